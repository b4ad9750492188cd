"""The paper's Sec. 4 experiments through the C ABI: runs end at t_end exactly,
record finite diagnostics, and the diagnostics track the state (checked
against the oracle's at the end of a short run)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ap_dvm_oracle as O  # noqa: E402
from paper_2512_19847_gb300 import api, experiments, tableaux  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["shear_thick", "shear_thin", "kelvin_helmholtz"])
def test_short_runs(case):
    h = experiments.run(case, 64, eps=1e-4, t_end=0.5, record_every=4)
    assert h.steps * h.dt == pytest.approx(0.5, rel=1e-12)
    assert len(h.t) == len(h.div_max) == math.ceil(h.steps / 4) + 1
    assert all(np.isfinite(h.div_max)) and all(np.isfinite(h.enstrophy))
    # the space discretisation does not preserve D_0 . u = 0 (the divergence history of
    # Figs. 2-3 grows from zero); it stays small against the velocity gradients, and the
    # enstrophy of these viscous 2D flows does not grow
    assert max(h.div_max) < 0.5
    assert h.enstrophy[-1] <= 1.01 * h.enstrophy[0]
    assert h.vorticity.shape == (64, 64)


def test_diagnostics_track_the_state():
    """The recorded final diagnostics equal the oracle's diagnostics of the state the
    solve holds at the end (4th-order central operators, [0, 4pi)^2)."""
    h = experiments.run("kelvin_helmholtz", 64, eps=1e-2, t_end=0.2, record_every=100)
    c = experiments.CASES["kelvin_helmholtz"]
    u1, u2, p = c["init"](64)
    A_ex, A_im = tableaux.gsa2()
    prm = api.default_params(64, 64, eps=1e-2, dt=h.dt, tau=0.05, mach=1e-2, Lx=c["L"], Ly=c["L"],
                             tableau=(A_ex, A_im))
    s = api.Solver(prm)
    s.set_equilibrium(*[torch.from_numpy(a).cuda() for a in (u1, u2, p)])
    s.step(h.steps)
    X = s.get_state().cpu().numpy()
    o = O.Params(64, 64, 1e-2, 0.05, h.dt, np.array(A_ex), np.array(A_im), scheme="WENO5_C4", Lx=c["L"], Ly=c["L"])
    ref = O.diagnostics(X, o)
    assert h.enstrophy[-1] == pytest.approx(ref["enstrophy"], rel=1e-12)
    assert h.div_max[-1] == pytest.approx(ref["div_max"], rel=1e-12)
    assert np.max(np.abs(h.vorticity.cpu().numpy() - ref["vorticity"])) <= 1e-12 * np.max(np.abs(ref["vorticity"]))


def _printed_orders(table, n):
    """Orders of the row N = n of Table 1 or 2 (L1, L2, max) from the golden file."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_1_2.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        t, nn, *vals = line.split()
        if int(t) == table and int(nn) == n:
            return [float(vals[k]) for k in (1, 3, 5)]
    raise KeyError((table, n))


def test_table_2_orders_at_the_paper_grids():
    """Sec. 4.1, Table 2 on the paper's grids of N = 33 .. 257 points (N - 1 cells, nested)
    against the 513-point reference: as in the printed table, the orders rise from about
    1.5 at N = 65 to about 2 at N = 129 (L1 and L2 between 1.8 and the printed order + 0.6).
    The last row compares with a reference only twice as fine, while the WENO3 weights
    (eps_W = 1e-6) are still leaving their pre-asymptotic range, and is not checked."""
    rows = {r["N"]: r for r in experiments.convergence(2)}
    assert sorted(rows) == [33, 65, 129, 257]
    printed = _printed_orders(2, 129)
    for k, name in enumerate(("L1_order", "L2_order", "Linf_order")):
        assert 1.2 < rows[65][name] < rows[129][name], (name, rows)
        if k < 2:
            assert 1.8 < rows[129][name] < printed[k] + 0.6, (name, rows[129][name], printed)


@pytest.mark.parametrize("n", [64, 128])
def test_kinetic_regime_blowup_is_the_schemes(n):
    """At eps = 1 (far from the low-Mach regime) a seeded random divergence-free
    field under the workloads' time-step rule (0.4 of the CFL bound, 0.32 of the
    viscous one) grows without bound in the oracle (the first step with
    max |u| > 1e3 or a non-finite value is found here, on the CPU); the CUDA path
    matches the oracle after 10 steps and leaves the same bound within two steps
    of it, so the blow-up is the discrete scheme's, not the kernel's."""
    from paper_2512_19847_gb300 import workloads as W
    u1, u2, pr = W.random_divfree(n, 2)
    dt = W.stable_dt(u1, u2, 2 * math.pi / n, 0.05)
    A_ex, A_im = tableaux.gsa2()
    p = api.default_params(n, n, eps=1.0, dt=dt, tau=0.05, mach=1e-2, tableau=(A_ex, A_im))
    o = O.Params(n, n, 1.0, 0.05, dt, np.array(A_ex), np.array(A_im), scheme="WENO5_C4")

    def bad(X):
        return not np.isfinite(X).all() or np.abs(X[:2]).max() > 1e3

    X = O.equilibrium_state(u1, u2, pr)
    s = api.Solver(p)
    s.set_state(torch.from_numpy(X).cuda())
    ref_blowup, gpu_blowup = None, None
    for k in range(1, 400):
        if ref_blowup is None:
            X = O.step(X, o)
            if bad(X):
                ref_blowup = k
        if gpu_blowup is None:
            s.step(1)
            g = s.get_state().cpu().numpy()
            if k == 10:
                err = np.max(np.abs(g - X), axis=(1, 2)) / np.max(np.abs(X), axis=(1, 2))
                assert np.all(err <= 1e-10), err
            if bad(g):
                gpu_blowup = k
        if ref_blowup is not None and gpu_blowup is not None:
            break
    assert ref_blowup is not None, "the oracle stayed bounded"
    assert gpu_blowup is not None and abs(gpu_blowup - ref_blowup) <= 2, (gpu_blowup, ref_blowup)
