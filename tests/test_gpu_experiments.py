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
