"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 form: element by element, max |gpu - oracle| <= 1e-12 * max |oracle| per
moment plane, on seeded inputs at sizes spanning several tiles, for every
spatial scheme and both tableaux of Sec. 4.1, non-square grids, eps from the
kinetic regime to the exact limit eps = 0, and multi-step runs.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ap_dvm_oracle as O  # noqa: E402
from paper_2512_19847_gb300 import api, tableaux, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _tab(name):
    return getattr(tableaux, name)()


def _pair(nx, ny, scheme, tab, eps, tau, dt, **kw):
    A_ex, A_im = _tab(tab)
    p = api.default_params(nx, ny, eps=eps, dt=dt, tau=tau, space_scheme=scheme, tableau=(A_ex, A_im), **kw)
    o = O.Params(nx, ny, eps, tau, dt, np.array(A_ex), np.array(A_im), scheme=scheme)
    return p, o


def rel_err(got, ref):
    scale = np.maximum(np.max(np.abs(ref), axis=(1, 2)), 1e-300)
    return np.max(np.abs(got - ref), axis=(1, 2)) / scale


def run_gpu(p, X0, nsteps, graph=0, tile=-1):
    s = api.Solver(p)
    if tile >= 0:
        s.set_tile(tile)
    s.set_graph_steps(graph)
    s.set_state(torch.from_numpy(X0).cuda())
    s.step(nsteps)
    s.sync_status()
    return s.get_state().cpu().numpy()


@pytest.mark.parametrize("scheme", ["LF1_C2", "WENO3_C4", "WENO5_C4"])
@pytest.mark.parametrize("tab", ["euler", "gsa2", "ars4"])
@pytest.mark.parametrize("eps", [1.0, 1e-2, 1e-6])
def test_one_step_random_state(scheme, tab, eps):
    nx, ny = 64, 32
    X0 = W.random_moment_state(nx, ny, seed=101, amp=0.5)
    p, o = _pair(nx, ny, scheme, tab, eps, 0.05, 0.02)
    got = run_gpu(p, X0, 1)
    ref = O.step(X0, o)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


@pytest.mark.parametrize("scheme", ["LF1_C2", "WENO5_C4"])
def test_exact_limit_eps_zero(scheme):
    n = 32
    u1, u2, pr = W.taylor_green(n)
    X0 = O.equilibrium_state(u1, u2, pr)
    p, o = _pair(n, n, scheme, "gsa2", 0.0, 0.0, 0.5 * 2 * math.pi / n)
    got = run_gpu(p, X0, 3)
    ref = O.run(X0, o, 3)
    err = rel_err(got, ref)
    assert np.all(err[:3] <= TOL), err            # v, q vanish identically in this limit


def test_taylor_green_64_100_steps():
    """Taylor-Green vortex, 64^2, eps = Ma = 1e-2, CFL 0.5, 100 steps, second-order
    IMEX with WENO5 + C4 (the small FP64 workload)."""
    n = 64
    u1, u2, pr = W.taylor_green(n)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.cfl_dt(u1, u2, 2 * math.pi / n, 0.5)
    p, o = _pair(n, n, "WENO5_C4", "gsa2", 1e-2, 0.05, dt, mach=1e-2)
    got = run_gpu(p, X0, 100, graph=10)
    ref = O.run(X0, o, 100)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


@pytest.mark.parametrize("eps", [1.0, 1e-2, 1e-4, 1e-6])
def test_double_shear_layer_sweep(eps):
    """Double shear layer (1/rho = 30, delta = 0.05), the asymptotic-preserving sweep
    over eps at a reduced size (128^2).  The thin layer is Kelvin-Helmholtz
    unstable: a 1e-14 perturbation of the oracle's own input grows ~2.5x per
    step (rate ~ U/delta = 30), so round-off differences between any two
    implementations are compared over a short horizon, 5 steps."""
    n = 128
    u1, u2, pr = W.double_shear_layer(n)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.cfl_dt(u1, u2, 2 * math.pi / n, 0.5)
    p, o = _pair(n, n, "WENO5_C4", "gsa2", eps, 0.05, dt, mach=1e-2)
    got = run_gpu(p, X0, 5)
    ref = O.run(X0, o, 5)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
def test_tile_shapes_agree(tile):
    n = 64
    X0 = W.random_moment_state(n, n, seed=5, amp=0.3)
    p, o = _pair(n, n, "WENO5_C4", "gsa2", 1e-3, 0.05, 0.02)
    got = run_gpu(p, X0, 2, tile=tile)
    ref = O.run(X0, o, 2)
    assert np.all(rel_err(got, ref) <= TOL)


def test_graph_replay_is_bitwise_direct():
    n = 64
    X0 = W.random_moment_state(n, n, seed=9, amp=0.3)
    p, _ = _pair(n, n, "WENO5_C4", "gsa2", 1e-2, 0.05, 0.02)
    a = run_gpu(p, X0, 6, graph=0)
    b = run_gpu(p, X0, 6, graph=3)
    assert np.array_equal(a, b)


def test_equilibrium_and_outputs():
    n = 32
    u1, u2, pr = W.taylor_green(n)
    p, _ = _pair(n, n, "WENO5_C4", "gsa2", 1e-2, 0.05, 0.01, mach=2e-3, rho0=1.2)
    s = api.Solver(p)
    s.set_equilibrium(*[torch.from_numpy(a).cuda() for a in (u1, u2, pr)])
    X = s.get_state().cpu().numpy()
    assert np.allclose(X, O.equilibrium_state(u1, u2, pr), rtol=0, atol=1e-15)
    rho, a1, a2, pp = [t.cpu().numpy() for t in s.moments()]
    r_ref = O.outputs(X, 1e-2, rho0=1.2, amp=2e-3)
    for g, r in zip((rho, a1, a2, pp), r_ref):
        assert np.max(np.abs(g - r)) <= 1e-14 * max(1.0, np.max(np.abs(r)))


def test_population_view_round_trip():
    n, eps, mach, rho0 = 32, 3e-2, 5e-3, 1.1
    X0 = W.random_moment_state(n, n, seed=17, amp=0.4)
    p, _ = _pair(n, n, "WENO5_C4", "gsa2", eps, 0.05, 0.01, mach=mach, rho0=rho0)
    s = api.Solver(p)
    dF_ref = O.populations_from_moments(X0, eps, rho0=rho0, amp=mach)
    s.set_populations(torch.from_numpy(dF_ref).cuda())
    X = s.get_state().cpu().numpy()
    power = np.array([0, 0, 1, 1, 1, 2])
    tol = 1e-14 * np.max(np.abs(X0)) * 8 / eps ** power
    assert np.all(np.max(np.abs(X - X0), axis=(1, 2)) <= tol)
    dF = s.get_populations().cpu().numpy()
    assert np.max(np.abs(dF - dF_ref)) <= 1e-13 * np.max(np.abs(dF_ref))


def test_nonfinite_state_is_reported():
    """A NaN planted in the input (on the host) is caught by the per-step check."""
    n = 16
    X0 = W.random_moment_state(n, n, seed=1)
    X0[0, 3, 4] = np.nan
    p, _ = _pair(n, n, "WENO5_C4", "gsa2", 1e-2, 0.05, 0.01)
    s = api.Solver(p)
    s.set_state(torch.from_numpy(X0).cuda())
    s.step(1)
    with pytest.raises(api.ApDvmError) as e:
        s.sync_status()
    assert e.value.status == 5
    s.set_state(torch.from_numpy(np.nan_to_num(X0)).cuda())
    s.step(1)
    s.sync_status()      # flag was cleared by the previous read


def test_run_host_matches_device_path():
    n = 32
    X0 = W.random_moment_state(n, n, seed=23, amp=0.3)
    p, _ = _pair(n, n, "WENO5_C4", "gsa2", 1e-2, 0.05, 0.01)
    a = run_gpu(p, X0, 3)
    s = api.Solver(p)
    b = s.run_host(torch.from_numpy(X0).pin_memory(), 3).numpy()
    assert np.array_equal(a, b)


def _pair_domain(nx, ny, Lx, Ly, scheme, eps, dt, tau=0.05):
    A_ex, A_im = tableaux.gsa2()
    p = api.default_params(nx, ny, eps=eps, dt=dt, tau=tau, space_scheme=scheme, tableau=(A_ex, A_im), Lx=Lx, Ly=Ly)
    o = O.Params(nx, ny, eps, tau, dt, np.array(A_ex), np.array(A_im), scheme=scheme, Lx=Lx, Ly=Ly)
    return p, o


@pytest.mark.parametrize("Lx,Ly", [(2 * math.pi, math.pi), (4 * math.pi, math.pi), (math.pi, 3.0)])
def test_domain_lengths(Lx, Ly):
    """Periodic domains other than [0, 2pi)^2, with dx != dy (the [0, 4pi)^2 of Sec. 4.3 below)."""
    nx, ny = 64, 32
    X0 = W.random_moment_state(nx, ny, seed=17, amp=0.4)
    p, o = _pair_domain(nx, ny, Lx, Ly, "WENO5_C4", 1e-2, 0.01)
    got = run_gpu(p, X0, 3)
    ref = O.run(X0, o, 3)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


def test_kelvin_helmholtz_domain():
    """Kelvin-Helmholtz data of Sec. 4.3 on [0, 4pi)^2 (tau = 0.05, the value of the figure caption; the text says 0), 5 steps
    (the layer is unstable, so round-off is compared over a short horizon)."""
    n = 128
    u1, u2, pr = W.kelvin_helmholtz(n)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.stable_dt(u1, u2, 4 * math.pi / n, 0.05)
    p, o = _pair_domain(n, n, 4 * math.pi, 4 * math.pi, "WENO5_C4", 1e-4, dt)
    got = run_gpu(p, X0, 5)
    ref = O.run(X0, o, 5)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


@pytest.mark.parametrize("scheme", ["LF1_C2", "WENO3_C4", "WENO5_C4"])
def test_diagnostics_match_oracle(scheme):
    """ap_dvm_diagnostics (max |D_0 . u|, its L2 norm, enstrophy, vorticity) against the oracle's."""
    nx, ny = 64, 32
    X0 = W.random_moment_state(nx, ny, seed=23, amp=0.5)
    p, o = _pair_domain(nx, ny, 2 * math.pi, 1.5 * math.pi, scheme, 1e-2, 0.01)
    s = api.Solver(p)
    s.set_state(torch.from_numpy(X0).cuda())
    got = s.diagnostics(vorticity=True)
    ref = O.diagnostics(X0, o)
    for k in ("div_max", "div_l2", "enstrophy"):
        assert abs(got[k] - ref[k]) <= TOL * abs(ref[k]), (k, got[k], ref[k])
    w = got["vorticity"].cpu().numpy()
    assert np.max(np.abs(w - ref["vorticity"])) <= TOL * np.max(np.abs(ref["vorticity"]))


def test_diagnostics_fp32_form():
    """The FP32 form's diagnostics come from its FP32 moment planes (the populations' moments
    rounded once): the enstrophy within 1e-5 relative, the divergence norms within 1e-5
    absolute, of the oracle's on the state the solve holds."""
    n = 64
    u1, u2, pr = W.random_divfree(n, 4, kmax=8)
    X0 = O.equilibrium_state(u1, u2, pr)
    X0[0] += 0.05 * np.sin(W.cell_centres(n, n)[0])          # a divergent part
    p, o = _pair_domain(n, n, 2 * math.pi, 2 * math.pi, "WENO5_C4", 1e-2, 0.01)
    p.precision = api.FP32_DEV
    s = api.Solver(p)
    s.set_state(torch.from_numpy(X0).cuda())
    got = s.diagnostics()
    ref = O.diagnostics(s.get_state().cpu().numpy(), o)
    assert abs(got["enstrophy"] - ref["enstrophy"]) <= 1e-5 * ref["enstrophy"]
    for k in ("div_max", "div_l2"):
        assert abs(got[k] - ref[k]) <= 1e-5, (k, got[k], ref[k])


@pytest.mark.parametrize("tab", ["type_a_euler", "type_a3"])
@pytest.mark.parametrize("scheme", ["LF1_C2", "WENO5_C4"])
@pytest.mark.parametrize("eps", [1.0, 1e-4, 0.0])
def test_type_a_tableaux(tab, scheme, eps):
    """Type-A tableaux (a_11 != 0): stage 1 by Algorithm 1 with i = 1, then the usual stages."""
    nx, ny = 64, 32
    X0 = W.random_moment_state(nx, ny, seed=31, amp=0.4)
    p, o = _pair(nx, ny, scheme, tab, eps, 0.05, 0.01)
    got = run_gpu(p, X0, 2)
    ref = O.run(X0, o, 2)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


def test_type_a_batch_equals_alone_and_fp32_form():
    """Type A in the batched form (bitwise equal to each solve alone) and in the
    FP32 deviation form (velocity within 1e-5 of FP64 on a resolved flow)."""
    n = 64
    u1, u2, pr = W.taylor_green(n)
    fields = [torch.from_numpy(a).cuda() for a in (u1, u2, pr)]
    out = {}
    for prec in (api.FP64, api.FP32_DEV):
        p = api.default_params(n, n, eps=1e-4, dt=0.01, tau=0.05, mach=1e-3, tableau=tableaux.type_a3(), precision=prec)
        s = api.Solver(p)
        s.set_equilibrium(*fields)
        s.step(10)
        out[prec] = s.get_state().cpu().numpy()
        b = api.Batch(p, capacity=2)
        q = p.copy()
        q.nx = q.ny = 32
        b.attach(0, q)
        b.attach(1, p)
        small = [torch.from_numpy(a).cuda() for a in W.taylor_green(32)]
        b.set_equilibrium(*small, slot=0)
        b.set_equilibrium(*fields, slot=1)
        b.set_tile(s.tile)
        b.step(10)
        assert np.array_equal(b.get_state(1).cpu().numpy(), out[prec])
    a, c = out[api.FP64], out[api.FP32_DEV]
    assert np.max(np.hypot(a[0] - c[0], a[1] - c[1])) / np.max(np.hypot(a[0], a[1])) <= 1e-5


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
def test_fp32_form_every_tile_shape(tile):
    """The FP32 form's register-run fluxes on every tile shape: velocity within 1e-5 of the
    oracle on a resolved flow after 5 steps, and all shapes agree to FP32 rounding."""
    n = 64
    u1, u2, pr = W.taylor_green(n)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.stable_dt(u1, u2, 2 * math.pi / n, 0.05)
    p, o = _pair(n, n, "WENO5_C4", "gsa2", 1e-4, 0.05, dt, mach=1e-3)
    p.precision = api.FP32_DEV
    got = run_gpu(p, X0, 5, tile=tile)
    ref = O.run(X0, o, 5)
    err = np.max(np.hypot(got[0] - ref[0], got[1] - ref[1])) / np.max(np.hypot(ref[0], ref[1]))
    assert err <= 1e-5, err


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("scheme", ["WENO3_C4", "WENO5_C4"])
def test_four_stages_every_tile_shape(tile, scheme):
    """s = 4 (the largest stage count the library takes; the ARS-type pair
    tableaux.ars4): the stage sums of Algorithm 1 over three earlier stages, the
    dissipation partner (the explicit-weight predictor) over three earlier stages and the update's
    largest staged plane set, on every tile shape, over 3 steps, on a grid with
    ragged edge tiles in both directions."""
    nx, ny = 72, 40
    X0 = W.random_moment_state(nx, ny, seed=404, amp=0.4)
    p, o = _pair(nx, ny, scheme, "ars4", 1e-2, 0.05, 0.01)
    got = run_gpu(p, X0, 3, tile=tile)
    ref = O.run(X0, o, 3)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


def test_four_stages_batch_graph_and_fp32_form():
    """s = 4 in the batched form (mixed sizes, CUDA graph: each solve bit for bit
    its result alone, and the oracle's within 1e-12) and in the FP32 deviation
    form (velocity within 1e-5 of the oracle on a resolved flow)."""
    sizes = [(64, 64), (64, 32), (32, 64)]
    eps = 1e-4
    ps, refs, alone = [], [], []
    for k, (nx, ny) in enumerate(sizes):
        X0 = W.random_moment_state(nx, ny, seed=50 + k, amp=0.4)
        p, o = _pair(nx, ny, "WENO5_C4", "ars4", eps, 0.05, 0.01, mach=1e-3)
        ps.append((p, X0))
        refs.append(O.run(X0, o, 4))
        alone.append(run_gpu(p, X0, 4, tile=3))
        assert np.all(rel_err(alone[-1], refs[-1]) <= TOL), rel_err(alone[-1], refs[-1])
    b = api.Batch(ps[0][0], capacity=len(sizes))
    for k, (p, X0) in enumerate(ps):
        b.attach(k, p)
        b.set_state(torch.from_numpy(X0).cuda(), slot=k)
    b.set_tile(3)
    b.set_graph_steps(2)
    b.step(4)
    b.sync_status()
    for k in range(len(sizes)):
        assert np.array_equal(b.get_state(k).cpu().numpy(), alone[k]), k
    n = 64
    u1, u2, pr = W.taylor_green(n)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.stable_dt(u1, u2, 2 * math.pi / n, 0.05)
    p, o = _pair(n, n, "WENO5_C4", "ars4", eps, 0.05, dt, mach=1e-3)
    p.precision = api.FP32_DEV
    got = run_gpu(p, X0, 5)
    ref = O.run(X0, o, 5)
    err = np.max(np.hypot(got[0] - ref[0], got[1] - ref[1])) / np.max(np.hypot(ref[0], ref[1]))
    assert err <= 1e-5, err


def test_fp32_carried_theta_form():
    """AP_DVM_FP32_DEV_TH: theta carried in its own FP32 plane.  Velocity within 1e-5
    and the pressure closer to the oracle's than the plain FP32 form's (theta is no
    longer summed back from the populations, where it rides at O(eps)); the
    populations are those of the FP32 form's packing; set_theta after
    set_populations restores a solve bit for bit (the autotuner's save/restore)."""
    n = 64
    u1, u2, pr = W.taylor_green(n)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.stable_dt(u1, u2, 2 * math.pi / n, 0.05)
    p, o = _pair(n, n, "WENO5_C4", "gsa2", 1e-4, 0.05, dt, mach=1e-3)
    ref = O.run(X0, o, 5)
    pref = ref[2] - 0.5 * (ref[0] ** 2 + ref[1] ** 2)
    out = {}
    for prec in (api.FP32_DEV, api.FP32_DEV_TH):
        p.precision = prec
        got = run_gpu(p, X0, 5)
        vel = np.max(np.hypot(got[0] - ref[0], got[1] - ref[1])) / np.max(np.hypot(ref[0], ref[1]))
        pg = got[2] - 0.5 * (got[0] ** 2 + got[1] ** 2)
        out[prec] = np.max(np.abs((pg - pg.mean()) - (pref - pref.mean()))) / np.max(np.abs(pref - pref.mean()))
        assert vel <= 1e-5, (prec, vel)
    assert out[api.FP32_DEV_TH] < 0.1 * out[api.FP32_DEV], out
    # bit-for-bit restore: populations + carried theta
    p.precision = api.FP32_DEV_TH
    s = api.Solver(p)
    s.set_state(torch.from_numpy(X0).cuda())
    s.step(2)
    pops = s.get_populations(dtype=torch.float32)
    theta = s.get_state()[2].clone()
    s.step(3)
    want = s.get_state().cpu().numpy()
    s.set_populations(pops)
    s.set_theta(theta)
    s.step(3)
    assert np.array_equal(s.get_state().cpu().numpy(), want)
