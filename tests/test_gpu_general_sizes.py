"""Grids of any size in [8, 4096]: ragged stencil tiles at the high edges, and
for the axes whose length is not a power of two mixed-radix transforms (lengths
that factor into 2, 3, 5, 7) or Bluestein's (the others).

FP64 parity with the oracle to 1e-12 (relative max-norm per moment plane) on
odd, even and mixed sizes (both with TMA staging, rows a multiple of 16 bytes,
and with plain loads), every spatial scheme and tile shape, type-A tableaux,
the diagnostics, the batched form (mixed sizes, bitwise equal to each solve
alone), the longest transforms (M = 8192 along either axis), and a 1000^2
grid; the FP32 form against the oracle on a resolved flow.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ap_dvm_oracle as O  # noqa: E402
from paper_2512_19847_gb300 import api, tableaux, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12

# (nx, ny): odd x odd (the paper's 2^k + 1 counts), even with 16-byte rows (TMA
# staging, ragged tiles in both directions), powers of two on one axis only,
# the smallest grids, and widths whose rows are not a multiple of 16 bytes
SIZES = [(33, 33), (65, 40), (100, 44), (64, 37), (45, 32), (9, 10), (8, 9), (50, 27)]


def _pair(nx, ny, scheme, tab, eps, tau, dt, **kw):
    A_ex, A_im = getattr(tableaux, tab)()
    p = api.default_params(nx, ny, eps=eps, dt=dt, tau=tau, space_scheme=scheme, tableau=(A_ex, A_im), **kw)
    o = O.Params(nx, ny, eps, tau, dt, np.array(A_ex), np.array(A_im), scheme=scheme)
    return p, o


def rel_err(got, ref):
    scale = np.maximum(np.max(np.abs(ref), axis=(1, 2)), 1e-300)
    return np.max(np.abs(got - ref), axis=(1, 2)) / scale


def run_gpu(p, X0, nsteps, tile=-1):
    s = api.Solver(p)
    if tile >= 0:
        s.set_tile(tile)
    s.set_state(torch.from_numpy(X0).cuda())
    s.step(nsteps)
    s.sync_status()
    return s.get_state().cpu().numpy()


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("scheme", ["LF1_C2", "WENO3_C4", "WENO5_C4"])
def test_sizes_match_oracle(nx, ny, scheme):
    X0 = W.random_moment_state(nx, ny, seed=nx * 1000 + ny, amp=0.4)
    p, o = _pair(nx, ny, scheme, "gsa2", 1e-2, 0.05, 0.01)
    got = run_gpu(p, X0, 2)
    ref = O.run(X0, o, 2)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


# lengths that factor into 2, 3, 5 and 7 take the mixed-radix transform (every radix,
# radix 7 repeated, long plans), the others Bluestein's
@pytest.mark.parametrize("nx,ny", [(98, 49), (96, 45), (2000, 30), (343, 10), (27, 2187), (84, 63)])
def test_mixed_radix_sizes(nx, ny):
    X0 = W.random_moment_state(nx, ny, seed=nx + 7 * ny, amp=0.4)
    p, o = _pair(nx, ny, "WENO5_C4", "gsa2", 1e-2, 0.05, 0.002)
    got = run_gpu(p, X0, 2)
    ref = O.run(X0, o, 2)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


def test_fp32_form_mixed_radix():
    """FP32 form on a resolved flow, 100 x 96 (mixed radix on both axes)."""
    nx, ny = 100, 96
    u1, u2, pr = W.taylor_green(nx, ny)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.stable_dt(u1, u2, 2 * math.pi / nx, 0.05)
    p, o = _pair(nx, ny, "WENO5_C4", "gsa2", 1e-4, 0.05, dt, mach=1e-3)
    p.precision = api.FP32_DEV
    got = run_gpu(p, X0, 5)
    ref = O.run(X0, o, 5)
    err = np.max(np.hypot(got[0] - ref[0], got[1] - ref[1])) / np.max(np.hypot(ref[0], ref[1]))
    assert err <= 1e-5, err


@pytest.mark.parametrize("eps", [1.0, 1e-4, 0.0])
def test_euler_tableau_and_eps_range(eps):
    nx, ny = 57, 35
    X0 = W.random_moment_state(nx, ny, seed=3, amp=0.4)
    p, o = _pair(nx, ny, "WENO5_C4", "euler", eps, 0.05, 0.01)
    got = run_gpu(p, X0, 3)
    ref = O.run(X0, o, 3)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
def test_every_tile_shape_ragged(tile):
    """77 x 51: ragged in both directions for every tile shape (plain staging, odd rows)."""
    nx, ny = 77, 51
    X0 = W.random_moment_state(nx, ny, seed=11, amp=0.3)
    p, o = _pair(nx, ny, "WENO5_C4", "gsa2", 1e-3, 0.05, 0.01)
    got = run_gpu(p, X0, 2, tile=tile)
    ref = O.run(X0, o, 2)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


@pytest.mark.parametrize("tile", [0, 4, 5])
def test_tma_staging_ragged(tile):
    """104 x 52 in FP64: 16-byte rows, so tiles are staged by TMA, with ragged edge tiles."""
    nx, ny = 104, 52
    X0 = W.random_moment_state(nx, ny, seed=12, amp=0.3)
    p, o = _pair(nx, ny, "WENO5_C4", "gsa2", 1e-3, 0.05, 0.01)
    got = run_gpu(p, X0, 2, tile=tile)
    ref = O.run(X0, o, 2)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


@pytest.mark.parametrize("tab", ["type_a_euler", "type_a3"])
def test_type_a_ragged(tab):
    nx, ny = 39, 29
    X0 = W.random_moment_state(nx, ny, seed=21, amp=0.4)
    p, o = _pair(nx, ny, "WENO5_C4", tab, 1e-2, 0.05, 0.01)
    got = run_gpu(p, X0, 2)
    ref = O.run(X0, o, 2)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


def test_diagnostics_ragged():
    nx, ny = 47, 33
    X0 = W.random_moment_state(nx, ny, seed=29, amp=0.5)
    p, o = _pair(nx, ny, "WENO5_C4", "gsa2", 1e-2, 0.05, 0.01)
    s = api.Solver(p)
    s.set_state(torch.from_numpy(X0).cuda())
    got = s.diagnostics(vorticity=True)
    ref = O.diagnostics(X0, o)
    for k in ("div_max", "div_l2", "enstrophy"):
        assert abs(got[k] - ref[k]) <= TOL * abs(ref[k]), (k, got[k], ref[k])
    w = got["vorticity"].cpu().numpy()
    assert np.max(np.abs(w - ref["vorticity"])) <= TOL * np.max(np.abs(ref["vorticity"]))


@pytest.mark.parametrize("nx,ny", [(4095, 12), (12, 4095)])
def test_longest_transforms(nx, ny):
    """n = 4095 on one axis: Bluestein with M = 8192, the longest transform."""
    X0 = W.random_moment_state(nx, ny, seed=31, amp=0.3)
    p, o = _pair(nx, ny, "WENO5_C4", "gsa2", 1e-2, 0.05, 0.2 * 2 * math.pi / max(nx, ny))
    got = run_gpu(p, X0, 1)
    ref = O.run(X0, o, 1)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


def test_thousand_squared():
    """1000^2 (125 x 32-wide tile columns, M = 2048 on both axes), one step of a shear layer."""
    n = 1000
    u1, u2, pr = W.double_shear_layer(n)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.stable_dt(u1, u2, 2 * math.pi / n, 0.05)
    p, o = _pair(n, n, "WENO5_C4", "gsa2", 1e-4, 0.05, dt)
    got = run_gpu(p, X0, 1)
    ref = O.run(X0, o, 1)
    assert np.all(rel_err(got, ref) <= TOL), rel_err(got, ref)


@pytest.mark.parametrize("nx,ny", [(60, 36), (61, 36), (64, 37)])
def test_fp32_form_ragged(nx, ny):
    """FP32 form on a resolved flow: 60 x 36 (16-byte rows, TMA; mixed radix), 61 x 36 (plain
    loads; Bluestein rows) and 64 x 37 (Bluestein columns)."""
    u1, u2, pr = W.taylor_green(nx, ny)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.stable_dt(u1, u2, 2 * math.pi / nx, 0.05)
    p, o = _pair(nx, ny, "WENO5_C4", "gsa2", 1e-4, 0.05, dt, mach=1e-3)
    p.precision = api.FP32_DEV
    got = run_gpu(p, X0, 5)
    ref = O.run(X0, o, 5)
    err = np.max(np.hypot(got[0] - ref[0], got[1] - ref[1])) / np.max(np.hypot(ref[0], ref[1]))
    assert err <= 1e-5, err


@pytest.mark.parametrize("nx,ny", [(8, 9), (9, 10), (27, 13), (16, 11), (50, 27)])
def test_fp32_form_narrow_and_short_grids(nx, ny):
    """FP32 form on grids narrower than one right-hand-side segment of 28 columns (lane
    columns wrapping more than once) and with few, odd rows (the last item of two row pairs
    ending past the last row), against the oracle on a resolved flow."""
    u1, u2, pr = W.taylor_green(nx, ny)
    X0 = O.equilibrium_state(u1, u2, pr)
    dt = W.stable_dt(u1, u2, 2 * math.pi / nx, 0.05)
    p, o = _pair(nx, ny, "WENO5_C4", "gsa2", 1e-4, 0.05, dt, mach=1e-3)
    p.precision = api.FP32_DEV
    got = run_gpu(p, X0, 5)
    ref = O.run(X0, o, 5)
    err = np.max(np.hypot(got[0] - ref[0], got[1] - ref[1])) / np.max(np.hypot(ref[0], ref[1]))
    assert err <= 1e-5, err


def test_batch_mixed_sizes_equal_alone():
    """One batch holding power-of-two and other sizes: each result equals the solve alone bit for bit."""
    tmpl = api.default_params(100, 100, eps=1e-2, dt=0.01, tableau=tableaux.gsa2())
    sizes = [(100, 100), (64, 64), (33, 50), (72, 17)]
    b = api.Batch(tmpl, capacity=len(sizes))
    states = {}
    for k, (nx, ny) in enumerate(sizes):
        q = tmpl.copy()
        q.nx, q.ny = nx, ny
        b.attach(k, q)
        states[k] = W.random_moment_state(nx, ny, seed=40 + k, amp=0.3)
        b.set_state(torch.from_numpy(states[k]).cuda(), slot=k)
    b.step(3)
    b.sync_status()
    # both transform kinds on both axes: 2 + 2 row launches and 2 column launches per implicit
    # stage; the last stage's update closes the step (no finish launch)
    assert b.launches_per_step == (3 + 6) * 2
    for k, (nx, ny) in enumerate(sizes):
        q = tmpl.copy()
        q.nx, q.ny = nx, ny
        alone = run_gpu(q, states[k], 3, tile=b.tile)
        assert np.array_equal(b.get_state(k).cpu().numpy(), alone), (nx, ny)


def test_launch_count_by_transform_kind():
    """A single solve launches one kernel per transform pass, whichever kind its axes need."""
    for nx, ny in ((64, 64), (33, 64), (64, 33), (33, 35)):
        s = api.Solver(api.default_params(nx, ny, eps=1e-2, dt=0.01, tableau=tableaux.gsa2()))
        assert s.launches_per_step == (3 + 3) * 2, (nx, ny)


def test_attach_rejects_longer_transforms():
    """A 64^2 batch has transforms of length 64; a 40-cell axis needs M = 128."""
    tmpl = api.default_params(64, 64, eps=1e-2, dt=0.01)
    b = api.Batch(tmpl, capacity=1)
    q = tmpl.copy()
    q.nx = 40
    with pytest.raises(api.ApDvmError):
        b.attach(0, q)


def test_graph_rebuilt_when_a_new_transform_kind_attaches():
    """A batch stepping through a captured CUDA graph with power-of-two solves only, then a
    solve of another size attached: the graph is re-captured with the Bluestein launches and
    every solve still equals itself alone."""
    tmpl = api.default_params(96, 96, eps=1e-2, dt=0.01, tableau=tableaux.gsa2())
    b = api.Batch(tmpl, capacity=2)
    b.set_graph_steps(2)
    q0 = tmpl.copy()
    q0.nx, q0.ny = 64, 32
    x0 = W.random_moment_state(64, 32, seed=50, amp=0.3)
    b.attach(0, q0)
    b.set_state(torch.from_numpy(x0).cuda(), slot=0)
    b.step(2)
    q1 = tmpl.copy()
    q1.nx, q1.ny = 96, 40
    x1 = W.random_moment_state(96, 40, seed=51, amp=0.3)
    b.attach(1, q1)
    b.set_state(torch.from_numpy(x1).cuda(), slot=1)
    b.step(4)
    b.sync_status()
    assert np.array_equal(b.get_state(0).cpu().numpy(), run_gpu(q0, x0, 6, tile=b.tile))
    assert np.array_equal(b.get_state(1).cpu().numpy(), run_gpu(q1, x1, 4, tile=b.tile))
