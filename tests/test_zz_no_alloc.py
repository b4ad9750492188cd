"""The no-allocation entry point ap_dvm_step_noalloc (include/ap_dvm.h).

Some callers cannot allocate device memory or hand the library a workspace:
code running under a host framework that owns every device allocation,
real-time loops that forbid allocation after start-up, plugins loaded into a
process whose allocator they may not touch.  This entry point gives them the
same IMEX steps with all scratch in one fixed file-scope device array.  The
tests check it against the handle path (ap_dvm_create + ap_dvm_step) and the
CPU oracle on two calls in a row, its size limits, and its error reporting.
This file runs last, so that a failure here does not stop the other tests.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ap_dvm_oracle as O  # noqa: E402
from paper_2512_19847_gb300 import api, tableaux, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _noalloc():
    fn = api.lib().ap_dvm_step_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(api.Params), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    return fn


def _rel(a, b):
    return np.max(np.abs(a - b), axis=(1, 2)) / np.maximum(np.max(np.abs(b), axis=(1, 2)), 1e-300)


# the largest layouts the 8 MiB scratch takes at 128 x 128: four stages of a CK/ARS tableau
# (ars4), three stages of a type-A tableau (type_a3, with its own stage-1 buffer)
@pytest.mark.parametrize("scheme,nx,ny,tab", [("WENO5_C4", 64, 64, "gsa2"), ("LF1_C2", 128, 128, "gsa2"),
                                              ("WENO3_C4", 16, 16, "gsa2"), ("WENO5_C4", 64, 64, "type_a3"),
                                              ("WENO5_C4", 128, 128, "type_a3"), ("WENO5_C4", 128, 128, "ars4")])
def test_noalloc_matches_handle_path_two_calls(scheme, nx, ny, tab):
    fn = _noalloc()
    X0 = W.random_moment_state(nx, ny, seed=404, amp=0.4)
    p = api.default_params(nx, ny, eps=1e-2, dt=0.01, tau=0.05, space_scheme=scheme, tableau=getattr(tableaux, tab)())
    ref = api.Solver(p)
    ref.set_state(torch.from_numpy(X0).cuda())
    d = torch.from_numpy(X0).cuda().contiguous()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        ref.step(3)
        want = ref.get_state().cpu().numpy()
        st = fn(ctypes.byref(p), d.data_ptr(), 3, stream)
        assert st == 0, st
        torch.cuda.synchronize()
        got = d.cpu().numpy()
        assert np.all(_rel(got, want) <= TOL), (call, _rel(got, want))


@pytest.mark.parametrize("nx,ny", [(128, 64), (32, 128)])
def test_noalloc_matches_the_oracle_on_non_square_grids(nx, ny):
    """Two calls in a row on non-square power-of-two grids (the transforms share
    twiddles built for the longer side) against the CPU oracle."""
    fn = _noalloc()
    X0 = W.random_moment_state(nx, ny, seed=17, amp=0.4)
    A_ex, A_im = tableaux.gsa2()
    dt = 0.25 * 2 * math.pi / max(nx, ny)
    p = api.default_params(nx, ny, eps=1e-3, dt=dt, tau=0.05, space_scheme="WENO5_C4", tableau=(A_ex, A_im))
    o = O.Params(nx, ny, 1e-3, 0.05, dt, np.array(A_ex), np.array(A_im), scheme="WENO5_C4")
    d = torch.from_numpy(X0).cuda().contiguous()
    stream = torch.cuda.current_stream().cuda_stream
    ref = X0
    for call in range(2):
        assert fn(ctypes.byref(p), d.data_ptr(), 2, stream) == 0
        torch.cuda.synchronize()
        ref = O.run(ref, o, 2)
        err = _rel(d.cpu().numpy(), ref)
        assert np.all(err <= TOL), (call, err)


def test_noalloc_reports_a_non_finite_state():
    """A NaN planted in the input state on the host: the call returns
    AP_DVM_ERR_NONFINITE (5), like ap_dvm_sync_status; the next call on a finite
    state returns 0 (the flags start cleared on every call)."""
    fn = _noalloc()
    n = 32
    X0 = W.random_moment_state(n, n, seed=8, amp=0.4)
    bad = X0.copy()
    bad[1, 5, 7] = float("nan")
    p = api.default_params(n, n, eps=1e-2, dt=0.01, tau=0.05)
    stream = torch.cuda.current_stream().cuda_stream
    d = torch.from_numpy(bad).cuda().contiguous()
    assert fn(ctypes.byref(p), d.data_ptr(), 1, stream) == 5
    d = torch.from_numpy(X0).cuda().contiguous()
    assert fn(ctypes.byref(p), d.data_ptr(), 1, stream) == 0
    assert torch.isfinite(d).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fn = _noalloc()
    stream = torch.cuda.current_stream().cuda_stream
    d = torch.zeros((6, 256, 256), dtype=torch.float64, device="cuda")
    p = api.default_params(256, 256, eps=1e-2, dt=0.01)
    assert fn(ctypes.byref(p), d.data_ptr(), 1, stream) == 1          # AP_DVM_ERR_ARG
    # a four-stage type-A tableau (its own stage-1 buffer) at 128^2 exceeds the 8 MiB
    A_ex = [[0, 0, 0, 0], [0.5, 0, 0, 0], [0.25, 0.25, 0, 0], [0.2, 0.3, 0.5, 0]]
    A_im = [[0.5, 0, 0, 0], [0, 0.5, 0, 0], [0, 0.25, 0.5, 0], [0, 0.25, 0.25, 0.5]]
    p4 = api.default_params(128, 128, eps=1e-2, dt=0.01, tableau=(A_ex, A_im))
    d4 = torch.zeros((6, 128, 128), dtype=torch.float64, device="cuda")
    assert fn(ctypes.byref(p4), d4.data_ptr(), 1, stream) == 1
    p5 = api.default_params(96, 64, eps=1e-2, dt=0.01)                 # not a power of two
    d5 = torch.zeros((6, 64, 96), dtype=torch.float64, device="cuda")
    assert fn(ctypes.byref(p5), d5.data_ptr(), 1, stream) == 7         # AP_DVM_ERR_UNSUPPORTED
