"""The no-allocation entry point ap_dvm_step_noalloc (include/ap_dvm.h) gives
the same result as the handle path (ap_dvm_create + ap_dvm_step), on two
calls in a row.  Callers that cannot allocate device memory use it; this
file runs last so that a failure here does not stop the other tests."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("scheme,n,tab", [("WENO5_C4", 64, "gsa2"), ("LF1_C2", 128, "gsa2"), ("WENO3_C4", 16, "gsa2"),
                                          ("WENO5_C4", 64, "type_a3")])
def test_noalloc_matches_handle_path_two_calls(scheme, n, tab):
    fn = _noalloc()
    X0 = W.random_moment_state(n, n, seed=404, amp=0.4)
    p = api.default_params(n, n, eps=1e-2, dt=0.01, tau=0.05, space_scheme=scheme, tableau=getattr(tableaux, tab)())
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


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fn = _noalloc()
    stream = torch.cuda.current_stream().cuda_stream
    d = torch.zeros((6, 256, 256), dtype=torch.float64, device="cuda")
    p = api.default_params(256, 256, eps=1e-2, dt=0.01)
    assert fn(ctypes.byref(p), d.data_ptr(), 1, stream) == 1          # AP_DVM_ERR_ARG
    p4 = api.default_params(128, 128, eps=1e-2, dt=0.01)
    A_ex = [[0, 0, 0, 0], [0.5, 0, 0, 0], [0, 0.5, 0, 0], [0, 0, 1.0, 0]]
    A_im = [[0, 0, 0, 0], [0, 0.5, 0, 0], [0, 0, 0.5, 0], [0, 0, 0.5, 0.5]]
    p4.set_tableau(A_ex, A_im)                                         # 4 stages at 128^2 exceed 8 MiB
    d4 = torch.zeros((6, 128, 128), dtype=torch.float64, device="cuda")
    assert fn(ctypes.byref(p4), d4.data_ptr(), 1, stream) == 1
    p5 = api.default_params(96, 64, eps=1e-2, dt=0.01)                 # not a power of two
    d5 = torch.zeros((6, 64, 96), dtype=torch.float64, device="cuda")
    assert fn(ctypes.byref(p5), d5.data_ptr(), 1, stream) == 7         # AP_DVM_ERR_UNSUPPORTED
