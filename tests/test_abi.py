"""The C-ABI library loads and exports every function include/ap_dvm.h declares
(no compute: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "ap_dvm.h")


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ap_dvm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ap_dvm_create", "ap_dvm_step", "ap_dvm_moments", "ap_dvm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2512_19847_gb300 import build_lib
    lib_path = build_lib.build()
    L = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_params_struct_layout_matches_c():
    from paper_2512_19847_gb300 import api
    # int nx, ny; double Lx, Ly; int vs; 5 doubles; int s; 2 x 16 doubles; 2 ints; double
    assert ctypes.sizeof(api.Params) == 352
    assert api.Params.A_ex.offset == 80 and api.Params.weno_eps.offset == 344


def test_validation_without_gpu():
    """Parameter and tableau validation happen on the host, before any CUDA call."""
    from paper_2512_19847_gb300 import api, tableaux
    p = api.default_params(64, 64, eps=1e-2, dt=0.01)
    assert api.lib().ap_dvm_workspace_size(ctypes.byref(p)) > 0
    g = p.copy(); g.nx, g.ny = 48, 33                # any size in [8, 4096]: Bluestein tables added
    assert api.lib().ap_dvm_workspace_size(ctypes.byref(g)) > 0
    for nx, ny in ((7, 64), (64, 4097), (0, 8)):
        bad = p.copy(); bad.nx, bad.ny = nx, ny
        assert api.lib().ap_dvm_workspace_size(ctypes.byref(bad)) == 0
    bad = p.copy(); bad.A_ex[0] = 1.0                # explicit diagonal
    assert api.lib().ap_dvm_workspace_size(ctypes.byref(bad)) == 0
    bad = p.copy(); bad.A_im[0] = -0.5               # negative a_11
    assert api.lib().ap_dvm_workspace_size(ctypes.byref(bad)) == 0
    a = p.copy(); a.A_im[0] = 0.5                    # type A: stage 1 gets its own buffers
    assert api.lib().ap_dvm_workspace_size(ctypes.byref(a)) > api.lib().ap_dvm_workspace_size(ctypes.byref(p))
    bad = p.copy(); bad.precision = api.FP32_DEV; bad.eps = 0.0
    assert api.lib().ap_dvm_workspace_size(ctypes.byref(bad)) == 0
    e = p.copy(); e.set_tableau(*tableaux.euler())
    assert api.lib().ap_dvm_workspace_size(ctypes.byref(e)) > 0
