"""Python binding of the C ABI in ``include/ap_dvm.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``libapdvm.so``; this
module loads it with ctypes, owns the device workspaces as PyTorch tensors,
and passes raw device pointers and the current CUDA stream.  There is no
CPU path: if the library or a GPU is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libapdvm.so")

MAX_STAGES = 4
D2V6 = 6
LF1_C2, WENO3_C4, WENO5_C4 = 0, 1, 2
SCHEMES = {"LF1_C2": LF1_C2, "WENO3_C4": WENO3_C4, "WENO5_C4": WENO5_C4}
FP64, FP32_DEV, FP32_DEV_TH = 0, 1, 2

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_TABLEAU", 3: "ERR_WORKSPACE", 4: "ERR_CUDA",
          5: "ERR_NONFINITE", 6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED"}


class ApDvmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of ``ap_dvm_params``."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
        ("velocity_set", ctypes.c_int),
        ("eps", ctypes.c_double), ("tau", ctypes.c_double), ("mach", ctypes.c_double),
        ("rho0", ctypes.c_double), ("dt", ctypes.c_double),
        ("s", ctypes.c_int),
        ("A_ex", ctypes.c_double * (MAX_STAGES * MAX_STAGES)),
        ("A_im", ctypes.c_double * (MAX_STAGES * MAX_STAGES)),
        ("space_scheme", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("weno_eps", ctypes.c_double),
    ]

    def set_tableau(self, A_ex, A_im):
        s = len(A_im)
        self.s = s
        for k in range(MAX_STAGES * MAX_STAGES):
            self.A_ex[k] = 0.0
            self.A_im[k] = 0.0
        for i in range(s):
            for j in range(s):
                self.A_ex[i * MAX_STAGES + j] = float(A_ex[i][j])
                self.A_im[i * MAX_STAGES + j] = float(A_im[i][j])
        return self

    def copy(self) -> "Params":
        q = Params()
        ctypes.pointer(q)[0] = self
        return q


_lib = None


def lib():
    """Load libapdvm.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing; build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(Params)
    vp, sz, i32, f64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double
    H = ctypes.c_void_p
    sig = {
        "ap_dvm_workspace_size": (sz, [P]),
        "ap_dvm_instance_workspace_size": (sz, [P]),
        "ap_dvm_batch_workspace_size": (sz, [P, i32]),
        "ap_dvm_create": (i32, [P, vp, sz, vp, ctypes.POINTER(H)]),
        "ap_dvm_batch_create": (i32, [P, i32, vp, sz, vp, ctypes.POINTER(H)]),
        "ap_dvm_attach": (i32, [H, i32, P, vp, sz]),
        "ap_dvm_detach": (i32, [H, i32]),
        "ap_dvm_set_state": (i32, [H, i32, vp]),
        "ap_dvm_set_equilibrium": (i32, [H, i32, vp, vp, vp]),
        "ap_dvm_set_populations": (i32, [H, i32, vp, i32]),
        "ap_dvm_get_state": (i32, [H, i32, vp]),
        "ap_dvm_set_theta": (i32, [H, i32, vp]),
        "ap_dvm_get_populations": (i32, [H, i32, vp, i32]),
        "ap_dvm_moments": (i32, [H, i32, vp, vp, vp, vp]),
        "ap_dvm_diagnostics": (i32, [H, i32, vp, ctypes.POINTER(f64)]),
        "ap_dvm_step": (i32, [H, i32]),
        "ap_dvm_step_slots": (i32, [H, i32, ctypes.POINTER(i32)]),
        "ap_dvm_set_graph_steps": (i32, [H, i32]),
        "ap_dvm_set_tile": (i32, [H, i32]),
        "ap_dvm_get_tile": (i32, [H]),
        "ap_dvm_launches_per_step": (i32, [H]),
        "ap_dvm_run_host": (i32, [H, i32, vp, vp, vp, i32]),
        "ap_dvm_sync_status": (i32, [H]),
        "ap_dvm_check_wait_timeout": (i32, [H, ctypes.c_longlong]),
        "ap_dvm_profile_enable": (i32, [H, i32]),
        "ap_dvm_profile_read": (i32, [H, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(f64),
                                      ctypes.POINTER(ctypes.c_long), i32]),
        "ap_dvm_last_error": (ctypes.c_char_p, [H]),
        "ap_dvm_destroy": (None, [H]),
        "ap_dvm_default_params": (None, [P, i32, i32, f64, f64]),
        "ap_dvm_step_noalloc": (i32, [P, vp, i32, vp]),
        "ap_dvm_fma_peak": (i32, [i32, i32, i32, vp, ctypes.POINTER(f64), ctypes.POINTER(f64)]),
        "ap_dvm_check_conversions": (i32, [vp, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def default_params(nx: int, ny: int | None = None, eps: float = 1e-2, dt: float = 1e-2, **kw) -> Params:
    """ap_dvm_default_params plus keyword overrides (scheme may be a name)."""
    p = Params()
    lib().ap_dvm_default_params(ctypes.byref(p), nx, nx if ny is None else ny, eps, dt)
    for k, v in kw.items():
        if k == "space_scheme" and isinstance(v, str):
            v = SCHEMES[v]
        if k == "tableau":
            p.set_tableau(*v)
            continue
        setattr(p, k, v)
    return p


def fma_peak(precision: int = FP64, iters: int = 256, reps: int = 50, stream=None) -> tuple[float, float]:
    """ap_dvm_fma_peak: (TFLOP/s, ms per launch) of an FMA-chain kernel in FP64
    (precision = FP64) or FP32 (FP32_DEV) on the current GPU."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    st = lib().ap_dvm_fma_peak(int(precision), int(iters), int(reps), _stream_ptr(stream), ctypes.byref(tf), ctypes.byref(ms))
    if st != 0:
        raise ApDvmError(st, "ap_dvm_fma_peak failed")
    return tf.value, ms.value


def check_conversions(x: torch.Tensor, stream=None) -> tuple[int, int]:
    """ap_dvm_check_conversions on the FP64 values of the device tensor x: the numbers of
    integer-pipe narrowings and widenings that differ from the conversion instructions."""
    x = x.contiguous()
    assert x.dtype == torch.float64 and x.is_cuda
    counts = torch.zeros(2, dtype=torch.int32, device=x.device)
    st = lib().ap_dvm_check_conversions(_ptr(x), int(x.numel()), _ptr(counts), _stream_ptr(stream))
    if st != 0:
        raise ApDvmError(st, "ap_dvm_check_conversions failed")
    c = counts.cpu().tolist()
    return c[0], c[1]


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream_ptr(stream) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


class _Handle:
    def __init__(self):
        self._h = ctypes.c_void_p()
        self._keep = {}

    def _check(self, st: int):
        if st != 0:
            msg = lib().ap_dvm_last_error(self._h).decode(errors="replace") if self._h else "no handle"
            raise ApDvmError(st, msg)

    def close(self):
        if self._h:
            lib().ap_dvm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- state of slot k
    def _shape(self, slot):
        p = self._params[slot]
        return p.ny, p.nx

    def set_state(self, X: torch.Tensor, slot: int = 0):
        """X: (6, ny, nx) float64 CUDA tensor (u1, u2, theta, v1, v2, q)."""
        X = X.contiguous()
        assert X.dtype == torch.float64 and X.is_cuda and X.shape == (6, *self._shape(slot))
        self._keep[("in", slot)] = X
        self._check(lib().ap_dvm_set_state(self._h, slot, _ptr(X)))

    def set_equilibrium(self, u1: torch.Tensor, u2: torch.Tensor, p: torch.Tensor, slot: int = 0):
        ts = [t.contiguous() for t in (u1, u2, p)]
        for t in ts:
            assert t.dtype == torch.float64 and t.is_cuda and t.shape == self._shape(slot)
        self._keep[("in", slot)] = ts
        self._check(lib().ap_dvm_set_equilibrium(self._h, slot, *[_ptr(t) for t in ts]))

    def set_populations(self, dF: torch.Tensor, slot: int = 0):
        dF = dF.contiguous()
        assert dF.is_cuda and dF.shape == (6, *self._shape(slot)) and dF.dtype in (torch.float64, torch.float32)
        self._keep[("in", slot)] = dF
        self._check(lib().ap_dvm_set_populations(self._h, slot, _ptr(dF), int(dF.dtype == torch.float32)))

    def set_theta(self, theta: torch.Tensor, slot: int = 0):
        """FP32_DEV_TH: overwrite the carried theta plane ((ny, nx) float64 CUDA tensor)."""
        theta = theta.contiguous()
        assert theta.dtype == torch.float64 and theta.is_cuda and theta.shape == self._shape(slot)
        self._keep[("theta", slot)] = theta
        self._check(lib().ap_dvm_set_theta(self._h, slot, _ptr(theta)))

    def get_state(self, slot: int = 0, out: torch.Tensor | None = None) -> torch.Tensor:
        out = torch.empty((6, *self._shape(slot)), dtype=torch.float64, device=self.device) if out is None else out
        self._check(lib().ap_dvm_get_state(self._h, slot, _ptr(out)))
        return out

    def get_populations(self, slot: int = 0, dtype=torch.float64) -> torch.Tensor:
        out = torch.empty((6, *self._shape(slot)), dtype=dtype, device=self.device)
        self._check(lib().ap_dvm_get_populations(self._h, slot, _ptr(out), int(dtype == torch.float32)))
        return out

    def moments(self, slot: int = 0):
        """(rho, u1, u2, p) as float64 CUDA tensors."""
        out = torch.empty((4, *self._shape(slot)), dtype=torch.float64, device=self.device)
        self._check(lib().ap_dvm_moments(self._h, slot, *[_ptr(out[k]) for k in range(4)]))
        return out[0], out[1], out[2], out[3]

    def diagnostics(self, slot: int = 0, vorticity: bool = False) -> dict:
        """Sec. 4 diagnostics of the current state: max |D_0 . u|, its area-weighted
        L2 norm, the enstrophy and (optionally) the vorticity plane (float64 CUDA tensor)."""
        out = (ctypes.c_double * 3)()
        w = torch.empty(self._shape(slot), dtype=torch.float64, device=self.device) if vorticity else None
        self._check(lib().ap_dvm_diagnostics(self._h, slot, _ptr(w), out))
        d = {"div_max": out[0], "div_l2": out[1], "enstrophy": out[2]}
        if w is not None:
            d["vorticity"] = w
        return d

    # ---- stepping
    def step(self, nsteps: int = 1):
        self._check(lib().ap_dvm_step(self._h, int(nsteps)))

    def set_graph_steps(self, k: int):
        self._check(lib().ap_dvm_set_graph_steps(self._h, int(k)))

    def set_tile(self, tile: int):
        self._check(lib().ap_dvm_set_tile(self._h, int(tile)))

    @property
    def tile(self) -> int:
        return lib().ap_dvm_get_tile(self._h)

    @property
    def launches_per_step(self) -> int:
        return lib().ap_dvm_launches_per_step(self._h)

    def sync_status(self):
        self._check(lib().ap_dvm_sync_status(self._h))

    def check_wait_timeout(self, wait_ns: int):
        """Enqueue one kernel whose bounded device wait expires after wait_ns (the next
        sync_status raises AP_DVM_ERR_TIMEOUT)."""
        self._check(lib().ap_dvm_check_wait_timeout(self._h, int(wait_ns)))

    def profile(self, enable: bool):
        """Per-kernel CUDA-event timing of the following ap_dvm_step calls."""
        self._check(lib().ap_dvm_profile_enable(self._h, int(enable)))

    def profile_read(self) -> dict:
        """{kernel: (total_ms, launches)} since profiling was enabled."""
        names = (ctypes.c_char_p * 8)()
        ms = (ctypes.c_double * 8)()
        cnt = (ctypes.c_long * 8)()
        n = lib().ap_dvm_profile_read(self._h, names, ms, cnt, 8)
        if n < 0:
            self._check(4)
        return {names[k].decode(): (ms[k], cnt[k]) for k in range(n) if cnt[k] > 0}


class Solver(_Handle):
    """One solve (ap_dvm_create)."""

    def __init__(self, params: Params, device="cuda", stream=None):
        super().__init__()
        self.device = torch.device(device)
        self.params = params.copy()
        self._params = {0: self.params}
        n = lib().ap_dvm_workspace_size(ctypes.byref(self.params))
        if n == 0:
            raise ApDvmError(1, "invalid parameters")
        self.workspace = torch.empty(n, dtype=torch.uint8, device=self.device)
        self._check(lib().ap_dvm_create(ctypes.byref(self.params), _ptr(self.workspace), n,
                                        _stream_ptr(stream), ctypes.byref(self._h)))

    def run_host(self, X_host: torch.Tensor, nsteps: int) -> torch.Tensor:
        """End-to-end call on host buffers (ap_dvm_run_host)."""
        X_host = X_host.contiguous()
        assert X_host.dtype == torch.float64 and not X_host.is_cuda
        out = torch.empty_like(X_host, pin_memory=X_host.is_pinned())
        stage = self._keep.get("stage")
        if stage is None or stage.shape != X_host.shape:
            stage = torch.empty(X_host.shape, dtype=torch.float64, device=self.device)
            self._keep["stage"] = stage
        self._check(lib().ap_dvm_run_host(self._h, 0, _ptr(X_host), _ptr(out), _ptr(stage), int(nsteps)))
        return out


class Batch(_Handle):
    """Many uneven solves stepped by the same launches (ap_dvm_batch_create)."""

    def __init__(self, template: Params, capacity: int, device="cuda", stream=None):
        super().__init__()
        self.device = torch.device(device)
        self.template = template.copy()
        self.capacity = capacity
        self._params = {}
        self._ws = {}
        n = lib().ap_dvm_batch_workspace_size(ctypes.byref(self.template), capacity)
        if n == 0:
            raise ApDvmError(1, "invalid batch template")
        self.workspace = torch.empty(n, dtype=torch.uint8, device=self.device)
        self._check(lib().ap_dvm_batch_create(ctypes.byref(self.template), capacity, _ptr(self.workspace), n,
                                              _stream_ptr(stream), ctypes.byref(self._h)))

    @staticmethod
    def instance_bytes(params: Params) -> int:
        return lib().ap_dvm_instance_workspace_size(ctypes.byref(params))

    def attach(self, slot: int, params: Params, workspace: torch.Tensor | None = None):
        params = params.copy()
        n = self.instance_bytes(params)
        if n == 0:
            raise ApDvmError(1, "invalid instance parameters")
        ws = torch.empty(n, dtype=torch.uint8, device=self.device) if workspace is None else workspace
        self._check(lib().ap_dvm_attach(self._h, slot, ctypes.byref(params), _ptr(ws), ws.numel()))
        self._params[slot] = params
        self._ws[slot] = ws

    def detach(self, slot: int):
        self._check(lib().ap_dvm_detach(self._h, slot))
        self._params.pop(slot, None)
        return self._ws.pop(slot, None)

    @property
    def slots(self):
        return sorted(self._params)

    def step_slots(self, nsteps: int, steps: dict):
        """ap_dvm_step_slots: advance the solve in slot k by steps[k] of at most nsteps
        steps (attached slots missing from steps advance by nsteps)."""
        arr = (ctypes.c_int * self.capacity)(*([0] * self.capacity))
        for k in self.slots:
            arr[k] = int(steps.get(k, nsteps))
        self._check(lib().ap_dvm_step_slots(self._h, int(nsteps), arr))
