"""Full-size checks in the launch configuration bench.py times (automatic
tile, one-step CUDA graph): element-wise parity with the oracle at 2048^2,
at the largest grids (4096^2, 4095^2) and at 512^2, the FP32 deviation
form's error on the 2048^2 precision workload, and properties that hold at
any size (incompressible limit, convergence)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ap_dvm_oracle as O  # noqa: E402
from paper_2512_19847_gb300 import api, tableaux, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
A_EX, A_IM = tableaux.gsa2()


def _gpu(n, fields, eps, mach, tau, dt, steps, prec=api.FP64):
    p = api.default_params(n, n, eps=eps, dt=dt, tau=tau, mach=mach, tableau=(A_EX, A_IM), precision=prec)
    s = api.Solver(p)
    s.set_graph_steps(1)
    s.set_equilibrium(*[torch.from_numpy(a).cuda() for a in fields])
    s.step(steps)
    s.sync_status()
    return s.get_state().cpu().numpy()


def _oracle(n, fields, eps, tau, dt, steps):
    o = O.Params(n, n, eps, tau, dt, np.array(A_EX), np.array(A_IM), scheme="WENO5_C4")
    return O.run(O.equilibrium_state(*fields), o, steps)


def _rel(a, b):
    return np.max(np.abs(a - b), axis=(1, 2)) / np.maximum(np.max(np.abs(b), axis=(1, 2)), 1e-300)


@pytest.mark.parametrize("field", ["taylor_green", "random_divfree"])
def test_precision_workload_2048_fp64_parity(field):
    """2048^2, eps = 1e-4, Ma = 1e-3, tau = 0.05 (the bench workload): one step, every cell."""
    n = 2048
    f = W.taylor_green(n) if field == "taylor_green" else W.random_divfree(n, seed=2048)
    dt = W.stable_dt(f[0], f[1], 2 * math.pi / n, 0.05)
    got = _gpu(n, f, 1e-4, 1e-3, 0.05, dt, 1)
    ref = _oracle(n, f, 1e-4, 0.05, dt, 1)
    assert np.all(_rel(got, ref) <= 1e-12), _rel(got, ref)


# bounds at about twice the measured errors (GB300): AP_DVM_FP32_DEV sums theta from the FP32
# populations, where it rides at O(eps); AP_DVM_FP32_DEV_TH carries it in its own FP32 plane
# measured (GB300, this workload, 10 steps): velocity 7.6e-7 for both, pressure 8.4e-4 and 7.0e-5
FP32_BOUNDS = {api.FP32_DEV: (1.6e-6, 1.7e-3), api.FP32_DEV_TH: (1.6e-6, 1.5e-4)}


@pytest.mark.parametrize("prec", [api.FP32_DEV, api.FP32_DEV_TH])
def test_precision_workload_2048_fp32_error(prec):
    """FP32 deviation storage vs all-FP64 on the 2048^2 random divergence-free field,
    eps = 1e-4, Ma = 1e-3, 10 steps: velocity within 1e-5 of max |u| (the stated
    target), velocity and pressure errors within about twice their measured values."""
    n = 2048
    f = W.random_divfree(n, seed=2048)
    dt = W.stable_dt(f[0], f[1], 2 * math.pi / n, 0.05)
    a = _gpu(n, f, 1e-4, 1e-3, 0.05, dt, 10)
    b = _gpu(n, f, 1e-4, 1e-3, 0.05, dt, 10, prec=prec)
    vel = np.max(np.hypot(a[0] - b[0], a[1] - b[1])) / np.max(np.hypot(a[0], a[1]))
    pa = a[2] - 0.5 * (a[0] ** 2 + a[1] ** 2)
    pb = b[2] - 0.5 * (b[0] ** 2 + b[1] ** 2)
    pr = np.max(np.abs((pb - pb.mean()) - (pa - pa.mean()))) / np.max(np.abs(pa - pa.mean()))
    print(f"FP32 form {prec}, 2048^2 random field, 10 steps: velocity {vel:.2e}, pressure {pr:.2e}")
    vb, pbnd = FP32_BOUNDS[prec]
    assert vel <= min(vb, 1e-5), vel
    assert pr <= pbnd, pr


@pytest.mark.parametrize("n", [4096, 4095])
def test_largest_grids_fp64_parity(n):
    """The largest grids: 4096^2 (power of two) and 4095^2 (Bluestein with M = 8192 on both
    axes, ragged tiles, plain staging), the bench workload's parameters, one step, every cell."""
    f = W.taylor_green(n)
    dt = W.stable_dt(f[0], f[1], 2 * math.pi / n, 0.05)
    got = _gpu(n, f, 1e-4, 1e-3, 0.05, dt, 1)
    ref = _oracle(n, f, 1e-4, 0.05, dt, 1)
    assert np.all(_rel(got, ref) <= 1e-12), _rel(got, ref)


@pytest.mark.parametrize("eps", [1.0, 1e-2, 1e-4, 1e-6])
def test_ap_sweep_shear_512_parity(eps):
    """Double shear layer 512^2 (1/rho = 30), Ma = 1e-2, eps sweep; 3 steps (the thin
    layer amplifies round-off differences ~2.5x per step)."""
    n = 512
    f = W.double_shear_layer(n)
    dt = W.stable_dt(f[0], f[1], 2 * math.pi / n, 0.05)
    got = _gpu(n, f, eps, 1e-2, 0.05, dt, 3)
    ref = _oracle(n, f, eps, 0.05, dt, 3)
    assert np.all(_rel(got, ref) <= 1e-12), _rel(got, ref)


def test_taylor_green_incompressible_limit_256():
    """eps = 1e-6: u follows the INS Taylor-Green solution with nu = tau/4, kinetic
    energy decays as exp(-4 nu t) (velocity as exp(-2 nu t))."""
    n, tau, T = 256, 0.4, 0.5
    f = W.taylor_green(n)
    dt, ns = W.fixed_time_dt(T, W.stable_dt(f[0], f[1], 2 * math.pi / n, tau))
    X = _gpu(n, f, 1e-6, 1e-2, tau, dt, ns)
    e1, e2, _ = W.taylor_green(n, t=T, nu=tau / 4)
    err = max(np.abs(X[0] - e1).max(), np.abs(X[1] - e2).max())
    ke = np.mean(X[0] ** 2 + X[1] ** 2) / np.mean(f[0] ** 2 + f[1] ** 2)
    assert err < 1e-6
    assert abs(ke / math.exp(-tau * T) - 1) < 1e-5


def test_taylor_green_refinement_order_64_to_512():
    """Grid and dt refinement 64 -> 512 (dt proportional to dx) in the limit eps = 1e-6:
    the error against the exact INS solution converges at second order or better
    (second-order tableau, fourth-order central differences, WENO5)."""
    tau, T = 0.05, 0.25
    errs = []
    for n in (64, 128, 256, 512):
        f = W.taylor_green(n)
        dt, ns = W.fixed_time_dt(T, 0.25 * 2 * math.pi / n)
        X = _gpu(n, f, 1e-6, 1e-2, tau, dt, ns)
        e1, e2, _ = W.taylor_green(n, t=T, nu=tau / 4)
        errs.append(max(np.abs(X[0] - e1).max(), np.abs(X[1] - e2).max()))
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(3)]
    print("TG refinement errors", errs, "orders", orders)
    assert min(orders) > 1.8, (errs, orders)
