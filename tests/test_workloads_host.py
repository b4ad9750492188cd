"""The seeded synthetic inputs (paper_2512_19847_gb300/workloads.py), which both the oracle
tests and the GPU path take: the properties their recipes state — divergence-free fields
with the stated spectrum and the incompressible pressure, the parameter draws' sets and
ranges, the Poisson arrival process — and the time-step rules, checked without a GPU."""
import math

import numpy as np
import pytest

from paper_2512_19847_gb300 import workloads as W


def _k(n):
    return np.fft.fftfreq(n, d=1.0 / n)


def _spectral_div(u1, u2):
    n = u1.shape[0]
    k = _k(n)
    return np.real(np.fft.ifft2(1j * k[None, :] * np.fft.fft2(u1) + 1j * k[:, None] * np.fft.fft2(u2)))


def _pressure_residual(u1, u2, p):
    """|Delta p + div((u.grad) u)| relative to its terms, spectrally."""
    n = u1.shape[0]
    k = _k(n)
    KX, KY = k[None, :], k[:, None]
    d = lambda f, K: np.real(np.fft.ifft2(1j * K * np.fft.fft2(f)))
    rhs = -(d(u1, KX) ** 2 + 2 * d(u1, KY) * d(u2, KX) + d(u2, KY) ** 2)
    lap = np.real(np.fft.ifft2(-(KX * KX + KY * KY) * np.fft.fft2(p)))
    return np.max(np.abs(lap - (rhs - rhs.mean()))) / np.max(np.abs(rhs))


@pytest.mark.parametrize("n,kmax", [(64, 16), (48, 8)])
def test_random_divfree_field(n, kmax):
    u1, u2, p = W.random_divfree(n, seed=5, kmax=kmax)
    assert np.max(np.hypot(u1, u2)) == pytest.approx(1.0)                # normalised
    assert np.max(np.abs(_spectral_div(u1, u2))) < 1e-12                  # divergence-free
    # spectral support: integer wave vectors with 0 < |k| <= kmax only
    k = _k(n)
    K2 = k[None, :] ** 2 + k[:, None] ** 2
    E = np.abs(np.fft.fft2(u1)) ** 2 + np.abs(np.fft.fft2(u2)) ** 2
    assert E[(K2 > kmax * kmax) | (K2 == 0)].sum() < 1e-20 * E.sum()
    assert abs(p.mean()) < 1e-14 and _pressure_residual(u1, u2, p) < 1e-10


def test_random_divfree_is_seeded():
    a = W.random_divfree(64, seed=9)
    b = W.random_divfree(64, seed=9)
    c = W.random_divfree(64, seed=10)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])
    with pytest.raises(ValueError):
        W.random_divfree(32, seed=1, kmax=16)


def test_taylor_green():
    n = 32
    u1, u2, p = W.taylor_green(n)
    X, Y = W.cell_centres(n, n)
    assert np.allclose(u1, np.sin(X) * np.cos(Y)) and np.allclose(u2, -np.cos(X) * np.sin(Y))
    assert np.max(np.abs(_spectral_div(u1, u2))) < 1e-13
    assert _pressure_residual(u1, u2, p) < 1e-12


def test_batched_draws():
    d = W.batched_draws(4096, seed=3)
    assert len(d) == 4096 and {x.n for x in d} == {64, 128, 256, 512}
    eps = np.array([x.eps for x in d])
    mach = np.array([x.mach for x in d])
    assert eps.min() >= 1e-6 and eps.max() <= 1.0 and mach.min() >= 1e-3 and mach.max() <= 1e-1
    # log-uniform: the mean of log eps sits at the middle of the log range
    assert np.mean(np.log10(eps)) == pytest.approx(-3.0, abs=0.1)
    assert np.mean(np.log10(mach)) == pytest.approx(-2.0, abs=0.05)
    again = W.batched_draws(4096, seed=3)
    assert [(x.n, x.eps, x.seed) for x in d] == [(x.n, x.eps, x.seed) for x in again]


def test_poisson_requests():
    r = W.poisson_requests(20000, rate_hz=25.0, seed=11)
    t = np.array([x.arrival for x in r])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / 25.0, rel=0.03)
    assert gaps.std() == pytest.approx(1 / 25.0, rel=0.05)                # exponential: std = mean
    assert {x.n for x in r} == {128, 256, 512, 1024}
    steps = np.array([x.steps for x in r])
    assert steps.min() >= 50 and steps.max() <= 500
    eps = np.array([x.eps for x in r])
    assert eps.min() >= 1e-6 and eps.max() <= 1e-1


def test_time_step_rules():
    u1, u2, _ = W.taylor_green(64)
    dx = 2 * math.pi / 64
    umax = float(np.max(np.hypot(u1, u2)))
    assert W.cfl_dt(u1, u2, dx) == pytest.approx(0.5 * dx / umax)
    assert W.stable_dt(u1, u2, dx, 0.0) == pytest.approx(0.4 * dx / umax)        # no viscous bound
    assert W.stable_dt(u1, u2, dx, 10.0) == pytest.approx(0.32 * dx * dx / 2.5)   # nu = tau / 4
    dt, n = W.fixed_time_dt(1.0, 0.03)
    assert n == 34 and n * dt == pytest.approx(1.0) and dt <= 0.03
