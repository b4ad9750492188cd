"""Seeded synthetic inputs for the AP IMEX-RK D2V6 solver.

This module is the only code shared by the CUDA path's tests/bench and the
CPU oracle.  It produces *inputs only*: initial velocity and pressure fields
on the cell-centred periodic grid, a CFL time step, random perturbation
fields and the parameter draws of the batched / served workloads.  It holds
none of the scheme's arithmetic (no equilibrium, no moment map, no stencil,
no relaxation, no Helmholtz solve of the method).

Grid convention (Sec. 3.2 of the paper: variables at cell centres): an
``ny x nx`` array indexed ``[j, i]`` holds the value at
``x_i = (i + 1/2) Lx/nx``, ``y_j = (j + 1/2) Ly/ny``; row-major, x fastest.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TWO_PI = 2.0 * math.pi


def cell_centres(nx: int, ny: int, Lx: float = TWO_PI, Ly: float = TWO_PI):
    """Return (X, Y) meshgrids of cell-centre coordinates, shape (ny, nx)."""
    x = (np.arange(nx, dtype=np.float64) + 0.5) * (Lx / nx)
    y = (np.arange(ny, dtype=np.float64) + 0.5) * (Ly / ny)
    return np.meshgrid(x, y, indexing="xy")


def taylor_green(nx: int, ny: int | None = None, t: float = 0.0, nu: float = 0.0):
    """Taylor-Green vortex on [0, 2pi)^2 (the headline benchmark workload; not one of the paper's experiments).

    u = (sin x cos y, -cos x sin y) e^{-2 nu t},  p = (cos 2x + cos 2y)/4 e^{-4 nu t}.
    This (u, p) solves the incompressible Navier-Stokes equations with
    viscosity nu exactly (checked by substitution); the scheme's limit has
    nu = tau/4 (Sec. 2.1, INS limit with Re = 4/tau).
    Returns (u1, u2, p), each (ny, nx) float64.
    """
    ny = nx if ny is None else ny
    X, Y = cell_centres(nx, ny)
    f = math.exp(-2.0 * nu * t)
    u1 = np.sin(X) * np.cos(Y) * f
    u2 = -np.cos(X) * np.sin(Y) * f
    p = 0.25 * (np.cos(2 * X) + np.cos(2 * Y)) * f * f
    return u1, u2, p


def double_shear_layer(nx: int, ny: int | None = None, inv_rho: float = 30.0, delta: float = 0.05,
                       nodes: bool = False):
    """Double shear layer of Sec. 4.1 (thick: inv_rho = 15/pi; thin, Sec. 4.2: 50/pi).

    u1 = tanh(inv_rho (y - pi/2)) for y <= pi, tanh(inv_rho (3pi/2 - y)) above;
    u2 = delta sin x; pressure input p = 0 (so theta^0 = |u^0|^2/2).
    Sampled at the cell centres, or with nodes=True at the points (i dx, j dy), so
    that grids of 2^k cells are nested (every coarse point is a fine one).
    Returns (u1, u2, p).
    """
    ny = nx if ny is None else ny
    if nodes:
        X, Y = np.meshgrid(np.arange(nx, dtype=np.float64) * (TWO_PI / nx),
                           np.arange(ny, dtype=np.float64) * (TWO_PI / ny), indexing="xy")
    else:
        X, Y = cell_centres(nx, ny)
    u1 = np.where(Y <= math.pi, np.tanh(inv_rho * (Y - math.pi / 2)), np.tanh(inv_rho * (1.5 * math.pi - Y)))
    u2 = delta * np.sin(X)
    p = np.zeros_like(u1)
    return u1, u2, p


def kelvin_helmholtz(nx: int, ny: int | None = None):
    """Kelvin-Helmholtz initial data of Sec. 4.3 on [0, 4pi)^2: u1 = cos y, u2 = 0.03 sin(x/2)."""
    ny = nx if ny is None else ny
    X, Y = cell_centres(nx, ny, 2 * TWO_PI, 2 * TWO_PI)
    return np.cos(Y), 0.03 * np.sin(0.5 * X), np.zeros((ny, nx))


def _spectral_derivatives(f_hat: np.ndarray, L: float):
    n = f_hat.shape[0]
    k = np.fft.fftfreq(n, d=1.0 / n) * (TWO_PI / L)
    KX = k[None, :]
    KY = k[:, None]
    return KX, KY


def random_divfree(n: int, seed: int, kmax: int = 16, normalise: bool = True):
    """Seeded random divergence-free field (precision-form and batched workloads).

    Stream function psi = sum_{0<|k|<=kmax} |k|^-2 cos(k.x + phi_k), phases
    phi_k ~ U[0, 2pi) drawn from numpy's PCG64 with ``seed`` for every
    integer wave vector in the half plane; u = (d_y psi, -d_x psi) evaluated
    spectrally (exact for the trigonometric polynomial), scaled so that
    max |u| = 1 on the grid.  The input pressure p solves
    Delta p = -div((u.grad) u) spectrally (well-prepared data for the INS
    limit; zero mean).  Requires n > 2*kmax.  Returns (u1, u2, p).
    """
    if n <= 2 * kmax:
        raise ValueError("grid too small for kmax")
    rng = np.random.Generator(np.random.PCG64(seed))
    psi_hat = np.zeros((n, n), dtype=np.complex128)
    for ky in range(0, kmax + 1):
        for kx in range(-kmax, kmax + 1):
            if ky == 0 and kx <= 0:
                continue  # half plane: (kx, ky) and (-kx, -ky) give the same cosine
            kk = kx * kx + ky * ky
            if kk == 0 or kk > kmax * kmax:
                continue
            phi = rng.uniform(0.0, TWO_PI)
            amp = 1.0 / kk
            # cos(k.x + phi) = (e^{i(k.x+phi)} + e^{-i(k.x+phi)})/2; grid origin at the cell centre offset
            psi_hat[ky % n, kx % n] += 0.5 * amp * np.exp(1j * phi) * n * n
            psi_hat[(-ky) % n, (-kx) % n] += 0.5 * amp * np.exp(-1j * phi) * n * n
    # account for cell-centred sampling x_i = (i+1/2) dx: shift by half a cell
    k = np.fft.fftfreq(n, d=1.0 / n)
    shift = np.exp(1j * np.pi * k / n)
    psi_hat = psi_hat * shift[None, :] * shift[:, None]
    KX, KY = _spectral_derivatives(psi_hat, TWO_PI)
    u1 = np.real(np.fft.ifft2(1j * KY * psi_hat))
    u2 = np.real(np.fft.ifft2(-1j * KX * psi_hat))
    if normalise:
        s = float(np.max(np.hypot(u1, u2)))
        u1 /= s
        u2 /= s
    # pressure of the incompressible limit: Delta p = -sum_ij d_i u_j d_j u_i
    def d(f, K):
        return np.real(np.fft.ifft2(1j * K * np.fft.fft2(f)))
    u1x, u1y = d(u1, KX), d(u1, KY)
    u2x, u2y = d(u2, KX), d(u2, KY)
    rhs = -(u1x * u1x + 2.0 * u1y * u2x + u2y * u2y)
    rhs_hat = np.fft.fft2(rhs)
    K2 = KX * KX + KY * KY
    K2[0, 0] = 1.0
    p_hat = -rhs_hat / K2
    p_hat[0, 0] = 0.0
    p = np.real(np.fft.ifft2(p_hat))
    return u1, u2, p


def random_moment_state(nx: int, ny: int, seed: int, amp: float = 1.0, modes: int = 4):
    """Seeded smooth random fields for all six moment planes (u1,u2,theta,v1,v2,q).

    Each plane is a sum of ``modes`` random low-wavenumber Fourier modes plus
    a small seeded white-noise component, so that stencils, WENO weights and
    the Helmholtz solve all see non-trivial data.  Not an equilibrium: used
    for element-wise parity tests of one IMEX step.
    Returns a float64 array of shape (6, ny, nx).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y = cell_centres(nx, ny)
    out = np.zeros((6, ny, nx))
    for m in range(6):
        f = np.zeros((ny, nx))
        for _ in range(modes):
            kx, ky = rng.integers(-3, 4, size=2)
            ph = rng.uniform(0, TWO_PI)
            f += rng.uniform(-1, 1) * np.cos(kx * X + ky * Y + ph)
        f += 0.05 * rng.standard_normal((ny, nx))
        out[m] = amp * f
    return out


def cfl_dt(u1: np.ndarray, u2: np.ndarray, dx: float, cfl: float = 0.5) -> float:
    """dt = cfl * dx / max|u| (the benchmark CFL rule; the paper does not state dt)."""
    umax = float(np.max(np.hypot(u1, u2)))
    return cfl * dx / max(umax, 1e-300)


def stable_dt(u1: np.ndarray, u2: np.ndarray, dx: float, tau: float, cfl: float = 0.4, visc: float = 0.32) -> float:
    """dt = min(cfl dx / max|u|, visc dx^2 / nu) with nu = tau/4.

    In the limit the viscous term (tau/4) Delta u of the scheme is explicit
    (Sec. 3.1, proof of Theorem 3.4), so besides the advective CFL bound the
    step obeys a parabolic bound; with the second-order tableau and WENO
    fluxes the explicit viscous part is stable up to nu dt/dx^2 ~ 0.5 over
    short runs (measured with the oracle).  Runs of thousands of steps on
    512^2 grids (the shear layers of Sec. 4, the random fields) need margin:
    cfl = 0.4 and visc = 0.32 keep them bounded where 0.5 and 0.4 did not."""
    dt = cfl_dt(u1, u2, dx, cfl)
    nu = 0.25 * tau
    if nu > 0:
        dt = min(dt, visc * dx * dx / nu)
    return dt


def fixed_time_dt(t_end: float, dt_cfl: float):
    """Split [0, t_end] into n = ceil(t_end/dt_cfl) equal steps; return (dt, n)."""
    n = max(1, int(math.ceil(t_end / dt_cfl - 1e-12)))
    return t_end / n, n


@dataclass
class InstanceDraw:
    n: int
    eps: float
    mach: float
    steps: int
    seed: int


def batched_draws(count: int = 256, seed: int = 2512, sides=(64, 128, 256, 512),
                  eps_range=(1e-6, 1.0), mach_range=(1e-3, 1e-1), steps: int = 200):
    """Parameter draws of the batched workload: side uniform in ``sides``,
    eps and Mach log-uniform in their ranges, one field seed per instance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        n = int(rng.choice(sides))
        eps = float(math.exp(rng.uniform(math.log(eps_range[0]), math.log(eps_range[1]))))
        mach = float(math.exp(rng.uniform(math.log(mach_range[0]), math.log(mach_range[1]))))
        out.append(InstanceDraw(n, eps, mach, steps, int(rng.integers(0, 2**31 - 1))))
    return out


@dataclass
class Request:
    arrival: float
    n: int
    eps: float
    steps: int
    seed: int


def poisson_requests(count: int, rate_hz: float, seed: int = 7, sides=(128, 256, 512, 1024),
                     eps_range=(1e-6, 1e-1), steps_range=(50, 500)):
    """Open-loop request stream of the served workload: Poisson arrivals at
    ``rate_hz``, side uniform in ``sides``, eps log-uniform, steps uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = int(rng.choice(sides))
        eps = float(math.exp(rng.uniform(math.log(eps_range[0]), math.log(eps_range[1]))))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(Request(t, n, eps, steps, int(rng.integers(0, 2**31 - 1))))
    return out
