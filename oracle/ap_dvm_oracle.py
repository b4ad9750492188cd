"""CPU oracle (test infrastructure only) for the AP IMEX-RK scheme of
"Asymptotic preserving methods for the low Mach limit in discrete velocity
models approximating kinetic equations" (Dimarco, Klar, Koefler, Pareschi).

THIS MODULE IS TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  The
product (the CUDA library and its Python binding) never imports, links or
executes anything under ``oracle/``; the two share no code.

It is a plain, slow, obviously-correct float64 numpy implementation of the
fully discrete scheme of Sec. 3.2 (the four update formulas that instantiate
Algorithm 1 of Sec. 3.1 with the finite-difference operators of Sec. 3.2),
executed stage by stage in the paper's order.  Every stage field is stored;
operators of a stage are evaluated once and cached, which does not change
the arithmetic.  Library primitives used as steps: numpy's FFT for the
periodic Helmholtz solve (Algorithm 1, step 2).

Readings of places where the paper is silent, garbled or at odds with itself
(each is pinned by a test in ``tests/test_oracle_pins.py``):

* G1  v1 is taken as sum((c2^2 - 1/2) F) = -sum((c1^2 - 1/2) F); with this sign
      the moment system of Sec. 2.1 and F(u) of Sec. 3 hold as printed.
* G2  the q equation carries div v = d_x v1 + d_y v2 (vector form, Sec. 3).
* G3  relaxation is -(F - F^eq)/(eps^2 tau) (the printed collision sign would
      anti-relax).
* G4  the theta-history term of the Helmholtz right-hand side (Algorithm 1,
      step 2 and the fully discrete scheme) enters with a MINUS sign, as the
      derivation of the theta stage equation in the proof of Theorem 3.4
      gives; ``theta_hist_sign=+1`` keeps the printed sign for experiments.
* G5  the mean (k = 0) Fourier mode of theta^(i) is set to mean(theta^n)
      (all other right-hand-side terms have zero periodic mean).
* G6  the dissipation partner of the LF flux of B(v^(j)) in step 3 is u^(j)
      for j < i and, for j = i (u^(i) is still unknown), the explicit-weight
      predictor P^(i) = (1/a_ii) sum_{j<i} (atilde_ij - a_ij) u^(j), which makes
      the LF dissipation accumulate with the explicit tableau, like the
      convective terms in the limit of Theorem 3.4.  The lagged u^(i-1) and
      u^n readings are linearly unstable for the second-order tableau of
      Sec. 4.1 at CFL 0.5 (kept as options to pin that).  x pairs
      (-v1 <-> u1), (v2 <-> u2), y pairs (v2 <-> u1), (v1 <-> u2).  The LF
      flux of q in step 1 pairs with v1 (x) and v2 (y).  alpha = 1.
* G7  high order: every alpha = 1 LF flux becomes component-wise
      finite-difference WENO with Lax-Friedrichs flux splitting
      g+- = (g +- alpha U)/2; every alpha0 = 0 flux and every central
      difference becomes the fourth-order central difference; the Laplacian
      and D_xx, D_yy become the fourth-order central second derivative and
      2 D_xy the product of the fourth-order first differences.
* G8  Jiang-Shu WENO weights alpha_k = d_k/(eps_W + beta_k)^2 with
      eps_W = 1e-6; WENO3 d = (1/3, 2/3), WENO5 d = (1/10, 6/10, 3/10).
* G9  N cells on [0, L), cell centred.
* G10 population view: f = dF/(rho0 A) with sum f/2 = eps theta,
      sum c f = u, sum (c1^2-1/2) f = -eps v1, sum c1 c2 f = eps v2,
      sum c1 (c2^2 - 1/4) f = eps^2 q.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SCHEMES = ("LF1_C2", "WENO3_C4", "WENO5_C4")
U1, U2, TH, V1, V2, Q = range(6)


# ---------------------------------------------------------------------------
# IMEX tableaux (Sec. 4.1)
# ---------------------------------------------------------------------------

def tableau_euler():
    """First-order GSA Euler IMEX scheme (Sec. 4.1).  Returns (A_ex, w_ex, A_im, w_im)."""
    A_ex = np.array([[0.0, 0.0], [1.0, 0.0]])
    A_im = np.array([[0.0, 0.0], [0.0, 1.0]])
    return A_ex, A_ex[-1].copy(), A_im, A_im[-1].copy()


def tableau_gsa2(c: float = 2.25):
    """Second-order GSA IMEX-RK scheme of Sec. 4.1 with gamma = (c - 1/2)/(c - 1).

    Explicit rows (0,0,0), (c,0,0), (1-1/(2c), 1/(2c), 0); implicit rows
    (0,0,0), (0,c,0), (0, 1-gamma, gamma); weights equal the last rows (GSA).
    """
    g = (c - 0.5) / (c - 1.0)
    A_ex = np.array([[0.0, 0.0, 0.0], [c, 0.0, 0.0], [1.0 - 1.0 / (2 * c), 1.0 / (2 * c), 0.0]])
    A_im = np.array([[0.0, 0.0, 0.0], [0.0, c, 0.0], [0.0, 1.0 - g, g]])
    return A_ex, A_ex[-1].copy(), A_im, A_im[-1].copy()


def tableau_ars4():
    """A four-stage second-order GSA IMEX pair of ARS type (Sec. 3.1 definitions:
    a_11 = 0 and a zero first implicit column, a_ii = 1/2 for i >= 2), with nodes
    c = (0, 1/2, 3/2, 1) shared by both tableaux, weights equal to the last rows
    (GSA), and sum w c = sum w~ c = 1/2.  Not one of the paper's pairs: it
    exercises Algorithm 1 with s = 4, every explicit entry below the diagonal
    nonzero, and every dissipation-partner weight atilde_ij - a_ij nonzero."""
    A_ex = np.array([[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.75, 0.75, 0.0, 0.0], [0.5, 0.25, 0.25, 0.0]])
    A_im = np.array([[0.0, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 1.0, 0.5, 0.0], [0.0, 0.75, -0.25, 0.5]])
    return A_ex, A_ex[-1].copy(), A_im, A_im[-1].copy()


# ---------------------------------------------------------------------------
# Parameters and state
# ---------------------------------------------------------------------------

@dataclass
class Params:
    nx: int
    ny: int
    eps: float
    tau: float
    dt: float
    A_ex: np.ndarray
    A_im: np.ndarray
    scheme: str = "WENO5_C4"
    Lx: float = 2 * math.pi
    Ly: float = 2 * math.pi
    weno_eps: float = 1e-6
    alpha: float = 1.0            # LF dissipation of the alpha = 1 fluxes (Sec. 3.2)
    theta_hist_sign: float = -1.0  # the theta-history sign (reading G4 above)
    # test-only: "consistent" replaces D_Delta by D_0.D_0, D_0^2:B(v) by D_0.(D_0.B(v))
    # and sets alpha = 0, so that the stage equations of Sec. 3.1 hold exactly.
    operators: str = "paper"
    # the j = i dissipation partner (reading G6 above): "explicit" (default) or the
    # rejected "lagged" u^(i-1) and "un" u^n readings (kept to pin their instability)
    partner: str = "explicit"

    @property
    def dx(self):
        return self.Lx / self.nx

    @property
    def dy(self):
        return self.Ly / self.ny

    @property
    def s(self):
        return self.A_im.shape[0]


# ---------------------------------------------------------------------------
# Periodic shifts and central differences (Sec. 3.2)
# ---------------------------------------------------------------------------

def sx(f, k):
    """f at (i+k, j), periodic: sx(f, k)[j, i] = f[j, (i+k) mod nx]."""
    return np.roll(f, -k, axis=1)


def sy(f, k):
    """f at (i, j+k), periodic."""
    return np.roll(f, -k, axis=0)


def _order(p: Params) -> int:
    return 2 if p.scheme == "LF1_C2" else 4


def dx_c(f, p: Params):
    """Central first difference in x: D_0 (2nd order) or its 4th-order version (G7)."""
    if _order(p) == 2:
        return (sx(f, 1) - sx(f, -1)) / (2 * p.dx)
    return (-sx(f, 2) + 8 * sx(f, 1) - 8 * sx(f, -1) + sx(f, -2)) / (12 * p.dx)


def dy_c(f, p: Params):
    if _order(p) == 2:
        return (sy(f, 1) - sy(f, -1)) / (2 * p.dy)
    return (-sy(f, 2) + 8 * sy(f, 1) - 8 * sy(f, -1) + sy(f, -2)) / (12 * p.dy)


def dxx_c(f, p: Params):
    """Central second difference in x (compact 3-point, or 5-point 4th order)."""
    if _order(p) == 2:
        return (sx(f, 1) - 2 * f + sx(f, -1)) / p.dx ** 2
    return (-sx(f, 2) + 16 * sx(f, 1) - 30 * f + 16 * sx(f, -1) - sx(f, -2)) / (12 * p.dx ** 2)


def dyy_c(f, p: Params):
    if _order(p) == 2:
        return (sy(f, 1) - 2 * f + sy(f, -1)) / p.dy ** 2
    return (-sy(f, 2) + 16 * sy(f, 1) - 30 * f + 16 * sy(f, -1) - sy(f, -2)) / (12 * p.dy ** 2)


def laplacian(f, p: Params):
    """D_Delta theta (Sec. 3.2): compact 5-point Laplacian (4th-order version under G7)."""
    if p.operators == "consistent":
        return dx_c(dx_c(f, p), p) + dy_c(dy_c(f, p), p)
    return dxx_c(f, p) + dyy_c(f, p)


def laplacian_symbol(n: int, h: float, p: Params):
    """Eigenvalue of the 1D second-difference operator on the DFT mode k = 0..n-1
    (the compact 3-point or the 4th-order 5-point stencil of Sec. 3.2)."""
    phi = 2 * math.pi * np.arange(n) / n
    if p.operators == "consistent":
        # D_0 D_0 with D_0 central: symbol (i sin(phi)/h)^2 (2nd order) or the 4th-order analogue
        if _order(p) == 2:
            d = np.sin(phi) / h
        else:
            d = (8 * np.sin(phi) - np.sin(2 * phi)) / (6 * h)
        return -d * d
    # (2 cos phi - 2) and (-2 cos 2phi + 32 cos phi - 30)/12 written without
    # cancellation for small phi: -4 sin^2(phi/2) and 2 sin^2(phi/2)(cos phi - 7)/3
    s2 = np.sin(0.5 * phi) ** 2
    if _order(p) == 2:
        return -4.0 * s2 / h ** 2
    return 2.0 * s2 * (np.cos(phi) - 7.0) / (3.0 * h ** 2)


def div_c(w1, w2, p: Params):
    """D_0 . w (Sec. 3.2, divergence of u in the Helmholtz equation; alpha0 = 0 fluxes)."""
    return dx_c(w1, p) + dy_c(w2, p)


def vorticity(u1, u2, p: Params):
    """omega = D_0x u2 - D_0y u1, the central vorticity of the Sec. 4 figures and
    Tables 1-2 (the paper does not define it; the central difference is the natural
    discrete curl), with the scheme's central difference."""
    return dx_c(u2, p) - dy_c(u1, p)


def diagnostics(X, p: Params) -> dict:
    """Flow diagnostics of Sec. 4: max |D_0 . u| (the divergence history of
    Figs. 2-3), its area-weighted L2 norm (sum (D_0 . u)^2 dx dy)^(1/2), the
    enstrophy (1/2) sum omega^2 dx dy, and the vorticity plane."""
    d = div_c(X[0], X[1], p)
    w = vorticity(X[0], X[1], p)
    area = p.dx * p.dy
    return {"div_max": float(np.max(np.abs(d))), "div_l2": float(math.sqrt(np.sum(d * d) * area)),
            "enstrophy": float(0.5 * np.sum(w * w) * area), "vorticity": w}


def d0sq_B(v1, v2, p: Params):
    """D_0^2 : B(v) = -D_xx v1 + 2 D_xy v2 + D_yy v1 (Sec. 3.2)."""
    if p.operators == "consistent":
        b1, b2 = divB_central(v1, v2, p)
        return div_c(b1, b2, p)
    return -dxx_c(v1, p) + 2 * dx_c(dy_c(v2, p), p) + dyy_c(v1, p)


def divB_central(w1, w2, p: Params):
    """D^0_LF . B(w) with alpha0 = 0, i.e. the central divergence of
    B(w) = [[-w1, w2], [w2, w1]] taken row-wise (Sec. 3 vector form):
    ( d_x(-w1) + d_y(w2),  d_x(w2) + d_y(w1) )."""
    return (dx_c(-w1, p) + dy_c(w2, p), dx_c(w2, p) + dy_c(w1, p))


# ---------------------------------------------------------------------------
# Upwind (Lax-Friedrichs / WENO) flux differences (Sec. 3.2, G6-G8)
# ---------------------------------------------------------------------------

def weno5_reconstruct(fm2, fm1, f0, fp1, fp2, eps_w):
    """Jiang-Shu WENO5 value at x_{i+1/2} from the left-biased stencil
    (f_{i-2}, ..., f_{i+2}): three quadratic candidates, smoothness
    indicators beta_k, nonlinear weights from linear weights (1/10, 6/10, 3/10)."""
    p0 = (2 * fm2 - 7 * fm1 + 11 * f0) / 6
    p1 = (-fm1 + 5 * f0 + 2 * fp1) / 6
    p2 = (2 * f0 + 5 * fp1 - fp2) / 6
    b0 = 13.0 / 12.0 * (fm2 - 2 * fm1 + f0) ** 2 + 0.25 * (fm2 - 4 * fm1 + 3 * f0) ** 2
    b1 = 13.0 / 12.0 * (fm1 - 2 * f0 + fp1) ** 2 + 0.25 * (fm1 - fp1) ** 2
    b2 = 13.0 / 12.0 * (f0 - 2 * fp1 + fp2) ** 2 + 0.25 * (3 * f0 - 4 * fp1 + fp2) ** 2
    a0 = 0.1 / (eps_w + b0) ** 2
    a1 = 0.6 / (eps_w + b1) ** 2
    a2 = 0.3 / (eps_w + b2) ** 2
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2)


def weno3_reconstruct(fm1, f0, fp1, eps_w):
    """Jiang-Shu WENO3 value at x_{i+1/2} from the left-biased stencil
    (f_{i-1}, f_i, f_{i+1}): linear candidates, linear weights (1/3, 2/3)."""
    p0 = (-fm1 + 3 * f0) / 2
    p1 = (f0 + fp1) / 2
    b0 = (f0 - fm1) ** 2
    b1 = (fp1 - f0) ** 2
    a0 = (1.0 / 3.0) / (eps_w + b0) ** 2
    a1 = (2.0 / 3.0) / (eps_w + b1) ** 2
    return (a0 * p0 + a1 * p1) / (a0 + a1)


def interface_flux(g, U, shift, p: Params):
    """Numerical flux at the interface (i+1/2) along the axis of ``shift``
    for the flux values g with dissipation partner U.

    LF1 (Sec. 3.2): hat g = (g_i + g_{i+1} - alpha (U_{i+1} - U_i))/2.
    WENO (G7): g+- = (g +- alpha U)/2, hat g = W_left(g+) + W_right(g-).
    Returned array: element i holds the flux at i+1/2.
    """
    a = p.alpha
    if p.scheme == "LF1_C2":
        return 0.5 * (g + shift(g, 1) - a * (shift(U, 1) - U))
    gp = 0.5 * (g + a * U)
    gm = 0.5 * (g - a * U)
    if p.scheme == "WENO3_C4":
        left = weno3_reconstruct(shift(gp, -1), gp, shift(gp, 1), p.weno_eps)
        right = weno3_reconstruct(shift(gm, 2), shift(gm, 1), gm, p.weno_eps)
        return left + right
    left = weno5_reconstruct(shift(gp, -2), shift(gp, -1), gp, shift(gp, 1), shift(gp, 2), p.weno_eps)
    right = weno5_reconstruct(shift(gm, 3), shift(gm, 2), shift(gm, 1), gm, shift(gm, -1), p.weno_eps)
    return left + right


def lf_dx(g, U, p: Params):
    """(hat g_{i+1/2} - hat g_{i-1/2})/dx."""
    fh = interface_flux(g, U, sx, p)
    return (fh - sx(fh, -1)) / p.dx


def lf_dy(g, U, p: Params):
    fh = interface_flux(g, U, sy, p)
    return (fh - sy(fh, -1)) / p.dy


def grad_lf_q(q, v1, v2, p: Params):
    """D_LF q (Sec. 3.2): x flux q with partner v1, y flux q with partner v2."""
    return lf_dx(q, v1, p), lf_dy(q, v2, p)


def divB_lf(v1, v2, u1, u2, p: Params):
    """D_LF . B(v) with dissipation partner u (Sec. 3.2 'the same approach', G6):
    component 1 = Dx(-v1; u1) + Dy(v2; u1), component 2 = Dx(v2; u2) + Dy(v1; u2)."""
    if p.operators == "consistent":
        return divB_central(v1, v2, p)
    return (lf_dx(-v1, u1, p) + lf_dy(v2, u1, p), lf_dx(v2, u2, p) + lf_dy(v1, u2, p))


def F_of_u(u1, u2):
    """F(u) = ((u2^2 - u1^2)/2, u1 u2) (Sec. 3, vector form)."""
    return 0.5 * (u2 * u2 - u1 * u1), u1 * u2


# ---------------------------------------------------------------------------
# Helmholtz solve (Algorithm 1, step 2)
# ---------------------------------------------------------------------------

def helmholtz_solve(R, kappa, theta_mean, p: Params):
    """Solve (D_Delta - kappa) theta = R on the periodic grid by FFT
    diagonalisation; the k = 0 mode is set to theta_mean (G5)."""
    ny, nx = R.shape
    lx = laplacian_symbol(nx, p.dx, p)
    ly = laplacian_symbol(ny, p.dy, p)
    den = ly[:, None] + lx[None, :] - kappa
    Rh = np.fft.fft2(R)
    den[0, 0] = 1.0
    th = Rh / den
    th[0, 0] = theta_mean * nx * ny
    return np.real(np.fft.ifft2(th))


# ---------------------------------------------------------------------------
# One IMEX step: Algorithm 1 (Sec. 3.1) with the operators of Sec. 3.2
# ---------------------------------------------------------------------------

class _Stage:
    __slots__ = ("u1", "u2", "th", "v1", "v2", "q", "cache")

    def __init__(self, u1, u2, th, v1, v2, q):
        self.u1, self.u2, self.th, self.v1, self.v2, self.q = u1, u2, th, v1, v2, q
        self.cache = {}


def _E(st: _Stage, p: Params):
    """Explicit term of step 1 for stage j:
    (tau/4) D0_LF . B(u) + tau eps^2 D_LF q - F(u)."""
    if "E" not in st.cache:
        b1, b2 = divB_central(st.u1, st.u2, p)
        g1, g2 = grad_lf_q(st.q, st.v1, st.v2, p)
        f1, f2 = F_of_u(st.u1, st.u2)
        te2 = p.tau * p.eps ** 2
        st.cache["E"] = (0.25 * p.tau * b1 + te2 * g1 - f1, 0.25 * p.tau * b2 + te2 * g2 - f2)
    return st.cache["E"]


def _explicit_partner(st, A_ex, A, i):
    """Dissipation partner of D_LF . B(v^(i)) in step 3 of stage i (reading G6):
    P^(i) = (1/a_ii) sum_{j<i} (atilde_ij - a_ij) u^(j).  With it the LF
    dissipation of the flux B(v) accumulates with the explicit weights,
    sum_{j<=i} a_ij diss(P_j) = sum_{j<i} atilde_ij diss(u^(j)), as the
    convective terms do in the limit (Theorem 3.4)."""
    a_ii = A[i - 1, i - 1]
    p1 = np.zeros_like(st[0].u1)        # stage 1 of a type-A tableau: the sum over j < 1 is empty
    p2 = np.zeros_like(st[0].u1)
    for j in range(1, i):
        w = A_ex[i - 1, j - 1] - A[i - 1, j - 1]
        if w != 0.0:
            p1 = p1 + w * st[j].u1
            p2 = p2 + w * st[j].u2
    return p1 / a_ii, p2 / a_ii


def _cached(st: _Stage, key, fn):
    if key not in st.cache:
        st.cache[key] = fn()
    return st.cache[key]


def step(X: np.ndarray, p: Params, return_stages: bool = False):
    """Advance the moment state X = (u1, u2, theta, v1, v2, q), shape (6, ny, nx),
    by one GSA IMEX-RK step (Algorithm 1; fully discrete scheme of Sec. 3.2).

    CK/ARS tableaux (a_11 = 0) take stage 1 = X^n (Appendix A); type-A
    tableaux compute stage 1 with the same four steps.  GSA: X^{n+1} = X^(s).
    With ``return_stages`` also returns {i: X^(i)}.
    """
    A_ex, A = p.A_ex, p.A_im
    s = p.s
    dt, eps, tau = p.dt, p.eps, p.tau
    te2 = tau * eps * eps
    Xn = _Stage(*[X[m] for m in range(6)])
    st = {0: Xn}                       # st[0] is only used as the lagged partner u^(0) = u^n
    first = 2 if A[0, 0] == 0.0 else 1
    if first == 2:
        st[1] = Xn
    theta_mean = float(np.mean(Xn.th))

    for i in range(first, s + 1):
        a_ii = A[i - 1, i - 1]
        den = te2 + dt * a_ii
        # ---- step 1: v^(i) in closed form
        sE1 = np.zeros_like(Xn.v1)
        sE2 = np.zeros_like(Xn.v1)
        sV1 = np.zeros_like(Xn.v1)
        sV2 = np.zeros_like(Xn.v1)
        for j in range(1, i):
            if A_ex[i - 1, j - 1] != 0.0:
                e1, e2 = _E(st[j], p)
                sE1 = sE1 + A_ex[i - 1, j - 1] * e1
                sE2 = sE2 + A_ex[i - 1, j - 1] * e2
            if A[i - 1, j - 1] != 0.0:
                sV1 = sV1 + A[i - 1, j - 1] * st[j].v1
                sV2 = sV2 + A[i - 1, j - 1] * st[j].v2
        v1 = (te2 * Xn.v1 - dt * sE1 - dt * sV1) / den
        v2 = (te2 * Xn.v2 - dt * sE2 - dt * sV2) / den
        cur = _Stage(None, None, None, v1, v2, None)

        # ---- step 2: Helmholtz equation for theta^(i)
        kappa = 2 * eps * eps / (dt * dt * a_ii * a_ii)
        R = -kappa * Xn.th
        for j in range(1, i):
            a = A[i - 1, j - 1]
            if a != 0.0:
                Sj = st[j]
                R = R + (a / (dt * a_ii * a_ii)) * _cached(Sj, "divu", lambda: div_c(Sj.u1, Sj.u2, p))
        R = R + (1.0 / (dt * a_ii)) * _cached(Xn, "divu", lambda: div_c(Xn.u1, Xn.u2, p))
        for j in range(1, i + 1):
            a = A[i - 1, j - 1]
            if a != 0.0:
                Sj = st[j] if j < i else cur
                R = R - (a / a_ii) * _cached(Sj, "d0sqB", lambda: d0sq_B(Sj.v1, Sj.v2, p))
        for j in range(1, i):
            a = A[i - 1, j - 1]
            if a != 0.0:
                Sj = st[j]
                R = R + p.theta_hist_sign * (a / a_ii) * _cached(Sj, "lapth", lambda: laplacian(Sj.th, p))
        th = helmholtz_solve(R, kappa, theta_mean, p)
        cur.th = th

        # ---- step 3: u^(i)
        s1 = np.zeros_like(Xn.u1)
        s2 = np.zeros_like(Xn.u1)
        for j in range(1, i + 1):
            a = A[i - 1, j - 1]
            if a == 0.0:
                continue
            Sj = st[j] if j < i else cur
            if j < i:
                pu1, pu2 = st[j].u1, st[j].u2
            elif p.partner == "lagged":
                pu1, pu2 = st[i - 1].u1, st[i - 1].u2
            elif p.partner == "un":
                pu1, pu2 = Xn.u1, Xn.u2
            else:
                pu1, pu2 = _explicit_partner(st, A_ex, A, i)
            key = ("divBv", j if j < i else -1)
            b1, b2 = _cached(Sj, key, lambda: divB_lf(Sj.v1, Sj.v2, pu1, pu2, p))
            g1, g2 = _cached(Sj, "gradth", lambda: (dx_c(Sj.th, p), dy_c(Sj.th, p)))
            s1 = s1 + a * (b1 + g1)
            s2 = s2 + a * (b2 + g2)
        cur.u1 = Xn.u1 - dt * s1
        cur.u2 = Xn.u2 - dt * s2

        # ---- step 4: q^(i) in closed form
        sD = np.zeros_like(Xn.q)
        sQ = np.zeros_like(Xn.q)
        for j in range(1, i + 1):
            a = A[i - 1, j - 1]
            if a == 0.0:
                continue
            Sj = st[j] if j < i else cur
            sD = sD + a * (0.5 * tau) * _cached(Sj, "divv", lambda: div_c(Sj.v1, Sj.v2, p))
            if j < i:
                sQ = sQ + a * st[j].q
        cur.q = (te2 * Xn.q - dt * (sD + sQ)) / den
        st[i] = cur

    last = st[s]
    out = np.stack([last.u1, last.u2, last.th, last.v1, last.v2, last.q])
    if return_stages:
        stages = {j: np.stack([st[j].u1, st[j].u2, st[j].th, st[j].v1, st[j].v2, st[j].q])
                  for j in range(1, s + 1)}
        return out, stages
    return out


def run(X: np.ndarray, p: Params, nsteps: int) -> np.ndarray:
    for _ in range(nsteps):
        X = step(X, p)
    return X


# ---------------------------------------------------------------------------
# Initial data, outputs and the population view (Sec. 2.1)
# ---------------------------------------------------------------------------

def equilibrium_state(u1, u2, p_in):
    """Moment state from equilibrium: theta = p + |u|^2/2 (Sec. 3.1, proof of
    Theorem 3.4), v = F(u), q = 0 (Sec. 2.1: v1, v2, q relax to F(u), 0)."""
    f1, f2 = F_of_u(u1, u2)
    th = p_in + 0.5 * (u1 * u1 + u2 * u2)
    return np.stack([u1, u2, th, f1, f2, np.zeros_like(u1)])


def outputs(X, eps, rho0=1.0, amp=1.0):
    """Macroscopic outputs: density rho = rho0 (1 + 2 A eps theta) (population
    view, G10), velocity u, pressure p = theta - |u|^2/2."""
    u1, u2, th = X[U1], X[U2], X[TH]
    return rho0 * (1.0 + 2.0 * amp * eps * th), u1, u2, th - 0.5 * (u1 * u1 + u2 * u2)


def d2v6_velocities():
    """c_i = (cos(pi(i-1)/3), sin(pi(i-1)/3)), i = 1..6 (Sec. 2.1)."""
    ang = np.pi * np.arange(6) / 3.0
    return np.stack([np.cos(ang), np.sin(ang)], axis=1)


def moment_basis():
    """Rows phi_m(c_i): 1, c1, c2, c1^2 - 1/2, c1 c2, c1 (c2^2 - 1/4) (Sec. 2.1)."""
    c = d2v6_velocities()
    c1, c2 = c[:, 0], c[:, 1]
    return np.stack([np.ones(6), c1, c2, c1 * c1 - 0.5, c1 * c2, c1 * (c2 * c2 - 0.25)])


def populations_from_moments(X, eps, rho0=1.0, amp=1.0):
    """Deviation populations dF_i = F_i - rho0/6 (shape (6, ny, nx)) of the
    moment state X under G10: the six unscaled f-moments are
    (2 eps theta, u1, u2, -eps v1, eps v2, eps^2 q), f = P^T diag(1/|phi_m|^2) M,
    dF = rho0 * amp * f."""
    P = moment_basis()
    norms = np.sum(P * P, axis=1)
    M = np.stack([2 * eps * X[TH], X[U1], X[U2], -eps * X[V1], eps * X[V2], eps * eps * X[Q]])
    f = np.einsum("mi,m,m...->i...", P, 1.0 / norms, M)
    return rho0 * amp * f


def moments_from_populations(dF, eps, rho0=1.0, amp=1.0):
    """Inverse of populations_from_moments: moment sums of dF/(rho0 amp), then the eps scalings."""
    P = moment_basis()
    f = dF / (rho0 * amp)
    M = np.einsum("mi,i...->m...", P, f)
    return np.stack([M[1], M[2], M[0] / (2 * eps), -M[3] / eps, M[4] / eps, M[5] / (eps * eps)])


def feq_populations(rho, m1, m2):
    """Equilibrium F_i^eq = rho/6 + c_i.m/3 + (2/3)(c_i c_i - I/2):m m (Sec. 2.1)
    for density rho and momentum m = sum c_i F_i."""
    c = d2v6_velocities()
    out = []
    for i in range(6):
        c1, c2 = c[i]
        quad = (c1 * c1 - 0.5) * m1 * m1 + 2 * c1 * c2 * m1 * m2 + (c2 * c2 - 0.5) * m2 * m2
        out.append(rho / 6.0 + (c1 * m1 + c2 * m2) / 3.0 + (2.0 / 3.0) * quad)
    return np.stack(out)
