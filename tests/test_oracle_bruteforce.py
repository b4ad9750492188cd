"""A second, deliberately naive implementation of one IMEX step on tiny grids,
written as scalar loops over cells and interfaces with explicit modulo
indexing, a dense Gaussian elimination for the Helmholtz equation of
Algorithm 1 (step 2), and every operator re-evaluated where the fully
discrete scheme of Sec. 3.2 uses it.  It shares no code with
``oracle/ap_dvm_oracle.py`` (only the tableau numbers and the inputs), and
the oracle's step must agree with it to round-off."""
import math

import numpy as np
import pytest

from oracle import ap_dvm_oracle as O
from paper_2512_19847_gb300 import workloads as W


class Brute:
    def __init__(self, n, eps, tau, dt, Aex, Aim, scheme, weno_eps=1e-6):
        self.n, self.eps, self.tau, self.dt = n, eps, tau, dt
        self.Aex, self.Aim = [list(r) for r in Aex], [list(r) for r in Aim]
        self.scheme, self.we = scheme, weno_eps
        self.h = 2 * math.pi / n
        self.o4 = scheme != "LF1_C2"

    # --- point access with periodic wrap: f[j][i], i along x
    def at(self, f, i, j):
        n = self.n
        return f[j % n][i % n]

    def d1(self, f, i, j, di, dj):
        a = lambda k: self.at(f, i + k * di, j + k * dj)
        if self.o4:
            return (a(-2) - 8 * a(-1) + 8 * a(1) - a(2)) / (12 * self.h)
        return (a(1) - a(-1)) / (2 * self.h)

    def d2(self, f, i, j, di, dj):
        a = lambda k: self.at(f, i + k * di, j + k * dj)
        if self.o4:
            return (-a(-2) + 16 * a(-1) - 30 * a(0) + 16 * a(1) - a(2)) / (12 * self.h * self.h)
        return (a(-1) - 2 * a(0) + a(1)) / (self.h * self.h)

    def field(self, fn):
        n = self.n
        return [[fn(i, j) for i in range(n)] for j in range(n)]

    # --- WENO / LF numerical flux at the interface between cell (i,j) and its +1 neighbour
    def weno_side(self, v):
        """Reconstruct at the interface from values v[0..] ordered from the
        upwind side towards the interface (v[k] = value k cells upwind-ish)."""
        we = self.we
        if self.scheme == "WENO3_C4":
            fm, f0, fp = v
            cand = [(3 * f0 - fm) / 2, (f0 + fp) / 2]
            beta = [(f0 - fm) ** 2, (fp - f0) ** 2]
            lin = [1 / 3, 2 / 3]
        else:
            f = v
            cand = [(11 * f[2] - 7 * f[1] + 2 * f[0]) / 6, (2 * f[3] + 5 * f[2] - f[1]) / 6,
                    (-f[4] + 5 * f[3] + 2 * f[2]) / 6]
            beta = []
            for k in range(3):
                a, b, c = f[k], f[k + 1], f[k + 2]
                first = [a - 4 * b + 3 * c, a - c, -3 * a + 4 * b - c][k]
                beta.append(13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * first ** 2)
            lin = [0.1, 0.6, 0.3]
        w = [lin[k] / (we + beta[k]) ** 2 for k in range(len(lin))]
        return sum(w[k] * cand[k] for k in range(len(w))) / sum(w)

    def flux(self, g, U, i, j, di, dj):
        A = 1.0
        gv = lambda k: self.at(g, i + k * di, j + k * dj)
        uv = lambda k: self.at(U, i + k * di, j + k * dj)
        if self.scheme == "LF1_C2":
            return 0.5 * (gv(0) + gv(1) - A * (uv(1) - uv(0)))
        plus = lambda k: 0.5 * (gv(k) + A * uv(k))
        minus = lambda k: 0.5 * (gv(k) - A * uv(k))
        r = 1 if self.scheme == "WENO3_C4" else 2
        left = [plus(k) for k in range(-r, r + 1)]
        right = [minus(k) for k in range(r + 1, -r, -1)]
        return self.weno_side(left) + self.weno_side(right)

    def dflux(self, g, U, i, j, di, dj):
        return (self.flux(g, U, i, j, di, dj) - self.flux(g, U, i - di, j - dj, di, dj)) / self.h

    # --- dense Helmholtz: (D_Delta - kappa) theta = R, mean of theta prescribed
    def helmholtz(self, R, kappa, mean_target):
        n = self.n
        N = n * n
        M = [[0.0] * N for _ in range(N)]
        for j in range(n):
            for i in range(n):
                r = j * n + i
                offs = [(-2, 1 / 12), (-1, -16 / 12), (0, 30 / 12), (1, -16 / 12), (2, 1 / 12)] if self.o4 \
                    else [(-1, -1.0), (0, 2.0), (1, -1.0)]
                for k, c in offs:
                    M[r][j * n + (i + k) % n] -= c / (self.h * self.h)
                    M[r][((j + k) % n) * n + i] -= c / (self.h * self.h)
                M[r][r] -= kappa
        mR = sum(R[j][i] for j in range(n) for i in range(n)) / N
        b = [R[j][i] - mR for j in range(n) for i in range(n)]
        # Gaussian elimination with partial pivoting
        for col in range(N):
            piv = max(range(col, N), key=lambda r: abs(M[r][col]))
            M[col], M[piv] = M[piv], M[col]
            b[col], b[piv] = b[piv], b[col]
            for r in range(col + 1, N):
                f = M[r][col] / M[col][col]
                if f != 0.0:
                    for c in range(col, N):
                        M[r][c] -= f * M[col][c]
                    b[r] -= f * b[col]
        x = [0.0] * N
        for r in range(N - 1, -1, -1):
            x[r] = (b[r] - sum(M[r][c] * x[c] for c in range(r + 1, N))) / M[r][r]
        return [[x[j * n + i] + mean_target for i in range(n)] for j in range(n)]

    def step(self, X):
        n, dt, eps, tau = self.n, self.dt, self.eps, self.tau
        u1n, u2n, thn, v1n, v2n, qn = [[list(r) for r in X[m]] for m in range(6)]
        A, Ae = self.Aim, self.Aex
        s = len(A)
        S = {1: dict(u1=u1n, u2=u2n, th=thn, v1=v1n, v2=v2n, q=qn)}
        te2 = tau * eps * eps
        mean_thn = sum(thn[j][i] for j in range(n) for i in range(n)) / (n * n)
        for st in range(2, s + 1):
            a = A[st - 1][st - 1]
            den = te2 + dt * a

            def E(Sj, i, j):
                u1, u2, q, v1, v2 = Sj["u1"], Sj["u2"], Sj["q"], Sj["v1"], Sj["v2"]
                b1 = -self.d1(u1, i, j, 1, 0) + self.d1(u2, i, j, 0, 1)
                b2 = self.d1(u2, i, j, 1, 0) + self.d1(u1, i, j, 0, 1)
                g1 = self.dflux(q, v1, i, j, 1, 0)
                g2 = self.dflux(q, v2, i, j, 0, 1)
                a1, a2 = u1[j][i], u2[j][i]
                return (tau / 4 * b1 + te2 * g1 - 0.5 * (a2 * a2 - a1 * a1), tau / 4 * b2 + te2 * g2 - a1 * a2)

            def v_at(i, j, comp):
                acc = 0.0
                for jj in range(1, st):
                    acc += Ae[st - 1][jj - 1] * E(S[jj], i, j)[comp] + A[st - 1][jj - 1] * S[jj]["v%d" % (comp + 1)][j][i]
                base = (v1n if comp == 0 else v2n)[j][i]
                return (te2 * base - dt * acc) / den

            v1 = self.field(lambda i, j: v_at(i, j, 0))
            v2 = self.field(lambda i, j: v_at(i, j, 1))
            cur = dict(v1=v1, v2=v2)
            kappa = 2 * eps * eps / (dt * dt * a * a)

            def divu(Sj, i, j):
                return self.d1(Sj["u1"], i, j, 1, 0) + self.d1(Sj["u2"], i, j, 0, 1)

            def ddB(Sj, i, j):
                w1, w2 = Sj["v1"], Sj["v2"]
                mixed = (self.d1(self.field(lambda ii, jj: self.d1(w2, ii, jj, 0, 1)), i, j, 1, 0))
                return -self.d2(w1, i, j, 1, 0) + 2 * mixed + self.d2(w1, i, j, 0, 1)

            def lap(f, i, j):
                return self.d2(f, i, j, 1, 0) + self.d2(f, i, j, 0, 1)

            def R_at(i, j):
                r = -kappa * thn[j][i] + divu(S[1], i, j) / (dt * a)
                for jj in range(1, st):
                    r += A[st - 1][jj - 1] * divu(S[jj], i, j) / (dt * a * a)
                    r -= A[st - 1][jj - 1] / a * lap(S[jj]["th"], i, j)       # theta-history term with a minus sign
                for jj in range(1, st + 1):
                    r -= A[st - 1][jj - 1] / a * ddB(S[jj] if jj < st else cur, i, j)
                return r

            R = self.field(R_at)
            th = self.helmholtz(R, kappa, mean_thn)
            cur["th"] = th
            # dissipation partner of D_LF.B(v^(st)) (j = i): explicit-weight predictor
            P1 = self.field(lambda i, j: sum((Ae[st - 1][k - 1] - A[st - 1][k - 1]) * S[k]["u1"][j][i]
                                             for k in range(1, st)) / a)
            P2 = self.field(lambda i, j: sum((Ae[st - 1][k - 1] - A[st - 1][k - 1]) * S[k]["u2"][j][i]
                                             for k in range(1, st)) / a)

            def upd(i, j, comp):
                acc = 0.0
                for jj in range(1, st + 1):
                    c = A[st - 1][jj - 1]
                    if c == 0.0:
                        continue
                    Sj = S[jj] if jj < st else cur
                    p1, p2 = (Sj["u1"], Sj["u2"]) if jj < st else (P1, P2)
                    neg_v1 = [[-x for x in row] for row in Sj["v1"]]
                    if comp == 0:
                        div = self.dflux(neg_v1, p1, i, j, 1, 0) + self.dflux(Sj["v2"], p1, i, j, 0, 1)
                        grad = self.d1(Sj["th"], i, j, 1, 0)
                    else:
                        div = self.dflux(Sj["v2"], p2, i, j, 1, 0) + self.dflux(Sj["v1"], p2, i, j, 0, 1)
                        grad = self.d1(Sj["th"], i, j, 0, 1)
                    acc += c * (div + grad)
                return (u1n if comp == 0 else u2n)[j][i] - dt * acc

            cur["u1"] = self.field(lambda i, j: upd(i, j, 0))
            cur["u2"] = self.field(lambda i, j: upd(i, j, 1))

            def q_at(i, j):
                acc = 0.0
                for jj in range(1, st + 1):
                    c = A[st - 1][jj - 1]
                    Sj = S[jj] if jj < st else cur
                    acc += c * tau / 2 * (self.d1(Sj["v1"], i, j, 1, 0) + self.d1(Sj["v2"], i, j, 0, 1))
                    if jj < st:
                        acc += c * Sj["q"][j][i]
                return (te2 * qn[j][i] - dt * acc) / den

            cur["q"] = self.field(q_at)
            S[st] = cur
        last = S[s]
        return np.array([last[k] for k in ("u1", "u2", "th", "v1", "v2", "q")])


@pytest.mark.parametrize("scheme", ["LF1_C2", "WENO3_C4", "WENO5_C4"])
@pytest.mark.parametrize("tab", ["euler", "gsa2"])
def test_oracle_matches_bruteforce_8x8(scheme, tab):
    n = 8
    A_ex, _, A_im, _ = O.tableau_gsa2() if tab == "gsa2" else O.tableau_euler()
    X = W.random_moment_state(n, n, seed=77, amp=0.5)
    eps, tau, dt = 0.2, 0.3, 0.05
    p = O.Params(n, n, eps, tau, dt, A_ex, A_im, scheme=scheme)
    Y = O.step(X, p)
    Z = Brute(n, eps, tau, dt, A_ex, A_im, scheme).step(X)
    scale = np.max(np.abs(Y), axis=(1, 2))
    err = np.max(np.abs(Y - Z), axis=(1, 2))
    assert np.all(err <= 1e-13 * np.maximum(scale, 1.0)), (err, scale)
