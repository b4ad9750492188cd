"""Convergence orders of the thick double shear layer (Sec. 4.1, Tables 1-2).

The printed error VALUES depend on an unstated time step and norm
normalisation (the t = 0 vorticity discretisation error alone exceeds the
printed N = 33 error), so only the ORDERS are compared: the second-order
GSA scheme with WENO3 must show orders near 2 on the last refinement, as
Table 2 prints (golden file ``tests/golden/paper_tables_1_2.txt``).
Grids are cell-centred powers of two (N = 32, 64, 128 against a 256
reference, resampled spectrally to the coarse cell centres); dt from CFL 0.5.
"""
import math
import os
import warnings

import numpy as np
import pytest

from oracle import ap_dvm_oracle as O
from paper_2512_19847_gb300 import workloads as W

warnings.filterwarnings("ignore", category=RuntimeWarning)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_1_2.txt")


def load_golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t, n, *vals = line.split()
        rows.append((int(t), int(n), [None if v == "-" else float(v) for v in vals]))
    return rows


def vorticity(X, p):
    """Vorticity diagnostic d_x u2 - d_y u1 with the scheme's central difference."""
    return O.dx_c(X[1], p) - O.dy_c(X[0], p)


def resample(f, n):
    """Trigonometric interpolation of a fine cell-centred field to the cell
    centres of an n x n grid (fine size a multiple of n)."""
    nf = f.shape[0]
    r = nf // n
    k = np.fft.fftfreq(nf, d=1.0 / nf)
    ph = np.exp(2j * np.pi * k * (r / 2 - 0.5) / nf)
    g = np.real(np.fft.ifft2(np.fft.fft2(f) * ph[None, :] * ph[:, None]))
    return g[::r, ::r]


def _interval(v_str):
    """Bounds of a printed number given its last printed digit."""
    v = float(v_str)
    mant = v_str.lower().split("e")[0]
    digits = len(mant.split(".")[1]) if "." in mant else 0
    exp = int(v_str.lower().split("e")[1]) if "e" in v_str.lower() else 0
    half = 0.5 * 10.0 ** (exp - digits)
    return v - half, v + half


# Table 2, N = 65, L2: the printed order 1.4447 does not follow from the
# printed errors 0.0039 -> 0.0012 (those give 1.62 .. 1.78); an inconsistency
# of the paper's table, not of the transcription.
KNOWN_INCONSISTENT = {(2, 65, 4)}   # (table, N, column of the L2 error)


def test_golden_file_is_consistent():
    """The printed orders are log2 ratios of the printed errors (Tables 1-2),
    up to the rounding of the printed errors."""
    raw = [l.split() for l in open(GOLDEN) if not l.startswith("#") and l.strip()]
    for t in (1, 2):
        tab = [r for r in raw if int(r[0]) == t]
        for a, b in zip(tab, tab[1:]):
            for k in (2, 4, 6):
                lo_a, hi_a = _interval(a[k])
                lo_b, hi_b = _interval(b[k])
                lo, hi = math.log2(lo_a / hi_b), math.log2(hi_a / lo_b)
                printed = float(b[k + 1])
                ok = lo - 1e-3 <= printed <= hi + 1e-3
                if (t, int(b[1]), k) in KNOWN_INCONSISTENT:
                    assert not ok
                else:
                    assert ok, (t, b[1], k, lo, hi, printed)


@pytest.mark.slow
def test_second_order_tableau_orders_like_table_2():
    A_ex, _, A_im, _ = O.tableau_gsa2()
    sols = {}
    for n in (32, 64, 128, 256):
        u1, u2, pr = W.double_shear_layer(n, inv_rho=15 / math.pi)
        X = O.equilibrium_state(u1, u2, pr)
        dt, ns = W.fixed_time_dt(1.0, W.cfl_dt(u1, u2, 2 * math.pi / n, 0.5))
        p = O.Params(n, n, 1e-6, 0.0, dt, A_ex, A_im, scheme="WENO3_C4")
        sols[n] = (vorticity(O.run(X, p, ns), p), p)
    ref = sols[256][0]
    norms = {}
    for n in (32, 64, 128):
        w, p = sols[n]
        e = w - resample(ref, n)
        h2 = p.dx * p.dy
        norms[n] = (h2 * np.abs(e).sum(), math.sqrt(h2 * (e * e).sum()), np.abs(e).max())
    orders = [math.log2(norms[64][k] / norms[128][k]) for k in range(3)]
    printed = [r for r in load_golden() if r[0] == 2 and r[1] == 257][0][2]
    for k, o in enumerate(orders):
        assert 1.8 < o < printed[2 * k + 1] + 0.6, (orders, printed)
