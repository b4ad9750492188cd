"""IMEX-RK tableaux of Sec. 4.1 as (A_ex, A_im) lists (GSA, type CK/ARS)."""


def euler():
    """First-order GSA Euler IMEX scheme."""
    return [[0.0, 0.0], [1.0, 0.0]], [[0.0, 0.0], [0.0, 1.0]]


def gsa2(c: float = 2.25):
    """Second-order GSA IMEX scheme, gamma = (c - 1/2)/(c - 1)."""
    g = (c - 0.5) / (c - 1.0)
    A_ex = [[0.0, 0.0, 0.0], [c, 0.0, 0.0], [1.0 - 1.0 / (2.0 * c), 1.0 / (2.0 * c), 0.0]]
    A_im = [[0.0, 0.0, 0.0], [0.0, c, 0.0], [0.0, 1.0 - g, g]]
    return A_ex, A_im
