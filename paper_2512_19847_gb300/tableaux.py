"""IMEX-RK tableaux as (A_ex, A_im) lists: the GSA schemes of Sec. 4.1 (type
CK/ARS: a_11 = 0), a four-stage GSA pair of ARS type, and type-A GSA tableaux
(a_ii != 0 for every i, Sec. 3.1)."""


def euler():
    """First-order GSA Euler IMEX scheme."""
    return [[0.0, 0.0], [1.0, 0.0]], [[0.0, 0.0], [0.0, 1.0]]


def gsa2(c: float = 2.25):
    """Second-order GSA IMEX scheme, gamma = (c - 1/2)/(c - 1)."""
    g = (c - 0.5) / (c - 1.0)
    A_ex = [[0.0, 0.0, 0.0], [c, 0.0, 0.0], [1.0 - 1.0 / (2.0 * c), 1.0 / (2.0 * c), 0.0]]
    A_im = [[0.0, 0.0, 0.0], [0.0, c, 0.0], [0.0, 1.0 - g, g]]
    return A_ex, A_im


def ars4():
    """A four-stage second-order GSA pair of ARS type (a_11 = 0, zero first
    implicit column, a_ii = 1/2 for i >= 2; nodes (0, 1/2, 3/2, 1)).  Not one
    of the paper's pairs: the largest stage count the library takes, with
    every explicit entry and every dissipation-partner weight nonzero."""
    A_ex = [[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.75, 0.75, 0.0, 0.0], [0.5, 0.25, 0.25, 0.0]]
    A_im = [[0.0, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 1.0, 0.5, 0.0], [0.0, 0.75, -0.25, 0.5]]
    return A_ex, A_im


def type_a_euler():
    """First-order type-A GSA pair: the implicit part takes an implicit Euler
    stage from t^n, the explicit part one explicit Euler step from it
    (A_ex = [[0, 0], [1, 0]], A_im = [[1, 0], [0, 1]])."""
    return [[0.0, 0.0], [1.0, 0.0]], [[1.0, 0.0], [0.0, 1.0]]


def type_a3():
    """A three-stage type-A GSA pair (consistent, first order) with every
    implicit diagonal entry and every off-diagonal coupling nonzero."""
    A_ex = [[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.3, 0.7, 0.0]]
    A_im = [[0.4, 0.0, 0.0], [0.1, 0.6, 0.0], [0.2, 0.5, 0.3]]
    return A_ex, A_im
