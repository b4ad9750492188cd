"""Host-side post-processing of the Sec. 4 experiments (no GPU): the trigonometric
interpolation that compares the convergence grids of Tables 1-2 with their
non-nested 513 x 513 reference reproduces band-limited fields exactly."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2512_19847_gb300.experiments import interpolate_periodic  # noqa: E402


@pytest.mark.parametrize("n", [33, 65, 129, 257])
def test_interpolation_is_exact_on_resolved_modes(n):
    m = 513
    x = (np.arange(m) + 0.5) * 2 * math.pi / m
    xc = (np.arange(n) + 0.5) * 2 * math.pi / n

    def field(xx):
        return (np.sin(3 * xx)[None, :] * np.cos(5 * xx)[:, None] + 0.3 * np.cos(11 * xx)[:, None]
                - 0.2 * np.sin(7 * xx)[None, :])

    assert np.max(np.abs(interpolate_periodic(field(x), n) - field(xc))) < 1e-12


def test_interpolation_keeps_the_mean_and_orientation():
    m, n = 513, 65
    x = (np.arange(m) + 0.5) * 2 * math.pi / m
    f = 2.5 + np.cos(2 * x)[:, None] * np.ones((1, m))       # varies along y (axis 0) only
    g = interpolate_periodic(f, n)
    xc = (np.arange(n) + 0.5) * 2 * math.pi / n
    assert np.max(np.abs(g - (2.5 + np.cos(2 * xc)[:, None]))) < 1e-12


def test_node_sampled_grids_are_nested():
    """Reading G14 of the Tables 1-2 grids: with nodes=True the double shear layer is sampled
    at (i dx, j dy), so every point of an N - 1 = 2^k cell grid is a point of the finer ones
    (injection compares the same physical points)."""
    from paper_2512_19847_gb300 import workloads as W
    coarse = W.double_shear_layer(32, inv_rho=15 / math.pi, nodes=True)
    fine = W.double_shear_layer(512, inv_rho=15 / math.pi, nodes=True)
    for c, f in zip(coarse, fine):
        assert np.array_equal(c, f[::16, ::16])
    centred = W.double_shear_layer(32, inv_rho=15 / math.pi)
    assert not np.array_equal(centred[1], coarse[1])
