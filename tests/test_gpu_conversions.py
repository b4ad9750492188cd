"""The integer-pipe FP32 <-> FP64 conversions of the FP32 forms (the moment sums of the
close and the FP64 relaxations use them in place of the conversion instructions) give
the instructions' results bit for bit on every class of value: zeros, normal values,
ties at every rounding position, the subnormal FP32 range, overflow, infinities, NaN."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_19847_gb300 import api  # noqa: E402

pytestmark = pytest.mark.gpu


def _special():
    f32 = np.finfo(np.float32)
    v = [0.0, -0.0, 1.0, -1.0, float(f32.max), -float(f32.max), float(f32.tiny), float(f32.smallest_subnormal),
         np.inf, -np.inf, np.nan, 1e300, -1e300, 5e-324, 1e-310, 2.0 ** -150, 3 * 2.0 ** -151, 2.0 ** -149 * 1.5,
         2.0 ** 128, 2.0 ** 127 * (2 - 2.0 ** -24), 2.0 ** 127 * (2 - 2.0 ** -25), 2.0 ** -126 * (1 - 2.0 ** -24)]
    # ties and near-ties at the 24-bit rounding position, across the exponent range
    for e in range(-155, 130, 3):
        base = 2.0 ** e
        for frac in (1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -52, 1.0 + 2.0 ** -24 - 2.0 ** -52,
                     2.0 - 2.0 ** -24, 2.0 - 2.0 ** -25):
            v += [base * frac, -base * frac]
    return np.array(v, dtype=np.float64)


def test_integer_conversions_match_the_instructions():
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 63, size=200_000, dtype=np.uint64) | (rng.integers(0, 2, 200_000, dtype=np.uint64) << 63)
    rand_all = bits.view(np.float64)                       # every double class, NaN payloads included
    # doubles whose FP32 rounding lands in the normal, subnormal and overflow ranges
    expo = rng.uniform(-160, 130, size=200_000)
    rand_f32 = np.sign(rng.standard_normal(200_000)) * np.exp2(expo) * (1 + rng.random(200_000))
    x = np.concatenate([_special(), rand_all, rand_f32])
    bad_narrow, bad_widen = api.check_conversions(torch.from_numpy(x).cuda())
    assert (bad_narrow, bad_widen) == (0, 0)
