"""The test-side emulation of the library's stored state forms (64-bit
fixed-point positions with 56 fraction bits, double-float pairs) against
exact integer arithmetic and the double-float error bound."""
from fractions import Fraction

import numpy as np

from parity_util import stored_df, stored_position


def test_stored_position_is_round_half_away_on_the_2_56_grid():
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(-63, 63, 2000), rng.uniform(-1e-3, 1e-3, 2000),
                         np.ldexp(np.array([1.0, 3.0, -5.0]), -57),  # exact ties
                         np.array([0.0, 1.0, -62.5, 2.0 ** -56, -(2.0 ** -60)])])
    got = stored_position(xs)
    for x, g in zip(xs, got):
        q = Fraction(float(x)) * 2 ** 56
        n = int(abs(q) + Fraction(1, 2)) * (1 if q >= 0 else -1)  # ties away from zero
        assert Fraction(float(g)) == Fraction(n, 2 ** 56), x


def test_stored_df_keeps_48_bits():
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.normal(size=5000), rng.normal(size=1000) * 1e-20, rng.normal(size=1000) * 1e20])
    got = stored_df(xs)
    assert np.all(np.abs(got - xs) <= np.abs(xs) * 2.0 ** -48)
    # FP32 numbers and sums of two FP32 numbers a few binades apart are exact
    f = rng.normal(size=1000).astype(np.float32).astype(np.float64)
    assert np.array_equal(stored_df(f), f)
    assert np.array_equal(stored_df(1.0 + 2.0 ** -30), 1.0 + 2.0 ** -30)
