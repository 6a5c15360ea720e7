"""Pins of the oracle's MLP: backpropagation against central finite
differences of the exact FP64 network, GELU against its definition via the
normal CDF (scipy), and BF16 rounding against the format's definition."""
import math

import numpy as np
from scipy import stats

import oracle.mlp as M


def test_bf16_rounding_is_round_to_nearest_even_on_8_bits():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -2.5, 3.0e-39, 65504.0])
    r = M.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # tie -> even
    assert r[2] == 1.0 + 2 ** -6          # tie -> even (up)
    assert r[3] == 1.0 + 2 ** -7          # representable
    assert r[4] == -2.5
    assert abs(r[6] - 65536.0) < 1e-9     # rounds up at 8 significant bits


def test_gelu_is_x_times_normal_cdf():
    z = np.linspace(-6, 6, 101)
    assert np.allclose(M.gelu(z), z * stats.norm.cdf(z), rtol=1e-13, atol=1e-15)
    h = 1e-6
    assert np.allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), atol=1e-8)


def test_backpropagation_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = M.init_params(3)
    for l in range(4):
        P["b%d" % l] = rng.normal(size=P["b%d" % l].shape) * 0.1
    X = rng.normal(size=(7, 11))
    Y = rng.normal(size=(7, 9))
    loss, g = M.loss_and_grads(P, X, Y, rounding=False)
    h = 1e-6
    for name in ("W0", "b0", "W1", "W2", "b2", "W3", "b3"):
        for idx in [tuple(rng.integers(0, s) for s in P[name].shape) for _ in range(6)]:
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][idx] += h
            Pm[name][idx] -= h
            lp = M.loss_and_grads(Pp, X, Y, rounding=False)[0]
            lm = M.loss_and_grads(Pm, X, Y, rounding=False)[0]
            fd = (lp - lm) / (2 * h)
            assert math.isclose(g[name][idx], fd, rel_tol=1e-5, abs_tol=1e-9), (name, idx, g[name][idx], fd)


def test_rounded_network_stays_close_to_the_exact_one():
    rng = np.random.default_rng(1)
    P = M.init_params(4)
    X = rng.normal(size=(32, 11))
    y1 = M.forward(P, X)
    y0 = M.forward(P, X, rounding=False)
    assert np.max(np.abs(y1 - y0)) < 0.05 * np.max(np.abs(y0))
