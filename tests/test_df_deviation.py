"""The statistics kernel forms each deviation x - k of two stored
double-floats with Fast2Sum as the final renormalization instead of
TwoSum.  The two agree bit for bit whenever the stored pairs are
normalized (|l| <= ulp(h) / 2), which is what the stored forms keep.  This
checks that claim in FP32 arithmetic emulated with numpy, on random pairs
and on the adversarial ones: equal or adjacent high parts, high parts on
both sides of a power of two, zeros, opposite signs and tiny values."""
import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = (a + b).astype(f32)
    bb = (s - a).astype(f32)
    e = ((a - (s - bb).astype(f32)).astype(f32) + (b - bb).astype(f32)).astype(f32)
    return s, e


def fast_two_sum(a, b):
    s = (a + b).astype(f32)
    return s, (b - (s - a).astype(f32)).astype(f32)


def normalized(h, rng):
    """A low part |l| <= ulp(h) / 2 for each high part (ties included)."""
    ulp = np.spacing(np.abs(h)).astype(f32)
    frac = rng.uniform(-0.5, 0.5, size=h.shape).astype(f32)
    frac[rng.random(h.shape) < 0.05] = f32(0.5)
    frac[rng.random(h.shape) < 0.05] = f32(-0.5)
    frac[rng.random(h.shape) < 0.05] = f32(0.0)
    return (frac * ulp).astype(f32)


def deviation_pairs(xh, xl, kh, kl):
    s, e = two_sum(xh, (-kh).astype(f32))
    t = (xl + (e + (-kl).astype(f32)).astype(f32)).astype(f32)
    return two_sum(s, t), fast_two_sum(s, t)


def check(xh, kh, rng):
    xh, kh = xh.astype(f32), kh.astype(f32)
    xl, kl = normalized(xh, rng), normalized(kh, rng)
    (a_h, a_l), (b_h, b_l) = deviation_pairs(xh, xl, kh, kl)
    assert np.array_equal(a_h.view(np.uint32), b_h.view(np.uint32))
    assert np.array_equal(a_l.view(np.uint32), b_l.view(np.uint32))


def test_fast_renormalization_equals_two_sum_on_normalized_pairs():
    rng = np.random.default_rng(7)
    n = 400_000
    # random values over many binades, both signs
    check(rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 3, n),
          rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 3, n), rng)
    # close values (the deviations of one element's particles)
    k = rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 1, n)
    check(k * (1 + rng.standard_normal(n) * 1e-3), k, rng)
    # equal and adjacent high parts
    k = (rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 1, n)).astype(f32)
    check(k, k, rng)
    check(np.nextafter(k, np.inf, dtype=f32), k, rng)
    check(np.nextafter(k, -np.inf, dtype=f32), k, rng)
    # on both sides of a power of two
    p = (2.0 ** rng.integers(-20, 6, n)).astype(f32) * np.where(rng.random(n) < 0.5, 1, -1).astype(f32)
    check(p, np.nextafter(p, np.zeros_like(p), dtype=f32), rng)
    check(np.nextafter(p, np.zeros_like(p), dtype=f32), p, rng)
    # zeros, opposite signs, tiny values
    z = np.zeros(n, dtype=f32)
    check(z, rng.standard_normal(n), rng)
    check(rng.standard_normal(n), z, rng)
    check(rng.standard_normal(n), -rng.standard_normal(n), rng)
    check(rng.standard_normal(n) * 1e-30, rng.standard_normal(n) * 1e-30, rng)


def test_the_check_sees_unnormalized_pairs():
    """A control: with low parts far beyond half an ulp (not a stored form),
    the sum of the high part and the low part is no longer exact and the
    two renormalizations part, so the comparison above can fail."""
    rng = np.random.default_rng(11)
    n = 100_000
    k = (rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 1, n)).astype(f32)
    xh = np.nextafter(k, np.inf, dtype=f32)
    xl = (rng.uniform(-1, 1, n) * np.spacing(np.abs(xh)) * 2.0 ** 30).astype(f32)
    kl = np.zeros(n, dtype=f32)
    (a_h, a_l), (b_h, b_l) = deviation_pairs(xh, xl, k, kl)
    assert (a_l.view(np.uint32) != b_l.view(np.uint32)).any()
