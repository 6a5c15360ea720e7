"""Tolerance helpers for comparing the CUDA library with the oracle.

Floating-point results must satisfy |a - b| <= rtol * max(|b|, s_f), where
s_f is the root-mean-square of that field over the domain (so quantities
that are near zero, such as <uv> or <W>, are compared on their natural
scale).  rtol = 1e-10 for the FP64 path.
"""
import numpy as np

RTOL = 1e-10


def field_close(a, b, rtol=RTOL, axis=0):
    """Per-column check of a against the reference b; returns (ok, worst)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    if a.ndim == 1:
        a = a[:, None]
        b = b[:, None]
    sf = np.sqrt(np.mean(b * b, axis=axis, keepdims=True))
    scale = np.maximum(np.abs(b), sf)
    scale = np.where(scale == 0, 1.0, scale)
    err = np.abs(a - b) / scale
    return bool(np.all(err <= rtol)), float(err.max()) if err.size else 0.0


def assert_field_close(a, b, what, rtol=RTOL):
    ok, worst = field_close(a, b, rtol)
    assert ok, "%s: worst scaled error %.3e > %.1e" % (what, worst, rtol)


def stored_position(x):
    """x rounded to the library's stored position format: 64-bit fixed
    point with 56 fraction bits, rounded to nearest with ties away from
    zero (returned as the FP64 value it reads back as; exact for |x| < 64)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.ldexp(np.abs(x), 56)
    fl = np.floor(s)
    r = np.where(s - fl >= 0.5, fl + 1.0, fl)
    return np.copysign(np.ldexp(r, -56), x)


def stored_df(x):
    """x rounded to the library's stored double-float pair (h = x rounded to
    FP32, l = the remainder rounded to FP32), read back as the FP64 sum."""
    x = np.asarray(x, dtype=np.float64)
    h = x.astype(np.float32).astype(np.float64)
    lo = (x - h).astype(np.float32).astype(np.float64)
    return h + lo
