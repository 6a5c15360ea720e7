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
