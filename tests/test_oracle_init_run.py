"""Pins of the oracle's particle initialisation (sec. 3.6) and invariants of
a full-method run on the small channel."""
import math

import numpy as np
import pytest
from scipy import stats

import inputs
import oracle


@pytest.fixture(scope="module")
def chan():
    m = inputs.channel_mesh(20, 40, seed=1)
    return m, oracle.Mesh(m)


def test_init_uniform_in_element_and_distributions(chan):
    m, M = chan
    ppe = 50
    counts = np.full(M.n_tri, ppe, dtype=np.int32)
    st = oracle.init(M, counts, seed=1, u_profile="parabola", u_sigma=0.1,
                     elem_psi0=inputs.scalar_slab(m))
    n = M.n_tri * ppe
    assert len(st["x"]) == n
    assert np.array_equal(np.bincount(st["elem"], minlength=M.n_tri), counts)
    # every particle inside the element it was generated in
    for p in range(0, n, 13):
        assert np.all(M.subareas(st["elem"][p], st["x"][p], st["y"][p]) >= 0)
    # uniform in the triangle: the area coordinate N^A / A_e has density 2(1-s)
    sA = np.array([M.subareas(st["elem"][p], st["x"][p], st["y"][p])[0] / M.area[st["elem"][p]]
                   for p in range(0, n, 3)])
    assert stats.kstest(sA, lambda s: 1 - (1 - s) ** 2).pvalue > 1e-4
    # velocity: mean profile 1 - y^2 plus N(0, 0.1^2)
    fu = st["u"] - (1 - st["y"] ** 2)
    for f in (fu, st["v"], st["w"]):
        assert abs(f.mean()) < 5 * 0.1 / math.sqrt(n)
        assert abs(f.std() / 0.1 - 1) < 5 * math.sqrt(0.5 / n)
    # frequency Gamma(k=4, theta=1/4): mean 1, variance 1/4 (sec. 3.6)
    assert abs(st["om"].mean() - 1) < 5 * 0.5 / math.sqrt(n)
    assert abs(st["om"].var() / 0.25 - 1) < 5 * math.sqrt((2 + 6 / 4) / n)
    assert stats.kstest(st["om"], stats.gamma(a=4, scale=0.25).cdf).pvalue > 1e-4
    # scalar slab
    slab = inputs.scalar_slab(m)
    assert np.array_equal(st["ps"], slab[st["elem"]])


def test_full_method_invariants_small_channel(chan):
    """Ten steps of the whole method (GLM with the local wp, channel pressure):
    particle count conserved, every particle inside its host element, omega
    non-negative, IEM keeps psi within [0, 1]."""
    m, M = chan
    counts = np.full(M.n_tri, 20, dtype=np.int32)
    st = oracle.init(M, counts, seed=1, u_profile="parabola", u_sigma=0.1,
                     elem_psi0=inputs.scalar_slab(m))
    P = oracle.make_params(dt=1e-3, nu=1e-3, Pi=2e-3, closure="glm", pressure="channel")
    es, ns, nd, kept = oracle.statistics(M, st)
    n = len(st["x"])
    for s in range(10):
        rows = oracle.elem_coeff(M, ns, nd, P)
        assert np.all(np.isfinite(rows))
        cnt, status = oracle.step(M, rows, P, 1, s, st)
        assert cnt["lost"] == 0
        es, ns, nd, kept = oracle.statistics(M, st, ns)
        assert es[:, 0].sum() == n
    for p in range(0, n, 7):
        assert np.all(M.subareas(st["elem"][p], st["x"][p], st["y"][p]) >= 0)
    assert np.all(st["om"] >= 0)
    assert st["ps"].min() >= 0.0 and st["ps"].max() <= 1.0
    assert np.all((st["y"] >= -1) & (st["y"] <= 1))
    assert np.all((st["x"] >= 0) & (st["x"] <= 2 * math.pi))


def test_threaded_particle_loop_matches_the_serial_one():
    """or_step_threads (the particle loop of loop design (ii) over host
    threads) gives or_step's results bit for bit: every particle reads only
    its own state and its element's coefficients within a step."""
    m = inputs.channel_mesh(20, 40, seed=1)
    M = oracle.Mesh(m)
    counts = np.full(M.n_tri, 12, dtype=np.int32)
    a = oracle.init(M, counts, 1, u_sigma=0.1, elem_psi0=inputs.scalar_slab(m))
    b = {k: v.copy() for k, v in a.items()}
    P = oracle.make_params(dt=1e-3, nu=1e-3, Pi=2e-3, closure="glm")
    es, ns, nd, _ = oracle.statistics(M, a)
    for s in range(4):
        rows = oracle.elem_coeff(M, ns, nd, P)
        ca, sa = oracle.step(M, rows, P, 1, s, a)
        cb, sb, used = oracle.step_threads(M, rows, P, 1, s, b, threads=4)
        assert used >= 1
        assert ca == cb and np.array_equal(sa, sb)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        es, ns, nd, _ = oracle.statistics(M, a, ns)
