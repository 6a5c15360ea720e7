"""Pins of the oracle's particle-in-cell statistics (sec. 3.3) and FEM
derivatives (sec. 3.4): library moments, linear-field reproduction,
partition of unity, constant preservation."""
import math

import numpy as np
import pytest

import inputs
import oracle


@pytest.fixture(scope="module")
def chan():
    m = inputs.channel_mesh(9, 7, seed=5)
    return m, oracle.Mesh(m)


def _random_particles(M, n, rng):
    st = {k: rng.normal(size=n) for k in ("u", "v", "w", "om", "ps")}
    st["elem"] = rng.integers(0, M.n_tri, n).astype(np.int32)
    return st


def test_element_moments_equal_library_mean_and_population_covariance(chan):
    m, M = chan
    rng = np.random.default_rng(0)
    st = _random_particles(M, 3000, rng)
    st["u"] = st["u"] + 5.0  # a large mean does not disturb the central moments
    es = oracle.elem_stats(M.n_tri, st)
    for e in range(M.n_tri):
        sel = st["elem"] == e
        n = int(sel.sum())
        assert es[e, 0] == n
        if n == 0:
            assert np.all(es[e] == 0)
            continue
        X = np.stack([st[k][sel] for k in ("u", "v", "w", "om", "ps")])
        assert np.allclose(es[e, 1:6], X.mean(axis=1), rtol=1e-13, atol=1e-14)
        C = np.cov(X[[0, 1, 2]], bias=True) if n > 1 else np.zeros((3, 3))
        got = es[e, 6:12]
        ref = [C[0, 0], C[1, 1], C[2, 2], C[0, 1], C[0, 2], C[1, 2]]
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-13)
        assert math.isclose(es[e, 12], np.var(X[4]), rel_tol=1e-11, abs_tol=1e-13)


def test_single_particle_and_constant_elements_have_zero_moments(chan):
    m, M = chan
    st = {k: np.array([0.3, 2.0, 2.0, 2.0]) for k in ("u", "v", "w", "om", "ps")}
    st["elem"] = np.array([0, 1, 1, 1], dtype=np.int32)
    es = oracle.elem_stats(M.n_tri, st)
    assert np.all(es[0, 6:] == 0) and np.all(es[1, 6:] == 0)
    assert es[1, 0] == 3 and es[1, 1] == 2.0


def test_linear_particle_field_gives_field_at_mean_position(chan):
    """PIC reproduces linear fields: the element mean of f(x) = a + b x + c y
    equals f at the element's mean particle position."""
    m, M = chan
    rng = np.random.default_rng(1)
    st = oracle.init(M, np.full(M.n_tri, 40), seed=3, u_profile="zero", u_sigma=1.0)
    a, b, c = 0.7, -1.3, 2.1
    st["u"] = a + b * st["x"] + c * st["y"]
    es = oracle.elem_stats(M.n_tri, st)
    for e in range(0, M.n_tri, 7):
        sel = st["elem"] == e
        mx, my = st["x"][sel].mean(), st["y"][sel].mean()
        assert math.isclose(es[e, 1], a + b * mx + c * my, rel_tol=1e-12, abs_tol=1e-12)


def test_node_pass_preserves_constants_and_merges_twins(chan):
    m, M = chan
    es = np.zeros((M.n_tri, oracle.NES))
    es[:, 0] = 10
    es[:, 1:] = np.arange(1, 13)
    ns, kept = oracle.node_stats(M, es)
    assert kept == 0
    assert np.all(ns == np.arange(1, 13))
    # a varying field: periodic twins get the same value
    rng = np.random.default_rng(2)
    es[:, 1:] = rng.normal(size=(M.n_tri, 12))
    ns, _ = oracle.node_stats(M, es)
    tw = m["twin"]
    for n in range(M.n_nodes):
        if tw[n] >= 0:
            assert np.array_equal(ns[n], ns[tw[n]])


def test_node_pass_skips_empty_elements_and_keeps_isolated_nodes(chan):
    m, M = chan
    es = np.zeros((M.n_tri, oracle.NES))
    es[:, 0] = 5
    es[:, 1:] = 1.0
    es[3, 0] = 0
    es[3, 1:] = 99.0  # garbage in an empty element is never read
    ns, kept = oracle.node_stats(M, es)
    assert kept == 0 and np.all(ns == 1.0)
    # every element around node n empty -> node keeps the previous value
    n = m["nx"] + 2  # an interior node
    around = [e for e in range(M.n_tri) if n in M.tri[e]]
    es[around, 0] = 0
    prev = np.full((M.n_nodes, oracle.NNS), -7.0)
    ns, kept = oracle.node_stats(M, es, prev)
    assert kept == 1 and np.all(ns[n] == -7.0)


def test_shape_function_derivatives_partition_of_unity(chan):
    m, M = chan
    for e in range(M.n_tri):
        dx, dy = M.shape_derivs(e)
        assert abs(dx.sum()) < 1e-12 and abs(dy.sum()) < 1e-12
        X = M.xy[M.tri[e]]
        # gradient of x is (1, 0), of y is (0, 1)
        assert math.isclose(dx @ X[:, 0], 1.0, rel_tol=1e-12)
        assert abs(dy @ X[:, 0]) < 1e-12
        assert math.isclose(dy @ X[:, 1], 1.0, rel_tol=1e-12)
        assert abs(dx @ X[:, 1]) < 1e-12


def test_derivatives_of_linear_nodal_fields_are_exact():
    """Linear fields: the element gradient is exact, the node average of exact
    gradients is exact, and the second derivatives vanish (sec. 3.4).  On a
    non-periodic mesh so that fields linear in x are admissible."""
    m = inputs.channel_mesh(9, 8, seed=11)
    m = dict(m)
    m["twin"] = np.full(len(m["xy"]), -1, dtype=np.int32)
    m["bnd"] = m["bnd"].copy()
    m["bnd"][m["bnd"][:, 2] == inputs.TAG_PERIODIC, 2] = inputs.TAG_WALL
    M = oracle.Mesh(m)
    x, y = M.xy[:, 0], M.xy[:, 1]
    ns = np.zeros((M.n_nodes, oracle.NNS))
    ns[:, 0] = 1.0 + 2.0 * x - 3.0 * y      # U
    ns[:, 1] = -0.5 * x + 0.25 * y          # V
    ns[:, 2] = 4.0 * y                      # W
    ns[:, 6] = 0.1 + 0.2 * y                # <vv>
    nd = oracle.node_derivs(M, ns)
    assert np.allclose(nd[:, 0:6], [2.0, -3.0, -0.5, 0.25, 0.0, 4.0], atol=1e-11)
    assert np.allclose(nd[:, 6:9], 0.0, atol=1e-9)
    assert np.allclose(nd[:, 9], 0.2, atol=1e-11)


def test_derivatives_on_the_periodic_channel_for_y_fields(chan):
    m, M = chan
    y = M.xy[:, 1]
    ns = np.zeros((M.n_nodes, oracle.NNS))
    ns[:, 0] = 3.0 - 2.0 * y
    nd = oracle.node_derivs(M, ns)
    assert np.allclose(nd[:, 0], 0.0, atol=1e-11)
    assert np.allclose(nd[:, 1], -2.0, atol=1e-11)
