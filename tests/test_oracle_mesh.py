"""Pins of the oracle's mesh connectivity and particle tracking (sec. 3.5)
against geometry: brute force over all triangles, exact areas, reflections."""
import math

import numpy as np
import pytest

import inputs
import oracle


@pytest.fixture(scope="module")
def small():
    m = inputs.channel_mesh(7, 6, seed=3)
    return m, oracle.Mesh(m)


def test_areas_partition_the_domain(small):
    m, M = small
    assert np.all(M.area > 0)
    assert math.isclose(M.area.sum(), 2 * math.pi * 2.0, rel_tol=1e-13)


def test_neighbour_lists_are_symmetric_and_tagged(small):
    m, M = small
    n_wall = 0
    for e in range(M.n_tri):
        for k in range(3):
            f = M.nbr[e, k]
            if f >= 0:
                assert e in M.nbr[f], (e, f)
                # a periodic crossing is undone by the way back
                kb = list(M.nbr[f]).index(e)
                assert M.shift[e, k] == -M.shift[f, kb]
            else:
                assert f == -1
                n_wall += 1
    nx, ny = m["nx"], m["ny"]
    assert n_wall == 2 * (nx - 1)
    assert np.count_nonzero(M.shift) == 2 * (ny - 1)


def test_subareas_partition_element_area(small):
    m, M = small
    rng = np.random.default_rng(0)
    for e in rng.integers(0, M.n_tri, 50):
        for _ in range(5):
            x, y = rng.uniform(-1, 7), rng.uniform(-1.5, 1.5)
            N = M.subareas(e, x, y)
            assert math.isclose(N.sum(), M.area[e], rel_tol=1e-12, abs_tol=1e-12)
        # the vertices get the unit shape-function values (area coordinates)
        t = M.tri[e]
        for j, node in enumerate(t):
            N = M.subareas(e, *M.xy[node])
            assert abs(N[j] - M.area[e]) < 1e-13 and all(abs(N[i]) < 1e-13 for i in range(3) if i != j)


def _random_interior_point(rng):
    return rng.uniform(0.0, 2 * math.pi), rng.uniform(-0.999, 0.999)


def test_walk_finds_the_brute_force_element(small):
    m, M = small
    rng = np.random.default_rng(1)
    for _ in range(400):
        x, y = _random_interior_point(rng)
        e_true = M.locate_brute(x, y)
        assert e_true >= 0
        # start from a nearby element: the brute-force host of a perturbed point
        x0 = min(max(x + rng.normal(0, 0.3), 1e-9), 2 * math.pi - 1e-9)
        y0 = min(max(y + rng.normal(0, 0.3), -0.999), 0.999)
        e0 = M.locate_brute(x0, y0)
        e, xn, yn, _, _, info = M.track(e0, x, y)
        N = M.subareas(e, xn, yn)
        assert np.all(N >= 0), (x, y, e, N)
        assert (xn, yn) == (x, y)
        if info["min_rel"] > 1e-12:
            assert e == e_true


def test_periodic_seam_round_trip(small):
    m, M = small
    rng = np.random.default_rng(2)
    P = 2 * math.pi
    for _ in range(100):
        y = rng.uniform(-0.99, 0.99)
        d = rng.uniform(1e-6, 0.2)
        e0 = M.locate_brute(P - 1e-3, y)
        e, xn, yn, _, _, info = M.track(e0, P + d, y)  # crosses the right seam
        assert info["crossings_periodic"] == 1
        assert math.isclose(xn, d, rel_tol=0, abs_tol=1e-14)
        assert np.all(M.subareas(e, xn, yn) >= 0)
        e2, x2, y2, _, _, info2 = M.track(e, xn - 2 * d, yn)  # and back again
        assert info2["crossings_periodic"] == 1
        assert math.isclose(x2, P - d, rel_tol=1e-15)
        assert e2 == M.locate_brute(x2, y2) or info2["min_rel"] < 1e-12


def test_wall_reflection_mirrors_position_and_normal_velocity(small):
    m, M = small
    rng = np.random.default_rng(5)
    for _ in range(100):
        x = rng.uniform(0.1, 6.1)
        d = rng.uniform(1e-6, 0.05)
        u, v = rng.normal(), -abs(rng.normal())
        e0 = M.locate_brute(x, -1 + 0.01)
        e, xn, yn, un, vn, info = M.track(e0, x, -1 - d, u, v)
        assert info["reflections"] == 1
        assert math.isclose(yn, -1 + d, rel_tol=0, abs_tol=1e-15)
        assert xn == x and un == u and vn == -v
        assert np.all(M.subareas(e, xn, yn) >= 0)
        # top wall
        e0 = M.locate_brute(x, 1 - 0.01)
        e, xn, yn, un, vn, info = M.track(e0, x, 1 + d, u, -v)
        assert math.isclose(yn, 1 - d, rel_tol=0, abs_tol=1e-15) and vn == v


def test_reflecting_twice_is_the_identity(small):
    m, M = small
    # an inclined wall: reflect a point across the line of an interior edge twice
    e = 10
    t = M.tri[e]
    a, b = M.xy[t[1]], M.xy[t[2]]
    tx, ty = b - a
    ln = math.hypot(tx, ty)
    n = np.array([ty / ln, -tx / ln])
    p = np.array([0.3, 0.1]) + a
    q = p - 2 * np.dot(p - a, n) * n
    r = q - 2 * np.dot(q - a, n) * n
    assert np.allclose(r, p, atol=1e-15)


def test_mesh_rejects_clockwise_triangle():
    m = inputs.channel_mesh(4, 3)
    m = dict(m)
    tri = m["tri"].copy()
    tri[0] = tri[0][::-1]
    m["tri"] = tri
    with pytest.raises(ValueError):
        oracle.Mesh(m)
