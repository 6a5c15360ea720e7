"""Pins of the oracle's elliptic-relaxation solve (Eq. elliptic-relaxation-
Lagrangian, P1 finite elements, sec. 3.2) against manufactured solutions of
the differential equation itself: with uniform statistics L is constant, and

    wp(y) = cos(pi (y + 1))   (zero normal derivative at the walls)
    wp(y) = sin(pi (y + 1))   (zero at the walls)

solve wp - L^2 wp'' = (1 + pi^2 L^2) wp.  The discrete solutions must
converge to them at second order; constants are reproduced exactly."""
import math

import numpy as np

import inputs
import oracle
import oracle.relax as R


def _uniform_stats(n, k=0.015, om=1.0):
    S = np.zeros((n, oracle.NNS))
    S[:, 3] = om
    S[:, 5:8] = 2.0 * k / 3.0
    return S


def _errors(nx, ny, nu=1e-3):
    m = inputs.channel_mesh(nx, ny, jitter=0.2, seed=2)
    n = len(m["xy"])
    S = _uniform_stats(n)
    y = m["xy"][:, 1]
    L2 = R.lengthscale2(S, nu, np.ones(n))[0]
    rhs = np.zeros((9, n))
    c = np.cos(math.pi * (y + 1))
    s = np.sin(math.pi * (y + 1))
    fac = 1.0 + math.pi ** 2 * L2
    rhs[0] = fac * c   # wp_11: diagonal, natural condition; C_xi = 1 + 1.3 n_x^2 = 1
    rhs[1] = fac * s   # wp_12: off-diagonal, zero at the walls
    wp = R.solve(m, S, rhs, nu)
    return np.max(np.abs(wp[0] - c)), np.max(np.abs(wp[1] - s)), L2


def test_manufactured_solutions_converge_at_second_order():
    """Meshes refined in both directions (about square cells): halving the
    spacing divides the maximum error by about 4."""
    e1 = _errors(51, 17)
    e2 = _errors(101, 33)
    e3 = _errors(201, 65)
    assert e1[2] > 1e-3  # the elliptic term matters at this L
    for k in (0, 1):
        r1, r2 = e1[k] / e2[k], e2[k] / e3[k]
        assert e3[k] < 1.5e-3
        assert r1 > 2.5 and r2 > 3.0, (k, e1[k], e2[k], e3[k])


def test_constant_right_hand_side_gives_the_constant():
    m = inputs.channel_mesh(10, 9, seed=3)
    n = len(m["xy"])
    S = _uniform_stats(n, k=0.02, om=1.3)
    rhs = np.zeros((9, n))
    rhs[0] = rhs[4] = rhs[8] = -0.7
    wp = R.solve(m, S, rhs, 1e-3)
    for ij in (0, 4, 8):
        assert np.allclose(wp[ij], -0.7, rtol=1e-11)
    assert np.allclose(wp[[1, 2, 3, 5, 6, 7]], 0.0, atol=1e-14)


def test_wall_normals_of_the_channel():
    m = inputs.channel_mesh(10, 9, seed=3)
    d, nrm = R.wall_normals(m)
    y = m["xy"][:, 1]
    assert np.allclose(d, 1.0 - np.abs(y), atol=1e-12)
    assert np.all(nrm[y < -1e-9, 1] == -1.0) and np.all(nrm[y > 1e-9, 1] == 1.0)
    assert np.all(nrm[:, 0] == 0.0)


def test_anisotropic_lengthscale_for_the_wall_normal_component():
    """Eq. Cxi: C_xi = 2.3 for wp_22 in the channel (normal (0, -1)), 1.0 for
    the others; Eq. L: L = C_L max(C_xi k^1.5 / eps, C_eta (nu^3/eps)^0.25)."""
    S = _uniform_stats(1, k=0.3, om=2.0)
    nu = 1e-4
    k, om = 0.3, 2.0
    eps = om * (k + nu * 36.0 * om)
    for cxi in (1.0, 2.3):
        L = 0.134 * max(cxi * k ** 1.5 / eps, 72.0 * (nu ** 3 / eps) ** 0.25)
        assert math.isclose(R.lengthscale2(S, nu, np.array([cxi]))[0], L * L, rel_tol=1e-14)


def _obstacles():
    cfg = inputs.OBSTACLES["obstacles_small_mean20"]
    return inputs.obstacle_mesh(h_min=cfg["h_min"], ratio=cfg["ratio"], growth=cfg["growth"])


def test_constant_right_hand_side_on_the_obstacle_mesh():
    """Graded elements, walls in both orientations and concave corners: with
    spatially varying statistics (so L^2 and C_xi vary) a constant right-hand
    side of a diagonal component is still reproduced (the stiffness matrix
    annihilates constants and the walls are natural boundaries for it), and
    the off-diagonal components with zero right-hand side stay zero."""
    m = _obstacles()
    n = len(m["xy"])
    rng = np.random.default_rng(7)
    S = _uniform_stats(n)
    S[:, 3] = rng.uniform(0.5, 2.0, n)
    S[:, 5:8] *= rng.uniform(0.5, 2.0, (n, 3))
    rhs = np.zeros((9, n))
    rhs[0], rhs[4], rhs[8] = 0.3, -1.1, 2.5
    wp = R.solve(m, S, rhs, 1e-3)
    for ij, c in ((0, 0.3), (4, -1.1), (8, 2.5)):
        assert np.allclose(wp[ij], c, rtol=1e-10), ij
    assert np.allclose(wp[[1, 2, 3, 5, 6, 7]], 0.0, atol=1e-14)


def test_wall_normals_of_the_obstacle_mesh():
    """Every node's nearest-wall normal is a unit vector; on a wall node it
    points out of the domain (away from the elements at that node) and the
    distance is 0."""
    m = _obstacles()
    d, nrm = R.wall_normals(m)
    assert np.allclose(np.hypot(nrm[:, 0], nrm[:, 1]), 1.0, atol=1e-12)
    assert np.all(d >= 0.0)
    xy, tri = m["xy"], m["tri"]
    walls = R.wall_nodes(m, 1)
    assert len(walls) > 0
    assert np.allclose(d[walls], 0.0, atol=1e-12)
    cent = xy[tri].mean(axis=1)
    for a in walls[:: max(1, len(walls) // 200)]:
        around = np.nonzero((tri == a).any(axis=1))[0]
        inward = cent[around].mean(axis=0) - xy[a]
        assert inward @ nrm[a] < 0.0, a
