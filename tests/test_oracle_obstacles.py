"""Pins of the complex-geometry parts: the obstacle mesh, the neighbour walk
around its concave corners (fall-back of sec. 3.5) against brute force, the
periodic inflow/outflow pair with scalar re-injection, the concentrated
source, and the source-dependent micromixing time scale
(eq. micromixing-timescale-canyon) in its two limits."""
import math

import numpy as np
import pytest

import inputs.obstacles as IO
import oracle


@pytest.fixture(scope="module")
def small():
    m = IO.obstacle_mesh(h_min=0.05, ratio=6.0, growth=1.3)
    return m, oracle.Mesh(m)


def _inside_obstacle(m, x, y):
    return any(o[0] < x < o[1] and y < o[2] for o in m["obstacles"])


def test_mesh_covers_the_fluid_domain(small):
    m, M = small
    obst = sum((o[1] - o[0]) * o[2] for o in m["obstacles"])
    assert np.all(M.area > 0)
    assert math.isclose(M.area.sum(), m["Lx"] * m["Ly"] - obst, rel_tol=1e-12)
    assert np.sum(M.shift != 0) == 2 * np.sum(m["bnd"][:, 2] == IO.TAG_OUTFLOW)


def test_walk_around_concave_corners_matches_brute_force(small):
    m, M = small
    rng = np.random.default_rng(0)
    checked = 0
    for (x0, x1, h) in m["obstacles"]:
        for cx, cy in ((x0, h), (x1, h)):  # the obstacle's top corners (re-entrant for the fluid)
            for _ in range(60):
                # start just beside the obstacle, end just above it: the
                # straight path may cut the corner
                xs, ys = cx + (-0.03 if cx == x0 else 0.03), cy - rng.uniform(0.01, 0.2)
                xe, ye = cx + rng.uniform(-0.1, 0.1) * (1 if cx == x0 else -1), cy + rng.uniform(0.005, 0.1)
                if _inside_obstacle(m, xs, ys) or _inside_obstacle(m, xe, ye):
                    continue
                e0 = M.locate_brute(xs, ys)
                e, xn, yn, _, _, info = M.track(e0, xe, ye)
                assert not (info["status"] & oracle.TRK_LOST)
                assert np.all(M.subareas(e, xn, yn) >= 0)
                if info["reflections"] == 0:
                    assert (xn, yn) == (xe, ye)
                    assert e == M.locate_brute(xe, ye) or info["min_rel"] < 1e-12
                checked += 1
    assert checked > 100


def test_outflow_reinjects_at_the_inflow(small):
    m, M = small
    rng = np.random.default_rng(1)
    Lx = m["Lx"]
    for _ in range(50):
        y = rng.uniform(0.1, 4.9)
        e0 = M.locate_brute(Lx - 1e-3, y)
        e, xn, yn, _, _, info = M.track(e0, Lx + 0.01, y)
        assert info["status"] & oracle.TRK_REINJECT
        assert math.isclose(xn, 0.01, abs_tol=1e-14)
        assert np.all(M.subareas(e, xn, yn) >= 0)
        # and back through the inflow: periodic, no re-injection
        e2, x2, y2, _, _, info2 = M.track(e, -0.01, yn)
        assert not (info2["status"] & oracle.TRK_REINJECT)
        assert math.isclose(x2, Lx - 0.01, rel_tol=1e-15)


def test_source_sets_the_scalar_and_reinjection_clears_it(small):
    m, M = small
    counts = IO.counts_by_area(m, mean=20)
    st = oracle.init(M, counts, 3, u_profile="uniform", u_sigma=0.1)
    st["ps"][:] = 0.5
    src = (2.0, 0.5, 0.05)
    P = oracle.make_params(dt=1e-2, nu=1e-3, Pi=2e-3, closure="slm", pressure="channel", tm_mode="source", src=src)
    es, ns, nd, _ = oracle.statistics(M, st)
    # push particles through the outflow: a strong uniform drift
    rows = oracle.elem_coeff(M, ns, nd, P)
    rows[:, 9] += 50.0  # a_x dt = 0.5 per step
    for s in range(3):
        before = st["x"].copy()
        cnt, status = oracle.step(M, rows, P, 1, s, st)
        d2 = (st["x"] - src[0]) ** 2 + (st["y"] - src[1]) ** 2
        assert np.all(st["ps"][d2 <= src[2] ** 2] == 1.0)
        re = (status & oracle.TRK_REINJECT) != 0
        assert re.any()
        assert np.all(st["ps"][re & (d2 > src[2] ** 2)] == 0.0)
        assert np.all(st["x"][re] < before[re])


def test_source_mixing_time_limits():
    """Far from the source t_m is the turbulence time max(k/eps, C_T sqrt(nu/eps));
    at the source it is min(C_s (r0^2/eps)^(1/3), that)."""
    S = np.zeros(oracle.NNS)
    S[0] = 1.0
    S[3] = 2.0
    S[5:8] = 0.02
    D = np.zeros(oracle.NND)
    nu, r0 = 1e-3, 0.05
    P = oracle.make_params(dt=1e-3, nu=nu, closure="glm", tm_mode="source", src=(2.0, 0.5, r0))
    k = 0.03
    eps = 2.0 * (k + nu * 36.0 * 2.0)
    tturb = max(k / eps, 6.0 * math.sqrt(nu / eps))
    far = oracle.node_coeff(S, D, None, P, xy=(19.0, 4.0))[25]
    assert math.isclose(far, 1.0 / tturb, rel_tol=1e-14)
    at = oracle.node_coeff(S, D, None, P, xy=(2.0, 0.5))[25]
    assert math.isclose(at, 1.0 / min(0.02 * (r0 * r0 / eps) ** (1 / 3), tturb), rel_tol=1e-14)
    # the same as the plain turbulence form when tm_mode is turb
    Pt = oracle.make_params(dt=1e-3, nu=nu, closure="glm", tm_mode="turb")
    assert oracle.node_coeff(S, D, None, Pt, xy=(2.0, 0.5))[25] == far
