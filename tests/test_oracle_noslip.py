"""The oracle's no-slip wall condition (the section on no-slip wall-boundary
conditions: eqs. fw, exp-wall-condition, frequency-wallstats), pinned by
geometry, limits of the crossing probability and the statistics of the
sampled frequency."""
import numpy as np

import inputs
import oracle


def _mesh(nx=12, ny=9):
    return inputs.channel_mesh(nx, ny, seed=2, wall_tag=inputs.TAG_NOSLIP)


def test_wall_lines_of_the_channel():
    m = _mesh()
    M = oracle.Mesh(m)
    # elements with a node on y = -1 or y = +1 are flagged; the line is that
    # wall with the normal into the fluid
    ys = m["xy"][m["tri"], 1]
    touch_lo = (ys == -1.0).any(axis=1)
    touch_hi = (ys == 1.0).any(axis=1)
    assert np.array_equal(M.noslip_flag.astype(bool), touch_lo | touch_hi)
    for e in np.flatnonzero(touch_lo):
        xa, ya, nx, ny = M.noslip_line[e]
        assert ya == -1.0 and abs(nx) < 1e-15 and ny == 1.0
    for e in np.flatnonzero(touch_hi):
        xa, ya, nx, ny = M.noslip_line[e]
        assert ya == 1.0 and abs(nx) < 1e-15 and ny == -1.0
    # free-slip walls carry no no-slip lines
    M2 = oracle.Mesh(inputs.channel_mesh(12, 9, seed=2))
    assert not M2.noslip_flag.any()


def test_particles_crossing_the_wall_are_reflected_and_stopped():
    # frozen velocity field pushing everything towards y = -1: every particle
    # that ends behind the wall is mirrored into the fluid with U = 0
    m = _mesh()
    M = oracle.Mesh(m)
    counts = np.zeros(M.n_tri, dtype=np.int32)
    counts[M.noslip_flag.astype(bool)] = 20
    st = oracle.init(M, counts, 4, u_profile="zero", u_sigma=0.0)
    st["v"][:] = -5.0
    rows = np.zeros((M.n_tri, 26))
    rows[:, 1] = -5.0           # <V>
    rows[:, 22] = 1.0           # <omega>
    P = oracle.make_params(dt=0.02, nu=1e-12, closure="slm", pressure="none")
    y0 = st["y"].copy()
    wall_w = np.full(M.n_tri, 3.0)
    cnt, status = oracle.step(M, rows, P, 1, 0, st, omega_wall=wall_w)
    behind = y0 - 5.0 * 0.02 < -1.0
    hit = (status & oracle.TRK_NOSLIP) != 0
    near_lo = M.noslip_line[:, 1] == -1.0
    assert behind.any()
    assert np.all(hit[behind])
    assert np.allclose(st["y"][behind], -2.0 - (y0[behind] - 0.1), atol=1e-14)   # mirror of y - 0.1
    assert np.all(st["u"][hit] == 0.0) and np.all(st["v"][hit] == 0.0) and np.all(st["w"][hit] == 0.0)
    assert np.all(st["y"] >= -1.0) and np.all(st["y"] <= 1.0)
    # with nu -> 0 the crossing probability of particles staying in front of the wall vanishes
    stay = ~behind & near_lo[oracle.init(M, counts, 4, u_profile="zero", u_sigma=0.0)["elem"]]
    assert not hit[stay].any()


def test_crossing_probability_of_trajectory_b():
    # particles kept at rest next to the wall (distance d before and after):
    # the wall condition fires with probability exp(-d^2 / (nu dt))
    m = _mesh(40, 6)
    M = oracle.Mesh(m)
    counts = np.zeros(M.n_tri, dtype=np.int32)
    lo = (M.noslip_line[:, 1] == -1.0) & M.noslip_flag.astype(bool)
    counts[lo] = 400
    st = oracle.init(M, counts, 5, u_profile="zero", u_sigma=0.0)
    d = st["y"] + 1.0
    rows = np.zeros((M.n_tri, 26))
    rows[:, 22] = 1.0
    nu, dt = 2e-3, 1e-2
    P = oracle.make_params(dt=dt, nu=nu, closure="slm", pressure="none")
    st["u"][:] = 0.0; st["v"][:] = 0.0; st["w"][:] = 0.0
    cnt, status = oracle.step(M, rows, P, 1, 0, st, omega_wall=np.full(M.n_tri, 2.0))
    hit = (status & oracle.TRK_NOSLIP) != 0
    fw = np.exp(-d * d / (nu * dt))
    # binomial check in bins of the expected probability (5 sigma)
    for lo_p, hi_p in ((0.0, 0.05), (0.05, 0.3), (0.3, 0.7), (0.7, 1.01)):
        sel = (fw >= lo_p) & (fw < hi_p)
        if sel.sum() < 50:
            continue
        expect = fw[sel].sum()
        sigma = np.sqrt((fw[sel] * (1 - fw[sel])).sum()) + 1e-9
        assert abs(hit[sel].sum() - expect) < 5 * sigma + 1


def test_wall_frequency_is_gamma_with_shape_four():
    # many particles forced through the wall: the new omega is Gamma with
    # mean <omega>_w and variance C4 <omega>_w^2 (C4 = 1/4)
    m = _mesh(60, 5)
    M = oracle.Mesh(m)
    counts = np.zeros(M.n_tri, dtype=np.int32)
    counts[M.noslip_flag.astype(bool)] = 200
    st = oracle.init(M, counts, 6, u_profile="zero", u_sigma=0.0)
    st["v"][:] = np.where(st["y"] < 0, -50.0, 50.0)
    rows = np.zeros((M.n_tri, 26))
    rows[:, 22] = 1.0
    P = oracle.make_params(dt=0.1, nu=1e-12, closure="slm", pressure="none")
    w_mean = 2.5
    cnt, status = oracle.step(M, rows, P, 1, 0, st, omega_wall=np.full(M.n_tri, w_mean))
    hit = (status & oracle.TRK_NOSLIP) != 0
    om = st["om"][hit]
    n = len(om)
    assert n > 5000
    assert abs(om.mean() - w_mean) < 5 * w_mean * 0.5 / np.sqrt(n)
    assert abs(om.var() / w_mean ** 2 - 0.25) < 0.05
    assert np.all(om > 0)


def test_wall_frequency_mean_from_the_kinetic_energy_gradient():
    # linear sqrt(2k) = a (y + 1) near the lower wall: <omega>_w = a / C_T;
    # without growth away from the wall the element <omega> is used
    m = _mesh(8, 7)
    M = oracle.Mesh(m)
    a = 3.0
    ns = np.zeros((M.n_nodes, 12))
    y = m["xy"][:, 1]
    sq = a * (y + 1.0)                 # sqrt(2k) = sqrt(uu + vv + ww)
    ns[:, 5] = ns[:, 6] = ns[:, 7] = sq * sq / 3.0
    ns[:, 3] = 7.0                     # <omega>
    w = oracle.noslip_omega(M, ns)
    lo = (M.noslip_line[:, 1] == -1.0) & M.noslip_flag.astype(bool)
    hi = (M.noslip_line[:, 1] == 1.0) & M.noslip_flag.astype(bool)
    assert np.allclose(w[lo], a / 6.0, rtol=1e-12)
    assert np.allclose(w[hi], 7.0)     # sqrt(2k) decreases towards y = +1
    assert np.all(w[~M.noslip_flag.astype(bool)] == 0.0)


def test_relaxation_holds_the_noslip_dirichlet_values():
    # eq. elliptic-relaxation-Lagrangian with no-slip walls: wp_ij = -4.5 eps
    # n_i n_j on the wall nodes for every component; interior values follow
    # the right-hand side when the lengthscale is small
    import oracle.relax as OR
    m = _mesh(10, 8)
    n = len(m["xy"])
    rng = np.random.default_rng(7)
    S = np.zeros((n, 12))
    S[:, 5:8] = rng.uniform(0.5, 1.0, (n, 3))
    S[:, 3] = rng.uniform(1.0, 2.0, n)
    rhs = rng.normal(size=(9, n))
    twin = np.asarray(m["twin"])   # periodic twins are one node: equal statistics
    t = np.flatnonzero(twin >= 0)
    S[t] = S[np.minimum(t, twin[t])]
    rhs[:, t] = rhs[:, np.minimum(t, twin[t])]
    nu = 1e-3
    wp = OR.solve(m, S, rhs, nu)
    _, nrm = OR.wall_normals(m)
    g = OR.noslip_values(S, nu, nrm)
    walls = OR.wall_nodes(m, 5)
    assert len(walls) == 2 * 10
    for ij in range(9):
        assert np.allclose(wp[ij][walls], g[ij][walls], rtol=1e-12, atol=1e-14)
    # wall-normal is +-y: only the (y, y) component is non-zero there
    assert np.allclose(g[4][walls], -4.5 * np.maximum(S[walls, 3] * (0.5 * S[walls, 5:8].sum(1)
                                                                    + nu * 36.0 * S[walls, 3]), 1e-12))
    assert np.allclose(g[0][walls], 0.0) and np.allclose(g[1][walls], 0.0)
