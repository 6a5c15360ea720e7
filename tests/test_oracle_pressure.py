"""Pins of the oracle's mean-pressure projection (sec. 3.2, eqs. pressure-
projection-smooth and velocity-correction; eq. wall-pressure-condition)
against closed forms: exact gradients of linear fields, the stiffness
matrix's null space and energy, the channel's cross-stream balance, the
stabilisation term, the weak divergence-free property of the corrected
field, and the wall load of linear fields."""
import numpy as np

import inputs
import oracle
import oracle.pressure as OP


def _mesh(nx=12, ny=10, wall_tag=None):
    return inputs.channel_mesh(nx, ny, seed=3, wall_tag=wall_tag)


def _rep_mask(m):
    rep = OP._rep(m)
    return rep == np.arange(len(rep))


def test_shape_gradients_are_exact_for_linear_fields():
    m = _mesh()
    x, y = m["xy"][:, 0], m["xy"][:, 1]
    A, g = OP.shape_gradients(m)
    assert np.all(A > 0)
    assert np.isclose(A.sum(), 2.0 * np.pi * 2.0)
    np.testing.assert_allclose(g.sum(axis=2), 0.0, atol=1e-12)
    gx = OP.element_gradient(m, 3.0 * x - 2.0 * y + 1.0)
    np.testing.assert_allclose(gx, np.tile([3.0, -2.0], (len(A), 1)), atol=1e-12)


def test_stiffness_null_space_and_energy():
    m = _mesh()
    K = OP.stiffness(m)
    mask = _rep_mask(m)
    y = m["xy"][:, 1]
    ones = mask.astype(float)
    np.testing.assert_allclose(K @ ones, 0.0, atol=1e-12)
    # int |grad y|^2 = area of the channel; y is a single-valued field on the
    # periodic mesh (twins share y)
    yr = np.where(mask, y, 0.0)
    assert np.isclose(yr @ (K @ yr), 2.0 * np.pi * 2.0)
    # y is discretely harmonic away from the walls
    interior = mask & (np.abs(np.abs(y) - 1.0) > 1e-12)
    np.testing.assert_allclose((K @ yr)[interior], 0.0, atol=1e-12)


def test_divergence_load_integrates_the_divergence():
    m = _mesh()
    x, y = m["xy"][:, 0], m["xy"][:, 1]
    ns = np.zeros((len(x), oracle.NNS))
    ns[:, 0] = 0.5 * x          # div = 0.5 + 2 = 2.5
    ns[:, 1] = 2.0 * y
    d = OP.divergence_load(m, ns)
    assert np.isclose(d.sum(), 2.5 * 2.0 * np.pi * 2.0)
    assert np.all(d[~_rep_mask(m)] == 0.0)


def test_wall_edges_point_out_of_the_channel():
    m = _mesh()
    E = OP.wall_edges(m)
    assert len(E) == 2 * 11
    for a, b, e, nx, ny, L in E:
        y = m["xy"][a, 1]
        assert np.isclose(nx, 0.0, atol=1e-12) and np.isclose(ny, np.sign(y))


def test_nodal_gradient_of_linear_fields():
    m = _mesh()
    x, y = m["xy"][:, 0], m["xy"][:, 1]
    np.testing.assert_allclose(OP.nodal_gradient(m, 0.7 * y), np.tile([0.0, 0.7], (len(y), 1)), atol=1e-12)
    np.testing.assert_allclose(OP.nodal_gradient(m, -1.3 * x), np.tile([-1.3, 0.0], (len(y), 1)), atol=1e-12)


def test_wall_load_of_linear_statistics():
    """h of eq. wall-pressure-condition on the channel's walls (outward
    normals -y at y = -1 and +y at y = 1) for each term alone: the load on
    a wall sums to h times its length 2 pi."""
    m = _mesh()
    x, y = m["xy"][:, 0], m["xy"][:, 1]
    n = len(x)
    bottom = np.isclose(y, -1.0) & _rep_mask(m)
    top = np.isclose(y, 1.0) & _rep_mask(m)
    L = 2.0 * np.pi
    nu = 0.01

    def load(ns, nd, slm=False):
        G = OP.wall_load(m, ns, nd, nu, slm)
        return G[bottom].sum(), G[top].sum()

    ns, nd = np.zeros((n, 12)), np.zeros((n, 10))
    ns[:, 6] = 0.4 * y                              # d<vv>/dy = 0.4
    gb, gt = load(ns, nd)
    assert np.isclose(gb, 0.4 * L) and np.isclose(gt, -0.4 * L)
    ns, nd = np.zeros((n, 12)), np.zeros((n, 10))
    ns[:, 8] = 0.3 * x                              # d<uv>/dx = 0.3
    gb, gt = load(ns, nd)
    assert np.isclose(gb, 0.3 * L) and np.isclose(gt, -0.3 * L)
    ns, nd = np.zeros((n, 12)), np.zeros((n, 10))
    nd[:, 7] = 5.0                                  # lap <V> = 5
    gb, gt = load(ns, nd)
    assert np.isclose(gb, -nu * 5.0 * L) and np.isclose(gt, nu * 5.0 * L)
    ns, nd = np.zeros((n, 12)), np.zeros((n, 10))
    ns[:, 0] = 1.5                                  # <U> = 1.5, <V> = 0.2 x
    ns[:, 1] = 0.2 * x
    gb, gt = load(ns, nd, slm=True)                 # advection: <U> d<V>/dx = 0.3
    assert np.isclose(gb, 0.3 * L) and np.isclose(gt, -0.3 * L)
    gb, gt = load(ns, nd, slm=False)
    assert gb == 0.0 and gt == 0.0


def test_projection_recovers_the_channel_cross_stream_balance():
    """With <vv> = c y and nothing else, the wall condition alone drives the
    projection: the solution is the linear dP = -c (y - mean), i.e. the
    channel's d<P>/dy = -d<v^2>/dy (eq. cross-stream-mean-momentum-
    channel), and every particle's V grows by dt c."""
    m = _mesh(wall_tag=inputs.TAG_NOSLIP)
    M = oracle.Mesh(m)
    n_tri = len(m["tri"])
    st = oracle.init(M, np.full(n_tri, 3, dtype=np.int32), 5, u_sigma=0.1)
    y = m["xy"][:, 1]
    n = len(y)
    c, dt = 0.25, 1e-3
    ns, nd = np.zeros((n, 12)), np.zeros((n, 10))
    ns[:, 6] = c * y
    v0 = st["v"].copy()
    u0 = st["u"].copy()
    dP, pres, G, gradP = OP.project(m, ns, nd, st, np.zeros(n), np.zeros(n), 0.01, dt, Cp=1e-3)
    mask = _rep_mask(m)
    ref = -c * (y - y[mask].mean())
    np.testing.assert_allclose(dP, ref, atol=1e-10)
    np.testing.assert_allclose(pres, ref, atol=1e-10)
    np.testing.assert_allclose(gradP, np.tile([0.0, -c], (n, 1)), atol=1e-9)
    np.testing.assert_allclose(st["v"] - v0, dt * c, atol=1e-12)
    np.testing.assert_allclose(st["u"], u0, atol=1e-12)
    # at the next projection with the same statistics nothing changes: the
    # field already satisfies the wall condition it was made with
    dP2, pres2, _, _ = OP.project(m, ns, nd, st, pres, G, 0.01, dt, Cp=0.0)
    np.testing.assert_allclose(dP2, 0.0, atol=1e-10)


def test_stabilisation_term_in_closed_form():
    """Divergence-free <U*>, no wall data: K dP = -C_p K P^n / dt, so dP =
    -(C_p / dt) (P^n - mean) (eq. pressure-projection-smooth)."""
    m = _mesh()
    n = len(m["xy"])
    rep = OP._rep(m)
    rng = np.random.default_rng(4)
    P = rng.standard_normal(n)[rep]
    ns, nd = np.zeros((n, 12)), np.zeros((n, 10))
    ns[:, 0] = 0.8                        # uniform flow along the channel
    Cp, dt = 1e-3, 2e-3
    dP, _ = OP.solve_increment(m, ns, nd, P, np.zeros(n), 0.01, dt, Cp)
    mask = rep == np.arange(n)
    np.testing.assert_allclose(dP, -(Cp / dt) * (P - P[mask].mean()), atol=1e-10)
    assert abs(dP[mask].mean()) < 1e-14


def test_corrected_field_is_weakly_divergence_free():
    """C_p = 0, no wall data, <U*> tangential at the walls: the corrected
    element velocities W = <U*> - dt grad dP satisfy int grad N_a . W = 0
    for every unknown a (the discrete form of eq. divergence)."""
    m = _mesh()
    x, y = m["xy"][:, 0], m["xy"][:, 1]
    n = len(x)
    rep = OP._rep(m)
    rng = np.random.default_rng(6)
    U = rng.standard_normal(n)[rep]
    V = (rng.standard_normal(n) * (1.0 - y * y))[rep]   # 0 on both walls
    ns, nd = np.zeros((n, 12)), np.zeros((n, 10))
    ns[:, 0], ns[:, 1] = U, V
    dt = 1e-2
    dP, _ = OP.solve_increment(m, ns, nd, np.zeros(n), np.zeros(n), 0.01, dt, 0.0)
    A, g = OP.shape_gradients(m)
    tri = m["tri"]
    ge = OP.element_gradient(m, dP)
    W = np.stack([U[tri].mean(axis=1), V[tri].mean(axis=1)], axis=1) - dt * ge
    r = np.zeros(n)
    for a in range(3):
        np.add.at(r, rep[tri[:, a]], A * (g[:, 0, a] * W[:, 0] + g[:, 1, a] * W[:, 1]))
    before = np.zeros(n)
    W0 = np.stack([U[tri].mean(axis=1), V[tri].mean(axis=1)], axis=1)
    for a in range(3):
        np.add.at(before, rep[tri[:, a]], A * (g[:, 0, a] * W0[:, 0] + g[:, 1, a] * W0[:, 1]))
    assert np.abs(before).max() > 0.1
    np.testing.assert_allclose(r, 0.0, atol=1e-10)


def test_projection_drift_in_the_coefficients():
    """make_params(pressure="projection"): the drift sees Pi - d<P'>/dx and
    -d<P'>/dy (eq. velocity-prediction), SLM and GLM alike."""
    S = np.zeros(12)
    S[3] = 1.0
    S[5:8] = 0.1
    Dv = np.zeros(10)
    Dv[9] = 7.0
    for closure in ("slm", "glm"):
        pj = oracle.make_params(dt=1e-3, nu=0.0, Pi=2.0, closure=closure, pressure="projection")
        c = oracle.node_coeff(S, Dv, None, pj, grad_p=np.array([0.5, -0.25]))
        assert np.isclose(c[9], 1.5) and np.isclose(c[10], 0.25)
        c0 = oracle.node_coeff(S, Dv, None, pj)
        assert np.isclose(c0[9], 2.0) and c0[10] == 0.0


def _coupled_run(Cp, steps=25):
    """Steps of the small channel with the projection after every step
    (eqs. velocity-prediction, pressure-projection-smooth, velocity-
    correction), all in the oracle."""
    m = inputs.channel_mesh(14, 24, seed=1)
    M = oracle.Mesh(m)
    n_tri, n = len(m["tri"]), len(m["xy"])
    st = oracle.init(M, np.full(n_tri, 30, dtype=np.int32), 1, u_sigma=0.1)
    dt, nu = 1e-3, 1e-3
    po = oracle.make_params(dt=dt, nu=nu, Pi=2 * nu, closure="glm", pressure="projection")
    _, ns, nd, _ = oracle.statistics(M, st)
    pres, G, gradP = np.zeros(n), np.zeros(n), np.zeros((n, 2))
    v0 = st["v"].std()
    dPs = []
    for s in range(steps):
        oracle.step(M, oracle.elem_coeff(M, ns, nd, po, grad_p=gradP), po, 1, s, st)
        _, ns, nd, _ = oracle.statistics(M, st, ns)
        dP, pres, G, gradP = OP.project(m, ns, nd, st, pres, G, nu, dt, Cp, False)
        _, ns, nd, _ = oracle.statistics(M, st, ns)
        dPs.append(np.abs(dP).max())
    return np.array(dPs), st["v"].std() / v0


def test_coupled_projection_stability_depends_on_cp_over_dt():
    """The reading of C_p as a time: with C_p = dt / 2 the coupled scheme
    stays bounded (the increments shrink, the cross-stream fluctuations keep
    their size), with C_p = dt the discrete pressure mode grows each step."""
    d, vr = _coupled_run(5e-4)
    assert d[-5:].max() < d[0] and 0.9 < vr < 1.05
    d, vr = _coupled_run(1e-3)
    assert d[-1] > 100 * d[0]


def test_inflow_outflow_condition_gives_the_imposed_drop():
    """The street canyon's inflow/outflow condition on a straight channel
    with constant <vv> = c and no flow: <P> = Pi L_x - c at the inflow, -c
    at the outflow, linear in between (the walls carry no load), so the
    drift's pressure gradient is exactly the imposed -Pi.  From <P'> = 0
    with C_p = 0 the increment is that linear field; from any <P'>^n with
    C_p = dt the stabilisation term replaces the interior by the harmonic
    extension of the boundary values, the same linear field; the next
    projection with the same statistics leaves it as it is."""
    m = inputs.channel_mesh(12, 10, seed=3, inout=True)
    x = m["xy"][:, 0]
    n = len(x)
    Pi, c, Lx, dt = 0.7, 0.05, 2.0 * np.pi, 1e-3
    ns, nd = np.zeros((n, 12)), np.zeros((n, 10))
    ns[:, 6] = c
    target = Pi * (Lx - x) - c
    dP, G = OP.solve_increment(m, ns, nd, np.zeros(n), np.zeros(n), 0.01, dt, 0.0, inout=True, Pi=Pi)
    np.testing.assert_allclose(dP, target, atol=1e-9)
    np.testing.assert_allclose(OP.nodal_gradient(m, dP), np.tile([-Pi, 0.0], (n, 1)), atol=1e-9)
    pres0 = np.random.default_rng(2).standard_normal(n)[OP._rep(m, inout=True)]
    dP, G = OP.solve_increment(m, ns, nd, pres0, np.zeros(n), 0.01, dt, dt, inout=True, Pi=Pi)
    P1 = pres0 + dP
    np.testing.assert_allclose(P1, target, atol=1e-9)
    dP2, _ = OP.solve_increment(m, ns, nd, P1, G, 0.01, dt, dt, inout=True, Pi=Pi)
    np.testing.assert_allclose(dP2, 0.0, atol=1e-9)
    io = OP.inout_nodes(m)
    assert (io == 1).sum() == 10 and (io == 2).sum() == 10
    # the drift sees the whole gradient of the field in this mode
    pj = oracle.make_params(dt=1e-3, nu=0.0, Pi=Pi, closure="slm", pressure="projection_inout")
    S = np.zeros(12)
    S[3] = 1.0
    S[5:8] = 0.1
    cf = oracle.node_coeff(S, np.zeros(10), None, pj, grad_p=np.array([-Pi, 0.0]))
    assert np.isclose(cf[9], Pi) and cf[10] == 0.0


def _obstacles():
    cfg = inputs.OBSTACLES["obstacles_small_mean20"]
    return inputs.obstacle_mesh(h_min=cfg["h_min"], ratio=cfg["ratio"], growth=cfg["growth"])


def test_obstacle_mesh_stiffness_null_space_and_energy():
    """Graded elements and concave corners: K annihilates the constants and
    the energy of y is the fluid area (the domain minus the obstacles)."""
    m = _obstacles()
    K = OP.stiffness(m)
    mask = _rep_mask(m)
    A, _ = OP.shape_gradients(m)
    assert np.all(A > 0)
    np.testing.assert_allclose(K @ mask.astype(float), 0.0, atol=1e-10)
    yr = np.where(mask, m["xy"][:, 1], 0.0)
    assert np.isclose(yr @ (K @ yr), A.sum(), rtol=1e-12)


def test_obstacle_mesh_divergence_load_integrates_the_divergence():
    m = _obstacles()
    x, y = m["xy"][:, 0], m["xy"][:, 1]
    rep = OP._rep(m)
    ns = np.zeros((len(x), oracle.NNS))
    ns[:, 0] = 0.0           # <U> = 0 keeps the field single-valued on the twins
    ns[:, 1] = -0.75 * y     # div = -0.75
    A, _ = OP.shape_gradients(m)
    d = OP.divergence_load(m, ns)
    assert np.isclose(d.sum(), -0.75 * A.sum(), rtol=1e-12)
    assert np.all(d[rep != np.arange(len(rep))] == 0.0)


def test_obstacle_mesh_wall_normals_close_the_boundary():
    """Divergence theorem: the outward normals times the lengths of all
    boundary edges sum to zero; the inflow and outflow edges are straight
    and of equal total length, so the wall edges alone sum to zero."""
    m = _obstacles()
    E = OP.wall_edges(m)
    assert len(E) > 50
    s = np.zeros(2)
    for a, b, e, nx, ny, L in E:
        assert np.isclose(nx * nx + ny * ny, 1.0)
        s += L * np.array([nx, ny])
    np.testing.assert_allclose(s, 0.0, atol=1e-10)
