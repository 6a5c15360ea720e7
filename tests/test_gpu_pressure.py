"""The stabilised mean-pressure projection (sec. 3.2: eqs. pressure-
projection-smooth and velocity-correction, with the wall condition of eq.
wall-pressure-condition) on the GPU against the oracle, each side on its own
from the same seeded state: the pressure field, the corrected particle
velocities, a second projection that carries the stored wall load, the
statistics estimated after it, and a step whose drift sees the projected
pressure gradient (eq. velocity-prediction)."""
import numpy as np
import pytest

import inputs
import oracle
import oracle.pressure as OP
from parity_util import assert_field_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402
from paper_1006_0720_gb300 import capi  # noqa: E402

KEYS = ("x", "y", "u", "v", "w", "om", "ps")


def _host(st):
    return {k: v.cpu().numpy() for k, v in st.items()}


def _setup(closure, wall_tag, seed=11, ppe=30, precision=capi.PDF_FP64):
    m = inputs.channel_mesh(16, 24, seed=2, wall_tag=wall_tag)
    n_tri = len(m["tri"])
    counts = np.full(n_tri, ppe, dtype=np.int32)
    psi = inputs.scalar_slab(m)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, seed, count=counts, u_sigma=0.3, elem_psi0=psi, precision=precision)
    M = oracle.Mesh(m)
    ost = oracle.init(M, counts, seed, u_sigma=0.3, elem_psi0=psi)
    p = pg.model_params(closure=closure, dt=2e-3, nu=5e-3, pressure="projection")
    return m, gm, gp, M, ost, p


@pytest.mark.parametrize("closure,wall_tag,persistent", [("slm", inputs.TAG_NOSLIP, True), ("glm", None, True),
                                                          ("slm", inputs.TAG_NOSLIP, False)])
def test_projection_matches_the_oracle(closure, wall_tag, persistent):
    m, gm, gp, M, ost, p = _setup(closure, wall_tag)
    pg.pdf_pressure_set_solver(gp, persistent)
    slm = closure == "slm"
    Cp = 1e-3
    n = gm.n_nodes
    pg.pdf_estimate_stats(gp, gm)
    _, ns, nd, _ = oracle.statistics(M, ost)
    pres, G = np.zeros(n), np.zeros(n)
    for k in range(2):
        it, res = pg.pdf_pressure_project(gp, gm, p, Cp=Cp, rtol=1e-13, max_it=20000)
        assert 0 < it < 20000 and res <= 1e-13
        dP, pres, G, gradP = OP.project(m, ns, nd, ost, pres, G, p.nu, p.dt, Cp, slm)
        got = pg.pdf_pressure_field(gp, gm).cpu().numpy()
        assert np.abs(dP).max() > 1e-3
        assert_field_close(got, pres, "projected pressure %d" % k, rtol=1e-9)
        st = _host(gp.get_state())
        assert np.array_equal(st["elem"], ost["elem"])
        for key in ("u", "v"):
            assert_field_close(st[key], ost[key], "corrected %s %d" % (key, k), rtol=1e-10)
        # the statistics the library carried through the correction (seen
        # through the coefficient rows, without estimating them again)
        es, ns, nd, _ = oracle.statistics(M, ost, ns)
        po_k = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=closure, pressure="projection")
        assert_field_close(pg.pdf_elem_coeff(gp, gm, p).cpu().numpy(),
                           oracle.elem_coeff(M, ns, nd, po_k, grad_p=gradP),
                           "rows after projection %d" % k, rtol=1e-9)
    # a step whose drift sees Pi - grad <P'>
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=closure, pressure="projection")
    rows = oracle.elem_coeff(M, ns, nd, po, grad_p=gradP)
    kw = {"omega_wall": oracle.noslip_omega(M, ns)} if wall_tag is not None else {}
    cnt, status = oracle.step(M, rows, po, 11, 0, ost, **kw)
    info = pg.pdf_step(gp, gm, p, step=0, info=True)
    assert info["lost"] == 0 and cnt["lost"] == 0
    st = _host(gp.get_state())
    flagged = (status & oracle.TRK_NEAR_FACE) != 0
    same = st["elem"] == ost["elem"]
    assert (same | flagged).all()
    for key in KEYS:
        assert_field_close(st[key][same], ost[key][same], "projection step %s" % key)


def test_pressure_field_set_and_get():
    """A field set through pdf_pressure_field reaches the drift: with the
    SLM closure the coefficient rows hold Pi - d<P'>/dx and -d<P'>/dy
    exactly (eq. velocity-prediction), here 0.5 y gives -0.5."""
    m, gm, gp, M, ost, p = _setup("slm", None)
    y = m["xy"][:, 1]
    f = torch.tensor(0.5 * y, dtype=torch.float64, device="cuda")
    back = pg.pdf_pressure_field(gp, gm, set=f).cpu().numpy()
    assert np.array_equal(back, 0.5 * y)
    ce = torch.empty((gm.n_tri, capi.PDF_NCOEF), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm)
    pg.pdf_elem_coeff(gp, gm, p, rows=ce)
    c = ce.cpu().numpy()
    np.testing.assert_allclose(c[:, 9], p.Pi, atol=1e-12)
    np.testing.assert_allclose(c[:, 10], -0.5, atol=1e-12)


def test_projection_fp32_state():
    m, gm, gp, M, ost, p = _setup("slm", inputs.TAG_NOSLIP, precision=capi.PDF_FP32_STATE)
    n = gm.n_nodes
    pg.pdf_estimate_stats(gp, gm)
    _, ns, nd, _ = oracle.statistics(M, ost)
    it, res = pg.pdf_pressure_project(gp, gm, p, Cp=1e-3, rtol=1e-12, max_it=20000)
    dP, pres, G, gradP = OP.project(m, ns, nd, ost, np.zeros(n), np.zeros(n), p.nu, p.dt, 1e-3, True)
    got = pg.pdf_pressure_field(gp, gm).cpu().numpy()
    # the FP32 state rounds the velocities the statistics come from
    assert_field_close(got, pres, "projected pressure (FP32 state)", rtol=1e-4)
    st = _host(gp.get_state())
    for key in ("u", "v"):
        assert_field_close(st[key], ost[key], "corrected %s (FP32 state)" % key, rtol=1e-5)


def test_both_solvers_give_the_same_iterates():
    """The persistent cooperative iteration and the separate kernels make the
    same iterates up to the order of the reductions: the same iteration
    count within one, the same pressure to the solve's tolerance."""
    out = []
    for persistent in (True, False):
        m, gm, gp, M, ost, p = _setup("slm", inputs.TAG_NOSLIP)
        pg.pdf_pressure_set_solver(gp, persistent)
        pg.pdf_estimate_stats(gp, gm)
        it, res = pg.pdf_pressure_project(gp, gm, p, Cp=1e-3, rtol=1e-10, max_it=500)
        out.append((it, pg.pdf_pressure_field(gp, gm).cpu().numpy()))
    assert abs(out[0][0] - out[1][0]) <= 1
    assert_field_close(out[0][1], out[1][1], "persistent vs separate kernels", rtol=1e-9)


def test_multigrid_keeps_the_iterations_few():
    """The multigrid-preconditioned iteration converges in tens of
    iterations on a 20 000-node channel (the Jacobi preconditioner needs
    about a thousand there) and reaches the same answer as the oracle's
    direct solve."""
    m = inputs.channel_mesh(100, 200, seed=2, wall_tag=inputs.TAG_NOSLIP)
    n_tri = len(m["tri"])
    counts = np.full(n_tri, 4, dtype=np.int32)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 3, count=counts, u_sigma=0.3)
    M = oracle.Mesh(m)
    ost = oracle.init(M, counts, 3, u_sigma=0.3)
    p = pg.model_params(closure="slm", dt=2e-3, nu=5e-3, pressure="projection")
    pg.pdf_estimate_stats(gp, gm)
    _, ns, nd, _ = oracle.statistics(M, ost)
    it, res = pg.pdf_pressure_project(gp, gm, p, Cp=1e-3, rtol=1e-10, max_it=400)
    assert it <= 80 and res <= 1e-10
    n = gm.n_nodes
    _, pres, _, _ = OP.project(m, ns, nd, ost, np.zeros(n), np.zeros(n), p.nu, p.dt, 1e-3, True)
    assert_field_close(pg.pdf_pressure_field(gp, gm).cpu().numpy(), pres, "pressure on 20k nodes", rtol=1e-7)


def test_not_converged_is_reported():
    m, gm, gp, M, ost, p = _setup("glm", None)
    pg.pdf_estimate_stats(gp, gm)
    with pytest.raises(capi.PdfError) as err:
        pg.pdf_pressure_project(gp, gm, p, Cp=1e-3, rtol=1e-14, max_it=2)
    assert err.value.status == capi.PDF_ENOTCONV


def test_projection_on_the_obstacle_mesh():
    """Graded mesh with three obstacles (wall edges on every obstacle side,
    inflow/outflow twins one unknown): the projection and the next step with
    its pressure gradient match the oracle."""
    cfg = inputs.OBSTACLES["obstacles_small_mean20"]
    m = inputs.obstacle_mesh(h_min=cfg["h_min"], ratio=cfg["ratio"], growth=cfg["growth"])
    counts = inputs.counts_by_area(m, cfg["mean_ppe"])
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, cfg["seed"], count=counts, u_profile=cfg["u_profile"], u_sigma=cfg["u_sigma"])
    M = oracle.Mesh(m)
    ost = oracle.init(M, counts, cfg["seed"], u_profile=cfg["u_profile"], u_sigma=cfg["u_sigma"])
    p = pg.model_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure=cfg["closure"], tm_mode=cfg["tm_mode"],
                        src_x=cfg["src"][0], src_y=cfg["src"][1], src_r=cfg["src"][2], pressure="projection")
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=cfg["closure"], tm_mode="source",
                            pressure="projection", src=cfg["src"])
    n = gm.n_nodes
    pg.pdf_estimate_stats(gp, gm)
    _, ns, nd, _ = oracle.statistics(M, ost)
    it, res = pg.pdf_pressure_project(gp, gm, p, Cp=1e-3, rtol=1e-13, max_it=5000)
    assert res <= 1e-13
    dP, pres, G, gradP = OP.project(m, ns, nd, ost, np.zeros(n), np.zeros(n), p.nu, p.dt, 1e-3,
                                    cfg["closure"] == "slm")
    assert np.abs(G).max() > 0
    assert_field_close(pg.pdf_pressure_field(gp, gm).cpu().numpy(), pres, "obstacle pressure", rtol=1e-9)
    st = _host(gp.get_state())
    for key in ("u", "v"):
        assert_field_close(st[key], ost[key], "obstacle corrected %s" % key, rtol=1e-10)
    _, ns, nd, _ = oracle.statistics(M, ost, ns)
    rows = oracle.elem_coeff(M, ns, nd, po, grad_p=gradP)
    assert_field_close(pg.pdf_elem_coeff(gp, gm, p).cpu().numpy(), rows, "obstacle rows with grad <P'>", rtol=1e-9)
    cnt, status = oracle.step(M, rows, po, cfg["seed"], 0, ost)
    pg.pdf_step(gp, gm, p, step=0)
    st = _host(gp.get_state())
    same = st["elem"] == ost["elem"]
    assert np.all(same | ((status & oracle.TRK_NEAR_FACE) != 0))
    for key in KEYS:
        assert_field_close(st[key][same], ost[key][same], "obstacle projection step %s" % key)


@pytest.mark.parametrize("where,persistent", [("channel", True), ("obstacles", True), ("channel", False)])
def test_inflow_outflow_projection_matches_the_oracle(where, persistent):
    """PDF_PRESSURE_PROJECTION_INOUT (the street canyon's inflow/outflow
    condition): two projections and a step, GPU and oracle each from the
    same seeded state."""
    if where == "channel":
        m = inputs.channel_mesh(16, 24, seed=2, inout=True, wall_tag=inputs.TAG_NOSLIP)
        counts = np.full(len(m["tri"]), 30, dtype=np.int32)
        closure, seed, prof, sig = "slm", 5, "parabola", 0.3
        extra = {}
    else:
        cfg = inputs.OBSTACLES["obstacles_small_mean20"]
        m = inputs.obstacle_mesh(h_min=cfg["h_min"], ratio=cfg["ratio"], growth=cfg["growth"])
        counts = inputs.counts_by_area(m, cfg["mean_ppe"])
        closure, seed, prof, sig = cfg["closure"], cfg["seed"], cfg["u_profile"], cfg["u_sigma"]
        extra = dict(tm_mode=cfg["tm_mode"], src_x=cfg["src"][0], src_y=cfg["src"][1], src_r=cfg["src"][2])
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, seed, count=counts, u_profile=prof, u_sigma=sig)
    pg.pdf_pressure_set_solver(gp, persistent)
    M = oracle.Mesh(m)
    ost = oracle.init(M, counts, seed, u_profile=prof, u_sigma=sig)
    p = pg.model_params(dt=2e-3, nu=5e-3, Pi=0.5, closure=closure, pressure="projection_inout", **extra)
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=closure, pressure="projection_inout",
                            tm_mode="source" if extra else "turb",
                            src=(p.src_x, p.src_y, p.src_r))
    n = gm.n_nodes
    Cp = 0.5 * p.dt
    pg.pdf_estimate_stats(gp, gm)
    _, ns, nd, _ = oracle.statistics(M, ost)
    pres, G = np.zeros(n), np.zeros(n)
    for k in range(2):
        it, res = pg.pdf_pressure_project(gp, gm, p, Cp=Cp, rtol=1e-13, max_it=5000)
        assert res <= 1e-13
        dP, pres, G, gradP = OP.project(m, ns, nd, ost, pres, G, p.nu, p.dt, Cp, closure == "slm", inout=True,
                                        Pi=p.Pi)
        assert_field_close(pg.pdf_pressure_field(gp, gm).cpu().numpy(), pres, "in/out pressure %d" % k, rtol=1e-9)
        st = _host(gp.get_state())
        for key in ("u", "v"):
            assert_field_close(st[key], ost[key], "in/out corrected %s %d" % (key, k), rtol=1e-10)
        _, ns, nd, _ = oracle.statistics(M, ost, ns)
    io = OP.inout_nodes(m)
    assert np.all(pres[io == 1] > pres[io == 2].mean())   # the imposed drop
    rows = oracle.elem_coeff(M, ns, nd, po, grad_p=gradP)
    assert_field_close(pg.pdf_elem_coeff(gp, gm, p).cpu().numpy(), rows, "in/out rows", rtol=1e-9)
    kw = {"omega_wall": oracle.noslip_omega(M, ns)} if where == "channel" else {}
    cnt, status = oracle.step(M, rows, po, seed, 0, ost, **kw)
    pg.pdf_step(gp, gm, p, step=0)
    st = _host(gp.get_state())
    same = st["elem"] == ost["elem"]
    assert np.all(same | ((status & oracle.TRK_NEAR_FACE) != 0))
    for key in KEYS:
        assert_field_close(st[key][same], ost[key][same], "in/out step %s" % key)
