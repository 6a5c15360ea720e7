"""The complex-geometry workload against the oracle: a small obstacle mesh
(concave corners, walls, periodic inflow/outflow with re-injection, a point
source, the source-dependent micromixing time), particles per element
proportional to the area.  FP64 states within 1e-10 of the oracle after 30
steps; the FP32-state form stays inside the domain and keeps its invariants."""
import numpy as np
import pytest

import inputs
import oracle
from parity_util import assert_field_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402
from paper_1006_0720_gb300 import capi  # noqa: E402

KEYS = ("x", "y", "u", "v", "w", "om", "ps")


def _setup(cfg, precision):
    m = inputs.obstacle_mesh(h_min=cfg["h_min"], ratio=cfg["ratio"], growth=cfg["growth"])
    counts = inputs.counts_by_area(m, cfg["mean_ppe"])
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, cfg["seed"], count=counts, u_profile=cfg["u_profile"], u_sigma=cfg["u_sigma"],
                      precision=precision)
    p = pg.model_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure=cfg["closure"], tm_mode=cfg["tm_mode"],
                        src_x=cfg["src"][0], src_y=cfg["src"][1], src_r=cfg["src"][2])
    return m, counts, gm, gp, p


def test_obstacles_fp64_parity_30_steps():
    cfg = inputs.OBSTACLES["obstacles_small_mean20"]
    m, counts, gm, gp, p = _setup(cfg, capi.PDF_FP64)
    M = oracle.Mesh(m)
    nbr, shift = gm.connectivity()
    assert np.array_equal(nbr, M.nbr) and np.array_equal(shift, M.shift)
    ost = oracle.init(M, counts, cfg["seed"], u_profile=cfg["u_profile"], u_sigma=cfg["u_sigma"])
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=cfg["closure"], tm_mode="source",
                            pressure="channel", src=cfg["src"])
    pg.pdf_estimate_stats(gp, gm)
    es, ns, nd, _ = oracle.statistics(M, ost)
    rows = pg.pdf_elem_coeff(gp, gm, p).cpu().numpy()
    assert_field_close(rows, oracle.elem_coeff(M, ns, nd, po), "obstacle coefficient rows")
    flagged_total = 0
    reinjected = 0
    for s in range(cfg["steps"]):
        rows = oracle.elem_coeff(M, ns, nd, po)
        cnt, status = oracle.step(M, rows, po, cfg["seed"], s, ost)
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        assert info["lost"] == 0 and cnt["lost"] == 0
        assert info["reflections"] == cnt["reflections"] and info["fallbacks"] == cnt["fallbacks"]
        reinjected += int(np.sum(status & oracle.TRK_REINJECT != 0))
        es, ns, nd, _ = oracle.statistics(M, ost, ns)
        pg.pdf_estimate_stats(gp, gm)
        st = {k: v.cpu().numpy() for k, v in gp.get_state().items()}
        flagged = (status & oracle.TRK_NEAR_FACE) != 0
        same = st["elem"] == ost["elem"]
        assert np.all(same | flagged)
        flagged_total += int(np.sum(~same))
        for k in KEYS:
            assert_field_close(st[k][same], ost[k][same], "step %d %s" % (s, k))
    assert reinjected > 0
    assert np.abs(ost["u"]).max() < 20 and np.abs(ost["v"]).max() < 20  # the run stays bounded
    src = cfg["src"]
    inside = (ost["x"] - src[0]) ** 2 + (ost["y"] - src[1]) ** 2 <= src[2] ** 2
    assert inside.any() and np.all(st["ps"][inside] == 1.0)


def test_obstacles_fp32_state_invariants():
    cfg = dict(inputs.OBSTACLES["obstacles_small_mean20"])
    m, counts, gm, gp, p = _setup(cfg, capi.PDF_FP32_STATE)
    pg.pdf_estimate_stats(gp, gm)
    n = int(counts.sum())
    for s in range(60):
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        assert info["lost"] == 0
        pg.pdf_estimate_stats(gp, gm)
    es = torch.empty((gm.n_tri, 13), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, es)
    assert int(es[:, 0].sum().item()) == n
    st = {k: v.cpu().numpy() for k, v in gp.get_state().items()}
    M = oracle.Mesh(m)
    for i in range(0, n, 97):
        assert np.all(M.subareas(st["elem"][i], st["x"][i], st["y"][i]) >= -1e-12 * M.area[st["elem"][i]])
    assert st["ps"].min() >= 0.0 and st["ps"].max() <= 1.0
    assert np.all(st["om"] >= 0) and st["om"].max() < 100
    assert np.abs(st["u"]).max() < 20 and np.abs(st["v"]).max() < 20


@pytest.mark.parametrize("multigrid", [True, False])
def test_obstacles_relaxation_solve_matches_the_oracle(multigrid):
    """The elliptic-relaxation solve on the obstacle mesh (walls in several
    orientations, concave corners, graded elements, inflow/outflow twins):
    the converged solution of both preconditioners agrees with the oracle's
    sparse direct solve of the GPU's own statistics."""
    import oracle.relax as OR
    cfg = inputs.OBSTACLES["obstacles_small_mean20"]
    m, counts, gm, gp, p = _setup(cfg, capi.PDF_FP64)
    pg.pdf_estimate_stats(gp, gm)
    for s in range(3):
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    ns = torch.empty((gm.n_nodes, capi.PDF_NNS), dtype=torch.float64, device="cuda")
    nd = torch.empty((gm.n_nodes, capi.PDF_NND), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, node_stats=ns, node_derivs=nd)
    S, Dv = ns.cpu().numpy(), nd.cpu().numpy()
    wp = torch.zeros((9, gm.n_nodes), dtype=torch.float64, device="cuda")
    pg.pdf_relax_set_solver(gp, multigrid)
    iters, res = pg.pdf_relax_solve_particles(gp, gm, p, wp, rtol=1e-13, max_it=6000)
    assert max(res) <= 1e-13
    rhs = np.stack([oracle.relax_rhs(S[n], Dv[n]) for n in range(gm.n_nodes)], axis=1)
    ref = OR.solve(m, S, rhs, p.nu)
    assert_field_close(wp.cpu().numpy().T, ref.T, "obstacle relaxation solution", rtol=1e-9)
    if multigrid:
        assert max(iters) < 200, iters
