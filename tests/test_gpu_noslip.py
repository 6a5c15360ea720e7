"""No-slip walls (the section on no-slip wall-boundary conditions) on the
GPU against the oracle, each side on its own from the same seeded state:
the wall lines, free-running steps of a channel with no-slip walls (wall
reflections, U = 0, the Gamma wall frequency and the crossing probability
of trajectory (b) all exercised), and the FP32-state form's invariants."""
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


def _host(st):
    return {k: v.cpu().numpy() for k, v in st.items()}


def _channel():
    return inputs.channel_mesh(20, 40, seed=1, wall_tag=inputs.TAG_NOSLIP)


def test_noslip_connectivity():
    m = _channel()
    nbr, shift = pg.Mesh(m).connectivity()
    M = oracle.Mesh(m)
    assert np.array_equal(nbr, M.nbr) and (nbr == -5).sum() == 2 * 19


@pytest.mark.parametrize("arith", ["fx", "fp64"])
def test_noslip_channel_steps_match_the_oracle(arith):
    m = _channel()
    n_tri = 2 * 19 * 39
    counts = np.full(n_tri, 40, dtype=np.int32)
    psi = inputs.scalar_slab(m)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 7, count=counts, u_sigma=0.2, elem_psi0=psi)
    M = oracle.Mesh(m)
    ost = oracle.init(M, counts, 7, u_sigma=0.2, elem_psi0=psi)
    # nu and dt such that the crossing probability of trajectory (b) is
    # well inside (0, 1) for the particles of the wall elements
    p = pg.model_params(closure="slm", dt=2e-3, nu=5e-3, arith=arith)
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure="slm", pressure="channel")
    pg.pdf_estimate_stats(gp, gm)
    es, ns, nd, _ = oracle.statistics(M, ost)
    flagged = np.zeros(len(ost["x"]), dtype=bool)
    events = 0
    for s in range(12):
        rows = oracle.elem_coeff(M, ns, nd, po)
        cnt, status = oracle.step(M, rows, po, 7, s, ost, omega_wall=oracle.noslip_omega(M, ns))
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        assert info["lost"] == 0 and cnt["lost"] == 0
        assert info["reflections"] == cnt["reflections"]
        events += int(((status & oracle.TRK_NOSLIP) != 0).sum())
        flagged |= (status & oracle.TRK_NEAR_FACE) != 0
        es, ns, nd, _ = oracle.statistics(M, ost, ns)
        pg.pdf_estimate_stats(gp, gm)
        st = _host(gp.get_state())
        same = st["elem"] == ost["elem"]
        assert (same | flagged).all()
        for k in KEYS:
            assert_field_close(st[k][same], ost[k][same], "no-slip step %d %s" % (s, k))
    assert events > 100
    wall_now = (st["u"] == 0.0) & (st["v"] == 0.0) & (st["w"] == 0.0)
    assert wall_now.any()


def test_noslip_fp32_state_invariants():
    m = _channel()
    n_tri = 2 * 19 * 39
    counts = np.full(n_tri, 30, dtype=np.int32)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 8, count=counts, u_sigma=0.2, elem_psi0=inputs.scalar_slab(m),
                      precision=capi.PDF_FP32_STATE)
    p = pg.model_params(closure="slm", dt=2e-3, nu=5e-3)
    pg.pdf_estimate_stats(gp, gm)
    for s in range(40):
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        assert info["lost"] == 0
        pg.pdf_estimate_stats(gp, gm)
    st = _host(gp.get_state())
    assert np.all(np.abs(st["y"]) <= 1.0)
    assert np.all(st["om"] >= 0)
    assert ((st["u"] == 0) & (st["v"] == 0) & (st["w"] == 0)).any()
    es = torch.empty((gm.n_tri, 13), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, es)
    assert int(es[:, 0].sum().item()) == int(counts.sum())


@pytest.mark.parametrize("multigrid", [True, False])
def test_noslip_relaxation_solve_matches_the_oracle(multigrid):
    """pdf_relax_solve_particles on the no-slip channel after a few steps: every
    component holds -4.5 eps n_i n_j on the no-slip nodes and the solution
    agrees with the oracle's sparse direct solve (each side with its own
    statistics)."""
    import oracle.relax as OR
    m = _channel()
    n_tri = 2 * 19 * 39
    counts = np.full(n_tri, 40, dtype=np.int32)
    psi = inputs.scalar_slab(m)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 9, count=counts, u_sigma=0.2, elem_psi0=psi)
    M = oracle.Mesh(m)
    ost = oracle.init(M, counts, 9, u_sigma=0.2, elem_psi0=psi)
    p = pg.model_params(closure="slm", dt=2e-3, nu=5e-3)
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure="slm", pressure="channel")
    pg.pdf_estimate_stats(gp, gm)
    es, ns, nd, _ = oracle.statistics(M, ost)
    for s in range(3):
        oracle.step(M, oracle.elem_coeff(M, ns, nd, po), po, 9, s, ost, omega_wall=oracle.noslip_omega(M, ns))
        es, ns, nd, _ = oracle.statistics(M, ost, ns)
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    wp = torch.zeros((9, gm.n_nodes), dtype=torch.float64, device="cuda")
    pg.pdf_relax_set_solver(gp, multigrid)
    iters, res = pg.pdf_relax_solve_particles(gp, gm, p, wp, rtol=1e-13, max_it=4000)
    got = wp.cpu().numpy()
    rhs = np.stack([oracle.relax_rhs(ns[n], nd[n]) for n in range(gm.n_nodes)], axis=1)
    ref = OR.solve(m, ns, rhs, p.nu)
    assert_field_close(got.T, ref.T, "no-slip relaxation solution", rtol=1e-9)
    walls = OR.wall_nodes(m, 5)
    _, nrm = OR.wall_normals(m)
    g = OR.noslip_values(ns, p.nu, nrm)
    assert np.allclose(got[:, walls], g[:, walls], rtol=1e-9, atol=1e-12)
    assert max(res) <= 1e-13
