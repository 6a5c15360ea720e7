"""Parity of the CUDA library (through its C-ABI) with the CPU oracle.

States and statistics: |gpu - oracle| <= 1e-10 * max(|oracle|, rms of the
field).  Random draws, the initial state and element ids: bit-exact, except
element ids of particles the oracle flags as within 1e-12 (relative) of an
element edge, whose fraction is reported.
"""
import math

import numpy as np
import pytest

import inputs
import oracle
from parity_util import RTOL, assert_field_close, stored_df, stored_position

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU only
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402

KEYS = ("x", "y", "u", "v", "w", "om", "ps")


def _host(st):
    return {k: v.cpu().numpy() for k, v in st.items()}


def _pair(m, counts, seed=1, psi=None, u_profile="parabola", u_sigma=0.1):
    gm = pg.Mesh(m)
    om_ = oracle.Mesh(m)
    gp = pg.Particles(gm, seed, count=counts, u_profile=u_profile, u_sigma=u_sigma, elem_psi0=psi)
    ost = oracle.init(om_, counts, seed, u_profile=u_profile, u_sigma=u_sigma, elem_psi0=psi)
    return gm, om_, gp, ost


def _oracle_params(p):
    names = {0: "glm", 1: "slm"}
    return oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=names[p.closure],
                              tm_mode={0: "turb", 1: "cphi"}[p.tm_mode], c_phi=p.c_phi,
                              pressure={0: "none", 1: "channel"}[p.pressure])


def test_gaussians_bit_exact():
    n = 200_003
    g = pg.pdf_rng_gauss(1, 7, 1, 0, n).cpu().numpy()
    ref = oracle.gauss_fill(1, n, 7, 1, 0)
    assert np.array_equal(g.view(np.uint32), ref.view(np.uint32))
    g2 = pg.pdf_rng_gauss(0xDEADBEEF12345678, 3, 0, 1, 1000).cpu().numpy()
    assert np.array_equal(g2, oracle.gauss_fill(0xDEADBEEF12345678, 1000, 3, 0, 1))


def test_connectivity_matches_oracle():
    for nx, ny in ((3, 2), (20, 40), (57, 31)):
        m = inputs.channel_mesh(nx, ny, seed=nx)
        nbr, shift = pg.Mesh(m).connectivity()
        M = oracle.Mesh(m)
        assert np.array_equal(nbr, M.nbr) and np.array_equal(shift, M.shift)


def test_init_bit_exact_with_ragged_counts():
    m = inputs.channel_mesh(20, 40, seed=1)
    rng = np.random.default_rng(0)
    counts = rng.integers(0, 9, 2 * 19 * 39).astype(np.int32)  # includes empty elements
    gm, M, gp, ost = _pair(m, counts, psi=inputs.scalar_slab(m))
    st = _host(gp.get_state())
    # the oracle's FP64 values, rounded to the stored forms
    for k in ("x", "y"):
        assert np.array_equal(st[k], stored_position(ost[k])), k
    for k in ("u", "v", "w", "om", "ps"):
        assert np.array_equal(st[k], stored_df(ost[k])), k
    assert np.array_equal(st["elem"], ost["elem"])


def _check_stats(gp, gm, M, ost, prev_ns=None):
    es = torch.empty((gm.n_tri, 13), dtype=torch.float64, device="cuda")
    ns = torch.empty((gm.n_nodes, 12), dtype=torch.float64, device="cuda")
    nd = torch.empty((gm.n_nodes, 10), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, es, ns, nd)
    es, ns, nd = es.cpu().numpy(), ns.cpu().numpy(), nd.cpu().numpy()
    oes, ons, ond, _ = oracle.statistics(M, ost, prev_ns)
    assert np.array_equal(es[:, 0], oes[:, 0]), "element counts"
    assert_field_close(es[:, 1:], oes[:, 1:], "element stats")
    assert_field_close(ns, ons, "node stats")
    assert_field_close(nd, ond, "node derivatives")
    return oes, ons, ond


def test_statistics_and_coefficients_after_init():
    m = inputs.channel_mesh(20, 40, seed=1)
    counts = np.full(2 * 19 * 39, 50, dtype=np.int32)
    gm, M, gp, ost = _pair(m, counts, psi=inputs.scalar_slab(m))
    oes, ons, ond = _check_stats(gp, gm, M, ost)
    for closure in ("glm", "slm"):
        p = pg.model_params(closure=closure)
        rows = pg.pdf_elem_coeff(gp, gm, p).cpu().numpy()
        ref = oracle.elem_coeff(M, ons, ond, _oracle_params(p))
        assert_field_close(rows, ref, "coefficient rows (%s)" % closure)
    # a given wp field
    rng = np.random.default_rng(3)
    wp = rng.normal(size=(9, gm.n_nodes)) * 0.01 - 0.02 * np.eye(3).reshape(9, 1)
    p = pg.model_params(closure="glm")
    rows = pg.pdf_elem_coeff(gp, gm, p, wp=torch.from_numpy(wp).cuda()).cpu().numpy()
    ref = oracle.elem_coeff(M, ons, ond, _oracle_params(p), wp=wp)
    assert_field_close(rows, ref, "coefficient rows (given wp)")


def _compare_states(st, ost, what, allow_flagged=None):
    el_ok = st["elem"] == ost["elem"]
    if allow_flagged is not None:
        bad = ~el_ok & ~allow_flagged
        assert not bad.any(), "%s: %d element ids differ outside the near-face band" % (what, bad.sum())
    else:
        assert el_ok.all(), "%s: %d element ids differ" % (what, (~el_ok).sum())
    for k in KEYS:
        assert_field_close(st[k][el_ok], ost[k][el_ok], "%s: %s" % (what, k))
    return float((~el_ok).mean())


@pytest.mark.parametrize("arith", ["fx", "fp64"])
def test_frozen_step_parity(arith):
    m = inputs.channel_mesh(20, 40, seed=1)
    counts = np.full(2 * 19 * 39, 30, dtype=np.int32)
    gm, M, gp, ost = _pair(m, counts, psi=inputs.scalar_slab(m))
    rng = np.random.default_rng(5)
    rows = np.zeros((gm.n_tri, 26))
    rows[:, 0:3] = rng.normal(size=(gm.n_tri, 3)) * 0.1
    rows[:, 3:9] = rng.normal(size=(gm.n_tri, 6))
    rows[:, 9:12] = rng.normal(size=(gm.n_tri, 3)) * 0.01
    G = rng.normal(size=(gm.n_tri, 9)) * 0.5
    G[:, [0, 4, 8]] -= 5.0
    rows[:, 12:21] = G
    rows[:, 21] = rng.uniform(0.1, 0.5, gm.n_tri)
    rows[:, 22] = rng.uniform(0.5, 2.0, gm.n_tri)
    rows[:, 23] = rng.normal(size=gm.n_tri)
    rows[:, 24] = rng.uniform(0, 1, gm.n_tri)
    rows[:, 25] = rng.uniform(0.5, 5, gm.n_tri)
    # the FROZEN closure moves positions with sqrt(2 nu) diffusion, as GLM
    # does (the SLM form, without it, runs in the free SLM runs of the
    # obstacle, no-slip and pressure tests)
    p = pg.model_params(closure="frozen", dt=2e-3, nu=1e-3, arith=arith)
    po = oracle.make_params(dt=2e-3, nu=1e-3, closure="glm")
    d_rows = torch.from_numpy(rows).cuda()
    info = pg.pdf_step(gp, gm, p, elem_coeff=d_rows, step=3, info=True)
    cnt, status = oracle.step(M, rows, po, 1, 3, ost)
    st = _host(gp.get_state())
    flagged = (status & oracle.TRK_NEAR_FACE) != 0
    _compare_states(st, ost, "frozen step", flagged)
    assert info["lost"] == 0 and cnt["lost"] == 0
    assert info["reflections"] == cnt["reflections"]
    assert info["crossings_periodic"] == cnt["crossings_periodic"]


def _run_config(name, steps, check_every=None, arith="fx", reorder=None):
    cfg = inputs.workload(name)
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], jitter=cfg["jitter"], seed=cfg["seed"])
    counts = np.full(cfg["n_tri"], cfg["ppe"], dtype=np.int32)
    psi = inputs.scalar_slab(m, cfg["psi_slab_x"])
    gm, M, gp, ost = _pair(m, counts, seed=cfg["seed"], psi=psi, u_sigma=cfg["u_sigma"])
    if reorder is not None:
        gp.set_reorder(reorder)
    p = pg.model_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure=cfg["closure"], arith=arith)
    po = _oracle_params(p)
    pg.pdf_estimate_stats(gp, gm)
    oes, ons, ond, _ = oracle.statistics(M, ost)
    near = []
    for s in range(steps):
        rows = oracle.elem_coeff(M, ons, ond, po)
        cnt, status = oracle.step(M, rows, po, cfg["seed"], s, ost)
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        assert info["lost"] == 0 and cnt["lost"] == 0
        oes, ons, ond, _ = oracle.statistics(M, ost, ons)
        pg.pdf_estimate_stats(gp, gm)
        if check_every and (s + 1) % check_every == 0:
            st = _host(gp.get_state())
            flagged = (status & oracle.TRK_NEAR_FACE) != 0
            near.append(_compare_states(st, ost, "step %d" % s, flagged))
    return gm, M, gp, ost, ons, near


@pytest.mark.parametrize("arith", ["fx", "fp64"])
def test_small_channel_free_run_100_steps(arith):
    """The small channel workload (20x40 nodes, 50 particles per element, GLM
    with the local wp, channel pressure), 100 steps free-running: states,
    statistics and element ids stay within the tolerance, for both the
    FP64-free default arithmetic and native FP64."""
    gm, M, gp, ost, ons, near = _run_config("channel_20x40_ppe50", 100, check_every=25, arith=arith)
    assert max(near) < 1e-4
    _check_stats(gp, gm, M, ost, ons)


def test_reordering_is_invisible_at_the_interface():
    """The state copied into element order at every statistics call (the
    densest reordering) against no reordering.  With frozen coefficients the
    steps do not depend on the statistics, so both runs hold bit-identical
    states (ids and random-number counters move with the particles) and
    counts; means and moments, summed in the storage order's grouping, agree
    to rounding.  A 30-step free run with every-call reordering still
    matches the oracle particle by particle."""
    m = inputs.channel_mesh(20, 40, seed=1)
    counts = np.random.default_rng(2).integers(0, 60, 2 * 19 * 39).astype(np.int32)
    rng = np.random.default_rng(7)
    n_tri = 2 * 19 * 39
    rows = np.zeros((n_tri, 26))
    rows[:, 0] = 1.0
    rows[:, 3:9] = rng.normal(size=(n_tri, 6)) * 0.1
    rows[:, 12:21] = np.tile(np.array([-5.0, 0, 0, 0, -5.0, 0, 0, 0, -5.0]), (n_tri, 1))
    rows[:, 21] = 0.3
    rows[:, 22] = 1.0
    rows[:, 24] = 0.5
    rows[:, 25] = 2.0
    d_rows = torch.from_numpy(rows).cuda()
    p = pg.model_params(closure="frozen", dt=5e-3, nu=1e-3)
    out = []
    for every in (0, 1):
        gm, M, gp, ost = _pair(m, counts, psi=inputs.scalar_slab(m))
        gp.set_reorder(every)
        pg.pdf_estimate_stats(gp, gm)
        for s in range(6):
            pg.pdf_step(gp, gm, p, elem_coeff=d_rows, step=s)
            pg.pdf_estimate_stats(gp, gm)
        es = torch.empty((gm.n_tri, 13), dtype=torch.float64, device="cuda")
        pg.pdf_estimate_stats(gp, gm, es)
        out.append((es.cpu().numpy(), _host(gp.get_state())))
    (es0, st0), (es1, st1) = out
    for k in KEYS + ("elem",):
        assert np.array_equal(st0[k], st1[k]), k
    assert (st0["elem"] != np.repeat(np.arange(n_tri), counts)).any()  # particles changed elements
    assert np.array_equal(es0[:, 0], es1[:, 0])
    assert_field_close(es1[:, 1:6], es0[:, 1:6], "means, reordered", rtol=1e-12)
    assert_field_close(es1[:, 6:], es0[:, 6:], "moments, reordered")
    gm, M, gp, ost, ons, near = _run_config("channel_20x40_ppe50", 30, check_every=10, reorder=1)
    assert max(near) < 1e-4
    _check_stats(gp, gm, M, ost, ons)


def test_tiny_mesh_edge_cases():
    """4 triangles, a handful of particles: warps and tiles mostly empty,
    empty elements, walls and seams crossed every step."""
    m = inputs.channel_mesh(3, 2, seed=2)
    counts = np.array([3, 0, 1, 5], dtype=np.int32)
    gm, M, gp, ost = _pair(m, counts, u_sigma=0.5)
    p = pg.model_params(closure="slm", dt=0.05, nu=1e-3)
    po = _oracle_params(p)
    assert p.arith == 0  # the default FP64-free kernel (walls go to its FP64 fall-back)
    pg.pdf_estimate_stats(gp, gm)
    oes, ons, ond, _ = oracle.statistics(M, ost)
    for s in range(20):
        rows = oracle.elem_coeff(M, ons, ond, po)
        cnt, status = oracle.step(M, rows, po, 1, s, ost)
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        oes, ons, ond, _ = oracle.statistics(M, ost, ons)
        pg.pdf_estimate_stats(gp, gm)
        st = _host(gp.get_state())
        _compare_states(st, ost, "tiny step %d" % s, (status & oracle.TRK_NEAR_FACE) != 0)
    _check_stats(gp, gm, M, ost, ons)


def test_full_size_steps_and_statistics():
    """The measured workload (200x400 nodes, 100 particles per element, ~16M
    particles) in the launch configuration the benchmark times: the oracle
    runs the same two steps at full size on its own, then every particle,
    every element statistic, every node statistic and derivative (80,000
    nodes) and every coefficient row is compared, except where a particle
    the oracle flagged within 1e-12 of a face took the other element: those
    elements, and the nodes and rows that depend on them (one ring of
    elements per averaging pass), are left out."""
    cfg = inputs.workload("channel_200x400_ppe100")
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], jitter=cfg["jitter"], seed=cfg["seed"])
    psi = inputs.scalar_slab(m, cfg["psi_slab_x"])
    counts = np.full(cfg["n_tri"], cfg["ppe"], dtype=np.int32)
    gm, M, gp, ost = _pair(m, counts, seed=cfg["seed"], psi=psi, u_sigma=cfg["u_sigma"])
    p = pg.model_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure=cfg["closure"])
    po = _oracle_params(p)
    pg.pdf_estimate_stats(gp, gm)
    oes, ons, ond, _ = oracle.statistics(M, ost)
    flagged = np.zeros(gp.n, dtype=bool)
    for s in range(2):
        rows = oracle.elem_coeff(M, ons, ond, po)
        cnt, status = oracle.step(M, rows, po, cfg["seed"], s, ost)
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        assert info["lost"] == 0 and cnt["lost"] == 0
        flagged |= (status & oracle.TRK_NEAR_FACE) != 0
        oes, ons, ond, _ = oracle.statistics(M, ost, ons)
        pg.pdf_estimate_stats(gp, gm)
    st = _host(gp.get_state())
    _compare_states(st, ost, "full-size, 2 steps", flagged)
    es = torch.empty((gm.n_tri, 13), dtype=torch.float64, device="cuda")
    ns = torch.empty((gm.n_nodes, 12), dtype=torch.float64, device="cuda")
    nd = torch.empty((gm.n_nodes, 10), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, es, ns, nd)
    es, ns, nd = es.cpu().numpy(), ns.cpu().numpy(), nd.cpu().numpy()
    touched = np.zeros(gm.n_tri, dtype=bool)
    moved = st["elem"] != ost["elem"]
    touched[st["elem"][moved]] = True
    touched[ost["elem"][moved]] = True
    assert np.array_equal(es[~touched, 0], oes[~touched, 0])
    assert_field_close(es[~touched, 1:], oes[~touched, 1:], "full-size element stats")
    tri = np.asarray(m["tri"])
    twin = np.asarray(m["twin"])

    def ring(bad_e):
        """Nodes of the given elements (periodic twins merged), and every
        element holding such a node."""
        bad_n = np.zeros(gm.n_nodes, dtype=bool)
        bad_n[tri[bad_e].ravel()] = True
        bad_n[twin[(twin >= 0) & bad_n]] = True
        return bad_n, bad_n[tri].any(axis=1)

    n1, e1 = ring(touched)   # node statistics
    n2, e2 = ring(e1)        # first derivatives
    n3, e3 = ring(e2)        # second derivatives
    assert (~n3).mean() > 0.99
    assert_field_close(ns[~n1], ons[~n1], "full-size node stats")
    assert_field_close(nd[~n3, :6], ond[~n3, :6], "full-size node gradients")
    assert_field_close(nd[~n3, 6:], ond[~n3, 6:], "full-size node second derivatives and d<vv>/dy")
    # coefficient rows: element means of the three nodal coefficient sets
    rows = pg.pdf_elem_coeff(gp, gm, p).cpu().numpy()
    ref = oracle.elem_coeff(M, ons, ond, po)
    _, e4 = ring(e3)
    assert_field_close(rows[~e4], ref[~e4], "full-size coefficient rows")


def test_grouping_beyond_one_scan_round_per_digit():
    """More radix tiles (4,096 keys each) than one scan block covers in a
    round (4,096): 132 particles per element of the 200x400 channel,
    20,961,864 particles in 5,118 tiles, so the per-digit scan of the tile
    counts runs two rounds.  After initialisation and after each of four
    steps (the fourth statistics call reorders the state) the element counts
    equal the bincount of the particles' element ids exactly, and the
    element means of u and psi agree with means taken on the host in FP64
    to 1e-12."""
    cfg = inputs.workload("channel_200x400_ppe100")
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], jitter=cfg["jitter"], seed=cfg["seed"])
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 5, ppe=132, u_sigma=cfg["u_sigma"], elem_psi0=inputs.scalar_slab(m, cfg["psi_slab_x"]))
    assert (gp.n + 4095) // 4096 > 4096
    p = pg.model_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure=cfg["closure"])
    es = torch.empty((gm.n_tri, 13), dtype=torch.float64, device="cuda")
    for s in range(5):
        if s > 0:
            assert pg.pdf_step(gp, gm, p, step=s - 1, info=True)["lost"] == 0
        pg.pdf_estimate_stats(gp, gm, es)
        st = _host(gp.get_state())
        e = es.cpu().numpy()
        cnt = np.bincount(st["elem"], minlength=gm.n_tri)
        assert np.array_equal(e[:, 0], cnt.astype(np.float64)), s
        nz = cnt > 0
        for k, col in (("u", 1), ("ps", 5)):
            mean = np.bincount(st["elem"], weights=st[k], minlength=gm.n_tri)[nz] / cnt[nz]
            scale = max(float(np.sqrt(np.mean(mean * mean))), 1e-300)
            assert float(np.max(np.abs(e[nz, col] - mean))) / scale < 1e-12, (s, k)


def test_fallbacks_for_values_outside_the_fixed_point_ranges():
    """Elements holding particles with |u| >= 128 or omega >= 2^14 (outside
    the range of the exact integer statistics) and particles that move two
    length units in the step (outside the fixed-point path of the step) are
    handled by the FP64 fall-backs; results still match."""
    m = inputs.channel_mesh(20, 40, seed=1)
    counts = np.full(2 * 19 * 39, 20, dtype=np.int32)
    gm, M, gp, ost = _pair(m, counts, psi=inputs.scalar_slab(m))
    sel = ost["elem"] < 12
    ost["u"][sel] += 300.0
    # scaled (not shifted) so that the element variances keep their relative
    # size: the stored double-float state carries 48 bits
    ost["u"][(ost["elem"] >= 12) & (ost["elem"] < 16)] *= 2.0e4
    ost["om"][ost["elem"] == 40] += 5000.0
    st = {k: torch.from_numpy(np.ascontiguousarray(ost[k])).cuda() for k in KEYS}
    st["elem"] = torch.from_numpy(ost["elem"]).cuda()
    gp.set_state(st)
    oes, ons, ond = _check_stats(gp, gm, M, ost)
    p = pg.model_params(closure="slm", dt=1e-4)
    po = _oracle_params(p)
    rows = oracle.elem_coeff(M, ons, ond, po)
    cnt, status = oracle.step(M, rows, po, 1, 0, ost)
    info = pg.pdf_step(gp, gm, p, step=0, info=True)
    got = _host(gp.get_state())
    _compare_states(got, ost, "fall-back step", (status & oracle.TRK_NEAR_FACE) != 0)
    assert info["lost"] == 0


@pytest.mark.parametrize("multigrid", [True, False])
def test_relaxation_solve_matches_the_oracle(multigrid):
    """pdf_relax_solve_particles on the small channel after a few steps: the nodal
    right-hand side, the L^2 fields and the converged solution agree with the
    oracle's assembly and sparse direct solve (multigrid and Jacobi
    preconditioners)."""
    import oracle.relax as OR
    m = inputs.channel_mesh(20, 40, seed=1)
    counts = np.full(2 * 19 * 39, 50, dtype=np.int32)
    gm, M, gp, ost = _pair(m, counts, psi=inputs.scalar_slab(m))
    p = pg.model_params(closure="glm")
    po = _oracle_params(p)
    pg.pdf_estimate_stats(gp, gm)
    oes, ons, ond, _ = oracle.statistics(M, ost)
    for s in range(3):   # both sides on their own
        oracle.step(M, oracle.elem_coeff(M, ons, ond, po), po, 1, s, ost)
        oes, ons, ond, _ = oracle.statistics(M, ost, ons)
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    S, Dv = ons, ond
    rhs, L2 = pg.pdf_relax_rhs(gp, gm, p)
    ref_rhs = np.stack([oracle.relax_rhs(S[n], Dv[n]) for n in range(gm.n_nodes)], axis=1)
    assert_field_close(rhs.cpu().numpy().T, ref_rhs.T, "relaxation right-hand side")
    dist, nrm = OR.wall_normals(m)
    gd, gn = gm.wall_distance()
    assert np.allclose(gd, dist, atol=1e-14) and np.array_equal(gn, nrm)
    for c, cxi in enumerate((1 + 1.3 * nrm[:, 0] ** 2, 1 + 1.3 * nrm[:, 1] ** 2, np.ones(gm.n_nodes))):
        assert_field_close(L2[c].cpu().numpy(), OR.lengthscale2(S, p.nu, cxi), "L^2 class %d" % c)
    wp = torch.zeros((9, gm.n_nodes), dtype=torch.float64, device="cuda")
    pg.pdf_relax_set_solver(gp, multigrid)
    iters, res = pg.pdf_relax_solve_particles(gp, gm, p, wp, rtol=1e-13, max_it=2000)
    ref = OR.solve(m, S, ref_rhs, p.nu)
    assert_field_close(wp.cpu().numpy().T, ref.T, "relaxation solution", rtol=1e-9)
    assert max(res) <= 1e-13
    # warm start from the solution: converged at once
    iters2, _ = pg.pdf_relax_solve_particles(gp, gm, p, wp, rtol=1e-10, max_it=2000)
    assert max(iters2) <= 1


def test_relaxation_multigrid_and_jacobi_agree_on_a_larger_channel():
    """The 100 x 200 channel (about 20,000 unknowns): both preconditioners
    reach the same solution; the multigrid needs far fewer iterations, and
    the choice can be switched between solves."""
    m = inputs.channel_mesh(100, 200, seed=3)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 4, ppe=30, u_sigma=0.1)
    p = pg.model_params(closure="glm")
    pg.pdf_estimate_stats(gp, gm)
    pg.pdf_step(gp, gm, p, step=0)
    pg.pdf_estimate_stats(gp, gm)
    out = {}
    for mg in (True, False, True):
        wp = torch.zeros((9, gm.n_nodes), dtype=torch.float64, device="cuda")
        pg.pdf_relax_set_solver(gp, mg)
        iters, res = pg.pdf_relax_solve_particles(gp, gm, p, wp, rtol=1e-12, max_it=20000)
        assert max(res) <= 1e-12
        if mg in out:
            assert list(iters) == out[mg][0]
            assert torch.equal(wp, out[mg][1])
        out[mg] = (list(iters), wp)
    it_mg, it_j = max(out[True][0]), max(out[False][0])
    assert it_mg * 4 < it_j, (it_mg, it_j)
    scale = out[False][1].abs().amax(dim=1, keepdim=True).clamp_min(1e-300)
    assert float(((out[True][1] - out[False][1]).abs() / scale).max()) < 1e-9


@pytest.mark.parametrize("multigrid", [True, False])
def test_relaxation_solve_on_a_tiny_mesh(multigrid):
    """An 8 x 6 channel (42 unknowns): the multigrid has no level and solves
    with the dense inverse of the whole matrix; both preconditioners agree
    with the oracle's direct solve."""
    import oracle.relax as OR
    m = inputs.channel_mesh(8, 6, seed=1)
    counts = np.full(2 * 7 * 5, 40, dtype=np.int32)
    gm, M, gp, ost = _pair(m, counts, psi=inputs.scalar_slab(m))
    p = pg.model_params(closure="glm")
    pg.pdf_estimate_stats(gp, gm)
    pg.pdf_step(gp, gm, p, step=0)
    ns = torch.empty((gm.n_nodes, pg.capi.PDF_NNS), dtype=torch.float64, device="cuda")
    nd = torch.empty((gm.n_nodes, pg.capi.PDF_NND), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, node_stats=ns, node_derivs=nd)
    S, Dv = ns.cpu().numpy(), nd.cpu().numpy()
    wp = torch.zeros((9, gm.n_nodes), dtype=torch.float64, device="cuda")
    pg.pdf_relax_set_solver(gp, multigrid)
    iters, res = pg.pdf_relax_solve_particles(gp, gm, p, wp, rtol=1e-13, max_it=500)
    assert max(res) <= 1e-13
    rhs = np.stack([oracle.relax_rhs(S[n], Dv[n]) for n in range(gm.n_nodes)], axis=1)
    ref = OR.solve(m, S, rhs, p.nu)
    assert_field_close(wp.cpu().numpy().T, ref.T, "tiny-mesh relaxation solution", rtol=1e-9)
    if multigrid:   # the exact inverse up to FP32 rounding: a few iterations
        assert max(iters) <= 12, iters


@pytest.mark.parametrize("nx,ny,ppe", [(20, 40, 50), (200, 400, 6)])
def test_relaxation_solve_of_the_oracle_statistics(nx, ny, ppe):
    """pdf_relax_solve, the mesh-level call: node statistics computed by the
    oracle go in through the C-ABI; the library forms the node derivatives,
    the right-hand side and L^2 itself and solves (multigrid PCG to 1e-13).
    On the small channel the solution matches the oracle's sparse direct
    solve; on the 80,000-node channel of the benchmark mesh (where that
    solve is slow) the solution's residual in each of the oracle's nine
    assembled systems is below 1e-12.  A second call warm-started from the
    solution stops at once."""
    import oracle.relax as OR
    m = inputs.channel_mesh(nx, ny, seed=1)
    M = oracle.Mesh(m)
    counts = np.full(M.n_tri, ppe, dtype=np.int32)
    ost = oracle.init(M, counts, 3, u_sigma=0.1, elem_psi0=inputs.scalar_slab(m))
    es, ns, nd, _ = oracle.statistics(M, ost)
    gm = pg.Mesh(m)
    p = pg.model_params(closure="glm")
    S = torch.from_numpy(np.ascontiguousarray(ns)).cuda()
    wp = torch.zeros((9, gm.n_nodes), dtype=torch.float64, device="cuda")
    iters, res = pg.pdf_relax_solve(gm, p, S, wp, rtol=1e-13, max_it=4000)
    assert max(res) <= 1e-13
    rhs = np.stack([oracle.relax_rhs(ns[n], nd[n]) for n in range(gm.n_nodes)], axis=1)
    x = wp.cpu().numpy()
    if gm.n_nodes <= 5000:
        ref = OR.solve(m, ns, rhs, p.nu)
        assert_field_close(x.T, ref.T, "mesh-level relaxation solution", rtol=1e-9)
    r = OR.residual(m, ns, rhs, p.nu, x)
    assert r.max() < 1e-12, r
    iters2, _ = pg.pdf_relax_solve(gm, p, S, wp, rtol=1e-10, max_it=4000)
    assert max(iters2) <= 1
