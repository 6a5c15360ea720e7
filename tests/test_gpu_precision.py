"""The precision form (PDF_FP32_STATE): velocity, frequency and scalar stored
and advanced in FP32, positions and the element search FP64-accurate,
statistics exact integer sums.  Compared with the FP64 oracle: the initial
state is the oracle's rounded to FP32; after 100 steps of the small
channel every statistic stays within a stated bound of the oracle's, and
after 1000 steps the domain statistics are compared with the FP64-accurate
form run alongside."""
import numpy as np
import pytest

import inputs
import oracle
from parity_util import stored_position

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402
from paper_1006_0720_gb300 import capi  # noqa: E402

KEYS = ("x", "y", "u", "v", "w", "om", "ps")


def _scaled_err(a, b):
    sf = np.sqrt(np.mean(b * b, axis=0, keepdims=True))
    scale = np.maximum(np.abs(b), sf)
    scale = np.where(scale == 0, 1.0, scale)
    return np.abs(a - b) / scale


def test_fp32_state_init_is_the_rounded_fp64_state():
    m = inputs.channel_mesh(20, 40, seed=1)
    counts = np.full(2 * 19 * 39, 10, dtype=np.int32)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 1, count=counts, u_sigma=0.1, elem_psi0=inputs.scalar_slab(m),
                      precision=capi.PDF_FP32_STATE)
    ost = oracle.init(oracle.Mesh(m), counts, 1, u_sigma=0.1, elem_psi0=inputs.scalar_slab(m))
    st = {k: v.cpu().numpy() for k, v in gp.get_state().items()}
    assert np.array_equal(st["x"], stored_position(ost["x"])) and np.array_equal(st["y"], stored_position(ost["y"]))
    for k in ("u", "v", "w", "om", "ps"):
        assert np.array_equal(st[k], ost[k].astype(np.float32).astype(np.float64)), k


def _run(steps):
    cfg = inputs.workload("channel_20x40_ppe50")
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], seed=1)
    counts = np.full(cfg["n_tri"], cfg["ppe"], dtype=np.int32)
    psi = inputs.scalar_slab(m)
    gm = pg.Mesh(m)
    M = oracle.Mesh(m)
    gp = pg.Particles(gm, 1, count=counts, u_sigma=0.1, elem_psi0=psi, precision=capi.PDF_FP32_STATE)
    ost = oracle.init(M, counts, 1, u_sigma=0.1, elem_psi0=psi)
    p = pg.model_params(closure="glm")
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure="glm", pressure="channel")
    pg.pdf_estimate_stats(gp, gm)
    es, ns, nd, _ = oracle.statistics(M, ost)
    es0 = es.copy()
    for s in range(steps):
        rows = oracle.elem_coeff(M, ns, nd, po)
        oracle.step(M, rows, po, 1, s, ost)
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        assert info["lost"] == 0
        es, ns, nd, _ = oracle.statistics(M, ost, ns)
        pg.pdf_estimate_stats(gp, gm)
    ges = torch.empty((gm.n_tri, 13), dtype=torch.float64, device="cuda")
    gns = torch.empty((gm.n_nodes, 12), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, ges, gns)
    ges, gns = ges.cpu().numpy(), gns.cpu().numpy()
    e_el = _scaled_err(ges[:, 1:], es[:, 1:]).max(axis=0)
    e_nd = _scaled_err(gns, ns).max(axis=0)
    # on the scale of the initial fields (RMS over the elements at step 0):
    # the largest element difference and the difference of the domain means
    S0 = np.sqrt(np.mean(es0[:, 1:] ** 2, axis=0))
    S0 = np.where(S0 > 0, S0, 1.0)
    e_phys = (np.abs(ges[:, 1:] - es[:, 1:]).max(axis=0)) / S0
    e_dom = np.abs(ges[:, 1:].mean(axis=0) - es[:, 1:].mean(axis=0)) / S0
    names = ["U", "V", "W", "omega", "phi", "uu", "vv", "ww", "uv", "uw", "vw", "phiphi"]
    print("after %d steps" % steps)
    print("max scaled error per element statistic:", dict(zip(names, np.round(e_el, 9))))
    print("max scaled error per node statistic:", dict(zip(names, np.round(e_nd, 9))))
    print("max element difference on the initial scale:", dict(zip(names, np.round(e_phys, 6))))
    print("domain-mean difference on the initial scale:", dict(zip(names, np.round(e_dom, 8))))
    moved = np.mean(ges[:, 0] != es[:, 0])
    print("fraction of elements whose particle count differs:", moved)
    return e_el, e_nd, e_phys, e_dom, moved


def test_fp32_state_statistics_after_100_steps():
    e_el, e_nd, e_phys, e_dom, moved = _run(100)
    assert e_nd.max() < 1e-3
    assert moved < 0.02


def test_fp32_state_statistics_after_1000_steps(capsys):
    """The precision form's report over the small channel's full run length
    (1000 steps), with the FP64-accurate form run alongside as the control.
    In this run the turbulent energy of some elements collapses after ~400
    steps; there the drift G_ij dt falls below -2 (G_11 dt = -3.1 in one
    element), the explicit step amplifies any rounding difference more than
    twofold per step, and both GPU forms depart from the oracle (the
    FP64-accurate one after agreeing to 1e-13 for 430 steps).  From then on
    the runs agree statistically: the FP32 form's domain means stay about as
    close to the oracle's as the FP64-accurate form's do."""
    cfg = inputs.workload("channel_20x40_ppe50")
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], seed=1)
    counts = np.full(cfg["n_tri"], cfg["ppe"], dtype=np.int32)
    psi = inputs.scalar_slab(m)
    gm = pg.Mesh(m)
    M = oracle.Mesh(m)
    runs = {f: pg.Particles(gm, 1, count=counts, u_sigma=0.1, elem_psi0=psi, precision=f)
            for f in (capi.PDF_FP64, capi.PDF_FP32_STATE)}
    ost = oracle.init(M, counts, 1, u_sigma=0.1, elem_psi0=psi)
    p = pg.model_params(closure="glm")
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure="glm", pressure="channel")
    for g in runs.values():
        pg.pdf_estimate_stats(g, gm)
    es, ns, nd, _ = oracle.statistics(M, ost)
    for s in range(1000):
        oracle.step(M, oracle.elem_coeff(M, ns, nd, po), po, 1, s, ost)
        es, ns, nd, _ = oracle.statistics(M, ost, ns)
        for g in runs.values():
            assert pg.pdf_step(g, gm, p, step=s, info=True)["lost"] == 0
            pg.pdf_estimate_stats(g, gm)

    def dom(st):
        u, v, w = st["u"], st["v"], st["w"]
        return np.array([u.mean(), v.mean(), w.mean(), st["om"].mean(), st["ps"].mean(), u.var(), v.var(), w.var(),
                         np.mean((u - u.mean()) * (v - v.mean())), st["ps"].var()])

    names = ["U", "V", "W", "omega", "phi", "uu", "vv", "ww", "uv", "phiphi"]
    ref = dom(ost)
    got = {f: dom({k: t.cpu().numpy() for k, t in g.get_state().items()}) for f, g in runs.items()}
    d64 = np.abs(got[capi.PDF_FP64] - ref)
    d32 = np.abs(got[capi.PDF_FP32_STATE] - ref)
    with capsys.disabled():
        print("\nafter 1000 steps, domain statistics: oracle / FP64-accurate / FP32 state")
        for i, nme in enumerate(names):
            print("  %-7s %.6e  %.6e  %.6e" % (nme, ref[i], got[capi.PDF_FP64][i], got[capi.PDF_FP32_STATE][i]))
    # the FP32 form stays about as close to the oracle as the FP64-accurate
    # form (two realisations that parted ways: a factor of three)
    assert np.all(d32 <= 3.0 * d64 + 1e-3 * np.abs(ref) + 1e-6), (d32, d64)
    assert abs(got[capi.PDF_FP32_STATE][3] / ref[3] - 1) < 1e-3
