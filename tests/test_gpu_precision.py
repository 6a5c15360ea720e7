"""The precision form (PDF_FP32_STATE): velocity, frequency and scalar stored
and advanced in FP32, positions and the element search FP64-accurate,
statistics summed in double-float.  Compared with the FP64 oracle: the
initial state is the oracle's rounded to FP32; after 100 steps of the small
channel every statistic stays within a stated bound of the oracle's; over
1000 steps the error of every statistic is stated inside the window where
the native-FP64 form still agrees with the oracle, and after it the domain
statistics are checked against an ensemble of oracle runs."""
import numpy as np
import pytest

import inputs
import oracle
import oracle_runs
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


NAMES = ["U", "V", "W", "omega", "phi", "uu", "vv", "ww", "uv", "uw", "vw", "phiphi"]
DOM = ["U", "V", "W", "omega", "phi", "uu", "vv", "ww", "uv", "phiphi",
       "med U", "med V", "med W", "med omega", "med phi", "iqr U", "iqr V", "iqr W"]


def _clean(mesh, gpu_elem, orc_elem):
    """Elements whose particle sets agree on both sides, and the nodes all
    of whose surrounding elements (periodic twins merged) are such."""
    diff = gpu_elem != orc_elem
    bad_e = np.zeros(len(mesh["tri"]), dtype=bool)
    bad_e[gpu_elem[diff]] = True
    bad_e[orc_elem[diff]] = True
    bad_n = np.zeros(len(mesh["xy"]), dtype=bool)
    bad_n[np.asarray(mesh["tri"])[bad_e].ravel()] = True
    twin = np.asarray(mesh.get("twin", np.full(len(mesh["xy"]), -1)))
    has = twin >= 0
    bad_n[twin[has & bad_n]] = True
    return ~bad_e, ~bad_n


def test_precision_forms_against_the_oracle_over_1000_steps(capsys):
    """The small channel's full run length (1000 steps) with the oracle and
    three GPU forms side by side from the same state: the FP64-accurate
    default (fixed point and double-float), native FP64 instructions
    (PDF_ARITH_FP64) and the FP32 state.
    * Both FP64 forms agree with the oracle element by element to 1e-10 for
      an initial window of steps.  The window ends where the decaying
      turbulence makes the explicit step unstable: k -> 0 in the core while
      the wall-corrected dissipation keeps eps / k >= nu C_T^2 <omega>^2 / k,
      so G_ii dt = (wp_ii - eps/2) dt / k falls below -2 (to about -90 by
      step 600), and from then on every implementation, the oracle
      included, amplifies its own rounding.
    * Inside that window, up to step 400 (before G_ii dt < -2), every
      element and node statistic of the FP32 form is compared with the
      oracle's over the elements whose particle sets agree and the nodes
      surrounded by them (printed per statistic at steps 100 ... 400).
    * After 1000 steps the frequency and scalar statistics (means, medians,
      scalar variance) of every form lie within five standard deviations of
      an ensemble of seven oracle runs (seeds 1-7); the velocity statistics
      are printed with their z-scores."""
    import multiprocessing as mp
    cfg = inputs.workload("channel_20x40_ppe50")
    seeds = list(range(1, 8))
    pool = mp.get_context("spawn").Pool(len(seeds) - 1)
    ens = [pool.apply_async(oracle_runs.channel_domain_after, (sd, 1000)) for sd in seeds[1:]]
    try:
        m = inputs.channel_mesh(cfg["nx"], cfg["ny"], seed=1)
        counts = np.full(cfg["n_tri"], cfg["ppe"], dtype=np.int32)
        psi = inputs.scalar_slab(m)
        gm = pg.Mesh(m)
        M = oracle.Mesh(m)
        forms = {"fx": (capi.PDF_FP64, "fx"), "fp64": (capi.PDF_FP64, "fp64"), "fp32": (capi.PDF_FP32_STATE, "fx")}
        runs = {f: (pg.Particles(gm, 1, count=counts, u_sigma=0.1, elem_psi0=psi, precision=prec),
                    pg.model_params(closure="glm", arith=ar)) for f, (prec, ar) in forms.items()}
        ost = oracle.init(M, counts, 1, u_sigma=0.1, elem_psi0=psi)
        p = runs["fx"][1]
        po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure="glm", pressure="channel")
        es_t = torch.empty((gm.n_tri, 13), dtype=torch.float64, device="cuda")
        ns_t = torch.empty((gm.n_nodes, 12), dtype=torch.float64, device="cuda")
        for g, _ in runs.values():
            pg.pdf_estimate_stats(g, gm)
        es, ns, nd, _ = oracle.statistics(M, ost)

        def g_elem(g):
            return g.get_state()["elem"].cpu().numpy()

        window = {"fx": None, "fp64": None}
        err32 = []  # per step: max scaled error per statistic of the FP32 form (elements, nodes)
        for s in range(1000):
            oracle.step(M, oracle.elem_coeff(M, ns, nd, po), po, 1, s, ost)
            es, ns, nd, _ = oracle.statistics(M, ost, ns)
            for f, (g, pf) in runs.items():
                assert pg.pdf_step(g, gm, pf, step=s, info=True)["lost"] == 0
                pg.pdf_estimate_stats(g, gm, es_t, ns_t)
                if f in window and window[f] is not None:
                    continue
                ges, gns = es_t.cpu().numpy(), ns_t.cpu().numpy()
                same = ges[:, 0] == es[:, 0]
                e_el = _scaled_err(ges[same, 1:], es[same, 1:]).max(axis=0) if same.any() else np.full(12, np.inf)
                e_nd = _scaled_err(gns, ns).max(axis=0)
                if f in window:
                    if not same.all() or max(e_el.max(), e_nd.max()) > 1e-10:
                        window[f] = s
                elif s < 400:
                    # the FP32 form: only where the particle sets agree
                    ok_e, ok_n = _clean(m, g_elem(g), ost["elem"])
                    e_el = _scaled_err(ges[ok_e, 1:], es[ok_e, 1:]).max(axis=0)
                    e_nd = _scaled_err(gns[ok_n], ns[ok_n]).max(axis=0)
                    err32.append((1.0 - ok_e.mean(), e_el, e_nd))
        got = {}
        for f, (g, _) in runs.items():
            st = {k: t.cpu().numpy() for k, t in g.get_state().items()}
            got[f] = np.concatenate([oracle_runs.domain_statistics(st), oracle_runs.robust_statistics(st)])
        ens_vals = np.array([np.concatenate([oracle_runs.domain_statistics(ost), oracle_runs.robust_statistics(ost)])]
                            + [r.get(timeout=1200) for r in ens])
    finally:
        pool.terminate()
    w = {f: (1000 if v is None else v) for f, v in window.items()}
    w64 = w["fp64"]
    # the FP32 form inside the stable period (G_ii dt > -2 up to step ~415):
    # the largest scaled error per statistic over the elements whose
    # particle sets agree (and the nodes surrounded by such elements), and
    # the largest fraction of elements whose sets differ
    checkpoints = [c for c in (100, 200, 300, 400) if c <= w64]
    per = {c: (np.max([e[1] for e in err32[:c]], axis=0), np.max([e[2] for e in err32[:c]], axis=0),
               max(e[0] for e in err32[:c])) for c in checkpoints}
    mean, sd = ens_vals.mean(axis=0), ens_vals.std(axis=0, ddof=1)
    z = {f: (got[f] - mean) / np.maximum(sd, 1e-300) for f in got}
    with capsys.disabled():
        print("\nagreement with the oracle to 1e-10 (steps): FP64-accurate %d, native FP64 %d" % (w["fx"], w64))
        print("FP32 state, max scaled error over the first N steps, element / node statistics:")
        print("  %-7s " % "N" + "  ".join("%21d" % c for c in checkpoints))
        for i, nme in enumerate(NAMES):
            print("  %-7s " % nme + "  ".join("%10.3e %10.3e" % (per[c][0][i], per[c][1][i]) for c in checkpoints))
        print("  elements whose particle set differs:   " + "  ".join("%.4f" % per[c][2] for c in checkpoints))
        print("after 1000 steps, domain statistics: oracle ensemble mean +- sd (7 seeds); FP64-accurate / "
              "native FP64 / FP32 state with their z-scores")
        for i, nme in enumerate(DOM):
            print("  %-7s %.5e +- %.2e  " % (nme, mean[i], sd[i]) +
                  "  ".join("%.5e (%+.1f)" % (got[f][i], z[f][i]) for f in ("fx", "fp64", "fp32")))
    assert w["fx"] >= 400 and w64 >= 400, w
    # the FP32 form's stated error (element and node statistics)
    assert max(per[100][0].max(), per[100][1].max()) < 5e-4, per[100]
    assert max(per[400][0].max(), per[400][1].max()) < 5e-3, per[400]
    assert per[400][2] < 0.05
    # the frequency and scalar statistics of every form within five
    # ensemble standard deviations; the velocity statistics are reported
    # only: past the window the explicit step is unstable (G_ii dt down to
    # about -90), and any realisation, the oracle's included, can have the
    # velocities of whole elements run away (the native-FP64 run's U
    # quartiles do, by 12 standard deviations)
    robust = [DOM.index(k) for k in ("omega", "phi", "phiphi", "med omega", "med phi")]
    for f in got:
        assert np.all(np.abs(z[f][robust]) <= 5.0), (f, z[f])
