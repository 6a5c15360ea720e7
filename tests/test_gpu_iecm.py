"""IECM (eq. IECM) on the GPU against the oracle, each side on its own from
the same seeded initial state: the velocity-conditioned scalar means of the
sort-and-divide binning, and free-running IECM steps.  The sorts see the
same values up to the stored state's rounding (2^-48), so only exact ties
could order differently; ties are broken by particle id on both sides."""
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


def _setup(precision=capi.PDF_FP64, big=True):
    m = inputs.channel_mesh(20, 40, seed=1)
    n_tri = 2 * 19 * 39
    counts = np.random.default_rng(5).integers(0, 120, n_tri).astype(np.int32)
    if big:
        counts[[7, 300, 301]] = [600, 777, 1500]   # above the shared-memory capacity of 256
    counts[[11, 12]] = [1, 2]
    psi = inputs.scalar_slab(m)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 3, count=counts, u_sigma=0.2, elem_psi0=psi, precision=precision)
    M = oracle.Mesh(m)
    ost = oracle.init(M, counts, 3, u_sigma=0.2, elem_psi0=psi)
    return m, gm, gp, n_tri, M, ost


def _run(gm, gp, M, ost, n_tri, steps, p, po, bins, m_min, iecm):
    """steps on both sides; returns the near-face flags of the oracle's steps"""
    pg.pdf_estimate_stats(gp, gm)
    es, ns, nd, _ = oracle.statistics(M, ost)
    flagged = np.zeros(len(ost["x"]), dtype=bool)
    for s in range(steps):
        cond = oracle.iecm_cond(n_tri, ost, bins=bins, m_min=m_min) if iecm else None
        cnt, status = oracle.step(M, oracle.elem_coeff(M, ns, nd, po), po, 3, s, ost, cond=cond)
        info = pg.pdf_step(gp, gm, p, step=s, info=True)
        assert info["lost"] == 0 and cnt["lost"] == 0
        flagged |= (status & oracle.TRK_NEAR_FACE) != 0
        es, ns, nd, _ = oracle.statistics(M, ost, ns)
        pg.pdf_estimate_stats(gp, gm)
    return flagged


@pytest.mark.parametrize("bins,m_min", [((5, 5, 5), 2), ((2, 2, 2), 2), ((4, 12, 5), 3), ((3, 1, 1), 1)])
def test_conditional_means_match_the_oracle(bins, m_min):
    m, gm, gp, n_tri, M, ost = _setup()
    p = pg.model_params(closure="slm", dt=2e-3)
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure="slm", pressure="channel")
    # particles change elements and the storage gets out of order
    flagged = _run(gm, gp, M, ost, n_tri, 3, p, po, bins, m_min, False)
    gp.set_iecm(bins, m_min)
    pg.pdf_estimate_stats(gp, gm)
    st = _host(gp.get_state())
    assert np.array_equal(st["elem"][~flagged], ost["elem"][~flagged])
    got = gp.iecm_cond().cpu().numpy()
    want = oracle.iecm_cond(n_tri, ost, bins=bins, m_min=m_min)
    bad = np.zeros(n_tri, dtype=bool)   # elements a near-face particle may have changed
    bad[st["elem"][flagged]] = True
    bad[ost["elem"][flagged]] = True
    ok = ~bad[ost["elem"]]
    assert_field_close(got[ok], want[ok], "IECM conditional means %s" % (bins,))
    # the conditional means preserve each element's scalar sum
    s_c = np.bincount(st["elem"], weights=got, minlength=n_tri)
    s_p = np.bincount(st["elem"], weights=st["ps"], minlength=n_tri)
    assert np.allclose(s_c, s_p, rtol=1e-12, atol=1e-12)


def test_iecm_steps_match_the_oracle():
    m, gm, gp, n_tri, M, ost = _setup(big=False)
    gp.set_iecm((5, 5, 5), 2)
    p = pg.model_params(closure="slm", dt=2e-3, mix="iecm")
    po = oracle.make_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure="slm", pressure="channel")
    flagged = _run(gm, gp, M, ost, n_tri, 6, p, po, (5, 5, 5), 2, True)
    got = _host(gp.get_state())
    ok = (got["elem"] == ost["elem"]) | flagged
    assert ok.all()
    same = got["elem"] == ost["elem"]
    for k in KEYS:
        assert_field_close(got[k][same], ost[k][same], "IECM steps %s" % k)


def test_iecm_needs_conditional_means():
    m, gm, gp, n_tri, M, ost = _setup(big=False)
    pg.pdf_estimate_stats(gp, gm)
    p = pg.model_params(closure="slm", mix="iecm")
    with pytest.raises(pg.PdfError):
        pg.pdf_step(gp, gm, p, step=0)


def test_fp32_state_conditional_means():
    # FP32 velocities: the GPU sorts the FP32 values, the oracle the FP64
    # ones; the binning agrees unless two values round to the same FP32
    # number, so compare the element sums and the bulk of the particles
    m, gm, gp, n_tri, M, ost = _setup(precision=capi.PDF_FP32_STATE)
    gp.set_iecm((5, 5, 5), 2)
    pg.pdf_estimate_stats(gp, gm)
    got = gp.iecm_cond().cpu().numpy()
    want = oracle.iecm_cond(n_tri, ost, bins=(5, 5, 5), m_min=2)
    close = np.abs(got - want) <= 1e-6 * np.maximum(1.0, np.abs(want))
    assert close.mean() > 0.999
    s_c = np.bincount(ost["elem"], weights=got, minlength=n_tri)
    s_p = np.bincount(ost["elem"], weights=ost["ps"], minlength=n_tri)
    assert np.allclose(s_c, s_p, rtol=1e-6, atol=1e-6)
