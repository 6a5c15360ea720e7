"""Particle redistribution (App. D) on the GPU: bit-exact against the
oracle from the same seeded state (FP64 and FP32 state forms, critical
elements with 0 to min_npel - 1 particles), and its invariants after steps
and a reordering of the state (particle ids then differ from the storage
slots)."""
import numpy as np
import pytest

import inputs
import oracle
from parity_util import stored_df, stored_position

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402
from paper_1006_0720_gb300 import capi  # noqa: E402

KEYS = ("x", "y", "u", "v", "w", "om", "ps")


def _host(st):
    return {k: v.cpu().numpy() for k, v in st.items()}


def _counts(n_tri, seed):
    rng = np.random.default_rng(seed)
    c = rng.integers(0, 40, size=n_tri).astype(np.int32)
    c[rng.choice(n_tri, 60, replace=False)] = rng.integers(0, 6, size=60)
    return c


@pytest.mark.parametrize("precision", [capi.PDF_FP64, capi.PDF_FP32_STATE])
def test_redistribution_matches_the_oracle(precision):
    m = inputs.channel_mesh(20, 40, seed=1)
    counts = _counts(2 * 19 * 39, 4)
    psi = inputs.scalar_slab(m)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 5, count=counts, u_sigma=0.3, elem_psi0=psi, precision=precision)
    M = oracle.Mesh(m)
    ost = oracle.init(M, counts, 5, u_sigma=0.3, elem_psi0=psi)
    mn = 8
    moved = pg.pdf_redistribute(gp, gm, mn, seed=5, step=17)
    moved_o = oracle.redistribute(M, ost, mn, seed=5, step=17)
    assert moved == moved_o > 100
    st = _host(gp.get_state())
    assert np.array_equal(st["elem"], ost["elem"])
    assert np.bincount(st["elem"], minlength=gm.n_tri).min() >= mn
    for k in ("x", "y"):
        assert np.array_equal(st[k], stored_position(ost[k])), k
    for k in ("u", "v", "w", "om", "ps"):
        ref = stored_df(ost[k]) if precision == capi.PDF_FP64 else ost[k].astype(np.float32).astype(np.float64)
        assert np.array_equal(st[k], ref), k
    # the next statistics see the new distribution; stepping needs them
    with pytest.raises(capi.PdfError):
        pg.pdf_step(gp, gm, pg.model_params(closure="slm"), step=18)
    es = torch.empty((gm.n_tri, capi.PDF_NES), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, es)
    assert np.array_equal(es[:, 0].cpu().numpy().astype(np.int64), np.bincount(ost["elem"], minlength=gm.n_tri))


def test_redistribution_invariants_after_steps_and_reordering():
    m = inputs.channel_mesh(20, 40, seed=1)
    counts = _counts(2 * 19 * 39, 7)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 9, count=counts, u_sigma=0.3, elem_psi0=inputs.scalar_slab(m))
    gp.set_reorder(1)
    p = pg.model_params(closure="slm")
    pg.pdf_estimate_stats(gp, gm)
    for s in range(5):
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    before = _host(gp.get_state())
    n_before = np.bincount(before["elem"], minlength=gm.n_tri)
    mn = 10
    moved = pg.pdf_redistribute(gp, gm, mn, seed=9, step=5)
    after = _host(gp.get_state())
    n_after = np.bincount(after["elem"], minlength=gm.n_tri)
    assert n_after.sum() == n_before.sum()
    assert moved == int(np.abs(n_after - n_before).sum() // 2) > 0
    crit = np.nonzero(n_before < mn)[0]
    assert np.all(n_after[crit] >= mn)
    changed = np.nonzero(after["elem"] != before["elem"])[0]
    for q in changed:
        j = after["elem"][q]
        own = np.nonzero((before["elem"] == j))[0]
        if len(own):
            # a copy of one of the receiving element's particles
            hit = np.ones(len(own), dtype=bool)
            for k in KEYS:
                hit &= before[k][own] == after[k][q]
            assert hit.any()
        else:
            assert all(after[k][q] == before[k][q] for k in ("u", "v", "w", "om", "ps"))
    # donors gave their lowest particle ids
    for e in np.unique(before["elem"][changed]):
        mine = np.nonzero(before["elem"] == e)[0]   # get_state is in particle-id order
        gone = np.isin(mine, changed)
        assert np.all(gone[:gone.sum()]) and not np.any(gone[gone.sum():])
    pg.pdf_estimate_stats(gp, gm)
    pg.pdf_step(gp, gm, p, step=6)


def test_redistribution_rejects_bad_minimum():
    m = inputs.channel_mesh(8, 6, seed=1)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 1, ppe=4)
    for bad in (0, 65):
        with pytest.raises(capi.PdfError):
            pg.pdf_redistribute(gp, gm, bad, seed=1, step=0)
    assert pg.pdf_redistribute(gp, gm, 4, seed=1, step=0) == 0
