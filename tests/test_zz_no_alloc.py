"""pdf_estimate_stats_noalloc: the statistics entry point for callers that
cannot allocate device memory (for example a host loop that must not take
the synchronization cudaMalloc/cudaFree may cause, or code whose device
memory is owned by another allocator).  It uses a fixed scratch array
compiled into the library instead of allocated buffers.

Called through the C-ABI twice in a row, its statistics must equal those of
pdf_estimate_stats on the same particle state; so must the IECM conditioned
means it computes from the grouping in its scratch array, on a mesh large
enough for two radix passes and on one small enough (fewer than 512
elements) for a single pass.  Sizes beyond the scratch array are refused.
This file is collected last so that a failure here does not stop the other
tests from running.
"""
import ctypes

import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU only
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402
from paper_1006_0720_gb300 import capi  # noqa: E402
from parity_util import assert_field_close  # noqa: E402


def _run(mesh_nx, mesh_ny, counts_fn, steps):
    m = inputs.channel_mesh(mesh_nx, mesh_ny, seed=4)
    gm = pg.Mesh(m)
    counts = counts_fn(gm.n_tri)
    gp = pg.Particles(gm, 3, count=counts, u_sigma=0.1, elem_psi0=inputs.scalar_slab(m))
    p = pg.model_params(closure="glm")
    pg.pdf_estimate_stats(gp, gm)
    for s in range(steps):  # scatter the particles so the grouping has work to do
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    return gm, gp


def _outputs(gm):
    return (torch.empty((gm.n_tri, capi.PDF_NES), dtype=torch.float64, device="cuda"),
            torch.empty((gm.n_nodes, capi.PDF_NNS), dtype=torch.float64, device="cuda"),
            torch.empty((gm.n_nodes, capi.PDF_NND), dtype=torch.float64, device="cuda"))


def test_noalloc_statistics_match_the_allocating_entry_point_twice():
    rng = np.random.default_rng(11)
    gm, gp = _run(20, 40, lambda nt: rng.integers(0, 60, nt).astype(np.int32), 5)
    ref = _outputs(gm)
    pg.pdf_estimate_stats(gp, gm, *ref)
    ref = [t.cpu().numpy() for t in ref]
    L = pg.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = _outputs(gm)
        st = L.pdf_estimate_stats_noalloc(gp.handle, gm.handle, *[ctypes.c_void_p(t.data_ptr()) for t in out],
                                          stream)
        assert st == capi.PDF_OK, pg.pdf_last_error()
        torch.cuda.synchronize()
        got = [t.cpu().numpy() for t in out]
        assert np.array_equal(got[0][:, 0], ref[0][:, 0]), "element counts, call %d" % call
        for g, r, what in zip(got, ref, ("element stats", "node stats", "node derivatives")):
            assert_field_close(g, r, "%s, call %d" % (what, call))


@pytest.mark.parametrize("nx,ny", [(20, 40), (8, 12)])
def test_noalloc_iecm_means_match_the_allocating_entry_point(nx, ny):
    """IECM conditioning runs on the segment offsets and sorted order that
    the allocation-free call leaves in its scratch array.  (8, 12): 154
    elements, a single radix pass."""
    m = inputs.channel_mesh(nx, ny, seed=4)
    gm = pg.Mesh(m)
    rng = np.random.default_rng(12)
    counts = rng.integers(0, 70, gm.n_tri).astype(np.int32)
    gp = pg.Particles(gm, 3, count=counts, u_sigma=0.1, elem_psi0=inputs.scalar_slab(m))
    gp.set_iecm((3, 3, 2))
    p = pg.model_params(closure="glm", mix="iecm")
    pg.pdf_estimate_stats(gp, gm)
    for s in range(3):
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    ref_es = _outputs(gm)[0]
    pg.pdf_estimate_stats(gp, gm, ref_es)
    ref_cond = gp.iecm_cond().cpu().numpy()
    ref_es = ref_es.cpu().numpy()
    L = pg.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        es = _outputs(gm)[0]
        st = L.pdf_estimate_stats_noalloc(gp.handle, gm.handle, ctypes.c_void_p(es.data_ptr()), None, None, stream)
        assert st == capi.PDF_OK, pg.pdf_last_error()
        torch.cuda.synchronize()
        assert_field_close(es.cpu().numpy(), ref_es, "element stats, call %d" % call)
        cond = gp.iecm_cond().cpu().numpy()
        assert_field_close(cond, ref_cond, "IECM conditioned means, call %d" % call)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    """A mesh with more elements than the scratch array holds is refused
    (the element check comes first, so a few particles suffice)."""
    m = inputs.channel_mesh(400, 400, seed=4)
    gm = pg.Mesh(m)
    assert gm.n_tri > capi.PDF_NOALLOC_MAX_ELEMENTS
    counts = np.zeros(gm.n_tri, dtype=np.int32)
    counts[::1000] = 1
    gp = pg.Particles(gm, 3, count=counts, u_sigma=0.1)
    assert gp.n <= capi.PDF_NOALLOC_MAX_PARTICLES
    st = pg.lib().pdf_estimate_stats_noalloc(gp.handle, gm.handle, None, None, None, None)
    assert st == capi.PDF_EINVAL
    assert "elements exceed the limit" in pg.pdf_last_error()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    m = inputs.channel_mesh(20, 40, seed=4)
    gm = pg.Mesh(m)
    n_tri = gm.n_tri
    ppe = capi.PDF_NOALLOC_MAX_PARTICLES // n_tri + 1
    gp = pg.Particles(gm, 3, ppe=ppe, u_sigma=0.1)
    assert gp.n > capi.PDF_NOALLOC_MAX_PARTICLES
    st = pg.lib().pdf_estimate_stats_noalloc(gp.handle, gm.handle, None, None, None, None)
    assert st == capi.PDF_EINVAL
    assert "exceed the limit" in pg.pdf_last_error()
