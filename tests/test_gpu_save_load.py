"""pdf_particles_save / pdf_particles_load through the C-ABI: a set saved
mid-run (after a reordering of its slots, with the statistics and, in one
case, the IECM conditioned means it carries) and loaded into a new handle
continues bit for bit like the original, in both state forms; saving the
loaded set gives the same bytes; corrupted, truncated and foreign buffers
are refused with PDF_EINVAL before anything reaches the device."""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402
from paper_1006_0720_gb300 import capi  # noqa: E402


def _stats(gp, gm):
    es = torch.empty((gm.n_tri, capi.PDF_NES), dtype=torch.float64, device="cuda")
    ns = torch.empty((gm.n_nodes, capi.PDF_NNS), dtype=torch.float64, device="cuda")
    pg.pdf_estimate_stats(gp, gm, es, ns)
    return es, ns


@pytest.mark.parametrize("precision,iecm", [(capi.PDF_FP64, False), (capi.PDF_FP32_STATE, False),
                                            (capi.PDF_FP64, True)])
def test_saved_set_continues_bit_for_bit(precision, iecm):
    m = inputs.channel_mesh(20, 40, seed=1)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 5, ppe=30, u_sigma=0.1, elem_psi0=inputs.scalar_slab(m), precision=precision)
    gp.set_reorder(3)
    if iecm:
        gp.set_iecm((3, 3, 2))
    p = pg.model_params(closure="glm", mix="iecm" if iecm else "iem")
    pg.pdf_estimate_stats(gp, gm)
    for s in range(5):   # a reordering of the slots at the third call
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    buf = gp.save()
    assert buf[:7].tobytes() == b"PDFGBPS"
    gq = pg.Particles.load(gm, buf)
    assert gq.n == gp.n
    assert np.array_equal(gq.save(), buf)
    if iecm:
        assert torch.equal(gp.iecm_cond(), gq.iecm_cond())
    for s in range(5, 12):   # two more reorderings on both, at the same calls
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_step(gq, gm, p, step=s)
        a, b = _stats(gp, gm), _stats(gq, gm)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), "statistics after step %d" % s
    sa, sb = gp.get_state(), gq.get_state()
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    assert np.array_equal(gp.save(), gq.save())


def test_load_refuses_bad_buffers():
    m = inputs.channel_mesh(20, 40, seed=1)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 5, ppe=10, u_sigma=0.1)
    pg.pdf_estimate_stats(gp, gm)
    buf = gp.save()

    def refused(b, mesh=gm, what=""):
        with pytest.raises(pg.PdfError) as ei:
            pg.Particles.load(mesh, b)
        assert ei.value.status == capi.PDF_EINVAL
        assert what in str(ei.value), str(ei.value)

    bad = buf.copy()
    bad[len(buf) // 2] ^= 1
    refused(bad, what="checksum")
    refused(buf[:-8], what="size")
    bad = buf.copy()
    bad[0] = ord("X")
    refused(bad, what="not a saved particle set")
    bad = buf.copy()
    bad[8] = 99   # version
    refused(bad, what="version")
    other = pg.Mesh(inputs.channel_mesh(12, 9, seed=4))
    refused(buf, mesh=other, what="another size")
    refused(buf[:40], what="too small")
    # the original is untouched and still loads
    pg.Particles.load(gm, buf)
