"""State transfers through the C-ABI with every kind of caller buffer:
device memory, page-locked host memory (read and written by the kernels
through its mapping) and pageable host memory (through the staging
buffer) give the same values, before and after a reordering of the state
(slots then differ from particle ids), in both state forms."""
import ctypes

import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402
from paper_1006_0720_gb300 import capi  # noqa: E402

KEYS = ("x", "y", "u", "v", "w", "om", "ps")


def _bufs(kind, n):
    if kind == "device":
        b = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in KEYS}
        b["elem"] = torch.empty(n, dtype=torch.int32, device="cuda")
    elif kind == "pinned":
        b = {k: torch.empty(n, dtype=torch.float64, pin_memory=True) for k in KEYS}
        b["elem"] = torch.empty(n, dtype=torch.int32, pin_memory=True)
    else:
        b = {k: torch.from_numpy(np.empty(n)) for k in KEYS}
        b["elem"] = torch.from_numpy(np.empty(n, dtype=np.int32))
    return b


def _ptrs(b):
    return [ctypes.c_void_p(b[k].data_ptr()) for k in KEYS + ("elem",)]


def _get(gp, kind):
    b = _bufs(kind, gp.n)
    capi.check(pg.lib().pdf_particles_get_state(gp.handle, *_ptrs(b), None), "get_state")
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().copy() for k, v in b.items()}


@pytest.mark.parametrize("precision", [capi.PDF_FP64, capi.PDF_FP32_STATE])
def test_state_round_trips_with_every_buffer_kind(precision):
    m = inputs.channel_mesh(20, 40, seed=1)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 3, ppe=30, u_sigma=0.2, elem_psi0=inputs.scalar_slab(m), precision=precision)
    gp.set_reorder(1)
    p = pg.model_params(closure="slm")
    pg.pdf_estimate_stats(gp, gm)
    for s in range(4):                      # moves particles; the reordering permutes the slots
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    ref = _get(gp, "device")
    for kind in ("pinned", "pageable"):
        got = _get(gp, kind)
        for k in KEYS + ("elem",):
            assert np.array_equal(got[k], ref[k]), (kind, k)
    # set from each kind, read back on the device: the same state
    for kind in ("pinned", "pageable", "device"):
        b = _bufs(kind, gp.n)
        for k in KEYS + ("elem",):
            b[k].copy_(torch.from_numpy(ref[k]))
        capi.check(pg.lib().pdf_particles_set_state(gp.handle, *_ptrs(b), None), "set_state")
        back = _get(gp, "device")
        for k in KEYS + ("elem",):
            assert np.array_equal(back[k], ref[k]), (kind, k)
    # positions out of range are refused from every kind
    for kind in ("pinned", "pageable"):
        b = _bufs(kind, gp.n)
        for k in KEYS + ("elem",):
            b[k].copy_(torch.from_numpy(ref[k]))
        b["x"][5] = 100.0
        with pytest.raises(capi.PdfError):
            capi.check(pg.lib().pdf_particles_set_state(gp.handle, *_ptrs(b), None), "set_state")


def _pinned_copy(st):
    out = {}
    for k, v in st.items():
        h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
        h.copy_(v)
        out[k] = h
    return out


@pytest.mark.parametrize("precision", [capi.PDF_FP64, capi.PDF_FP32_STATE])
def test_step_host_matches_set_step_get(precision):
    """pdf_step_host (chunked loads, steps and stores of a page-locked host
    state) gives, bit for bit, the state and the statistics of
    set_state + pdf_step + get_state, over several steps with the state
    reordered by every statistics call in between."""
    m = inputs.channel_mesh(50, 100, seed=2)
    gm = pg.Mesh(m)
    psi = inputs.scalar_slab(m)
    a = pg.Particles(gm, 6, ppe=30, u_sigma=0.2, elem_psi0=psi, precision=precision)
    b = pg.Particles(gm, 6, ppe=30, u_sigma=0.2, elem_psi0=psi, precision=precision)
    assert a.n > 4 * 65536   # several chunks
    for q in (a, b):
        q.set_reorder(1)
        pg.pdf_estimate_stats(q, gm)
    p = pg.model_params(closure="slm")
    host_a = _pinned_copy(a.get_state())
    dev_b = b.get_state()
    ea = torch.empty((gm.n_tri, capi.PDF_NES), dtype=torch.float64, device="cuda")
    eb = torch.empty_like(ea)
    for s in range(3):
        ia = pg.pdf_step_host(a, gm, p, host_a, step=s, info=True)
        b.set_state(dev_b)
        ib = pg.pdf_step(b, gm, p, step=s, info=True)
        dev_b = b.get_state()
        torch.cuda.synchronize()
        for k in KEYS + ("elem",):
            assert torch.equal(host_a[k], dev_b[k].cpu()), (s, k)
        assert ia == ib
        pg.pdf_estimate_stats(a, gm, ea)
        pg.pdf_estimate_stats(b, gm, eb)
        assert torch.equal(ea, eb), s
    # the device copy holds the stepped state too
    da = a.get_state()
    for k in KEYS + ("elem",):
        assert torch.equal(da[k].cpu(), host_a[k]), k


def test_step_host_stats_matches_step_host_then_statistics():
    """pdf_step_host_stats gives, bit for bit, the state of pdf_step_host and
    the statistics (element, node, derivatives) of a following
    pdf_estimate_stats, into device and page-locked host outputs, over
    several steps that include reorderings of the device state."""
    m = inputs.channel_mesh(50, 100, seed=3)
    gm = pg.Mesh(m)
    psi = inputs.scalar_slab(m)
    a = pg.Particles(gm, 8, ppe=30, u_sigma=0.2, elem_psi0=psi)
    b = pg.Particles(gm, 8, ppe=30, u_sigma=0.2, elem_psi0=psi)
    for q in (a, b):
        q.set_reorder(2)
        pg.pdf_estimate_stats(q, gm)
    p = pg.model_params(closure="glm")
    host_a = _pinned_copy(a.get_state())
    host_b = _pinned_copy(b.get_state())
    shapes = {"e": (gm.n_tri, capi.PDF_NES), "n": (gm.n_nodes, capi.PDF_NNS), "d": (gm.n_nodes, capi.PDF_NND)}
    out_a = {k: torch.empty(v, dtype=torch.float64, pin_memory=True) for k, v in shapes.items()}
    out_b = {k: torch.empty(v, dtype=torch.float64, device="cuda") for k, v in shapes.items()}
    for s in range(4):
        ia = pg.pdf_step_host_stats(a, gm, p, host_a, out_a["e"], out_a["n"], out_a["d"], step=s, info=True)
        ib = pg.pdf_step_host(b, gm, p, host_b, step=s, info=True)
        pg.pdf_estimate_stats(b, gm, out_b["e"], out_b["n"], out_b["d"])
        torch.cuda.synchronize()
        assert ia == ib
        for k in KEYS + ("elem",):
            assert torch.equal(host_a[k], host_b[k]), (s, k)
        for k in shapes:
            assert torch.equal(out_a[k], out_b[k].cpu()), (s, k)


def test_step_host_rejects_pageable_buffers_and_iecm():
    m = inputs.channel_mesh(8, 6, seed=1)
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, 1, ppe=4)
    pg.pdf_estimate_stats(gp, gm)
    p = pg.model_params(closure="slm")
    st = _pinned_copy(gp.get_state())
    pageable = {k: v.clone() for k, v in st.items()}
    args = [ctypes.c_void_p(pageable[k].data_ptr()) for k in KEYS + ("elem",)]
    rc = pg.lib().pdf_step_host(gp.handle, gm.handle, ctypes.byref(p), None, None, 0, *args, None, None)
    assert rc == capi.PDF_EINVAL
    gp.set_iecm((2, 2, 2), 2)
    pg.pdf_estimate_stats(gp, gm)
    pi = pg.model_params(closure="slm", mix="iecm")
    with pytest.raises(capi.PdfError):
        pg.pdf_step_host(gp, gm, pi, st, step=0)
    pg.pdf_step_host(gp, gm, p, st, step=0)   # the plain model still runs
    # the conditioned means belonged to the old slot order: IECM waits for
    # the next statistics
    with pytest.raises(capi.PdfError):
        pg.pdf_step(gp, gm, pi, step=1)
    pg.pdf_estimate_stats(gp, gm)
    pg.pdf_step(gp, gm, pi, step=1)
