"""The precision form (PDF_FP32_STATE): velocity, frequency and scalar stored
and advanced in FP32, positions and the element search FP64-accurate,
statistics exact integer sums.  Compared with the FP64 oracle: the initial
state is the oracle's rounded to FP32, and after 100 steps of the small
channel every statistic stays within a stated bound of the oracle's."""
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


def test_fp32_state_statistics_after_100_steps():
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
    for s in range(100):
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
    names = ["U", "V", "W", "omega", "phi", "uu", "vv", "ww", "uv", "uw", "vw", "phiphi"]
    print("max scaled error per element statistic:", dict(zip(names, np.round(e_el, 9))))
    print("max scaled error per node statistic:", dict(zip(names, np.round(e_nd, 9))))
    moved = np.mean(ges[:, 0] != es[:, 0])
    print("fraction of elements whose particle count differs:", moved)
    assert e_nd.max() < 1e-3
    assert moved < 0.02
