"""Whole oracle runs for the GPU tests' ensembles, importable by spawned
worker processes (numpy, inputs and the oracle only; no GPU)."""
import numpy as np

import inputs
import oracle


def domain_statistics(st):
    """Domain means and (co)variances of a particle state: U, V, W, omega,
    phi, uu, vv, ww, uv, phiphi."""
    u, v, w = st["u"], st["v"], st["w"]
    return np.array([u.mean(), v.mean(), w.mean(), st["om"].mean(), st["ps"].mean(), u.var(), v.var(), w.var(),
                     np.mean((u - u.mean()) * (v - v.mean())), st["ps"].var()])


def robust_statistics(st):
    """Medians of U, V, W, omega, phi and the interquartile ranges of U, V,
    W: statistics of the particle distribution that a few runaway
    particles cannot move."""
    med = [np.median(st[k]) for k in ("u", "v", "w", "om", "ps")]
    iqr = [np.subtract(*np.percentile(st[k], [75, 25])) for k in ("u", "v", "w")]
    return np.array(med + iqr)


def channel_domain_after(seed, steps, workload="channel_20x40_ppe50"):
    """The oracle's run of a channel workload from `seed` (GLM closure, the
    channel's imposed pressure gradient): the domain statistics after
    `steps` steps (domain_statistics, then robust_statistics)."""
    cfg = inputs.workload(workload)
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], seed=1)
    M = oracle.Mesh(m)
    counts = np.full(cfg["n_tri"], cfg["ppe"], dtype=np.int32)
    st = oracle.init(M, counts, seed, u_sigma=cfg["u_sigma"], elem_psi0=inputs.scalar_slab(m))
    po = oracle.make_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure="glm", pressure="channel")
    es, ns, nd, _ = oracle.statistics(M, st)
    for s in range(steps):
        oracle.step(M, oracle.elem_coeff(M, ns, nd, po), po, seed, s, st)
        es, ns, nd, _ = oracle.statistics(M, st, ns)
    return np.concatenate([domain_statistics(st), robust_statistics(st)])
