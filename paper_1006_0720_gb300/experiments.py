"""The learned warm start experiment (argument marshalling and orchestration
only: every computation runs in libpdfgb's kernels).

collect_solves  run the small channel with the elliptic-relaxation solve each
                step and keep (node features, wp - rhs) pairs: the network
                learns the correction that the elliptic term makes to the
                local model wp = rhs;
train           fit the per-node MLP on them with the library's Adam steps
                (batches drawn by the library's Philox gather);
compare         on a given state, solve from four initial guesses -- zero,
                the previous step's solution (the paper's warm start, sec.
                3.2), the local model rhs and rhs plus the network's
                correction -- to the same residual and report iterations
                and times.
"""
import time

import numpy as np
import torch

import inputs

from . import api as A


def setup(workload, seed=1, arith="fx"):
    cfg = inputs.workload(workload)
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], jitter=cfg["jitter"], seed=cfg["seed"])
    gm = A.Mesh(m)
    gp = A.Particles(gm, seed, ppe=cfg["ppe"], u_sigma=cfg["u_sigma"],
                     elem_psi0=inputs.scalar_slab(m, cfg["psi_slab_x"]))
    p = A.model_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure="glm", arith=arith)
    A.pdf_estimate_stats(gp, gm)
    wp = torch.zeros((9, gm.n_nodes), dtype=torch.float64, device="cuda")
    return cfg, gm, gp, p, wp


def advance(gm, gp, p, wp, steps, step0=0, rtol=1e-10, max_it=5000, collect=False):
    """Steps of the whole method with the relaxation solved every step (warm
    start from the previous solution).  Returns per-step iteration counts
    and, with collect, the (features, wp - rhs) pairs of every solve."""
    its, Xs, Ys = [], [], []
    for s in range(steps):
        it, _ = A.pdf_relax_solve_particles(gp, gm, p, wp, rtol=rtol, max_it=max_it)
        its.append(max(it))
        if collect:
            X, Y = A.pdf_mlp_features(gp, gm, p, wp)
            Xs.append(X)
            Ys.append(Y)
        A.pdf_step(gp, gm, p, wp=wp, step=step0 + s)
        A.pdf_estimate_stats(gp, gm)
    if collect:
        return its, torch.cat(Xs), torch.cat(Ys)
    return its


def collect_solves(n_solves, workload="channel_20x40_ppe50", seed=1, rtol=1e-10):
    cfg, gm, gp, p, wp = setup(workload, seed)
    Xs, Ys = [], []
    for s in range(n_solves):
        A.pdf_relax_solve_particles(gp, gm, p, wp, rtol=rtol, max_it=5000)
        X, Y = A.pdf_mlp_features(gp, gm, p, wp)
        Xs.append(X)
        Ys.append(Y)
        A.pdf_step(gp, gm, p, wp=wp, step=s)
        A.pdf_estimate_stats(gp, gm)
    return torch.cat(Xs), torch.cat(Ys)


def train(X, Y, steps=3000, batch=8192, lr=2e-3, seed=0, log_every=0):
    net = A.Mlp(seed)
    net.fit_norm(X, Y)
    Xb = torch.empty((batch, X.shape[1]), dtype=torch.float32, device="cuda")
    Yb = torch.empty((batch, Y.shape[1]), dtype=torch.float32, device="cuda")
    losses = []
    for s in range(steps):
        A.pdf_mlp_batch(X, Y, seed, s, batch, Xb, Yb)
        lr_s = lr * (0.5 * (1 + np.cos(np.pi * s / steps)))  # cosine decay
        want = log_every and (s % log_every == 0 or s == steps - 1)
        loss = net.train_step(Xb, Yb, lr_s, want_loss=bool(want))
        if want:
            losses.append((s, loss))
    return net, losses


def compare(gm, gp, p, wp_prev, net, rtol=1e-10, max_it=20000, multigrid=True):
    """Iterations and times to rtol from zero, from the previous solution and
    from the network's guess (each from its own copy), with the multigrid or
    the Jacobi preconditioner (the choice is restored to multigrid after)."""
    A.pdf_relax_set_solver(gp, multigrid)
    try:
        return _compare(gm, gp, p, wp_prev, net, rtol, max_it)
    finally:
        A.pdf_relax_set_solver(gp, True)


def _compare(gm, gp, p, wp_prev, net, rtol, max_it):
    out = {}
    for name in ("zero", "previous", "local", "mlp"):
        if name == "zero":
            w = torch.zeros_like(wp_prev)
        elif name == "previous":
            w = wp_prev.clone()
        else:
            w = torch.empty_like(wp_prev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if name == "local":
            rhs, _ = A.pdf_relax_rhs(gp, gm, p)
            w.copy_(rhs)
        elif name == "mlp":
            net.guess(gp, gm, p, w)
        it, res = A.pdf_relax_solve_particles(gp, gm, p, w, rtol=rtol, max_it=max_it)
        torch.cuda.synchronize()
        out[name] = {"iterations_max": max(it), "iterations_total": sum(it),
                     "seconds": time.perf_counter() - t0, "rel_res_max": max(res)}
    return out
