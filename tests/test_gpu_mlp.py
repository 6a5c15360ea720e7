"""The learned warm start's kernels against the CPU oracle: forward values,
loss and gradients (BF16 rounding points reproduced by the oracle), and that
training reduces the loss."""
import numpy as np
import pytest

import oracle.mlp as OM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1006_0720_gb300 as pg  # noqa: E402


def _flat(P):
    return np.concatenate([P["W0"].ravel(), P["b0"], P["W1"].ravel(), P["b1"], P["W2"].ravel(), P["b2"],
                           P["W3"].ravel(), P["b3"]]).astype(np.float32)


def _unflat(f):
    P, o = {}, 0
    for l, (n, k) in enumerate(((64, 11), (64, 64), (64, 64), (9, 64))):
        P["W%d" % l] = f[o:o + n * k].reshape(n, k).astype(np.float64)
        o += n * k
        P["b%d" % l] = f[o:o + n].astype(np.float64)
        o += n
    return P


def _identity_norm():
    nrm = np.zeros(64, dtype=np.float32)
    nrm[16:32] = 1.0
    nrm[48:64] = 1.0
    return nrm


def _random_params(seed):
    rng = np.random.default_rng(seed)
    P = OM.init_params(seed)
    for l in range(4):
        P["b%d" % l] = rng.normal(size=P["b%d" % l].shape) * 0.1
    # parameters exactly representable in FP32 so both sides start equal
    return _unflat(_flat(P))


def test_forward_matches_the_oracle():
    P = _random_params(1)
    net = pg.Mlp(0)
    rng = np.random.default_rng(2)
    mean_in = rng.normal(size=11).astype(np.float32)
    std_in = rng.uniform(0.5, 2, 11).astype(np.float32)
    mean_out = rng.normal(size=9).astype(np.float32)
    std_out = rng.uniform(0.5, 2, 9).astype(np.float32)
    nrm = np.zeros(64, dtype=np.float32)
    nrm[:11] = mean_in
    nrm[16:27] = 1.0 / std_in
    nrm[32:41] = mean_out
    nrm[48:57] = std_out
    net.set_params(_flat(P), nrm)
    X = rng.normal(size=(1000, 11)).astype(np.float32) * std_in + mean_in
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Xn = (X.astype(np.float64) - mean_in) * nrm[16:27].astype(np.float64)
    ref = OM.forward(P, Xn) * std_out + mean_out
    err = np.abs(Y - ref) / (np.abs(ref).max())
    assert err.max() < 2e-3, err.max()
    assert np.median(err) < 1e-5


def test_gradients_match_the_oracle():
    P = _random_params(3)
    net = pg.Mlp(0)
    net.set_params(_flat(P), _identity_norm())
    rng = np.random.default_rng(4)
    n = 300  # not a multiple of the 64-row blocks
    X = rng.normal(size=(n, 11)).astype(np.float32)
    Yt = rng.normal(size=(n, 9)).astype(np.float32)
    loss, g = net.grad(torch.from_numpy(X).cuda(), torch.from_numpy(Yt).cuda())
    g = g.cpu().numpy().astype(np.float64)
    ref_loss, G = OM.loss_and_grads(P, X.astype(np.float64), Yt.astype(np.float64))
    ref = _flat({k: G[k] for k in G}).astype(np.float64)
    assert abs(loss - ref_loss) < 1e-4 * ref_loss
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < 5e-3, rel
    # every layer's gradient points the same way
    for name in ("W0", "W1", "W2", "W3"):
        a = _unflat(g.astype(np.float32))[name].ravel()
        b = G[name].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cos > 0.9999, (name, cos)


def test_training_reduces_the_loss():
    rng = np.random.default_rng(5)
    n = 4096
    X = rng.normal(size=(n, 11)).astype(np.float32)
    W = rng.normal(size=(11, 9)).astype(np.float32) * 0.5
    Yt = np.tanh(X @ W).astype(np.float32) + 0.1 * X[:, :9] ** 2
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Yt).cuda()
    net = pg.Mlp(7)
    net.fit_norm(Xd, Yd)
    first = net.train_step(Xd, Yd, 3e-3, want_loss=True)
    for _ in range(300):
        net.train_step(Xd, Yd, 3e-3)
    last = net.grad(Xd, Yd)[0]
    assert last < 0.1 * first, (first, last)


def test_learned_warm_start_beats_a_cold_start(capsys):
    """Train briefly on solves of the small channel, then on a later state of
    the same run compare CG iterations: the network's guess needs fewer
    iterations than a zero guess with the paper's Jacobi preconditioner.
    The previous-step start (the paper's warm start, the judge of the
    learned one) is printed beside them, not asserted: no learned start has
    beaten it (the quantified negative result is in the design notes)."""
    from paper_1006_0720_gb300 import experiments as E
    X, Y = E.collect_solves(120)
    net, _ = E.train(X, Y, steps=600, batch=4096, lr=3e-3)
    cfg, gm, gp, p, wp = E.setup("channel_20x40_ppe50", seed=5)
    E.advance(gm, gp, p, wp, 40)
    res = E.compare(gm, gp, p, wp, net, multigrid=False)
    with capsys.disabled():
        print("\nJacobi-PCG iterations to 1e-10 (max over 9 components / total):",
              ", ".join("%s %d / %d" % (k, res[k]["iterations_max"], res[k]["iterations_total"])
                        for k in ("zero", "previous", "local", "mlp")))
    assert res["mlp"]["iterations_total"] < res["zero"]["iterations_total"], res
    assert res["mlp"]["rel_res_max"] <= 1e-10 and res["zero"]["rel_res_max"] <= 1e-10
