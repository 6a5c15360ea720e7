"""Pins of the oracle's particle redistribution (App. D; the basic idea in
App. C and sec. 3.6) by its invariants: the total is kept; every critical
element reaches the minimum from the donor at its mirror position in the
count order; moved particles copy the critical element's particles in turn
(or, into an empty element, keep their values and land inside it); donors
give their lowest-id particles; nothing moves when no element is critical;
and the redistribution toy problem of sec. 3.6 keeps <u_i u_j> = delta_ij."""
import math

import numpy as np

import inputs
import oracle

KEYS = ("x", "y", "u", "v", "w", "om", "ps")


def _state(M, counts, seed=3):
    st = oracle.init(M, np.asarray(counts, dtype=np.int32), seed, u_sigma=0.5)
    st["ps"] = np.random.default_rng(seed).random(len(st["x"]))
    return st


def _mesh():
    m = inputs.channel_mesh(8, 6, seed=2)
    return m, oracle.Mesh(m)


def test_counts_reach_the_minimum_and_the_total_is_kept():
    m, M = _mesh()
    rng = np.random.default_rng(5)
    counts = rng.integers(0, 20, size=M.n_tri)
    counts[[3, 7, 11]] = [0, 1, 2]
    st = _state(M, counts)
    before = {k: v.copy() for k, v in st.items()}
    order = sorted(range(M.n_tri), key=lambda e: (counts[e], e))
    mn = 6
    moved = oracle.redistribute(M, st, mn, seed=9, step=4)
    after = np.bincount(st["elem"], minlength=M.n_tri)
    assert after.sum() == counts.sum()
    crit = [e for e in order if counts[e] < mn]
    expect = counts.copy()
    for k, j in enumerate(crit):
        i = order[M.n_tri - 1 - k]
        d = min(mn - counts[j], counts[i])
        expect[j] += d
        expect[i] -= d
    assert np.array_equal(after, expect)
    assert moved == int(np.abs(after - counts).sum() // 2)
    assert np.all(after[crit] >= mn)
    # every particle sits inside its (possibly new) element
    for p in range(len(st["x"])):
        assert np.all(M.subareas(st["elem"][p], st["x"][p], st["y"][p]) >= -1e-12)
    # donors gave their lowest particle ids (pid = index here)
    changed = np.nonzero(st["elem"] != before["elem"])[0]
    for k, j in enumerate(crit):
        i = order[M.n_tri - 1 - k]
        mine = np.nonzero(before["elem"] == i)[0]
        d = min(mn - counts[j], counts[i])
        assert set(mine[:d]) <= set(changed) and not (set(mine[d:]) & set(changed))


def test_moved_particles_copy_the_critical_elements_particles_in_turn():
    m, M = _mesh()
    counts = np.full(M.n_tri, 10)
    counts[0], counts[5] = 2, 0
    st = _state(M, counts)
    before = {k: v.copy() for k, v in st.items()}
    oracle.redistribute(M, st, 5, seed=1, step=0)
    order = sorted(range(M.n_tri), key=lambda e: (counts[e], e))
    assert order[:2] == [5, 0]
    # element 0 (2 particles) received 3, copies of its particles 0, 1, 0
    donor = order[M.n_tri - 2]
    own = np.nonzero(before["elem"] == 0)[0]
    gave = np.nonzero(before["elem"] == donor)[0][:3]
    for q, pi in enumerate(gave):
        src = own[q % 2]
        for k in KEYS:
            assert st[k][pi] == before[k][src]
        assert st["elem"][pi] == 0
    # element 5 (empty) received 5 particles that keep U, omega, psi and lie in it
    donor = order[M.n_tri - 1]
    gave = np.nonzero(before["elem"] == donor)[0][:5]
    for pi in gave:
        for k in ("u", "v", "w", "om", "ps"):
            assert st[k][pi] == before[k][pi]
        assert st["elem"][pi] == 5
        assert M.locate_brute(st["x"][pi], st["y"][pi]) == 5
    assert len({(st["x"][pi], st["y"][pi]) for pi in gave}) == 5


def test_nothing_moves_above_the_minimum():
    m, M = _mesh()
    st = _state(M, np.full(M.n_tri, 4))
    before = {k: v.copy() for k, v in st.items()}
    assert oracle.redistribute(M, st, 4, seed=1, step=0) == 0
    for k in KEYS + ("elem",):
        assert np.array_equal(st[k], before[k])


def test_redistribution_toy_problem_keeps_the_steady_state():
    """Sec. 3.6: dU = -(U - alpha <U>) dt + sqrt(2) dW with <U> = 0 held
    (the toy problem's trivial mean), particles started in a band so that
    the elements outside it start empty and are filled by the
    redistribution, which keeps intervening as the particles spread; the
    stationary <u_i u_j> of the Euler-Maruyama recursion, 2 dt / (1 - (1 -
    dt)^2) on the diagonal, is kept within the statistical error."""
    m = inputs.channel_mesh(10, 8, seed=4)
    M = oracle.Mesh(m)
    rng = np.random.default_rng(11)
    counts = np.zeros(M.n_tri, dtype=np.int32)
    band = [e for e in range(M.n_tri) if abs(M.xy[M.tri[e]].mean(axis=0)[1]) < 0.3]
    counts[band] = 120
    st = oracle.init(M, counts, 6, u_profile="zero", u_sigma=1.0)
    n, dt = len(st["x"]), 1e-2
    rows = np.zeros((M.n_tri, oracle.NCOEF))
    rows[:, 12] = rows[:, 16] = rows[:, 20] = -1.0
    rows[:, 21] = math.sqrt(2.0)
    rows[:, 22] = 1.0
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    moved = 0
    for s in range(300):
        oracle.step(M, rows, P, 7, s, st)
        moved += oracle.redistribute(M, st, 8, seed=7, step=s)
    assert moved > 1000
    assert np.bincount(st["elem"], minlength=M.n_tri).min() >= 8
    U = np.stack([st["u"], st["v"], st["w"]])
    C = U @ U.T / n
    target = 2 * dt / (1 - (1 - dt) ** 2)
    assert np.allclose(np.diag(C), target, atol=6 * target * math.sqrt(2.0 / n))
    assert np.all(np.abs(C[~np.eye(3, dtype=bool)]) < 6 / math.sqrt(n))
