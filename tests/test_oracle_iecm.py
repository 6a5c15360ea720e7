"""The oracle's velocity-conditioned scalar mean for the IECM model (eq.
IECM; the sort-and-divide binning of the section on conditional statistics
and its appendix), pinned by special cases and invariants."""
import numpy as np

import oracle


def _state(elem, u, v, w, ps):
    return {"elem": np.asarray(elem, dtype=np.int32), "u": np.asarray(u, float), "v": np.asarray(v, float),
            "w": np.asarray(w, float), "ps": np.asarray(ps, float)}


def _random_state(n_tri=40, seed=0):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 60, n_tri)
    elem = np.repeat(np.arange(n_tri), counts)
    rng.shuffle(elem)
    n = len(elem)
    return _state(elem, rng.normal(size=n), rng.normal(size=n), rng.normal(size=n), rng.uniform(size=n))


def test_single_bin_is_the_element_mean():
    st = _random_state()
    cond = oracle.iecm_cond(40, st, bins=(1, 1, 1))
    for e in range(40):
        sel = st["elem"] == e
        if sel.any():
            assert np.allclose(cond[sel], st["ps"][sel].mean(), rtol=0, atol=1e-15)


def test_conditioning_preserves_the_element_mean():
    st = _random_state(seed=1)
    for bins in ((2, 2, 2), (5, 5, 5), (4, 12, 5), (3, 1, 7)):
        cond = oracle.iecm_cond(40, st, bins=bins)
        s_c = np.bincount(st["elem"], weights=cond, minlength=40)
        s_p = np.bincount(st["elem"], weights=st["ps"], minlength=40)
        assert np.allclose(s_c, s_p, rtol=1e-13, atol=1e-13)


def test_one_dimensional_bins_are_equal_count_runs_in_U():
    rng = np.random.default_rng(2)
    for n, k in ((10, 3), (37, 5), (100, 5), (8, 8)):
        u = rng.normal(size=n)
        st = _state(np.zeros(n), u, rng.normal(size=n), rng.normal(size=n), np.arange(n, dtype=float))
        cond = oracle.iecm_cond(1, st, bins=(k, 1, 1), m_min=1)
        order = np.argsort(u)
        kk = min(k, n)
        expect_bin = (kk * np.arange(n)) // n            # the appendix's index, in U order
        for j in range(kk):
            members = order[expect_bin == j]
            assert np.allclose(cond[members], members.mean())


def test_five_particles_with_125_bins_use_two_groups():
    # the example of the conditional-statistics section: 5 particles, a
    # (5x5x5) structure and at least 2 particles per subgroup -> two groups
    u = np.array([0.3, -1.0, 2.0, 0.1, -0.5])
    ps = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    st = _state(np.zeros(5), u, np.zeros(5), np.zeros(5), ps)
    cond = oracle.iecm_cond(1, st, bins=(5, 5, 5), m_min=2)
    low = [1, 4, 3]   # the three smallest U (floor(2 i / 5) = 0 for i = 0, 1, 2)
    high = [0, 2]
    assert np.allclose(cond[low], ps[low].mean()) and np.allclose(cond[high], ps[high].mean())


def test_cube_corners_are_divided_by_U_then_V():
    # 8 particles at the corners of a velocity cube, (2x2x2), m_min = 2: the
    # U halves hold 4, the V halves of those hold 2, which cannot be divided
    # by W any more; with m_min = 1 every particle is its own bin
    rng = np.random.default_rng(3)
    corners = np.array([[a, b, c] for a in (-1, 1) for b in (-1, 1) for c in (-1, 1)], dtype=float)
    corners += 1e-3 * rng.normal(size=corners.shape)
    perm = rng.permutation(8)
    uvw = corners[perm]
    ps = rng.uniform(size=8)
    st = _state(np.zeros(8), uvw[:, 0], uvw[:, 1], uvw[:, 2], ps)
    cond = oracle.iecm_cond(1, st, bins=(2, 2, 2), m_min=2)
    for a in (-1, 1):
        for b in (-1, 1):
            sel = (np.sign(uvw[:, 0]) == a) & (np.sign(uvw[:, 1]) == b)
            assert sel.sum() == 2 and np.allclose(cond[sel], ps[sel].mean())
    assert np.allclose(oracle.iecm_cond(1, st, bins=(2, 2, 2), m_min=1), ps)


def test_ties_are_ordered_by_particle_id():
    # equal U (e.g. after a no-slip reset): the lower particle id comes first;
    # 5 particles in 2 bins of 3 and 2
    u = np.zeros(5)
    ps = np.array([0.0, 1.0, 2.0, 3.0, 4.0])
    st = _state(np.zeros(5), u, np.zeros(5), np.zeros(5), ps)
    cond = oracle.iecm_cond(1, st, bins=(2, 1, 1), m_min=1)
    assert np.allclose(cond, [1.0, 1.0, 1.0, 3.5, 3.5])
    pid = np.array([4, 3, 2, 1, 0], dtype=np.int32)
    cond = oracle.iecm_cond(1, st, bins=(2, 1, 1), m_min=1, pid=pid)
    assert np.allclose(cond, [0.5, 0.5, 3.0, 3.0, 3.0])


def test_iecm_step_relaxes_towards_the_conditional_mean():
    # frozen particles (zero rows apart from <phi> and dt/t_m): the IECM step
    # moves each psi by (cond - psi) dt / t_m exactly as eq. IECM says
    import inputs
    m = inputs.channel_mesh(6, 5, seed=1)
    M = oracle.Mesh(m)
    counts = np.full(M.n_tri, 12, dtype=np.int32)
    st = oracle.init(M, counts, 3, u_sigma=0.5, elem_psi0=np.linspace(0, 1, M.n_tri))
    rng = np.random.default_rng(4)
    st["ps"] = rng.uniform(size=len(st["ps"]))
    cond = oracle.iecm_cond(M.n_tri, st, bins=(3, 2, 1))
    rows = np.zeros((M.n_tri, 26))
    rows[:, 22] = 1.0
    rows[:, 25] = 4.0          # 1 / t_m
    P = oracle.make_params(dt=1e-2, nu=0.0, closure="slm", pressure="none")
    ps0 = st["ps"].copy()
    st["u"][:] = 0.0; st["v"][:] = 0.0; st["w"][:] = 0.0
    oracle.step(M, rows, P, 1, 0, st, cond=cond)
    assert np.allclose(st["ps"], ps0 - (ps0 - cond) * 1e-2 * 4.0, rtol=0, atol=1e-15)
