"""Pins of the oracle's particle time step against closed forms of the
discretised SDEs (frozen coefficients):

* Ornstein-Uhlenbeck velocity: stationary variance and lag autocorrelation of
  the Euler-Maruyama AR(1) recursion; the redistribution toy problem of
  sec. 3.6 (alpha = 0.5 -> <u_i u_j> = delta_ij);
* Taylor dispersion of the position driven by the OU velocity (ch. 4,
  eq. ms-particle-displacement) in its discrete form;
* frequency SDE (eq. frequency-model) with constant <omega>: mean relaxation
  and the stationary Gamma variance C4 <omega>^2;
* IEM mixing (eq. IEM) with the element's own mean: scalar mean preserved,
  variance ratio exactly (1 - dt/t_m)^2 per step, exp(-C_phi <omega> t) decay;
* SLM energy decay per step E[k'] = k (1 - <omega> dt + a^2 dt^2);
* conservation: particle count and host-element validity every step;
* the terms the OU pins leave at zero: the velocity-gradient noise equals
  the mean-velocity gradient times the particle's own diffusive displacement
  (one shared dW_j); a non-symmetric G_ij against the matrix power
  (I + G dt)^N and expm(G t); a constant drift a_i and the position advanced
  with the time-n velocity; S_omega by an exact one-step difference and the
  stationary mean C3 <omega> / (C3 + S_omega).
"""
import math

import numpy as np
import pytest

import inputs
import oracle


@pytest.fixture(scope="module")
def chan():
    m = inputs.channel_mesh(12, 9, seed=4)
    return m, oracle.Mesh(m)


def _frozen_rows(M, a=0.0, b=0.0, om=1.0, phi=0.0, inv_tm=0.0, mean=(0.0, 0.0, 0.0), drift=(0, 0, 0)):
    rows = np.zeros((M.n_tri, oracle.NCOEF))
    rows[:, 0:3] = mean
    rows[:, 9:12] = drift
    rows[:, 12] = rows[:, 16] = rows[:, 20] = -a
    rows[:, 21] = b
    rows[:, 22] = om
    rows[:, 23] = 0.0
    rows[:, 24] = phi
    rows[:, 25] = inv_tm
    return rows


def _particles_in_band(M, n, rng, ylo=-0.5, yhi=0.5):
    x = rng.uniform(0.05, 2 * math.pi - 0.05, n)
    y = rng.uniform(ylo, yhi, n)
    st = {"x": x, "y": y, "u": np.zeros(n), "v": np.zeros(n), "w": np.zeros(n),
          "om": np.ones(n), "ps": np.zeros(n)}
    st["elem"] = np.array([M.locate_brute(xi, yi) for xi, yi in zip(x, y)], dtype=np.int32)
    assert np.all(st["elem"] >= 0)
    return st


def test_ou_stationary_variance_and_autocorrelation(chan):
    m, M = chan
    rng = np.random.default_rng(0)
    n, dt, a = 20000, 1e-3, 10.0
    var_inf = 1e-4
    b = math.sqrt(2 * a * var_inf)
    rows = _frozen_rows(M, a=a, b=b)
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng)
    rho = 1.0 - a * dt
    disc_inf = b * b * dt / (1.0 - rho * rho)
    for s in range(600):
        oracle.step(M, rows, P, 1, s, st)
    u0 = st["u"].copy()
    for comp in ("u", "v", "w"):
        var = st[comp].var()
        assert abs(var / disc_inf - 1.0) < 5 * math.sqrt(2.0 / n), (comp, var, disc_inf)
    lag = 50
    for s in range(600, 600 + lag):
        oracle.step(M, rows, P, 1, s, st)
    corr = np.mean(u0 * st["u"]) / disc_inf
    assert abs(corr - rho ** lag) < 5 / math.sqrt(n), (corr, rho ** lag)
    # counts conserved and every particle inside its host element
    assert len(st["elem"]) == n
    for p in range(0, n, 97):
        assert np.all(M.subareas(st["elem"][p], st["x"][p], st["y"][p]) >= 0)


def test_redistribution_toy_problem_steady_state(chan):
    """dU = -(U - alpha <U>) dt + sqrt(2) dW with <U> = 0: <u_i u_j> -> delta_ij
    (sec. 3.6); the Euler-Maruyama recursion gives 2 dt / (1 - (1-dt)^2)."""
    m, M = chan
    rng = np.random.default_rng(1)
    n, dt = 10000, 1e-2
    rows = _frozen_rows(M, a=1.0, b=math.sqrt(2.0))
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng, -0.01, 0.01)
    st["u"] = rng.normal(size=n)
    st["v"] = rng.normal(size=n)
    st["w"] = rng.normal(size=n)
    for s in range(400):
        oracle.step(M, rows, P, 7, s, st)
    U = np.stack([st["u"], st["v"], st["w"]])
    C = U @ U.T / n
    target = 2 * dt / (1 - (1 - dt) ** 2)
    assert np.allclose(np.diag(C), target, atol=5 * target * math.sqrt(2.0 / n))
    assert np.all(np.abs(C[~np.eye(3, dtype=bool)]) < 5 / math.sqrt(n))


def test_taylor_dispersion_discrete(chan):
    """Stationary OU velocity, position X += U dt: E[(X_N - X_0)^2] =
    dt^2 var [N + 2 sum_k (N-k) rho^k]; its continuum limit is
    2 var T_L^2 (t/T_L - 1 + exp(-t/T_L)) with T_L = 1/a."""
    m, M = chan
    rng = np.random.default_rng(2)
    n, dt, a, var = 20000, 1e-3, 20.0, 0.01
    rho = 1 - a * dt
    b = math.sqrt(var * (1 - rho * rho) / dt)  # exactly stationary discrete variance
    rows = _frozen_rows(M, a=a, b=b)
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng, -0.3, 0.3)
    st["u"] = rng.normal(size=n) * math.sqrt(var)
    st["v"] = rng.normal(size=n) * math.sqrt(var)
    y0 = st["y"].copy()
    N = 200
    for s in range(N):
        oracle.step(M, rows, P, 3, s, st)
    d2 = np.mean((st["y"] - y0) ** 2)
    ref = dt * dt * var * (N + 2 * sum((N - k) * rho ** k for k in range(1, N)))
    assert abs(d2 / ref - 1) < 5 * math.sqrt(2.0 / n), (d2, ref)
    t, TL = N * dt, 1 / a
    cont = 2 * var * TL * TL * (t / TL - 1 + math.exp(-t / TL))
    assert abs(ref / cont - 1) < 0.05


def test_frequency_relaxation_and_gamma_variance(chan):
    m, M = chan
    rng = np.random.default_rng(3)
    n, dt, mo = 20000, 1e-3, 1.0
    rows = _frozen_rows(M, om=mo)
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng)
    st["om"][:] = 2.0
    C3, C4 = 5.0, 0.25
    for s in range(100):
        oracle.step(M, rows, P, 11, s, st)
    mean_ref = mo + (2.0 - mo) * (1 - C3 * mo * dt) ** 100
    sd = math.sqrt(st["om"].var() / n)
    assert abs(st["om"].mean() - mean_ref) < 5 * sd + 1e-12
    for s in range(100, 1500):
        oracle.step(M, rows, P, 11, s, st)
    # stationary variance of the recursion: 2 C3 C4 <w>^3 dt / (1 - (1 - C3 <w> dt)^2)
    r = 1 - C3 * mo * dt
    var_ref = 2 * C3 * C4 * mo ** 3 * dt / (1 - r * r)
    assert abs(st["om"].mean() - mo) < 5 * math.sqrt(var_ref / n)
    assert abs(st["om"].var() / var_ref - 1) < 5 * math.sqrt(2 * (1 + 3 * C4) / n)
    assert np.all(st["om"] >= 0)


def test_iem_mean_preserved_and_variance_ratio_exact(chan):
    m, M = chan
    rng = np.random.default_rng(4)
    n, dt = 6000, 1e-3
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng)
    st["ps"] = rng.uniform(0, 1, n)
    c_phi, om = 2.0, 3.0
    inv_tm = 0.5 * c_phi * om
    for s in range(50):
        es = oracle.elem_stats(M.n_tri, st)
        rows = _frozen_rows(M, om=om, inv_tm=inv_tm)
        rows[:, 24] = es[:, 5]  # the element's own particle mean of psi
        var0 = es[:, 12].copy()
        mean0 = es[:, 5].copy()
        oracle.step(M, rows, P, 5, s, st)
        es1 = oracle.elem_stats(M.n_tri, st)
        occ = es[:, 0] > 1
        assert np.array_equal(es1[:, 0], es[:, 0])  # frozen particles stay
        assert np.allclose(es1[occ, 5], mean0[occ], rtol=0, atol=1e-15)
        ratio = (1 - dt * inv_tm) ** 2
        assert np.allclose(es1[occ, 12], ratio * var0[occ], rtol=1e-12, atol=1e-18)
    # 50 steps of ratio r: exp(-C_phi <w> t) within O(dt)
    t = 50 * dt
    tot = (1 - dt * inv_tm) ** 100
    # log-ratio is -N (dt/t_m)^2 + O(N (dt/t_m)^3)
    assert abs(tot / math.exp(-c_phi * om * t) - 1) < 2 * 50 * (dt * inv_tm) ** 2


def test_slm_energy_decay_one_step(chan):
    m, M = chan
    rng = np.random.default_rng(5)
    n, dt, om = 40000, 1e-2, 2.0
    C0 = 3.5
    a = (0.5 + 0.75 * C0) * om
    st = _particles_in_band(M, n, rng, -0.2, 0.2)
    for c in ("u", "v", "w"):
        st[c] = rng.normal(size=n) * 0.1
    k = 0.5 * sum(np.mean(st[c] ** 2) for c in ("u", "v", "w"))
    eps = k * om
    rows = _frozen_rows(M, a=a, b=math.sqrt(C0 * eps), om=om)
    P = oracle.make_params(dt=dt, nu=0.0, closure="slm", pressure="none")
    oracle.step(M, rows, P, 9, 0, st)
    k1 = 0.5 * sum(np.mean(st[c] ** 2) for c in ("u", "v", "w"))
    ref = k * (1 - om * dt + a * a * dt * dt)
    assert abs(k1 / ref - 1) < 5 * math.sqrt(2.0 / (3 * n))


# ---------------------------------------------------------------------------
# Terms of the velocity and frequency updates that the OU pins above leave
# at zero: the velocity-gradient noise (and its sharing of dW_j with the
# position), a full non-symmetric G_ij, the drift a_i, and S_omega.
# ---------------------------------------------------------------------------
def _wrap(d, period):
    """Periodic displacement in (-period/2, period/2]."""
    return d - period * np.round(d / period)


def test_velocity_gradient_noise_is_the_position_noise(chan):
    """eq. velocity-prediction with U^n = <U> = 0, G = 0, a = 0, C0 eps = 0:
    U_i^{n+1} = sqrt(2 nu) d<U_i>/dx_j dW_j, and the position moves by
    sqrt(2 nu) dW_j with the same dW_j (eq. Lagrangian-position-exact), so
    particle by particle U_i^{n+1} = d<U_i>/dx_j (X_j^{n+1} - X_j^n): a uniform
    shear of the mean field carries each particle's velocity along with its
    diffusive displacement.  Distinct gradient entries make any index swap,
    and any noise not shared with the position, visible."""
    m, M = chan
    rng = np.random.default_rng(21)
    n, dt, nu = 4000, 1e-3, 1e-3
    grad = np.array([1.5, -2.25, 3.0, 0.75, -1.25, 2.5])  # dU/dx dU/dy dV/dx dV/dy dW/dx dW/dy
    rows = _frozen_rows(M)
    rows[:, 3:9] = grad
    P = oracle.make_params(dt=dt, nu=nu, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng, -0.5, 0.5)
    x0, y0 = st["x"].copy(), st["y"].copy()
    cnt, _ = oracle.step(M, rows, P, 13, 4, st)
    assert cnt["reflections"] == 0
    dx = _wrap(st["x"] - x0, M.period)
    dy = st["y"] - y0
    # the displacement is the diffusion alone: variance 2 nu dt per axis
    for d in (dx, dy):
        assert abs(d.var() / (2 * nu * dt) - 1) < 5 * math.sqrt(2.0 / n)
    for i, comp in enumerate(("u", "v", "w")):
        ref = grad[2 * i] * dx + grad[2 * i + 1] * dy
        assert np.allclose(st[comp], ref, rtol=0, atol=1e-13), comp
    assert np.array_equal(st["om"] > 0, np.ones(n, dtype=bool))


def test_nonsymmetric_relaxation_tensor_matrix_power(chan):
    """With nu = 0, C0 eps = 0 and a = 0 the velocity recursion is linear:
    U^{n+1} - <U> = (I + G dt)(U^n - <U>), so after N steps U^N - <U> =
    (I + G dt)^N (U^0 - <U>) to rounding (the matrix power by numpy), and
    within O(N dt^2 |G|^2) of the continuum solution expm(G t) (U^0 - <U>)
    (scipy).  G is non-symmetric, so a transposed G_ij fails."""
    linalg = pytest.importorskip("scipy.linalg")
    m, M = chan
    rng = np.random.default_rng(22)
    n, dt, N = 500, 1e-3, 200
    G = np.array([[-2.0, 1.5, 0.3],
                  [-0.7, -1.0, 0.4],
                  [0.2, -0.5, -3.0]])
    mean = np.array([0.3, -0.2, 0.1])
    rows = _frozen_rows(M, mean=tuple(mean))
    rows[:, 12:21] = G.reshape(-1)
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng, -0.3, 0.3)
    U0 = np.stack([rng.normal(0.3, 0.2, n), rng.normal(0.0, 0.2, n), rng.normal(0.0, 0.2, n)])
    st["u"], st["v"], st["w"] = U0[0].copy(), U0[1].copy(), U0[2].copy()
    for s in range(N):
        cnt, _ = oracle.step(M, rows, P, 17, s, st)
        assert cnt["reflections"] == 0
    UN = np.stack([st["u"], st["v"], st["w"]])
    dev0 = U0 - mean[:, None]
    ref = np.linalg.matrix_power(np.eye(3) + G * dt, N) @ dev0 + mean[:, None]
    assert np.allclose(UN, ref, rtol=1e-12, atol=1e-14)
    cont = linalg.expm(G * N * dt) @ dev0 + mean[:, None]
    bound = N * dt * dt * np.linalg.norm(G, 2) ** 2 * np.abs(dev0).max()
    assert np.abs(UN - cont).max() < bound
    # the transposed tensor is a different trajectory, far outside that bound
    wrong = np.linalg.matrix_power(np.eye(3) + G.T * dt, N) @ dev0 + mean[:, None]
    assert np.abs(UN - wrong).max() > 10 * bound


def test_constant_drift_and_position_uses_time_n_velocity(chan):
    """Drift alone (G = 0, C0 eps = 0, nu = 0): U^N = U^0 + N a dt per
    component, and the position, advanced with the time-n velocity
    (Euler-Maruyama, eq. Lagrangian-position-exact), moves by
    N U^0 dt + a dt^2 N (N - 1) / 2 (with U^{n+1} it would be N (N + 1) / 2)."""
    m, M = chan
    rng = np.random.default_rng(23)
    n, dt, N = 400, 1e-3, 100
    a = np.array([0.5, -1.25, 2.0])
    rows = _frozen_rows(M, mean=(0.7, -0.4, 0.9), drift=tuple(a))
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng, -0.3, 0.3)
    U0 = np.stack([rng.normal(0.5, 0.2, n), rng.normal(0.0, 0.2, n), rng.normal(0.0, 0.2, n)])
    st["u"], st["v"], st["w"] = U0[0].copy(), U0[1].copy(), U0[2].copy()
    x0, y0 = st["x"].copy(), st["y"].copy()
    for s in range(N):
        cnt, _ = oracle.step(M, rows, P, 19, s, st)
        assert cnt["reflections"] == 0
    for i, comp in enumerate(("u", "v", "w")):
        assert np.allclose(st[comp], U0[i] + N * a[i] * dt, rtol=0, atol=1e-13), comp
    tri = dt * dt * N * (N - 1) / 2
    assert np.allclose(_wrap(st["x"] - x0, M.period), N * U0[0] * dt + a[0] * tri, rtol=0, atol=1e-13)
    assert np.allclose(st["y"] - y0, N * U0[1] * dt + a[1] * tri, rtol=0, atol=1e-13)
    # the U^{n+1} reading differs by a dt^2 N, far above rounding
    assert abs(a[1]) * dt * dt * N > 1e-8


def test_frequency_source_term(chan):
    """eq. frequency-model with eq. frequency-source's S_omega.  One step from
    the same state and draws with S_omega = s and with S_omega = 0 differs by
    exactly -s <omega> omega dt (the noise does not involve S_omega).  Over
    many steps the mean obeys m' = (1 - (C3 + S_omega) <omega> dt) m
    + C3 <omega>^2 dt, whose fixed point C3 <omega> / (C3 + S_omega) the
    ensemble reaches (5 sigma)."""
    m, M = chan
    rng = np.random.default_rng(24)
    n, dt, mo, s_om = 20000, 2e-3, 1.5, 2.0
    C3, C4 = 5.0, 0.25
    P = oracle.make_params(dt=dt, nu=0.0, closure="glm", pressure="none")
    st = _particles_in_band(M, n, rng)
    st["om"] = rng.uniform(0.5, 2.0, n)
    rows0 = _frozen_rows(M, om=mo)
    rows1 = rows0.copy()
    rows1[:, 23] = s_om
    a, b = {k: v.copy() for k, v in st.items()}, {k: v.copy() for k, v in st.items()}
    oracle.step(M, rows0, P, 29, 0, a)
    oracle.step(M, rows1, P, 29, 0, b)
    assert np.allclose(b["om"] - a["om"], -s_om * mo * st["om"] * dt, rtol=1e-9, atol=1e-15)
    # stationary mean with the source term
    N = 800
    for s in range(N):
        oracle.step(M, rows1, P, 31, s, st)
    r = 1 - (C3 + s_om) * mo * dt
    m_star = C3 * mo * mo * dt / (1 - r)
    assert abs(m_star - C3 * mo / (C3 + s_om)) < 1e-15
    m0 = 1.25  # the initial uniform mean
    ref = m_star + (m0 - m_star) * r ** N
    se = math.sqrt(st["om"].var() / n)
    assert abs(st["om"].mean() - ref) < 5 * se, (st["om"].mean(), ref, se)
    # without the source term the fixed point is <omega>: far outside 5 sigma
    assert abs(mo - ref) > 50 * se
