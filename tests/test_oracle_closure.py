"""Pins of the oracle's closure at the nodes: the kinetic-energy constraint
(eq. constraint-on-c0) that eq. GandC is built to satisfy, the SLM special
case, hand-evaluated special cases of the elliptic-relaxation right-hand
side (eqs. elliptic-relaxation-Lagrangian, H, A_v, bij), and the model
constants printed in the paper."""
import math
import os

import numpy as np
import pytest

import inputs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "model_constants.txt")


def _golden_constants():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_oracle_constants_match_the_printed_table():
    assert oracle.constants() == _golden_constants()


def _stats(rng, k_scale=1.0):
    A = rng.normal(size=(3, 3))
    R = k_scale * (A @ A.T / 3.0 + 0.05 * np.eye(3))  # symmetric positive definite
    S = np.zeros(oracle.NNS)
    S[0:3] = rng.normal(size=3)
    S[3] = rng.uniform(0.5, 2.0)      # <omega>
    S[4] = rng.uniform(0, 1)          # <phi>
    S[5:11] = [R[0, 0], R[1, 1], R[2, 2], R[0, 1], R[0, 2], R[1, 2]]
    S[11] = 0.01
    D = np.zeros(oracle.NND)
    D[0:6] = rng.normal(size=6)
    D[6:10] = rng.normal(size=4)
    return S, D, R


def _eps(S, nu, closure):
    k = 0.5 * (S[5] + S[6] + S[7])
    if closure == "slm":
        return k * S[3]
    # eq. dissipation-from-frequency_wall
    return S[3] * (k + nu * 36.0 * S[3])


@pytest.mark.parametrize("closure", ["glm", "slm"])
def test_kinetic_energy_constraint_holds(closure):
    rng = np.random.default_rng(0)
    P = oracle.make_params(dt=1e-3, nu=1e-3, Pi=0.0, closure=closure)
    for _ in range(50):
        S, D, R = _stats(rng)
        # a wp whose C0 stays positive: a negative-definite part dominates
        B = rng.normal(size=(3, 3))
        wp = -2.0 * np.eye(3) + 0.3 * B
        c = oracle.node_coeff(S, D, wp.ravel(), P)
        G = c[12:21].reshape(3, 3)
        eps = _eps(S, 1e-3, closure)
        C0 = c[21] ** 2 / eps
        resid = (1.0 + 1.5 * C0) * eps + np.sum(G * R)
        assert abs(resid) < 1e-12 * (1 + eps + np.abs(G).max()), resid
        if closure == "slm":
            assert math.isclose(C0, 3.5, rel_tol=1e-13)
            assert np.allclose(G, -(0.5 + 0.75 * 3.5) * S[3] * np.eye(3), rtol=1e-14)


def test_local_wp_is_the_relaxation_right_hand_side():
    rng = np.random.default_rng(1)
    P = oracle.make_params(dt=1e-3, nu=1e-3, closure="glm")
    S, D, R = _stats(rng)
    rhs = oracle.relax_rhs(S, D)
    assert np.allclose(oracle.node_coeff(S, D, None, P), oracle.node_coeff(S, D, rhs, P), rtol=0, atol=0)


def test_relax_rhs_isotropic_simple_shear_closed_form():
    """Isotropic stresses R = 2k/3 I give b = 0 and A_v = min(1, C_v) = 1, so
    with a single gradient dU/dy = s the right-hand side is, by hand from
    eq. H: rhs_ii = (1-C1)/2 k<w>, rhs_12 = k (C2 + g5/3) s,
    rhs_21 = -k g5/3 s, all others 0."""
    k, om, s = 0.6, 1.7, 2.5
    S = np.zeros(oracle.NNS)
    S[3] = om
    S[5:8] = 2.0 * k / 3.0
    D = np.zeros(oracle.NND)
    D[1] = s  # dU/dy
    rhs = oracle.relax_rhs(S, D).reshape(3, 3)
    C1, C2, g5 = 1.85, 0.63, 0.1
    ref = np.zeros((3, 3))
    for i in range(3):
        ref[i, i] = 0.5 * (1 - C1) * k * om
    ref[0, 1] = k * (C2 + g5 / 3.0) * s
    ref[1, 0] = -k * g5 / 3.0 * s
    assert np.allclose(rhs, ref, rtol=1e-14, atol=1e-15)


def test_relax_rhs_anisotropic_av_below_one():
    """A strongly anisotropic (two-component-limit-like) stress gives
    det R small, A_v = C_v det R / (2k/3)^3 < 1; with dU/dx = s only:
    rhs_11 = (1-C1)/2 k<w> + k s (C2 A_v + g5/3 - g5/3 + g5 b11 - g5 b11)."""
    R = np.diag([1.0, 0.02, 0.5])
    k = 0.5 * np.trace(R)
    om, s = 1.0, 0.7
    S = np.zeros(oracle.NNS)
    S[3] = om
    S[5:8] = np.diag(R)
    D = np.zeros(oracle.NND)
    D[0] = s
    Av = 1.4 * np.linalg.det(R) / (2 * k / 3) ** 3
    assert Av < 1.0
    rhs = oracle.relax_rhs(S, D).reshape(3, 3)
    assert math.isclose(rhs[0, 0], 0.5 * (1 - 1.85) * k * om + k * s * 0.63 * Av, rel_tol=1e-13)
    assert math.isclose(rhs[1, 1], 0.5 * (1 - 1.85) * k * om, rel_tol=1e-13)


def test_frequency_source_and_mixing_time_special_cases():
    P = oracle.make_params(dt=1e-3, nu=1e-3, closure="glm")
    S = np.zeros(oracle.NNS)
    S[3] = 2.0
    S[5:8] = [0.1, 0.1, 0.1]
    D = np.zeros(oracle.NND)
    c = oracle.node_coeff(S, D, None, P)
    assert c[23] == 0.73                     # no production: S_omega = C_omega2
    k = 0.15
    eps = 2.0 * (k + 1e-3 * 36.0 * 2.0)      # eq. dissipation-from-frequency_wall
    tm = max(k / eps, 6.0 * math.sqrt(1e-3 / eps))
    assert math.isclose(c[25], 1.0 / tm, rel_tol=1e-14)
    Pc = oracle.make_params(dt=1e-3, nu=1e-3, closure="glm", tm_mode="cphi", c_phi=2.0)
    assert oracle.node_coeff(S, D, None, Pc)[25] == 2.0  # 1/t_m = C_phi <omega> / 2


def test_element_rows_average_nodal_coefficients():
    """Constant nodal statistics give identical rows everywhere; the rows are
    the mean of the three nodal coefficient sets (loop (ii))."""
    m = inputs.channel_mesh(6, 5, seed=2)
    M = oracle.Mesh(m)
    P = oracle.make_params(dt=1e-3, nu=1e-3, Pi=2e-3, closure="glm")
    rng = np.random.default_rng(3)
    S, D, R = _stats(rng)
    ns = np.tile(S, (M.n_nodes, 1))
    nd = np.tile(D, (M.n_nodes, 1))
    rows = oracle.elem_coeff(M, ns, nd, P)
    ref = oracle.node_coeff(S, D, None, P)
    assert np.allclose(rows, ref[None, :], rtol=1e-14, atol=1e-15)
    # varying nodal stats: row = mean of the element's three node coefficient sets
    ns = ns + 0.01 * rng.normal(size=ns.shape)
    ns[:, 5:8] = np.abs(ns[:, 5:8])
    rows = oracle.elem_coeff(M, ns, nd, P)
    for e in (0, 7, 13):
        t = M.tri[e]
        ref = np.mean([oracle.node_coeff(ns[n], nd[n], None, P) for n in t], axis=0)
        assert np.allclose(rows[e], ref, rtol=1e-13, atol=1e-15)
