"""The synthetic workloads: sizes, step counts and run parameters.

Values, not arithmetic.  Each entry names what it is; the mesh itself comes
from inputs.channel.  Model constants (C1, C2, ...) are not here: the library
and the oracle each carry the paper's table themselves.
"""
import math

CHANNEL_COMMON = dict(
    jitter=0.2,
    seed=1,
    dt=1e-3,
    nu=1e-3,           # Re ~ 1000 on centreline velocity and half width
    Pi=2e-3,           # imposed -d<P>/dx = 2*nu: laminar balance of U = 1 - y^2
    u_profile="parabola",  # initial mean U(y) = 1 - y^2
    u_sigma=0.1,       # N(0, 0.1^2) fluctuations on every component
    omega_init="gamma4",   # Gamma(k=4, theta=0.25): mean 1, variance 1/4
    psi_slab_x=0.5,    # psi = 1 in elements touching x = 0.5
    closure="glm",
)

CONFIGS = {
    # small case: the oracle finishes it in seconds
    "channel_20x40_ppe50": dict(CHANNEL_COMMON, nx=20, ny=40, ppe=50, steps=100),
    # the measured workload: ~16M particles on ~160k triangles
    "channel_200x400_ppe100": dict(CHANNEL_COMMON, nx=200, ny=400, ppe=100, steps=1000),
    # the same mesh with fewer particles (3.2M, state 200 MB > L2): profiler captures
    "channel_200x400_ppe20": dict(CHANNEL_COMMON, nx=200, ny=400, ppe=20, steps=1000),
    # a quarter of the mesh at the measured density (3.9M particles, state 240 MB
    # > L2): profiler captures of per-element work that depends on the density
    "channel_100x200_ppe100": dict(CHANNEL_COMMON, nx=100, ny=200, ppe=100, steps=1000),
}

# Complex geometry: 20 x 5 domain, obstacles 1x1, 1x2, 0.5x1.5 on the bottom
# wall, graded triangulation (535,720 triangles, 50:1 spacing), particles per
# element proportional to its area with mean 128 (68.6M), a point source of
# scalar at (2, 0.5) of radius 0.05 with the source-dependent micromixing
# time, periodic inflow/outflow re-injecting clean fluid, FP32 velocity /
# frequency / scalar state with FP64 positions.  Closure: the simplified
# Langevin model (eq. wall-GandC): with counts proportional to area the
# smallest wall elements hold a few particles, k -> 0 there and the GLM's
# G = (wp - eps/2)/k is unbounded without particle redistribution.
OBSTACLES = {
    "obstacles_20x5_mean128": dict(mesh="obstacles", h_min=0.0025, ratio=37.0, growth=1.04, mean_ppe=128,
                                   steps=2000, seed=1, dt=1e-3, nu=1e-3, Pi=2e-2, u_profile="uniform",
                                   u_sigma=0.1, closure="slm", tm_mode="source", src=(2.0, 0.5, 0.05),
                                   precision="fp32_state"),
    # a small version for parity tests
    "obstacles_small_mean20": dict(mesh="obstacles", h_min=0.05, ratio=6.0, growth=1.3, mean_ppe=20,
                                   steps=30, seed=1, dt=2e-3, nu=1e-3, Pi=2e-2, u_profile="uniform",
                                   u_sigma=0.1, closure="slm", tm_mode="source", src=(2.0, 0.5, 0.05),
                                   precision="fp64"),
}


def workload(name):
    cfg = dict(CONFIGS[name])
    cfg["name"] = name
    cfg["n_tri"] = 2 * (cfg["nx"] - 1) * (cfg["ny"] - 1)
    cfg["n_particles"] = cfg["n_tri"] * cfg["ppe"]
    cfg["period"] = 2.0 * math.pi
    return cfg
