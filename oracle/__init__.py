"""CPU oracle (TEST INFRASTRUCTURE ONLY).

A plain, slow, single-threaded FP64 implementation of the particle time step,
written from the paper, used to check the CUDA library.  Only the tests, the
smoke check in ``__graft_entry__`` and the benchmark's CPU-baseline leg may
import it.  It shares no code with the CUDA library.

The arithmetic lives in ``pdf_oracle.c`` (compiled here with gcc); this module
only marshals numpy arrays.  Every function here has pins of its own in
``tests/test_oracle_*.py``; what no pin fixes is the composition of many
steps (the paper prints no worked trajectory): parity unpinned there,
covered by agreement with the GPU and by invariants.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NES = 13   # element stats: N, U, V, W, omega, phi, uu, vv, ww, uv, uw, vw, phiphi
NNS = 12   # node stats: the same without N
NND = 10   # node derivatives: dU/dx dU/dy dV/dx dV/dy dW/dx dW/dy lapU lapV lapW d<vv>/dy
NCOEF = 26

CLOSURE = {"glm": 0, "slm": 1}
TM_MODE = {"turb": 0, "cphi": 1, "source": 2}
PRESSURE = {"none": 0, "channel": 1, "projection": 2, "projection_inout": 3}

TRK_FALLBACK, TRK_BRUTE, TRK_LOST, TRK_EXIT_OUT, TRK_EXIT_IN, TRK_REINJECT, TRK_NEAR_FACE = 1, 2, 4, 8, 16, 32, 256
TRK_NOSLIP = 64     # the no-slip wall condition was applied


def build(force=False):
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC]
    # OpenMP only spreads the particle loop of or_step_threads over threads;
    # without it that loop runs on one thread
    if subprocess.call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL) != 0:
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("nu", ctypes.c_double), ("Pi", ctypes.c_double),
                ("c_phi", ctypes.c_double), ("closure", ctypes.c_int), ("tm_mode", ctypes.c_int),
                ("pressure", ctypes.c_int), ("src_x", ctypes.c_double), ("src_y", ctypes.c_double),
                ("src_r", ctypes.c_double)]


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


D = ctypes.c_double
I = ctypes.c_int
U32 = ctypes.c_uint32
PD = ctypes.POINTER(D)
PI = ctypes.POINTER(I)
PL = ctypes.POINTER(ctypes.c_long)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_constants.argtypes = [PD]
            L.or_philox.argtypes = [ctypes.POINTER(U32), ctypes.POINTER(U32), ctypes.POINTER(U32)]
            L.or_u01.argtypes = [U32]
            L.or_u01.restype = ctypes.c_float
            L.or_logf.argtypes = [ctypes.c_float]
            L.or_logf.restype = ctypes.c_float
            L.or_sincos2pi.argtypes = [ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_float)]
            L.or_gauss4.argtypes = [ctypes.c_uint64, U32, U32, U32, U32, ctypes.POINTER(ctypes.c_float)]
            L.or_gauss_fill.argtypes = [ctypes.c_uint64, ctypes.c_long, U32, U32, U32,
                                        ctypes.POINTER(ctypes.c_float)]
            L.or_mesh_create.argtypes = [I, PD, I, PI, PI, I, PI, D]
            L.or_mesh_create.restype = ctypes.c_void_p
            L.or_mesh_free.argtypes = [ctypes.c_void_p]
            L.or_mesh_get.argtypes = [ctypes.c_void_p, PD, PI, PI]
            L.or_subareas.argtypes = [ctypes.c_void_p, I, D, D, PD]
            L.or_track.argtypes = [ctypes.c_void_p, I, PD, PD, PD, PD, ctypes.c_void_p]
            L.or_track.restype = I
            L.or_locate_brute.argtypes = [ctypes.c_void_p, D, D]
            L.or_locate_brute.restype = I
            L.or_init.argtypes = [ctypes.c_void_p, PI, ctypes.c_uint64, I, D, PD] + [PD] * 7 + [PI]
            L.or_elem_stats.argtypes = [I, ctypes.c_long, PI, PD, PD, PD, PD, PD, PD]
            L.or_node_stats.argtypes = [ctypes.c_void_p, PD, PD]
            L.or_node_stats.restype = I
            L.or_shape_derivs.argtypes = [ctypes.c_void_p, I, PD, PD]
            L.or_node_derivs.argtypes = [ctypes.c_void_p, PD, PD]
            L.or_relax_rhs.argtypes = [PD, PD, PD]
            L.or_node_coeff.argtypes = [PD, PD, PD, ctypes.POINTER(_Params), PD, PD, PD]
            L.or_elem_coeff.argtypes = [ctypes.c_void_p, PD, PD, PD, ctypes.POINTER(_Params), PD, PD]
            L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_long, PD, ctypes.POINTER(_Params),
                                  ctypes.c_uint64, U32, PD, PD, PD, PD, PD, PD, PD, PI, PI, PL, PI, PD, PD]
            L.or_step_threads.argtypes = L.or_step.argtypes + [I]
            L.or_step_threads.restype = I
            L.or_noslip_omega.argtypes = [ctypes.c_void_p, PD, PD]
            L.or_mesh_noslip.argtypes = [ctypes.c_void_p, PI, PD]
            L.or_iecm_cond.argtypes = [I, ctypes.c_long, PI, PD, PD, PD, PD, PI, I, I, I, I, PD]
            L.or_redistribute.argtypes = [ctypes.c_void_p, ctypes.c_long] + [PD] * 7 + [PI, PI, I,
                                                                                       ctypes.c_uint64, U32]
            L.or_redistribute.restype = ctypes.c_long
            _lib = L
    return _lib


def constants():
    """The model constants the oracle carries: C1, C2, C3, C4, C_T, C_L, C_eta,
    C_v, gamma5, C_omega1, C_omega2 (channel constants table) and the SLM C0."""
    c = np.zeros(12)
    lib().or_constants(_p(c, D))
    names = ["C1", "C2", "C3", "C4", "CT", "CL", "Ceta", "Cv", "gamma5", "Comega1", "Comega2", "C0_slm"]
    return dict(zip(names, c.tolist()))


# ---------------------------------------------------------------- random numbers
def philox(ctr, key):
    c = (U32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (U32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (U32 * 4)()
    lib().or_philox(c, k, o)
    return [int(v) for v in o]


def u01(word):
    return lib().or_u01(int(word) & 0xFFFFFFFF)


def logf(u):
    return lib().or_logf(float(u))


def sincos2pi(u):
    s, c = ctypes.c_float(), ctypes.c_float()
    lib().or_sincos2pi(float(u), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def gauss4(seed, c0, c1, c2, c3):
    g = (ctypes.c_float * 4)()
    lib().or_gauss4(int(seed), c0, c1, c2, c3, g)
    return np.array(list(g), dtype=np.float32)


def gauss_fill(seed, n, c1, c2, c3):
    out = np.zeros(4 * n, dtype=np.float32)
    lib().or_gauss_fill(int(seed), int(n), c1, c2, c3, _p(out, ctypes.c_float))
    return out.reshape(n, 4)


# ---------------------------------------------------------------- mesh
class Mesh:
    def __init__(self, mesh):
        xy = np.ascontiguousarray(mesh["xy"], dtype=np.float64)
        tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
        twin = np.ascontiguousarray(mesh.get("twin", np.full(len(xy), -1)), dtype=np.int32)
        bnd = np.ascontiguousarray(mesh["bnd"], dtype=np.int32)
        self.n_nodes, self.n_tri = len(xy), len(tri)
        self.xy, self.tri = xy, tri
        self.period = float(mesh.get("period", 0.0))
        h = lib().or_mesh_create(self.n_nodes, _p(xy, D), self.n_tri, _p(tri, I), _p(twin, I),
                                 len(bnd), _p(bnd, I), self.period)
        if not h:
            raise ValueError("oracle: inconsistent mesh")
        self._h = h
        self.area = np.zeros(self.n_tri)
        self.nbr = np.zeros((self.n_tri, 3), dtype=np.int32)
        self.shift = np.zeros((self.n_tri, 3), dtype=np.int32)
        lib().or_mesh_get(h, _p(self.area, D), _p(self.nbr, I), _p(self.shift, I))
        self.noslip_flag = np.zeros(self.n_tri, dtype=np.int32)
        self.noslip_line = np.zeros((self.n_tri, 4))
        lib().or_mesh_noslip(h, _p(self.noslip_flag, I), _p(self.noslip_line, D))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_mesh_free(self._h)
            self._h = None

    def subareas(self, e, x, y):
        N = np.zeros(3)
        lib().or_subareas(self._h, int(e), float(x), float(y), _p(N, D))
        return N

    def shape_derivs(self, e):
        a, b = np.zeros(3), np.zeros(3)
        lib().or_shape_derivs(self._h, int(e), _p(a, D), _p(b, D))
        return a, b

    def track(self, e0, x, y, u=0.0, v=0.0):
        """Returns (element, x, y, u, v, info dict)."""
        X, Y, Uu, Vv = D(x), D(y), D(u), D(v)

        class Info(ctypes.Structure):
            _fields_ = [("walk_steps", I), ("reflections", I), ("crossings_periodic", I),
                        ("status", I), ("min_rel", D)]
        info = Info()
        e = lib().or_track(self._h, int(e0), ctypes.byref(X), ctypes.byref(Y), ctypes.byref(Uu),
                           ctypes.byref(Vv), ctypes.byref(info))
        return e, X.value, Y.value, Uu.value, Vv.value, {
            "walk_steps": info.walk_steps, "reflections": info.reflections,
            "crossings_periodic": info.crossings_periodic, "status": info.status,
            "min_rel": info.min_rel}

    def locate_brute(self, x, y):
        return lib().or_locate_brute(self._h, float(x), float(y))


# ---------------------------------------------------------------- particles
STATE_KEYS = ("x", "y", "u", "v", "w", "om", "ps")


U_PROFILE = {"zero": 0, "parabola": 1, "uniform": 2}


def init(mesh, counts, seed, u_profile="parabola", u_sigma=0.1, elem_psi0=None):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    n = int(counts.sum())
    st = {k: np.zeros(n) for k in STATE_KEYS}
    st["elem"] = np.zeros(n, dtype=np.int32)
    psi0 = None if elem_psi0 is None else np.ascontiguousarray(elem_psi0, dtype=np.float64)
    lib().or_init(mesh._h, _p(counts, I), int(seed), U_PROFILE[u_profile],
                  float(u_sigma), None if psi0 is None else _p(psi0, D),
                  *[_p(st[k], D) for k in STATE_KEYS], _p(st["elem"], I))
    return st


def elem_stats(n_tri, st):
    es = np.zeros((n_tri, NES))
    args = [np.ascontiguousarray(st[k], dtype=np.float64) for k in ("u", "v", "w", "om", "ps")]
    el = np.ascontiguousarray(st["elem"], dtype=np.int32)
    lib().or_elem_stats(n_tri, len(el), _p(el, I), *[_p(a, D) for a in args], _p(es, D))
    return es


def node_stats(mesh, es, prev=None):
    ns = np.zeros((mesh.n_nodes, NNS)) if prev is None else np.array(prev, dtype=np.float64)
    es = np.ascontiguousarray(es, dtype=np.float64)
    kept = lib().or_node_stats(mesh._h, _p(es, D), _p(ns, D))
    return ns, kept


def node_derivs(mesh, ns):
    nd = np.zeros((mesh.n_nodes, NND))
    ns = np.ascontiguousarray(ns, dtype=np.float64)
    lib().or_node_derivs(mesh._h, _p(ns, D), _p(nd, D))
    return nd


def make_params(dt, nu, Pi=0.0, closure="glm", tm_mode="turb", c_phi=2.0, pressure="channel",
                src=(0.0, 0.0, 0.0)):
    return _Params(dt, nu, Pi, c_phi, CLOSURE[closure], TM_MODE[tm_mode], PRESSURE[pressure],
                   float(src[0]), float(src[1]), float(src[2]))


def relax_rhs(S, Dv):
    out = np.zeros(9)
    S = np.ascontiguousarray(S, dtype=np.float64)
    Dv = np.ascontiguousarray(Dv, dtype=np.float64)
    lib().or_relax_rhs(_p(S, D), _p(Dv, D), _p(out, D))
    return out


def node_coeff(S, Dv, wp, params, xy=(0.0, 0.0), grad_p=None):
    out = np.zeros(NCOEF)
    S = np.ascontiguousarray(S, dtype=np.float64)
    Dv = np.ascontiguousarray(Dv, dtype=np.float64)
    w = None if wp is None else np.ascontiguousarray(wp, dtype=np.float64)
    P = np.ascontiguousarray(xy, dtype=np.float64)
    g = None if grad_p is None else np.ascontiguousarray(grad_p, dtype=np.float64)
    lib().or_node_coeff(_p(S, D), _p(Dv, D), None if w is None else _p(w, D),
                        ctypes.byref(params), _p(P, D), None if g is None else _p(g, D), _p(out, D))
    return out


def elem_coeff(mesh, ns, nd, params, wp=None, grad_p=None):
    """grad_p: [n_nodes, 2] nodal gradient of the projected pressure (for
    make_params(pressure="projection"))."""
    rows = np.zeros((mesh.n_tri, NCOEF))
    ns = np.ascontiguousarray(ns, dtype=np.float64)
    nd = np.ascontiguousarray(nd, dtype=np.float64)
    w = None if wp is None else np.ascontiguousarray(wp, dtype=np.float64)
    g = None if grad_p is None else np.ascontiguousarray(grad_p, dtype=np.float64)
    lib().or_elem_coeff(mesh._h, _p(ns, D), _p(nd, D), None if w is None else _p(w, D),
                        ctypes.byref(params), None if g is None else _p(g, D), _p(rows, D))
    return rows


def iecm_cond(n_tri, st, bins=(5, 5, 5), m_min=2, pid=None):
    """Velocity-conditioned scalar mean of every particle (eq. IECM) by the
    sort-and-divide binning over the particles of each element."""
    el = np.ascontiguousarray(st["elem"], dtype=np.int32)
    arrs = [np.ascontiguousarray(st[k], dtype=np.float64) for k in ("u", "v", "w", "ps")]
    pid = None if pid is None else np.ascontiguousarray(pid, dtype=np.int32)
    out = np.zeros(len(el))
    lib().or_iecm_cond(n_tri, len(el), _p(el, I), *[_p(a, D) for a in arrs],
                       None if pid is None else _p(pid, I), int(bins[0]), int(bins[1]), int(bins[2]),
                       int(m_min), _p(out, D))
    return out


def redistribute(mesh, st, min_npel, seed, step, pid=None):
    """The particle redistribution of App. D, in place; returns the number
    of particles moved."""
    for k in STATE_KEYS:
        st[k] = np.ascontiguousarray(st[k], dtype=np.float64)
    st["elem"] = np.ascontiguousarray(st["elem"], dtype=np.int32)
    pid = None if pid is None else np.ascontiguousarray(pid, dtype=np.int32)
    return int(lib().or_redistribute(mesh._h, len(st["x"]), *[_p(st[k], D) for k in STATE_KEYS],
                                     _p(st["elem"], I), None if pid is None else _p(pid, I), int(min_npel),
                                     int(seed), int(step)))


def noslip_omega(mesh, ns):
    """Per element: the mean frequency given to particles striking a no-slip
    wall (eq. frequency-wallstats); 0 away from no-slip walls."""
    out = np.zeros(mesh.n_tri)
    ns = np.ascontiguousarray(ns, dtype=np.float64)
    lib().or_noslip_omega(mesh._h, _p(ns, D), _p(out, D))
    return out


def step(mesh, rows, params, seed, step_no, st, pid=None, cond=None, omega_wall=None):
    """Advance every particle one step in place.  Returns (counters, status).
    pid: particle ids of the entries (default: their index); cond: the
    velocity-conditioned scalar means for eq. IECM (default: eq. IEM);
    omega_wall: noslip_omega() for meshes with no-slip walls."""
    n = len(st["x"])
    pid = None if pid is None else np.ascontiguousarray(pid, dtype=np.int32)
    cond = None if cond is None else np.ascontiguousarray(cond, dtype=np.float64)
    omega_wall = None if omega_wall is None else np.ascontiguousarray(omega_wall, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    status = np.zeros(n, dtype=np.int32)
    counters = np.zeros(8, dtype=np.int64)
    lib().or_step(mesh._h, n, _p(rows, D), ctypes.byref(params), int(seed), int(step_no),
                  *[_p(st[k], D) for k in STATE_KEYS], _p(st["elem"], I), _p(status, I),
                  counters.ctypes.data_as(PL), None if pid is None else _p(pid, I),
                  None if cond is None else _p(cond, D), None if omega_wall is None else _p(omega_wall, D))
    names = ["walk_steps", "reflections", "crossings_periodic", "fallbacks", "brute", "lost",
             "omega_reflections", "near_face"]
    return dict(zip(names, counters.tolist())), status


def step_threads(mesh, rows, params, seed, step_no, st, threads=0, pid=None, cond=None, omega_wall=None):
    """step() with its particle loop over `threads` host threads (0: all;
    OpenMP).  Bit for bit the results of step().  Returns (counters, status,
    threads used)."""
    n = len(st["x"])
    pid = None if pid is None else np.ascontiguousarray(pid, dtype=np.int32)
    cond = None if cond is None else np.ascontiguousarray(cond, dtype=np.float64)
    omega_wall = None if omega_wall is None else np.ascontiguousarray(omega_wall, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    status = np.zeros(n, dtype=np.int32)
    counters = np.zeros(8, dtype=np.int64)
    used = lib().or_step_threads(mesh._h, n, _p(rows, D), ctypes.byref(params), int(seed), int(step_no),
                                 *[_p(st[k], D) for k in STATE_KEYS], _p(st["elem"], I), _p(status, I),
                                 counters.ctypes.data_as(PL), None if pid is None else _p(pid, I),
                                 None if cond is None else _p(cond, D),
                                 None if omega_wall is None else _p(omega_wall, D), int(threads))
    names = ["walk_steps", "reflections", "crossings_periodic", "fallbacks", "brute", "lost",
             "omega_reflections", "near_face"]
    return dict(zip(names, counters.tolist())), status, int(used)


def statistics(mesh, st, prev_ns=None):
    """Element stats, node stats and node derivatives at the end of a step."""
    es = elem_stats(mesh.n_tri, st)
    ns, kept = node_stats(mesh, es, prev_ns)
    nd = node_derivs(mesh, ns)
    return es, ns, nd, kept
