"""Python binding of libpdfgb with the C names (argument marshalling only).

Device buffers are torch CUDA tensors; every step of the computation runs in
the library's CUDA kernels.  Streams default to torch's current stream.
"""
import ctypes

import numpy as np
import torch

from . import capi
from .capi import check, lib


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t, dtype=None, numel=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError("expected %s, got %s" % (dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d elements, got %d" % (numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def model_params(**kw):
    """pdf_model_params with the library defaults, then the given overrides.
    closure / tm_mode / pressure accept names ("glm", "slm", "frozen"; "turb",
    "cphi"; "none", "channel")."""
    p = capi.ModelParams()
    lib().pdf_model_params_default(ctypes.byref(p))
    names = {"closure": {"glm": 0, "slm": 1, "frozen": 2}, "tm_mode": {"turb": 0, "cphi": 1, "source": 2},
             "pressure": {"none": 0, "channel": 1, "projection": 2, "projection_inout": 3}, "arith": {"fx": 0, "fp64": 1}, "mix": {"iem": 0, "iecm": 1}}
    for k, v in kw.items():
        if k in names and isinstance(v, str):
            v = names[k][v]
        setattr(p, k, v)
    return p


class Mesh:
    """Owns a pdf_mesh handle."""

    def __init__(self, mesh):
        xy = np.ascontiguousarray(mesh["xy"], dtype=np.float64)
        tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
        twin = mesh.get("twin")
        twin = None if twin is None else np.ascontiguousarray(twin, dtype=np.int32)
        bnd = np.ascontiguousarray(mesh["bnd"], dtype=np.int32)
        h = ctypes.c_void_p()
        check(lib().pdf_mesh_create(
            xy.ctypes.data_as(capi.PD), len(xy), tri.ctypes.data_as(capi.PI32), len(tri),
            None if twin is None else twin.ctypes.data_as(capi.PI32),
            bnd.ctypes.data_as(capi.PI32), len(bnd), float(mesh.get("period", 0.0)),
            ctypes.byref(h)), "pdf_mesh_create")
        self.handle = h
        self.n_nodes, self.n_tri = len(xy), len(tri)

    def connectivity(self):
        nbr = np.zeros((self.n_tri, 3), dtype=np.int32)
        shift = np.zeros((self.n_tri, 3), dtype=np.int32)
        check(lib().pdf_mesh_connectivity(self.handle, nbr.ctypes.data_as(capi.PI32),
                                          shift.ctypes.data_as(capi.PI32)), "pdf_mesh_connectivity")
        return nbr, shift

    def wall_distance(self):
        d = np.zeros(self.n_nodes)
        nrm = np.zeros((self.n_nodes, 2))
        check(lib().pdf_mesh_wall_distance(self.handle, d.ctypes.data_as(capi.PD), nrm.ctypes.data_as(capi.PD)),
              "pdf_mesh_wall_distance")
        return d, nrm

    def close(self):
        if getattr(self, "handle", None):
            lib().pdf_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Particles:
    """Owns a pdf_particles handle (the particle state lives in the library)."""

    def __init__(self, mesh, seed, ppe=None, count=None, u_profile="parabola", u_sigma=0.1,
                 elem_psi0=None, precision=capi.PDF_FP64, stream=None):
        ip = capi.InitParams()
        keep = []
        if count is not None:
            c = np.ascontiguousarray(count, dtype=np.int32)
            keep.append(c)
            ip.count = c.ctypes.data_as(capi.PI32)
        ip.ppe = int(ppe or 0)
        ip.u_profile = ({"zero": 0, "parabola": 1, "uniform": 2}[u_profile] if isinstance(u_profile, str)
                        else int(u_profile))
        ip.u_sigma = float(u_sigma)
        if elem_psi0 is not None:
            ps = np.ascontiguousarray(elem_psi0, dtype=np.float64)
            keep.append(ps)
            ip.elem_psi0 = ps.ctypes.data_as(capi.PD)
        h = ctypes.c_void_p()
        check(lib().pdf_particles_init(mesh.handle, ctypes.byref(ip), int(seed), int(precision),
                                       _stream(stream), ctypes.byref(h)), "pdf_particles_init")
        self.handle = h
        self.mesh = mesh
        n = ctypes.c_int64()
        check(lib().pdf_particles_count(h, ctypes.byref(n)), "pdf_particles_count")
        self.n = n.value

    def get_state(self, stream=None):
        dev = torch.device("cuda")
        out = {k: torch.empty(self.n, dtype=torch.float64, device=dev)
               for k in ("x", "y", "u", "v", "w", "om", "ps")}
        out["elem"] = torch.empty(self.n, dtype=torch.int32, device=dev)
        check(lib().pdf_particles_get_state(self.handle, *[_ptr(out[k]) for k in
                                                            ("x", "y", "u", "v", "w", "om", "ps", "elem")],
                                            _stream(stream)), "pdf_particles_get_state")
        return out

    def set_iecm(self, bins=(5, 5, 5), m_min=2):
        """Compute velocity-conditioned scalar means (IECM) at every statistics
        call with the given sort-and-divide binning; bins=None disables it."""
        b = (0, 0, 0) if bins is None else tuple(int(x) for x in bins)
        check(lib().pdf_particles_set_iecm(self.handle, b[0], b[1], b[2], int(m_min)), "pdf_particles_set_iecm")

    def iecm_cond(self, stream=None):
        out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        check(lib().pdf_iecm_cond(self.handle, _ptr(out), _stream(stream)), "pdf_iecm_cond")
        return out

    def set_reorder(self, every):
        """Copy the state into element order every `every` statistics calls (0: never)."""
        check(lib().pdf_particles_set_reorder(self.handle, int(every)), "pdf_particles_set_reorder")

    def set_state(self, st, stream=None):
        args = []
        for k in ("x", "y", "u", "v", "w", "om", "ps"):
            args.append(_ptr(st[k], torch.float64, self.n))
        args.append(_ptr(st["elem"], torch.int32, self.n))
        check(lib().pdf_particles_set_state(self.handle, *args, _stream(stream)), "pdf_particles_set_state")

    def save(self, stream=None):
        """The saved byte form of the set (pdf_particles_save) as a numpy uint8 array."""
        size = ctypes.c_size_t()
        check(lib().pdf_particles_save_size(self.handle, ctypes.byref(size)), "pdf_particles_save_size")
        buf = np.empty(size.value, dtype=np.uint8)
        check(lib().pdf_particles_save(self.handle, ctypes.c_void_p(buf.ctypes.data), size.value, _stream(stream)),
              "pdf_particles_save")
        return buf

    @classmethod
    def load(cls, mesh, buf, stream=None):
        """A new set from a saved byte form (pdf_particles_load)."""
        b = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if not isinstance(buf, np.ndarray) else buf,
                                 dtype=np.uint8)
        h = ctypes.c_void_p()
        check(lib().pdf_particles_load(mesh.handle, ctypes.c_void_p(b.ctypes.data), b.size, _stream(stream),
                                       ctypes.byref(h)), "pdf_particles_load")
        self = cls.__new__(cls)
        self.handle = h
        self.mesh = mesh
        n = ctypes.c_int64()
        check(lib().pdf_particles_count(h, ctypes.byref(n)), "pdf_particles_count")
        self.n = n.value
        return self

    def close(self):
        if getattr(self, "handle", None):
            lib().pdf_particles_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pdf_mesh_create(mesh):
    return Mesh(mesh)


def pdf_particles_save(particles, stream=None):
    return particles.save(stream)


def pdf_particles_load(mesh, buf, stream=None):
    return Particles.load(mesh, buf, stream)


def pdf_particles_init(mesh, seed, **kw):
    return Particles(mesh, seed, **kw)


def pdf_step(particles, mesh, params, wp=None, elem_coeff=None, step=0, stream=None, info=False):
    """One particle time step.  Returns the counters dict when info=True."""
    si = capi.StepInfo() if info else None
    st = lib().pdf_step(particles.handle, mesh.handle, ctypes.byref(params),
                        _ptr(wp, torch.float64, None if wp is None else 9 * mesh.n_nodes),
                        _ptr(elem_coeff, torch.float64, None if elem_coeff is None else capi.PDF_NCOEF * mesh.n_tri),
                        int(step) & 0xFFFFFFFF, _stream(stream), ctypes.byref(si) if si is not None else None)
    if info and st == capi.PDF_ELOST:
        d = si.as_dict()
        d["status"] = "lost"
        return d
    check(st, "pdf_step")
    return si.as_dict() if info else None


def _host_ptr(t, dtype, numel):
    if t.is_cuda or not t.is_pinned() or not t.is_contiguous():
        raise ValueError("expected a contiguous page-locked host tensor")
    if t.dtype != dtype or t.numel() != numel:
        raise ValueError("expected %d elements of %s" % (numel, dtype))
    return ctypes.c_void_p(t.data_ptr())


def _out_ptr(t, numel):
    """An optional output: a CUDA tensor or a page-locked host tensor."""
    if t is None:
        return None
    return _ptr(t, torch.float64, numel) if t.is_cuda else _host_ptr(t, torch.float64, numel)


def pdf_step_host(particles, mesh, params, state, wp=None, elem_coeff=None, step=0, stream=None, info=False):
    """pdf_step for a state held in page-locked host tensors (dict x, y, u,
    v, w, om, ps float64 and elem int32, particle-id order), which is read
    and overwritten with the stepped state; the loads, the step and the
    stores run overlapped in chunks.  Returns the counters dict when
    info=True."""
    si = capi.StepInfo()
    args = [_host_ptr(state[k], torch.float64, particles.n) for k in ("x", "y", "u", "v", "w", "om", "ps")]
    args.append(_host_ptr(state["elem"], torch.int32, particles.n))
    st = lib().pdf_step_host(particles.handle, mesh.handle, ctypes.byref(params),
                             _ptr(wp, torch.float64, None if wp is None else 9 * mesh.n_nodes),
                             _ptr(elem_coeff, torch.float64, None if elem_coeff is None else capi.PDF_NCOEF * mesh.n_tri),
                             int(step) & 0xFFFFFFFF, *args, _stream(stream), ctypes.byref(si))
    if info and st == capi.PDF_ELOST:
        d = si.as_dict()
        d["status"] = "lost"
        return d
    check(st, "pdf_step_host")
    return si.as_dict() if info else None


def pdf_step_host_stats(particles, mesh, params, state, elem_stats=None, node_stats=None, node_derivs=None,
                        wp=None, elem_coeff=None, step=0, stream=None, info=False):
    """pdf_step_host followed by pdf_estimate_stats in one call (the same
    results); the statistics run while the last chunks are written back.
    The optional statistics outputs are device or page-locked host tensors
    laid out as for pdf_estimate_stats."""
    si = capi.StepInfo()
    args = [_host_ptr(state[k], torch.float64, particles.n) for k in ("x", "y", "u", "v", "w", "om", "ps")]
    args.append(_host_ptr(state["elem"], torch.int32, particles.n))
    st = lib().pdf_step_host_stats(particles.handle, mesh.handle, ctypes.byref(params),
                                   _ptr(wp, torch.float64, None if wp is None else 9 * mesh.n_nodes),
                                   _ptr(elem_coeff, torch.float64, None if elem_coeff is None else capi.PDF_NCOEF * mesh.n_tri),
                                   int(step) & 0xFFFFFFFF, *args,
                                   _out_ptr(elem_stats, capi.PDF_NES * mesh.n_tri),
                                   _out_ptr(node_stats, capi.PDF_NNS * mesh.n_nodes),
                                   _out_ptr(node_derivs, capi.PDF_NND * mesh.n_nodes),
                                   _stream(stream), ctypes.byref(si))
    if info and st == capi.PDF_ELOST:
        d = si.as_dict()
        d["status"] = "lost"
        return d
    check(st, "pdf_step_host_stats")
    return si.as_dict() if info else None


def pdf_estimate_stats(particles, mesh, elem_stats=None, node_stats=None, node_derivs=None, stream=None):
    check(lib().pdf_estimate_stats(particles.handle, mesh.handle,
                                   _ptr(elem_stats, torch.float64, None if elem_stats is None else capi.PDF_NES * mesh.n_tri),
                                   _ptr(node_stats, torch.float64, None if node_stats is None else capi.PDF_NNS * mesh.n_nodes),
                                   _ptr(node_derivs, torch.float64, None if node_derivs is None else capi.PDF_NND * mesh.n_nodes),
                                   _stream(stream)), "pdf_estimate_stats")


def pdf_estimate_stats_noalloc(particles, mesh, elem_stats=None, node_stats=None, node_derivs=None,
                               stream=None):
    """pdf_estimate_stats without any device allocation (fixed library scratch;
    see include/pdfgb.h for its limits and the rule on overlapping calls)."""
    check(lib().pdf_estimate_stats_noalloc(
        particles.handle, mesh.handle,
        _ptr(elem_stats, torch.float64, None if elem_stats is None else capi.PDF_NES * mesh.n_tri),
        _ptr(node_stats, torch.float64, None if node_stats is None else capi.PDF_NNS * mesh.n_nodes),
        _ptr(node_derivs, torch.float64, None if node_derivs is None else capi.PDF_NND * mesh.n_nodes),
        _stream(stream)), "pdf_estimate_stats_noalloc")


def pdf_elem_coeff(particles, mesh, params, wp=None, rows=None, stream=None):
    if rows is None:
        rows = torch.empty((mesh.n_tri, capi.PDF_NCOEF), dtype=torch.float64, device="cuda")
    check(lib().pdf_elem_coeff(particles.handle, mesh.handle, ctypes.byref(params),
                               _ptr(wp, torch.float64, None if wp is None else 9 * mesh.n_nodes),
                               _ptr(rows, torch.float64, capi.PDF_NCOEF * mesh.n_tri), _stream(stream)),
          "pdf_elem_coeff")
    return rows


def pdf_rng_gauss(seed, c1, c2, c3, n, out=None, stream=None):
    if out is None:
        out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    check(lib().pdf_rng_gauss(int(seed), c1, c2, c3, int(n), _ptr(out, torch.float32, 4 * n), _stream(stream)),
          "pdf_rng_gauss")
    return out


def pdf_last_error():
    m = lib().pdf_last_error()
    return m.decode() if m else ""


def pdf_profile_enable(on=True):
    check(lib().pdf_profile_enable(1 if on else 0), "pdf_profile_enable")


def pdf_pressure_project(particles, mesh, params, Cp=None, rtol=1e-10, max_it=20000, stream=None):
    """Stabilised pressure projection after a step's statistics; returns
    (iterations, relative residual).  The particles' velocities are corrected
    and the statistics follow.  Cp defaults to dt / 2."""
    if Cp is None:
        Cp = 0.5 * params.dt
    it = ctypes.c_int32()
    res = ctypes.c_double()
    check(lib().pdf_pressure_project(particles.handle, mesh.handle, ctypes.byref(params), float(Cp), float(rtol),
                                     int(max_it), ctypes.byref(it), ctypes.byref(res), _stream(stream)),
          "pdf_pressure_project")
    return it.value, res.value


def pdf_redistribute(particles, mesh, min_npel, seed, step, stream=None):
    """Particle redistribution (App. D); returns the number of particles
    moved.  Estimate the statistics again before the next step."""
    moved = ctypes.c_int32()
    check(lib().pdf_redistribute(particles.handle, mesh.handle, int(min_npel), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                 int(step) & 0xFFFFFFFF, ctypes.byref(moved), _stream(stream)), "pdf_redistribute")
    return moved.value


def pdf_pressure_set_solver(particles, persistent=False):
    check(lib().pdf_pressure_set_solver(particles.handle, 1 if persistent else 0), "pdf_pressure_set_solver")


def pdf_pressure_field(particles, mesh, set=None, stream=None):
    """The projection's nodal pressure <P'> (device FP64 tensor); `set`
    replaces it first."""
    out = torch.empty(mesh.n_nodes, dtype=torch.float64, device="cuda")
    check(lib().pdf_pressure_field(particles.handle, _ptr(set, torch.float64, mesh.n_nodes) if set is not None else None,
                                   _ptr(out), _stream(stream)), "pdf_pressure_field")
    return out


def pdf_profile_only(kernel=None):
    check(lib().pdf_profile_only(kernel.encode() if kernel else None), "pdf_profile_only")


def pdf_profile_reset():
    check(lib().pdf_profile_reset(), "pdf_profile_reset")


def pdf_profile_query(kernel):
    """(launches, total_ms) of the named kernel since the last reset."""
    n, ms = ctypes.c_int64(), ctypes.c_double()
    check(lib().pdf_profile_query(kernel.encode(), ctypes.byref(n), ctypes.byref(ms)), "pdf_profile_query")
    return n.value, ms.value


def pdf_kernel_launches():
    return int(lib().pdf_kernel_launches())


def pdf_relax_solve(mesh, params, node_stats, wp, rtol=1e-10, max_it=1000, stream=None):
    """Solve for wp in place (device [9, n_nodes] float64, in: initial guess)
    from caller node statistics (device [n_nodes, 12] float64).
    Returns (iterations [9], relative residuals [9]); raises on PDF_ENOTCONV."""
    it = (ctypes.c_int32 * 9)()
    rr = (ctypes.c_double * 9)()
    check(lib().pdf_relax_solve(mesh.handle, ctypes.byref(params),
                                _ptr(node_stats, torch.float64, capi.PDF_NNS * mesh.n_nodes),
                                _ptr(wp, torch.float64, 9 * mesh.n_nodes), float(rtol), int(max_it), it, rr,
                                _stream(stream)), "pdf_relax_solve")
    return list(it), list(rr)


def pdf_relax_solve_particles(particles, mesh, params, wp, rtol=1e-10, max_it=1000, stream=None):
    """Solve for wp in place from the particle set's last statistics.
    Returns (iterations [9], relative residuals [9]); raises on PDF_ENOTCONV."""
    it = (ctypes.c_int32 * 9)()
    rr = (ctypes.c_double * 9)()
    check(lib().pdf_relax_solve_particles(particles.handle, mesh.handle, ctypes.byref(params),
                                          _ptr(wp, torch.float64, 9 * mesh.n_nodes), float(rtol), int(max_it),
                                          it, rr, _stream(stream)), "pdf_relax_solve_particles")
    return list(it), list(rr)


def pdf_relax_set_solver(particles, multigrid=True):
    check(lib().pdf_relax_set_solver(particles.handle, 1 if multigrid else 0), "pdf_relax_set_solver")


def pdf_relax_rhs(particles, mesh, params, stream=None):
    rhs = torch.empty((9, mesh.n_nodes), dtype=torch.float64, device="cuda")
    L2 = torch.empty((3, mesh.n_nodes), dtype=torch.float64, device="cuda")
    check(lib().pdf_relax_rhs(particles.handle, mesh.handle, ctypes.byref(params), _ptr(rhs), _ptr(L2),
                              _stream(stream)), "pdf_relax_rhs")
    return rhs, L2


class Mlp:
    """Owns a pdf_mlp handle (the learned warm start of the relaxation solve)."""

    def __init__(self, seed=0):
        h = ctypes.c_void_p()
        check(lib().pdf_mlp_create(int(seed), ctypes.byref(h)), "pdf_mlp_create")
        self.handle = h

    def params(self):
        out = np.zeros(capi.PDF_MLP_NPARAM, dtype=np.float32)
        nrm = np.zeros(64, dtype=np.float32)
        check(lib().pdf_mlp_params(self.handle, None, ctypes.c_void_p(out.ctypes.data), None,
                                   ctypes.c_void_p(nrm.ctypes.data)), "pdf_mlp_params")
        return out, nrm

    def set_params(self, flat=None, norm=None):
        f = None if flat is None else np.ascontiguousarray(flat, dtype=np.float32)
        n = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        check(lib().pdf_mlp_params(self.handle, None if f is None else ctypes.c_void_p(f.ctypes.data), None,
                                   None if n is None else ctypes.c_void_p(n.ctypes.data), None), "pdf_mlp_params")

    def fit_norm(self, X, Y, stream=None):
        check(lib().pdf_mlp_fit_norm(self.handle, _ptr(X, torch.float32), _ptr(Y, torch.float32), X.shape[0],
                                     _stream(stream)), "pdf_mlp_fit_norm")

    def forward(self, X, stream=None):
        Y = torch.empty((X.shape[0], 9), dtype=torch.float32, device="cuda")
        check(lib().pdf_mlp_forward(self.handle, _ptr(X, torch.float32), X.shape[0], _ptr(Y), _stream(stream)),
              "pdf_mlp_forward")
        return Y

    def grad(self, X, Y, stream=None):
        g = torch.empty(capi.PDF_MLP_NPARAM, dtype=torch.float32, device="cuda")
        loss = ctypes.c_float()
        check(lib().pdf_mlp_grad(self.handle, _ptr(X, torch.float32), _ptr(Y, torch.float32), X.shape[0], _ptr(g),
                                 ctypes.byref(loss), _stream(stream)), "pdf_mlp_grad")
        return loss.value, g

    def train_step(self, X, Y, lr, want_loss=False, stream=None):
        loss = ctypes.c_float()
        check(lib().pdf_mlp_train_step(self.handle, _ptr(X, torch.float32), _ptr(Y, torch.float32), X.shape[0],
                                       float(lr), ctypes.byref(loss) if want_loss else None, _stream(stream)),
              "pdf_mlp_train_step")
        return loss.value if want_loss else None

    def guess(self, particles, mesh, params, wp, stream=None):
        """wp = the relaxation's right-hand side + the network's correction."""
        scratch = torch.empty(20 * mesh.n_nodes, dtype=torch.float32, device="cuda")
        check(lib().pdf_mlp_guess(self.handle, particles.handle, mesh.handle, ctypes.byref(params),
                                  _ptr(wp, torch.float64), _ptr(scratch), _stream(stream)), "pdf_mlp_guess")
        return wp

    def close(self):
        if getattr(self, "handle", None):
            lib().pdf_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pdf_mlp_batch(X, Y, seed, step, batch, Xb=None, Yb=None, stream=None):
    """A training batch drawn (Philox, with replacement) from the pairs (X, Y)."""
    n = X.shape[0]
    Xb = torch.empty((batch, X.shape[1]), dtype=torch.float32, device="cuda") if Xb is None else Xb
    Yb = torch.empty((batch, Y.shape[1]), dtype=torch.float32, device="cuda") if Yb is None else Yb
    check(lib().pdf_mlp_batch(_ptr(X, torch.float32), _ptr(Y, torch.float32), n, int(seed), int(step), int(batch),
                              _ptr(Xb), _ptr(Yb), _stream(stream)), "pdf_mlp_batch")
    return Xb, Yb


def pdf_mlp_features(particles, mesh, params, wp=None, stream=None):
    """Node features X [n, 11] and, with a solution wp, targets Y [n, 9] = wp - rhs."""
    X = torch.empty((mesh.n_nodes, 11), dtype=torch.float32, device="cuda")
    Y = None if wp is None else torch.empty((mesh.n_nodes, 9), dtype=torch.float32, device="cuda")
    check(lib().pdf_mlp_features(particles.handle, mesh.handle, ctypes.byref(params), _ptr(wp, torch.float64),
                                 _ptr(X), _ptr(Y), _stream(stream)), "pdf_mlp_features")
    return X, Y
