"""ctypes declarations of the C-ABI in include/pdfgb.h (argument marshalling only)."""
import ctypes
import os
import threading

from . import build as _build

PDF_OK, PDF_EINVAL, PDF_ENOMEM, PDF_ECUDA, PDF_ELOST, PDF_ENOTCONV, PDF_ENUMERIC, PDF_ESTATE = range(8)
STATUS_NAMES = ["PDF_OK", "PDF_EINVAL", "PDF_ENOMEM", "PDF_ECUDA", "PDF_ELOST", "PDF_ENOTCONV",
                "PDF_ENUMERIC", "PDF_ESTATE"]
PDF_TAG_WALL, PDF_TAG_PERIODIC, PDF_TAG_INFLOW, PDF_TAG_OUTFLOW = 1, 2, 3, 4
PDF_CLOSURE_GLM, PDF_CLOSURE_SLM, PDF_CLOSURE_FROZEN = 0, 1, 2
PDF_TM_TURB, PDF_TM_CPHI, PDF_TM_SOURCE = 0, 1, 2
PDF_PRESSURE_NONE, PDF_PRESSURE_CHANNEL, PDF_PRESSURE_PROJECTION, PDF_PRESSURE_PROJECTION_INOUT = 0, 1, 2, 3
PDF_FP64, PDF_FP32_STATE = 0, 1
PDF_ARITH_FX, PDF_ARITH_FP64 = 0, 1
PDF_NCOEF, PDF_NES, PDF_NNS, PDF_NND = 26, 13, 12, 10
PDF_NOALLOC_MAX_PARTICLES, PDF_NOALLOC_MAX_ELEMENTS = 524288, 262144
PDF_MLP_NPARAM = 9673


class PdfError(RuntimeError):
    def __init__(self, status, where, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s: %s" % (where, name, msg))


class ModelParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("nu", ctypes.c_double), ("Pi", ctypes.c_double),
                ("c_phi", ctypes.c_double), ("closure", ctypes.c_int32), ("tm_mode", ctypes.c_int32),
                ("pressure", ctypes.c_int32), ("arith", ctypes.c_int32)] + [
        (n, ctypes.c_double) for n in ("C1", "C2", "C3", "C4", "CT", "CL", "Ceta", "Cv", "gamma5",
                                       "Comega1", "Comega2", "C0_slm", "src_x", "src_y", "src_r", "Cs", "Ct")] + [
        ("mix", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class InitParams(ctypes.Structure):
    _fields_ = [("count", ctypes.POINTER(ctypes.c_int32)), ("ppe", ctypes.c_int32),
                ("u_profile", ctypes.c_int32), ("u_sigma", ctypes.c_double),
                ("elem_psi0", ctypes.POINTER(ctypes.c_double))]


class StepInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("walk_steps", "reflections", "crossings_periodic",
                                              "fallbacks", "brute", "lost", "omega_reflections",
                                              "near_face")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lock = threading.Lock()
_lib = None

V = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
U32 = ctypes.c_uint32
U64 = ctypes.c_uint64
D = ctypes.c_double
PD = ctypes.POINTER(ctypes.c_double)
PI32 = ctypes.POINTER(ctypes.c_int32)
PV = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes)
PROTOTYPES = {
    "pdf_model_params_default": (None, [ctypes.POINTER(ModelParams)]),
    "pdf_mesh_create": (I32, [PD, I32, PI32, I32, PI32, PI32, I32, D, PV]),
    "pdf_mesh_destroy": (I32, [V]),
    "pdf_mesh_connectivity": (I32, [V, PI32, PI32]),
    "pdf_mesh_size": (I32, [V, PI32, PI32]),
    "pdf_particles_init": (I32, [V, ctypes.POINTER(InitParams), U64, I32, V, PV]),
    "pdf_particles_destroy": (I32, [V]),
    "pdf_particles_count": (I32, [V, ctypes.POINTER(I64)]),
    "pdf_particles_set_reorder": (I32, [V, I32]),
    "pdf_particles_set_iecm": (I32, [V, I32, I32, I32, I32]),
    "pdf_iecm_cond": (I32, [V, V, V]),
    "pdf_pressure_project": (I32, [V, V, ctypes.POINTER(ModelParams), D, D, I32, ctypes.POINTER(I32), ctypes.POINTER(D), V]),
    "pdf_redistribute": (I32, [V, V, I32, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(I32), V]),
    "pdf_pressure_set_solver": (I32, [V, I32]),
    "pdf_pressure_field": (I32, [V, V, V, V]),
    "pdf_particles_get_state": (I32, [V, V, V, V, V, V, V, V, V, V]),
    "pdf_particles_save_size": (I32, [V, ctypes.POINTER(ctypes.c_size_t)]),
    "pdf_particles_save": (I32, [V, V, ctypes.c_size_t, V]),
    "pdf_particles_load": (I32, [V, V, ctypes.c_size_t, V, ctypes.POINTER(V)]),
    "pdf_particles_set_state": (I32, [V, V, V, V, V, V, V, V, V, V]),
    "pdf_step": (I32, [V, V, ctypes.POINTER(ModelParams), V, V, U32, V, ctypes.POINTER(StepInfo)]),
    "pdf_step_host": (I32, [V, V, ctypes.POINTER(ModelParams), V, V, U32, V, V, V, V, V, V, V, V, V,
                            ctypes.POINTER(StepInfo)]),
    "pdf_step_host_stats": (I32, [V, V, ctypes.POINTER(ModelParams), V, V, U32, V, V, V, V, V, V, V, V, V, V, V,
                                  V, ctypes.POINTER(StepInfo)]),
    "pdf_estimate_stats": (I32, [V, V, V, V, V, V]),
    "pdf_estimate_stats_noalloc": (I32, [V, V, V, V, V, V]),
    "pdf_elem_coeff": (I32, [V, V, ctypes.POINTER(ModelParams), V, V, V]),
    "pdf_relax_solve": (I32, [V, ctypes.POINTER(ModelParams), V, V, D, I32, ctypes.POINTER(I32), PD, V]),
    "pdf_relax_solve_particles": (I32, [V, V, ctypes.POINTER(ModelParams), V, D, I32, ctypes.POINTER(I32), PD, V]),
    "pdf_relax_rhs": (I32, [V, V, ctypes.POINTER(ModelParams), V, V, V]),
    "pdf_relax_set_solver": (I32, [V, I32]),
    "pdf_mesh_wall_distance": (I32, [V, PD, PD]),
    "pdf_mlp_create": (I32, [U64, PV]),
    "pdf_mlp_destroy": (I32, [V]),
    "pdf_mlp_params": (I32, [V, V, V, V, V]),
    "pdf_mlp_fit_norm": (I32, [V, V, V, I64, V]),
    "pdf_mlp_forward": (I32, [V, V, I64, V, V]),
    "pdf_mlp_grad": (I32, [V, V, V, I64, V, ctypes.POINTER(ctypes.c_float), V]),
    "pdf_mlp_train_step": (I32, [V, V, V, I64, ctypes.c_float, ctypes.POINTER(ctypes.c_float), V]),
    "pdf_mlp_batch": (I32, [V, V, I64, U64, U32, I64, V, V, V]),
    "pdf_mlp_features": (I32, [V, V, ctypes.POINTER(ModelParams), V, V, V, V]),
    "pdf_mlp_guess": (I32, [V, V, V, ctypes.POINTER(ModelParams), V, V, V]),
    "pdf_rng_gauss": (I32, [U64, U32, U32, U32, I64, V, V]),
    "pdf_profile_enable": (I32, [I32]),
    "pdf_profile_only": (I32, [ctypes.c_char_p]),
    "pdf_profile_reset": (I32, []),
    "pdf_profile_query": (I32, [ctypes.c_char_p, ctypes.POINTER(I64), ctypes.POINTER(D)]),
    "pdf_kernel_launches": (I64, []),
    "pdf_last_error": (ctypes.c_char_p, []),
}


def lib():
    """The loaded libpdfgb (built from source on first use if needed).  Raises
    if the library cannot be built or loaded: there is no fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or _build._stale():
                path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status, where):
    if status != PDF_OK:
        msg = lib().pdf_last_error()
        raise PdfError(status, where, msg.decode() if msg else "")
    return status
