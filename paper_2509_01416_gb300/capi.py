"""ctypes binding of libnop.so: the C ABI of include/nop.h under the same names.

Argument marshalling only -- every computation happens in the CUDA library.
Importing this module loads the in-tree library and fails loudly when it is
missing; there is no fallback.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnop.so")

NOP_OK, NOP_EINVAL, NOP_ECUDA, NOP_ENOMEM = 0, -1, -2, -3
NOP_ENOCONV, NOP_EDIVERGE, NOP_ETIMEOUT, NOP_ENAN, NOP_ESTATE, NOP_EIO = -4, -5, -6, -7, -8, -9
NOP_GEOM_SLAB, NOP_GEOM_XY = 1, 2
NOP_BC_VACUUM, NOP_BC_REFLECTIVE = 0, 1
NOP_PREC_F32, NOP_PREC_F64 = 0, 1
NOP_WARM_NONE, NOP_WARM_RECAST, NOP_WARM_RECAST_CP = 0, 1, 2
NOP_PHI0_DEVICE, NOP_OUT_DEVICE, NOP_SP_CONSTRAINED, NOP_DSA = 1, 2, 4, 8
NOP_SWEEP_CHUNKED = 16
NOP_GAUSS_SEIDEL = 64
NOP_COLD_SCHEDULE = 32
NOP_SCHED_AUTO, NOP_SCHED_WARP, NOP_SCHED_BLOCK, NOP_SCHED_MODEL = 0, 1, 2, 3
NOP_SCHED_TUNE_MIN = 256
NOP_NOALLOC_MAX_CELLS, NOP_NOALLOC_MAX_ORDER = 65536, 128

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class nop_problem(C.Structure):
    _fields_ = [("geometry", C.c_int), ("n_inst", C.c_int), ("n_cells", _ip),
                ("width", _dp), ("order", _ip), ("nx", C.c_int), ("ny", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("n_groups", C.c_int),
                ("sigma_t", _dp), ("sigma_s", _dp), ("source", _dp),
                ("nu_sigma_f", _dp), ("chi", _dp), ("bc", C.c_int * 4),
                ("sigma_s1", _dp)]


class nop_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("tol_k", C.c_double), ("tol_inner", C.c_double),
                ("itmax", C.c_int), ("itmax_inner", C.c_int), ("precision", C.c_int),
                ("warm_start", C.c_int), ("recast_tol", C.c_double),
                ("recast_itmax", C.c_int), ("flags", C.c_int), ("schedule", C.c_int)]


class nop_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("max_iterations", C.c_int),
                ("sum_iterations", C.c_longlong), ("max_outer", C.c_int),
                ("recast_iterations", C.c_int), ("recast_status", C.c_int),
                ("max_change", C.c_double), ("inst_iterations", _ip),
                ("inst_status", _ip)]


class nop_timings(C.Structure):
    _fields_ = [("sweep_ms", C.c_double), ("operator_ms", C.c_double),
                ("setup_ms", C.c_double), ("launches", C.c_longlong),
                ("sweep_launches", C.c_longlong), ("cell_angle_updates", C.c_double),
                ("last_span_ms", C.c_double), ("last_inst_max_ms", C.c_double),
                ("last_inst_mean_ms", C.c_double), ("last_block_instances", C.c_int),
                ("last_direct_instances", C.c_int), ("last_tune_ms", C.c_double)]


NOP_NO_DEEPONET, NOP_NO_FNO1D, NOP_NO_FNO2D = 1, 2, 3


class nop_no_config(C.Structure):
    _fields_ = [("kind", C.c_int), ("sensors", C.c_int), ("width", C.c_int),
                ("basis", C.c_int), ("depth", C.c_int), ("modes", C.c_int),
                ("proj", C.c_int), ("sigma_t_star", C.c_double),
                ("sigma_s_star", C.c_double), ("length", C.c_double)]


class nop_train_config(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("order", _ip)]


_fp = C.POINTER(C.c_float)

# every symbol include/nop.h declares, with its ctypes signature
SIGNATURES = {
    "nop_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "nop_destroy": (C.c_int, [C.c_void_p]),
    "nop_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nop_status_str": (C.c_char_p, [C.c_int]),
    "nop_last_error": (C.c_char_p, [C.c_void_p]),
    "nop_set_problem": (C.c_int, [C.c_void_p, C.POINTER(nop_problem)]),
    "nop_get_quadrature": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, _ip]),
    "nop_solve_fixed_source": (C.c_int, [C.c_void_p, C.POINTER(nop_solve_opts), C.c_void_p,
                                         C.c_void_p, C.POINTER(nop_stats)]),
    "nop_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "nop_set_wait_limit": (C.c_int, [C.c_void_p, C.c_longlong]),
    "nop_set_diffusion": (C.c_int, [C.c_void_p, C.c_int, _ip, _dp, _dp, _dp, _dp]),
    "nop_diffusion_solve": (C.c_int, [C.c_void_p, _dp]),
    "nop_measure_alu_peaks": (C.c_int, [C.c_void_p, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "nop_sched_select_teams": (C.c_int, [C.c_int, _dp, _dp, C.c_int, C.c_int, C.c_int, C.c_double, _ip,
                                         C.POINTER(C.c_double)]),
    "nop_slab_solve_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                         C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                         C.c_void_p]),
    "nop_no_param_count": (C.c_int, [C.POINTER(nop_no_config), C.POINTER(C.c_longlong)]),
    "nop_no_set": (C.c_int, [C.c_void_p, C.POINTER(nop_no_config), _fp]),
    "nop_no_get": (C.c_int, [C.c_void_p, _fp]),
    "nop_no_write_file": (C.c_int, [C.c_char_p, C.POINTER(nop_no_config), _fp]),
    "nop_no_read_file": (C.c_int, [C.c_char_p, C.POINTER(nop_no_config), _fp,
                                   C.POINTER(C.c_longlong)]),
    "nop_no_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "nop_no_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "nop_no_forward": (C.c_int, [C.c_void_p, C.c_int, _fp, _fp, C.c_int, _fp]),
    "nop_no_loss_grad": (C.c_int, [C.c_void_p, C.c_int, _fp, _fp, C.c_int, _fp,
                                   C.POINTER(C.c_double), _fp]),
    "nop_no_train": (C.c_int, [C.c_void_p, C.POINTER(nop_train_config), C.c_int, _fp, _fp,
                               C.c_int, _fp, _dp]),
    "nop_no_sensors": (C.c_int, [C.c_void_p, _dp, _fp]),
    "nop_no_predict": (C.c_int, [C.c_void_p, _dp, _dp]),
    "nop_recast_iterate": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_void_p,
                                     C.POINTER(nop_stats)]),
    "nop_sp_eigen": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_void_p,
                               C.c_void_p, C.POINTER(nop_stats)]),
    "nop_get_timing": (C.c_int, [C.c_void_p, C.POINTER(nop_timings)]),
    "nop_get_trace": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nop_solve_eigen": (C.c_int, [C.c_void_p, C.POINTER(nop_solve_opts), C.c_void_p,
                                  C.c_double, C.c_void_p, C.c_void_p,
                                  C.POINTER(nop_stats)]),
}

_lib = None


def lib():
    """Load libnop.so (built by paper_2509_01416_gb300.build) or raise."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnop.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class NopError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (lib().nop_status_str(code).decode(), code, msg))
        self.code = code


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)
