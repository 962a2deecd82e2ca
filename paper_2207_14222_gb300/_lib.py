"""ctypes binding of libusp.so (declarations in include/usp.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Loading fails loudly if the library has not been built.
"""

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libusp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "usp.h")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class Grid(ctypes.Structure):
    _fields_ = [("ndim", c_int32), ("n", c_int64 * 3), ("dx", c_double)]


class LSymbol(ctypes.Structure):
    _fields_ = [("a_re", c_double), ("a_im", c_double), ("b_re", c_double), ("b_im", c_double),
                ("kind", c_int32), ("table", c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("converged", c_int32), ("refinements", c_int32),
                ("stagnated", c_int32), ("final_rel_residual", c_double),
                ("ref_norm", c_double), ("alpha", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Options(ctypes.Structure):
    _fields_ = [("plain", c_int32), ("schedule", c_int32), ("chunk", c_int32),
                ("max_refinements", c_int32), ("no_tma", c_int32), ("cols_tile", c_int32),
                ("tc_dft", c_int32),
                ("onchip_rows", c_int32),
                ("test_wait_fault", c_int32),
                ("residual_fp64", c_int32)]


class FnoConfig(ctypes.Structure):
    _fields_ = [("h", c_int32), ("w", c_int32), ("c_in", c_int32), ("width", c_int32),
                ("layers", c_int32), ("modes", c_int32), ("max_batch", c_int32)]


class PassTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", c_int32), ("ms", c_double),
                ("bytes", c_double)]


STATUS = {
    0: "USP_OK", 1: "USP_ERR_INVALID_ARG", 2: "USP_ERR_UNSUPPORTED_SIZE",
    3: "USP_ERR_V_NOT_CONTRACTIVE", 4: "USP_ERR_NOT_ACCRETIVE", 5: "USP_ERR_ALPHA_RANGE",
    6: "USP_ERR_NOT_CONVERGED", 7: "USP_ERR_DIVERGED", 8: "USP_ERR_NONFINITE",
    9: "USP_ERR_CUDA", 10: "USP_ERR_OOM",
}
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED_SIZE, ERR_V_NOT_CONTRACTIVE = 0, 1, 2, 3
ERR_NOT_ACCRETIVE, ERR_ALPHA_RANGE, ERR_NOT_CONVERGED, ERR_DIVERGED = 4, 5, 6, 7
ERR_NONFINITE, ERR_CUDA, ERR_OOM = 8, 9, 10


class UspError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, message))
        self.status = status


_P = ctypes.POINTER
_SIGNATURES = {
    "usp_solver_create": (c_int32, [_P(Grid), _P(LSymbol), c_void_p, c_int32, c_double,
                                    c_void_p, _P(c_void_p)]),
    "usp_batch_create": (c_int32, [_P(Grid), c_int32, _P(LSymbol), c_void_p, c_int32,
                                   _P(c_double), c_void_p, _P(c_void_p)]),
    "usp_batch_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_int32,
                                  _P(c_double), _P(Result), _P(c_int32)]),
    "usp_batch_history": (c_int32, [c_void_p, c_int32, _P(c_double), c_int32, _P(c_int32)]),
    "usp_solve_many": (c_int32, [_P(c_void_p), c_int32, _P(c_void_p), _P(c_void_p), c_int32,
                                 c_double, c_int32, _P(Result), _P(c_int32)]),
    "usp_autotune": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, _P(Options)]),
    "usp_solver_set_options": (c_int32, [c_void_p, _P(Options)]),
    "usp_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_int32,
                            c_double, _P(Result)]),
    "usp_solve_host": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_int32,
                                 c_double, _P(Result)]),
    "usp_residual_history": (c_int32, [c_void_p, _P(c_double), c_int32, _P(c_int32)]),
    "usp_apply_A": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "usp_residual": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, _P(c_double)]),
    "usp_solver_alpha": (c_int32, [c_void_p, _P(c_double)]),
    "usp_solver_destroy": (None, [c_void_p]),
    "usp_canon_helmholtz": (c_int32, [c_void_p, c_void_p, c_int64, c_double, c_void_p,
                                      c_void_p, _P(LSymbol), c_void_p, c_void_p]),
    "usp_canon_diffusion": (c_int32, [c_void_p, c_double, c_void_p, c_int64, c_double,
                                      c_void_p, c_void_p, _P(LSymbol), c_void_p, c_void_p]),
    "usp_solve_noalloc": (c_int32, [_P(Grid), _P(LSymbol), c_void_p, c_int32, c_double,
                                    c_void_p, c_void_p, c_double, c_int32, c_void_p,
                                    _P(Result)]),
    "usp_time_passes": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, _P(PassTime),
                                  c_int32, _P(c_int32)]),
    "usp_fno_param_count": (c_int64, [_P(FnoConfig)]),
    "usp_fno_create": (c_int32, [_P(FnoConfig), ctypes.c_uint64, c_void_p, _P(c_void_p)]),
    "usp_fno_get_params": (c_int32, [c_void_p, _P(ctypes.c_float), c_int64]),
    "usp_fno_set_params": (c_int32, [c_void_p, _P(ctypes.c_float), c_int64]),
    "usp_fno_predict": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "usp_fno_gradients": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, _P(ctypes.c_float),
                                    _P(c_double)]),
    "usp_fno_train_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double,
                                     _P(c_double)]),
    "usp_fno_destroy": (None, [c_void_p]),
    "usp_variant_create": (c_int32, [_P(Grid), c_int32, _P(c_double), c_void_p, c_double,
                                     c_void_p, _P(c_void_p)]),
    "usp_variant_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_int32,
                                    c_double, _P(Result)]),
    "usp_variant_history": (c_int32, [c_void_p, _P(c_double), c_int32, _P(c_int32)]),
    "usp_variant_destroy": (None, [c_void_p]),
    "usp_variant_set_schedule": (c_int32, [c_void_p, c_int32]),
    "usp_canon_antisymmetric": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_double,
                                          c_void_p, c_void_p, _P(c_double), _P(c_double)]),
    "usp_canon_flux_diffusion": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32,
                                           c_double, c_void_p, c_void_p, _P(c_double),
                                           _P(c_double)]),
    "usp_kernel_launches": (c_int64, []),
    "usp_status_string": (ctypes.c_char_p, [c_int32]),
    "usp_last_error": (ctypes.c_char_p, []),
    "usp_version": (c_int32, []),
}

_lib = None


def header_functions(path=HEADER):
    """Names of the functions include/usp.h declares."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(usp_\w+)\s*\(", src)))


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libusp.so is not built (expected at %s); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error():
    return lib().usp_last_error().decode()


def check(status, allow=(OK,)):
    if status not in allow:
        raise UspError(status, last_error())
    return status
