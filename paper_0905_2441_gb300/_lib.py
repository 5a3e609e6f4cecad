"""ctypes declarations of the C ABI in include/smc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# SMC_LIB_VARIANT=debug selects the bounds-checked build (libsmc_debug.so,
# build.build(debug=True)); there is no fallback between the two
LIB_PATH = os.path.join(_HERE, "libsmc_debug.so" if os.environ.get("SMC_LIB_VARIANT") == "debug"
                        else "libsmc.so")

SMC_OK, SMC_ERR_ARG, SMC_ERR_CUDA, SMC_ERR_NONFINITE = 0, -1, -2, -3
SMC_ERR_ZERO_WEIGHT, SMC_ERR_TIMEOUT, SMC_ERR_UNSUPPORTED = -4, -5, -6
SMC_ERR_BOUNDS = -7
RNG_MOVE, RNG_ACCEPT, RNG_RESAMPLE, RNG_EXCHANGE, RNG_PFNOISE, RNG_MULTINOMIAL = 1, 2, 3, 4, 5, 6
RNG_PROPOSAL = 7
OP_LOGLIK, OP_MOVE, OP_POPMCMC = 0, 1, 2
GMM_1D, GMM_DIAG = 0, 1
PREC_FP32, PREC_BF16SPLIT = 0, 1
MOVE_RW, MOVE_MALA = 0, 1
PF_MSV, PF_LG, PF_FSV = 0, 1, 2

# every entry point include/smc.h declares
EXPORTS = ("smc_create", "smc_destroy", "smc_reserve", "smc_ctx_check", "smc_status_string",
           "smc_set_launch", "smc_get_launch", "smc_loglik_batch", "smc_reweight", "smc_ess",
           "smc_resample_systematic", "smc_gather", "smc_mh_move", "smc_popmcmc_sweep",
           "pf_step", "smc_rng_words", "smc_rng_normals", "smc_measure_peak",
           "smc_resample_systematic_noalloc", "smc_resample_multinomial",
           "smc_resample_residual", "smc_is_moments", "smc_rng_mrg32k3a",
           "smc_reweight_resample", "smc_set_wait_limit", "smc_pf_filter_step")
PEAK_EX2, PEAK_LG2, PEAK_FFMA, PEAK_DFMA = 0, 1, 2, 3


class SmcGmm(C.Structure):
    _fields_ = [("kind", C.c_int32), ("K", C.c_int32), ("d", C.c_int32),
                ("precision", C.c_int32), ("log_w", C.POINTER(C.c_float)),
                ("sigma", C.c_float), ("lo", C.c_float), ("hi", C.c_float)]


class SmcIsProblem(C.Structure):
    _fields_ = [("K", C.c_int32), ("mu", C.c_float * 8), ("a", C.c_float * 8), ("var", C.c_float),
                ("prop_mean", C.c_float), ("prop_sd", C.c_float), ("power", C.c_int32)]


class SmcPfModel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("d", C.c_int32), ("phi", C.c_float * 8),
                ("chol", C.c_float * 64), ("beta", C.c_float), ("m", C.c_int32),
                ("B", C.c_float * 64), ("psi", C.c_float * 8)]


_vp, _i64, _u64, _i32, _u32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_int32, C.c_uint32
_st = C.c_int


def _declare(L):
    L.smc_create.argtypes = [C.POINTER(_vp), C.c_int]
    L.smc_destroy.argtypes = [_vp]
    L.smc_reserve.argtypes = [_vp, _i64, _i32]
    L.smc_ctx_check.argtypes = [_vp, _vp]
    L.smc_status_string.argtypes = [_st]
    L.smc_status_string.restype = C.c_char_p
    L.smc_set_launch.argtypes = [_vp, _i32, _i32, _i32]
    L.smc_set_wait_limit.argtypes = [_vp, _u32]
    L.smc_get_launch.argtypes = [_vp, _i32, _i64, _i64, _i32, C.POINTER(_i32), C.POINTER(_i32)]
    L.smc_loglik_batch.argtypes = [_vp, C.POINTER(SmcGmm), _vp, _i64, _vp, _i64, _vp, _vp, _vp]
    L.smc_reweight.argtypes = [_vp, _vp, C.c_double, _vp, _i64, _vp, _vp, _vp, C.c_double, _vp]
    L.smc_ess.argtypes = [_vp, _vp, _i64, _vp, _vp]
    L.smc_resample_systematic.argtypes = [_vp, _vp, _i64, _u64, _u64, _vp, _vp, _vp, _vp, _vp]
    L.smc_resample_systematic_noalloc.argtypes = [_vp, _i64, _u64, _u64, _vp, _vp, _vp, _vp, _vp,
                                                  _vp]
    L.smc_resample_multinomial.argtypes = [_vp, _vp, _i64, _u64, _u64, _vp, _vp, _vp, _vp]
    L.smc_resample_residual.argtypes = [_vp, _vp, _i64, _u64, _u64, _vp, _vp, _vp, _vp]
    L.smc_gather.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp, _vp]
    L.smc_reweight_resample.argtypes = [_vp, _vp, C.c_double, _vp, _i64, _vp, _vp, _vp, C.c_double,
                                        _u64, _u64, _vp, _vp, _vp]
    L.smc_rng_mrg32k3a.argtypes = [_vp, C.POINTER(C.c_uint32 * 6), _u64, _i64, _i64, _vp, _vp,
                                   _vp]
    L.smc_is_moments.argtypes = [_vp, C.POINTER(SmcIsProblem), _vp, _i64, _u64, _u64, _vp, _vp]
    L.smc_mh_move.argtypes = [_vp, C.POINTER(SmcGmm), _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                              _vp, _i64, _vp, _i64, C.c_float, _i32, _u64, _u64, _vp, _vp]
    L.smc_popmcmc_sweep.argtypes = [_vp, C.POINTER(SmcGmm), _vp, _i64, _vp, _vp, _i64, _vp, _vp,
                                    _i32, C.c_float, _u64, _u64, _vp, _vp]
    L.pf_step.argtypes = [_vp, C.POINTER(SmcPfModel), _vp, _vp, _vp, _vp, _vp, _i64, _u64, _u64,
                          _vp]
    L.smc_pf_filter_step.argtypes = [_vp, C.POINTER(SmcPfModel), _vp, _vp, _vp, _vp, _vp, _vp,
                                     _i64, _vp, _vp, _vp, C.c_double, _u64, _u64, _vp, _vp]
    L.smc_rng_words.argtypes = [_vp, _u64, _u32, _u64, _u32, _u32, _vp, _vp]
    L.smc_rng_normals.argtypes = [_vp, _u64, _u32, _u64, _u32, _u32, _vp, _vp]
    L.smc_measure_peak.argtypes = [_i32, _i32, _i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    for name in EXPORTS:
        if name != "smc_status_string":
            getattr(L, name).restype = _st


_lib = None


def load(path: str = LIB_PATH):
    """Load libsmc.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it first (python -m "
                               "paper_0905_2441_gb300.build or __graft_entry__.build())")
        L = C.CDLL(path)
        _declare(L)
        _lib = L
    return _lib
