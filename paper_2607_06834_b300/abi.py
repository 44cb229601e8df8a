"""ctypes declarations of the C ABI in include/ptahmc.h (argument marshalling only).

Importing this module loads the in-tree libptahmc.so (its check build libptahmc_check.so
when PTA_CHECK_BUILD=1) and raises ImportError if it is missing: there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libptahmc_check.so" if os.environ.get("PTA_CHECK_BUILD") == "1" else "libptahmc.so")

PTA_OK, PTA_EINVAL, PTA_ESTATE, PTA_ECUDA, PTA_ENOMEM, PTA_ETIMEOUT, PTA_ECHECK = 0, -1, -2, -3, -4, -5, -6
PREC = {"fp64": 0, "fp32": 1, "tf32x3": 2, "tf32": 3, "bf16x3": 4, "gram": 5, "f16split": 6}
TRANSFORM = {"prior": 0, "curn": 1}
CHOLESKY = {"dw": 0, "fp64": 1}

EXPORTED = ["pta_create", "pta_add_pulsar", "pta_finalize", "pta_layout", "pta_set_precision",
            "pta_set_hyperprior", "pta_logp_and_grad", "pta_hmc_trajectory", "pta_logp_constant",
            "pta_profile_enable", "pta_profile_read", "pta_logp_and_grad_noalloc", "pta_autotune",
            "pta_set_toa_config", "pta_toa_config_info", "pta_debug_inject", "pta_set_beta", "pta_set_transform",
            "pta_set_cholesky",
            "pta_param_bounds", "pta_last_error", "pta_destroy"]
NSTAGES = 8
STAGES = ["prior_forward", "toa", "epilogue", "adjoint", "final"]
# single kernels timed inside those stages (not part of the stage sum)
KERNEL_TIMERS = ["chol_forward", "toa_res", "toa_ftw"]


class ModelDesc(C.Structure):
    _fields_ = [("n_gwb", C.c_int), ("n_rn", C.c_int), ("n_dm", C.c_int), ("cw", C.c_int),
                ("precision", C.c_int), ("nu_ref_mhz", C.c_double), ("spectrum", C.c_int)]


class PulsarDesc(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("n_backend", C.c_int),
                ("toas_s", C.POINTER(C.c_double)), ("freqs_mhz", C.POINTER(C.c_double)),
                ("resid_s", C.POINTER(C.c_double)), ("sigma_s", C.POINTER(C.c_double)),
                ("backend", C.POINTER(C.c_int32)), ("efac", C.POINTER(C.c_double)),
                ("equad_s", C.POINTER(C.c_double)), ("M", C.POINTER(C.c_double)),
                ("pos", C.c_double * 3), ("dist_kpc", C.c_double)]


class Layout(C.Structure):
    _fields_ = [("npsr", C.c_int), ("n_ach", C.c_int), ("n_dm", C.c_int), ("P", C.c_int),
                ("d_z", C.c_int), ("d", C.c_int), ("z_ach", C.c_int), ("z_dm", C.c_int),
                ("th_rn", C.c_int), ("th_dm", C.c_int), ("th_gwb", C.c_int), ("th_cw", C.c_int),
                ("ntoa", C.c_longlong), ("tspan_s", C.c_double), ("t0_s", C.c_double),
                ("n_th_rn", C.c_int), ("n_th_gwb", C.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run `python -m paper_2607_06834_b300.build` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i32p, f64p, f32p = C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p
    lib.pta_create.argtypes = [C.POINTER(vp), C.POINTER(ModelDesc)]
    lib.pta_add_pulsar.argtypes = [vp, C.POINTER(PulsarDesc)]
    lib.pta_finalize.argtypes = [vp, vp]
    lib.pta_layout.argtypes = [vp, C.POINTER(Layout)]
    lib.pta_set_precision.argtypes = [vp, C.c_int]
    lib.pta_set_hyperprior.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double]
    lib.pta_logp_and_grad.argtypes = [vp, C.c_int, f32p, f64p, f32p, i32p, vp]
    lib.pta_logp_and_grad_noalloc.argtypes = [vp, C.c_int, f32p, f64p, f32p, i32p, vp]
    lib.pta_hmc_trajectory.argtypes = [vp, C.c_int, f32p, f64p, f32p, f32p, f32p, C.c_int,
                                       C.c_uint64, C.c_uint64, i32p, vp]
    lib.pta_logp_constant.argtypes = [vp, C.POINTER(C.c_double)]
    lib.pta_profile_enable.argtypes = [vp, C.c_int]
    lib.pta_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]
    lib.pta_autotune.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int]
    lib.pta_set_toa_config.argtypes = [vp, C.c_int]
    lib.pta_debug_inject.argtypes = [vp, C.c_int]
    lib.pta_set_beta.argtypes = [vp, C.c_int, vp, vp]
    lib.pta_set_transform.argtypes = [vp, C.c_int]
    lib.pta_set_cholesky.argtypes = [vp, C.c_int]
    lib.pta_param_bounds.argtypes = [vp, vp, vp]
    lib.pta_toa_config_info.argtypes = [C.c_int] + [C.POINTER(C.c_int)] * 4
    lib.pta_last_error.argtypes = [vp]
    lib.pta_last_error.restype = C.c_char_p
    lib.pta_destroy.argtypes = [vp]
    lib.pta_destroy.restype = None
    for name in EXPORTED:
        if name not in ("pta_last_error", "pta_destroy"):
            getattr(lib, name).restype = C.c_int
    return lib


lib = _load()
