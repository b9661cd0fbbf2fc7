"""ctypes loader for libsgp.so, the sm_103a lattice library (C-ABI in include/sgp.h and
include/sgp_serve.h).

This module only declares the C signatures.  It never substitutes another
implementation: if the library is missing, loading fails with an error.
"""

from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsgp.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
HEADERS = [os.path.join(INCLUDE, "sgp.h"), os.path.join(INCLUDE, "sgp_serve.h")]

SGP_OK = 0
STATUS_NAMES = {0: "SGP_OK", 1: "SGP_ERR_INVALID_ARG", 2: "SGP_ERR_OOM", 3: "SGP_ERR_RANGE",
                4: "SGP_ERR_HASH_FULL", 5: "SGP_ERR_NONFINITE", 6: "SGP_ERR_CUDA",
                7: "SGP_ERR_TIMEOUT"}

KERNELS = {"rbf_binomial": 0, "rbf_coverage": 1, "matern32_coverage": 2}
BLURS = {"sequential": 0, "transpose": 1, "symmetric": 2}
GRADS = {"lattice": 0, "filter": 1}
VALUE_DTYPES = {"f32": 0, "bf16": 1}


class sgp_opts(ctypes.Structure):
    _fields_ = [("order_r", ctypes.c_int), ("kernel", ctypes.c_int),
                ("spacing_s", ctypes.c_double), ("outputscale", ctypes.c_float),
                ("value_dtype", ctypes.c_int), ("check_every", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("precond_rank", ctypes.c_int),
                ("precond_seed", ctypes.c_ulonglong), ("precond_power_iters", ctypes.c_int)]


class sgp_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_ulonglong), ("max_active", ctypes.c_int),
                ("probes", ctypes.c_int), ("order_r", ctypes.c_int), ("kernel", ctypes.c_int),
                ("spacing_s", ctypes.c_double), ("value_dtype", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("check_every", ctypes.c_int), ("precond_rank", ctypes.c_int),
                ("precond_min_kappa", ctypes.c_double), ("lane_classes", ctypes.c_int)]


class sgp_request(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n", ctypes.c_longlong),
                ("Xs", ctypes.c_void_p), ("ns", ctypes.c_longlong), ("d", ctypes.c_int),
                ("lengthscales", ctypes.c_void_p), ("outputscale", ctypes.c_float),
                ("noise", ctypes.c_float), ("seed", ctypes.c_ulonglong),
                ("mean", ctypes.c_void_p), ("var", ctypes.c_void_p),
                ("arrival_us", ctypes.c_double), ("timeout_us", ctypes.c_double),
                ("lattice_key", ctypes.c_ulonglong)]


class sgp_request_stats(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("arrival_us", ctypes.c_double),
                ("admit_us", ctypes.c_double), ("done_us", ctypes.c_double),
                ("m", ctypes.c_longlong), ("bytes", ctypes.c_ulonglong),
                ("setup_us", ctypes.c_double), ("lattice_reused", ctypes.c_int),
                ("precond_rank", ctypes.c_int), ("kappa_est", ctypes.c_double),
                ("value_dtype", ctypes.c_int)]


class SGPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


_lib = None


def declared_functions() -> list:
    """Names of the functions the headers under include/ declare."""
    names = set()
    for header in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(header).read(), flags=re.S)
        names.update(re.findall(r"\b(sgp_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def load():
    """Load libsgp.so (built by paper_2106_06695_gb300.build_lib) and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsgp.so is not built; run paper_2106_06695_gb300.build_lib.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I, I64, F, Dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    sigs = {
        "sgp_opts_init": (None, [ctypes.POINTER(sgp_opts)]),
        "sgp_stencil": (I, [I, I, Dbl, ctypes.POINTER(Dbl), P, P]),
        "sgp_lattice_build": (I, [P, P, I64, I, ctypes.POINTER(sgp_opts), ctypes.POINTER(P)]),
        "sgp_lattice_info": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_size_t)]),
        "sgp_lattice_stencil": (I, [P, ctypes.POINTER(I), ctypes.POINTER(Dbl), P, P]),
        "sgp_lattice_blur_lists": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I64)]),
        "sgp_lattice_export": (I, [P, P, P, P]),
        "sgp_set_stream": (I, [P, P]),
        "sgp_mvm": (I, [P, P, I, P]),
        "sgp_mvm_ex": (I, [P, P, I, I, F, F, P]),
        "sgp_mvm_static": (I, [P, P, I, I, F, F, P]),
        "sgp_cg_solve": (I, [P, P, I, F, F, I, P, P, P]),
        "sgp_mvm_backward": (I, [P, P, P, P, P, I, I, F, I, P, P, P]),
        "sgp_logdet": (I, [P, P, I, F, I, F, ctypes.POINTER(Dbl), P]),
        "sgp_cg_solve_ex": (I, [P, P, I, I, F, F, I, P, P, P]),
        "sgp_cg_solve_history": (I, [P, P, I, I, F, F, I, P, P, P, P]),
        "sgp_lattice_free": (None, [P]),
        "sgp_profile_blur": (I, [P, I]),
        "sgp_profile_read": (I, [P, ctypes.POINTER(Dbl), ctypes.POINTER(I64)]),
        "sgp_profile_read_stages": (I, [P, P, ctypes.POINTER(I64)]),
        "sgp_kernel_launches": (I64, []),
        "sgp_trim_memory": (I, []),
        "sgp_last_error": (ctypes.c_char_p, []),
        "sgp_version": (I, []),
        "sgp_server_opts_init": (None, [ctypes.POINTER(sgp_server_opts)]),
        "sgp_request_bytes_bound": (ctypes.c_ulonglong, [ctypes.c_longlong, I, I, I, I, I]),
        "sgp_server_create": (I, [ctypes.POINTER(sgp_server_opts), ctypes.POINTER(P)]),
        "sgp_server_submit": (I, [P, ctypes.POINTER(sgp_request),
                                  ctypes.POINTER(ctypes.c_longlong)]),
        "sgp_server_step": (I, [P, ctypes.POINTER(I)]),
        "sgp_server_stats": (I, [P, ctypes.c_longlong, ctypes.POINTER(sgp_request_stats)]),
        "sgp_server_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I),
                                ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(I)]),
        "sgp_server_clock_us": (Dbl, [P]),
        "sgp_server_cache_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_ulonglong)]),
        "sgp_server_destroy": (None, [P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != SGP_OK:
        raise SGPError(status, load().sgp_last_error().decode(errors="replace"))
