"""ctypes binding of ``liblmep.so`` (include/lmep.h).

Argument marshalling only: every function forwards to the C entry point of
the same name.  The library must have been built (``build.build()``); there is
no fallback of any kind -- a missing library raises at load time.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblmep.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lmep.h")

OK, ERR_INVALID, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_NOMEM = range(7)
BC = {"periodic": 0, "dirichlet": 1, "neumann": 2}
PREC = {"fp64": 0, "mixed": 1}
SCHEME = {"linear": 0, "etd1": 1, "etdrk2": 2, "etdrk4": 3}
NONLIN = {"none": 0, "allen_cahn": 1, "kdv": 2, "burgers": 3}
EXPM = {"auto": 0, "pade": 1, "series": 2}


class LmepGrid(C.Structure):
    _fields_ = [("N", C.c_int64), ("h", C.c_double), ("bc", C.c_int32), ("n", C.c_int32),
                ("departure_centring", C.c_int32), ("batch", C.c_int32), ("window_shift", C.c_int32),
                ("reserved", C.c_int32), ("bc_lo", C.c_double), ("bc_hi", C.c_double)]


class LmepOperator(C.Structure):
    _fields_ = [("c0", C.c_double), ("c1", C.c_double), ("c2", C.c_double), ("c3", C.c_double),
                ("frozen_adv", C.c_double)]


class LmepBatchDesc(C.Structure):
    _fields_ = [("B", C.c_int64), ("N_host", C.POINTER(C.c_int64)), ("h_host", C.POINTER(C.c_double)),
                ("bc_host", C.POINTER(C.c_int32)), ("n", C.c_int32), ("scheme", C.c_int32),
                ("nonlin", C.c_int32), ("tile", C.c_int32), ("block", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("dt", C.c_double), ("op", LmepOperator)]


class LmepFrozenSetDesc(C.Structure):
    _fields_ = [("B", C.c_int64), ("grids_host", C.POINTER(LmepGrid)), ("ops_host", C.POINTER(LmepOperator)),
                ("dt_host", C.POINTER(C.c_double)), ("block", C.c_int32), ("points_per_thread", C.c_int32)]


class LmepError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_P = C.c_void_p
_SIGS = {
    "lmep_create": [C.POINTER(_P)],
    "lmep_destroy": [_P],
    "lmep_build_operator": [_P, C.POINTER(LmepGrid), C.POINTER(LmepOperator), C.c_double, C.c_int32, _P,
                            C.c_int64, C.c_int64, _P, _P, _P, _P],
    "lmep_expm": [_P, _P, C.c_int64, C.c_int32, _P, C.c_int32, _P, _P],
    "lmep_harvest_weights": [_P, C.POINTER(LmepGrid), C.POINTER(LmepOperator), C.c_double, C.c_int32, _P,
                             _P, C.c_int32, _P],
    "lmep_harvest_scheme_weights": [_P, C.POINTER(LmepGrid), C.POINTER(LmepOperator), C.c_double, C.c_int32, _P,
                                    C.c_int32, _P],
    "lmep_step": [_P, C.POINTER(LmepGrid), C.POINTER(LmepOperator), C.c_int32, C.c_int32, C.c_double, _P,
                  _P, _P, C.c_int64, C.c_int32, _P],
    "lmep_batch_workspace_bytes": [C.POINTER(LmepBatchDesc), C.c_int32, C.POINTER(C.c_size_t)],
    "lmep_batch_prepare": [_P, C.POINTER(LmepBatchDesc), _P, C.c_size_t, C.c_int32, _P],
    "lmep_step_batched": [_P, _P, _P, _P, C.c_int64, _P],
    "lmep_step_batched_once": [_P, _P, _P, _P, _P],
    "lmep_frozen_set_workspace_bytes": [C.POINTER(LmepFrozenSetDesc), C.c_int32, C.POINTER(C.c_size_t)],
    "lmep_frozen_set_prepare": [_P, C.POINTER(LmepFrozenSetDesc), _P, C.c_size_t, C.c_int32, _P],
    "lmep_frozen_set_refresh": [_P, _P, _P],
    "lmep_frozen_set_step_once": [_P, _P, _P, _P, _P],
    "lmep_adjoint_scratch_bytes": [C.POINTER(LmepGrid), C.c_int32, C.POINTER(C.c_size_t)],
    "lmep_adjoint_step": [_P, C.POINTER(LmepGrid), C.POINTER(LmepOperator), C.c_double, _P, _P, _P, _P, _P,
                          C.c_size_t, C.c_int32, _P],
    "lmep_adjoint_step_noalloc": [C.POINTER(LmepGrid), C.POINTER(LmepOperator), C.c_double, _P, _P, _P, _P,
                                  C.c_int32, _P],
    "lmep_frozen_stats": [_P, C.POINTER(LmepGrid), C.POINTER(LmepOperator), C.c_double, _P, _P, C.c_int32, _P],
    "lmep_set_expm_method": [_P, C.c_int32],
    "lmep_set_wait_limit": [_P, C.c_int64],
    "lmep_sync_status": [_P, _P],
    "lmep_fma_peak": [C.c_int32, C.POINTER(C.c_double)],
    "lmep_harvest_nodes": [_P, C.c_int64, _P, C.c_int32, C.POINTER(LmepOperator), C.c_double, C.c_int32, _P,
                           C.c_int32, _P],
    "lmep_step_nodes": [_P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, _P,
                        _P, _P, C.c_int64, C.c_int32, _P],
    "lmep_amplification": [_P, C.c_int32, C.c_int32, _P, C.c_int64, _P, _P],
    "lmep_status_string": [C.c_int],
    "lmep_last_error": [],
    "lmep_version": [],
}
_STRING_RESULT = {"lmep_status_string", "lmep_last_error", "lmep_version"}

_lib = None


def declared_symbols(header: str = HEADER) -> list[str]:
    """Names of every entry point declared with LMEP_API in include/lmep.h."""
    with open(header) as f:
        text = f.read()
    return sorted(set(re.findall(r"LMEP_API\s+[\w\s\*]+?\b(lmep_\w+)\s*\(", text)))


def load() -> C.CDLL:
    """Load liblmep.so once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2603_15964_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name in _STRING_RESULT else C.c_int
    _lib = lib
    return lib


def check(status: int, where: str) -> None:
    if status != OK:
        lib = load()
        raise LmepError(status, where, lib.lmep_last_error().decode() or lib.lmep_status_string(status).decode())


def call(name: str, *args) -> None:
    check(getattr(load(), name)(*args), name)
