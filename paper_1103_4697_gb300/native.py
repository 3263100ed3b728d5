"""ctypes declarations for libgbres.so (the C ABI in include/gbres.h).

Loading fails loudly: there is no CPU fallback for any computation.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgbres.so")

OK, EINVAL, ENOMEM, EDEVICE, ETIMEOUT, EAGAIN, EVERIFY, ELIMIT, ECANCELED, ENOTFOUND = range(10)
OPT_DROP_UNLUCKY, OPT_STATS, OPT_GRAPH, OPT_EXTRA_PRIMES, OPT_INTERP_GEMM, OPT_REGISTER_FORM, OPT_INTERP_TC, \
    OPT_PIPELINE, OPT_POINTS = (1, 2, 3, 4, 5, 6, 7, 8, 9)
JOB_RESULTANT, JOB_DISC, JOB_GCD = 0, 1, 2


class BiPoly(C.Structure):
    _fields_ = [("deg_x", C.c_int32), ("deg_y", C.c_int32), ("words", C.c_int32), ("coef", C.c_void_p)]


class UPoly(C.Structure):
    _fields_ = [("deg", C.c_int32), ("words", C.c_int32), ("coef", C.c_void_p)]


class BigPoly(C.Structure):
    _fields_ = [("deg", C.c_int32), ("limbs", C.c_int32), ("mag", C.POINTER(C.c_uint32)),
                ("sign", C.POINTER(C.c_int8))]


class BigBiPoly(C.Structure):
    _fields_ = [("deg_x", C.c_int32), ("deg_y", C.c_int32), ("c", BigPoly)]


class Sqf(C.Structure):
    _fields_ = [("unit", BigPoly), ("count", C.c_int32), ("factors", C.POINTER(BigPoly))]


class Stats(C.Structure):
    _fields_ = [("bounds_ms", C.c_double), ("reduce_ms", C.c_double), ("evalres_ms", C.c_double),
                ("interp_ms", C.c_double), ("crt_ms", C.c_double), ("gcd_ms", C.c_double),
                ("total_ms", C.c_double), ("kernels", C.c_int64), ("subproblems", C.c_int64),
                ("modmul", C.c_int64), ("modmul_evalres", C.c_int64), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64), ("dropped_points", C.c_int64), ("dropped_primes", C.c_int64),
                ("graph_replayed", C.c_int64), ("redo_warps", C.c_int64), ("root_pairs", C.c_int64),
                ("quad_pairs", C.c_int64)]


class Calib(C.Structure):
    _fields_ = [("modmul_per_s", C.c_double), ("mulsub_per_s", C.c_double), ("sm_clock_mhz", C.c_double),
                ("sms", C.c_int32), ("fma3_per_s", C.c_double), ("shoup_per_s", C.c_double)]


class ResInfo(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("deg_bound", C.c_int32), ("primes", C.c_int32),
                ("limbs", C.c_int32), ("log2_bound", C.c_double)]


class Job(C.Structure):
    _fields_ = [("kind", C.c_int32), ("var", C.c_int32), ("f", BiPoly), ("g", BiPoly), ("p", UPoly),
                ("q", UPoly)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("batches", C.c_int64),
                ("max_batch", C.c_int64), ("peak_bytes", C.c_int64), ("waits_for_memory", C.c_int64)]


# name -> (restype, argtypes); every symbol include/gbres.h declares
SIGNATURES = {
    "gbr_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t, C.c_void_p, C.c_void_p]),
    "gbr_destroy": (None, [C.c_void_p]),
    "gbr_strerror": (C.c_char_p, [C.c_int]),
    "gbr_last_error": (C.c_char_p, [C.c_void_p]),
    "gbr_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int64]),
    "gbr_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "gbr_resultant": (C.c_int, [C.c_void_p, C.POINTER(BiPoly), C.POINTER(BiPoly), C.c_int, C.POINTER(BigPoly)]),
    "gbr_discriminant_res": (C.c_int, [C.c_void_p, C.POINTER(BiPoly), C.c_int, C.POINTER(BigPoly)]),
    "gbr_gcd": (C.c_int, [C.c_void_p, C.POINTER(UPoly), C.POINTER(UPoly), C.POINTER(BigPoly)]),
    "gbr_resultant_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(BigPoly)]),
    "gbr_discriminant_res_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(BigPoly)]),
    "gbr_gcd_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(BigPoly)]),
    "gbr_mixed_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(BigPoly), C.c_int,
                                  C.c_void_p, C.c_void_p, C.POINTER(BigPoly)]),
    "gbr_gcd_cofactors_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(BigPoly),
                                          C.POINTER(BigPoly), C.POINTER(BigPoly)]),
    "gbr_gcd2_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(BigBiPoly),
                                 C.POINTER(BigBiPoly), C.POINTER(BigBiPoly)]),
    "gbr_free_bigbipoly": (None, [C.c_void_p, C.POINTER(BigBiPoly)]),
    "gbr_content_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(BigPoly)]),
    "gbr_teissier_res_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(BigPoly)]),
    "gbr_squarefree": (C.c_int, [C.c_void_p, C.POINTER(BigPoly), C.POINTER(Sqf)]),
    "gbr_squarefree_batch": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(BigPoly), C.POINTER(Sqf)]),
    "gbr_free_sqf": (None, [C.c_void_p, C.POINTER(Sqf)]),
    "gbr_upload_pairs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                   C.POINTER(C.c_void_p)]),
    "gbr_run_resident": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gbr_upload_arrangement": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "gbr_arrangement_resultants": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(BigPoly)]),
    "gbr_fetch_resident": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(BigPoly)]),
    "gbr_free_resident": (None, [C.c_void_p, C.c_void_p]),
    "gbr_free_result": (None, [C.c_void_p, C.POINTER(BigPoly)]),
    "gbr_submit": (C.c_int, [C.c_void_p, C.POINTER(Job), C.POINTER(C.c_uint64)]),
    "gbr_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(BigPoly), C.c_int]),
    "gbr_wait_any": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint64), C.POINTER(BigPoly),
                               C.POINTER(C.c_double)]),
    "gbr_clock": (C.c_double, []),
    "gbr_get_serve_stats": (C.c_int, [C.c_void_p, C.POINTER(ServeStats)]),
    "gbr_calibrate": (C.c_int, [C.c_void_p, C.POINTER(Calib)]),
    "gbr_crt_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int, C.c_void_p,
                                  C.c_void_p]),
    "gbr_num_primes": (C.c_int, []),
    "gbr_prime": (C.c_int, [C.c_int, C.POINTER(C.c_uint32)]),
    "gbr_primes_for_bits": (C.c_int, [C.c_double]),
    "gbr_resident_plan": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(ResInfo)]),
    "gbr_resultant_info": (C.c_int, [C.POINTER(BiPoly), C.POINTER(BiPoly), C.c_int, C.c_int, C.POINTER(ResInfo)]),
}

_lib = None
_missing: list[str] = []


def missing_symbols() -> list[str]:
    lib()
    return list(_missing)


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name, None)
            if fn is None:
                _missing.append(name)
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GbrError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"gbres error {status}: {msg}")


def check(status: int, ctx=None) -> None:
    if status != OK:
        L = lib()
        text = L.gbr_strerror(status).decode()
        if ctx is not None:
            detail = L.gbr_last_error(ctx)
            if detail:
                text += " (" + detail.decode() + ")"
        raise GbrError(status, text)
