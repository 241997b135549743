"""ctypes declarations of libtera.so (include/tera.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# TERA_DEBUG_BOUNDS=1 in the environment selects the bounds-checking build
# (libtera_debug.so, `build.build(debug_bounds=True)`): the same kernels with
# every write checked against the range its pair or buffer owns
DEBUG_BOUNDS = os.environ.get("TERA_DEBUG_BOUNDS", "") == "1"
LIB_PATH = os.path.join(HERE, "libtera_debug.so" if DEBUG_BOUNDS else "libtera.so")

OK, EINVAL, ENOMEM, ECAPACITY, ECORRUPT, EDOMAIN, EREFMISMATCH, ETIMEOUT, ECUDA, EBOUNDS = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECAPACITY", "ECORRUPT", "EDOMAIN", "EREFMISMATCH",
                "ETIMEOUT", "ECUDA", "EBOUNDS"]
MODE_RAW, MODE_XOR, MODE_RESIDUAL = 0, 1, 2
MLP_PARAMS = 4931
HIST_BYTES = 48
SAMPLE_FLOATS = 12


class TeraError(RuntimeError):
    def __init__(self, status: int, where: str, required: int | None = None):
        self.status = status
        self.required = required
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        extra = f" (required capacity {required})" if required else ""
        super().__init__(f"{where}: {name}{extra}")


class Grid(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n", C.c_int32 * 3),
                ("w", C.c_double), ("periodic", C.c_uint32), ("reserved", C.c_uint32)]


class Soa(C.Structure):
    _fields_ = [("id", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("diameter", C.c_void_p), ("volume", C.c_void_p), ("adherence", C.c_void_p),
                ("density", C.c_void_p), ("n", C.c_int64)]


class PartitionOut(C.Structure):
    _fields_ = [("owner", C.c_void_p), ("mask", C.c_void_p), ("pair_count", C.c_void_p),
                ("pair_off", C.c_void_p), ("pair_idx", C.c_void_p), ("idx_capacity", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("iterations", "agents", "records", "ref_slots", "holes",
                                          "new_records", "payload_bytes", "wire_bytes")]


class Tune(C.Structure):
    _fields_ = [("block", C.c_int), ("ctas_per_sm", C.c_int), ("table_records", C.c_int),
                ("team_blocks", C.c_int), ("wait_limit_us", C.c_int), ("reserved", C.c_int)]


class Ids(C.Structure):
    _fields_ = [("msg", C.c_void_p), ("ref_prev", C.c_void_p), ("ref_next", C.c_void_p)]


class Predictor(C.Structure):
    _fields_ = [("params", C.c_void_p), ("hist_prev", C.c_void_p), ("hist_next", C.c_void_p),
                ("samples", C.c_void_p), ("allow_residual", C.c_int)]


# name -> (restype, argtypes); every symbol include/tera.h declares
P, u32, u64, i64 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int64
SIGNATURES = {
    "tera_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Grid), C.c_int, u32]),
    "tera_ctx_destroy": (C.c_int, [P]),
    "tera_n_pairs": (u64, [P]),
    "tera_ctx_reserve": (C.c_int, [P, i64, u64]),
    "tera_partition": (C.c_int, [P, C.POINTER(Soa), C.POINTER(PartitionOut), P]),
    "tera_pack": (C.c_int, [P, C.POINTER(Soa), C.POINTER(PartitionOut), u32, u32, P, u64, P]),
    "tera_pack_ids": (C.c_int, [P, C.POINTER(Soa), C.POINTER(PartitionOut), P, u64, P, P]),
    "tera_codec_batched_ids": (C.c_int, [P, P, P, P, P, P, P, u64, P, P, P, P, P, u64, P,
                                         C.c_int, C.POINTER(Tune), C.POINTER(Ids), P]),
    "tera_delta_encode": (C.c_int, [P, P, P, P, P, u32, u32, P, P, u64, P, P, C.c_int, P]),
    "tera_delta_decode": (C.c_int, [P, P, P, P, P, u32, u32, P, u64, P, P]),
    "tera_delta_decode_noalloc": (C.c_int, [P, P, P, P, u64, u32, P, u64, P,
                                            C.POINTER(C.c_uint64), P]),
    "tera_codec_batched": (C.c_int, [P, P, P, P, P, P, P, u64, P, P, P, P, P, u64, P, C.c_int,
                                     C.POINTER(Tune), P]),
    "tera_delta_encode_pred": (C.c_int, [P, P, P, P, P, u32, u32, P, P, u64, P, P, C.c_int,
                                         C.POINTER(Predictor), P]),
    "tera_delta_decode_pred": (C.c_int, [P, P, P, P, P, u32, u32, P, u64, P,
                                         C.POINTER(Predictor), P]),
    "tera_codec_batched_pred": (C.c_int, [P, P, P, P, P, P, P, u64, P, P, P, P, P, u64, P,
                                          C.c_int, C.POINTER(Tune), C.POINTER(Predictor),
                                          C.POINTER(Predictor), P]),
    "tera_mlp_grad": (C.c_int, [P, P, u64, P, P, C.POINTER(C.c_uint64), P]),
    "tera_mlp_train": (C.c_int, [P, P, u64, P, C.c_int, C.c_int, C.c_float, C.c_float,
                                 C.POINTER(C.c_uint64), P]),
    "tera_unpack_inplace": (C.c_int, [P, u64, u32, C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_uint64), P]),
    "tera_unpack_validate": (C.c_int, [P, P, P, P]),
    "tera_wire_to_host": (C.c_int, [P, P, P, P, u64, P, P]),
    # tera_soa_mut has the layout of tera_soa
    "tera_migrate_send": (C.c_int, [P, C.POINTER(Soa), P, P, u64, P, C.POINTER(Soa), P, P]),
    "tera_migrate_recv": (C.c_int, [P, P, u64, P, P, C.POINTER(Soa), P]),
    "tera_ctx_status": (C.c_int, [P, C.POINTER(C.c_uint64), P]),
    "tera_reset_reference": (C.c_int, [P, u32]),
    "tera_ctx_launches": (u64, [P]),
    "tera_ctx_stats": (C.c_int, [P, C.POINTER(Stats), C.c_int, P]),
    "tera_ctx_profile": (C.c_int, [P, C.c_int]),
    "tera_ctx_profile_collect": (C.c_int, [P]),
    "tera_ctx_profile_entries": (C.c_int, [P]),
    "tera_ctx_profile_entry": (C.c_int, [P, C.c_int, C.POINTER(C.c_char_p),
                                         C.POINTER(C.c_uint64), C.POINTER(C.c_double)]),
    "tera_ctx_profile_reset": (C.c_int, [P]),
    "tera_version": (C.c_char_p, []),
    "tera_ref_schedule": (C.c_int, [u64, u32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_uint64)]),
    "tera_cell_thresholds": (C.c_int, [C.c_double, C.c_double, C.c_double, u64, P]),
    "tera_axis_buckets": (C.c_int, [C.POINTER(Grid), P, P, P, C.POINTER(C.c_int)]),
}

_lock = threading.Lock()
_lib = None


def load():
    """Load the in-tree libtera.so.  Fails loudly if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU path)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int, where: str):
    if status != OK:
        raise TeraError(status, where)
