"""ctypes declarations of the C ABI in include/ns.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_lib = None

P = ctypes.c_void_p
U64 = ctypes.c_uint64
I32 = ctypes.c_int
ST = ctypes.c_int  # ns_status


class NsConfig(ctypes.Structure):
    _fields_ = [("path", I32), ("hbm_budget_bytes", U64), ("max_slots", I32), ("tuner_cache", ctypes.c_char_p),
                ("cta_cache", I32), ("column_sort", I32), ("hash_load", ctypes.c_double), ("sort_split", I32),
                ("sort_tile", I32), ("sort_digits", I32)]


class NsStats(ctypes.Structure):
    _fields_ = [(f, U64) for f in (
        "valid_packets", "unique_links", "unique_sources", "unique_destinations",
        "max_src_packets", "max_src_fanout", "max_dst_packets", "max_dst_fanin", "max_link_packets")]


FIELDS = tuple(f for f, _ in NsStats._fields_)


class NsBatchParams(ctypes.Structure):
    _fields_ = [("tile_packets", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32), ("max_load", ctypes.c_double),
                ("cta_cache", ctypes.c_uint32)]


class NsStreamTiming(ctypes.Structure):
    _fields_ = [("submit_us", ctypes.c_double), ("admit_us", ctypes.c_double), ("complete_us", ctypes.c_double),
                ("window_id", U64)]


class NsTraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", U64), ("total_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double)]

# name -> (restype, argtypes)
SIGNATURES = {
    "ns_create": (ST, [ctypes.POINTER(P), ctypes.POINTER(NsConfig), I32]),
    "ns_destroy": (None, [P]),
    "ns_sync": (ST, [P, P]),
    "ns_matrix_create": (ST, [P, ctypes.POINTER(P)]),
    "ns_matrix_reserve": (ST, [P, U64, P]),
    "ns_matrix_clear": (ST, [P, P]),
    "ns_matrix_free": (None, [P]),
    "ns_matrix_nnz": (ST, [P, ctypes.POINTER(U64), P]),
    "ns_matrix_export": (ST, [P, P, P, U64, ctypes.POINTER(U64), P]),
    "ns_window_build": (ST, [P, P, P, U64, P, P]),
    "ns_window_build_host": (ST, [P, P, P, U64, P, ctypes.POINTER(NsStats), P]),
    "ns_path_tune": (ST, [P, P, P, U64, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                          ctypes.POINTER(ctypes.c_float)]),
    "ns_path_resolve": (ST, [P, U64, ctypes.POINTER(ctypes.c_int)]),
    "ns_sort_resolve": (ST, [P, U64, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
    "ns_sort_split_info": (ST, [P, ctypes.POINTER(I32), ctypes.POINTER(U64), ctypes.POINTER(U64), P]),
    "ns_column_split_info": (ST, [P, ctypes.POINTER(I32), ctypes.POINTER(U64), ctypes.POINTER(U64), P]),
    "ns_matrix_nodes": (ST, [P, P, ctypes.c_int, P, P, P, U64, ctypes.POINTER(U64), P]),
    "ns_anonymize": (ST, [P, P, P, U64, P, U64, P, P, ctypes.POINTER(U64), P]),
    "ns_server_reserve": (ST, [P, U64]),
    "ns_server_clear": (ST, [P]),
    "ns_slider_create": (ST, [P, ctypes.c_uint32, ctypes.POINTER(P)]),
    "ns_slider_free": (None, [P]),
    "ns_slider_push": (ST, [P, P, P, P, U64, P, P, P]),
    "ns_slider_matrix": (ST, [P, ctypes.POINTER(P)]),
    "ns_accumulate": (ST, [P, P, P, P]),
    "ns_window_ingest": (ST, [P, P, P, P, U64, P]),
    "ns_window_ingest_stats": (ST, [P, P, P, P, U64, P, P]),
    "ns_network_stats": (ST, [P, P, ctypes.POINTER(NsStats), P]),
    "ns_network_stats_async": (ST, [P, P, P, P]),
    "ns_window_stats_static": (ST, [P, P, U64, P, P]),
    "ns_trace_enable": (ST, [P, I32]),
    "ns_trace_read": (ST, [P, ctypes.POINTER(NsTraceEntry), I32, ctypes.POINTER(I32)]),
    "ns_matrix_reserve_ex": (ST, [P, U64, U64, P]),
    "ns_matrix_save": (ST, [P, ctypes.c_char_p, P]),
    "ns_owner": (ctypes.c_uint32, [ctypes.c_uint32, ctypes.c_uint32]),
    "ns_matrix_partition": (ST, [P, P, I32, ctypes.c_uint32, P, P, U64, ctypes.POINTER(U64), P]),
    "ns_matrix_add_entries": (ST, [P, P, P, P, U64, P]),
    "ns_matrix_load": (ST, [P, ctypes.c_char_p, P, P]),
    "ns_batch_create": (ST, [P, U64, U64, ctypes.POINTER(P)]),
    "ns_batch_free": (None, [P]),
    "ns_batch_get_params": (ST, [P, ctypes.POINTER(NsBatchParams)]),
    "ns_batch_set_params": (ST, [P, ctypes.POINTER(NsBatchParams)]),
    "ns_batch_run": (ST, [P, P, P, P, ctypes.POINTER(U64), U64, P, P, P]),
    "ns_batch_tune": (ST, [P, P, P, P, ctypes.POINTER(U64), U64, P, P, ctypes.POINTER(NsBatchParams)]),
    "ns_batch_run_device": (ST, [P, P, P, P, P, U64, P, P, P]),
    "ns_batch_sync": (ST, [P, P]),
    "ns_server_create": (ST, [P, P, ctypes.POINTER(P)]),
    "ns_server_destroy": (None, [P]),
    "ns_stream_submit": (ST, [P, P, P, U64, U64, ctypes.POINTER(U64)]),
    "ns_stream_poll": (ST, [P, U64, ctypes.POINTER(I32)]),
    "ns_stream_wait": (ST, [P, U64, ctypes.POINTER(NsStats), ctypes.POINTER(NsStats), ctypes.c_int64,
                           ctypes.POINTER(NsStreamTiming)]),
    "ns_diag_wait_timeout": (ST, [I32, P]),
    "ns_diag_random_atomics": (ST, [U64, U64, I32, ctypes.POINTER(ctypes.c_double), P]),
    "ns_diag_random_claims": (ST, [U64, U64, I32, I32, ctypes.POINTER(ctypes.c_double), P]),
    "ns_last_error": (ctypes.c_char_p, []),
    "ns_status_string": (ctypes.c_char_p, [ST]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libns.so (building it first if it is missing or stale and nvcc is
    available).  Raises if the library cannot be loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libns.so is not built; run python -m paper_2509_03653_b300.build")
    L = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class NsError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = load()
        self.status = status
        self.name = L.ns_status_string(status).decode()
        self.message = L.ns_last_error().decode()
        super().__init__(f"{where}: {self.name}: {self.message}")


def check(status: int, where: str):
    if status != 0:
        raise NsError(status, where)
