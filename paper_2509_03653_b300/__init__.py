"""B300-native traffic-matrix engine for the network-sensing graph challenge.

Python binding of the C ABI in include/ns.h, with the same names.  Every step
of the path runs in the CUDA library (libns.so, built for sm_103a); this
module only marshals arguments: torch tensors supply device pointers and
torch streams supply cudaStream_t handles.  If the library is missing or
cannot be loaded, every call raises -- there is no CPU fallback.

Quantities (the paper's Table 2, matrix notation) come back as a dict with
the keys in ``FIELDS``.
"""
from __future__ import annotations

import ctypes
import os

import torch

from ._native import (FIELDS, NsBatchParams, NsConfig, NsError, NsStats, NsStreamTiming, NsTraceEntry, check,
                      load)

__all__ = [
    "FIELDS", "NsError", "Context", "Matrix", "window_build", "window_build_host", "accumulate", "window_ingest",
    "window_ingest_stats", "network_stats", "network_stats_async", "matrix_export", "matrix_nnz", "matrix_reserve",
    "matrix_clear", "sync", "PATHS", "SORT_TILES", "SORT_DIGITS", "path_tune", "path_resolve", "sort_resolve", "sort_split_info", "matrix_nodes", "NODES", "anonymize", "Slider",
    "slider_push", "window_stats_static", "STATIC_MAX_PACKETS",
    "trace_enable", "trace_read", "Batch", "batch_run", "batch_run_device", "batch_sync", "batch_tune", "matrix_reserve_ex",
    "owner", "matrix_partition", "matrix_add_entries", "Server", "stream_submit", "stream_poll", "stream_wait", "diag_random_atomics", "diag_random_claims", "column_split_info", "matrix_save", "matrix_load",
]

STATIC_MAX_PACKETS = 32768  # NS_STATIC_MAX_PACKETS in include/ns.h

PATHS = {"auto": 0, "sort": 1, "hash": 2}
# digit-pass tiles of the sort path (ns_config.sort_tile): threads x keys per thread
SORT_TILES = {"auto": 0, "512x16": 1, "512x12": 2, "256x16": 3}
# digit plan of the sort path's 64-bit radix sorts (ns_config.sort_digits):
# eight 8-bit passes, or "wide": one 10-bit pass, then six 9-bit passes
SORT_DIGITS = {"auto": 0, "8": 1, "wide": 2}


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _column(t: torch.Tensor, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.element_size() != 4 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous 32-bit tensor (uint32/int32)")
    if t.numel() and not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    return ctypes.c_void_p(t.data_ptr() if t.numel() else 0)


class Context:
    """A library context on one CUDA device (ns_create / ns_destroy)."""

    def __init__(self, device: int = 0, path: str = "auto", hbm_budget_bytes: int = 0,
                 max_slots: int = 0, tuner_cache: str | None = None, cta_cache: str = "auto",
                 column_sort: str = "auto", hash_load: float = 0.0, sort_split: str = "auto",
                 sort_tile: str = "auto", sort_digits: str = "auto"):
        self._L = load()
        cfg = NsConfig(PATHS[path], hbm_budget_bytes, max_slots,
                       tuner_cache.encode() if tuner_cache else None, {"auto": 0, "on": 1, "off": 2}[cta_cache],
                       {"auto": 0, "pairs": 1}[column_sort], hash_load, {"auto": 0, "on": 1, "off": 2}[sort_split],
                       SORT_TILES[sort_tile], SORT_DIGITS[sort_digits])
        h = ctypes.c_void_p()
        check(self._L.ns_create(ctypes.byref(h), ctypes.byref(cfg), device), "ns_create")
        self.handle = h
        self.device = device
        self.path = path

    def close(self):
        if getattr(self, "handle", None):
            self._L.ns_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """A library-owned traffic matrix (ns_matrix_create / ns_matrix_free)."""

    def __init__(self, ctx: Context):
        self._L = ctx._L
        self.ctx = ctx
        h = ctypes.c_void_p()
        check(self._L.ns_matrix_create(ctx.handle, ctypes.byref(h)), "ns_matrix_create")
        self.handle = h

    def free(self):
        if getattr(self, "handle", None):
            self._L.ns_matrix_free(self.handle)
            self.handle = None

    def live(self):
        """The handle, while this matrix and its context are both open (the
        library would otherwise reach the closed context's freed memory)."""
        if not getattr(self, "handle", None):
            raise RuntimeError("the matrix has been freed")
        if not getattr(self.ctx, "handle", None):
            raise RuntimeError("the matrix's context has been closed")
        return self.handle

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def window_build(ctx: Context, src: torch.Tensor, dst: torch.Tensor, out: Matrix, stream=None):
    """out := A_t of one window (ns_window_build)."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("src and dst differ in length")
    check(ctx._L.ns_window_build(ctx.handle, _column(src, "src"), _column(dst, "dst"), n, out.live(),
                                 _stream(stream)), "ns_window_build")


def _host_column(t, name: str) -> ctypes.c_void_p:
    if isinstance(t, torch.Tensor):
        if t.element_size() != 4 or not t.is_contiguous() or t.is_cuda:
            raise ValueError(f"{name} must be a contiguous 32-bit host tensor")
        return ctypes.c_void_p(t.data_ptr() if t.numel() else 0)
    import numpy as np
    if not isinstance(t, np.ndarray) or t.dtype.itemsize != 4 or not t.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name} must be a contiguous 32-bit host array")
    return ctypes.c_void_p(t.ctypes.data if t.size else 0)


def window_build_host(ctx: Context, src, dst, out: Matrix, stream=None) -> dict:
    """out := A_t of packets held in host memory (torch CPU tensors or numpy
    arrays of 32-bit addresses), and its nine quantities, returned
    (ns_window_build_host; blocking)."""
    n = src.numel() if isinstance(src, torch.Tensor) else src.size
    m = dst.numel() if isinstance(dst, torch.Tensor) else dst.size
    if m != n:
        raise ValueError("src and dst differ in length")
    st = NsStats()
    check(ctx._L.ns_window_build_host(ctx.handle, _host_column(src, "src"), _host_column(dst, "dst"), n, out.live(),
                                      ctypes.byref(st), _stream(stream)), "ns_window_build_host")
    return {f: int(getattr(st, f)) for f in FIELDS}


_PATH_NAMES = {v: k for k, v in PATHS.items()}


def path_tune(ctx: Context, src: torch.Tensor, dst: torch.Tensor, stream=None) -> dict:
    """Times both paths on this window and makes the faster one the
    context's "auto" choice for its size (ns_path_tune)."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("src and dst differ in length")
    chosen = ctypes.c_int(0)
    ms_sort, ms_hash = ctypes.c_float(0), ctypes.c_float(0)
    check(ctx._L.ns_path_tune(ctx.handle, _column(src, "src"), _column(dst, "dst"), n, _stream(stream),
                              ctypes.byref(chosen), ctypes.byref(ms_sort), ctypes.byref(ms_hash)), "ns_path_tune")
    return {"path": _PATH_NAMES[chosen.value], "sort_ms": ms_sort.value, "hash_ms": ms_hash.value}


def sort_split_info(ctx: Context, stream=None) -> dict:
    """What the context's last sort-path build did with the hot-key split
    (ns_sort_split_info): {"used", "hot_keys", "cold_packets"}."""
    used = ctypes.c_int(0)
    h, cold = ctypes.c_uint64(0), ctypes.c_uint64(0)
    check(ctx._L.ns_sort_split_info(ctx.handle, ctypes.byref(used), ctypes.byref(h), ctypes.byref(cold),
                                    _stream(stream)), "ns_sort_split_info")
    return {"used": bool(used.value), "hot_keys": int(h.value), "cold_packets": int(cold.value)}


def column_split_info(ctx: Context, stream=None) -> dict:
    """What the context's last sort-path build did with the column side's
    hot-destination split (ns_column_split_info): {"used",
    "hot_destinations", "cold_words"}."""
    used = ctypes.c_int(0)
    h, cold = ctypes.c_uint64(0), ctypes.c_uint64(0)
    check(ctx._L.ns_column_split_info(ctx.handle, ctypes.byref(used), ctypes.byref(h), ctypes.byref(cold),
                                      _stream(stream)), "ns_column_split_info")
    return {"used": bool(used.value), "hot_destinations": int(h.value), "cold_words": int(cold.value)}


def path_resolve(ctx: Context, n: int) -> str:
    """The path window_build takes for n packets (ns_path_resolve)."""
    p = ctypes.c_int(0)
    check(ctx._L.ns_path_resolve(ctx.handle, n, ctypes.byref(p)), "ns_path_resolve")
    return _PATH_NAMES[p.value]


def sort_resolve(ctx: Context, n: int) -> dict:
    """The sort variant a sort-path build of n packets takes (ns_sort_resolve):
    {"split": bool, "tile": one of SORT_TILES' shapes, "digits": "8" or "wide"}."""
    sp, tl, dg = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    check(ctx._L.ns_sort_resolve(ctx.handle, n, ctypes.byref(sp), ctypes.byref(tl), ctypes.byref(dg)),
          "ns_sort_resolve")
    tiles = {v: k for k, v in SORT_TILES.items()}
    digits = {v: k for k, v in SORT_DIGITS.items()}
    return {"split": bool(sp.value), "tile": tiles[tl.value], "digits": digits[dg.value]}


def accumulate(ctx: Context, acc: Matrix, add: Matrix, stream=None):
    """acc := acc + add (ns_accumulate)."""
    check(ctx._L.ns_accumulate(ctx.handle, acc.live(), add.live(), _stream(stream)), "ns_accumulate")


def window_ingest(ctx: Context, acc: Matrix, src: torch.Tensor, dst: torch.Tensor, stream=None):
    """acc := acc + A_t(src, dst), fused (ns_window_ingest)."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("src and dst differ in length")
    check(ctx._L.ns_window_ingest(ctx.handle, acc.live(), _column(src, "src"), _column(dst, "dst"), n,
                                  _stream(stream)), "ns_window_ingest")


def window_ingest_stats(ctx: Context, acc: Matrix, src: torch.Tensor, dst: torch.Tensor, out: torch.Tensor,
                        stream=None):
    """acc := acc + A_t(src, dst) and its nine quantities written into `out`
    (a device tensor of >= 9 64-bit elements), in one launch
    (ns_window_ingest_stats)."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("src and dst differ in length")
    if out.element_size() != 8 or out.numel() < 9 or not out.is_contiguous():
        raise ValueError("out must be a contiguous 64-bit tensor with >= 9 elements")
    check(ctx._L.ns_window_ingest_stats(ctx.handle, acc.live(), _column(src, "src"), _column(dst, "dst"), n,
                                        ctypes.c_void_p(out.data_ptr()), _stream(stream)),
          "ns_window_ingest_stats")


def network_stats(ctx: Context, m: Matrix, stream=None) -> dict:
    """The nine Table 2 quantities (ns_network_stats; blocking)."""
    out = NsStats()
    check(ctx._L.ns_network_stats(ctx.handle, m.live(), ctypes.byref(out), _stream(stream)),
          "ns_network_stats")
    return {f: int(getattr(out, f)) for f in FIELDS}


def network_stats_async(ctx: Context, m: Matrix, out: torch.Tensor, stream=None):
    """Writes the nine quantities into `out` (a device tensor of >= 9 64-bit
    elements) when the stream gets there (ns_network_stats_async)."""
    if out.element_size() != 8 or out.numel() < 9 or not out.is_contiguous():
        raise ValueError("out must be a contiguous 64-bit tensor with >= 9 elements")
    check(ctx._L.ns_network_stats_async(ctx.handle, m.live(), ctypes.c_void_p(out.data_ptr()),
                                        _stream(stream)), "ns_network_stats_async")


def matrix_nnz(m: Matrix, stream=None) -> int:
    v = ctypes.c_uint64()
    check(m._L.ns_matrix_nnz(m.live(), ctypes.byref(v), _stream(stream)), "ns_matrix_nnz")
    return int(v.value)


def matrix_export(m: Matrix, stream=None, device=None):
    """A's nonzeros ascending by key = src << 32 | dst, as two int64 device
    tensors holding uint64 bit patterns (ns_matrix_export)."""
    nnz = matrix_nnz(m, stream)
    dev = device if device is not None else torch.device("cuda", m.ctx.device)
    keys = torch.empty(max(nnz, 1), dtype=torch.int64, device=dev)
    counts = torch.empty(max(nnz, 1), dtype=torch.int64, device=dev)
    got = ctypes.c_uint64()
    check(m._L.ns_matrix_export(m.live(), ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(counts.data_ptr()),
                                max(nnz, 1), ctypes.byref(got), _stream(stream)), "ns_matrix_export")
    return keys[: got.value], counts[: got.value]


NODES = {"src": 0, "dst": 1, "any": 2}


def matrix_nodes(m: Matrix, which: str = "src", stream=None):
    """Per-entity vectors of A, ascending by address (ns_matrix_nodes):
    which="src" -> (ids, A 1, |A|_0 1); "dst" -> (ids, 1^T A, 1^T |A|_0);
    "any" -> the distinct addresses of src and dst together.  Device
    tensors: ids int32 holding uint32 bit patterns, the others int64."""
    nnz = matrix_nnz(m, stream)
    dev = torch.device("cuda", m.ctx.device)
    cap = max(2 * nnz, 1)
    ids = torch.empty(cap, dtype=torch.int32, device=dev)
    pk = torch.empty(cap, dtype=torch.int64, device=dev)
    dg = torch.empty(cap, dtype=torch.int64, device=dev)
    got = ctypes.c_uint64()
    check(m._L.ns_matrix_nodes(m.ctx.handle, m.live(), NODES[which], ctypes.c_void_p(ids.data_ptr()),
                               ctypes.c_void_p(pk.data_ptr()), ctypes.c_void_p(dg.data_ptr()), cap,
                               ctypes.byref(got), _stream(stream)), "ns_matrix_nodes")
    k = got.value
    if which == "any":
        return ids[:k]
    return ids[:k], pk[:k], dg[:k]


def anonymize(ctx: Context, src: torch.Tensor, dst: torch.Tensor, rand: torch.Tensor,
              out_src: torch.Tensor | None = None, out_dst: torch.Tensor | None = None, stream=None):
    """Relabels the addresses of both columns by the random permutation the
    int64 (uint64 bit patterns) device tensor `rand` defines (ns_anonymize).
    Returns (out_src, out_dst, number of distinct addresses)."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("src and dst differ in length")
    if rand.dtype != torch.int64 or not rand.is_contiguous():
        raise ValueError("rand must be a contiguous int64 tensor")
    out_src = torch.empty_like(src) if out_src is None else out_src
    out_dst = torch.empty_like(dst) if out_dst is None else out_dst
    nu = ctypes.c_uint64()
    check(ctx._L.ns_anonymize(ctx.handle, _column(src, "src"), _column(dst, "dst"), n,
                              ctypes.c_void_p(rand.data_ptr() if rand.numel() else None), rand.numel(),
                              _column(out_src, "out_src"), _column(out_dst, "out_dst"), ctypes.byref(nu),
                              _stream(stream)), "ns_anonymize")
    return out_src, out_dst, nu.value


def matrix_reserve(m: Matrix, max_links: int, stream=None):
    check(m._L.ns_matrix_reserve(m.live(), max_links, _stream(stream)), "ns_matrix_reserve")


def matrix_clear(m: Matrix, stream=None):
    check(m._L.ns_matrix_clear(m.live(), _stream(stream)), "ns_matrix_clear")


def sync(ctx: Context, stream=None):
    check(ctx._L.ns_sync(ctx.handle, _stream(stream)), "ns_sync")


def window_stats_static(src: torch.Tensor, dst: torch.Tensor, out: torch.Tensor, stream=None):
    """The nine quantities of one window of at most STATIC_MAX_PACKETS packets
    written into `out` (a device tensor of >= 9 64-bit elements), without any
    device allocation by the library (ns_window_stats_static).  For callers
    that cannot allocate device memory at this point; calls share one fixed
    device array, so order them on one stream."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("src and dst differ in length")
    if out.element_size() != 8 or out.numel() < 9 or not out.is_contiguous():
        raise ValueError("out must be a contiguous 64-bit tensor with >= 9 elements")
    L = load()
    check(L.ns_window_stats_static(_column(src, "src"), _column(dst, "dst"), n, ctypes.c_void_p(out.data_ptr()),
                                   _stream(stream)), "ns_window_stats_static")


def trace_enable(ctx: Context, on: bool = True):
    """Per-kernel timing of the context's launches (ns_trace_enable)."""
    check(ctx._L.ns_trace_enable(ctx.handle, 1 if on else 0), "ns_trace_enable")


def trace_read(ctx: Context) -> dict:
    """{kernel name: (launches, total ms, max ms)} since the last read
    (ns_trace_read; waits for the recorded events)."""
    cap = 64
    buf = (NsTraceEntry * cap)()
    cnt = ctypes.c_int()
    check(ctx._L.ns_trace_read(ctx.handle, buf, cap, ctypes.byref(cnt)), "ns_trace_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms), float(buf[i].max_ms))
            for i in range(min(cnt.value, cap))}


def matrix_save(m: Matrix, path: str, stream=None):
    """Checkpoint: writes A's sorted nonzero list and its nine quantities to
    `path` (ns_matrix_save)."""
    check(m._L.ns_matrix_save(m.live(), os.fsencode(path), _stream(stream)), "ns_matrix_save")


def matrix_load(ctx: Context, path: str, m: Matrix, stream=None):
    """Resume: replaces m's contents with the checkpoint in `path`; its
    quantities are recomputed and checked against the saved ones
    (ns_matrix_load)."""
    check(ctx._L.ns_matrix_load(ctx.handle, os.fsencode(path), m.live(), _stream(stream)), "ns_matrix_load")


def matrix_reserve_ex(m: Matrix, max_links: int, max_nodes: int, stream=None):
    """Reserve with a promise on the number of sources/destinations
    (ns_matrix_reserve_ex)."""
    check(m._L.ns_matrix_reserve_ex(m.live(), max_links, max_nodes, _stream(stream)), "ns_matrix_reserve_ex")


class _BorrowedMatrix(Matrix):
    """A matrix owned by another library object (not freed from Python); it
    stays usable while that owner is open."""

    def __init__(self, ctx: Context, handle, owner=None):
        self._L = ctx._L
        self.ctx = ctx
        self.handle = handle
        self.owner = owner

    def live(self):
        if self.owner is not None and not getattr(self.owner, "handle", None):
            raise RuntimeError("the matrix's owner has been freed")
        return super().live()

    def free(self):
        self.handle = None


class Slider:
    """Per-window and sliding-window statistics over the last `windows`
    windows (ns_slider_create / ns_slider_free)."""

    def __init__(self, ctx: Context, windows: int):
        self._L = ctx._L
        self.ctx = ctx
        h = ctypes.c_void_p()
        check(self._L.ns_slider_create(ctx.handle, windows, ctypes.byref(h)), "ns_slider_create")
        self.handle = h

    def matrix(self) -> Matrix:
        """The current sliding sum (valid until the next push)."""
        h = ctypes.c_void_p()
        check(self._L.ns_slider_matrix(self.handle, ctypes.byref(h)), "ns_slider_matrix")
        return _BorrowedMatrix(self.ctx, h, owner=self)

    def free(self):
        if getattr(self, "handle", None):
            self._L.ns_slider_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def slider_push(ctx: Context, slider: Slider, src: torch.Tensor, dst: torch.Tensor,
                out_window: torch.Tensor | None = None, out_sliding: torch.Tensor | None = None, stream=None):
    """Builds the next window and writes its quantities and the sliding sum's
    into int64 device tensors of at least 9 entries (ns_slider_push)."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("src and dst differ in length")
    for t in (out_window, out_sliding):
        if t is not None and (t.dtype != torch.int64 or t.numel() < 9 or not t.is_cuda):
            raise ValueError("statistics outputs must be int64 CUDA tensors of >= 9 entries")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    check(ctx._L.ns_slider_push(ctx.handle, slider.handle, _column(src, "src"), _column(dst, "dst"), n,
                                ptr(out_window), ptr(out_sliding), _stream(stream)), "ns_slider_push")


class Batch:
    """A plan for batched windows (ns_batch_create / ns_batch_free)."""

    def __init__(self, ctx: Context, max_windows: int, max_packets: int):
        self._L = ctx._L
        self.ctx = ctx
        h = ctypes.c_void_p()
        check(self._L.ns_batch_create(ctx.handle, max_windows, max_packets, ctypes.byref(h)), "ns_batch_create")
        self.handle = h

    @property
    def params(self) -> dict:
        p = NsBatchParams()
        check(self._L.ns_batch_get_params(self.handle, ctypes.byref(p)), "ns_batch_get_params")
        return {"tile_packets": p.tile_packets, "ctas_per_sm": p.ctas_per_sm, "max_load": p.max_load,
                "cta_cache": p.cta_cache}

    def set_params(self, tile_packets: int, ctas_per_sm: int, max_load: float, cta_cache: int = 1):
        p = NsBatchParams(tile_packets, ctas_per_sm, max_load, cta_cache)
        check(self._L.ns_batch_set_params(self.handle, ctypes.byref(p)), "ns_batch_set_params")

    def free(self):
        if getattr(self, "handle", None):
            self._L.ns_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _offsets(offsets):
    import numpy as _np
    off = _np.ascontiguousarray(offsets, dtype=_np.uint64)
    return off, off.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def batch_run(ctx: Context, batch: Batch, src: torch.Tensor, dst: torch.Tensor, offsets, out: torch.Tensor,
              acc: Matrix | None = None, stream=None):
    """Per-window quantities of a batch into `out` (device, int64, windows x
    >= 9, contiguous rows of 9) and optionally acc += the sum (ns_batch_run).
    `offsets` (host, windows + 1) must stay alive until the stream reaches the
    call's copy; keep a reference."""
    off, ptr = _offsets(offsets)
    W = off.size - 1
    if out.element_size() != 8 or out.numel() < 9 * W or not out.is_contiguous():
        raise ValueError("out must be a contiguous 64-bit tensor with >= 9 * windows elements")
    check(ctx._L.ns_batch_run(ctx.handle, batch.handle, _column(src, "src"), _column(dst, "dst"), ptr, W,
                              ctypes.c_void_p(out.data_ptr()), acc.live() if acc is not None else None,
                              _stream(stream)), "ns_batch_run")
    return off


def batch_run_device(ctx: Context, batch: Batch, src: torch.Tensor, dst: torch.Tensor, offsets: torch.Tensor,
                     out: torch.Tensor, acc: Matrix | None = None, stream=None):
    """ns_batch_run with the windows + 1 offsets in a device tensor (int64
    holding uint64), planned on the device (ns_batch_run_device); a graph
    captured around it replays any layout later written into `offsets`."""
    W = offsets.numel() - 1
    if W < 0 or not offsets.is_cuda or offsets.element_size() != 8 or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous 64-bit CUDA tensor of windows + 1 entries")
    if out.element_size() != 8 or out.numel() < 9 * W or not out.is_contiguous():
        raise ValueError("out must be a contiguous 64-bit tensor of >= 9 * windows elements")
    check(ctx._L.ns_batch_run_device(ctx.handle, batch.handle, _column(src, "src"), _column(dst, "dst"),
                                     ctypes.c_void_p(offsets.data_ptr()), W, ctypes.c_void_p(out.data_ptr()),
                                     acc.live() if acc is not None else None, _stream(stream)),
          "ns_batch_run_device")


def batch_sync(batch: Batch, stream=None):
    """Raises NS_ERR_CAPACITY if the batch's last device-planned run refused
    its offsets (ns_batch_sync; blocking)."""
    check(batch._L.ns_batch_sync(batch.handle, _stream(stream)), "ns_batch_sync")


def batch_tune(ctx: Context, batch: Batch, src: torch.Tensor, dst: torch.Tensor, offsets, stream=None) -> dict:
    """Autotune the batch's launch parameters on this batch (ns_batch_tune)."""
    off, ptr = _offsets(offsets)
    W = off.size - 1
    scratch = torch.empty(max(9 * W, 9), dtype=torch.int64, device=src.device)
    p = NsBatchParams()
    check(ctx._L.ns_batch_tune(ctx.handle, batch.handle, _column(src, "src"), _column(dst, "dst"), ptr, W,
                               ctypes.c_void_p(scratch.data_ptr()), _stream(stream), ctypes.byref(p)),
          "ns_batch_tune")
    return {"tile_packets": p.tile_packets, "ctas_per_sm": p.ctas_per_sm, "max_load": p.max_load,
            "cta_cache": p.cta_cache}


class Server:
    """Streaming service over `acc` (ns_server_create / ns_server_destroy).
    The server owns ctx and acc until close()."""

    def __init__(self, ctx: Context, acc: Matrix):
        self._L = ctx._L
        self.ctx, self.acc = ctx, acc
        h = ctypes.c_void_p()
        check(self._L.ns_server_create(ctx.handle, acc.live(), ctypes.byref(h)), "ns_server_create")
        self.handle = h
        self._keep = {}  # ticket -> host arrays that must outlive the window

    def reserve(self, max_window: int):
        """Sizes every slot for windows of up to max_window packets
        (ns_server_reserve; while idle)."""
        check(self._L.ns_server_reserve(self.handle, max_window), "ns_server_reserve")

    def clear(self):
        """Empties the aggregate while idle (ns_server_clear)."""
        check(self._L.ns_server_clear(self.handle), "ns_server_clear")

    def close(self):
        if getattr(self, "handle", None):
            self._L.ns_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_col(a):
    import numpy as _np
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.element_size() != 4 or not a.is_contiguous():
            raise ValueError("host columns must be contiguous 32-bit CPU tensors")
        return a, ctypes.c_void_p(a.data_ptr() if a.numel() else 0)
    a = _np.ascontiguousarray(a, dtype=_np.uint32)
    return a, ctypes.c_void_p(a.ctypes.data if a.size else 0)


def stream_submit(server: Server, src, dst, window_id: int = 0) -> int:
    """Queue one window (host arrays; kept alive by the server until its
    wait) and return its ticket; raises NsError(NS_ERR_BUSY) if full."""
    s, ps = _host_col(src)
    d, pd = _host_col(dst)
    n = s.numel() if isinstance(s, torch.Tensor) else s.size
    t = ctypes.c_uint64()
    check(server._L.ns_stream_submit(server.handle, ps, pd, n, window_id, ctypes.byref(t)), "ns_stream_submit")
    server._keep[t.value] = (s, d)
    return int(t.value)


def stream_poll(server: Server, ticket: int) -> bool:
    d = ctypes.c_int()
    check(server._L.ns_stream_poll(server.handle, ticket, ctypes.byref(d)), "ns_stream_poll")
    return bool(d.value)


def stream_wait(server: Server, ticket: int, timeout_us: int = -1):
    """(per_window quantities, running quantities, timing dict)."""
    pw, rn, tm = NsStats(), NsStats(), NsStreamTiming()
    st = server._L.ns_stream_wait(server.handle, ticket, ctypes.byref(pw), ctypes.byref(rn), timeout_us,
                                  ctypes.byref(tm))
    if st != 5:  # a timeout keeps the ticket (and its arrays) alive
        server._keep.pop(ticket, None)
    check(st, "ns_stream_wait")
    as_dict = lambda x: {f: int(getattr(x, f)) for f in FIELDS}
    return as_dict(pw), as_dict(rn), {"submit_us": tm.submit_us, "admit_us": tm.admit_us,
                                      "complete_us": tm.complete_us, "window_id": int(tm.window_id)}


def diag_random_atomics(table_words: int, threads: int, reps: int = 5, stream=None) -> float:
    """Microseconds for `threads` x 3 random 8-byte atomics into three tables
    of `table_words` words (ns_diag_random_atomics): the ceiling the hash
    ingest's access pattern is bound by."""
    L = load()
    us = ctypes.c_double()
    check(L.ns_diag_random_atomics(table_words, threads, reps, ctypes.byref(us), _stream(stream)),
          "ns_diag_random_atomics")
    return float(us.value)


DIAG_CLAIM_MODES = {"claim": 0, "claim_add": 1, "claim_stale": 2}


def diag_random_claims(table_slots: int, threads: int, mode: str = "claim_add", reps: int = 5,
                       stream=None) -> float:
    """Microseconds for `threads` x three random 16-byte slot claims into
    three tables of `table_slots` slots (ns_diag_random_claims).  mode:
    "claim" (one round trip), "claim_add" (the claims, then the dependent row
    and column adds: the hash ingest's two round trips) or "claim_stale"
    (claims of slots holding old entries, as an epoch mark instead of a
    table clear would need, then the adds)."""
    L = load()
    us = ctypes.c_double()
    check(L.ns_diag_random_claims(table_slots, threads, DIAG_CLAIM_MODES[mode], reps, ctypes.byref(us),
                                  _stream(stream)), "ns_diag_random_claims")
    return float(us.value)


_BY = {"src": 0, "dst": 1}


def owner(addr: int, parts: int) -> int:
    """The rank among `parts` that owns an address (ns_owner)."""
    return int(load().ns_owner(addr & 0xFFFFFFFF, parts))


def matrix_partition(ctx: Context, m: Matrix, by: str, parts: int, stream=None):
    """A's nonzeros grouped by the owner of their source (by="src") or
    destination (by="dst"): (keys, counts, offsets) -- two int64 device
    tensors holding uint64 bit patterns, and the parts + 1 group starts
    (ns_matrix_partition; blocking)."""
    nnz = matrix_nnz(m, stream)
    dev = torch.device("cuda", ctx.device)
    keys = torch.empty(max(nnz, 1), dtype=torch.int64, device=dev)
    counts = torch.empty(max(nnz, 1), dtype=torch.int64, device=dev)
    offs = (ctypes.c_uint64 * (parts + 1))()
    check(ctx._L.ns_matrix_partition(ctx.handle, m.live(), _BY[by], parts, ctypes.c_void_p(keys.data_ptr()),
                                     ctypes.c_void_p(counts.data_ptr()), max(nnz, 1), offs, _stream(stream)),
          "ns_matrix_partition")
    return keys[:nnz], counts[:nnz], [int(x) for x in offs]


def matrix_add_entries(ctx: Context, m: Matrix, keys: torch.Tensor, counts: torch.Tensor, stream=None):
    """m := m + the (key, count) entries of two device tensors of 64-bit
    elements (ns_matrix_add_entries)."""
    n = keys.numel()
    if counts.numel() != n:
        raise ValueError("keys and counts differ in length")
    for t, name in ((keys, "keys"), (counts, "counts")):
        if n and (t.element_size() != 8 or not t.is_contiguous() or not t.is_cuda):
            raise ValueError(f"{name} must be a contiguous 64-bit CUDA tensor")
    check(ctx._L.ns_matrix_add_entries(ctx.handle, m.live(), ctypes.c_void_p(keys.data_ptr() if n else 0),
                                       ctypes.c_void_p(counts.data_ptr() if n else 0), n, _stream(stream)),
          "ns_matrix_add_entries")

