"""CPU oracle for the traffic-matrix hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the package's smoke check and the benchmark's
CPU-baseline leg may import this module.  The CUDA library never calls it and
shares no code with it.

``ns_oracle.cpp`` follows the paper's Table 2 definitions (matrix notation)
with std::sort and linear scans; see its header for the steps.  This wrapper
only compiles it and marshals numpy arrays.

Statistics record field order (``FIELDS``): valid packets, unique links,
unique sources, unique destinations, max source packets, max source fan-out,
max destination packets, max destination fan-in, max link packets.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

FIELDS = (
    "valid_packets",
    "unique_links",
    "unique_sources",
    "unique_destinations",
    "max_src_packets",
    "max_src_fanout",
    "max_dst_packets",
    "max_dst_fanin",
    "max_link_packets",
)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ns_oracle.cpp")
_LIB = os.path.join(_HERE, "libns_oracle.so")
_lib = None

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_U64 = ctypes.c_uint64
_P64 = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False, src: str = _SRC, out: str = _LIB, defines=()) -> str:
    """Compile the oracle (plain g++ -O2; std::thread for the all-cores
    variants) when missing or stale."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", "-o", tmp, src]
        cmd += ["-D%s" % d for d in defines]
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load an oracle library (the default one, or a test variant)."""
    L = ctypes.CDLL(path or build())
    L.oracle_build.argtypes = [_u32p, _u32p, _U64, _u64p, _u64p, _P64]
    L.oracle_accumulate.argtypes = [_u64p, _u64p, _U64, _u64p, _u64p, _U64, _u64p, _u64p, _P64]
    L.oracle_stats.argtypes = [_u64p, _u64p, _U64, _u64p]
    L.oracle_rows.argtypes = [_u64p, _u64p, _U64, _u32p, _u64p, _u64p, _P64]
    L.oracle_digest.argtypes = [_u64p, _u64p, _U64]
    L.oracle_digest.restype = _U64
    L.oracle_cols.argtypes = [_u64p, _u64p, _U64, _u32p, _u64p, _u64p, _P64]
    L.oracle_unique_addresses.argtypes = [_u64p, _U64, _u32p, _P64]
    L.oracle_anonymize.argtypes = [_u32p, _u32p, _U64, _u64p, _U64, _u32p, _u32p, _P64]
    L.oracle_anonymize.restype = ctypes.c_int
    L.oracle_build_parallel.argtypes = [_u32p, _u32p, _U64, _u64p, _u64p, _P64, ctypes.c_int]
    L.oracle_stats_parallel.argtypes = [_u64p, _u64p, _U64, _u64p, ctypes.c_int]
    L.oracle_hardware_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def build_matrix(src, dst, L=None):
    """A's sorted nonzero list (keys, counts) for one packet window."""
    L = L or lib()
    src = _c(src, np.uint32)
    dst = _c(dst, np.uint32)
    n = src.size
    assert dst.size == n
    keys = np.empty(max(n, 1), dtype=np.uint64)
    counts = np.empty(max(n, 1), dtype=np.uint64)
    nnz = ctypes.c_uint64(0)
    L.oracle_build(src, dst, n, keys, counts, ctypes.byref(nnz))
    return keys[: nnz.value].copy(), counts[: nnz.value].copy()


def hardware_threads(L=None) -> int:
    """Threads the all-cores variants use by default (the host's hardware
    concurrency)."""
    return int((L or lib()).oracle_hardware_threads())


def build_matrix_parallel(src, dst, threads: int = 0, L=None):
    """build_matrix on all host cores (threads <= 0: every hardware thread):
    chunk matrices by build_matrix's own step, summed pairwise by
    accumulate's.  Same result as build_matrix."""
    L = L or lib()
    src = _c(src, np.uint32)
    dst = _c(dst, np.uint32)
    n = src.size
    assert dst.size == n
    # np.empty pages are touched only up to nnz
    keys = np.empty(max(n, 1), dtype=np.uint64)
    counts = np.empty(max(n, 1), dtype=np.uint64)
    nnz = ctypes.c_uint64(0)
    L.oracle_build_parallel(src if n else np.zeros(1, np.uint32), dst if n else np.zeros(1, np.uint32), n,
                            keys, counts, ctypes.byref(nnz), int(threads))
    return keys[: nnz.value].copy(), counts[: nnz.value].copy()


def stats_parallel(keys, counts, threads: int = 0, L=None) -> dict:
    """stats on all host cores (the columns' sort split over the threads)."""
    L = L or lib()
    keys = _c(keys, np.uint64)
    counts = _c(counts, np.uint64)
    out = np.zeros(len(FIELDS), dtype=np.uint64)
    L.oracle_stats_parallel(keys if keys.size else np.zeros(1, np.uint64),
                            counts if counts.size else np.zeros(1, np.uint64), keys.size, out, int(threads))
    return {f: int(v) for f, v in zip(FIELDS, out)}


def accumulate(a, b, L=None):
    """(keys, counts) of A + B for two sorted nonzero lists."""
    L = L or lib()
    ka, ca = _c(a[0], np.uint64), _c(a[1], np.uint64)
    kb, cb = _c(b[0], np.uint64), _c(b[1], np.uint64)
    cap = max(ka.size + kb.size, 1)
    keys = np.empty(cap, dtype=np.uint64)
    counts = np.empty(cap, dtype=np.uint64)
    nnz = ctypes.c_uint64(0)
    L.oracle_accumulate(ka, ca, ka.size, kb, cb, kb.size, keys, counts, ctypes.byref(nnz))
    return keys[: nnz.value].copy(), counts[: nnz.value].copy()


def stats(keys, counts, L=None) -> dict:
    """The nine quantities of a matrix given by its sorted nonzero list."""
    L = L or lib()
    keys = _c(keys, np.uint64)
    counts = _c(counts, np.uint64)
    out = np.zeros(len(FIELDS), dtype=np.uint64)
    L.oracle_stats(keys if keys.size else np.zeros(1, np.uint64),
                   counts if counts.size else np.zeros(1, np.uint64), keys.size, out)
    return {f: int(v) for f, v in zip(FIELDS, out)}


def stats_of_packets(src, dst, L=None) -> dict:
    k, c = build_matrix(src, dst, L)
    return stats(k, c, L)


def rows(keys, counts, L=None):
    """Per-source (src, packets A1, fan-out |A|_0 1), ascending by src."""
    L = L or lib()
    keys = _c(keys, np.uint64)
    counts = _c(counts, np.uint64)
    n = max(keys.size, 1)
    s = np.empty(n, np.uint32)
    p = np.empty(n, np.uint64)
    f = np.empty(n, np.uint64)
    ns = ctypes.c_uint64(0)
    L.oracle_rows(keys if keys.size else np.zeros(1, np.uint64),
                  counts if counts.size else np.zeros(1, np.uint64), keys.size, s, p, f,
                  ctypes.byref(ns))
    m = ns.value
    return s[:m].copy(), p[:m].copy(), f[:m].copy()


def cols(keys, counts, L=None):
    """Per-destination (dst, packets 1^T A, fan-in 1^T |A|_0), ascending by dst."""
    L = L or lib()
    keys = _c(keys, np.uint64)
    counts = _c(counts, np.uint64)
    n = max(keys.size, 1)
    d = np.empty(n, np.uint32)
    p = np.empty(n, np.uint64)
    f = np.empty(n, np.uint64)
    nd = ctypes.c_uint64(0)
    L.oracle_cols(keys if keys.size else np.zeros(1, np.uint64),
                  counts if counts.size else np.zeros(1, np.uint64), keys.size, d, p, f,
                  ctypes.byref(nd))
    m = nd.value
    return d[:m].copy(), p[:m].copy(), f[:m].copy()


def unique_addresses(keys, L=None) -> np.ndarray:
    """Distinct addresses of src and dst together, ascending (|src u dst|)."""
    L = L or lib()
    keys = _c(keys, np.uint64)
    out = np.empty(max(2 * keys.size, 1), np.uint32)
    cnt = ctypes.c_uint64(0)
    L.oracle_unique_addresses(keys if keys.size else np.zeros(1, np.uint64), keys.size, out,
                              ctypes.byref(cnt))
    return out[:cnt.value].copy()


def anonymize(src, dst, rnd, L=None):
    """(out_src, out_dst, n_unique): every address replaced by its label under
    the random permutation that the random keys rnd define."""
    L = L or lib()
    src = _c(src, np.uint32)
    dst = _c(dst, np.uint32)
    rnd = _c(rnd, np.uint64)
    n = src.size
    os_ = np.empty(max(n, 1), np.uint32)
    od = np.empty(max(n, 1), np.uint32)
    nu = ctypes.c_uint64(0)
    rc = L.oracle_anonymize(src if n else np.zeros(1, np.uint32), dst if n else np.zeros(1, np.uint32), n,
                            rnd if rnd.size else np.zeros(1, np.uint64), rnd.size, os_, od, ctypes.byref(nu))
    if rc != 0:
        raise ValueError("fewer random keys than distinct addresses")
    return os_[:n].copy(), od[:n].copy(), nu.value


def digest(keys, counts, L=None) -> int:
    L = L or lib()
    keys = _c(keys, np.uint64)
    counts = _c(counts, np.uint64)
    if keys.size == 0:
        return 0
    return int(L.oracle_digest(keys, counts, keys.size))
