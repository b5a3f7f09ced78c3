"""Seeded synthetic packet-stream generators (input side only).

Both the CPU oracle and the CUDA library consume these arrays; this module
holds none of the traffic-matrix arithmetic.  The C source is ``nsgen.c``;
it is compiled on first use into ``libnsgen.so`` next to it.

The workload recipes that stand in for the challenge dataset (paper, section
"Graph Challenge Setup", paragraph "Inputs": one graph of 2^30 packets; the
GraphBLAS release splits it into 128 x 64 = 8192 matrices, i.e. 2^17 packets
each) live in :mod:`gen.workloads`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nsgen.c")
_LIB = os.path.join(_HERE, "libnsgen.so")
_lib = None

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U64 = ctypes.c_uint64


def build(force: bool = False) -> str:
    """Compile nsgen.c into libnsgen.so when it is missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.nsg_splitmix64.argtypes = [_U64]
        L.nsg_splitmix64.restype = _U64
        L.nsg_rand64.argtypes = [_U64, _U64, _U64]
        L.nsg_rand64.restype = _U64
        L.nsg_feistel.argtypes = [ctypes.c_uint32, _U64]
        L.nsg_feistel.restype = ctypes.c_uint32
        L.nsg_feistel_inv.argtypes = [ctypes.c_uint32, _U64]
        L.nsg_feistel_inv.restype = ctypes.c_uint32
        L.nsg_feistel_fill.argtypes = [_u32p, _u32p, _U64, _U64]
        L.nsg_zipf_fill.argtypes = [_u32p, _U64, ctypes.c_double, _U64, _U64, _U64, _U64]
        L.nsg_zipf_ranks.argtypes = [_u32p, _U64, ctypes.c_double, _U64, _U64, _U64]
        L.nsg_rmat_fill.argtypes = [_u32p, _u32p, _U64, _U64, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, _U64, _U64]
        L.nsg_loguniform_sizes.argtypes = [_u64p, _U64, ctypes.c_double, ctypes.c_double, _U64, _U64]
        L.nsg_uniform_doubles.argtypes = [_f64p, _U64, ctypes.c_double, ctypes.c_double, _U64, _U64]
        L.nsg_poisson_arrivals.argtypes = [_f64p, _U64, ctypes.c_double, _U64, _U64]
        L.nsg_uniform_pairs.argtypes = [_u32p, _u32p, _U64, ctypes.c_int, _U64]
        L.nsg_rand64_fill.argtypes = [_u64p, _U64, _U64, _U64]
        _lib = L
    return _lib


def random_u64(n: int, seed: int, stream: int, out=None) -> np.ndarray:
    """n random 64-bit keys (counter-based: key i = splitmix64(seed ^ stream << 40 ^ i))."""
    out = np.empty(n, np.uint64) if out is None else out
    if n:
        lib().nsg_rand64_fill(out, n, seed, stream)
    return out


def splitmix64(x: int) -> int:
    return int(lib().nsg_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def bijection_key(seed: int) -> int:
    """Key of the anonymizing Feistel bijection used with a given seed."""
    return splitmix64(seed ^ 0xB1)


def feistel(x: np.ndarray, key: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint32)
    out = np.empty_like(x)
    lib().nsg_feistel_fill(x, out, x.size, key)
    return out


def feistel_inv_scalar(y: int, key: int) -> int:
    return int(lib().nsg_feistel_inv(y, key))


def zipf_addresses(n: int, s: float, K: int, seed: int, stream: int, bij_key: int,
                   out: np.ndarray | None = None) -> np.ndarray:
    """n addresses whose ranks are Zipf(s) over K, relabelled into 32 bits."""
    if out is None:
        out = np.empty(n, dtype=np.uint32)
    lib().nsg_zipf_fill(out, n, s, K, seed, stream, bij_key)
    return out


def zipf_ranks(n: int, s: float, K: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    lib().nsg_zipf_ranks(out, n, s, K, seed, stream)
    return out


def rmat_pairs(n: int, seed: int, bij_key: int, i0: int = 0, scale: int = 32,
               a: float = 0.57, b: float = 0.19, c: float = 0.19, bg_frac: float = 0.10,
               src: np.ndarray | None = None, dst: np.ndarray | None = None):
    """n RMAT packets (packet indices i0..i0+n-1) plus uniform background."""
    if src is None:
        src = np.empty(n, dtype=np.uint32)
    if dst is None:
        dst = np.empty(n, dtype=np.uint32)
    lib().nsg_rmat_fill(src, dst, n, i0, scale, a, b, c, bg_frac, seed, bij_key)
    return src, dst


def loguniform_sizes(k: int, lo: float, hi: float, seed: int, stream: int) -> np.ndarray:
    out = np.empty(k, dtype=np.uint64)
    lib().nsg_loguniform_sizes(out, k, lo, hi, seed, stream)
    return out


def uniform_doubles(k: int, lo: float, hi: float, seed: int, stream: int) -> np.ndarray:
    out = np.empty(k, dtype=np.float64)
    lib().nsg_uniform_doubles(out, k, lo, hi, seed, stream)
    return out


def poisson_arrivals(k: int, rate: float, seed: int, stream: int) -> np.ndarray:
    out = np.empty(k, dtype=np.float64)
    lib().nsg_poisson_arrivals(out, k, rate, seed, stream)
    return out


def uniform_pairs(n: int, bits: int, seed: int):
    src = np.empty(n, dtype=np.uint32)
    dst = np.empty(n, dtype=np.uint32)
    lib().nsg_uniform_pairs(src, dst, n, bits, seed)
    return src, dst
