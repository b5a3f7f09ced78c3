"""Helpers for the GPU parity tests: host arrays <-> device tensors."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2509_03653_b300 as ns


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).cuda()


def export_np(m):
    k, c = ns.matrix_export(m)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64).copy(), c.cpu().numpy().view(np.uint64).copy()


def stats_row(t: torch.Tensor) -> dict:
    v = t.cpu().numpy().view(np.uint64)
    return {f: int(x) for f, x in zip(oracle.FIELDS, v[:9])}


def assert_matrix_equal(m, want_keys, want_counts):
    k, c = export_np(m)
    assert k.size == want_keys.size, (k.size, want_keys.size)
    np.testing.assert_array_equal(k, want_keys)
    np.testing.assert_array_equal(c, want_counts)
