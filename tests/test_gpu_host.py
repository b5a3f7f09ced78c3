"""ns_window_build_host: packets in host memory in, the nine quantities out.
Against the oracle, for both paths, from pageable numpy arrays and from
pinned tensors, on a ragged size, an empty window and a window that reuses
the context's staging buffers after a larger one."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import export_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("path", ["sort", "hash"])
def test_host_build_matches_oracle(path):
    ctx = ns.Context(0, path=path)
    m = ns.Matrix(ctx)
    for n, pinned in ((300007, False), (4097, True), (0, False), (65536 + 3, True)):
        s, d = W.large_build(n) if n else (np.zeros(0, np.uint32), np.zeros(0, np.uint32))
        if pinned:
            hs = torch.from_numpy(s.view(np.int32)).pin_memory()
            hd = torch.from_numpy(d.view(np.int32)).pin_memory()
            got = ns.window_build_host(ctx, hs, hd, m)
        else:
            got = ns.window_build_host(ctx, s, d, m)
        wk, wc = oracle.build_matrix(s, d)
        assert got == oracle.stats(wk, wc), (n, pinned)
        k, c = export_np(m)
        np.testing.assert_array_equal(k, wk)
        np.testing.assert_array_equal(c, wc)
    m.free()
    ctx.close()


def test_host_build_rejects_device_tensors():
    ctx = ns.Context(0)
    m = ns.Matrix(ctx)
    t = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        ns.window_build_host(ctx, t, t, m)
    m.free()
    ctx.close()
