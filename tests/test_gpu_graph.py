"""Sort-path builds captured in a CUDA graph and replayed on new data.

The digit passes and run kernels coordinate their tiles through look-back
status words tagged per launch; a graph fixes those tags at capture, so every
replay must start from cleared words.  These tests capture a build once and
replay it on windows with different contents, comparing A and the nine
quantities with the oracle after every replay."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import export_np, to_dev

pytestmark = pytest.mark.gpu


def _replays(ctx, windows, n):
    ts = torch.empty(n, dtype=torch.int32, device="cuda")
    td = torch.empty(n, dtype=torch.int32, device="cuda")
    s0, d0 = windows[0]
    ts.copy_(to_dev(s0))
    td.copy_(to_dev(d0))
    m = ns.Matrix(ctx)
    cap = torch.cuda.Stream()
    with torch.cuda.stream(cap):
        ns.window_build(ctx, ts, td, m)  # eager: every buffer reaches its size
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        ns.window_build(ctx, ts, td, m)
    for s, d in windows[1:] + windows[:1] + windows[1:]:
        ts.copy_(to_dev(s))
        td.copy_(to_dev(d))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        wk, wc = oracle.build_matrix(s, d)
        assert ns.network_stats(ctx, m) == oracle.stats(wk, wc)
        k, c = export_np(m)
        np.testing.assert_array_equal(k, wk)
        np.testing.assert_array_equal(c, wc)
    m.free()


@pytest.mark.parametrize("digits", ["8", "wide"])
@pytest.mark.parametrize("split", ["on", "off"])
def test_sort_build_graph_replays_new_windows(split, digits):
    n = (1 << 21) + 13
    windows = [W.zipf_window(n, 1.2, 1 << 16, 5), W.zipf_window(n, 1.05, 1 << 18, 6),
               gen.uniform_pairs(n, 32, 7)]
    ctx = ns.Context(0, path="sort", sort_split=split, sort_digits=digits)
    _replays(ctx, windows, n)
    ctx.close()
