"""Per-window and sliding-window statistics (ns_slider_*): every window's
own quantities and those of the sum of the last K windows, bit-exact against
the CPU oracle, for K = 1, 3 and more windows than pushed; with empty and
ragged windows, sort-path window matrices, and the sliding sum's nonzero
list."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import assert_matrix_equal, to_dev

pytestmark = pytest.mark.gpu


def rows_of(t):
    return {f: int(x) for f, x in zip(oracle.FIELDS, t.cpu().numpy().view(np.uint64)[:9])}


SIZES = [5000, 0, 70001, 1, 4096, 33333, 20000, 1 << 17]


@pytest.mark.parametrize("K", [1, 3, 16])
def test_slider_matches_oracle(K):
    ctx = ns.Context(0)
    sl = ns.Slider(ctx, K)
    wins = []
    for w, n in enumerate(SIZES):
        s, d = W.rmat_stream(n, i0=w * 200000) if w % 2 else W.zipf_window(n, 1.2, 1 << 12, 500 + w)
        wins.append((s, d))
        ow = torch.zeros(16, dtype=torch.int64, device="cuda")
        os_ = torch.zeros(16, dtype=torch.int64, device="cuda")
        ns.slider_push(ctx, sl, to_dev(s), to_dev(d), ow, os_)
        torch.cuda.synchronize()
        assert rows_of(ow) == oracle.stats_of_packets(s, d), w
        last = wins[max(0, w + 1 - K):]
        ss = np.concatenate([x[0] for x in last])
        dd = np.concatenate([x[1] for x in last])
        assert rows_of(os_) == oracle.stats_of_packets(ss, dd), w
        if w == len(SIZES) - 1:
            assert_matrix_equal(sl.matrix(), *oracle.build_matrix(ss, dd))
    sl.free()


def test_slider_with_sort_path_windows():
    """With the context on the sort path the window matrices are sorted
    lists; the sliding sum (a hash matrix) still comes out exact."""
    ctx = ns.Context(0, path="sort")
    sl = ns.Slider(ctx, 2)
    wins = []
    for w in range(3):
        s, d = W.zipf_window(300000, 1.1, 1 << 14, 900 + w)
        wins.append((s, d))
        os_ = torch.zeros(16, dtype=torch.int64, device="cuda")
        ns.slider_push(ctx, sl, to_dev(s), to_dev(d), None, os_)
        torch.cuda.synchronize()
        last = wins[max(0, w - 1):]
        want = oracle.stats_of_packets(np.concatenate([x[0] for x in last]), np.concatenate([x[1] for x in last]))
        assert rows_of(os_) == want, w
