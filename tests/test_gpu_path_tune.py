"""NS_PATH_AUTO and the path tuner (ns_path_tune / ns_path_resolve): the
default size rule, a tuned choice applied to every window of the same power
of two, its persistence in the tuner cache next to the batch tuner's
entries, and builds through the chosen path equal to the CPU oracle."""
from __future__ import annotations

import json
import os
import tempfile

import numpy as np
import pytest
import torch

import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def test_auto_default_rule():
    ctx = ns.Context(0, path="auto")
    assert ns.path_resolve(ctx, 0) == "hash"
    assert ns.path_resolve(ctx, 1 << 17) == "hash"
    assert ns.path_resolve(ctx, (1 << 24) - 1) == "hash"
    assert ns.path_resolve(ctx, 1 << 24) == "sort"
    assert ns.path_resolve(ctx, 1 << 30) == "sort"
    for fixed in ("sort", "hash"):
        c = ns.Context(0, path=fixed)
        assert ns.path_resolve(c, 1 << 17) == fixed and ns.path_resolve(c, 1 << 30) == fixed


def test_path_tune_choice_cache_and_parity():
    s, d = W.zipf_window(1 << 17, 1.1, 1 << 14, W.seed_of(1) + 5)
    ds, dd = to_dev(s), to_dev(d)
    with tempfile.TemporaryDirectory() as tmp:
        cache = os.path.join(tmp, "tuner.json")
        ctx = ns.Context(0, path="auto", tuner_cache=cache)
        # a batch-tuner entry already in the file must survive the path tuner's write
        src_b, dst_b = W.zipf_window(16 * 3000, 1.0, 1 << 12, 99)
        off = np.arange(17, dtype=np.uint64) * 3000
        b = ns.Batch(ctx, 16, int(off[-1]))
        ns.batch_tune(ctx, b, to_dev(src_b), to_dev(dst_b), off)
        b.free()
        r = ns.path_tune(ctx, ds, dd)
        assert r["path"] in ("sort", "hash")
        assert r["sort_ms"] > 0 and r["hash_ms"] > 0
        assert r["path"] == ("sort" if r["sort_ms"] < r["hash_ms"] else "hash")
        for n in (1 << 17, (1 << 17) + 12345, (1 << 18) - 1):
            assert ns.path_resolve(ctx, n) == r["path"]
        assert ns.path_resolve(ctx, 1 << 16) == "hash"  # other sizes keep the default rule
        entries = json.load(open(cache))
        kinds = sorted(k.split("|")[1] for k in entries)
        assert kinds == ["batch", "path"]
        key = next(k for k in entries if "|path|" in k)
        assert key.endswith("|path|n2^17") and entries[key]["path"] == r["path"]
        # a later context on the same GPU starts from the stored choice
        ctx2 = ns.Context(0, path="auto", tuner_cache=cache)
        assert ns.path_resolve(ctx2, 1 << 17) == r["path"]
        m = ns.Matrix(ctx2)
        ns.window_build(ctx2, ds, dd, m)
        assert ns.network_stats(ctx2, m) == oracle.stats_of_packets(s, d)


def test_path_tune_forced_choice_from_cache():
    """A cache entry naming the sort path for a size makes auto take it there;
    results stay equal to the oracle."""
    s, d = W.zipf_window(5000, 1.2, 1 << 10, 17)
    with tempfile.TemporaryDirectory() as tmp:
        cache = os.path.join(tmp, "tuner.json")
        ctx = ns.Context(0, path="auto", tuner_cache=cache)
        ns.path_tune(ctx, to_dev(s), to_dev(d))
        entries = json.load(open(cache))
        (key,) = [k for k in entries if "|path|" in k]
        want = "hash" if entries[key]["path"] == "sort" else "sort"
        entries[key]["path"] = want
        with open(cache, "w") as f:
            json.dump(entries, f)
        ctx2 = ns.Context(0, path="auto", tuner_cache=cache)
        assert ns.path_resolve(ctx2, 5000) == want
        m = ns.Matrix(ctx2)
        ns.window_build(ctx2, to_dev(s), to_dev(d), m)
        assert ns.network_stats(ctx2, m) == oracle.stats_of_packets(s, d)


def test_path_tune_rejects_empty():
    ctx = ns.Context(0, path="auto")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(ns.NsError) as err:
        ns.path_tune(ctx, e, e)
    assert err.value.name == "NS_ERR_INVALID"
