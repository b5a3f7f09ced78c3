"""The sharded multi-GPU form of the traffic-matrix path, simulated over CPU
ranks (two gloo processes, no GPU; the multi-GPU benchmark runs independent
replicas, and this checks the sharded decomposition's arithmetic).

Each rank takes a disjoint share of the packets and aggregates it locally;
the oracle stands in for the rank's GPU.  Then:

1. every local (key, count) entry goes to the rank that owns its source
   (the library's ns_owner rule), which merges equal keys.  Each rank now
   holds whole rows of A, so its unique links, unique sources, max link
   packets, max source packets and max fan-out are exact for those rows;
2. every owned entry goes on to the rank that owns its destination.  Links
   are unique after step 1, so per-destination sums and entry counts there
   are whole columns: unique destinations, max destination packets and max
   fan-in;
3. counts and packet totals add across ranks; maxima take the max.

The reduced quantities must equal the oracle's on the whole stream (Table 2),
and the ranks' rows together must be A's nonzero list."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.slow  # spawns processes; a few seconds


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _packets(kind):
    import gen
    import gen.workloads as W
    if kind == "zipf":
        return W.zipf_window(60001, 1.2, 1 << 12, 0x5AD)
    return gen.rmat_pairs(50000, 0x5AE, gen.bijection_key(0x5AE))


def _owner(addr: np.ndarray, world: int) -> np.ndarray:
    """The library's owner rule (ns_owner, a host function of libns: no GPU
    needed), so the CPU simulation splits exactly as the GPU ranks do."""
    from paper_2509_03653_b300 import _native
    L = _native.load()
    return np.array([L.ns_owner(int(a), world) for a in addr], dtype=np.int64)


def _exchange(dist, parts):
    """All-to-all of per-destination lists: parts[j] goes to rank j."""
    world = dist.get_world_size()
    gathered = [None] * world
    dist.all_gather_object(gathered, parts)
    me = dist.get_rank()
    return [gathered[j][me] for j in range(world)]


def _merge(oracle, lists):
    keys = np.zeros(0, np.uint64)
    counts = np.zeros(0, np.uint64)
    for k, c in lists:
        keys, counts = oracle.accumulate((keys, counts), (k, c))
    return keys, counts


def _rank(rank, world, port, kind, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle

    src, dst = _packets(kind)
    mine = np.arange(rank, src.size, world)  # data-parallel share of the packets
    lk, lc = oracle.build_matrix(src[mine], dst[mine])

    # step 1: entries to the owner of their source; merge equal keys
    own_src = _owner((lk >> np.uint64(32)).astype(np.uint32), world)
    parts = [(lk[own_src == j], lc[own_src == j]) for j in range(world)]
    rk, rc = _merge(oracle, _exchange(dist, parts))
    row = oracle.stats(rk, rc)  # exact for this rank's whole rows

    # step 2: owned entries to the owner of their destination
    own_dst = _owner((rk & np.uint64(0xFFFFFFFF)).astype(np.uint32), world)
    parts = [(rk[own_dst == j], rc[own_dst == j]) for j in range(world)]
    ck, cc = _merge(oracle, _exchange(dist, parts))
    ids, pk, deg = oracle.cols(ck, cc)  # whole columns of this rank's destinations

    part = {
        "valid_packets": row["valid_packets"], "unique_links": row["unique_links"],
        "unique_sources": row["unique_sources"], "unique_destinations": int(ids.size),
        "max_src_packets": row["max_src_packets"], "max_src_fanout": row["max_src_fanout"],
        "max_dst_packets": int(pk.max()) if pk.size else 0, "max_dst_fanin": int(deg.max()) if deg.size else 0,
        "max_link_packets": row["max_link_packets"],
    }
    # step 3: sums and maxima over the ranks
    allp = [None] * world
    dist.all_gather_object(allp, part)
    sums = ("valid_packets", "unique_links", "unique_sources", "unique_destinations")
    total = {f: (sum(p[f] for p in allp) if f in sums else max(p[f] for p in allp)) for f in part}
    out[rank] = (total, rk.tobytes(), rc.tobytes())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["zipf", "rmat"])
def test_sharded_decomposition_equals_the_whole(kind):
    import oracle
    ctx = mp.get_context("spawn")
    world = 2
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, kind, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    src, dst = _packets(kind)
    wk, wc = oracle.build_matrix(src, dst)
    want = oracle.stats(wk, wc)
    for r in range(world):
        assert res[r][0] == want
    # the ranks' rows are disjoint and together form A
    keys = np.concatenate([np.frombuffer(res[r][1], np.uint64) for r in range(world)])
    counts = np.concatenate([np.frombuffer(res[r][2], np.uint64) for r in range(world)])
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(keys[order], wk)
    np.testing.assert_array_equal(counts[order], wc)
