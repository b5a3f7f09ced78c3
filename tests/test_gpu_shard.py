"""The sharded form of the traffic-matrix path through the library: two
gloo ranks (processes) each drive libns on cuda:0 -- every rank builds the
matrix of its share of the packets on the GPU, groups its nonzeros by the
rank that owns their source (ns_matrix_partition), the groups are exchanged
over gloo as host copies, and each rank adds what it received
(ns_matrix_add_entries) and reads its row quantities; the same again by
destination owner for the column quantities; sums and maxima are then
reduced over the ranks.  The oracle only checks the result: the reduced
quantities equal the whole stream's, and the ranks' rows together are A's
nonzero list.  (Two processes on one GPU: their kernels never wait on each
other; the exchange is on the host.)"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


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
        return W.zipf_window(300007, 1.2, 1 << 14, 0x5AD)
    return gen.rmat_pairs(250000, 0x5AE, gen.bijection_key(0x5AE))


def _exchange(dist, ns, ctx, m, by, world):
    """Groups m's nonzeros by owner, sends group j to rank j, and returns a
    new matrix holding everything this rank received."""
    import torch
    keys, counts, offs = ns.matrix_partition(ctx, m, by, world)
    hk = keys.cpu().numpy().view(np.uint64)
    hc = counts.cpu().numpy().view(np.uint64)
    parts = [(hk[offs[j]:offs[j + 1]].tobytes(), hc[offs[j]:offs[j + 1]].tobytes()) for j in range(world)]
    gathered = [None] * world
    dist.all_gather_object(gathered, parts)
    me = dist.get_rank()
    got = ns.Matrix(ctx)
    for j in range(world):
        k = np.frombuffer(gathered[j][me][0], np.uint64)
        c = np.frombuffer(gathered[j][me][1], np.uint64)
        if k.size:
            ns.matrix_add_entries(ctx, got, torch.from_numpy(k.view(np.int64).copy()).cuda(),
                                  torch.from_numpy(c.view(np.int64).copy()).cuda())
    return got


def _rank(rank, world, port, kind, path, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2509_03653_b300 as ns

    torch.cuda.set_device(0)
    ctx = ns.Context(0, path=path)
    src, dst = _packets(kind)
    mine = np.arange(rank, src.size, world)  # data-parallel share of the packets
    local = ns.Matrix(ctx)
    ns.window_build(ctx, torch.from_numpy(src[mine].view(np.int32)).cuda(),
                    torch.from_numpy(dst[mine].view(np.int32)).cuda(), local)
    rows = _exchange(dist, ns, ctx, local, "src", world)  # whole rows of A owned here
    row = ns.network_stats(ctx, rows)
    cols = _exchange(dist, ns, ctx, rows, "dst", world)  # whole columns owned here
    col = ns.network_stats(ctx, cols)
    part = dict(row)
    for f in ("unique_destinations", "max_dst_packets", "max_dst_fanin"):
        part[f] = col[f]
    allp = [None] * world
    dist.all_gather_object(allp, part)
    sums = ("valid_packets", "unique_links", "unique_sources", "unique_destinations")
    total = {f: (sum(p[f] for p in allp) if f in sums else max(p[f] for p in allp)) for f in part}
    k, c = ns.matrix_export(rows)
    owners = {ns.owner(int(x) >> 32, world) for x in k.cpu().numpy().view(np.uint64)[:64]}
    out[rank] = (total, k.cpu().numpy().view(np.uint64).tobytes(), c.cpu().numpy().view(np.uint64).tobytes(),
                 sorted(owners))
    for mm in (local, rows, cols):
        mm.free()
    ctx.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind,path", [("zipf", "sort"), ("rmat", "hash")])
def test_sharded_path_through_the_library(kind, path):
    import oracle
    ctx = mp.get_context("spawn")
    world = 2
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, kind, path, out)) for r in range(world)]
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
        assert res[r][3] in ([], [r])  # a rank's rows are the ones it owns
    keys = np.concatenate([np.frombuffer(res[r][1], np.uint64) for r in range(world)])
    counts = np.concatenate([np.frombuffer(res[r][2], np.uint64) for r in range(world)])
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(keys[order], wk)
    np.testing.assert_array_equal(counts[order], wc)


def test_partition_groups_by_owner_in_key_order():
    """One process: groups are the owners' entries, ascending, covering A."""
    import torch
    import gen.workloads as W
    import oracle
    import paper_2509_03653_b300 as ns
    s, d = W.zipf_window(100003, 1.1, 1 << 13, 44)
    ctx = ns.Context(0)
    m = ns.Matrix(ctx)
    ns.window_build(ctx, torch.from_numpy(s.view(np.int32)).cuda(), torch.from_numpy(d.view(np.int32)).cuda(), m)
    wk, wc = oracle.build_matrix(s, d)
    for by, shift in (("src", 32), ("dst", 0)):
        for parts in (1, 3, 8):
            k, c, offs = ns.matrix_partition(ctx, m, by, parts)
            k = k.cpu().numpy().view(np.uint64)
            c = c.cpu().numpy().view(np.uint64)
            assert offs[0] == 0 and offs[-1] == wk.size
            own = np.array([ns.owner(int(x >> np.uint64(shift)) & 0xFFFFFFFF, parts) for x in wk])
            for p in range(parts):
                sel = own == p
                np.testing.assert_array_equal(k[offs[p]:offs[p + 1]], wk[sel])
                np.testing.assert_array_equal(c[offs[p]:offs[p + 1]], wc[sel])
    # adding a matrix's own entries doubles every count
    k, c, _ = ns.matrix_partition(ctx, m, "src", 1)
    ns.matrix_add_entries(ctx, m, k, c)
    k2, c2 = ns.matrix_export(m)
    np.testing.assert_array_equal(k2.cpu().numpy().view(np.uint64), wk)
    np.testing.assert_array_equal(c2.cpu().numpy().view(np.uint64), 2 * wc)
    ctx.close()
