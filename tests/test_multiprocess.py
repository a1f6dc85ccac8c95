"""The multi-rank path of the benchmark on CPU with the gloo backend (world size 2): the
barrier and max-over-ranks timing helper, and the partition of the batch into disjoint
contiguous slices, one per rank, built by the counter-based generators with no data moving
between ranks (the path shards with no exchange step)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import bench
    from paper_2407_13116_gb300 import inputs as I
    D = bench.Dist()
    try:
        D.barrier()
        m = D.max(float(10 + 7 * rank))
        n = 1000
        i0 = bench.shard_offset(n, rank)
        G = I.general(n, 0x240713116 + 2, "d", "wide", i0=i0)
        # all ranks see each other's first index and an exact checksum of their slice
        x = int(np.bitwise_xor.reduce(G.view(np.uint64), axis=None)) & ((1 << 63) - 1)
        t = torch.tensor([i0, x], dtype=torch.int64)
        out = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
        D.dist.all_gather(out, t)
        q.put((rank, m, [o.tolist() for o in out], bench.shard_seed(7, rank)))
    finally:
        D.close()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # max over ranks reaches every rank
    assert all(r[1] == 17.0 for r in res)
    # slices are contiguous and disjoint: [0, n) and [n, 2n) of one global batch
    firsts = [g[0] for g in res[0][2]]
    assert firsts == [0, 1000]
    # each rank's slice equals the matching part of one global generation
    sys.path.insert(0, ROOT)
    from paper_2407_13116_gb300 import inputs as I
    full = I.general(2000, 0x240713116 + 2, "d", "wide")
    for r in range(world):
        part = np.ascontiguousarray(full[:, r * 1000:(r + 1) * 1000])
        assert res[0][2][r][1] == int(np.bitwise_xor.reduce(part.view(np.uint64), axis=None)) & ((1 << 63) - 1)
    assert res[0][2][0][1] != res[0][2][1][1]
    # per-rank seeds of the per-batch workloads differ, rank 0 keeps the base seed
    assert res[0][3] == 7 and res[1][3] != 7
