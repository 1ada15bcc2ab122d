"""Multi-GPU host logic on CPU with world_size-2 gloo ranks: query sharding
covers every query once; a query split on median-of-means block boundaries
gives the unsharded estimate bit for bit (block means from the oracle's Q_R,
gathered with the product's gather, reduced with the library's host median);
the timing reduction is a max over ranks."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import oracle
    from paper_2512_05460_gb300 import build, probewalk as pw, sharding
    from pw_inputs import er_cycle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    build.build()
    host = er_cycle(200, 8 / 199, 0)
    results = {}
    for (s, t, seed) in ((3, 77, 12345), (150, 9, 99)):
        full = oracle.query(host, s, t, 0.2, 32, seed, want_q=True)
        B, G = full["B"], full["G"]
        g0, g1 = sharding.shard_blocks(G, rank, world)
        q = full["q"]
        local = []
        for g in range(g0, g1):  # block means in the oracle's order
            acc = 0.0
            for k in range(g * B, (g + 1) * B):
                acc = acc + float(q[k])
            local.append(acc / B)
        means = sharding.gather_block_means(local, G)
        if rank == 0:
            results[(s, t)] = (pw.pw_block_median(means), full["beta"])
    mx = sharding.max_over_ranks(float(rank + 1))
    covered = sharding.shard_range(1001, rank, world)
    if rank == 0:
        np.save(out_path, np.array([[v[0], v[1]] for v in results.values()] + [[mx, world]] +
                                   [[covered[0], covered[1]]]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_median_equals_unsharded(tmp_path):
    import torch.multiprocessing as mp

    out = str(tmp_path / "res.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = np.load(out)
    for got, want in res[:2]:
        assert got == want
    assert res[2][0] == 2.0  # max over ranks of (rank + 1)
    assert tuple(res[3]) == (0.0, 501.0)


def test_shard_ranges_partition():
    from paper_2512_05460_gb300 import sharding

    for count in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = sharding.shard_range(count, r, world)
                seen.extend(range(lo, hi))
            assert seen == list(range(count))
    with pytest.raises(ValueError):
        sharding.shard_range(10, 2, 2)
