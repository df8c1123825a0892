"""Multi-rank host logic on CPU ranks (gloo, world size 2 and 3).

The scan of each rank's share is the oracle here (CPU), so these tests check
the split and merge arithmetic of paper_1403_1305_gb300.shard — text ranges
with a warm-up halo, pattern id ranges, gather and merge of sorted matches,
summed counts — and bench.py's max-over-ranks timing, without a GPU.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, split, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    import workloads
    from paper_1403_1305_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(77)
        results = []
        for case in range(6):
            text = workloads.dna_text(rng, int(rng.integers(1, 20_000)))
            text[rng.random(text.size) < 0.01] = ord("N")
            pats = workloads.draw_patterns(rng, [text, workloads.dna_text(rng, 64)], 40, 2, 25, 0.6,
                                           np.frombuffer(b"ACGT", np.uint8))
            got = shard.sharded_scan(pats, text, split=split, scanner=oracle.scan, dist=dist)
            if rank == 0:
                want = oracle.scan(pats, text)
                results.append(bool(np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])))
        # bench.py's timing reduction: the slowest rank counts
        import bench
        t = bench.max_over_ranks(dist, float(rank + 1))
        if rank == 0:
            q.put((results, t))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("split,world", [("text", 2), ("patterns", 2), ("text", 3)])
def test_sharded_scan_equals_single_scan(split, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, split, q)) for r in range(world)]
    for p in procs:
        p.start()
    results, t = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(results) and len(results) == 6
    assert t == float(world)


def test_ranges_cover_the_text_and_patterns():
    from paper_1403_1305_gb300 import shard
    for n in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            rs = shard.text_ranges(n, world, 5)
            assert rs[0][1] == 0 and rs[-1][2] == n
            assert all(rs[i][2] == rs[i + 1][1] for i in range(world - 1))
            assert all(s == max(0, lo - 5) for s, lo, _ in rs)
    pr = shard.pattern_ranges(10, 4)
    assert pr[0][0] == 0 and pr[-1][1] == 10 and all(pr[i][1] == pr[i + 1][0] for i in range(3))
