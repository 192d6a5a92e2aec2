"""The multi-process path on CPU: two gloo ranks shard events and counter ranges, take the
job time as the maximum over ranks, and merge their reducer states with the library's
mbis_merge_summaries; the merged evidence and ESS equal the oracle's on all samples."""
import os
import socket

import numpy as np
import pytest

import oracle

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, ll, lp, lq, out_path):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import paper_2410_05190_gb300 as m
        from paper_2410_05190_gb300.dist import counter_range, max_over_ranks, merge_over_ranks, shard
        a, b = counter_range(len(ll), rank, WORLD)
        part = oracle.reduce(ll[a:b], lp[a:b], lq[a:b])
        merged = merge_over_ranks(part, merge=m.mbis_merge_summaries)
        t = max_over_ranks(1.0 + rank)
        mine = shard(range(10), rank, WORLD)
        np.save(out_path + f".{rank}.npy", np.array([merged["ess"], merged["log_z"], merged["n"], t, len(mine),
                                                      a, b]))
    finally:
        tdist.destroy_process_group()


def test_counter_ranges_and_shards_partition():
    from paper_2410_05190_gb300.dist import counter_range, shard
    for n in (0, 1, 7, 1 << 20, 1000003):
        for world in (1, 2, 3, 8):
            spans = [counter_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
    items = list(range(11))
    got = sorted(x for r in range(3) for x in shard(items, r, 3))
    assert got == items
    with pytest.raises(ValueError):
        shard(items, 3, 3)


def test_two_gloo_ranks_merge_to_the_whole():
    import __graft_entry__
    __graft_entry__._build_module().build()
    oracle.build()
    import torch.multiprocessing as mp
    rng = np.random.default_rng(5)
    n = 10007
    ll = rng.normal(50.0, 4.0, n)
    lp = np.where(rng.uniform(size=n) < 0.2, -np.inf, rng.normal(-3.0, 0.5, n))
    lq = rng.normal(-2.0, 1.0, n)
    scratch = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2410_05190_gb300",
                           "_build")
    os.makedirs(scratch, exist_ok=True)
    out = os.path.join(scratch, "dist_test_rank")
    mp.start_processes(_worker, args=(_free_port(), ll, lp, lq, out), nprocs=WORLD, join=True, start_method="spawn")
    whole = oracle.reduce(ll, lp, lq)
    res = [np.load(out + f".{r}.npy") for r in range(WORLD)]
    for r in res:
        ess, log_z, nn, t, n_items, a, b = r
        assert nn == n and t == float(WORLD)
        assert abs(ess / whole["ess"] - 1) < 1e-12
        assert abs(log_z - whole["log_z"]) < 1e-12
    assert res[0][4] + res[1][4] == 10
    assert res[0][6] == res[1][5]
