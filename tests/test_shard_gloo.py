"""Multi-rank host logic on CPU ranks (gloo, world size 2): walker sharding, the gather of
per-walker chi^2 to the sampler rank, max-over-ranks timing, and a rank that leaves before
the exchange (failure made on the host; no GPU involved)."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1501_06576_gb300 import shard


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def fake_chi2(walkers):
    return np.array([0.5 * w * w + 1.0 for w in walkers], dtype=np.float64)


@pytest.mark.parametrize("n,world", [(128, 2), (5, 2), (7, 3), (1, 4), (0, 2)])
def test_walker_slices_partition(n, world):
    seen = []
    sizes = []
    for r in range(world):
        s, e = shard.walker_slice(n, r, world)
        seen.extend(range(s, e))
        sizes.append(e - s)
    assert seen == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, n_walkers, mode, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
        store = dist.TCPStore("127.0.0.1", port + 1, world, is_master=(rank == 0),
                              timeout=datetime.timedelta(seconds=30))
        hb = shard.Heartbeat(store, rank, world, timeout_s=10.0)
        s, e = shard.walker_slice(n_walkers, rank, world)
        local = fake_chi2(range(s, e))
        if mode == "leave" and rank == 1:
            hb.leave(0)                       # leaves between steps, nothing in flight
            q.put((rank, "left"))
            return
        hb.wait_all(0)                        # membership known on the host before the exchange
        full = shard.gather_chi2(local, n_walkers)
        tmax = shard.max_over_ranks(10.0 + rank)
        q.put((rank, "ok", None if full is None else full.tolist(), tmax))
        dist.destroy_process_group()
    except Exception as exc:   # reported to the parent
        q.put((rank, "error", type(exc).__name__))
        q.close()
        q.join_thread()                       # the report is on its way before the process ends
        os._exit(0)                           # leave without tearing down a group a peer abandoned


def run(world, n_walkers, mode="normal"):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_walkers, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    return sorted(out, key=lambda x: x[0])


def test_gather_chi2_and_max_over_two_gloo_ranks():
    res = run(2, 9)
    assert [r[1] for r in res] == ["ok", "ok"]
    np.testing.assert_array_equal(np.array(res[0][2]), fake_chi2(range(9)))
    assert res[1][2] is None
    assert res[0][3] == res[1][3] == 11.0


def test_rank_leaving_before_the_exchange_is_seen_as_an_error():
    res = run(2, 6, mode="leave")
    assert res[1][1] == "left"
    assert res[0][1] == "error" and res[0][2] == "RankLeft"   # learnt on the host, no collective entered
