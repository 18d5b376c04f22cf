"""Walker sharding across processes, one GPU each.

The likelihood path partitions by walker: every rank evaluates its own walkers on its own
GPU against its own copy of the density spectra, with no exchange on the data path. The
one exchange step is the sampler's: it needs every walker's chi^2 on one rank (a few KB
per batch). These helpers do that over any torch.distributed backend (gloo on CPU, NCCL
on GPUs), plus the max-over-ranks of a timing.
"""
from __future__ import annotations

import numpy as np


def walker_slice(n_walkers: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of this rank's walkers: contiguous, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n_walkers < 0:
        raise ValueError("bad rank/world/walker count")
    base, extra = divmod(n_walkers, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _device_for(backend: str):
    import torch
    return torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")


def gather_chi2(chi2_local: np.ndarray, n_walkers: int, dst: int = 0) -> np.ndarray | None:
    """Every rank's chi^2 (in walker order) on rank `dst`; None on the other ranks."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(), dist.get_rank()
    dev = _device_for(dist.get_backend())
    width = -(-n_walkers // world)                       # ceil: equal-size chunks for all_gather
    buf = torch.full((width,), float("nan"), dtype=torch.float64, device=dev)
    start, stop = walker_slice(n_walkers, rank, world)
    if stop - start != len(chi2_local):
        raise ValueError("chi2_local does not match this rank's walker slice")
    buf[: stop - start] = torch.as_tensor(np.asarray(chi2_local, dtype=np.float64), device=dev)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    if rank != dst:
        return None
    out = np.empty(n_walkers)
    for r in range(world):
        s, e = walker_slice(n_walkers, r, world)
        out[s:e] = parts[r][: e - s].cpu().numpy()
    return out


def max_over_ranks(value: float) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device_for(dist.get_backend()))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class RankLeft(RuntimeError):
    """A rank announced that it left before an exchange step."""


class Heartbeat:
    """Host-side membership check before each exchange step, over a key-value store
    (torch.distributed.TCPStore): each rank marks step s as reached ("arrive") or
    announces that it leaves ("left"); wait_all(s) returns when every rank has arrived,
    raises RankLeft if one left, and TimeoutError if one neither arrives nor leaves within
    the timeout. Ranks thus learn of a departure on the host, before their next collective
    or kernel launch, instead of inside a collective."""

    def __init__(self, store, rank: int, world: int, timeout_s: float = 30.0, poll_s: float = 0.01):
        self.store, self.rank, self.world = store, rank, world
        self.timeout_s, self.poll_s = timeout_s, poll_s

    def arrive(self, step: int) -> None:
        self.store.set(f"hb/{step}/arrive/{self.rank}", "1")

    def leave(self, step: int) -> None:
        self.store.set(f"hb/{step}/left/{self.rank}", "1")

    def wait_all(self, step: int) -> None:
        import time
        self.arrive(step)
        deadline = time.monotonic() + self.timeout_s
        pending = set(range(self.world))
        while pending:
            for r in list(pending):
                if self.store.check([f"hb/{step}/left/{r}"]):
                    raise RankLeft(f"rank {r} left before step {step}")
                if self.store.check([f"hb/{step}/arrive/{r}"]):
                    pending.discard(r)
            if pending:
                if time.monotonic() > deadline:
                    raise TimeoutError(f"ranks {sorted(pending)} did not reach step {step}")
                time.sleep(self.poll_s)
