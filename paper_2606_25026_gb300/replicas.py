"""Multi-rank bookkeeping for the replica benchmark.

The split-step grid does not shard here: N ranks (one process per GPU, launched by
``torch.distributed.run``) each step their own replica of the same workload, and the job's
throughput is the units every rank processed over the slowest rank's time (weak scaling).  The
only collectives are a barrier around the timed region and one MAX reduction of the measured
times; nothing is exchanged on the data path.

Everything here works on any ``torch.distributed`` backend: ``nccl`` on the GPUs, ``gloo`` on the
host (which the CPU tests use with world size 2).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class Ranks:
    rank: int
    world: int
    local: int

    @property
    def leader(self) -> bool:
        return self.rank == 0


def from_env(env=None) -> Ranks:
    """RANK / WORLD_SIZE / LOCAL_RANK as ``torch.distributed.run`` sets them (1 rank without)."""
    env = os.environ if env is None else env
    r = Ranks(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0")))
    if r.world < 1 or not 0 <= r.rank < r.world or r.local < 0:
        raise ValueError(f"inconsistent rank environment {r}")
    return r


def init(r: Ranks, backend: str = "nccl", device=None) -> None:
    """Join the process group (a no-op for one rank)."""
    if r.world == 1:
        return
    import torch.distributed as dist
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=device)
    else:
        dist.init_process_group(backend)
    dist.barrier()


def finish(r: Ranks) -> None:
    if r.world == 1:
        return
    import torch.distributed as dist
    dist.barrier()
    dist.destroy_process_group()


def barrier(r: Ranks, cuda: bool = True) -> None:
    """Device work drained on this rank, then all ranks meet, then drained again."""
    import torch
    if cuda:
        torch.cuda.synchronize()
    if r.world > 1:
        import torch.distributed as dist
        dist.barrier()
        if cuda:
            torch.cuda.synchronize()


def max_over_ranks(r: Ranks, x: float, device="cpu") -> float:
    """The largest of the ranks' values (the slowest rank's time)."""
    if r.world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(r: Ranks, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's seconds."""
    if seconds <= 0:
        raise ValueError("non-positive time")
    return r.world * units_per_rank / seconds
