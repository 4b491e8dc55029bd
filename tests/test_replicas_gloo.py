"""The multi-rank bookkeeping of the benchmark (independent replicas, one process per rank) on
the host: two gloo ranks meet at the barriers, the slowest rank's time wins, and the whole-job
rate counts every rank's units.  No GPU: the device synchronisations are switched off."""
import json
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2606_25026_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, times):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r = replicas.from_env()
    replicas.init(r, backend="gloo")
    replicas.barrier(r, cuda=False)
    slowest = replicas.max_over_ranks(r, times[rank])
    rate = replicas.job_rate(r, 1000.0, slowest)
    replicas.barrier(r, cuda=False)
    replicas.finish(r)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"rank": r.rank, "world": r.world, "leader": r.leader, "slowest": slowest, "rate": rate}, f)


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    times = [0.5, 2.0]
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path), times), nprocs=2,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(2)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == 2 for x in res)
    assert [x["leader"] for x in res] == [True, False]
    for x in res:
        assert x["slowest"] == 2.0
        assert x["rate"] == pytest.approx(2 * 1000.0 / 2.0)


def test_one_rank_needs_no_process_group():
    r = replicas.from_env({})
    assert (r.rank, r.world, r.local, r.leader) == (0, 1, 0, True)
    replicas.init(r)                      # no process group for one rank
    assert replicas.max_over_ranks(r, 3.5) == 3.5
    assert replicas.job_rate(r, 10.0, 2.0) == 5.0
    replicas.finish(r)


@pytest.mark.parametrize("env", [{"RANK": "2", "WORLD_SIZE": "2"}, {"WORLD_SIZE": "0"},
                                 {"RANK": "-1", "WORLD_SIZE": "2"}, {"LOCAL_RANK": "-1"}])
def test_inconsistent_rank_environment_is_rejected(env):
    with pytest.raises(ValueError):
        replicas.from_env(env)


def test_job_rate_rejects_a_zero_time():
    with pytest.raises(ValueError):
        replicas.job_rate(replicas.Ranks(0, 1, 0), 1.0, 0.0)


def test_reference_arm_runs_on_the_leader_only(monkeypatch):
    """Under torchrun the CPU reference arm runs on rank 0 alone; other ranks exit 0 at once."""
    import bench

    def boom(*a, **k):
        raise AssertionError("a non-leader rank built inputs")

    monkeypatch.setattr(bench, "make_inputs", boom)
    args = types.SimpleNamespace(workload="halo256_stars1e6", steps=1, warmup=1)
    assert bench.reference_arm(args, 1, 2) == 0
