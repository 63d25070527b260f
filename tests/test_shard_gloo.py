"""The multi-rank path on CPU: two gloo ranks in child processes.

Independent systems shard with no data exchange.  Every rank computes the
same partition; the ranks agree on the slowest rank's time and gather their
reports on rank 0, which is all the bench's N-GPU arm needs from them.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2604_01800_gb300 import inputs as I  # noqa: E402
from paper_2604_01800_gb300 import shard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_is_a_balanced_cover():
    ws = I.config4(64)
    costs = [shard.system_cost(w.nx, w.ny) for w in ws]
    for world in (1, 2, 3, 8):
        parts = shard.partition(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(64))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: no rank exceeds the mean by more than the largest system
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
    assert shard.partition([3.0, 1.0, 2.0], 2) == [[0], [1, 2]]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def test_single_rank_helpers_without_a_process_group():
    assert shard.max_over_ranks(2.5) == 2.5
    assert shard.gather_to_rank0({"a": 1}) == [{"a": 1}]
    assert shard.job_rate([10, 6], [2.0, 4.0]) == 4.0


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws = I.config4(16)
        costs = [shard.system_cost(w.nx, w.ny) for w in ws]
        mine = shard.partition(costs, world)[rank]
        # a stand-in for each rank's timed work: its share's cost
        seconds = sum(costs[i] for i in mine) / 1e9
        t = shard.max_over_ranks(seconds)
        reports = shard.gather_to_rank0({"rank": rank, "systems": mine, "seconds": seconds})
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(repr((t, reports)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_partition_time_and_reports(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    res = [eval(open(tmp_path / f"r{r}.txt").read()) for r in range(world)]
    (t0, rep0), (t1, rep1) = res
    assert rep1 is None and len(rep0) == world
    assert [r["rank"] for r in rep0] == [0, 1]
    got = sorted(i for r in rep0 for i in r["systems"])
    assert got == list(range(16))                             # disjoint cover, no system twice
    assert t0 == t1 == max(r["seconds"] for r in rep0)        # both ranks hold the slowest rank's time
    rate = shard.job_rate([len(r["systems"]) for r in rep0], [r["seconds"] for r in rep0])
    assert abs(rate - 16 / t0) <= 1e-12 * rate
