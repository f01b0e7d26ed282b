"""The N > 1 path of bench.py on CPU: two gloo ranks shard the subdomains (independent split
draws per rank, no data-path collective) and agree on the job's time (max over ranks) and value."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import bench
    from paper_2512_11087_gb300 import workloads as WL
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank
    t = bench.job_time_ms(local_ms, dist, "cpu")
    B, steps = 100, 3
    value = bench.job_value(world, B, steps, t)
    ids = np.arange(40, 140, dtype=np.int64)
    so, si = WL.draw_splits(ids, B, 1, 4, seed=bench.shard_seed(rank))
    shards = [None] * world
    dist.all_gather_object(shards, si.tolist())
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(dict(t=t, value=value, shards=shards, so=so.tolist()), f)


def test_two_gloo_ranks_shard_and_agree(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    # the job's time is the slowest rank's, on every rank
    assert r[0]["t"] == r[1]["t"] == 15.0
    assert r[0]["value"] == r[1]["value"] == pytest.approx(world * 100 * 3 / 0.015)
    # each rank bounds its own batch: different split draws, each a valid CSR over the candidates
    assert r[0]["shards"][0] != r[0]["shards"][1]
    for k in range(world):
        so = np.array(r[k]["so"])
        assert so[0] == 0 and np.all(np.diff(so) >= 1) and np.all(np.diff(so) <= 4)
        codes = np.abs(np.array(r[0]["shards"][k])) - 1
        assert np.all((codes >= 40) & (codes < 140))


def test_single_rank_time_is_local():
    import bench
    assert bench.job_time_ms(12.5) == 12.5
    assert bench.job_value(1, 4096, 10, 1000.0) == pytest.approx(40960.0)


def _summary_rank(rank, world, port, out_dir):
    from paper_2512_11087_gb300 import engine as E
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    # the layout cv_round_summary writes: [least lower bound, least unverified lower bound], [verified, infeasible]
    local = {0: ([-0.5, -0.5], [10, 2]), 1: ([0.25, float("inf")], [30, 0])}[rank]
    s = E.reduce_round_summary(torch.tensor(local[0], dtype=torch.float32), torch.tensor(local[1], dtype=torch.int32),
                               dist)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"sum{rank}.json"), "w") as f:
        json.dump(s, f)


def test_round_summary_reduces_over_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_summary_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"sum{k}.json")) for k in range(world)]
    assert r[0] == r[1]
    assert r[0] == dict(lower_min=-0.5, lower_min_unverified=-0.5, verified=40, infeasible=2)


def test_round_summary_without_a_group_is_local():
    from paper_2512_11087_gb300 import engine as E
    s = E.reduce_round_summary(torch.tensor([1.0, float("inf")]), torch.tensor([3, 1], dtype=torch.int32))
    assert s == dict(lower_min=1.0, lower_min_unverified=float("inf"), verified=3, infeasible=1)
