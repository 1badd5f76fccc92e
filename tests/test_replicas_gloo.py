"""The multi-rank bench path on CPU: two gloo ranks (processes) run the
replica aggregation the bench uses under torchrun, with no GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_reduce(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, c = bench.reduce_over_ranks([3.0, 5.0][rank], {"scenarios": 10 + rank, "converged": rank})
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"reduce{rank}.txt"), "w") as f:
        f.write(f"{t!r} {c['scenarios']!r} {c['converged']!r}\n")


def _rank_gather(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = bench.gather_objects({"rank": rank, "recs": list(range(rank + 1))})
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"gather{rank}.txt"), "w") as f:
        f.write(repr(parts) + "\n")


def _rank_main(rank, world, port, times, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    rate, tmax = bench.whole_job_rate(times[rank], steps=20)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{rate!r} {tmax!r}\n")


def test_whole_job_rate_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    times = [0.5, 0.8]
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, times, str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    for rank in range(2):
        rate, tmax = map(float, (tmp_path / f"rank{rank}.txt").read_text().split())
        # every rank sees the slowest rank's time and the whole job's rate
        assert tmax == 0.8
        assert rate == pytest.approx(2 * 20 / 0.8)


def test_whole_job_rate_single_process():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    rate, tmax = bench.whole_job_rate(0.25, steps=10)
    assert tmax == 0.25 and rate == pytest.approx(40.0)


def test_shard_scenarios_partition_is_balanced_and_covering():
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    rng = np.random.default_rng(3)
    sizes = list(np.exp(rng.uniform(np.log(500), np.log(20000), 256)).astype(int))
    for ws in (1, 2, 3, 8):
        parts = [bench.shard_scenarios(sizes, ws, r) for r in range(ws)]
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(sizes)))                 # disjoint and covering
        loads = [sum(sizes[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)           # longest-first balance
        assert parts == [bench.shard_scenarios(sizes, ws, r) for r in range(ws)]


def test_reduce_over_ranks_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_reduce, args=(2, port, str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    for rank in range(2):
        t, n, conv = map(float, (tmp_path / f"reduce{rank}.txt").read_text().split())
        assert (t, n, conv) == (5.0, 21.0, 1.0)


def test_gather_objects_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    import ast
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_gather, args=(2, port, str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    want = [{"rank": 0, "recs": [0]}, {"rank": 1, "recs": [0, 1]}]
    for rank in range(2):
        assert ast.literal_eval((tmp_path / f"gather{rank}.txt").read_text()) == want
