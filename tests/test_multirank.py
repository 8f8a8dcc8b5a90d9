"""The multi-rank path of bench.py on the host (no GPU): two gloo ranks launched
as torchrun would launch them (RANK / WORLD_SIZE / MASTER_ADDR in the
environment).  Every rank times its own replica; the job's time is the slowest
rank's (max over ranks) and its throughput the units of all ranks over that
time (weak scaling, no collective on the data path)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [0.8, 1.25][rank]  # rank 1 is the slow one
    tmax = bench._max_over_ranks(seconds, dist)
    rate = bench.whole_job_rate(1000, ws, tmax)
    assert bench._sum_over_ranks([100.0, 250.0][rank], dist) == 350.0
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{tmax} {rate}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in (0, 1):
        tmax, rate = map(float, open(tmp_path / f"rank{rank}.txt").read().split())
        assert tmax == 1.25
        assert abs(rate - 2 * 1000 / 1.25) < 1e-9


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def _study_rank(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2404_14195_gb300 import studies
    dist, r, ws, local = studies.dist_env()
    assert (r, ws, local) == (rank, world, rank)
    seen = []

    def fn(x):
        seen.append(x)
        return dict(x=x, rank=rank)
    res = studies.run_sharded(fn, [0.1, 0.2, 0.3, 0.4, 0.5], dist, r, ws)
    with open(os.path.join(out_dir, f"study{rank}.txt"), "w") as f:
        f.write(repr((seen, res)) + "\n")
    dist.destroy_process_group()


def test_studies_shard_runs_over_gloo_ranks(tmp_path):
    """The studies' runs (independent cells) go round-robin to the ranks; every
    rank ends with all results in item order."""
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_study_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    import ast
    got = [ast.literal_eval(open(tmp_path / f"study{r}.txt").read()) for r in (0, 1)]
    assert got[0][0] == [0.1, 0.3, 0.5] and got[1][0] == [0.2, 0.4]
    want = [dict(x=x, rank=i % 2) for i, x in enumerate([0.1, 0.2, 0.3, 0.4, 0.5])]
    assert got[0][1] == want and got[1][1] == want


def test_studies_single_process():
    sys.path.insert(0, ROOT)
    from paper_2404_14195_gb300 import studies
    assert studies.run_sharded(lambda x: 2 * x, [1, 2, 3]) == [2, 4, 6]


def test_batch_cells_are_disjoint_per_rank():
    """Rank r's cells of the batched workload are the r-th block of one seeded
    sequence: rank 0 keeps the one-GPU cells, the ranks share no cell."""
    sys.path.insert(0, ROOT)
    import bench
    one = bench.config3_jobs(4)
    two = bench.config3_jobs(8)
    assert bench.config3_jobs(4, rank=0) == one == two[:4]
    assert bench.config3_jobs(4, rank=1) == two[4:]
    seeds = [j[2] for j in bench.config3_jobs(4, rank=0) + bench.config3_jobs(4, rank=1)]
    assert len(set(seeds)) == 8
