"""The multi-rank logic of bench.py on CPU: world_size-2 gloo ranks reduce
the timed region to the maximum wall time and the summed work, and the
reference arm runs on rank 0 only."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 + 5 r ms of wall time, 1e12 (r + 1) flops
        t, w = bench.aggregate(10.0 + 5.0 * rank, 1e12 * (rank + 1), world, "cpu")
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"t": t, "w": w}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_work(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as f:
            got = json.load(f)
        assert got == {"t": 15.0, "w": 3e12}


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(7.5, 2.0, 1) == (7.5, 2.0)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(workload="plummer-2^14", warmup=0, steps=1, cpu_groups=10)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("rank", [0, 3])
def test_replica_workloads_are_seeded_per_rank(rank):
    import bench
    m0, _ = bench._workload("plummer-2^14", 0)
    m, _ = bench._workload("plummer-2^14", rank)
    assert m.n == m0.n
    assert (m.pos == m0.pos).all() == (rank == 0)
