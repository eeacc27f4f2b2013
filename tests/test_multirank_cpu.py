"""The N > 1 path of bench.py on CPU: two gloo ranks (independent replicas).
The job's time is the slowest rank's, the value counts every rank's units,
and the reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_setup(None) == (world, rank, rank)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    value = bench.whole_job_value(1e6, 4, world, ms)
    # the reference arm: ranks other than 0 return at once, without work
    ref = None
    if rank != 0:
        ref = bench.run_reference(None, world, rank)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(result_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{ms} {value} {ref}")


def test_two_gloo_ranks(tmp_path):
    world, port = 2, _free_port()
    ctx = torch.multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, value, ref = open(tmp_path / f"r{r}.txt").read().split()
        assert float(ms) == 15.0                       # the slowest rank's time
        assert float(value) == pytest.approx(2 * 1e6 * 4 / 0.015)
        assert ref == "None"
