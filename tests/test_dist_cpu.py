"""The bench's multi-process path (one process per GPU, independent replicas,
barrier + max-over-ranks timing) exercised with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local = bench.dist_init()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    m = bench.max_over_ranks(1.5 + rank, ws)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{m}\n")
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_barrier_and_max(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    vals = [float(open(tmp_path / f"rank{r}.txt").read()) for r in range(world)]
    assert vals == [2.5, 2.5]


def _ref_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    ws, r, _ = bench.dist_init()
    # non-zero ranks of the reference arm do no work and produce no line
    if r != 0:
        assert bench.run_reference(None, ws, r) is None
    with open(os.path.join(out_dir, f"ok{rank}"), "w") as f:
        f.write("ok")
    import torch.distributed as dist
    dist.destroy_process_group()


def test_reference_arm_other_ranks_idle(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_ref_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    assert (tmp_path / "ok0").exists() and (tmp_path / "ok1").exists()
