"""Replicas across processes (one per GPU in a real run), exercised on CPU with gloo.

Windows are independent, so N GPUs run N replicas with no collective on the data path; the
only cross-rank steps are the timing barrier and the max over ranks of the step time. Two
gloo ranks check those helpers of bench.py, the whole-job rate and that each rank draws its
own frames.
"""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from dh_synth import SpeckleParams, SpeckleStream
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    step_ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    ms_max = bench.max_over_ranks(step_ms, ws)
    rate = bench.whole_job_rate(64, ws, ms_max)
    # the bench's per-rank stream: seed 1000 + rank
    f = SpeckleStream(SpeckleParams(32, 32), seed=1000 + rank).next(2)
    ref_rc = None
    if rank == 1:  # the reference arm does its work on rank 0 only
        class A:  # minimal argument namespace
            steps, warmup, gpus = 1, 0, world
        ref_rc = bench.run_reference(A, ws, rank)
    torch.save({"ms_max": ms_max, "rate": rate, "frames": f, "ref_rc": ref_rc},
               os.path.join(out_dir, f"r{rank}.pt"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r0 = torch.load(tmp_path / "r0.pt")
    r1 = torch.load(tmp_path / "r1.pt")
    assert r0["ms_max"] == r1["ms_max"] == 15.0      # every rank sees the slowest rank's time
    assert r0["rate"] == r1["rate"] == pytest.approx(2 * 64 / 0.015)
    assert not torch.equal(r0["frames"], r1["frames"])  # each replica has its own data
    assert r1["ref_rc"] == 0
