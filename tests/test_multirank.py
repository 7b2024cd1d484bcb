"""Host logic of bench.py's multi-process run (one process per GPU under
torchrun), exercised on CPU with the gloo backend and two ranks: whole-job
totals (segments and solves summed, time the maximum over ranks), distinct
atmospheres per rank, and the reference arm's non-zero ranks exiting
without work."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2102_01734_gb300 import inputs

    # rank r: 10 + r formal solutions of 1000 segments, 2 + r seconds, 3 solves
    segs, secs, solves = bench.job_totals((10 + rank) * 1000, 2.0 + rank, 3)
    chi, _, _, _ = inputs.cartesian_config(9, 1e-6, seed=1 + rank)
    digest = torch.tensor([float(np.sum(chi))], dtype=torch.float64)
    digests = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(digests, digest)
    out[rank] = (segs, secs, solves, [d.item() for d in digests])
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    for rank in range(world):
        segs, secs, solves, digests = res[rank]
        assert segs == (10 + 11) * 1000  # summed over ranks
        assert secs == 3.0  # the slower rank
        assert solves == 6
        assert digests[0] != digests[1]  # each rank its own atmosphere


def test_job_totals_single_process():
    import bench

    assert bench.job_totals(5, 2.0, 1) == (5.0, 2.0, 1.0)


def test_reference_arm_rank1_exits_without_work(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(None) == 0
