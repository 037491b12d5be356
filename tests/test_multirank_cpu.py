"""The multi-GPU path of bench.py is query-parallel replicas: every rank runs
the same index on its own batch, the only cross-rank steps are a barrier and a
max-reduction of the timed region, and the job throughput divides all ranks'
queries by the slowest rank's time.  These host-side steps run here as two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as distd  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    distd.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        ms = [120.0, 180.0][rank]  # rank 1 is the slow one
        distd.barrier()
        slowest = bench.max_over_ranks(ms, w, "cpu")
        out[rank] = (r, w, lr, slowest, bench.job_qps(10_000, 20, w, slowest))
    finally:
        distd.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][:3] == (0, 2, 0) and res[1][:3] == (1, 2, 1)
    for r in (0, 1):
        assert res[r][3] == 180.0  # every rank sees the slowest rank's time
        assert res[r][4] == pytest.approx(2 * 10_000 * 20 / 0.180)


def test_single_rank_needs_no_group():
    assert bench.max_over_ranks(42.5, 1) == 42.5
    assert bench.job_qps(100, 3, 1, 1000.0) == pytest.approx(300.0)
