"""The multi-process path of bench.py on CPU (gloo, world size 2).

Every rank runs an independent replica of the workload (its own seeded
blocks, no collective on the data path); the only exchanges are the barrier
around the timed region and the max-over-ranks of the step time, and the
reported value is all ranks' bytes over the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.rank_env()
        ms = 1.0 + 2.0 * r                         # rank 1 is the slow one
        dist.barrier()
        ms_max = bench.max_over_ranks(ms, w, device="cpu")
        seeds = [bench.replica_seed(1000, r)]
        gathered = [None] * w
        dist.all_gather_object(gathered, seeds)
        out[rank] = (w, r, l, ms_max, bench.job_gbs(1e9, ms_max, w), gathered)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_report_max_time_and_summed_bytes():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (w, r, l, ms_max, gbs, gathered) in res.items():
        assert (w, r, l) == (2, rank, rank)
        assert ms_max == 3.0                      # the slowest rank's time, seen by every rank
        assert gbs == pytest.approx(2 * 1e9 / 3e-3 / 1e9)
        s0, s1 = gathered[0][0], gathered[1][0]
        assert s0 != s1                           # independent replicas draw different blocks


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.rank_env() == (1, 0, 0)
        assert bench.max_over_ranks(2.5, 1) == 2.5
        assert bench.job_gbs(2e9, 1.0, 1) == pytest.approx(2000.0)
    finally:
        os.environ.update(env)
