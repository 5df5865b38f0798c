"""The multi-rank (N > 1) path of bench.py on CPU: two gloo ranks over
127.0.0.1 check that each rank gets its own volume, that the only collective
(the max of the ranks' times) gives every rank the slowest time, and that the
whole-job value counts every rank's volumes over that time."""
import importlib.util
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("sift3d_bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        import sys
        sys.path.insert(0, ROOT)
        from workloads.volumes import brain_like_volume
        vol = brain_like_volume(seed=b.rank_volume_seed(rank), shape=(24, 20, 18))
        my_ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
        total = b._max_over_ranks(dist, my_ms, device="cpu")
        value = b.whole_job_value(world, 7, vol.size, total)
        out[rank] = (float(vol.sum()), total, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_reduction():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn",
                           join=True)
        res = dict(out)
    (s0, t0, v0), (s1, t1, v1) = res[0], res[1]
    assert s0 != s1                                    # distinct volumes per rank
    assert t0 == t1 == 15.0                            # every rank sees the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 7 * 24 * 20 * 18 / 15e-3)


def test_single_rank_needs_no_collective():
    b = _bench()
    assert b._max_over_ranks(None, 3.5) == 3.5
    assert b.whole_job_value(1, 10, 1000, 2.0) == pytest.approx(5e6)
    assert b.rank_volume_seed(0) != b.rank_volume_seed(1)
