"""The multi-GPU form is replicas only (every glyph and query is independent; no data-path
collective).  What runs across ranks is the benchmark's timing aggregation: a barrier, the max of
the per-rank step times and the whole-job rate.  Exercised here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = bench.reduce_over_ranks(times[rank], dist, "cpu")
    rate = bench.whole_job_rate(1000.0, world, ms)
    # per-rank replicas draw different inputs (weak scaling)
    args = bench.parse_args(["--glyphs", "4", "--per-glyph", "8", "--engine", "simt"])
    w = bench.GlyphField(args, rank)
    out[rank] = (ms, rate, float(w.c_host[0, 1]))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, _free_port(), [3.0, 5.0], out), nprocs=world, join=True)
    (ms0, r0, c0), (ms1, r1, c1) = out[0], out[1]
    assert ms0 == ms1 == 5.0                         # the slowest replica
    assert r0 == r1 == pytest.approx(2 * 1000.0 / 5e-3)
    assert c0 != c1                                  # different glyphs per rank


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(4.0, None) == 4.0
    assert bench.whole_job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
