"""The multi-rank host logic of bench.py on two gloo ranks (CPU): every rank
traces its own Philox streams of the same workload (weak scaling, no data
exchange) and the job's time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    streams = [bench.rank_stream_base(rank, g) for g in range(4)]
    gathered = [None] * world
    dist.all_gather_object(gathered, streams)
    t = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))
    dist.barrier()
    q.put((rank, gathered, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_trace_disjoint_streams_and_report_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t in out:
        assert t == 11.0
        ids = [s for per_rank in gathered for s in per_rank]
        assert len(set(ids)) == len(ids)  # no two (rank, group) pairs share a Philox stream
        # a sweep group spans at most 128 stream ids (96 cases): the ranges do not overlap
        spans = sorted((s, s + 96) for s in ids)
        assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
