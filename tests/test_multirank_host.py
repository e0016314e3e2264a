"""The multi-rank bench path on CPU: world_size-2 gloo ranks combine their step
times (max) and their work units (sum) the way bench.py does on NCCL, and each
rank traces its own paths of the same workload (distinct Philox seeds)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]
        units = [1000, 3000][rank]
        out[rank] = bench.job_totals(ms, units, dist, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_combine_max_time_and_summed_units():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        ctx_procs = []
        port = _free_port()
        for r in range(2):
            p = ctx.Process(target=_rank, args=(r, 2, port, out))
            p.start()
            ctx_procs.append(p)
        for p in ctx_procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == (150.0, 4000.0) and out[1] == (150.0, 4000.0)


def test_ranks_trace_independent_paths_of_the_same_workload():
    """Rank r keys its Philox stream with seed + 1000 r: same scene and image, other paths."""
    import bench
    a = bench.workload("heterogeneous", seed_offset=0, image=16, spp=1)
    b = bench.workload("heterogeneous", seed_offset=1000, image=16, spp=1)
    assert a["opts"]["seed"] != b["opts"]["seed"]
    assert a["camera"] == b["camera"] and a["opts"]["spp"] == b["opts"]["spp"]


def test_single_rank_is_identity():
    import bench
    assert bench.job_totals(12.5, 7) == (12.5, 7.0)
