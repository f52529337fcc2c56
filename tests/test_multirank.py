"""The benchmark's multi-rank path on the host: two gloo ranks (one process per GPU on a GPU machine).

The sweep runs as independent replicas, one per rank (no data-path collective); only the timing
is combined: the whole-job rate is every rank's updates over the slowest rank's time, and the
reference arm runs on rank 0 alone.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    try:
        local_ms = 10.0 * (rank + 1)                       # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, ws, "cpu")
        lups = 512 ** 3 * 64
        rate = bench.whole_job_glups(lups, 5, ws, ms)
        ws_env, rank_env, local_env = bench._dist()
        ref_rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": ws})(), "7pt_const_f64_512") \
            if rank != 0 else None                         # ranks other than 0 return at once
        q.put((rank, ms, rate, (ws_env, rank_env, local_env), ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_timing():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    lups = 512 ** 3 * 64
    for rank, ms, rate, env, ref_rc in out:
        assert ms == 20.0                                  # the slowest rank's time on every rank
        assert rate == pytest.approx(lups * 5 * 2 / 0.020 * 1e-9)
        assert env == (2, rank, rank)
        assert ref_rc == (None if rank == 0 else 0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_glups(1e9, 2, 1, 1000.0) == pytest.approx(2.0)
