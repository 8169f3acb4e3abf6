"""Multi-process (replica) path of bench.py on CPU: two gloo ranks on 127.0.0.1.

On N GPUs every rank renders its own replica of the workload with no collective on the data
path; the only cross-rank steps are the barrier around the timed region and the maximum of
the per-rank times.  These tests run that host-side logic with the gloo backend, and check
that the reference arm does its work on rank 0 only.
"""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.dist_env()
        ms = bench.max_over_ranks(10.0 + 5.0 * r, w, "cpu")  # rank 1 is the slow one
        dist.barrier()
        out.put((r, w, lr, ms, bench.job_mpix_s(2_073_600, w, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res) and [r[2] for r in res] == [0, 1]
    assert all(r[3] == 15.0 for r in res)  # both ranks report the max of 10 and 15 ms
    # whole-job rate: both replicas' pixels in the slowest rank's time
    assert all(abs(r[4] - 2 * 2_073_600 / 15e-3 / 1e6) < 1e-9 for r in res)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_mpix_s(1_000_000, 1, 1.0) == pytest.approx(1000.0)


def _reference_rank(rank, out):
    sys.path.insert(0, ROOT)
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank))
    import contextlib
    import io
    import bench

    class A:  # the arguments run_reference reads
        workload, steps, warmup, cpu_seconds, gpus = "pinhole_1k_64", 1, 0, 0.5, 2

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A())
    out.put((rank, buf.getvalue()))


def test_reference_arm_runs_on_rank_zero_only():
    pytest.importorskip("oracle")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_reference_rank, args=(r, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[1] == ""
    line = json.loads(res[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
