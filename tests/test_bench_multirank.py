"""The multi-rank host logic of bench.py on CPU (two gloo ranks).

Under torchrun every rank solves its own replica of the scene (views are
independent until the additive sum over views, Eq. 6, and this build runs one
GPU per process: replicas only).  The line rank 0 prints takes the slowest
rank's time and all ranks' pixels; the reference arm runs on rank 0 alone.
"""
import contextlib
import io
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduce_worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 180.0][rank]          # rank 1 is the slower replica
        total = bench.max_over_ranks(ms, world, "cpu")
        q.put((rank, total, bench.whole_job_gpix(world, 76_204_800, 5, total)))
    finally:
        dist.destroy_process_group()


def _reference_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                "--n", "3000", "--views", "2"]
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.main()
    q.put((rank, out.getvalue()))


def _spawn(fn, world=2):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=fn, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res)


def test_slowest_rank_sets_the_time_and_all_pixels_count():
    pytest.importorskip("torch")
    res = _spawn(_reduce_worker)
    for rank, total, gpix in res:
        assert total == 180.0
        assert gpix == pytest.approx(2 * 76_204_800 * 5 / 0.180 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    pytest.importorskip("torch")
    res = _spawn(_reference_worker)
    (r0, out0), (r1, out1) = res
    assert r0 == 0 and r1 == 1
    lines = [l for l in out0.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert out1.strip() == ""
