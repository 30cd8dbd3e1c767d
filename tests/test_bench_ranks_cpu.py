"""The benchmark's multi-rank path on the CPU: two gloo ranks run bench.py's
barrier, max-over-ranks timing and whole-job throughput, and the reference
arm prints its contract line (no GPU needed)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.rank_barrier(world)
        local_ms = 10.0 + 5.0 * rank          # the slower rank takes 15 ms
        ms = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        value = bench.job_rate(1000, world, ms)
        bench.rank_barrier(world)
        out.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0                      # every rank sees the maximum
        assert value == pytest.approx(2 * 1000 / 0.015)   # units of both ranks over the slowest time


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    bench.rank_barrier(1)
    assert bench.job_rate(500, 1, 250.0) == pytest.approx(2000.0)


def test_reference_arm_prints_its_contract_line():
    env = dict(os.environ, RSC_REF_QUERIES="16")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "3000",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"
