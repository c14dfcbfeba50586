"""Host logic of `bench.py --gpus N` on CPU ranks (gloo, world size 2): every rank runs an
independent replica, the job's time is the largest per-rank time (all-reduce MAX) and the
value counts the units of all ranks; under torchrun the reference arm runs on rank 0 alone
and prints one JSON line while the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, r = bench.dist_setup()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, ws)
    rate = bench.job_rate(1_000_000, ws, ms)
    out_q.put((r, ws, ms, rate))
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for _, ws, ms, rate in res:
        assert ws == 2 and ms == 15.0  # the slower rank's time on every rank
        assert abs(rate - 2 * 1_000_000 / 15e-3 / 1e9) < 1e-12


def test_reference_arm_under_torchrun_prints_on_rank_zero_only():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["e2e"]["h2d_bytes_per_step"] == 0
