"""The multi-rank side of bench.py on CPU ranks (gloo, world size 2): the job time is the
maximum over ranks, ranks solve disjoint images, and the reference arm prints on rank 0
only. The GPU work itself runs one replica per GPU with no data-path collective."""
import io
import contextlib
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)
    seeds = bench.problem_seeds(rank)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        if rank != 0:
            bench.run_reference(None, rank, world)   # returns at once on rank != 0
    dist.barrier()
    q.put((rank, t, seeds, out.getvalue()))
    dist.destroy_process_group()


def test_two_gloo_ranks_time_is_max_and_images_are_disjoint():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, t, seeds, printed = q.get(timeout=120)
        res[rank] = (t, seeds, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 15.0
    assert not set(res[0][1]) & set(res[1][1])
    assert len(res[0][1]) == len(res[1][1]) == 10
    assert res[1][2] == ""


def test_single_rank_time_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.problem_seeds(0) == list(range(10))


def test_reference_arm_prints_one_valid_line():
    """`bench.py --impl reference` times the FP64 oracle on the host and prints one JSON
    line with the contract's keys (no GPU involved)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
