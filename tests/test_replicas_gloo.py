"""The multi-process path of bench.py (independent replicas, one per GPU) on CPU ranks
with the gloo backend: the timed region is the maximum over ranks and the value counts
the steps of every rank; the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.reduce_timing(100.0 + 50.0 * rank, 3, world, dist)
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_timing_is_max_over_ranks_and_value_counts_all_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()   # both ranks rendezvous on one port
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == 150.0
        assert value == pytest.approx(world * 3 / 0.150)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_keeps_the_contract():
    """Rank 0's reference line: the keys of the benchmark line, the oracle as cpu_baseline,
    e2e with zero host-device bytes, and the ILO width in the config when asked for."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    for extra, want_rb in (([], None), (["--r-bond", "2"], 2)):
        r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                            "--warmup", "0", "--D", "6"] + extra,
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        line = json.loads(r.stdout.strip().splitlines()[-1])
        for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
                  "ms_per_step", "higher_is_better", "config", "cpu_baseline", "e2e"):
            assert k in line, k
        assert line["impl"] == "reference" and line["value"] > 0
        assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
        assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
        assert line["config"].get("r_bond") == want_rb
