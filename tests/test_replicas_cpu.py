"""Multi-GPU form of the benchmark: replicas only (vehicles are independent,
the path has no exchange step).  The host logic — per-rank problem
(distinct Philox stream, same workload), max-over-ranks timing and the
whole-job rate — runs here as world-size-2 gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fleet = bench.Fleet(4, stream_base=rank * bench.N_FLEET)
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
    mx = bench.barrier_max(local_ms, world)
    bench.barrier(world)
    rate = bench.whole_job_rate(fleet.rollout_steps, 4, mx, world)
    sids = {int(p["params"]["stream_id"]) for p in fleet.probs}
    out.put((rank, mx, rate, min(sids), max(sids), fleet.rollout_steps, float(np.sum(fleet.obs))))
    dist.destroy_process_group()


def test_replicas_reduce_max_and_whole_job_rate():
    import torch.multiprocessing as mp
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
    (r0, mx0, rate0, lo0, hi0, st0, obs0), (r1, mx1, rate1, lo1, hi1, st1, obs1) = res
    assert mx0 == mx1 == 15.0  # the slowest rank's time on every rank
    assert st0 == st1 and rate0 == rate1 == pytest.approx(2 * st0 * 4 / 15e-3)
    assert hi0 < lo1  # independent noise streams per replica and vehicle
    assert obs0 == obs1  # same workload on every replica


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    """`bench.py --impl reference` launched like the multi-GPU bench (two
    ranks): rank 0 alone times the oracle and prints the one JSON line, the
    other rank exits 0 without work; no GPU is touched."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "3", "--ref-seconds", "3"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
