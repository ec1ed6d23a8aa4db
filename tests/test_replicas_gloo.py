"""The N > 1 path of bench.py on CPU, world size 2 over gloo.

The hot path has no data exchange between ranks: each rank runs its own
geometry (replicas), and the only collectives are the timing ones -- a barrier
around the timed steps and the maximum of the ranks' elapsed times, which sets
the whole-job throughput.  These tests run that host logic as real processes
(spawned, rendezvous on 127.0.0.1), and the reference arm under torchrun, where
rank 0 alone works and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_setup()
    bench.barrier(pg)
    ms = 10.0 * (r + 1)                     # rank 1 is the slower replica
    ms_max = bench.allreduce_max(pg, ms, local)
    bench.barrier(pg)
    steps = 5
    q.put((r, w, ms_max, w * steps / (ms_max / 1e3)))
    pg.destroy_process_group()


def test_timing_collectives_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(60)
    assert all(p.exitcode == 0 for p in procs)
    # both ranks see the slower rank's time; throughput = all ranks' steps / that time
    assert [(r, w, m) for r, w, m, _ in res] == [(0, 2, 20.0), (1, 2, 20.0)]
    assert res[0][3] == pytest.approx(2 * 5 / 0.020)


def _json_lines(text):
    return [json.loads(line) for line in text.splitlines() if line.startswith("{")]


def test_reference_arm_single_process():
    import bench
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "0", "--ref-molecule", "monomer"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # whole steps were timed and the line says how many; its time per step and
    # that count fit the run's own wall clock
    assert d["steps_timed"] >= 1 and d["steps_timed"] <= d["steps"]
    assert "whole steps timed" in d["cpu_baseline"]["sample"]


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-molecule", "monomer"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1                  # rank 0 alone runs the oracle and prints
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0
