"""The N > 1 launch path on CPU: world-size-2 gloo process groups on 127.0.0.1.

Ranks are independent replicas (one seeded scene each, weak scaling): the process
group only carries the barrier and the reductions of the timings.  These tests run
those host-side pieces of bench.py with two gloo ranks, and the reference arm under
torchrun with two ranks (rank 0 alone runs the oracle and prints one line).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from paper_1906_05260_gb300 import scenes as S
    dist, r, ws, local = bench.dist_setup()
    assert (r, ws, local) == (rank, 2, rank) and dist.get_backend() == "gloo"
    bench.barrier(dist)
    # each rank steps its own seeded scene: different inputs, fixed work per rank
    sc = S.muscle_rig(seed=1 + rank, n_rods=20, mesh_verts=0)
    units = sc.nv * sc.substeps
    ms = 1.0 + rank  # the slower rank sets the time
    value, ms_max = bench.whole_job(dist, units, ms)
    res = {"rank": r, "value": value, "ms_max": ms_max, "units": units, "units_all": bench.reduce_sum(dist, units),
           "max_rank": bench.reduce_max(dist, r)}
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    bench.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timings_and_units(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    assert res[0]["units_all"] == res[1]["units_all"] == res[0]["units"] + res[1]["units"]
    assert res[0]["units"] != res[1]["units"]  # each rank its own seeded scene
    assert res[0]["max_rank"] == res[1]["max_rank"] == 1
    assert res[0]["ms_max"] == res[1]["ms_max"] == 2.0
    assert res[0]["value"] == pytest.approx(res[0]["units_all"] / 2e-3)
    assert res[0]["value"] == res[1]["value"]


def test_reference_arm_under_torchrun_with_two_ranks():
    """`bench.py --impl reference` launched as the driver launches it for N = 2:
    rank 0 times the oracle and prints exactly one JSON line; rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_clock_sampler_keeps_only_the_timed_window():
    """bench.py's clock record: lines that arrive before begin() or after end()
    are dropped; the median SM clock, the maximum and the active throttle
    reasons come from the window alone."""
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    row = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"
    cs.lines = [(1.0, row.format(sm=1000, hw="Active", pc="Not Active")),    # before the window
                (2.1, row.format(sm=2000, hw="Not Active", pc="Active")),
                (2.2, row.format(sm=2070, hw="Not Active", pc="Not Active")),
                (2.3, row.format(sm=2060, hw="Not Active", pc="Not Active")),
                (3.5, row.format(sm=500, hw="Active", pc="Not Active"))]     # after it
    cs.t0, cs.t1 = 2.0, 3.0
    out = cs.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2060 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]
    assert out["window_s"] == pytest.approx(1.0)
