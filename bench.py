"""Benchmark of the VIPER per-substep rod solve on GB300.

A step is one frame of the muscle-rig workload: kinematic bones animated
towards the frame's pose, 10 substeps x 4 iterations of prediction, constraint
projection, pill-pill contacts and velocity update, then linear blend skinning
of the 200k-vertex mesh.  Reported metric: rod-vertex substeps per second
(vertices x substeps / frame time), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: W untimed frames; then K frames each bracketed by CUDA events on the
scene stream, with a 256 MB buffer written between frames (outside the events)
so that every frame starts with a cold L2; barrier + synchronize around the
timed region; max over ranks.  Under torchrun every rank steps its own
independent seeded scene (weak scaling; no data-path collective).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_DESC = ("muscle_rig: 200 tapered rods of 8-64 vertices pinned to 20 animated bones, "
                 "pill-pill contacts, volume on, dt=1/60 s, 10 substeps x 4 iterations, "
                 "LBS of a 200k-vertex mesh (4 weights)")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs: the
    sampler is started (and has printed its first line) before the region, and
    only the lines that arrive between begin() and end() are kept."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.monotonic() + 5.0
            while not self.lines and time.monotonic() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def begin(self):
        self.t0 = time.monotonic()

    def end(self):
        self.t1 = time.monotonic()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        t0 = self.t0 if self.t0 is not None else 0.0
        t1 = self.t1 if self.t1 is not None else float("inf")
        lines = [ln for t, ln in self.lines if t0 <= t <= t1]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window_s": (t1 - t0) if self.t1 is not None and self.t0 is not None else None}


def dist_setup():
    """Process group of a torchrun launch (RANK / WORLD_SIZE / LOCAL_RANK / MASTER_*
    from the environment): NCCL with GPUs, gloo without.  Ranks are independent
    replicas; the group carries only the barrier and the timing reductions."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        return dist, rank, ws, local
    return None, 0, 1, 0


def barrier(dist):
    if dist is not None:
        dist.barrier()


def _reduce(dist, x, op):
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=op)
    return float(t.item())


def reduce_max(dist, x):
    return _reduce(dist, x, dist.ReduceOp.MAX) if dist is not None else x


def reduce_sum(dist, x):
    return _reduce(dist, x, dist.ReduceOp.SUM) if dist is not None else x


def whole_job(dist, units, ms):
    """Whole-job throughput of a weak-scaling step: the units of all ranks over the
    slowest rank's time per step.  Returns (units per second, max ms per step)."""
    ms_max = reduce_max(dist, ms)
    return reduce_sum(dist, units) / (ms_max * 1e-3), ms_max


# ---------------------------------------------------------------------------- oracle arm

def oracle_run(scene, frames: int, skin: bool = True):
    """Step the FP64 oracle `frames` frames (plus LBS); returns seconds."""
    import oracle
    o = oracle.OracleScene(scene)
    t0 = time.perf_counter()
    for _ in range(frames):
        o.frame()
        if skin and scene.mesh is not None:
            o.skin()
    return time.perf_counter() - t0


def cpu_baseline(scene, budget_s: float = 20.0):
    """The oracle on this host's cores (single-threaded), on a bounded sample."""
    t1 = oracle_run(scene, 1)
    frames = max(1, min(10, int(budget_s / max(t1, 1e-3))))
    t = oracle_run(scene, frames)
    val = scene.nv * scene.substeps * frames / t
    return {"value": val, "unit": "rod-vertex substeps/s", "cores": 1, "kind": "oracle",
            "sample": f"{frames} frame(s) of the same muscle_rig scene incl. LBS of {scene.mesh.n} vertices, "
                      f"FP64, single thread, {os.cpu_count()} host cores present"}


def run_reference(args):
    from paper_1906_05260_gb300 import scenes as S
    # the oracle runs on rank 0's host cores alone; the other ranks exit without work
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    import oracle
    oracle.build()
    sc = S.muscle_rig(seed=1)
    # bound the whole run to a few minutes: each step is one oracle frame of a
    # rod sample of the workload if full frames would not fit
    t1 = oracle_run(sc, 1)
    budget = 150.0
    per_step_budget = budget / max(1, args.steps + args.warmup)
    sample_desc = "full frame"
    if t1 > per_step_budget:
        frac = max(0.02, per_step_budget / t1)
        n_rods = max(4, int(sc.n_rods * frac))
        sc = S.muscle_rig(seed=1, n_rods=n_rods, mesh_verts=max(1000, int(sc.mesh.n * frac)))
        sample_desc = f"{n_rods} of 200 rods and a {sc.mesh.n}-vertex mesh per frame"
    import oracle as O
    o = O.OracleScene(sc)
    for _ in range(args.warmup):
        o.frame()
        o.skin()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.frame()
        o.skin()
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    val = sc.nv * sc.substeps / mean
    line = {
        "impl": "reference", "metric": "rod-vertex substeps/sec", "value": val, "unit": "rod-vertex substeps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "sample": sample_desc},
        "cpu_baseline": {"value": val, "unit": "rod-vertex substeps/s", "cores": 1, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": val, "unit": "rod-vertex substeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------- our arm

def bench_batching(V, torch, flush, dist, peaks, peak_kind, fp32_peak_tflops, frames):
    """4096 independent rods (log-uniform 4..256 vertices), 20 substeps x 8 iterations."""
    from paper_1906_05260_gb300 import scenes as S
    sc = S.batching()
    out = {"workload": "batching: 4096 rods, log-uniform 4-256 vertices (250,612 total), "
                       "random initial bends, 20 substeps x 8 iterations, no contacts"}
    units = sc.nv * sc.substeps
    for mode, name in ((V.SOLVER_FRAME, "frame"), (V.SOLVER_BATCHED, "batched"), (V.SOLVER_PLAIN, "plain")):
        g = V.Scene(sc, solver=mode, resident_max=256)
        st = g.stream
        for _ in range(3):
            g.step()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ts = []
        for i in range(frames):
            with torch.cuda.stream(st):
                flush.fill_(i & 0xFF)
                e0.record(st)
                g.step()
                e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = reduce_max(dist, sum(ts) / len(ts))
        out[name] = {"value": reduce_sum(dist, units) / (ms * 1e-3), "unit": "rod-vertex substeps/s",
                     "ms_per_frame": ms, "p50_ms": float(np.percentile(ts, 50)),
                     "p99_ms": float(np.percentile(ts, 99))}
        if mode in (V.SOLVER_BATCHED, V.SOLVER_FRAME):
            g.profile(V.PROF_ROD)
            g.step()
            g.profile_read()
            tot, nl = 0.0, 0
            for i in range(min(frames, 10)):
                with torch.cuda.stream(st):
                    flush.fill_(i & 0xFF)
                g.step()
                ms_k, n = g.profile_read()
                tot += ms_k
                nl += n
            us = 1e3 * tot / max(nl, 1)
            per_launch = sc.substeps if mode == V.SOLVER_FRAME else 1  # substeps per launch
            flops = sc.nv * sc.iterations * 1030.0 * per_launch
            bytes_ = sc.nv * 140.0 * (1 if mode == V.SOLVER_FRAME else 1)  # state in/out + rest once per launch
            out["rod_kernel" if mode == V.SOLVER_BATCHED else "frame_kernel"] = {
                "us_per_launch": us, "launches_per_frame": nl / min(frames, 10),
                "alu": {"achieved": flops / (us * 1e-6) / 1e12, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                        "frac": flops / (us * 1e-6) / 1e12 / fp32_peak_tflops},
                "hbm": {"achieved": bytes_ / (us * 1e-6) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": bytes_ / (us * 1e-6) / 1e9 / peaks["hbm_gbs"], "peak_kind": peak_kind},
            }
            g.profile(V.PROF_NONE)
        g.close()
    out["batched_over_plain"] = out["batched"]["value"] / out["plain"]["value"]
    out["frame_over_plain"] = out["frame"]["value"] / out["plain"]["value"]
    # the same workload with the paper's Jacobi ordering, and with surface bending
    import dataclasses
    for key, variant in (("jacobi", dict(jacobi=True)), ("surface_bending", dict(surface_bending=True))):
        g = V.Scene(dataclasses.replace(sc, **variant), resident_max=256)
        st = g.stream
        for _ in range(3):
            g.step()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ts = []
        for i in range(frames):
            with torch.cuda.stream(st):
                flush.fill_(i & 0xFF)
                e0.record(st)
                g.step()
                e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        if g.sync() != 0:
            raise SystemExit(f"{key} variant failed")
        ms = reduce_max(dist, sum(ts) / len(ts))
        out[key] = {"value": reduce_sum(dist, units) / (ms * 1e-3), "unit": "rod-vertex substeps/s",
                    "ms_per_frame": ms, "over_colours": out["batched"]["ms_per_frame"] / ms}
        g.close()
    return out


def bench_convergence(V, np_):
    """E9 (the paper's convergence test): a 12-vertex rod whose end bars are
    pulled to twice its length at once; distance of the state after N
    iterations (one substep) to the ordering's own limit, on the GPU."""
    import dataclasses
    from paper_1906_05260_gb300 import scenes as S
    n = 12
    off = np_.array([0, n], np_.int32)
    pos = np_.zeros((n, 3))
    pos[:, 0] = np_.arange(n) * 0.01
    q = np_.tile(S.quat_from_z(np_.array([1.0, 0, 0])), (n - 1, 1))
    sc = S.Scene(name="e9", rod_offsets=off, rest_pos=pos, rest_quat=q, radius=np_.full(n, 0.01),
                 density=np_.array([1000.0]), c_stretch=np_.array([1e-9]), c_bend=np_.array([1e-7]),
                 c_volume=np_.array([1e-9]), group=np_.zeros(1, np_.int32), gravity=np_.zeros(3),
                 pin_vertex=np_.array([0, n - 1], np_.int32), pin_bone=np_.array([-1, -1], np_.int32),
                 pin_offset=np_.array([[0, 0, 0], [2.0 * 0.01 * (n - 1), 0, 0]]), bones=None,
                 planes=np_.zeros((0, 4)), contact_compliance=1e-9, contacts=False, volume=True,
                 dt=1 / 60, substeps=1, iterations=1, frames=1)

    def run(jacobi, iters):
        g = V.Scene(dataclasses.replace(sc, jacobi=jacobi))
        g.step(sc.dt, 1, iters)
        x = g.get_state()["x4"][:, :3].astype(np_.float64)
        g.close()
        return x

    out = {"workload": "E9: 12-vertex rod, bars pulled to 2x rest length at once, one substep of N iterations",
           "metric": "max |x_N - x_limit| (m), limit = 4096 iterations (colours) / 16384 (Jacobi)"}
    for jacobi, limit_iters, key in ((False, 4096, "colours"), (True, 16384, "jacobi")):
        lim = run(jacobi, limit_iters)
        out[key] = {str(it): float(np_.abs(run(jacobi, it) - lim).max()) for it in (1, 4, 16, 64, 256)}
    return out


def bench_multi_scene(V, torch, flush, dist, frames, n_scenes=64, rank=0):
    """n serving-size muscle rigs advanced together by the multi-scene step, against
    the same scenes stepped one after another (graph-replayed, per scene)."""
    from paper_1906_05260_gb300 import serving as SV
    temps = SV.scene_templates(seed=4 + rank)
    objs = [V.Scene(temps[k % len(temps)]) for k in range(n_scenes)]
    meshes = [V.Mesh(o.scene.mesh) for o in objs]
    sc0 = objs[0].scene
    nv = sum(o.nv for o in objs)
    nm = sum(m.n for m in meshes)
    units = reduce_sum(dist, nv * sc0.substeps)
    Bt = V.Batch()
    st = Bt.stream
    poses = [[o.scene.bone_pose((f + 1) * sc0.dt) for o in objs] for f in range(frames + 3)]
    for f in range(3):
        Bt.step(objs, poses[f], meshes, sc0.dt, sc0.substeps, sc0.iterations)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ts = []
    l0 = Bt.launch_count()
    for i in range(frames):
        with torch.cuda.stream(st):
            flush.fill_(i & 0xFF)
            e0.record(st)
            Bt.step(objs, poses[3 + i], meshes, sc0.dt, sc0.substeps, sc0.iterations)
            e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    launches = (Bt.launch_count() - l0) / frames
    ms = reduce_max(dist, sum(ts) / len(ts))
    out = {"workload": f"{n_scenes} muscle rigs of 50-500 rods (templates of the serving mix), "
                       f"{nv} rod vertices and {nm} mesh vertices in all, 10 substeps x 4 iterations + LBS",
           "batched": {"value": units / (ms * 1e-3), "unit": "rod-vertex substeps/s", "ms_per_frame": ms,
                       "skinned_vertices_per_s": reduce_sum(dist, nm) / (ms * 1e-3),
                       "launches_per_frame": launches,
                       "solver": "multi-scene step: one launch sequence for all scenes"}}
    # the same scenes, one graph-replayed frame each, serially on one stream
    for o in objs:
        o.close()
    one = torch.cuda.Stream()
    objs = [V.Scene(temps[k % len(temps)], stream=one) for k in range(n_scenes)]
    for f in range(2):
        for o, m in zip(objs, meshes):
            o.frame()
            o.skin(m)
    torch.cuda.synchronize()
    tp = []
    for i in range(max(3, frames // 4)):
        with torch.cuda.stream(one):
            flush.fill_(i & 0xFF)
            e0.record(one)
            for o, m in zip(objs, meshes):
                o.frame()
                o.skin(m)
            e1.record(one)
        e1.synchronize()
        tp.append(e0.elapsed_time(e1))
    pm = reduce_max(dist, sum(tp) / len(tp))
    out["per_scene_graphs"] = {"value": units / (pm * 1e-3), "unit": "rod-vertex substeps/s", "ms_per_frame": pm,
                               "solver": "each scene's frame graph replayed in turn on one stream"}
    out["batched_over_per_scene"] = out["batched"]["value"] / out["per_scene_graphs"]["value"]
    for o in objs:
        o.close()
    return out


def time_scene(V, torch, flush, dist, sc, frames, per_frame=None, solver=None):
    """Frame time of one scene (bones set per frame, LBS when it has a mesh):
    device time between CUDA events on its stream, L2 flushed between frames,
    and the host wall clock of the same frames."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    g = V.Scene(sc) if solver is None else V.Scene(sc, solver=solver)
    mesh = V.Mesh(sc.mesh) if sc.mesh is not None else None
    st = g.stream

    def one(f):
        if per_frame is not None:
            per_frame(g, f)
        g.frame()
        if mesh is not None:
            g.skin(mesh)

    for f in range(3):
        one(f)
    torch.cuda.synchronize()
    ts, tw = [], []
    l0 = g.launch_count()
    for i in range(frames):
        with torch.cuda.stream(st):
            flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(st):
            e0.record(st)
            one(3 + i)
            e1.record(st)
        e1.synchronize()
        tw.append((time.perf_counter() - t0) * 1e3)
        ts.append(e0.elapsed_time(e1))
    rc = g.sync()
    if rc != 0:
        raise SystemExit(f"solver error {rc}: {V.error_string(rc)}")
    ms = reduce_max(dist, sum(ts) / len(ts))
    wall = reduce_max(dist, sum(tw) / len(tw))
    units = reduce_sum(dist, sc.nv * sc.substeps)
    out = {"value": units / (ms * 1e-3), "unit": "rod-vertex substeps/s", "ms_per_frame": ms,
           "wall_ms_per_frame": wall, "launches_per_frame": (g.launch_count() - l0) / frames}
    g.close()
    return out


def bench_lbs(V, torch, flush, dist, frames, peaks, peak_kind, rank=0):
    """Skinning alone on a large mesh (the HBM-streaming stage): 8M mesh vertices
    bound to the headline rig's 7,110-segment frames; algorithmic bytes 64 per
    vertex (rest position, frame ids, weights in; skinned position out)."""
    from paper_1906_05260_gb300 import scenes as S
    sc = S.muscle_rig(seed=1 + rank, mesh_verts=8_000_000)
    g = V.Scene(sc)
    mesh = V.Mesh(sc.mesh)
    st = g.stream
    g.frame()
    g.skin(mesh)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ts = []
    for i in range(frames):
        with torch.cuda.stream(st):
            flush.fill_(i & 0xFF)
            e0.record(st)
            g.skin(mesh)
            e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = reduce_max(dist, float(np.median(ts)))
    n = sc.mesh.n
    gbs = n * 64.0 / (ms * 1e-3) / 1e9
    g.close()
    return {"workload": f"LBS of {n} mesh vertices (4 frames each, random order) on the muscle_rig's "
                        f"{sc.ns} segment frames; frames rebuilt and gathered every call",
            "ms_per_call": ms, "skinned_vertices_per_s": reduce_sum(dist, n) / (ms * 1e-3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / peaks["hbm_gbs"], "peak_kind": f"{peak_kind} HBM copy bandwidth",
                         "bytes_per_vertex": 64}}


def bench_muscles(V, torch, flush, dist, frames, rank=0):
    """Muscle features on the headline rig and on bundled muscles (Sec. 7.3, 8.2):
    per-frame time with a time-varying activation (rest tables recomputed on the
    host and uploaded every frame, inside the timed region) and the bone-driven
    warm start, against the same rig without them; bundled fibre muscles with
    shape matching after every substep."""
    from paper_1906_05260_gb300 import scenes as S
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed_scene(sc, per_frame=None, solver=None):
        return time_scene(V, torch, flush, dist, sc, frames, per_frame, solver)

    base = S.muscle_rig(seed=1 + rank)
    warm = dataclasses.replace(base, warm_start=True)
    phase = np.random.default_rng(7).uniform(0, 2 * math.pi, base.n_rods)

    # the activation of every frame: inputs, generated before timing
    acts = [(0.3 * (0.5 + 0.5 * np.sin(2 * math.pi * f / 60.0 + phase))).astype(np.float32)
            for f in range(frames + 3)]

    def activate(g, f):
        g.set_activation(acts[f])

    res = {"workload": f"muscle_rig {base.n_rods} rods / {base.nv} vertices, {base.mesh.n} mesh vertices, "
                       "10 substeps x 4 iterations + LBS",
           "plain_rig": timed_scene(base),
           "activation_and_warm_start": timed_scene(warm, activate)}
    # the activation update alone: upload + device recompute of the rest tables
    g = V.Scene(warm)
    st = g.stream
    for f in range(3):
        activate(g, f)
    torch.cuda.synchronize()
    ta = []
    for i in range(frames):
        with torch.cuda.stream(st):
            e0.record(st)
            activate(g, i)
            e1.record(st)
        e1.synchronize()
        ta.append(e0.elapsed_time(e1))
    g.close()
    res["set_activation_us"] = 1e3 * reduce_max(dist, sum(ta) / len(ta))
    res["activation_and_warm_start"]["note"] = ("per-rod activation 0.3 (1 + sin) / 2 set every frame: the rods "
                                                "thicken and shorten, so contacts and pairs change too; "
                                                "(n_rods floats uploaded, rest tables recomputed on the device), warm start from the bones")
    bm = S.bundled_muscles(n_muscles=96)
    res["bundled_muscles"] = timed_scene(bm)
    # the printed vector volume form (plain solver only) against the scalar form on the plain solver
    res["volume_forms_plain_solver"] = {
        "scalar": timed_scene(base, solver=V.SOLVER_PLAIN),
        "vector": timed_scene(dataclasses.replace(base, volume_vector=True), solver=V.SOLVER_PLAIN)}
    res["bundled_muscles"]["workload"] = (f"{bm.n_rods // 7} muscles x 7 fibre rods x 16 vertices "
                                          f"({bm.nv} vertices), shape matching of every cross-section per substep, "
                                          "contacts between muscles, 10 substeps x 4 iterations")
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-multi", action="store_true")
    ap.add_argument("--no-muscles", action="store_true")
    ap.add_argument("--no-lbs", action="store_true")
    ap.add_argument("--serving", type=float, default=10.0,
                    help="seconds of the real-time serving load (0 disables)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_1906_05260_gb300 import build as B
    B.build()
    from paper_1906_05260_gb300 import scenes as S
    from paper_1906_05260_gb300 import viper as V

    dist, rank, ws, local = dist_setup()
    torch.cuda.set_device(local)
    sc = S.muscle_rig(seed=1 + rank)
    g = V.Scene(sc)
    mesh = V.Mesh(sc.mesh)
    stream = g.stream
    nb = sc.bones.n
    K, W = args.steps, args.warmup
    sec_frames = max(10, min(K, 60) // 2)  # frames per timed section beside the main line

    # per-frame bone poses: the inputs, generated before timing
    total_frames = 10 * (W + K) + 400
    poses_q = np.zeros((total_frames, nb, 4), np.float32)
    poses_t = np.zeros((total_frames, nb, 3), np.float32)
    for f in range(total_frames):
        q, t = sc.bone_pose((f + 1) * sc.dt)
        poses_q[f], poses_t[f] = q, t
    dev_q = torch.from_numpy(poses_q).cuda()
    dev_t = torch.from_numpy(poses_t).cuda()
    pin_q = torch.from_numpy(poses_q).pin_memory()
    pin_t = torch.from_numpy(poses_t).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    frame_no = [0]

    def device_frame():
        f = frame_no[0]
        frame_no[0] += 1
        g.set_bones(dev_q[f], dev_t[f])
        g.step()
        g.skin(mesh)

    def timed(nframes, fn):
        ts = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for i in range(nframes):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
                e0.record(stream)
                fn()
                e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts

    # ---- batched (graph) path: warmup + timed region
    for _ in range(W):
        device_frame()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    l0 = g.launch_count()
    clocks.begin()
    ts = timed(K, device_frame)
    torch.cuda.synchronize()
    clocks.end()
    barrier(dist)
    launches = g.launch_count() - l0
    clk = clocks.stop()
    rc = g.sync()
    if rc != 0:
        raise SystemExit(f"solver error {rc}: {V.error_string(rc)}")
    mean_ms = sum(ts) / len(ts)
    value, mean_ms_max = whole_job(dist, sc.nv * sc.substeps, mean_ms)
    units = reduce_sum(dist, sc.nv * sc.substeps)
    p50 = float(np.percentile(ts, 50))
    p99 = float(np.percentile(ts, 99))

    # ---- end to end through the public API with host buffers
    out_host = torch.empty((sc.mesh.n, 4), dtype=torch.float32).pin_memory()
    rest4 = np.zeros((sc.mesh.n, 4), np.float32)
    rest4[:, :3] = sc.mesh.rest
    idx4 = np.ascontiguousarray(sc.mesh.idx, np.int32)
    w4 = np.ascontiguousarray(sc.mesh.w, np.float32)
    rest_pin = torch.from_numpy(rest4).pin_memory()
    idx_pin = torch.from_numpy(idx4).pin_memory()
    w_pin = torch.from_numpy(w4).pin_memory()
    import ctypes as C

    def host_frame():
        f = frame_no[0]
        frame_no[0] += 1
        rcb = V.lib().viper_set_bones(g.handle, nb, C.c_void_p(pin_q[f].data_ptr()), C.c_void_p(pin_t[f].data_ptr()))
        rcs = V.lib().viper_step(g.handle, float(sc.dt), sc.substeps, sc.iterations)
        rck = V.lib().viper_skin(g.handle, sc.mesh.n, C.c_void_p(rest_pin.data_ptr()), C.c_void_p(idx_pin.data_ptr()),
                                 C.c_void_p(w_pin.data_ptr()), C.c_void_p(out_host.data_ptr()))
        if rcb or rcs or rck:
            raise SystemExit(f"e2e frame failed: {rcb} {rcs} {rck}")

    for _ in range(3):
        host_frame()
    torch.cuda.synchronize()
    barrier(dist)
    te = []
    for i in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_frame()
        te.append((time.perf_counter() - t0) * 1e3)
    barrier(dist)
    e2e_ms = reduce_max(dist, sum(te) / len(te))
    e2e = {"value": units / (e2e_ms * 1e-3), "unit": "rod-vertex substeps/s",
           "h2d_bytes_per_step": int(nb * (16 + 12) + sc.mesh.n * 48),
           "d2h_bytes_per_step": int(sc.mesh.n * 16), "ms_per_step": e2e_ms,
           "note": "host pinned bone poses and mesh operands in, skinned mesh out, wall clock per frame"}

    # ---- per-kernel-class device time (events around each launch inside the graph)
    classes = {"rod": V.PROF_ROD, "contact": V.PROF_CONTACT, "broadphase": V.PROF_BROADPHASE,
               "pairs": V.PROF_PAIRS, "lbs_gather": V.PROF_LBS, "elementwise": V.PROF_ELEMENTWISE}
    per_class = {}
    prof_frames = min(K, 20)
    for name, cls in classes.items():
        g.profile(cls)
        device_frame()
        g.profile_read()
        tot = 0.0
        nl = 0
        for i in range(prof_frames):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
            device_frame()
            ms, n = g.profile_read()
            tot += ms
            nl += n
        if nl == 0:
            continue  # class not launched by this solver (the frame kernel fuses it)
        per_class[name] = {"ms_per_frame": tot / prof_frames, "launches_per_frame": nl / prof_frames,
                           "us_per_launch": 1e3 * tot / max(nl, 1)}
    g.profile(V.PROF_NONE)
    dominant = max(per_class, key=lambda k: per_class[k]["ms_per_frame"])

    peaks, peak_kind = load_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    # FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x max clock
    fp32_peak_tflops = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    nv, ns = sc.nv, sc.ns
    d = per_class[dominant]
    # algorithmic work per launch of each class: 1030 FP32 flop per vertex per colour
    # sweep, 1500 per candidate pair per contact pass, 64 B per skinned vertex, and for
    # the broadphase about 60 B per pill plus 8 B per emitted pair
    pairs_last = g.pairs().shape[0]
    if dominant == "rod" and g.solver == V.SOLVER_FRAME:
        # the whole frame: colour sweeps (1030 flop per vertex per sweep) + contact passes
        # (1500 flop per candidate pair per pass, pair count of the frame's last substep)
        flops = sc.substeps * sc.iterations * (nv * 1030.0 + pairs_last * 1500.0)
        roof = {"bound": "alu", "achieved": flops / (d["us_per_launch"] * 1e-6) / 1e12, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "peak_kind": f"FP32 SIMT 152x128x2x{sm_max:.0f} MHz ({peak_kind} clock)",
                "kernel_name": "frame_kernel<true,true>", "pairs": pairs_last}
    elif dominant == "rod":
        flops = nv * 1030.0  # FP32 flop per vertex per colour sweep (segment + vertex constraints)
        roof = {"bound": "alu", "achieved": flops / (d["us_per_launch"] * 1e-6) / 1e12, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "peak_kind": f"FP32 SIMT 152x128x2x{sm_max:.0f} MHz ({peak_kind} clock)"}
    elif dominant == "lbs_gather":
        bytes_ = sc.mesh.n * 64.0
        roof = {"bound": "hbm", "achieved": bytes_ / (d["us_per_launch"] * 1e-6) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "peak_kind": f"{peak_kind} HBM copy bandwidth"}
    else:
        pairs = g.pairs().shape[0]
        if dominant == "contact":
            flops = pairs * 1500.0
            roof = {"bound": "alu", "achieved": flops / (d["us_per_launch"] * 1e-6) / 1e12,
                    "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                    "peak_kind": f"FP32 SIMT 152x128x2x{sm_max:.0f} MHz ({peak_kind} clock)", "pairs": pairs}
        else:
            bytes_ = (ns * 60.0 + pairs * 8.0) / max(d["launches_per_frame"] / sc.substeps, 1)
            roof = {"bound": "hbm", "achieved": bytes_ / (d["us_per_launch"] * 1e-6) / 1e9,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "peak_kind": f"{peak_kind} HBM copy bandwidth",
                    "pairs": pairs}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = dominant
    # DRAM bytes per launch of the dominant class from one ncu capture of this workload
    # (first sweep 0.716 MB, later sweeps 1.092 MB, one and three per substep; the
    # velocity update and prediction run in the advance kernel before them); other
    # classes or solvers: not captured
    roof["traffic"] = (0.716e6 + 3 * 1.092e6) / 4 if (dominant == "rod" and g.solver == V.SOLVER_BATCHED) else None
    roof["traffic_unit"] = "bytes per launch (dram read + write, ncu)"
    roof["per_class"] = per_class

    # ---- the other solvers on the same scene: graph-replayed launches and plain per-colour launches
    main_solver = g.solver
    plain = None
    graph = None
    if not args.no_plain:
        for mode, label in ((V.SOLVER_BATCHED, "batched: one shared-memory rod launch per iteration, broadphase and "
                                               "contact launches, frame replayed as a CUDA graph"),
                            (V.SOLVER_PLAIN, "plain: one launch per constraint colour")):
            if mode == main_solver:
                continue
            g.set_solver(mode)
            for _ in range(3):
                device_frame()
            tp = timed(sec_frames, device_frame)
            pm = reduce_max(dist, sum(tp) / len(tp))
            res = {"value": units / (pm * 1e-3), "ms_per_step": pm, "p50_ms": float(np.percentile(tp, 50)),
                   "p99_ms": float(np.percentile(tp, 99)), "solver": label}
            if mode == V.SOLVER_PLAIN:
                plain = res
            else:
                graph = res
        g.set_solver(main_solver)

    # ---- batching workload (4096 rods, 20 x 8, no contacts): batched vs plain and
    # the shared-memory rod kernel's roofline
    batching = None
    convergence = None
    if not args.no_batching:
        batching = bench_batching(V, torch, flush, dist, peaks, peak_kind, fp32_peak_tflops, sec_frames)
        convergence = bench_convergence(V, np)

    # ---- skinning alone on a large mesh: the HBM-streaming stage's roofline
    lbs = None
    if not args.no_lbs:
        lbs = bench_lbs(V, torch, flush, dist, sec_frames, peaks, peak_kind, rank=rank)

    # ---- muscle features: activation + warm start, bundled muscles
    muscles = None
    if not args.no_muscles:
        muscles = bench_muscles(V, torch, flush, dist, sec_frames, rank=rank)

    # ---- many scenes at once: the multi-scene step against per-scene graphs
    multi = None
    if not args.no_multi:
        g.close()
        multi = bench_multi_scene(V, torch, flush, dist, sec_frames, rank=rank)

    # ---- serving: Poisson stream of muscle-rig scenes, 60 Hz frame requests each
    serving = None
    if args.serving > 0:
        from paper_1906_05260_gb300 import serving as SV
        g.close()
        temps = SV.scene_templates(seed=4 + rank)
        conc = SV.run_load(duration=args.serving, rate=6.4, mean_life=10.0, budget=150 << 30, max_inflight=256,
                           seed=4 + rank, templates=temps, warm_scenes=64)
        ser = SV.run_load(duration=max(3.0, args.serving / 2), rate=6.4, mean_life=10.0, budget=150 << 30,
                          max_inflight=1, seed=4 + rank, templates=temps, warm_scenes=64)
        serving = {
            "workload": "Poisson arrivals 6.4/s, lifetimes Exp(10 s), 64 scenes live at start (mean 64 "
                        "concurrent); muscle rigs of log-uniform 50-500 rods and 10k-300k mesh vertices; "
                        "60 Hz frame requests per scene, dt=1/60 s, 10 substeps x 4 iterations + LBS; "
                        "HBM budget 150 GB",
            "continuous_batching": conc, "serial_per_scene": ser,
            "throughput_over_serial": conc["rod_vertex_substeps_per_s"] / max(ser["rod_vertex_substeps_per_s"], 1e-9),
        }

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cpu = cpu_baseline(sc)

    line = {
        "metric": "rod-vertex substeps/sec", "value": value, "unit": "rod-vertex substeps/s", "n_gpus": ws,
        "steps": K, "warmup": W, "ms_per_step": mean_ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "rods": sc.n_rods, "vertices": sc.nv, "mesh_vertices": sc.mesh.n,
                   "solver": ("frame: one persistent cooperative launch per frame, rods resident in shared memory, "
                              "grid barriers between broadphase / sweep / contact phases")
                             if main_solver == V.SOLVER_FRAME else
                             "batched: shared-memory rod kernel, frame replayed as a CUDA graph",
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "parallelism": f"replicas x{ws} (independent seeded scenes)"},
        "latency_ms": {"p50": p50, "p99": p99},
        "skinned_vertices_per_s": reduce_sum(dist, sc.mesh.n) / (mean_ms_max * 1e-3),
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
        "plain": plain,
        "graph_batched": graph,
        "batching": batching,
        "convergence": convergence,
        "multi_scene": multi,
        "muscles": muscles,
        "lbs": lbs,
        "serving": serving,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
