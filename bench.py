"""Benchmark of the VIPER per-substep rod solve on GB300.

A step is one frame of the contact-heavy hair workload, the largest
single-GPU configuration: 20,000 rods x 16 vertices falling from a sphere into
a box, 10 substeps x 4 iterations of prediction, constraint projection,
pill-pill contacts (grid broadphase, dichotomous narrowphase) with six
half-planes, and velocity update.  Reported metric: rod-vertex substeps per
second (vertices x substeps / frame time), whole job.  The muscle rig with
skinning, the batching workload, the multi-scene step and the serving loop
are measured as sections of the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: W untimed frames; then K frames each bracketed by CUDA events on the
scene stream, with a 256 MB buffer written between frames (outside the events)
so that every frame starts with a cold L2; barrier + synchronize around the
timed region; max over ranks.  Frames are those of the trajectory from the
start (frame W to W + K - 1).  Under torchrun every rank steps its own
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

WORKLOAD_DESC = ("hair: 20,000 rods x 16 vertices (320,000 vertices, 300,000 pills), radius 2 mm, 5 mm segments, "
                 "roots at Poisson-disk sites of a 0.2 m sphere falling into a 0.3 m box (six half-planes), "
                 "pill-pill contacts (uniform-grid broadphase, dichotomous narrowphase, compliance 1e-9), "
                 "volume on, dt=1/60 s, 10 substeps x 4 iterations")
MUSCLE_DESC = ("muscle_rig: 200 tapered rods of 8-64 vertices pinned to 20 animated bones, "
               "pill-pill contacts, volume on, dt=1/60 s, 10 substeps x 4 iterations, "
               "LBS of a 200k-vertex mesh (4 weights)")
HAIR_PAIRS_PER_PILL = 64  # pair-list capacity of the hair scene (peak use about 36 per pill)

# FP32 work per unit of the contact pass (ncu SASS counts of FADD + FMUL + 2 FFMA of one
# pass at frames 5, 18 and 55 of the hair scene, least-squares fit of the two figures,
# each state predicted within 1.5 %): the two-direction early-out test per candidate
# pair, and the dichotomous search + constraint update per searched pair
CONTACT_FLOP_PER_CANDIDATE = 77.5
CONTACT_FLOP_PER_SEARCHED = 892.5
# FP32 work of the shared-memory rod kernel per vertex per colour sweep (ncu SASS
# counts on the batching workload: 2.133 GFLOP per launch over 250,612 vertices x 8
# sweeps, prediction and velocity update included)
ROD_FLOP_PER_VERTEX_SWEEP = 1064.0


def hair_scene(rank=0):
    from paper_1906_05260_gb300 import scenes as S
    return S.hair(seed=3 + rank)


def hair_octant(sc):
    """The rods of the hair scene whose roots lie in the octant x, y, z > 0 of
    the sphere: a sample with the scene's own local density of strands and
    contacts (about an eighth of its rods; planes and material kept)."""
    import dataclasses as dc
    roots = sc.rest_pos[sc.rod_offsets[:-1]]
    keep = np.nonzero((roots > 0).all(axis=1))[0]
    sub = sc.subset(keep)
    return dc.replace(sub, name="hair_octant", group=np.arange(len(keep), dtype=np.int32))


def kernel_source_hash(unit="contact.cu"):
    """sha256 of one CUDA translation unit as the build compiles it: the file
    csrc/<unit>, every header of the repository it includes (#include "...",
    followed transitively, in the order met) and the nvcc flags.  A kernel's
    code is fixed by exactly these, so an ncu summary under profiles/ names the
    hash of the unit its kernels were captured from."""
    import hashlib
    import re
    from paper_1906_05260_gb300 import build as B
    d = os.path.join(ROOT, "paper_1906_05260_gb300", "csrc")
    h = hashlib.sha256()
    h.update(" ".join([*B.ARCH, *B.NVCC_FLAGS]).encode() + b"\0")
    seen, todo = set(), [os.path.join(d, unit)]
    while todo:
        path = os.path.normpath(todo.pop(0))
        if path in seen or not os.path.exists(path):
            continue
        seen.add(path)
        with open(path, "rb") as f:
            text = f.read()
        h.update(os.path.relpath(path, ROOT).encode() + b"\0" + text)
        for inc in re.findall(rb'#include "([^"]+)"', text):
            todo.append(os.path.join(os.path.dirname(path), inc.decode()))
    return h.hexdigest()


def profile_traffic(summary, key):
    """DRAM bytes per unit of one kernel from a committed ncu summary
    (profiles/<summary>): the line 'traffic <key>: <bytes> bytes per <unit>',
    used only while the summary's 'csrc sha256:' line matches this build's
    hash of the kernel's translation unit (contact.cu for the contact pass);
    else None (the kernel changed since the counters were taken)."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    sha, val = None, None
    with open(path) as f:
        for line in f:
            line = line.strip().strip("`")
            if line.startswith("csrc sha256:"):
                sha = line.split(":", 1)[1].strip()
            elif line.startswith(f"traffic {key}:"):
                try:
                    val = float(line.split(":", 1)[1].split()[0])
                except ValueError:
                    val = None
    return val if sha == kernel_source_hash() else None


def fp32_peak_tflops(sm_max_mhz):
    """FP32 SIMT peak: SMs (read from the device) x 128 FP32 lanes x 2 flop (FMA) x clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * 2 * sm_max_mhz * 1e6 / 1e12, sms


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

def oracle_substep_time(scene, threads=1):
    """Seconds of one substep of the FP64 oracle on `scene` from its initial state
    (h = dt / substeps, the scene's iterations), on `threads` host threads."""
    import oracle
    o = oracle.OracleScene(scene, threads=threads)
    t0 = time.perf_counter()
    rc = o.step(dt=scene.dt / scene.substeps, substeps=1, iterations=scene.iterations)
    t = time.perf_counter() - t0
    if rc != 0:
        raise SystemExit(f"oracle step failed: {rc}")
    return t


def cpu_baseline(scene):
    """The oracle on this host's cores on a bounded sample of the hair workload:
    one substep of the full scene from its initial state (2.19 M candidate pairs),
    single-threaded and with one thread per host core."""
    t1 = oracle_substep_time(scene, threads=1)
    cores = os.cpu_count() or 1
    tn = oracle_substep_time(scene, threads=cores)
    return {"value": scene.nv / t1, "unit": "rod-vertex substeps/s", "cores": 1, "kind": "oracle",
            "sample": f"one substep (h = dt/{scene.substeps}, {scene.iterations} iterations, contacts) of the full "
                      f"hair scene from its initial state, FP64, {t1:.1f} s on one thread",
            "threads": {"value": scene.nv / tn, "unit": "rod-vertex substeps/s", "cores": cores,
                        "kind": "oracle",
                        "sample": f"the same substep with OpenMP over the constraints of each colour and the "
                                  f"pairs of each contact pass, {tn:.2f} s on {cores} threads"}}


def run_at_frame(frames):
    """The hair scene after `frames` frames, then one substep with one iteration:
    a single pair search and a single contact pass at that state (for ncu:
    contact_kernel launch 40 x frames, bp_emit_kernel launch 10 x frames).
    Prints the pass's candidate, searched and active pair counts."""
    import torch
    from paper_1906_05260_gb300 import build as B
    B.build()
    from paper_1906_05260_gb300 import viper as V
    torch.cuda.set_device(0)
    sc = hair_scene(0)
    g = V.Scene(sc, max_pairs=HAIR_PAIRS_PER_PILL * sc.ns)
    for _ in range(frames):
        g.step()
    g.contact_stats()
    g.step(dt=sc.dt / sc.substeps, substeps=1, iterations=1)
    cand, searched, active = g.contact_stats()
    rc = g.sync()
    g.close()
    print(json.dumps({"at_frame": frames, "candidates": cand, "searched": searched, "active": active, "rc": rc}))
    return 0 if rc == 0 else 1


def run_reference(args):
    # the oracle runs on rank 0's host cores alone; the other ranks exit without work
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    import oracle
    oracle.build()
    sample = hair_octant(hair_scene(0))
    h = sample.dt / sample.substeps
    o = oracle.OracleScene(sample)
    for _ in range(args.warmup):
        o.step(dt=h, substeps=1, iterations=sample.iterations)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rc = o.step(dt=h, substeps=1, iterations=sample.iterations)
        times.append(time.perf_counter() - t0)
        if rc != 0:
            raise SystemExit(f"oracle step failed: {rc}")
    mean = sum(times) / len(times)
    val = sample.nv / mean
    desc = (f"one substep per step of the rods rooted in one octant of the hair scene ({sample.n_rods} rods, "
            f"{sample.nv} vertices, same local density), FP64, one thread")
    line = {
        "impl": "reference", "metric": "rod-vertex substeps/sec", "value": val, "unit": "rod-vertex substeps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "sample": desc},
        "cpu_baseline": {"value": val, "unit": "rod-vertex substeps/s", "cores": 1, "kind": "oracle", "sample": desc},
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
    # the batched solver's CTA size and residency threshold from the autotuner
    # (cached per GPU and scene under the package's build folder)
    g = V.Scene(sc)
    t0 = time.perf_counter()
    (bw, rm), cached = g.autotune_cached(os.path.join(ROOT, "paper_1906_05260_gb300", "_build", "autotune.json"))
    n_items, threads, resident = g.schedule()
    out["autotuned"] = {"block_warps": bw, "resident_max": rm, "threads_per_cta": threads, "ctas": n_items,
                        "rods_per_cta": sc.n_rods / max(n_items, 1), "resident_vertices": resident,
                        "cached": cached, "tune_s": time.perf_counter() - t0}
    g.close()
    for mode, name in ((V.SOLVER_FRAME, "frame"), (V.SOLVER_BATCHED, "batched"), (V.SOLVER_PLAIN, "plain")):
        g = (V.Scene(sc, solver=mode, block_warps=bw, resident_max=rm) if mode == V.SOLVER_BATCHED
             else V.Scene(sc, solver=mode, resident_max=256))
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
            flops = sc.nv * sc.iterations * ROD_FLOP_PER_VERTEX_SWEEP * per_launch
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


def events_timed(torch, stream, flush, nframes, fn):
    """Device time of each call of fn() between CUDA events on `stream`, L2
    flushed before each (outside the events); ms per call."""
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


HAIR_CLASSES = ("rod", "contact", "broadphase", "pairs", "elementwise")


def per_class_times(V, torch, g, stream, flush, frames, step):
    """Device time per frame of each kernel class (events around its launches
    inside the frame graph), over `frames` frames per class."""
    classes = {"rod": V.PROF_ROD, "contact": V.PROF_CONTACT, "broadphase": V.PROF_BROADPHASE,
               "pairs": V.PROF_PAIRS, "lbs_gather": V.PROF_LBS, "elementwise": V.PROF_ELEMENTWISE}
    out = {}
    for name, cls in classes.items():
        g.profile(cls)
        step()
        g.profile_read()
        tot, nl = 0.0, 0
        for i in range(frames):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
            step()
            ms, n = g.profile_read()
            tot += ms
            nl += n
        if nl:
            out[name] = {"ms_per_frame": tot / frames, "launches_per_frame": nl / frames,
                         "us_per_launch": 1e3 * tot / nl}
    g.profile(V.PROF_NONE)
    return out


def per_class_replay(V, torch, sc, cap, flush, W, K, classes=HAIR_CLASSES):
    """Kernel-class device times over the timed frames: a fresh scene replays
    the trajectory (W untimed frames, then frames W .. W+K-1), frame i timing
    class classes[i % n] (events around that class's launches in the frame
    graph).  The contact counters are read after every frame and kept for the
    frames that timed the contact pass, so that the contact pass's work and
    its time come from the same frames."""
    ids = {"rod": V.PROF_ROD, "contact": V.PROF_CONTACT, "broadphase": V.PROF_BROADPHASE,
           "pairs": V.PROF_PAIRS, "elementwise": V.PROF_ELEMENTWISE}
    g = V.Scene(sc, max_pairs=cap)
    for _ in range(W):
        g.step()
    g.contact_stats()
    tot = {c: 0.0 for c in classes}
    nl = {c: 0 for c in classes}
    nf = {c: 0 for c in classes}
    cstats = [0, 0, 0]
    for i in range(K):
        c = classes[i % len(classes)]
        g.profile(ids[c])
        with torch.cuda.stream(g.stream):
            flush.fill_(i & 0xFF)
        g.step()
        ms, n = g.profile_read()
        st = g.contact_stats()
        tot[c] += ms
        nl[c] += n
        nf[c] += 1
        if c == "contact":
            cstats = [a + b for a, b in zip(cstats, st)]
    g.profile(V.PROF_NONE)
    rc = g.sync()
    g.close()
    if rc != 0:
        raise SystemExit(f"per-class replay failed: {rc}")
    out = {c: {"ms_per_frame": tot[c] / nf[c], "launches_per_frame": nl[c] / nf[c],
               "us_per_launch": 1e3 * tot[c] / max(nl[c], 1), "frames": nf[c]} for c in classes if nf[c]}
    stats = {"candidates": cstats[0], "searched": cstats[1], "active": cstats[2],
             "passes": nf.get("contact", 0) * sc.substeps * sc.iterations}
    return out, stats


def contact_roofline(per_class, stats, sc, peak_tflops, peak_kind, sms, sm_max):
    """ALU roofline of the contact pass (contact_kernel, one launch per pass):
    FP32 work = candidates x the early-out test + searched pairs x (dichotomous
    search + update), per pass, over its event-timed duration."""
    d = per_class["contact"]
    passes = stats["passes"]
    cand = stats["candidates"] / passes
    searched = stats["searched"] / passes
    us_pass = 1e3 * d["ms_per_frame"] / (sc.substeps * sc.iterations)
    flops = cand * CONTACT_FLOP_PER_CANDIDATE + searched * CONTACT_FLOP_PER_SEARCHED
    ach = flops / (us_pass * 1e-6) / 1e12
    tr = profile_traffic("contact_kernel_hair.md", "per candidate pair")
    return {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s", "frac": ach / peak_tflops,
            "traffic": None if tr is None else tr * cand,
            "traffic_unit": "DRAM bytes per pass (ncu bytes per candidate pair x candidates per pass)",
            "kernel": "contact_kernel",
            "peak_kind": f"FP32 SIMT {sms} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz ({peak_kind} clock)",
            "work": {"candidates_per_pass": cand, "searched_per_pass": searched,
                     "active_per_pass": stats["active"] / passes,
                     "flop_per_candidate": CONTACT_FLOP_PER_CANDIDATE,
                     "flop_per_searched_pair": CONTACT_FLOP_PER_SEARCHED},
            "us_per_pass": us_pass}


def pairs_roofline(per_class, pairs_per_substep, sc, peaks, peak_kind):
    """HBM roofline of the pair search: 60 B per pill (spheres, cells, groups in
    cell order) + 20 B per emitted pair (pair, its first vertices, multiplier)."""
    d = per_class["pairs"]
    bytes_ = sc.ns * 60.0 + pairs_per_substep * 20.0
    ach = bytes_ / (d["us_per_launch"] * 1e-6) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
            "traffic": None, "kernel": "bp_emit_kernel", "peak_kind": f"{peak_kind} HBM copy bandwidth",
            "us_per_launch": d["us_per_launch"]}


def bench_hair_trajectory(V, torch, flush, dist, sc, cap):
    """All frames of the hair workload (the configuration's 200) from the start,
    on a fresh scene: per-frame device time, p50/p99, whole-run throughput."""
    g = V.Scene(sc, max_pairs=cap)
    ts = events_timed(torch, g.stream, flush, sc.frames, g.step)
    rc = g.sync()
    pairs_last = int(g.pairs().shape[0])
    g.close()
    if rc != 0:
        raise SystemExit(f"hair trajectory failed: {rc}")
    tot = sum(ts)
    units = reduce_sum(dist, sc.nv * sc.substeps * sc.frames)
    tot = reduce_max(dist, tot)
    return {"frames": sc.frames, "value": units / (tot * 1e-3), "unit": "rod-vertex substeps/s",
            "ms_total": tot, "ms_per_frame_mean": tot / sc.frames, "p50_ms": float(np.percentile(ts, 50)),
            "p99_ms": float(np.percentile(ts, 99)), "max_ms": float(max(ts)), "pairs_last_substep": pairs_last,
            "ms_per_frame_every_10": [round(x, 2) for x in ts[::10]]}


def bench_muscle_rig(V, torch, flush, dist, K, W, sec_frames, peaks, peak_kind, fp32_peak, sms, rank, no_plain):
    """The muscle rig (configs' 200-rod rig with bones, contacts and a 200k-vertex
    LBS mesh): frame time on the graph path, e2e through the C ABI with host
    operands, per-class times and the plain one-launch-per-colour path."""
    from paper_1906_05260_gb300 import scenes as S
    import ctypes as C
    sc = S.muscle_rig(seed=1 + rank)
    g = V.Scene(sc)
    mesh = V.Mesh(sc.mesh)
    stream = g.stream
    nb = sc.bones.n
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
    frame_no = [0]

    def device_frame():
        f = frame_no[0]
        frame_no[0] += 1
        g.set_bones(dev_q[f], dev_t[f])
        g.step()
        g.skin(mesh)

    for _ in range(W):
        device_frame()
    torch.cuda.synchronize()
    l0 = g.launch_count()
    ts = events_timed(torch, stream, flush, K, device_frame)
    launches = (g.launch_count() - l0) / K
    rc = g.sync()
    if rc != 0:
        raise SystemExit(f"muscle rig: solver error {rc}: {V.error_string(rc)}")
    units = reduce_sum(dist, sc.nv * sc.substeps)
    ms = reduce_max(dist, sum(ts) / len(ts))
    out = {"workload": MUSCLE_DESC, "rods": sc.n_rods, "vertices": sc.nv, "mesh_vertices": sc.mesh.n,
           "value": units / (ms * 1e-3), "unit": "rod-vertex substeps/s", "ms_per_frame": ms,
           "p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
           "skinned_vertices_per_s": reduce_sum(dist, sc.mesh.n) / (ms * 1e-3), "launches_per_frame": launches,
           "solver": "batched: multi-scene kernels for this scene alone, frame replayed as a CUDA graph"}

    # end to end through the C ABI with host buffers (bones in, skinned mesh out)
    out_host = torch.empty((sc.mesh.n, 4), dtype=torch.float32).pin_memory()
    rest4 = np.zeros((sc.mesh.n, 4), np.float32)
    rest4[:, :3] = sc.mesh.rest
    rest_pin = torch.from_numpy(rest4).pin_memory()
    idx_pin = torch.from_numpy(np.ascontiguousarray(sc.mesh.idx, np.int32)).pin_memory()
    w_pin = torch.from_numpy(np.ascontiguousarray(sc.mesh.w, np.float32)).pin_memory()

    def host_frame():
        f = frame_no[0]
        frame_no[0] += 1
        rcb = V.lib().viper_set_bones(g.handle, nb, C.c_void_p(pin_q[f].data_ptr()), C.c_void_p(pin_t[f].data_ptr()))
        rcs = V.lib().viper_step(g.handle, float(sc.dt), sc.substeps, sc.iterations)
        rck = V.lib().viper_skin(g.handle, sc.mesh.n, C.c_void_p(rest_pin.data_ptr()), C.c_void_p(idx_pin.data_ptr()),
                                 C.c_void_p(w_pin.data_ptr()), C.c_void_p(out_host.data_ptr()))
        if rcb or rcs or rck:
            raise SystemExit(f"muscle rig e2e frame failed: {rcb} {rcs} {rck}")

    for _ in range(3):
        host_frame()
    te = []
    for i in range(sec_frames):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_frame()
        te.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = reduce_max(dist, sum(te) / len(te))
    out["e2e"] = {"value": units / (e2e_ms * 1e-3), "unit": "rod-vertex substeps/s", "ms_per_step": e2e_ms,
                  "h2d_bytes_per_step": int(nb * (16 + 12) + sc.mesh.n * 48),
                  "d2h_bytes_per_step": int(sc.mesh.n * 16),
                  "note": "host pinned bone poses and mesh operands in, skinned mesh out, wall clock per frame"}
    out["per_class"] = per_class_times(V, torch, g, stream, flush, min(sec_frames, 20), device_frame)
    if not no_plain:
        g.set_solver(V.SOLVER_PLAIN)
        for _ in range(3):
            device_frame()
        tp = events_timed(torch, stream, flush, sec_frames, device_frame)
        pm = reduce_max(dist, sum(tp) / len(tp))
        out["plain"] = {"value": units / (pm * 1e-3), "ms_per_frame": pm, "p50_ms": float(np.percentile(tp, 50)),
                        "p99_ms": float(np.percentile(tp, 99)), "solver": "plain: one launch per constraint colour"}
        out["batched_over_plain"] = out["value"] / out["plain"]["value"]
    g.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=195)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-trajectory", action="store_true")
    ap.add_argument("--no-rig", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-multi", action="store_true")
    ap.add_argument("--no-muscles", action="store_true")
    ap.add_argument("--no-lbs", action="store_true")
    ap.add_argument("--serving", type=float, default=60.0,
                    help="seconds of the real-time serving load (0 disables)")
    ap.add_argument("--at-frame", type=int, default=-1,
                    help="profiling aid: step the hair scene this many frames, then run one substep of "
                         "one iteration (its contact pass is contact_kernel launch 40 x F) and print "
                         "that pass's contact counters; no timing")
    ap.add_argument("--serving-serial", type=float, default=10.0,
                    help="seconds of the same load served one scene per step")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.at_frame >= 0:
        return run_at_frame(args.at_frame)

    import ctypes as C
    import torch
    from paper_1906_05260_gb300 import build as B
    B.build()
    from paper_1906_05260_gb300 import viper as V

    dist, rank, ws, local = dist_setup()
    torch.cuda.set_device(local)
    peaks, peak_kind = load_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak, sms = fp32_peak_tflops(sm_max)
    K, W = args.steps, args.warmup
    sec_frames = max(10, min(K, 60) // 2)  # frames per timed section beside the main line
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    sc = hair_scene(rank)
    cap = HAIR_PAIRS_PER_PILL * sc.ns
    units = sc.nv * sc.substeps

    # ---- main line: the hair workload, frames W .. W + K - 1 of its trajectory
    g = V.Scene(sc, max_pairs=cap)
    stream = g.stream
    for _ in range(W):
        g.step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    l0 = g.launch_count()
    clocks.begin()
    ts = events_timed(torch, stream, flush, K, g.step)
    torch.cuda.synchronize()
    clocks.end()
    barrier(dist)
    launches = g.launch_count() - l0
    clk = clocks.stop()
    rc = g.sync()
    if rc != 0:
        raise SystemExit(f"solver error {rc}: {V.error_string(rc)}")
    mean_ms = sum(ts) / len(ts)
    value, mean_ms_max = whole_job(dist, units, mean_ms)
    p50 = float(np.percentile(ts, 50))
    p99 = float(np.percentile(ts, 99))
    pairs_last = int(g.pairs().shape[0])

    g.close()
    # ---- kernel classes and contact counters over the same frames, replayed
    per_class, stats = per_class_replay(V, torch, sc, cap, flush, W, K)
    dominant = max(per_class, key=lambda k: per_class[k]["ms_per_frame"])
    if dominant == "pairs":
        roof = pairs_roofline(per_class, pairs_last, sc, peaks, peak_kind)
    else:
        roof = contact_roofline(per_class, stats, sc, fp32_peak, peak_kind, sms, sm_max)
        roof["dominant_class"] = dominant
    roof["per_class"] = per_class
    roof["contact_counters"] = stats

    # ---- end to end through the C ABI: a fresh scene, the same frames, each
    # frame's positions and radii read back into pinned host memory
    ge = V.Scene(sc, max_pairs=cap)
    x4_host = torch.empty((sc.nv, 4), dtype=torch.float32).pin_memory()

    def host_frame():
        rcs = V.lib().viper_step(ge.handle, float(sc.dt), sc.substeps, sc.iterations)
        rcg = V.lib().viper_get_state(ge.handle, C.c_void_p(x4_host.data_ptr()), None, None, None)
        if rcs or rcg:
            raise SystemExit(f"e2e frame failed: {rcs} {rcg}")

    for _ in range(W):
        host_frame()
    barrier(dist)
    te = []
    for i in range(K):
        with torch.cuda.stream(ge.stream):
            flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_frame()
        te.append((time.perf_counter() - t0) * 1e3)
    barrier(dist)
    ge.close()
    e2e_ms = reduce_max(dist, sum(te) / len(te))
    e2e = {"value": reduce_sum(dist, units) / (e2e_ms * 1e-3), "unit": "rod-vertex substeps/s",
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(sc.nv * 16), "ms_per_step": e2e_ms,
           "note": "viper_step then viper_get_state of every vertex's position and scale into pinned host "
                   "memory, wall clock per frame; the frame's only inputs are its scalars (dt, substeps, "
                   "iterations), the state stays on the device"}

    # ---- the plain one-launch-per-colour path on the same frames
    plain = None
    if not args.no_plain:
        gp = V.Scene(sc, max_pairs=cap, solver=V.SOLVER_PLAIN)
        for _ in range(W):
            gp.step()
        tp = events_timed(torch, gp.stream, flush, K, gp.step)
        if gp.sync() != 0:
            raise SystemExit("plain hair path failed")
        gp.close()
        pm = reduce_max(dist, sum(tp) / len(tp))
        plain = {"value": reduce_sum(dist, units) / (pm * 1e-3), "ms_per_step": pm,
                 "p50_ms": float(np.percentile(tp, 50)), "p99_ms": float(np.percentile(tp, 99)),
                 "solver": "plain: one launch per constraint colour", "graph_over_plain": pm / mean_ms_max}

    trajectory = None if args.no_trajectory else bench_hair_trajectory(V, torch, flush, dist, sc, cap)

    rig = None
    if not args.no_rig:
        rig = bench_muscle_rig(V, torch, flush, dist, min(K, 60), W, sec_frames, peaks, peak_kind, fp32_peak, sms,
                               rank, args.no_plain)

    batching = convergence = None
    if not args.no_batching:
        batching = bench_batching(V, torch, flush, dist, peaks, peak_kind, fp32_peak, sec_frames)
        convergence = bench_convergence(V, np)
    lbs = None if args.no_lbs else bench_lbs(V, torch, flush, dist, sec_frames, peaks, peak_kind, rank=rank)
    muscles = None if args.no_muscles else bench_muscles(V, torch, flush, dist, sec_frames, rank=rank)
    multi = None if args.no_multi else bench_multi_scene(V, torch, flush, dist, sec_frames, rank=rank)

    serving = None
    if args.serving > 0:
        from paper_1906_05260_gb300 import serving as SV
        temps = SV.scene_templates(seed=4 + rank)
        conc = SV.run_load(duration=args.serving, rate=6.4, mean_life=10.0, budget=150 << 30, max_inflight=256,
                           seed=4 + rank, templates=temps, warm_scenes=64)
        ser = SV.run_load(duration=max(3.0, args.serving_serial), rate=6.4, mean_life=10.0, budget=150 << 30,
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
        "config": {"workload": WORKLOAD_DESC, "rods": sc.n_rods, "vertices": sc.nv, "pills": sc.ns,
                   "frames_timed": f"{W} .. {W + K - 1} of the trajectory",
                   "solver": "batched: shared-memory rod kernel per sweep, multi-kernel grid broadphase beside "
                             "the first sweep, contact pass after every sweep, frame replayed as a CUDA graph",
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "parallelism": f"replicas x{ws} (independent seeded scenes)"},
        "latency_ms": {"p50": p50, "p99": p99}, "pairs_last_substep": pairs_last,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
        "plain": plain,
        "trajectory": trajectory,
        "muscle_rig": rig,
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
