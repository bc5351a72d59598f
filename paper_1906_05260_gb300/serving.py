"""Serving driver: many independent scenes stepped as frame requests arrive.

`Server` wraps the C ABI's viper_server_* calls (marshalling only; admission,
queueing, dispatch through the multi-scene frame step and timing run in
libviper.so's native dispatcher).
`run_load` replays a seeded Poisson stream of muscle-rig scenes with
exponential lifetimes, each issuing 60 Hz frame-step requests, in real time,
and reports latency percentiles and aggregate throughput.
"""
from __future__ import annotations

import ctypes as C
import math
import time

import numpy as np

from . import scenes as S
from . import viper as V


class Server:
    def __init__(self, budget_bytes: int, max_inflight: int = 64):
        h = C.c_void_p()
        V._check(V.lib().viper_server_create(int(budget_bytes), int(max_inflight), C.byref(h)), "viper_server_create")
        self._h = h
        self.scenes = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            V.lib().viper_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, scene, solver=V.SOLVER_BATCHED):
        """Scene id, or None if it does not fit the memory budget now."""
        desc, keep = V.make_desc(scene, None)
        sid = C.c_int()
        n = 0
        args = [None, None, None]
        if scene.mesh is not None:
            n = scene.mesh.n
            rest = np.zeros((n, 4), np.float32)
            rest[:, :3] = scene.mesh.rest
            idx = np.ascontiguousarray(scene.mesh.idx, np.int32)
            w = np.ascontiguousarray(scene.mesh.w, np.float32)
            keep += [rest, idx, w]
            args = [C.c_void_p(a.ctypes.data) for a in (rest, idx, w)]
        rc = V.lib().viper_server_admit(self._h, C.byref(desc), n, *args, int(solver), float(scene.dt),
                                        int(scene.substeps), int(scene.iterations), C.byref(sid))
        if rc == V.EBUDGET:
            return None
        V._check(rc, "viper_server_admit")
        self.scenes[sid.value] = scene
        return sid.value

    def submit(self, sid: int, t_end: float, dt=None, substeps=None, iterations=None):
        sc = self.scenes[sid]
        q, tr = sc.bone_pose(t_end)
        q = np.ascontiguousarray(q, np.float32)
        tr = np.ascontiguousarray(tr, np.float32)
        tk = C.c_longlong()
        V._check(V.lib().viper_server_submit(self._h, sid, C.c_void_p(q.ctypes.data), C.c_void_p(tr.ctypes.data),
                                             float(dt or sc.dt), int(substeps or sc.substeps),
                                             int(iterations if iterations is not None else sc.iterations),
                                             C.byref(tk)), "viper_server_submit")
        return tk.value

    def wait(self, ticket: int, timeout_ms: float = 60_000.0):
        st = C.c_int()
        lat = C.c_double()
        V._check(V.lib().viper_server_wait(self._h, ticket, float(timeout_ms), C.byref(st), C.byref(lat)),
                 "viper_server_wait")
        return st.value, lat.value

    def idle(self, timeout_ms: float = 60_000.0):
        V._check(V.lib().viper_server_idle(self._h, float(timeout_ms)), "viper_server_idle")

    def release(self, sid: int):
        V._check(V.lib().viper_server_release(self._h, sid), "viper_server_release")
        self.scenes.pop(sid, None)

    def state(self, sid: int):
        """State of an idle scene (x4, v4, q4, w4 in the scene's numbering)."""
        h = V.lib().viper_server_scene(self._h, sid)
        sc = self.scenes[sid]
        x4 = np.zeros((sc.nv, 4), np.float32); v4 = np.zeros((sc.nv, 4), np.float32)
        q4 = np.zeros((sc.ns, 4), np.float32); w4 = np.zeros((sc.ns, 4), np.float32)
        V._check(V.lib().viper_get_state(C.c_void_p(h), *[C.c_void_p(a.ctypes.data) for a in (x4, v4, q4, w4)]),
                 "viper_get_state")
        return {"x4": x4, "v4": v4, "q4": q4, "w4": w4}

    def mesh_out(self, sid: int):
        sc = self.scenes[sid]
        out = np.zeros((sc.mesh.n, 4), np.float32)
        V._check(V.lib().viper_server_mesh_out(self._h, sid, C.c_void_p(out.ctypes.data)), "viper_server_mesh_out")
        return out

    def stats(self):
        st = V.ServerStats()
        V._check(V.lib().viper_server_get_stats(self._h, C.byref(st)), "viper_server_get_stats")
        return {k: getattr(st, k) for k, _ in V.ServerStats._fields_}

    def reset_stats(self):
        V.lib().viper_server_reset_stats(self._h)


def scene_templates(seed: int = 4, n: int = 12, rods_lo: int = 50, rods_hi: int = 500, mesh_lo: int = 10_000,
                    mesh_hi: int = 300_000):
    """Muscle rigs spanning the log-uniform size range (rods, mesh vertices)."""
    out = []
    for i in range(n):
        f = (i + 0.5) / n
        nr = int(round(math.exp(math.log(rods_lo) + f * (math.log(rods_hi) - math.log(rods_lo)))))
        fm = ((i * 7) % n + 0.5) / n  # decorrelate mesh size from rod count
        nm = int(round(math.exp(math.log(mesh_lo) + fm * (math.log(mesh_hi) - math.log(mesh_lo)))))
        out.append(S.muscle_rig(seed=10_000 * seed + i, n_rods=nr, mesh_verts=nm, frames=1))
    return out


def run_load(duration: float = 60.0, rate: float = 6.4, mean_life: float = 10.0, budget: int = 150 << 30,
             max_inflight: int = 256, seed: int = 4, hz: float = 60.0, templates=None, warm_scenes: int = 0):
    """Replay a Poisson stream of scenes in real time; returns a summary dict.

    Scene arrivals are Poisson(rate), lifetimes Exp(mean_life); a live scene
    submits one frame request every 1/hz seconds of wall time; scenes that do
    not fit the budget wait in an admission queue.
    """
    templates = templates or scene_templates(seed)
    rng = np.random.default_rng(seed)
    arrivals = S.poisson_arrivals(seed, rate, mean_life, duration)
    # steady state from the start: `warm_scenes` scenes alive at t = 0
    arrivals = [(0.0, rng.exponential(mean_life)) for _ in range(warm_scenes)] + arrivals
    arrivals.sort()
    srv = Server(budget, max_inflight)
    live = {}  # sid -> [next_request_time, leave_time, local_time]
    waiting = []
    ai = 0
    t0 = time.perf_counter()
    peak_live = 0
    submitted = 0
    refused = 0
    admit_ms = []
    while True:
        now = time.perf_counter() - t0
        if now >= duration:
            break
        while ai < len(arrivals) and arrivals[ai][0] <= now:
            waiting.append(arrivals[ai])
            ai += 1
        still = []
        for t_arr, t_leave in waiting:
            sc = templates[int(rng.integers(len(templates)))]
            ta = time.perf_counter()
            sid = srv.admit(sc)
            if sid is None:
                refused += 1
                still.append((t_arr, t_leave))
                continue
            admit_ms.append((time.perf_counter() - ta) * 1e3)
            live[sid] = [time.perf_counter() - t0, t_arr + (t_leave - t_arr), 0.0]
        waiting = still
        now = time.perf_counter() - t0
        for sid in list(live):
            nxt, leave, tloc = live[sid]
            if now >= leave:
                srv.release(sid)
                del live[sid]
                continue
            while nxt <= now:
                sc = srv.scenes[sid]
                tloc += sc.dt
                srv.submit(sid, tloc)
                submitted += 1
                nxt += 1.0 / hz
            live[sid] = [nxt, leave, tloc]
        peak_live = max(peak_live, len(live))
        nexts = [v[0] for v in live.values()] + ([arrivals[ai][0]] if ai < len(arrivals) else [])
        wake = min(nexts) if nexts else now + 0.001
        delay = wake - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(min(delay, 0.002))
    elapsed = time.perf_counter() - t0
    srv.idle(120_000.0)
    st = srv.stats()
    for sid in list(live):
        srv.release(sid)
    srv.close()
    return {"duration_s": elapsed, "frames": st["frames"], "failed": st["failed"], "submitted": submitted,
            "rod_vertex_substeps_per_s": st["rod_vertex_substeps"] / elapsed, "p50_ms": st["p50_ms"],
            "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "mean_ms": st["mean_ms"], "peak_live_scenes": peak_live,
            "arrivals": len(arrivals), "budget_refusals": refused, "max_inflight": max_inflight,
            "steps": st["steps"], "mean_scenes_per_step": st["frames"] / max(st["steps"], 1),
            "admit_ms_p50": float(np.percentile(admit_ms, 50)) if admit_ms else None}
