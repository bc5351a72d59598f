"""Thin Python binding of the VIPER C ABI (include/viper.h).

Argument marshalling only: every step of the solver runs in libviper.so's CUDA
kernels.  PyTorch supplies device memory (through the library's allocator
hook, backed by torch's caching allocator) and CUDA streams.  There is no CPU
fallback: if the compiled library is missing or no GPU is present, calls fail.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libviper.so")

OK = 0
EINVAL, ENOMEM, ECUDA, ENONFINITE, EOVERFLOW, ETIMEOUT, EBUDGET, ENOCONV, ECONTACTS = -1, -2, -3, -4, -5, -6, -7, -8, -9
FLAG_CONTACTS, FLAG_VOLUME, FLAG_SURFACE_BENDING, FLAG_JACOBI, FLAG_WARM_START = 1, 2, 4, 8, 16
FLAG_VOLUME_VECTOR = 32
FLAG_CONTACT_THREADS = 64  # contact pass with one thread per pair always (timing only)
SOLVER_PLAIN, SOLVER_BATCHED, SOLVER_FRAME = 0, 1, 2
SOLVER_AUTO = -1
PROF_NONE, PROF_ROD, PROF_CONTACT, PROF_BROADPHASE, PROF_LBS, PROF_ELEMENTWISE, PROF_PAIRS = 0, 1, 2, 3, 4, 5, 6

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_fp = C.POINTER(C.c_float)


class ViperError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} ({code})")


class Desc(C.Structure):
    """Mirror of viper_scene_desc."""
    _fields_ = [
        ("n_rods", C.c_int), ("rod_offsets", _ip), ("rest_pos", _dp), ("rest_quat", _dp),
        ("radius", _dp), ("density", _dp), ("c_stretch", _dp), ("c_bend", _dp), ("c_volume", _dp),
        ("group", _ip), ("gravity", C.c_double * 3), ("n_pins", C.c_int), ("pin_vertex", _ip),
        ("pin_bone", _ip), ("pin_offset", _dp), ("n_bones", C.c_int), ("bone_quat", _dp),
        ("bone_trans", _dp), ("n_planes", C.c_int), ("planes", _dp),
        ("contact_compliance", C.c_double), ("flags", C.c_int), ("max_pairs", C.c_int),
        ("stream", C.c_void_p), ("n_bundles", C.c_int), ("bundle_offsets", _ip), ("bundle_rods", _ip),
    ]


class ServerStats(C.Structure):
    """Mirror of viper_server_stats."""
    _fields_ = [("frames", C.c_longlong), ("failed", C.c_longlong), ("rod_vertex_substeps", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("scenes", C.c_int), ("inflight", C.c_int), ("queued", C.c_int), ("used_bytes", C.c_size_t),
                ("steps", C.c_longlong)]


class BatchItem(C.Structure):
    """Mirror of viper_batch_item."""
    _fields_ = [("scene", C.c_void_p), ("bone_quat", C.c_void_p), ("bone_trans", C.c_void_p),
                ("n_mesh", C.c_int), ("rest4", C.c_void_p), ("idx4", C.c_void_p), ("w4", C.c_void_p),
                ("out4", C.c_void_p)]


_lib = None
_ALLOC_T = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_T = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_torch_hooks = None
_live = weakref.WeakSet()


def lib():
    """Load libviper.so (built by paper_1906_05260_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.viper_scene_create.argtypes = [C.POINTER(Desc), C.POINTER(vp)]
        L.viper_scene_destroy.argtypes = [vp]
        L.viper_scene_destroy.restype = None
        L.viper_scene_counts.argtypes = [vp, _ip, _ip, _ip]
        L.viper_set_solver.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.viper_autotune.argtypes = [vp, C.c_float, C.c_int, C.c_int, _ip]
        L.viper_step.argtypes = [vp, C.c_float, C.c_int, C.c_int]
        L.viper_set_bones.argtypes = [vp, C.c_int, vp, vp]
        L.viper_set_activation.argtypes = [vp, vp]
        L.viper_skin.argtypes = [vp, C.c_int, vp, vp, vp, vp]
        L.viper_get_state.argtypes = [vp, vp, vp, vp, vp]
        L.viper_set_state.argtypes = [vp, vp, vp, vp, vp]
        L.viper_sync.argtypes = [vp]
        L.viper_get_pairs.argtypes = [vp, _ip, C.c_int, _ip]
        L.viper_get_colouring.argtypes = [vp, _ip, _ip]
        L.viper_get_predicted.argtypes = [vp, vp, vp]
        L.viper_set_allocator.argtypes = [vp, vp, vp]
        L.viper_scene_footprint.argtypes = [C.POINTER(Desc)]
        L.viper_scene_footprint.restype = C.c_size_t
        L.viper_profile.argtypes = [vp, C.c_int]
        L.viper_profile_read.argtypes = [vp, _dp, _ip]
        L.viper_broadphase.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp, C.c_int, vp, vp]
        L.viper_broadphase_noalloc.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp, C.c_int, vp, vp]
        L.viper_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(vp)]
        L.viper_server_destroy.argtypes = [vp]
        L.viper_server_destroy.restype = None
        L.viper_server_admit.argtypes = [vp, C.POINTER(Desc), C.c_int, vp, vp, vp, C.c_int, C.c_float, C.c_int,
                                         C.c_int, _ip]
        L.viper_prepare.argtypes = [vp, C.c_float, C.c_int, C.c_int]
        L.viper_server_submit.argtypes = [vp, C.c_int, vp, vp, C.c_float, C.c_int, C.c_int,
                                          C.POINTER(C.c_longlong)]
        L.viper_server_wait.argtypes = [vp, C.c_longlong, C.c_double, _ip, _dp]
        L.viper_server_idle.argtypes = [vp, C.c_double]
        L.viper_server_release.argtypes = [vp, C.c_int]
        L.viper_server_scene.argtypes = [vp, C.c_int]
        L.viper_server_scene.restype = vp
        L.viper_server_mesh_out.argtypes = [vp, C.c_int, vp]
        L.viper_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.viper_server_reset_stats.argtypes = [vp]
        L.viper_batch_create.argtypes = [vp, C.POINTER(vp)]
        L.viper_batch_destroy.argtypes = [vp]
        L.viper_batch_destroy.restype = None
        L.viper_batch_step.argtypes = [vp, C.POINTER(BatchItem), C.c_int, C.c_float, C.c_int, C.c_int, _ip]
        L.viper_batch_stream.argtypes = [vp]
        L.viper_batch_stream.restype = vp
        L.viper_batch_launch_count.argtypes = [vp]
        L.viper_batch_launch_count.restype = C.c_longlong
        L.viper_launch_count.argtypes = [vp]
        L.viper_launch_count.restype = C.c_longlong
        L.viper_contact_stats.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.viper_schedule.argtypes = [vp, _ip, _ip, _ip]
        L.viper_error_string.argtypes = [C.c_int]
        L.viper_error_string.restype = C.c_char_p
        _lib = L
    return _lib


def error_string(code: int) -> str:
    try:
        return lib().viper_error_string(int(code)).decode()
    except Exception:  # library not loadable: still report the number
        return "error"


def _check(rc, where):
    if rc != OK:
        raise ViperError(rc, where)
    return rc


def use_torch_allocator():
    """Route all later scene allocations through torch's CUDA caching allocator."""
    global _torch_hooks
    import torch
    if _torch_hooks is not None:
        return

    def _alloc(nbytes, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:
            return None

    def _free(ptr, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    _torch_hooks = (_ALLOC_T(_alloc), _FREE_T(_free))
    _check(lib().viper_set_allocator(C.cast(_torch_hooks[0], C.c_void_p), C.cast(_torch_hooks[1], C.c_void_p),
                                     None), "viper_set_allocator")


def _d(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32).reshape(-1)
    return a, a.ctypes.data_as(_ip)


def make_desc(scene, stream_handle=None, max_pairs=0, extra_flags=0):
    """Marshal a scenes.Scene into a viper_scene_desc; returns (desc, keepalive)."""
    keep = []

    def d(a):
        arr, p = _d(a)
        keep.append(arr)
        return p

    def i(a):
        arr, p = _i(a)
        keep.append(arr)
        return p

    desc = Desc()
    desc.n_rods = scene.n_rods
    desc.rod_offsets = i(scene.rod_offsets)
    desc.rest_pos = d(scene.rest_pos)
    desc.rest_quat = d(scene.rest_quat)
    desc.radius = d(scene.radius)
    desc.density = d(scene.density)
    desc.c_stretch = d(scene.c_stretch)
    desc.c_bend = d(scene.c_bend)
    desc.c_volume = d(scene.c_volume)
    desc.group = i(scene.group)
    for c in range(3):
        desc.gravity[c] = float(scene.gravity[c])
    n_pins = int(scene.pin_vertex.shape[0])
    desc.n_pins = n_pins
    desc.pin_vertex = i(scene.pin_vertex if n_pins else np.zeros(1))
    desc.pin_bone = i(scene.pin_bone if n_pins else np.zeros(1))
    desc.pin_offset = d(scene.pin_offset if n_pins else np.zeros(3))
    nb = 0 if scene.bones is None else scene.bones.n
    desc.n_bones = nb
    q0, t0 = scene.bone_pose(0.0) if nb else (np.zeros(4), np.zeros(3))
    desc.bone_quat = d(q0)
    desc.bone_trans = d(t0)
    n_planes = int(scene.planes.shape[0])
    desc.n_planes = n_planes
    desc.planes = d(scene.planes if n_planes else np.zeros(4))
    desc.contact_compliance = float(scene.contact_compliance)
    desc.flags = ((FLAG_CONTACTS if scene.contacts else 0) | (FLAG_VOLUME if scene.volume else 0)
                  | (FLAG_SURFACE_BENDING if getattr(scene, "surface_bending", False) else 0)
                  | (FLAG_JACOBI if getattr(scene, "jacobi", False) else 0)
                  | (FLAG_WARM_START if getattr(scene, "warm_start", False) else 0)
                  | (FLAG_VOLUME_VECTOR if getattr(scene, "volume_vector", False) else 0) | int(extra_flags))
    desc.max_pairs = int(max_pairs)
    desc.stream = stream_handle
    if getattr(scene, "bundle_offsets", None) is not None and len(scene.bundle_offsets) > 1:
        desc.n_bundles = len(scene.bundle_offsets) - 1
        desc.bundle_offsets = i(scene.bundle_offsets)
        desc.bundle_rods = i(scene.bundle_rods)
    return desc, keep


def footprint(scene, max_pairs=0) -> int:
    desc, keep = make_desc(scene, None, max_pairs)
    return int(lib().viper_scene_footprint(C.byref(desc)))


class Mesh:
    """Skinning mesh staged on the device as 128-bit-aligned float4/int4 rows."""

    def __init__(self, mesh, device="cuda"):
        import torch
        m = mesh.n
        rest = np.zeros((m, 4), np.float32)
        rest[:, :3] = mesh.rest
        self.n = m
        self.rest = torch.from_numpy(rest).to(device)
        self.idx = torch.from_numpy(np.ascontiguousarray(mesh.idx, np.int32)).to(device)
        self.w = torch.from_numpy(np.ascontiguousarray(mesh.w, np.float32)).to(device)
        self.out = torch.empty((m, 4), dtype=torch.float32, device=device)


class Scene:
    """A device-resident VIPER scene (one viper_scene handle)."""

    def __init__(self, scene, stream=None, solver=SOLVER_AUTO, block_warps=4, resident_max=256,
                 max_pairs=0, torch_allocator=True, extra_flags=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required")
        L = lib()
        if torch_allocator:
            use_torch_allocator()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        desc, keep = make_desc(scene, C.c_void_p(self.stream.cuda_stream), max_pairs, extra_flags)
        h = C.c_void_p()
        with torch.cuda.stream(self.stream):
            _check(L.viper_scene_create(C.byref(desc), C.byref(h)), "viper_scene_create")
        self._h = h
        self.scene = scene
        self.n_rods, self.nv, self.ns = scene.n_rods, scene.nv, scene.ns
        self.t = 0.0
        _live.add(self)
        # auto: the graph-replayed shared-memory path (measured fastest on contact scenes;
        # the persistent frame kernel is an explicit option); the vector volume form
        # runs on the plain path only
        if solver == SOLVER_AUTO:
            solver = SOLVER_PLAIN if (scene.volume and getattr(scene, "volume_vector", False)) else SOLVER_BATCHED
        self.set_solver(solver, block_warps, resident_max)
        if scene.init_pos is not None or scene.init_quat is not None:
            x4 = self.get_state()["x4"]
            q4 = None
            if scene.init_pos is not None:
                x4[:, :3] = scene.init_pos
            if scene.init_quat is not None:
                q4 = np.ascontiguousarray(scene.init_quat, np.float32)
            self.set_state(x4=x4, q4=q4)

    # -- lifecycle
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().viper_scene_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- solver
    def set_solver(self, mode=SOLVER_BATCHED, block_warps=4, resident_max=256):
        _check(lib().viper_set_solver(self._h, int(mode), int(block_warps), int(resident_max)), "viper_set_solver")
        self.solver = mode

    def autotune(self, dt=None, substeps=None, iterations=None):
        sc = self.scene
        out = C.c_int()
        _check(lib().viper_autotune(self._h, float(dt or sc.dt), int(substeps or sc.substeps),
                                    int(iterations if iterations is not None else sc.iterations),
                                    C.byref(out)), "viper_autotune")
        return divmod(out.value, 1000)

    def autotune_cached(self, path, dt=None, substeps=None, iterations=None):
        """autotune(), its choice kept in the JSON file `path` under a key of the
        GPU's name and a hash of the rod lengths, step parameters and contact
        flag; a cached choice is applied without timing.  Returns
        ((block_warps, resident_max), cached)."""
        import hashlib
        import json
        import torch
        sc = self.scene
        params = (float(dt or sc.dt), int(substeps or sc.substeps),
                  int(iterations if iterations is not None else sc.iterations), bool(sc.contacts))
        digest = hashlib.sha256(np.ascontiguousarray(np.diff(sc.rod_offsets), np.int64).tobytes() +
                                repr(params).encode()).hexdigest()[:16]
        key = f"{torch.cuda.get_device_name()}:{digest}"
        cache = {}
        if os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if key in cache:
            bw, rm = cache[key]
            self.set_solver(SOLVER_BATCHED, bw, rm)
            return (bw, rm), True
        bw, rm = self.autotune(dt, substeps, iterations)
        cache[key] = [bw, rm]
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, path)
        return (bw, rm), False

    def schedule(self):
        """(work items, threads per CTA, resident vertices) of the batched solver."""
        n, t, r = C.c_int(), C.c_int(), C.c_int()
        _check(lib().viper_schedule(self._h, C.byref(n), C.byref(t), C.byref(r)), "viper_schedule")
        return n.value, t.value, r.value

    # -- stepping
    def step(self, dt=None, substeps=None, iterations=None, check=True):
        sc = self.scene
        rc = lib().viper_step(self._h, float(dt if dt is not None else sc.dt),
                              int(substeps if substeps is not None else sc.substeps),
                              int(iterations if iterations is not None else sc.iterations))
        self.t += float(dt if dt is not None else sc.dt)
        if check:
            _check(rc, "viper_step")
        return rc

    def set_bones(self, quat, trans):
        """quat [nb,4], trans [nb,3]: numpy (host) or torch CUDA tensors."""
        q, t = _ptr_f32(quat), _ptr_f32(trans)
        _check(lib().viper_set_bones(self._h, int(self.scene.bones.n), q[1], t[1]), "viper_set_bones")

    def set_activation(self, a=None):
        """Muscle activation per rod in [0, 0.9] (None: the original rest state)."""
        if a is None:
            rc = lib().viper_set_activation(self._h, None)
        else:
            arr = np.ascontiguousarray(a, dtype=np.float32)
            if arr.shape != (self.scene.n_rods,):
                raise ValueError("one activation per rod")
            rc = lib().viper_set_activation(self._h, arr.ctypes.data_as(C.c_void_p))
        _check(rc, "viper_set_activation")

    def frame(self):
        """One frame of the scene's schedule with bones set to their pose at the frame end."""
        sc = self.scene
        if sc.bones is not None:
            self.set_bones(*sc.bone_pose(self.t + sc.dt))
        return self.step()

    def skin(self, mesh: Mesh):
        """LBS of the current state into mesh.out (enqueued on the scene stream;
        torch's current stream is made to wait for it before later torch work)."""
        import torch
        _check(lib().viper_skin(self._h, mesh.n, C.c_void_p(mesh.rest.data_ptr()), C.c_void_p(mesh.idx.data_ptr()),
                                C.c_void_p(mesh.w.data_ptr()), C.c_void_p(mesh.out.data_ptr())), "viper_skin")
        torch.cuda.current_stream().wait_stream(self.stream)
        return mesh.out

    def skin_host(self, rest4, idx4, w4, out4):
        """Skinning with host (numpy) operands; synchronous."""
        args = [np.ascontiguousarray(a) for a in (rest4, idx4, w4)]
        _check(lib().viper_skin(self._h, int(args[0].shape[0]), *[C.c_void_p(a.ctypes.data) for a in args],
                                C.c_void_p(out4.ctypes.data)), "viper_skin")
        return out4

    def sync(self):
        return lib().viper_sync(self._h)

    # -- state
    def get_state(self):
        x4 = np.zeros((self.nv, 4), np.float32); v4 = np.zeros((self.nv, 4), np.float32)
        q4 = np.zeros((self.ns, 4), np.float32); w4 = np.zeros((self.ns, 4), np.float32)
        rc = lib().viper_get_state(self._h, *[C.c_void_p(a.ctypes.data) for a in (x4, v4, q4, w4)])
        return {"x4": x4, "v4": v4, "q4": q4, "w4": w4, "rc": rc}

    def set_state(self, x4=None, v4=None, q4=None, w4=None):
        arrs = [None if a is None else np.ascontiguousarray(a, np.float32) for a in (x4, v4, q4, w4)]
        _check(lib().viper_set_state(self._h, *[None if a is None else C.c_void_p(a.ctypes.data) for a in arrs]),
               "viper_set_state")

    # -- introspection
    def pairs(self):
        n = C.c_int()
        _check(lib().viper_get_pairs(self._h, None, 0, C.byref(n)), "viper_get_pairs")
        out = np.zeros((max(n.value, 1), 2), np.int32)
        _check(lib().viper_get_pairs(self._h, out.ctypes.data_as(_ip), n.value, C.byref(n)), "viper_get_pairs")
        return out[: n.value]

    def colouring(self):
        sc = np.zeros(self.ns, np.int32); vc = np.zeros(self.nv, np.int32)
        rc = lib().viper_get_colouring(self._h, sc.ctypes.data_as(_ip), vc.ctypes.data_as(_ip))
        _check(rc, "viper_get_colouring")
        return sc, vc

    def predicted(self):
        x4 = np.zeros((self.nv, 4), np.float32); rb = np.zeros(self.nv, np.float32)
        _check(lib().viper_get_predicted(self._h, C.c_void_p(x4.ctypes.data), C.c_void_p(rb.ctypes.data)),
               "viper_get_predicted")
        return x4, rb

    def profile(self, kernel_class: int):
        """Bracket one kernel class with CUDA events (drops cached graphs)."""
        _check(lib().viper_profile(self._h, int(kernel_class)), "viper_profile")

    def profile_read(self):
        """(device ms, launches) of the profiled class in the last frame + skin calls."""
        ms = C.c_double(); n = C.c_int()
        _check(lib().viper_profile_read(self._h, C.byref(ms), C.byref(n)), "viper_profile_read")
        return ms.value, n.value

    def launch_count(self) -> int:
        return int(lib().viper_launch_count(self._h))

    def contact_stats(self):
        """(candidate pairs, searched pairs, active constraints) summed over the
        contact passes since the previous call; resets the counters."""
        out = (C.c_longlong * 3)()
        _check(lib().viper_contact_stats(self._h, out), "viper_contact_stats")
        return int(out[0]), int(out[1]), int(out[2])


def broadphase(rod_offsets, group, x4, rbar, max_pairs, stream=None):
    """Stand-alone broadphase on device tensors (torch): returns (pairs[n,2] sorted, total count).

    rod_offsets/group int32, x4 float32 [nv,4] (x, y, z, scale), rbar float32 [nv]."""
    import torch
    dev = x4.device
    n_rods = int(rod_offsets.numel() - 1)
    pairs = torch.empty((max(int(max_pairs), 1), 2), dtype=torch.int32, device=dev)
    n = torch.zeros(1, dtype=torch.int32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().viper_broadphase(n_rods, int(x4.shape[0]), C.c_void_p(rod_offsets.data_ptr()),
                                  None if group is None else C.c_void_p(group.data_ptr()),
                                  C.c_void_p(x4.data_ptr()), C.c_void_p(rbar.data_ptr()),
                                  C.c_void_p(pairs.data_ptr()), int(max_pairs), C.c_void_p(n.data_ptr()),
                                  C.c_void_p(st.cuda_stream)), "viper_broadphase")
    st.synchronize()
    total = int(n.item())
    got = pairs[: min(total, int(max_pairs))].cpu().numpy()
    order = np.lexsort((got[:, 1], got[:, 0])) if got.size else np.zeros(0, np.int64)
    return got[order], total


class Batch:
    """A multi-scene step context (viper_batch): one launch sequence per frame for many scenes."""

    def __init__(self, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        _check(lib().viper_batch_create(C.c_void_p(self.stream.cuda_stream), C.byref(h)), "viper_batch_create")
        self._h = h
        _live.add(self)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().viper_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, scenes, poses=None, meshes=None, dt=1.0 / 60, substeps=10, iterations=4, check=True):
        """One frame of every scene.  poses[i] = (quat [nb,4], trans [nb,3]) host arrays or None;
        meshes[i] = Mesh or None.  Returns the per-scene latched status codes."""
        n = len(scenes)
        items = (BatchItem * max(n, 1))()
        keep = []
        for i, sc in enumerate(scenes):
            it = items[i]
            it.scene = sc.handle.value
            pose = poses[i] if poses is not None else None
            if pose is not None:
                q = np.ascontiguousarray(pose[0], np.float32)
                t = np.ascontiguousarray(pose[1], np.float32)
                keep += [q, t]
                it.bone_quat, it.bone_trans = q.ctypes.data, t.ctypes.data
            m = meshes[i] if meshes is not None else None
            if m is not None:
                it.n_mesh = m.n
                it.rest4, it.idx4 = m.rest.data_ptr(), m.idx.data_ptr()
                it.w4, it.out4 = m.w.data_ptr(), m.out.data_ptr()
        status = (C.c_int * max(n, 1))()
        rc = lib().viper_batch_step(self._h, items, n, float(dt), int(substeps), int(iterations), status)
        if check:
            _check(rc, "viper_batch_step")
        return [status[i] for i in range(n)]

    def frame(self, scenes, meshes=None):
        """One frame of each scene's own schedule (dt, substeps, iterations must agree), bones at the frame end."""
        sc0 = scenes[0].scene
        poses = []
        for s in scenes:
            sc = s.scene
            if (sc.dt, sc.substeps, sc.iterations) != (sc0.dt, sc0.substeps, sc0.iterations):
                raise ValueError("scenes of one batched frame share dt, substeps and iterations")
            poses.append(sc.bone_pose(s.t + sc.dt) if sc.bones is not None else None)
        st = self.step(scenes, poses, meshes, sc0.dt, sc0.substeps, sc0.iterations)
        for s in scenes:
            s.t += sc0.dt
        return st

    def synchronize(self):
        self.stream.synchronize()

    def launch_count(self) -> int:
        return int(lib().viper_batch_launch_count(self._h))


def _ptr_f32(a):
    """(keepalive, pointer) for a float32 numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            t = a.contiguous().float()
            return t, C.c_void_p(t.data_ptr())
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, np.float32)
    return arr, C.c_void_p(arr.ctypes.data)


@atexit.register
def _close_all():
    for s in list(_live):
        try:
            s.close()
        except Exception:
            pass
