"""FP64 CPU oracle of the VIPER rod solve -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
use this package.  The product library never imports it.  The C source
(``vo.c``) restates the paper step by step; this module compiles it with gcc
(``-ffp-contract=off`` so that the single-precision broadphase predicate keeps
its fixed operation order) and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vo.c")
_HDR = os.path.join(_HERE, "vo.h")
_LIB = os.path.join(_HERE, "libvo.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_fp = C.POINTER(C.c_float)


class _Desc(C.Structure):
    _fields_ = [
        ("n_rods", C.c_int), ("rod_offsets", _ip), ("rest_pos", _dp), ("rest_quat", _dp),
        ("radius", _dp), ("density", _dp), ("c_stretch", _dp), ("c_bend", _dp),
        ("c_volume", _dp), ("group", _ip), ("gravity", C.c_double * 3), ("n_pins", C.c_int),
        ("pin_vertex", _ip), ("pin_bone", _ip), ("pin_offset", _dp), ("n_bones", C.c_int),
        ("bone_quat", _dp), ("bone_trans", _dp), ("n_planes", C.c_int), ("planes", _dp),
        ("contact_compliance", C.c_double), ("contacts", C.c_int), ("volume", C.c_int),
        ("surface_bending", C.c_int), ("jacobi", C.c_int),
        ("volume_vector", C.c_int), ("warm_start", C.c_int), ("n_bundles", C.c_int), ("bundle_offsets", _ip), ("bundle_rods", _ip),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libvo.so (plain C11, -O2, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.vo_create.restype = C.c_void_p
        L.vo_create.argtypes = [C.POINTER(_Desc)]
        L.vo_destroy.argtypes = [C.c_void_p]
        L.vo_set_threads.argtypes = [C.c_void_p, C.c_int]
        L.vo_set_state.argtypes = [C.c_void_p] + [_dp] * 6
        L.vo_get_state.argtypes = [C.c_void_p] + [_dp] * 6
        L.vo_set_bones.argtypes = [C.c_void_p, _dp, _dp]
        L.vo_step.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int]
        L.vo_skin.argtypes = [C.c_void_p, C.c_int, _dp, _ip, _dp, _dp]
        L.vo_last_pairs.argtypes = [C.c_void_p, _ip, C.c_int]
        L.vo_broadphase_f32.argtypes = [C.c_int, _ip, _ip, _fp, _fp, C.c_int, _ip, C.c_int]
        L.vo_pill_project.restype = C.c_double
        L.vo_pill_project.argtypes = [_dp, C.c_double, _dp, C.c_double, _dp]
        L.vo_narrowphase.argtypes = [_dp, C.c_double, _dp, C.c_double, _dp, C.c_double, _dp,
                                     C.c_double, _dp, _dp, _dp]
        L.vo_segment_constraint.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, _dp,
                                            C.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
        L.vo_vertex_constraint.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                           _dp, _dp, _dp, _dp, _dp]
        L.vo_segment_compliance.argtypes = [C.c_void_p, C.c_int, _dp]
        L.vo_vertex_compliance.argtypes = [C.c_void_p, C.c_int, _dp]
        L.vo_vertex_inverse_inertia.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.vo_rest.argtypes = [C.c_void_p, _dp, _dp]
        L.vo_colouring.argtypes = [C.c_void_p, _ip, _ip]
        L.vo_constraint_rms.argtypes = [C.c_void_p, _dp]
        L.vo_laplacian_constraint.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                              _dp, _dp]
        L.vo_polar_rotation.argtypes = [_dp, _dp]
        L.vo_set_activation.argtypes = [C.c_void_p, _dp]
        L.vo_shape_match.argtypes = [C.c_void_p]
        L.vo_laplacian_compliance.restype = C.c_double
        L.vo_laplacian_compliance.argtypes = [C.c_void_p, C.c_int]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


class OracleScene:
    """FP64 oracle scene built from a ``scenes.Scene``."""

    def __init__(self, scene, threads=1):
        L = lib()
        self.scene = scene
        keep = []

        def d(a):
            arr, p = _d(a)
            keep.append(arr)
            return p

        def i(a):
            arr, p = _i(a)
            keep.append(arr)
            return p

        desc = _Desc()
        desc.n_rods = scene.n_rods
        desc.rod_offsets = i(scene.rod_offsets)
        desc.rest_pos = d(scene.rest_pos.reshape(-1))
        desc.rest_quat = d(scene.rest_quat.reshape(-1))
        desc.radius = d(scene.radius)
        desc.density = d(scene.density)
        desc.c_stretch = d(scene.c_stretch)
        desc.c_bend = d(scene.c_bend)
        desc.c_volume = d(scene.c_volume)
        desc.group = i(scene.group)
        for c in range(3):
            desc.gravity[c] = float(scene.gravity[c])
        desc.n_pins = int(scene.pin_vertex.shape[0])
        desc.pin_vertex = i(scene.pin_vertex if desc.n_pins else np.zeros(1))
        desc.pin_bone = i(scene.pin_bone if desc.n_pins else np.zeros(1))
        desc.pin_offset = d(scene.pin_offset.reshape(-1) if desc.n_pins else np.zeros(3))
        nb = 0 if scene.bones is None else scene.bones.n
        desc.n_bones = nb
        if nb:
            q0, t0 = scene.bone_pose(0.0)
        else:
            q0, t0 = np.zeros(4), np.zeros(3)
        desc.bone_quat = d(q0.reshape(-1))
        desc.bone_trans = d(t0.reshape(-1))
        desc.n_planes = int(scene.planes.shape[0])
        desc.planes = d(scene.planes.reshape(-1) if desc.n_planes else np.zeros(4))
        desc.contact_compliance = float(scene.contact_compliance)
        desc.contacts = int(bool(scene.contacts))
        desc.volume = int(bool(scene.volume))
        desc.surface_bending = int(bool(getattr(scene, "surface_bending", False)))
        desc.jacobi = int(bool(getattr(scene, "jacobi", False)))
        desc.volume_vector = int(bool(getattr(scene, "volume_vector", False)))
        desc.warm_start = int(bool(getattr(scene, "warm_start", False)))
        if getattr(scene, "bundle_offsets", None) is not None and len(scene.bundle_offsets) > 1:
            desc.n_bundles = len(scene.bundle_offsets) - 1
            desc.bundle_offsets = i(scene.bundle_offsets)
            desc.bundle_rods = i(scene.bundle_rods)
        h = L.vo_create(C.byref(desc))
        if not h:
            raise ValueError("vo_create rejected the scene")
        self._h = h
        if threads != 1 and L.vo_set_threads(h, int(threads)) != 0:
            raise ValueError("vo_set_threads rejected the thread count")
        self.n_rods, self.nv, self.ns = scene.n_rods, scene.nv, scene.ns
        self.t = 0.0
        if scene.init_pos is not None or scene.init_quat is not None:
            self.set_state(x=scene.init_pos, q=scene.init_quat)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().vo_destroy(h)
            self._h = None

    def set_state(self, x=None, s=None, v=None, sdot=None, q=None, w=None):
        arrs = []
        ptrs = []
        for a in (x, s, v, sdot, q, w):
            if a is None:
                ptrs.append(None)
            else:
                arr, p = _d(np.asarray(a).reshape(-1))
                arrs.append(arr)
                ptrs.append(p)
        lib().vo_set_state(self._h, *ptrs)

    def get_state(self):
        x = np.zeros((self.nv, 3)); s = np.zeros(self.nv); v = np.zeros((self.nv, 3))
        sd = np.zeros(self.nv); q = np.zeros((self.ns, 4)); w = np.zeros((self.ns, 3))
        lib().vo_get_state(self._h, *[_d(a)[1] for a in (x, s, v, sd, q, w)])
        return {"x": x, "s": s, "v": v, "sdot": sd, "q": q, "w": w}

    def set_bones(self, quat, trans):
        qa, qp = _d(np.asarray(quat).reshape(-1))
        ta, tp = _d(np.asarray(trans).reshape(-1))
        lib().vo_set_bones(self._h, qp, tp)

    def step(self, dt=None, substeps=None, iterations=None):
        sc = self.scene
        dt = sc.dt if dt is None else dt
        substeps = sc.substeps if substeps is None else substeps
        iterations = sc.iterations if iterations is None else iterations
        rc = lib().vo_step(self._h, float(dt), int(substeps), int(iterations))
        self.t += dt
        return rc

    def frame(self):
        """One frame of the scene's own schedule, bones set to their pose at the frame end."""
        sc = self.scene
        if sc.bones is not None:
            self.set_bones(*sc.bone_pose(self.t + sc.dt))
        return self.step()

    def skin(self, mesh=None):
        mesh = mesh if mesh is not None else self.scene.mesh
        out = np.zeros((mesh.n, 3))
        ra, rp = _d(mesh.rest.reshape(-1))
        ia, ip = _i(mesh.idx.reshape(-1))
        wa, wp = _d(mesh.w.reshape(-1))
        rc = lib().vo_skin(self._h, mesh.n, rp, ip, wp, _d(out)[1])
        if rc != 0:
            raise ValueError("vo_skin: bad frame index")
        return out

    def last_pairs(self):
        n = lib().vo_last_pairs(self._h, None, 0)
        out = np.zeros((max(n, 1), 2), np.int32)
        lib().vo_last_pairs(self._h, out.ctypes.data_as(_ip), n)
        return out[:n]

    def segment_compliance(self, g):
        out = np.zeros(4)
        if lib().vo_segment_compliance(self._h, int(g), _d(out)[1]) != 0:
            raise IndexError(g)
        return out

    def vertex_compliance(self, i):
        out = np.zeros(4)
        if lib().vo_vertex_compliance(self._h, int(i), _d(out)[1]) != 0:
            raise IndexError(i)
        return out

    def vertex_inverse_inertia(self, i):
        a = np.zeros(1); b = np.zeros(1)
        lib().vo_vertex_inverse_inertia(self._h, int(i), _d(a)[1], _d(b)[1])
        return float(a[0]), float(b[0])

    def rest(self):
        lb = np.zeros(self.ns); ob = np.zeros((self.nv, 3))
        lib().vo_rest(self._h, _d(lb)[1], _d(ob)[1])
        return lb, ob

    def colouring(self):
        sc = np.zeros(self.ns, np.int32); vc = np.zeros(self.nv, np.int32)
        lib().vo_colouring(self._h, sc.ctypes.data_as(_ip), vc.ctypes.data_as(_ip))
        return sc, vc

    def set_activation(self, a=None):
        """Muscle activation per rod in [0, 0.9] (None: back to rest)."""
        if a is None:
            rc = lib().vo_set_activation(self._h, None)
        else:
            arr = np.ascontiguousarray(a, dtype=np.float64)
            rc = lib().vo_set_activation(self._h, arr.ctypes.data_as(_dp))
        if rc != 0:
            raise ValueError("activation outside [0, 0.9]")

    def shape_match(self):
        """Apply the bundles' shape matching (Sec. 7.3) to the current state once."""
        lib().vo_shape_match(self._h)

    def laplacian_compliance(self, i):
        return float(lib().vo_laplacian_compliance(self._h, int(i)))

    def constraint_rms(self):
        out = np.zeros(6)
        lib().vo_constraint_rms(self._h, _d(out)[1])
        return dict(zip(["S", "V", "X", "G", "B", "Vb"], out))


def polar_rotation(A):
    """The rotation maximising trace(R^T A) (3x3, row-major)."""
    a = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    r = np.zeros(9)
    lib().vo_polar_rotation(_d(a)[1], _d(r)[1])
    return r.reshape(3, 3)


def laplacian_constraint(s_prev, s, s_next, la, lb):
    """Surface-bending constraint value and its three scale Jacobian entries."""
    c = np.zeros(1)
    j = np.zeros(3)
    lib().vo_laplacian_constraint(float(s_prev), float(s), float(s_next), float(la), float(lb), _d(c)[1],
                                  _d(j)[1])
    return float(c[0]), j


def broadphase_f32(rod_offsets, group, x4, rbar, brute=False):
    """Candidate pairs on FP32 (x, y, z, scale) vertex states; sorted (a, b), a < b."""
    L = lib()
    off, op = _i(rod_offsets)
    grp, gp = _i(group)
    x4 = np.ascontiguousarray(x4, dtype=np.float32).reshape(-1)
    rb = np.ascontiguousarray(rbar, dtype=np.float32)
    xp = x4.ctypes.data_as(_fp)
    rp = rb.ctypes.data_as(_fp)
    n = L.vo_broadphase_f32(len(off) - 1, op, gp, xp, rp, int(brute), None, 0)
    out = np.zeros((max(n, 1), 2), np.int32)
    L.vo_broadphase_f32(len(off) - 1, op, gp, xp, rp, int(brute), out.ctypes.data_as(_ip), n)
    return out[:n]


def pill_project(c1, r1, c2, r2, x):
    return lib().vo_pill_project(_d(c1)[1], float(r1), _d(c2)[1], float(r2), _d(x)[1])


def narrowphase(a1, ra1, a2, ra2, b1, rb1, b2, rb2):
    al = np.zeros(1); be = np.zeros(1); c = np.zeros(1)
    lib().vo_narrowphase(_d(a1)[1], float(ra1), _d(a2)[1], float(ra2), _d(b1)[1], float(rb1),
                         _d(b2)[1], float(rb2), _d(al)[1], _d(be)[1], _d(c)[1])
    return float(al[0]), float(be[0]), float(c[0])


def segment_constraint(kind, xa, xb, sa, sb, q, lbar):
    """kind 0 S, 1 V, 2 X, 3 G, 4 V in the printed vector form."""
    rows = 3 if kind in (0, 4) else 1
    Cv = np.zeros(rows); Jxa = np.zeros((rows, 3)); Jxb = np.zeros((rows, 3))
    Jsa = np.zeros(rows); Jsb = np.zeros(rows); Jth = np.zeros((rows, 3))
    args = [_d(a)[1] for a in (Cv, Jxa, Jxb, Jsa, Jsb, Jth)]
    xa_, xb_, q_ = _d(xa), _d(xb), _d(q)
    lib().vo_segment_constraint(int(kind), xa_[1], xb_[1], float(sa), float(sb), q_[1], float(lbar), *args)
    return {"C": Cv, "Jxa": Jxa, "Jxb": Jxb, "Jsa": Jsa, "Jsb": Jsb, "Jth": Jth}


def vertex_constraint(kind, qa, qb, s, la, lb, obar):
    rows = 3 if kind == 0 else 2
    Cv = np.zeros(rows); Ja = np.zeros((rows, 3)); Jb = np.zeros((rows, 3)); Js = np.zeros(rows)
    qa_, qb_, ob_ = _d(qa), _d(qb), _d(obar)
    lib().vo_vertex_constraint(int(kind), qa_[1], qb_[1], float(s), float(la), float(lb), ob_[1],
                               _d(Cv)[1], _d(Ja)[1], _d(Jb)[1], _d(Js)[1])
    return {"C": Cv, "Jtha": Ja, "Jthb": Jb, "Js": Js}
