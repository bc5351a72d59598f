"""Seeded synthetic scene generators for the VIPER rod solver.

This module produces *inputs only*: rest geometry, per-rod material parameters,
pin attachments, bone animation tracks, half-planes and skinning meshes.  It holds
none of the solver's arithmetic (no masses, inertias, compliances, constraint
values or integration): both the CUDA path and the CPU oracle derive those
independently from the same scene description.

The paper's own scenes (an octopus rig and Ziva muscle assets, Sec. 7 and
Sec. 8) are not available, so these generators stand in for them with the
shapes, sizes and value distributions of the five workloads this library is
measured on:

* ``plain_small``   16 rods x 32 vertices hanging from a pinned vertex.
* ``muscle_rig``    tapered rods pinned at both ends to animated bones, with
                    pill-pill contacts and a linear-blend-skinned surface.
* ``batching``      4096 rods of log-uniform 4..256 vertices with random bends.
* ``hair``          20,000 radial strands falling into a box of half-planes.
* serving mixes     many independent muscle rigs of log-uniform size.

Conventions: quaternions are stored (x, y, z, w) (Hamilton product); the rod
material frame's third axis d3 = R(q) e_z is the rod tangent; rods are given as
a vertex CSR ``rod_offsets``; segment j of rod r joins its local vertices j and
j+1 and has global index ``rod_offsets[r] - r + j``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

GRAVITY = np.array([0.0, -9.81, 0.0])


@dataclasses.dataclass
class Mesh:
    """Skinning mesh: rest positions, 4 segment-frame ids and 4 weights per vertex."""
    rest: np.ndarray      # float64 [m, 3]
    idx: np.ndarray       # int32  [m, 4]  global segment ids
    w: np.ndarray         # float64 [m, 4] normalised weights

    @property
    def n(self) -> int:
        return int(self.rest.shape[0])


@dataclasses.dataclass
class BoneTrack:
    """Smooth random bone rotations: per bone, per axis, a sum of 3 sinusoids.

    The rotation vector of bone b at time t is
    theta_c(t) = sum_m A[b,c,m] * (sin(omega[b,c,m] * t + phi[b,c,m]) - sin(phi[b,c,m])),
    (zero at t = 0, so the rig starts in its rest pose) and the bone rotates
    about its own origin ``trans0[b]``.
    """
    quat0: np.ndarray     # [nb, 4] rest orientation
    trans0: np.ndarray    # [nb, 3] rest origin
    amp: np.ndarray       # [nb, 3, 3]
    omega: np.ndarray     # [nb, 3, 3]
    phase: np.ndarray     # [nb, 3, 3]

    @property
    def n(self) -> int:
        return int(self.quat0.shape[0])

    def pose(self, t: float):
        """Bone orientations (x,y,z,w) and origins at time ``t``."""
        theta = (self.amp * (np.sin(self.omega * t + self.phase) - np.sin(self.phase))).sum(axis=2)
        dq = axis_angle_quat(theta)
        q = quat_mul(dq, self.quat0)
        return q, self.trans0.copy()


@dataclasses.dataclass
class Scene:
    name: str
    rod_offsets: np.ndarray           # int32 [n_rods+1]
    rest_pos: np.ndarray              # float64 [nv, 3]
    rest_quat: np.ndarray             # float64 [ns, 4]
    radius: np.ndarray                # float64 [nv] rest radius r(z) of the disc
    density: np.ndarray               # float64 [n_rods] kg/m^3
    c_stretch: np.ndarray             # float64 [n_rods] stretch/shear compliance (1/Pa)
    c_bend: np.ndarray                # float64 [n_rods] bend/twist compliance (1/Pa)
    c_volume: np.ndarray              # float64 [n_rods] volume compliance (1/Pa)
    group: np.ndarray                 # int32 [n_rods] collision group
    gravity: np.ndarray               # [3]
    pin_vertex: np.ndarray            # int32 [n_pins]
    pin_bone: np.ndarray              # int32 [n_pins] (-1: fixed in world)
    pin_offset: np.ndarray            # float64 [n_pins, 3] offset in the bone frame
    bones: Optional[BoneTrack]
    planes: np.ndarray                # float64 [n_planes, 4] (n, d): n.x - d - radius >= 0
    contact_compliance: float
    contacts: bool
    volume: bool
    dt: float
    substeps: int
    iterations: int
    frames: int
    init_pos: Optional[np.ndarray] = None
    init_quat: Optional[np.ndarray] = None
    mesh: Optional[Mesh] = None
    surface_bending: bool = False     # scale-Laplacian constraints (Sec. 5, E_bending)
    jacobi: bool = False              # rod constraints by Jacobi with averaging (Sec. 7 engine)
    volume_vector: bool = False       # volume constraint in the printed vector form (Sec. 5)
    warm_start: bool = False          # bone-driven LBS initialisation per frame (Sec. 8.2)
    bundle_offsets: Optional[np.ndarray] = None  # int32 [n_bundles+1] CSR into bundle_rods (Sec. 7.3)
    bundle_rods: Optional[np.ndarray] = None     # int32 rods of each bundle (equal vertex counts)

    @property
    def n_rods(self) -> int:
        return int(self.rod_offsets.shape[0] - 1)

    @property
    def nv(self) -> int:
        return int(self.rod_offsets[-1])

    @property
    def ns(self) -> int:
        return self.nv - self.n_rods

    def rod_lengths(self) -> np.ndarray:
        return np.diff(self.rod_offsets)

    def bone_pose(self, t: float):
        if self.bones is None:
            return np.zeros((0, 4)), np.zeros((0, 3))
        return self.bones.pose(t)

    def subset(self, rods) -> "Scene":
        """Scene holding only the listed rods (no contacts between rods needed).

        Used to step a sample of an independent-rod workload on the oracle.
        Pins, bones, planes and material parameters of the kept rods are kept;
        the skinning mesh is dropped.
        """
        rods = np.asarray(rods, dtype=np.int64)
        off = self.rod_offsets
        vsel = np.concatenate([np.arange(off[r], off[r + 1]) for r in rods])
        ssel = np.concatenate([np.arange(off[r] - r, off[r + 1] - r - 1) for r in rods])
        lens = off[rods + 1] - off[rods]
        new_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        vmap = -np.ones(self.nv, dtype=np.int64)
        vmap[vsel] = np.arange(vsel.size)
        keep = vmap[self.pin_vertex] >= 0
        return dataclasses.replace(
            self,
            name=self.name + "_subset",
            rod_offsets=new_off,
            rest_pos=self.rest_pos[vsel].copy(),
            rest_quat=self.rest_quat[ssel].copy(),
            radius=self.radius[vsel].copy(),
            density=self.density[rods].copy(),
            c_stretch=self.c_stretch[rods].copy(),
            c_bend=self.c_bend[rods].copy(),
            c_volume=self.c_volume[rods].copy(),
            group=self.group[rods].copy(),
            pin_vertex=vmap[self.pin_vertex[keep]].astype(np.int32),
            pin_bone=self.pin_bone[keep].copy(),
            pin_offset=self.pin_offset[keep].copy(),
            init_pos=None if self.init_pos is None else self.init_pos[vsel].copy(),
            init_quat=None if self.init_quat is None else self.init_quat[ssel].copy(),
            mesh=None,
        )


# ----------------------------------------------------------------------------
# quaternion helpers used to *build* input geometry (not by the solver)
# ----------------------------------------------------------------------------

def quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    ax, ay, az, aw = np.moveaxis(a, -1, 0)
    bx, by, bz, bw = np.moveaxis(b, -1, 0)
    return np.stack([
        aw * bx + bw * ax + ay * bz - az * by,
        aw * by + bw * ay + az * bx - ax * bz,
        aw * bz + bw * az + ax * by - ay * bx,
        aw * bw - ax * bx - ay * by - az * bz,
    ], axis=-1)


def axis_angle_quat(v: np.ndarray) -> np.ndarray:
    """Quaternion of the rotation by |v| about v/|v| (v: [..., 3])."""
    ang = np.linalg.norm(v, axis=-1, keepdims=True)
    half = 0.5 * ang
    with np.errstate(invalid="ignore", divide="ignore"):
        k = np.where(ang > 1e-300, np.sin(half) / np.where(ang > 1e-300, ang, 1.0), 0.5)
    return np.concatenate([v * k, np.cos(half)], axis=-1)


def quat_rotate(q: np.ndarray, v: np.ndarray) -> np.ndarray:
    qv = q[..., :3]
    w = q[..., 3:4]
    t = 2.0 * np.cross(qv, v)
    return v + w * t + np.cross(qv, t)


def quat_from_z(t: np.ndarray) -> np.ndarray:
    """Minimal rotation taking e_z to the unit vectors t ([..., 3])."""
    t = t / np.linalg.norm(t, axis=-1, keepdims=True)
    ez = np.zeros_like(t)
    ez[..., 2] = 1.0
    c = np.cross(ez, t)
    w = 1.0 + t[..., 2]
    q = np.concatenate([c, w[..., None]], axis=-1)
    bad = w < 1e-9
    q[bad] = np.array([1.0, 0.0, 0.0, 0.0])
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


def _perp_basis(t: np.ndarray):
    """Two unit vectors orthogonal to unit t (arrays [..., 3])."""
    a = np.where(np.abs(t[..., :1]) < 0.9, np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]))
    u = np.cross(t, a)
    u /= np.linalg.norm(u, axis=-1, keepdims=True)
    v = np.cross(t, u)
    return u, v


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _empty_pins():
    return (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros((0, 3)))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def plain_small(seed: int = 0, n_rods: int = 16, n_verts: int = 32, seg_len: float = 0.01,
                frames: int = 100) -> Scene:
    """16 rods x 32 vertices straight along +x, vertex 0 pinned, under gravity.

    Radius uniform [0.02, 0.05] m per rod, density 1000 kg/m^3, stretch/shear and
    bend/twist compliances log-uniform [1e-8, 1e-5] 1/Pa, volume constraint on,
    dt = 1/60 s, 10 substeps x 4 iterations.
    """
    rng = np.random.default_rng(seed)
    off = np.arange(n_rods + 1, dtype=np.int32) * n_verts
    nv = n_rods * n_verts
    pos = np.zeros((nv, 3))
    rad = np.zeros(nv)
    r_rod = rng.uniform(0.02, 0.05, n_rods)
    for r in range(n_rods):
        sl = slice(off[r], off[r + 1])
        pos[sl, 0] = np.arange(n_verts) * seg_len
        pos[sl, 2] = 0.15 * r
        rad[sl] = r_rod[r]
    ns = nv - n_rods
    quat = np.tile(quat_from_z(np.array([1.0, 0.0, 0.0])), (ns, 1))
    cs = _log_uniform(rng, 1e-8, 1e-5, n_rods)
    cb = _log_uniform(rng, 1e-8, 1e-5, n_rods)
    pin_v = off[:-1].astype(np.int32)
    return Scene(
        name="plain_small", rod_offsets=off, rest_pos=pos, rest_quat=quat, radius=rad,
        density=np.full(n_rods, 1000.0), c_stretch=cs, c_bend=cb, c_volume=cs.copy(),
        group=np.arange(n_rods, dtype=np.int32), gravity=GRAVITY.copy(),
        pin_vertex=pin_v, pin_bone=np.full(n_rods, -1, np.int32), pin_offset=pos[pin_v].copy(),
        bones=None, planes=np.zeros((0, 4)), contact_compliance=1e-9, contacts=False,
        volume=True, dt=1.0 / 60.0, substeps=10, iterations=4, frames=frames)


def _bone_track(rng, n_bones: int, spacing: float, max_rate_deg: float = 30.0) -> BoneTrack:
    trans0 = np.zeros((n_bones, 3))
    trans0[:, 0] = spacing * np.arange(n_bones)
    quat0 = np.tile(np.array([0.0, 0.0, 0.0, 1.0]), (n_bones, 1))
    omega = rng.uniform(0.5, 3.0, (n_bones, 3, 3))
    # |d theta/dt| <= sum_m A*omega per axis; keep the vector rate below the cap
    cap = math.radians(max_rate_deg) / math.sqrt(3.0) / 3.0
    amp = cap / omega * rng.uniform(0.5, 1.0, (n_bones, 3, 3))
    phase = rng.uniform(0.0, 2.0 * math.pi, (n_bones, 3, 3))
    return BoneTrack(quat0=quat0, trans0=trans0, amp=amp, omega=omega, phase=phase)


def _pill_surface_mesh(rng, off, pos, rad, n_mesh: int, rods=None) -> Mesh:
    """Points on the rest pill surfaces; frames j-1..j+2 (clamped) with Dirichlet(1) weights."""
    n_rods = off.shape[0] - 1
    lens = np.diff(off)
    if rods is None:
        rods = np.arange(n_rods)
    r_of = rng.choice(rods, n_mesh)
    nseg = lens[r_of] - 1
    j = (rng.random(n_mesh) * nseg).astype(np.int64)
    t = rng.random(n_mesh)
    v0 = off[r_of] + j
    a = pos[v0]
    b = pos[v0 + 1]
    c = a + t[:, None] * (b - a)
    rr = (1 - t) * rad[v0] + t * rad[v0 + 1]
    tang = (b - a) / np.linalg.norm(b - a, axis=1, keepdims=True)
    u, v = _perp_basis(tang)
    phi = rng.uniform(0, 2 * math.pi, n_mesh)
    p = c + rr[:, None] * (np.cos(phi)[:, None] * u + np.sin(phi)[:, None] * v)
    seg0 = off[r_of] - r_of  # first global segment id of the rod
    loc = np.clip(j[:, None] + np.arange(-1, 3)[None, :], 0, nseg[:, None] - 1)
    idx = (seg0[:, None] + loc).astype(np.int32)
    w = rng.dirichlet(np.ones(4), n_mesh)
    return Mesh(rest=p, idx=idx, w=w)


def muscle_rig(seed: int = 1, n_rods: int = 200, mesh_verts: int = 200_000, n_bones: int = 20,
               nmin: int = 8, nmax: int = 64, frames: int = 600) -> Scene:
    """Tapered rods pinned at both ends to animated bones, contacts and LBS on.

    Bones sit 0.3 m apart on the x axis and rotate about their origins with
    seeded smooth random rotations (<= 30 deg/s).  Rod k spans bone b_k -> b_k+1
    (b_k uniform); its attachment offsets form a y-z grid per bone gap with
    0.13 m spacing so that no two rods overlap at rest.  Vertex counts are
    uniform integers in [nmin, nmax]; the radius profile is
    r(t) = r0 (0.5 + sin(pi t)), r0 uniform [0.01, 0.04] m.
    """
    rng = np.random.default_rng(seed)
    spacing = 0.3
    bones = _bone_track(rng, n_bones, spacing)
    nvert = rng.integers(nmin, nmax + 1, n_rods)
    gap = rng.integers(0, n_bones - 1, n_rods)
    r0 = rng.uniform(0.01, 0.04, n_rods)
    off = np.concatenate([[0], np.cumsum(nvert)]).astype(np.int32)
    nv = int(off[-1])
    pos = np.zeros((nv, 3))
    rad = np.zeros(nv)
    slot_in_gap = np.zeros(n_rods, np.int64)
    counts = np.zeros(n_bones, np.int64)
    for k in range(n_rods):
        slot_in_gap[k] = counts[gap[k]]
        counts[gap[k]] += 1
    pin_v, pin_b, pin_o = [], [], []
    for k in range(n_rods):
        s = slot_in_gap[k]
        y = (s // 4 - 2) * 0.13
        z = (s % 4 - 1.5) * 0.13
        start_local = np.array([0.04, y, z])
        end_local = np.array([-0.04, y, z])
        A = bones.trans0[gap[k]] + start_local
        B = bones.trans0[gap[k] + 1] + end_local
        t = np.linspace(0.0, 1.0, nvert[k])
        sl = slice(off[k], off[k + 1])
        pos[sl] = A[None, :] + t[:, None] * (B - A)[None, :]
        rad[sl] = r0[k] * (0.5 + np.sin(math.pi * t))
        pin_v += [off[k], off[k + 1] - 1]
        pin_b += [gap[k], gap[k] + 1]
        pin_o += [start_local, end_local]
    ns = nv - n_rods
    quat = np.tile(quat_from_z(np.array([1.0, 0.0, 0.0])), (ns, 1))
    cs = _log_uniform(rng, 1e-8, 1e-5, n_rods)
    cb = _log_uniform(rng, 1e-8, 1e-5, n_rods)
    mesh = _pill_surface_mesh(rng, off, pos, rad, mesh_verts) if mesh_verts > 0 else None
    return Scene(
        name="muscle_rig", rod_offsets=off, rest_pos=pos, rest_quat=quat, radius=rad,
        density=np.full(n_rods, 1000.0), c_stretch=cs, c_bend=cb, c_volume=cs.copy(),
        group=np.arange(n_rods, dtype=np.int32), gravity=GRAVITY.copy(),
        pin_vertex=np.array(pin_v, np.int32), pin_bone=np.array(pin_b, np.int32),
        pin_offset=np.array(pin_o), bones=bones, planes=np.zeros((0, 4)),
        contact_compliance=1e-9, contacts=True, volume=True, dt=1.0 / 60.0, substeps=10,
        iterations=4, frames=frames, mesh=mesh)


def bundled_muscles(seed: int = 6, n_muscles: int = 24, fibers: int = 7, n_verts: int = 16, n_bones: int = 8,
                    frames: int = 300) -> Scene:
    """Muscles made of bundled fibre rods (Sec. 7.3, Sec. 8.2 muscles).

    Bones as in muscle_rig.  Each muscle spans a random bone gap and holds
    `fibers` rods of `n_verts` vertices in a hexagonal pattern (one central
    fibre, the others 22 mm around it) whose ends are pinned to the two bones;
    radius profile r(t) = r0 (0.5 + sin(pi t)), r0 = 8 mm.  The fibres of a
    muscle form one bundle (one shape-matching cross-section per vertex index)
    and one collision group (no intra-muscle contacts); muscles collide with
    each other.  Stretch / bend compliances log-uniform [1e-8, 1e-5] per muscle.
    """
    rng = np.random.default_rng(seed)
    spacing = 0.3
    bones = _bone_track(rng, n_bones, spacing)
    gap = rng.integers(0, n_bones - 1, n_muscles)
    n_rods = n_muscles * fibers
    off = (np.arange(n_rods + 1) * n_verts).astype(np.int32)
    nv = int(off[-1])
    pos = np.zeros((nv, 3))
    rad = np.zeros(nv)
    ring = [np.zeros(2)] + [0.022 * np.array([math.cos(a), math.sin(a)])
                            for a in np.arange(fibers - 1) * 2 * math.pi / max(fibers - 1, 1)]
    counts = np.zeros(n_bones, np.int64)
    pin_v, pin_b, pin_o = [], [], []
    group = np.zeros(n_rods, np.int32)
    cs_m = _log_uniform(rng, 1e-8, 1e-5, n_muscles)
    cb_m = _log_uniform(rng, 1e-8, 1e-5, n_muscles)
    t = np.linspace(0.0, 1.0, n_verts)
    for m in range(n_muscles):
        s = counts[gap[m]]
        counts[gap[m]] += 1
        y0 = (s // 4 - 2) * 0.13
        z0 = (s % 4 - 1.5) * 0.13
        for f in range(fibers):
            k = m * fibers + f
            oyz = ring[f]
            start_local = np.array([0.04, y0 + oyz[0], z0 + oyz[1]])
            end_local = np.array([-0.04, y0 + oyz[0], z0 + oyz[1]])
            A = bones.trans0[gap[m]] + start_local
            B = bones.trans0[gap[m] + 1] + end_local
            sl = slice(off[k], off[k + 1])
            pos[sl] = A[None, :] + t[:, None] * (B - A)[None, :]
            rad[sl] = 0.008 * (0.5 + np.sin(math.pi * t))
            pin_v += [off[k], off[k + 1] - 1]
            pin_b += [gap[m], gap[m] + 1]
            pin_o += [start_local, end_local]
            group[k] = m
    ns = nv - n_rods
    quat = np.tile(quat_from_z(np.array([1.0, 0.0, 0.0])), (ns, 1))
    cs = np.repeat(cs_m, fibers)
    cb = np.repeat(cb_m, fibers)
    return Scene(
        name="bundled_muscles", rod_offsets=off, rest_pos=pos, rest_quat=quat, radius=rad,
        density=np.full(n_rods, 1000.0), c_stretch=cs, c_bend=cb, c_volume=cs.copy(), group=group,
        gravity=GRAVITY.copy(), pin_vertex=np.array(pin_v, np.int32), pin_bone=np.array(pin_b, np.int32),
        pin_offset=np.array(pin_o), bones=bones, planes=np.zeros((0, 4)), contact_compliance=1e-9,
        contacts=True, volume=True, dt=1.0 / 60.0, substeps=10, iterations=4, frames=frames,
        bundle_offsets=(np.arange(n_muscles + 1) * fibers).astype(np.int32),
        bundle_rods=np.arange(n_rods, dtype=np.int32))


def batching(seed: int = 2, n_rods: int = 4096, nmin: int = 4, nmax: int = 256,
             seg_len: float = 0.01, frames: int = 300) -> Scene:
    """Independent rods of log-uniform 4..256 vertices with random initial bends.

    Rest shape straight along +x; the initial state rotates each segment by a
    uniform angle in [-45, 45] deg about a random axis orthogonal to the rest
    tangent (positions follow the bent frames).  Vertex 0 is pinned, gravity on,
    radius uniform [0.005, 0.02] m per rod, 20 substeps x 8 iterations.
    """
    rng = np.random.default_rng(seed)
    nvert = np.clip(np.rint(_log_uniform(rng, nmin, nmax, n_rods)), nmin, nmax).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(nvert)]).astype(np.int32)
    nv = int(off[-1])
    ns = nv - n_rods
    side = int(math.ceil(math.sqrt(n_rods)))
    pos = np.zeros((nv, 3))
    ipos = np.zeros((nv, 3))
    rad = np.zeros(nv)
    q_rest = quat_from_z(np.array([1.0, 0.0, 0.0]))
    quat = np.tile(q_rest, (ns, 1))
    iquat = np.zeros((ns, 4))
    r_rod = rng.uniform(0.005, 0.02, n_rods)
    for k in range(n_rods):
        n = int(nvert[k])
        root = np.array([0.0, 0.1 * (k // side), 0.1 * (k % side)])
        sl = slice(off[k], off[k + 1])
        pos[sl] = root[None, :] + np.arange(n)[:, None] * np.array([seg_len, 0.0, 0.0])[None, :]
        rad[sl] = r_rod[k]
        ang = np.radians(rng.uniform(-45.0, 45.0, n - 1))
        phi = rng.uniform(0.0, 2 * math.pi, n - 1)
        axis = np.stack([np.zeros(n - 1), np.cos(phi), np.sin(phi)], axis=1)  # orthogonal to +x
        qs = quat_mul(axis_angle_quat(axis * ang[:, None]), np.tile(q_rest, (n - 1, 1)))
        s0 = off[k] - k
        iquat[s0:s0 + n - 1] = qs
        d3 = quat_rotate(qs, np.tile(np.array([0.0, 0.0, 1.0]), (n - 1, 1)))
        p = np.zeros((n, 3))
        p[0] = root
        p[1:] = root[None, :] + np.cumsum(seg_len * d3, axis=0)
        ipos[sl] = p
    cs = _log_uniform(rng, 1e-8, 1e-5, n_rods)
    cb = _log_uniform(rng, 1e-8, 1e-5, n_rods)
    pin_v = off[:-1].astype(np.int32)
    return Scene(
        name="batching", rod_offsets=off, rest_pos=pos, rest_quat=quat, radius=rad,
        density=np.full(n_rods, 1000.0), c_stretch=cs, c_bend=cb, c_volume=cs.copy(),
        group=np.arange(n_rods, dtype=np.int32), gravity=GRAVITY.copy(),
        pin_vertex=pin_v, pin_bone=np.full(n_rods, -1, np.int32), pin_offset=pos[pin_v].copy(),
        bones=None, planes=np.zeros((0, 4)), contact_compliance=1e-9, contacts=False,
        volume=True, dt=1.0 / 60.0, substeps=20, iterations=8, frames=frames,
        init_pos=ipos, init_quat=iquat)


def poisson_sphere(rng, n: int, radius: float, min_dist: float, batch: int = 4096,
                   max_rounds: int = 4000) -> np.ndarray:
    """Dart throwing on a sphere surface: n points at pairwise distance >= min_dist."""
    from scipy.spatial import cKDTree
    pts = np.zeros((0, 3))
    tree = None
    for _ in range(max_rounds):
        c = rng.normal(size=(batch, 3))
        c = radius * c / np.linalg.norm(c, axis=1, keepdims=True)
        if tree is not None:
            d, _ = tree.query(c, k=1)
            c = c[d >= min_dist]
        if c.shape[0] == 0:
            continue
        # greedy acceptance inside the batch, in draw order
        bt = cKDTree(c)
        pairs = bt.query_pairs(min_dist, output_type="ndarray")
        keep = np.ones(c.shape[0], bool)
        if pairs.size:
            nb = [[] for _ in range(c.shape[0])]
            for a, b in pairs:
                nb[max(a, b)].append(min(a, b))
            for i in range(c.shape[0]):
                if keep[i]:
                    for j in nb[i]:
                        if keep[j]:
                            keep[i] = False
                            break
        c = c[keep]
        pts = np.concatenate([pts, c[: n - pts.shape[0]]])
        if pts.shape[0] >= n:
            return pts
        tree = cKDTree(pts)
    raise RuntimeError(f"poisson_sphere: only {pts.shape[0]} of {n} points placed")


def hair(seed: int = 3, n_rods: int = 20_000, n_verts: int = 16, radius: float = 0.002,
         seg_len: float = 0.005, sphere: float = 0.2, box: float = 0.3,
         min_dist: float = 0.004, frames: int = 200) -> Scene:
    """Radial strands rooted at Poisson-disk sites of a sphere, falling into a box.

    Six half-planes bound the box [-box, box]^3; no pins; contacts on with
    contact compliance 1e-9; stretch compliance 1e-8, bend compliance
    log-uniform [1e-7, 1e-5]; 10 substeps x 4 iterations.
    """
    rng = np.random.default_rng(seed)
    roots = poisson_sphere(rng, n_rods, sphere, min_dist)
    normals = roots / np.linalg.norm(roots, axis=1, keepdims=True)
    off = np.arange(n_rods + 1, dtype=np.int32) * n_verts
    nv = int(off[-1])
    pos = (roots[:, None, :] + seg_len * np.arange(n_verts)[None, :, None] * normals[:, None, :]).reshape(nv, 3)
    rad = np.full(nv, radius)
    quat = np.repeat(quat_from_z(normals), n_verts - 1, axis=0)
    planes = np.array([
        [1, 0, 0, -box], [-1, 0, 0, -box],
        [0, 1, 0, -box], [0, -1, 0, -box],
        [0, 0, 1, -box], [0, 0, -1, -box],
    ], dtype=np.float64)
    cb = _log_uniform(rng, 1e-7, 1e-5, n_rods)
    cs = np.full(n_rods, 1e-8)
    p = _empty_pins()
    return Scene(
        name="hair", rod_offsets=off, rest_pos=pos, rest_quat=quat, radius=rad,
        density=np.full(n_rods, 1000.0), c_stretch=cs, c_bend=cb, c_volume=cs.copy(),
        group=np.arange(n_rods, dtype=np.int32), gravity=GRAVITY.copy(),
        pin_vertex=p[0], pin_bone=p[1], pin_offset=p[2], bones=None, planes=planes,
        contact_compliance=1e-9, contacts=True, volume=True, dt=1.0 / 60.0, substeps=10,
        iterations=4, frames=frames)


def serving_mix(seed: int = 4, n_scenes: int = 8, rods_lo: int = 50, rods_hi: int = 500,
                mesh_lo: int = 10_000, mesh_hi: int = 300_000):
    """Independent muscle rigs of log-uniform size (rods 50..500, mesh 10k..300k)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        nr = int(round(_log_uniform(rng, rods_lo, rods_hi, 1)[0]))
        nm = int(round(_log_uniform(rng, mesh_lo, mesh_hi, 1)[0]))
        out.append(muscle_rig(seed=1000 * seed + i, n_rods=nr, mesh_verts=nm, frames=1))
    return out


def poisson_arrivals(seed: int, rate: float, mean_life: float, duration: float):
    """Poisson scene arrivals with exponential lifetimes: list of (t_arrive, t_leave)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append((t, t + rng.exponential(mean_life)))


WORKLOADS = {
    "plain_small": plain_small,
    "muscle_rig": muscle_rig,
    "batching": batching,
    "hair": hair,
    "bundled_muscles": bundled_muscles,
}


def make(name: str, **kw) -> Scene:
    return WORKLOADS[name](**kw)
