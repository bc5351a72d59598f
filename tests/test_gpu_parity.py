"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every test runs both sides on the same seeded synthetic scene.  Float results
are compared with the tolerances stated in parity_util; the candidate-pair set
and the colouring are compared bit for bit (the pair set is recomputed by the
oracle's FP32 predicate on the GPU's own predicted positions, since the two
trajectories legitimately differ at threshold pairs).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1906_05260_gb300 import scenes as S
from parity_util import ANG_TOL, POS_TOL_1, POS_TOL_100, RAD_TOL, assert_parity, errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1906_05260_gb300 import build
    build.build()
    from paper_1906_05260_gb300 import viper
    return viper


def _pair(V, scene, solver, **kw):
    return V.Scene(scene, solver=solver, **kw), oracle.OracleScene(scene)


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_plain_small_one_frame(V, solver):
    sc = S.plain_small()
    g, o = _pair(V, sc, solver)
    g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="plain_small 1 frame")
    print("plain_small 1 frame errors vs FP64:", e)


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_plain_small_100_frames(V, solver):
    sc = S.plain_small()
    g, o = _pair(V, sc, solver)
    for _ in range(100):
        g.frame(); o.frame()
    assert g.sync() == 0
    # Angles: twist about the rod axis drifts as t^2 in FP32 (4e-4 rad after 100
    # frames, 1e-4 after 50).  The FP64 oracle is stable (a 1e-7 rad perturbation
    # stays at 6e-8 rad after 100 frames); the same algorithm compiled with every
    # double as float drifts to 3.2e-4 rad: the rounding of each orientation update
    # becomes an angular-velocity error that the free twist mode integrates.
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_100, rad_tol=RAD_TOL, ang_tol=1e-3,
                      what="plain_small 100 frames")
    print("plain_small 100 frames errors vs FP64:", e)


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_colouring_bit_exact(V, solver):
    sc = S.batching(n_rods=300)
    g, o = _pair(V, sc, solver, resident_max=128 if solver != 2 else 256)
    gs, gv = g.colouring()
    os_, ov = o.colouring()
    np.testing.assert_array_equal(gs, os_)
    np.testing.assert_array_equal(gv, ov)


def _ragged_scene():
    """Rods of 2..9 vertices, around the warp / CTA boundaries, and long rods."""
    lens = [2, 3, 4, 5, 6, 7, 8, 9, 31, 32, 33, 63, 64, 65, 66, 127, 128, 129, 255, 256, 257, 300]
    base = S.batching(n_rods=len(lens))
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    nv = int(off[-1])
    rng = np.random.default_rng(9)
    pos = np.zeros((nv, 3))
    ipos = np.zeros((nv, 3))
    iq = []
    for r, n in enumerate(lens):
        root = np.array([0.0, 0.3 * r, 0.0])
        pos[off[r]:off[r + 1]] = root + np.arange(n)[:, None] * np.array([0.01, 0, 0])
        ang = np.radians(rng.uniform(-30, 30, n - 1))
        phi = rng.uniform(0, 2 * np.pi, n - 1)
        axis = np.stack([np.zeros(n - 1), np.cos(phi), np.sin(phi)], 1)
        qr = S.quat_from_z(np.array([1.0, 0, 0]))
        qs = S.quat_mul(S.axis_angle_quat(axis * ang[:, None]), np.tile(qr, (n - 1, 1)))
        d3 = S.quat_rotate(qs, np.tile([0, 0, 1.0], (n - 1, 1)))
        ipos[off[r]] = root
        ipos[off[r] + 1:off[r + 1]] = root + np.cumsum(0.01 * d3, axis=0)
        iq.append(qs)
    nr = len(lens)
    return dataclasses.replace(
        base, rod_offsets=off, rest_pos=pos, rest_quat=np.tile(S.quat_from_z(np.array([1.0, 0, 0])), (nv - nr, 1)),
        radius=np.repeat(rng.uniform(0.004, 0.02, nr), lens), density=np.full(nr, 1000.0),
        c_stretch=np.exp(rng.uniform(np.log(1e-8), np.log(1e-5), nr)),
        c_bend=np.exp(rng.uniform(np.log(1e-8), np.log(1e-5), nr)), c_volume=np.full(nr, 1e-7),
        group=np.arange(nr, dtype=np.int32), pin_vertex=off[:-1].copy(), pin_bone=np.full(nr, -1, np.int32),
        pin_offset=pos[off[:-1]].copy(), init_pos=ipos, init_quat=np.concatenate(iq), substeps=10, iterations=4)


@pytest.mark.parametrize("solver,warps,resident", [(0, 4, 256), (1, 1, 64), (1, 4, 256), (1, 8, 512), (2, 4, 512),
                                                   (2, 8, 512)],
                         ids=["plain", "b1w-res64", "b4w-res256", "b8w-res512", "frame-4w", "frame-8w"])
def test_ragged_rod_lengths(V, solver, warps, resident):
    sc = _ragged_scene()
    g = V.Scene(sc, solver=solver, block_warps=warps, resident_max=resident)
    o = oracle.OracleScene(sc)
    for _ in range(3):
        g.frame(); o.frame()
    assert g.sync() == 0
    assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="ragged")
    gs, gv = g.colouring()
    os_, ov = o.colouring()
    np.testing.assert_array_equal(gs, os_)
    np.testing.assert_array_equal(gv, ov)


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_muscle_rig_one_frame_with_contacts_and_skinning(V, solver):
    sc = S.muscle_rig()
    g, o = _pair(V, sc, solver)
    for _ in range(2):
        g.frame(); o.frame()
    assert g.sync() == 0
    gst, ost = g.get_state(), o.get_state()
    e = assert_parity(sc, gst, ost, POS_TOL_1, what="muscle_rig")
    print("muscle_rig 2 frames errors vs FP64:", e)
    # skinning: GPU LBS of the GPU state against the oracle's LBS of the same
    # FP32 state (tight), and against the oracle's LBS of its own state
    mesh = V.Mesh(sc.mesh)
    out = g.skin(mesh).cpu().numpy()[:, :3].astype(np.float64)
    o2 = oracle.OracleScene(sc)
    o2.set_state(x=gst["x4"][:, :3], s=gst["x4"][:, 3] / sc.radius, q=gst["q4"])
    ref_same = o2.skin()
    scale = np.abs(sc.mesh.rest).max()
    assert np.abs(out - ref_same).max() < 2e-6 * scale
    ref_own = o.skin()
    assert np.abs(out - ref_own).max() < POS_TOL_1 * 0.3 * 3  # rods are ~0.22 m; frames move by pos error


@pytest.mark.parametrize("solver,n_rods", [(1, 200), (2, 200), (1, 500)], ids=["batched", "frame", "batched-500"])
def test_muscle_rig_pairs_bit_exact(V, solver, n_rods):
    """Candidate pairs of the first five frames against the oracle's FP32 predicate
    on the GPU's predicted state (500 rods, about 18k vertices, take the one-CTA grid
    build's general path; 200 rods its shared-memory path)."""
    sc = S.muscle_rig(n_rods=n_rods, mesh_verts=0)
    g = V.Scene(sc, solver=solver)
    total = 0
    for f in range(5):
        g.frame()
        x4, rb = g.predicted()
        ref = oracle.broadphase_f32(sc.rod_offsets, sc.group, x4, rb)
        got = g.pairs()
        np.testing.assert_array_equal(got, ref)
        total += len(ref)
    assert g.sync() == 0


def test_hair_pairs_bit_exact_first_five_frames(V):
    sc = S.hair()
    g = V.Scene(sc)
    counts = []
    for f in range(5):
        g.frame()
        x4, rb = g.predicted()
        ref = oracle.broadphase_f32(sc.rod_offsets, sc.group, x4, rb)
        got = g.pairs()
        assert got.shape == ref.shape, (got.shape, ref.shape)
        np.testing.assert_array_equal(got, ref)
        counts.append(len(ref))
    assert g.sync() == 0
    print("hair candidate pairs per substep (last substep of frames 0-4):", counts)
    assert min(counts) > 100_000


@pytest.mark.parametrize("solver", [1, 2], ids=["batched", "frame"])
def test_hair_small_one_frame(V, solver):
    sc = S.hair(n_rods=400)
    g, o = _pair(V, sc, solver)
    g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="hair-400")
    print("hair (400 rods) 1 frame errors vs FP64:", e)


def test_batching_full_size_sampled_rods(V):
    sc = S.batching()
    g = V.Scene(sc)
    sample = np.unique(np.concatenate([np.argsort(sc.rod_lengths())[[0, 1, -1, -2]],
                                       np.random.default_rng(0).choice(sc.n_rods, 12, replace=False)]))
    sub = sc.subset(sample)
    o = oracle.OracleScene(sub)
    g.frame(); o.frame()
    assert g.sync() == 0
    gst = g.get_state()
    off = sc.rod_offsets
    vsel = np.concatenate([np.arange(off[r], off[r + 1]) for r in sample])
    ssel = np.concatenate([np.arange(off[r] - r, off[r + 1] - r - 1) for r in sample])
    gsub = {"x4": gst["x4"][vsel], "q4": gst["q4"][ssel]}
    e = assert_parity(sub, gsub, o.get_state(), POS_TOL_1, what="batching sample")
    print("batching (20x8, sampled rods) 1 frame errors vs FP64:", e)


def test_batching_sampled_rods_20_frames(V):
    """20 frames (400 substeps x 8 iterations) of the full batching workload on
    the GPU against the oracle on a sample of its rods (the rods are
    independent: no contacts)."""
    sc = S.batching()
    g = V.Scene(sc)
    sample = np.unique(np.concatenate([np.argsort(sc.rod_lengths())[[0, 1, -1, -2]],
                                       np.random.default_rng(1).choice(sc.n_rods, 12, replace=False)]))
    sub = sc.subset(sample)
    o = oracle.OracleScene(sub)
    for _ in range(20):
        g.frame(); o.frame()
    assert g.sync() == 0
    gst = g.get_state()
    off = sc.rod_offsets
    vsel = np.concatenate([np.arange(off[r], off[r + 1]) for r in sample])
    ssel = np.concatenate([np.arange(off[r] - r, off[r + 1] - r - 1) for r in sample])
    gsub = {"x4": gst["x4"][vsel], "q4": gst["q4"][ssel]}
    # Angles: 20 frames of strongly bent, fast rods amplify perturbations (the FP64
    # oracle moves by 1.2e-5 rad after 20 frames from a 1e-7 rad perturbation), and
    # the FP32 rounding of every orientation update feeds the nearly free twist
    # mode; the plain C oracle run entirely in FP32 drifts the same way.
    e = assert_parity(sub, gsub, o.get_state(), POS_TOL_100, ang_tol=5e-3, what="batching sample, 20 frames")
    print("batching (20x8, sampled rods) 20 frames errors vs FP64:", e)


@pytest.mark.parametrize("solver", [0, 1], ids=["plain", "batched"])
def test_muscle_rig_20_frames_with_contacts(V, solver):
    """20 frames of the muscle rig (bones, pill-pill contacts): the horizon over
    which the oracle's own trajectory stays within 3e-6 of rod length when its
    inputs are rounded to FP32 (later frames of this rig amplify rounding)."""
    import os
    sc = S.muscle_rig(mesh_verts=0)
    g = V.Scene(sc, solver=solver)
    o = oracle.OracleScene(sc, threads=os.cpu_count() or 1)
    for _ in range(20):
        g.frame(); o.frame()
    assert g.sync() == 0
    # angles: the FP32 twist drift of the plain_small 100-frame case, here after 20 frames
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_100, ang_tol=1e-3, what="muscle rig, 20 frames")
    print("muscle_rig 20 frames errors vs FP64:", e)


def test_hair_full_size_one_frame(V):
    """One frame of the full 20,000 x 16 hair scene (2.19 M candidate pairs per
    substep, six half-planes) against the oracle on every host core."""
    import os
    sc = S.hair()
    g = V.Scene(sc, max_pairs=64 * sc.ns)
    o = oracle.OracleScene(sc, threads=os.cpu_count() or 1)
    g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="hair full size, 1 frame")
    print("hair full size 1 frame errors vs FP64:", e)


def test_plain_and_batched_agree_on_batching(V):
    sc = S.batching(n_rods=512)
    a = V.Scene(sc, solver=0)
    b = V.Scene(sc, solver=1)
    for _ in range(3):
        a.frame(); b.frame()
    sa, sb = a.get_state(), b.get_state()
    assert np.abs(sa["x4"] - sb["x4"]).max() < 1e-4
    qa, qb = sa["q4"].astype(np.float64), sb["q4"].astype(np.float64)
    ang = 2 * np.arccos(np.clip(np.abs((qa * qb).sum(1)) / np.linalg.norm(qa, axis=1) / np.linalg.norm(qb, axis=1), 0, 1))
    print("plain vs batched (two FP32 schedules), 3 frames of 20x8: max angle", ang.max(),
          "max |dx|", np.abs(sa["x4"] - sb["x4"]).max())


def test_deterministic_replay(V):
    sc = S.muscle_rig(mesh_verts=0)
    a, b = V.Scene(sc), V.Scene(sc)
    for _ in range(3):
        a.frame(); b.frame()
    sa, sb = a.get_state(), b.get_state()
    scale = np.abs(sa["x4"][:, :3]).max() + 1e-3
    assert np.abs(sa["x4"] - sb["x4"]).max() < 4e-6 * scale
    assert np.abs(sa["q4"] - sb["q4"]).max() < 1e-4


def test_zero_iterations_is_pure_prediction(V):
    sc = dataclasses.replace(S.plain_small(n_rods=2), pin_vertex=np.zeros(0, np.int32),
                             pin_bone=np.zeros(0, np.int32), pin_offset=np.zeros((0, 3)))
    g, o = _pair(V, sc, 1)
    g.step(iterations=0); o.step(iterations=0)
    assert_parity(sc, g.get_state(), o.get_state(), 1e-6, what="iterations=0")


def test_nonfinite_state_is_quarantined(V):
    sc = S.plain_small(n_rods=4)
    g = V.Scene(sc)
    st = g.get_state()
    x4 = st["x4"].copy()
    x4[5, 1] = np.nan
    g.set_state(x4=x4)
    g.step(check=False)
    assert g.sync() == V.ENONFINITE
    assert g.step(check=False) == V.ENONFINITE
    g.set_state(x4=st["x4"], v4=np.zeros_like(st["v4"]), q4=st["q4"], w4=np.zeros_like(st["w4"]))
    assert g.step(check=False) == 0
    assert g.sync() == 0


def test_state_roundtrip_and_host_skinning(V):
    sc = S.muscle_rig(n_rods=20, mesh_verts=3000)
    g = V.Scene(sc)
    g.frame()
    st = g.get_state()
    g.set_state(**{k: st[k] for k in ("x4", "v4", "q4", "w4")})
    st2 = g.get_state()
    for k in ("x4", "v4", "w4"):
        np.testing.assert_allclose(st2[k], st[k], rtol=2e-7, atol=1e-7)
    mesh = V.Mesh(sc.mesh)
    dev = g.skin(mesh).cpu().numpy()
    rest4 = np.zeros((sc.mesh.n, 4), np.float32); rest4[:, :3] = sc.mesh.rest
    host = np.zeros((sc.mesh.n, 4), np.float32)
    g.skin_host(rest4, sc.mesh.idx.astype(np.int32), sc.mesh.w.astype(np.float32), host)
    np.testing.assert_array_equal(dev, host)


def test_host_skinning_beside_frames_and_staging_reuse(V):
    """Host operands are uploaded on a copy stream beside the frame's kernels:
    each call's result (device, pageable host or page-locked host output)
    equals the device-operand path on the same operands, also when a call with
    device output (no sync) is followed at once by a call that refills the
    staging buffer."""
    import ctypes as C
    import torch
    sc = S.muscle_rig(n_rods=20, mesh_verts=3000)
    g = V.Scene(sc)
    n = sc.mesh.n
    rest4 = np.zeros((n, 4), np.float32); rest4[:, :3] = sc.mesh.rest
    idx4 = np.ascontiguousarray(sc.mesh.idx, np.int32)
    rng = np.random.default_rng(5)
    L = V.lib()
    for f in range(4):
        g.frame()  # still running while the next uploads start
        w_a = np.ascontiguousarray(rng.dirichlet(np.ones(4), n), np.float32)
        w_b = np.ascontiguousarray(rng.dirichlet(np.ones(4), n), np.float32)
        dev_out = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
        assert L.viper_skin(g.handle, n, C.c_void_p(rest4.ctypes.data), C.c_void_p(idx4.ctypes.data),
                            C.c_void_p(w_a.ctypes.data), C.c_void_p(dev_out.data_ptr())) == 0
        host = np.zeros((n, 4), np.float32)
        g.skin_host(rest4, idx4, w_b, host)
        # page-locked host output: written by the kernel directly
        pinned = torch.zeros((n, 4), dtype=torch.float32).pin_memory()
        assert L.viper_skin(g.handle, n, C.c_void_p(rest4.ctypes.data), C.c_void_p(idx4.ctypes.data),
                            C.c_void_p(w_b.ctypes.data), C.c_void_p(pinned.data_ptr())) == 0
        assert g.sync() == 0
        ref_a = g.skin(V.Mesh(dataclasses.replace(sc.mesh, w=w_a.astype(np.float64))))
        ref_b = g.skin(V.Mesh(dataclasses.replace(sc.mesh, w=w_b.astype(np.float64))))
        torch.cuda.synchronize()  # the scene stream included
        np.testing.assert_array_equal(dev_out.cpu().numpy(), ref_a.cpu().numpy())
        np.testing.assert_array_equal(host, ref_b.cpu().numpy())
        np.testing.assert_array_equal(pinned.numpy(), host)


def test_autotune_keeps_results(V):
    sc = S.batching(n_rods=256)
    g = V.Scene(sc)
    bw, res = g.autotune()
    assert bw in (1, 2, 4, 8) and res in (64, 128, 256, 512)
    o = oracle.OracleScene(sc)
    g.frame(); o.frame()
    assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="after autotune")


def test_autotune_cache_applies_the_stored_choice(V, tmp_path):
    """autotune_cached times once per GPU and scene, then applies the stored
    (block_warps, resident_max) without timing; the schedule follows it."""
    sc = S.batching(n_rods=128)
    path = str(tmp_path / "tune.json")
    a = V.Scene(sc)
    choice, cached = a.autotune_cached(path)
    assert not cached
    b = V.Scene(sc)
    choice_b, cached_b = b.autotune_cached(path)
    assert cached_b and choice_b == choice
    assert a.schedule() == b.schedule()
    n_items, threads, resident = b.schedule()
    assert n_items >= 1 and threads >= 32 * choice[0] and 0 < resident <= sc.nv


@pytest.mark.parametrize("name", ["muscle_rig", "hair", "plain_small", "batching"])
def test_frame_kernel_equals_graph_path(V, name):
    """The persistent frame kernel runs the same device functions in the same
    order as the graph-replayed launches (contacts summed in fixed point); the
    two agree to FP32 rounding (the compiler may contract multiply-adds
    differently in the two kernels, so not bit for bit)."""
    kw = {"muscle_rig": dict(n_rods=120, mesh_verts=0), "hair": dict(n_rods=600), "plain_small": {},
          "batching": dict(n_rods=300)}[name]
    sc = S.make(name, **kw)
    a = V.Scene(sc, solver=1)
    b = V.Scene(sc, solver=2)
    for _ in range(3):
        a.frame(); b.frame()
    assert a.sync() == 0 and b.sync() == 0
    sa, sb = a.get_state(), b.get_state()
    scale = np.abs(sa["x4"][:, :3]).max() + 1e-3
    assert np.abs(sa["x4"] - sb["x4"]).max() < 4e-6 * scale
    assert np.abs(sa["q4"] - sb["q4"]).max() < 1e-4


# --------------------------------------------------------------------------
# surface bending (scale Laplacian, three extra vertex colours)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_surface_bending_plain_small(V, solver):
    sc = dataclasses.replace(S.plain_small(), surface_bending=True)
    g, o = _pair(V, sc, solver)
    g.frame(); o.frame()
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="surface bending, 1 frame")
    for _ in range(19):
        g.frame(); o.frame()
    assert g.sync() == 0
    e20 = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_100, rad_tol=RAD_TOL, ang_tol=ANG_TOL,
                        what="surface bending, 20 frames")
    print("surface bending plain_small errors vs FP64, 1 / 20 frames:", e, e20)


@pytest.mark.parametrize("solver", [1, 2], ids=["batched", "frame"])
def test_surface_bending_with_contacts(V, solver):
    sc = dataclasses.replace(S.muscle_rig(n_rods=60, mesh_verts=0), surface_bending=True)
    g, o = _pair(V, sc, solver)
    for _ in range(2):
        g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="surface bending, muscle rig")
    print("surface bending muscle_rig 2 frames errors vs FP64:", e)


def test_surface_bending_scale_bump_matches_oracle(V):
    """A sharp scale bump on a free straight rod: the scale profile the GPU
    relaxes to matches the oracle's (radii are what the constraint moves)."""
    sc = dataclasses.replace(S.plain_small(), surface_bending=True, gravity=np.zeros(3))
    g, o = _pair(V, sc, 1)
    st = g.get_state()
    x4 = st["x4"].copy()
    x4[5::32, 3] *= 1.3
    g.set_state(x4=x4)
    o.set_state(s=x4[:, 3].astype(np.float64) / sc.radius)
    for _ in range(3):
        g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, rad_tol=1e-5, what="scale bump")
    print("surface bending scale bump errors vs FP64:", e)


# --------------------------------------------------------------------------
# Jacobi with averaging (Sec. 7 engine) instead of the four colours
# --------------------------------------------------------------------------

@pytest.mark.parametrize("solver", [1, 2], ids=["batched", "frame"])
def test_jacobi_plain_small(V, solver):
    sc = dataclasses.replace(S.plain_small(), jacobi=True)
    g, o = _pair(V, sc, solver)
    g.frame(); o.frame()
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="jacobi, 1 frame")
    for _ in range(19):
        g.frame(); o.frame()
    assert g.sync() == 0
    e20 = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_100, rad_tol=RAD_TOL, ang_tol=ANG_TOL,
                        what="jacobi, 20 frames")
    print("jacobi plain_small errors vs FP64, 1 / 20 frames:", e, e20)


@pytest.mark.parametrize("solver", [1, 2], ids=["batched", "frame"])
def test_jacobi_muscle_rig_with_surface_bending(V, solver):
    sc = dataclasses.replace(S.muscle_rig(n_rods=60, mesh_verts=0), jacobi=True, surface_bending=True)
    g, o = _pair(V, sc, solver)
    for _ in range(2):
        g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="jacobi + surface bending, muscle rig")
    print("jacobi + surface bending muscle_rig 2 frames errors vs FP64:", e)


def test_jacobi_batching_sampled_rods(V):
    """Ragged rods of 4..256 vertices, 20 x 8: a sample of rods against the oracle."""
    sc = dataclasses.replace(S.batching(n_rods=512), jacobi=True)
    g = V.Scene(sc, resident_max=256)
    g.frame()
    assert g.sync() == 0
    rods = np.arange(0, sc.n_rods, 37)
    sub = sc.subset(rods)
    o = oracle.OracleScene(sub)
    o.frame()
    st = g.get_state()
    off = sc.rod_offsets
    vsel = np.concatenate([np.arange(off[r], off[r + 1]) for r in rods])
    ssel = np.concatenate([np.arange(off[r] - r, off[r + 1] - r - 1) for r in rods])
    gs = {"x4": st["x4"][vsel], "q4": st["q4"][ssel]}
    e = assert_parity(sub, gs, o.get_state(), POS_TOL_1, what="jacobi batching sample")
    print("jacobi batching sample errors vs FP64:", e)


def test_jacobi_needs_the_shared_memory_solvers(V):
    sc = dataclasses.replace(S.plain_small(), jacobi=True)
    g = V.Scene(sc)
    assert V.lib().viper_set_solver(g.handle, V.SOLVER_PLAIN, 4, 256) == V.EINVAL
    g.frame()  # the scene keeps its previous solver
    assert g.sync() == 0


# --------------------------------------------------------------------------
# bundles: scale-invariant shape matching (Sec. 7.3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("solver", [0, 1], ids=["plain", "batched"])
def test_bundled_muscles(V, solver):
    sc = S.bundled_muscles(n_muscles=12)
    g, o = _pair(V, sc, solver)
    for _ in range(2):
        g.frame(); o.frame()
    assert g.sync() == 0
    st = g.get_state()
    e = assert_parity(sc, st, o.get_state(), POS_TOL_1, what="bundled muscles, 2 frames")
    print("bundled_muscles 2 frames errors vs FP64:", e)
    # every unpinned cross-section leaves the substep as a similarity of its rest
    n_v = int(sc.rod_offsets[1] - sc.rod_offsets[0])
    worst = 0.0
    for b in range(len(sc.bundle_offsets) - 1):
        rods = sc.bundle_rods[sc.bundle_offsets[b]:sc.bundle_offsets[b + 1]]
        for k in range(1, n_v - 1):
            v = sc.rod_offsets[rods] + k
            x = st["x4"][v, :3].astype(np.float64)
            d = np.linalg.norm(x[:, None] - x[None], axis=2)
            d0 = np.linalg.norm(sc.rest_pos[v][:, None] - sc.rest_pos[v][None], axis=2)
            ratio = d[d0 > 0] / d0[d0 > 0]
            worst = max(worst, float(np.abs(ratio / ratio.mean() - 1).max()))
    print("bundle cross-sections: worst relative deviation from a similarity", worst)
    assert worst < 1e-4


def _turned_free_bundles(deg, seed=11):
    """Free bundled muscles (no pins, bones, gravity or contacts) whose rest
    state, perturbed by 0.5 mm, is turned by `deg` degrees about a random axis
    through its centroid: every cross-section starts far from its rest frame."""
    rng = np.random.default_rng(seed)
    base = S.bundled_muscles(n_muscles=4)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    qr = S.axis_angle_quat(np.radians(deg) * axis)
    c = base.rest_pos.mean(axis=0)
    x = base.rest_pos + rng.normal(scale=5e-4, size=base.rest_pos.shape)
    x = c + S.quat_rotate(np.tile(qr, (base.nv, 1)), x - c)
    q = S.quat_mul(np.tile(qr, (base.ns, 1)), base.rest_quat)
    x = x.astype(np.float32).astype(np.float64)  # both sides start from the same FP32 state
    q = q.astype(np.float32).astype(np.float64)
    return dataclasses.replace(base, gravity=np.zeros(3), pin_vertex=np.zeros(0, np.int32),
                               pin_bone=np.zeros(0, np.int32), pin_offset=np.zeros((0, 3)), bones=None,
                               contacts=False, init_pos=x, init_quat=q)


@pytest.mark.parametrize("deg", [90, 135, 170])
@pytest.mark.parametrize("solver", [0, 1], ids=["plain", "batched"])
def test_bundle_cross_sections_turned_far_from_rest(V, solver, deg):
    """Shape matching (Sec. 7.3) of cross-sections turned 90-170 degrees from
    rest: the GPU's iterative rotation extraction (warm-started from the
    members' frames) against the oracle's exact quaternion solution, and no
    non-convergence reported."""
    sc = _turned_free_bundles(deg)
    g, o = _pair(V, sc, solver)
    g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what=f"bundles turned {deg} deg, 1 frame")
    print(f"bundles turned {deg} deg, 1 frame errors vs FP64:", e)


def test_bundles_in_a_multi_scene_step(V):
    scenes = [S.bundled_muscles(n_muscles=8), S.muscle_rig(seed=1, n_rods=40, mesh_verts=0)]
    a = [V.Scene(sc) for sc in scenes]
    b = [V.Scene(sc) for sc in scenes]
    B = V.Batch()
    for f in range(2):
        B.step(a, [sc.bone_pose((f + 1) * sc.dt) for sc in scenes], None, scenes[0].dt, 10, 4)
    B.synchronize()
    for f in range(2):
        for o, sc in zip(b, scenes):
            o.set_bones(*sc.bone_pose((f + 1) * sc.dt))
            o.step(sc.dt, 10, 4)
    for ga, gb in zip(a, b):
        assert ga.sync() == 0 and gb.sync() == 0
        sa, sb = ga.get_state(), gb.get_state()
        scale = np.abs(sa["x4"][:, :3]).max() + 1e-3
        assert np.abs(sa["x4"] - sb["x4"]).max() < 4e-6 * scale
        assert np.abs(sa["q4"] - sb["q4"]).max() < 1e-4


def test_bundles_refuse_the_frame_solver(V):
    g = V.Scene(S.bundled_muscles(n_muscles=2))
    assert V.lib().viper_set_solver(g.handle, V.SOLVER_FRAME, 4, 256) == V.EINVAL
    g.frame()
    assert g.sync() == 0


# ---------------------------------------------------------------- muscle activation, warm start (Sec. 8.2)

def _activation(sc, seed=3):
    """Per-rod activations in [0, 0.6], multiples of 1/64 (exact in FP32)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 39, sc.n_rods) / 64.0


def _activated(sc, a):
    """The scene with the rest radii the activation gives (for the radius comparison)."""
    rod_of_v = np.repeat(np.arange(sc.n_rods), np.diff(sc.rod_offsets))
    return dataclasses.replace(sc, radius=sc.radius / np.sqrt(1.0 - a[rod_of_v]))


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
@pytest.mark.parametrize("seeds,contacts", [((2, 3), True), ((7, 8), False)], ids=["contacts", "no-contacts"])
def test_activation_matches_oracle(V, solver, seeds, contacts):
    """Activated muscles against the oracle, 3 frames.  With contacts the scene
    is one whose activated (thicker) rods do not start in deep, near-parallel
    overlaps: there the narrowphase's probe comparisons are decided by rounding
    (an FP64 oracle with only those comparisons rounded to FP32 moves by
    3.6e-4 L in a frame on scene 7 with activation 8), so that case runs
    without contacts."""
    sc = dataclasses.replace(S.muscle_rig(seed=seeds[0], n_rods=40, mesh_verts=0), contacts=contacts)
    a = _activation(sc, seeds[1])
    g, o = _pair(V, sc, solver)
    g.set_activation(a)
    o.set_activation(a)
    # rest radii on the device: rbar0 / sqrt(1 - a), rounded once to FP32
    _, rb = g.predicted()
    ref = _activated(sc, a).radius
    assert np.abs(rb - ref).max() <= 1e-6 * ref.max()
    for _ in range(3):
        g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(_activated(sc, a), g.get_state(), o.get_state(), POS_TOL_1,
                      what=f"activated muscle_rig {seeds}, contacts {contacts}, 3 frames")
    print(f"activated muscle_rig {seeds} contacts {contacts}, 3 frames errors vs FP64:", e)


def test_activation_reset_restores_the_rest_tables_bitwise(V):
    sc = S.muscle_rig(seed=2, n_rods=40, mesh_verts=0)
    a, b = V.Scene(sc), V.Scene(sc)
    a.set_activation(_activation(sc))
    a.set_activation(None)
    for _ in range(2):
        a.frame(); b.frame()
    sa, sb = a.get_state(), b.get_state()
    for key in ("x4", "v4", "q4", "w4"):
        np.testing.assert_array_equal(sa[key], sb[key], err_msg=key)
    with pytest.raises(RuntimeError):
        a.set_activation(np.full(sc.n_rods, 0.95, np.float32))


def _jump_scene(warm):
    """One rod between two bones that jump (translate) within a frame, no gravity."""
    sc = dataclasses.replace(S.muscle_rig(seed=1, n_rods=1, n_bones=2, mesh_verts=0), warm_start=warm,
                             gravity=np.zeros(3))
    q0, t0 = sc.bones.pose(0.0)
    return sc, q0, t0 + np.array([[0.05, 0.0, 0.01], [-0.02, 0.03, 0.0]])


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_warm_start_blend_before_the_first_substep(V, solver):
    """Translating bones, one substep without iterations: every vertex moves by
    (1 - t) d0 + t d1 exactly as in the oracle."""
    sc, q0, t1 = _jump_scene(True)
    g, o = _pair(V, sc, solver)
    for x in (g, o):
        x.set_bones(q0, t1)
        x.step(1 / 60, 1, 0)
    assert g.sync() == 0
    xg = g.get_state()["x4"][:, :3].astype(np.float64)
    xo = o.get_state()["x"]
    assert np.abs(xg - xo).max() < 1e-6, np.abs(xg - xo).max()
    assert np.abs(xo - sc.rest_pos).max() > 1e-2  # the blend moved the interior


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_warm_start_muscle_rig_matches_oracle(V, solver):
    sc = dataclasses.replace(S.muscle_rig(seed=2, n_rods=40, mesh_verts=0), warm_start=True)
    a = _activation(sc, 3)
    g, o = _pair(V, sc, solver)
    g.set_activation(a)
    o.set_activation(a)
    for f in range(3):
        g.frame(); o.frame()
        assert g.sync() == 0
        e = assert_parity(_activated(sc, a), g.get_state(), o.get_state(), POS_TOL_1,
                          what=f"warm-started, activated muscle_rig, {f + 1} frames")
    print("warm-started activated muscle_rig 3 frames errors vs FP64:", e)


def test_warm_start_and_activation_in_a_multi_scene_step(V):
    warm = dataclasses.replace(S.muscle_rig(seed=2, n_rods=40, mesh_verts=0), warm_start=True)
    scenes = [warm, S.muscle_rig(seed=1, n_rods=40, mesh_verts=0)]
    act = _activation(warm, 3)
    a = [V.Scene(sc) for sc in scenes]
    b = [V.Scene(sc) for sc in scenes]
    a[0].set_activation(act)
    b[0].set_activation(act)
    B = V.Batch()
    counts = []
    for f in range(2):
        c0 = B.launch_count()
        B.step(a, [sc.bone_pose((f + 1) * sc.dt) for sc in scenes], None, warm.dt, 10, 4)
        counts.append(B.launch_count() - c0)
    B.synchronize()
    # per substep 2 I + 3, velocity update and frame end, one warm-start launch (no mesh: no skinning)
    assert counts == [10 * (2 * 4 + 3) + 2 + 1] * 2, counts
    for f in range(2):
        for o, sc in zip(b, scenes):
            o.set_bones(*sc.bone_pose((f + 1) * sc.dt))
            o.step(sc.dt, 10, 4)
    for ga, gb in zip(a, b):
        assert ga.sync() == 0 and gb.sync() == 0
        sa, sb = ga.get_state(), gb.get_state()
        scale = np.abs(sa["x4"][:, :3]).max() + 1e-3
        assert np.abs(sa["x4"] - sb["x4"]).max() < 4e-6 * scale
        assert np.abs(sa["q4"] - sb["q4"]).max() < 1e-4


# ---------------------------------------------------------------- the printed vector volume form

@pytest.mark.parametrize("frames,tol", [(1, "one"), (100, "hundred")])
def test_vector_volume_plain_small(V, frames, tol):
    sc = dataclasses.replace(S.plain_small(), volume_vector=True)
    g, o = _pair(V, sc, V.SOLVER_AUTO)
    assert g.solver == V.SOLVER_PLAIN
    for _ in range(frames):
        g.frame(); o.frame()
    assert g.sync() == 0
    if frames == 1:
        e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="vector volume, plain_small 1 frame")
    else:
        e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_100, rad_tol=RAD_TOL, ang_tol=1e-3,
                          what="vector volume, plain_small 100 frames")
    print(f"vector volume plain_small {frames} frames errors vs FP64:", e)


def test_vector_volume_muscle_rig(V):
    sc = dataclasses.replace(S.muscle_rig(seed=2, n_rods=40, mesh_verts=0), volume_vector=True)
    g, o = _pair(V, sc, V.SOLVER_AUTO)
    for _ in range(2):
        g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="vector volume, muscle_rig 2 frames")
    print("vector volume muscle_rig 2 frames errors vs FP64:", e)
    # the two forms give different trajectories (shear is resisted by the vector form)
    o2 = oracle.OracleScene(dataclasses.replace(sc, volume_vector=False))
    for _ in range(2):
        o2.frame()
    assert np.abs(o2.get_state()["x"] - o.get_state()["x"]).max() > 1e-6


def test_vector_volume_stays_on_the_plain_solver(V):
    sc = dataclasses.replace(S.muscle_rig(seed=2, n_rods=20, mesh_verts=0), volume_vector=True)
    g = V.Scene(sc)
    for mode in (V.SOLVER_BATCHED, V.SOLVER_FRAME):
        assert V.lib().viper_set_solver(g.handle, mode, 4, 256) == V.EINVAL
    assert g.solver == V.SOLVER_PLAIN
    # in a multi-scene step it is stepped by viper_step on its own stream
    a, b = V.Scene(sc), V.Scene(sc)
    B = V.Batch()
    for f in range(2):
        B.step([a], [sc.bone_pose((f + 1) * sc.dt)], None, sc.dt, 10, 4)
        b.set_bones(*sc.bone_pose((f + 1) * sc.dt))
        b.step(sc.dt, 10, 4)
    B.synchronize()
    assert a.sync() == 0 and b.sync() == 0
    for key in ("x4", "v4", "q4", "w4"):
        np.testing.assert_array_equal(a.get_state()[key], b.get_state()[key], err_msg=key)


# ---------------------------------------------------------------- degenerate inputs

def _two_vertex_rods(n_rods=5, contacts=True):
    """Rods of a single segment (no interior vertex: no bend constraints) in a
    zig-zag chain: consecutive rods head +-60 deg off the x axis with seeded
    jitter, and each rod's end sphere overlaps the next rod's start sphere by
    0.1 mm, so every contact is end to end.  There the separation grows with
    slope ~l/2 away from both closest points, and the ten dichotomous decisions
    stay far above FP32 rounding; where two pills cross away from their ends the
    last decisions compare values that differ by less than FP32 resolves, the
    contact point is known to ~2^-7 of the segment, and free rods carry the
    resulting velocity differences (1e-4 of their length after two frames)."""
    rng = np.random.default_rng(4)
    r, l, depth = 0.01, 0.05, 1e-4
    off = (np.arange(n_rods + 1) * 2).astype(np.int32)
    pos = np.zeros((2 * n_rods, 3))
    quats = []
    start = np.zeros(3)
    prev = None
    for k in range(n_rods):
        th = np.radians((60.0 if k % 2 == 0 else -60.0) + rng.uniform(-10, 10))
        d = np.array([np.cos(th), np.sin(th), 0.0])
        if prev is not None:
            g = prev + d
            start = pos[2 * k - 1] + (2 * r - depth) * g / np.linalg.norm(g)
        pos[2 * k], pos[2 * k + 1] = start, start + l * d
        quats.append(S.quat_from_z(d))
        prev = d
    return S.Scene(name="two-vertex", rod_offsets=off, rest_pos=pos, rest_quat=np.array(quats),
                   radius=np.full(2 * n_rods, r), density=np.full(n_rods, 1000.0),
                   c_stretch=np.full(n_rods, 1e-6), c_bend=np.full(n_rods, 1e-6), c_volume=np.full(n_rods, 1e-6),
                   group=np.arange(n_rods, dtype=np.int32), gravity=np.array([0.0, -9.81, 0.0]),
                   pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32), pin_offset=np.zeros((0, 3)),
                   bones=None, planes=np.zeros((0, 4)), contact_compliance=1e-9, contacts=contacts, volume=True,
                   dt=1 / 60, substeps=10, iterations=4, frames=2)


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_single_segment_rods_with_contacts(V, solver):
    """The smallest rods (two vertices, one segment, no interior vertex) in
    shallow crossing contact: the slot layout, colouring and contacts still
    match.  (Deep, near-parallel initial overlaps are left out: there the
    dichotomous probe's comparisons flip with rounding and FP32 and FP64
    legitimately part ways.)"""
    sc = _two_vertex_rods()
    g, o = _pair(V, sc, solver)
    g.frame(); o.frame()
    assert len(g.pairs()) > 0  # the rods do touch
    g.frame(); o.frame()
    assert g.sync() == 0
    e = assert_parity(sc, g.get_state(), o.get_state(), POS_TOL_1, what="two-vertex rods, 2 frames")
    print("two-vertex rods with contacts, 2 frames errors vs FP64:", e)


def test_empty_skin_and_empty_batch_calls(V):
    sc = S.muscle_rig(seed=1, n_rods=10, mesh_verts=100)
    g = V.Scene(sc)
    L = V.lib()
    assert L.viper_skin(g.handle, 0, None, None, None, None) == 0
    B = V.Batch()
    assert B.step([], None, None, 1 / 60, 10, 4) == []
    g.frame()
    assert g.sync() == 0
