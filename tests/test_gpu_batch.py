"""GPU: the multi-scene step (viper_batch_step) through the C ABI.

A scene stepped in a batch runs the one-scene kernels' device code on the
same schedule, so it must (1) match the FP64 oracle within the parity
tolerances, (2) agree with the same scene stepped alone by viper_step to FP32
rounding, and (3) give bit-identical results alone in a batch and mixed with
other scenes (no state is shared between scenes; contacts are summed in fixed
point, so the order in which pairs are found does not matter).
"""
import numpy as np
import pytest

import oracle
from paper_1906_05260_gb300 import scenes as S
from parity_util import POS_TOL_1, assert_parity

pytestmark = pytest.mark.gpu

DT, SUB, IT = 1.0 / 60, 10, 4


@pytest.fixture(scope="module")
def V():
    from paper_1906_05260_gb300 import build
    build.build()
    from paper_1906_05260_gb300 import viper
    return viper


def _mix():
    """Scenes of different kinds and sizes: contacts + bones + mesh, contacts
    only, half-planes + contacts, no contacts (its own launch group)."""
    return [S.muscle_rig(seed=1, n_rods=60, mesh_verts=5000),
            S.muscle_rig(seed=5, n_rods=150, mesh_verts=0),
            S.hair(n_rods=300),
            S.plain_small()]


def _pose(sc, t):
    return sc.bone_pose(t) if sc.bones is not None else None


def _batch_frames(V, B, scenes, objs, meshes, frames):
    for f in range(frames):
        poses = [_pose(sc, (f + 1) * DT) for sc in scenes]
        st = B.step(objs, poses, meshes, DT, SUB, IT)
        assert all(c == 0 for c in st), st
    B.synchronize()


def _solo_frames(objs, scenes, frames):
    for f in range(frames):
        for o, sc in zip(objs, scenes):
            p = _pose(sc, (f + 1) * DT)
            if p is not None:
                o.set_bones(*p)
            o.step(DT, SUB, IT)


def test_batch_scene_matches_oracle(V):
    scenes = _mix()
    objs = [V.Scene(sc) for sc in scenes]
    mesh = V.Mesh(scenes[0].mesh)
    B = V.Batch()
    _batch_frames(V, B, scenes, objs, [mesh, None, None, None], 2)
    o = oracle.OracleScene(scenes[0])
    for f in range(2):
        o.set_bones(*scenes[0].bone_pose((f + 1) * DT))
        o.step(DT, SUB, IT)
    assert objs[0].sync() == 0
    gst = objs[0].get_state()
    e = assert_parity(scenes[0], gst, o.get_state(), POS_TOL_1, what="muscle_rig in a batch, 2 frames")
    print("muscle_rig in a 4-scene batch, 2 frames, errors vs FP64:", e)
    # skinning of the batched state against the oracle's LBS of the same FP32 state
    o2 = oracle.OracleScene(scenes[0])
    o2.set_state(x=gst["x4"][:, :3], s=gst["x4"][:, 3] / scenes[0].radius, q=gst["q4"])
    ref = o2.skin()
    out = mesh.out.cpu().numpy()[:, :3].astype(np.float64)
    assert np.abs(out - ref).max() < 2e-6 * np.abs(scenes[0].mesh.rest).max()


def test_batch_agrees_with_single_scene_steps(V):
    scenes = _mix()
    a = [V.Scene(sc) for sc in scenes]
    b = [V.Scene(sc) for sc in scenes]
    ma = V.Mesh(scenes[0].mesh)
    mb = V.Mesh(scenes[0].mesh)
    B = V.Batch()
    _batch_frames(V, B, scenes, a, [ma, None, None, None], 3)
    _solo_frames(b, scenes, 3)
    b[0].skin(mb)
    for k, (ga, gb) in enumerate(zip(a, b)):
        assert ga.sync() == 0 and gb.sync() == 0
        sa, sb = ga.get_state(), gb.get_state()
        scale = np.abs(sa["x4"][:, :3]).max() + 1e-3
        dx = np.abs(sa["x4"] - sb["x4"]).max()
        dq = np.abs(sa["q4"] - sb["q4"]).max()
        print(f"scene {k}: batch vs viper_step max |dx| = {dx:.3e} (scale {scale:.3f}), max |dq| = {dq:.3e}")
        assert dx < 4e-6 * scale
        assert dq < 1e-4
    out_a, out_b = ma.out.cpu().numpy(), mb.out.cpu().numpy()
    assert np.abs(out_a - out_b).max() < 4e-6 * np.abs(scenes[0].mesh.rest).max()


def test_batch_alone_equals_in_mix_bitwise(V):
    scenes = _mix()
    alone = [V.Scene(sc) for sc in scenes[:2]]
    mixed = [V.Scene(sc) for sc in scenes]
    m_alone, m_mixed = V.Mesh(scenes[0].mesh), V.Mesh(scenes[0].mesh)
    B1, B2 = V.Batch(), V.Batch()
    for f in range(3):
        # scene 0 alone; scene 1 alone in its own call
        B1.step([alone[0]], [_pose(scenes[0], (f + 1) * DT)], [m_alone], DT, SUB, IT)
        B1.step([alone[1]], [_pose(scenes[1], (f + 1) * DT)], None, DT, SUB, IT)
        # the same two among the others, in another order
        order = [2, 1, 3, 0]
        B2.step([mixed[k] for k in order], [_pose(scenes[k], (f + 1) * DT) for k in order],
                [m_mixed if k == 0 else None for k in order], DT, SUB, IT)
    B1.synchronize(); B2.synchronize()
    for k in range(2):
        sa, sb = alone[k].get_state(), mixed[k].get_state()
        for key in ("x4", "v4", "q4", "w4"):
            np.testing.assert_array_equal(sa[key], sb[key], err_msg=f"scene {k} {key}")
    np.testing.assert_array_equal(m_alone.out.cpu().numpy(), m_mixed.out.cpu().numpy())


def test_batch_launch_count_independent_of_scene_count(V):
    sc = S.muscle_rig(seed=1, n_rods=40, mesh_verts=1000)
    one = [V.Scene(sc)]
    many = [V.Scene(S.muscle_rig(seed=10 + k, n_rods=40, mesh_verts=1000)) for k in range(6)]
    B = V.Batch()
    counts = []
    for objs in (one, many):
        meshes = [V.Mesh(o.scene.mesh) for o in objs]
        c0 = B.launch_count()
        B.step(objs, [o.scene.bone_pose(DT) for o in objs], meshes, DT, SUB, IT)
        counts.append(B.launch_count() - c0)
    B.synchronize()
    # per substep: advance, grid, pair search, first sweep, contact, (I - 1) x (sweep, contact);
    # then the velocity update, the frame end and the skinning
    assert counts[0] == counts[1] == SUB * (2 * IT + 3) + 3, counts


def test_batch_quarantines_nonfinite_scene_only(V):
    scenes = [S.muscle_rig(seed=1, n_rods=40, mesh_verts=0), S.muscle_rig(seed=6, n_rods=40, mesh_verts=0)]
    objs = [V.Scene(sc) for sc in scenes]
    twin = V.Scene(scenes[0])
    st = objs[1].get_state()
    st["x4"][3, 0] = np.nan
    objs[1].set_state(x4=st["x4"])
    B = V.Batch()
    for f in range(3):
        poses = [_pose(sc, (f + 1) * DT) for sc in scenes]
        status = B.step(objs, poses, None, DT, SUB, IT)
        B.synchronize()
        assert status[0] == 0
        if f >= 1:
            assert status[1] == V.ENONFINITE
        twin.set_bones(*_pose(scenes[0], (f + 1) * DT))
        twin.step(DT, SUB, IT)
    assert objs[1].sync() == V.ENONFINITE
    sa, sb = objs[0].get_state(), twin.get_state()
    assert np.isfinite(sa["x4"]).all()
    assert np.abs(sa["x4"] - sb["x4"]).max() < 4e-6 * (np.abs(sa["x4"][:, :3]).max() + 1e-3)


def test_batch_rejects_bad_arguments(V):
    sc = S.muscle_rig(seed=1, n_rods=20, mesh_verts=0)
    g = V.Scene(sc)
    B = V.Batch()
    items = (V.BatchItem * 2)()
    items[0].scene = items[1].scene = g.handle.value
    L = V.lib()
    assert L.viper_batch_step(B._h, items, 2, DT, SUB, IT, None) == V.EINVAL  # same scene twice
    assert L.viper_batch_step(B._h, items, 1, 0.0, SUB, IT, None) == V.EINVAL  # dt <= 0
    items[0].n_mesh = 10  # mesh without pointers
    assert L.viper_batch_step(B._h, items, 1, DT, SUB, IT, None) == V.EINVAL
    assert L.viper_batch_step(B._h, items, 0, DT, SUB, IT, None) == 0  # empty call


def test_batch_large_scene_and_zero_iterations(V):
    """A scene too large for the one-CTA grid build (the multi-CTA broadphase
    sequence), and frames without iterations (prediction, broadphase and
    velocity update only), against viper_step."""
    big = S.hair()  # 20,000 strands: 300,000 pills
    small = S.muscle_rig(seed=3, n_rods=40, mesh_verts=0)
    for iters, scenes in ((IT, [big, small]), (0, [small])):
        a = [V.Scene(sc) for sc in scenes]
        b = [V.Scene(sc) for sc in scenes]
        B = V.Batch()
        for f in range(2):
            B.step(a, [_pose(sc, (f + 1) * DT) for sc in scenes], None, DT, SUB, iters)
        B.synchronize()
        for f in range(2):
            for o, sc in zip(b, scenes):
                p = _pose(sc, (f + 1) * DT)
                if p is not None:
                    o.set_bones(*p)
                o.step(DT, SUB, iters)
        for ga, gb in zip(a, b):
            assert ga.sync() == 0 and gb.sync() == 0
            sa, sb = ga.get_state(), gb.get_state()
            scale = np.abs(sa["x4"][:, :3]).max() + 1e-3
            assert np.abs(sa["x4"] - sb["x4"]).max() < 4e-6 * scale
            assert np.abs(sa["q4"] - sb["q4"]).max() < 1e-4


def test_misaligned_mesh_arrays_are_rejected(V):
    """The skinning arrays are read and written as float4 / int4: device pointers
    that are not 16-byte aligned are refused (no misaligned access on the GPU)."""
    import ctypes as C
    import torch
    sc = S.muscle_rig(seed=1, n_rods=20, mesh_verts=100)
    g = V.Scene(sc)
    mesh = V.Mesh(sc.mesh)
    L = V.lib()
    bad = torch.empty(4 * mesh.n + 1, dtype=torch.float32, device="cuda")
    bad_ptr = C.c_void_p(bad.data_ptr() + 4)  # 4-byte offset
    assert L.viper_skin(g.handle, mesh.n, bad_ptr, C.c_void_p(mesh.idx.data_ptr()), C.c_void_p(mesh.w.data_ptr()),
                        C.c_void_p(mesh.out.data_ptr())) == V.EINVAL
    items = (V.BatchItem * 1)()
    items[0].scene = g.handle.value
    items[0].n_mesh = mesh.n
    items[0].rest4 = bad_ptr.value
    items[0].idx4 = mesh.idx.data_ptr()
    items[0].w4 = mesh.w.data_ptr()
    items[0].out4 = mesh.out.data_ptr()
    B = V.Batch()
    assert L.viper_batch_step(B._h, items, 1, DT, SUB, IT, None) == V.EINVAL
    # aligned arrays still skin
    g.skin(mesh)
    assert g.sync() == 0


def test_batch_pairs_bit_exact_in_a_large_group(V):
    """Four 200-rod muscle rigs in one multi-scene step (about 28k pills: the pair
    search runs a chunk with all its neighbour lists per warp): every scene's
    candidate pairs equal the oracle's FP32 predicate on its predicted state."""
    scenes = [S.muscle_rig(seed=11 + k, n_rods=200, mesh_verts=0) for k in range(4)]
    assert sum(sc.ns for sc in scenes) > 16384
    objs = [V.Scene(sc) for sc in scenes]
    B = V.Batch()
    for f in range(2):
        B.step(objs, [sc.bone_pose((f + 1) * DT) for sc in scenes], None, DT, SUB, IT)
        B.synchronize()
        for o, sc in zip(objs, scenes):
            x4, rb = o.predicted()
            ref = oracle.broadphase_f32(sc.rod_offsets, sc.group, x4, rb)
            np.testing.assert_array_equal(o.pairs(), ref)
    assert all(o.sync() == 0 for o in objs)


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["plain", "batched", "frame"])
def test_contact_warp_search_matches_thread_search_bitwise(V, solver):
    """The contact pass gives each pair a warp while the pairs fit its warps
    (the dichotomous search four steps per round); with FLAG_CONTACT_THREADS
    it searches with one thread per pair.  Both make the same decisions on the
    same values, so the states agree bit for bit."""
    sc = S.muscle_rig(mesh_verts=0)
    a = V.Scene(sc, solver=solver, extra_flags=V.FLAG_CONTACT_THREADS)
    b = V.Scene(sc, solver=solver)
    warps = min(64, -(-sc.ns // 256)) * 8  # the batched contact pass's warps (the others have more)
    for _ in range(3):
        a.frame(); b.frame()
        assert 0 < len(b.pairs()) <= 2 * warps  # the warp-per-pair branch ran
    assert a.sync() == 0 and b.sync() == 0
    sa, sb = a.get_state(), b.get_state()
    for k in ("x4", "v4", "q4", "w4"):
        np.testing.assert_array_equal(sa[k], sb[k])
