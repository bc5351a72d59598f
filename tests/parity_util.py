"""Comparison helpers shared by the GPU parity tests.

Tolerances (stated for the FP32 CUDA path against the FP64 oracle on the same
seeded inputs): positions within 1e-4 of the rod's length after one frame and
1e-3 after 100 frames, radii within 1e-5 relative, quaternion angle below 1e-4
rad; candidate-pair sets and the colouring bit-exact.
"""
import numpy as np

POS_TOL_1 = 1e-4
POS_TOL_100 = 1e-3
RAD_TOL = 1e-5
ANG_TOL = 1e-4


def rod_lengths(scene):
    off = scene.rod_offsets
    seg = np.linalg.norm(np.diff(scene.rest_pos, axis=0), axis=1)
    L = np.zeros(scene.n_rods)
    for r in range(scene.n_rods):
        L[r] = seg[off[r]:off[r + 1] - 1].sum()
    return L


def errors(scene, gpu_state, oracle_state):
    """Per-quantity errors: max |dx| / L_rod, max relative radius error, max
    quaternion angle (rad), plus the raw absolute maxima."""
    off = scene.rod_offsets
    L = rod_lengths(scene)
    rod_of_v = np.repeat(np.arange(scene.n_rods), np.diff(off))
    xg = gpu_state["x4"][:, :3].astype(np.float64)
    xo = oracle_state["x"]
    dx = np.linalg.norm(xg - xo, axis=1) / L[rod_of_v]
    rad_o = oracle_state["s"] * scene.radius
    drad = np.abs(gpu_state["x4"][:, 3].astype(np.float64) - rad_o) / rad_o
    qg = gpu_state["q4"].astype(np.float64)
    qg /= np.linalg.norm(qg, axis=1, keepdims=True)
    dot = np.clip(np.abs((qg * oracle_state["q"]).sum(1)), 0.0, 1.0)
    ang = 2.0 * np.arccos(dot)
    return {"pos": float(dx.max()), "rad": float(drad.max()), "ang": float(ang.max()),
            "pos_abs": float(np.linalg.norm(xg - xo, axis=1).max())}


def assert_parity(scene, gpu_state, oracle_state, pos_tol=POS_TOL_1, rad_tol=RAD_TOL, ang_tol=ANG_TOL, what=""):
    e = errors(scene, gpu_state, oracle_state)
    msg = f"{what}: {e}"
    assert np.isfinite(list(e.values())).all(), msg
    assert e["pos"] < pos_tol, msg
    assert e["rad"] < rad_tol, msg
    assert e["ang"] < ang_tol, msg
    return e
