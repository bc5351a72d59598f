"""Stand-alone broadphase (viper_broadphase) against the oracle's FP32 predicate."""
import numpy as np
import pytest

import oracle
from paper_1906_05260_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1906_05260_gb300 import build
    build.build()
    from paper_1906_05260_gb300 import viper
    return viper


def _random_rods(seed, n_rods=300, spread=0.4):
    rng = np.random.default_rng(seed)
    lens = rng.integers(2, 20, n_rods)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    nv = int(off[-1])
    x4 = np.zeros((nv, 4), np.float32)
    for r in range(n_rods):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        x4[off[r]:off[r + 1], :3] = rng.uniform(-spread, spread, 3) + np.arange(lens[r])[:, None] * 0.02 * d
    x4[:, 3] = rng.uniform(0.6, 1.4, nv)
    rbar = rng.uniform(0.002, 0.02, nv).astype(np.float32)
    group = rng.integers(0, n_rods // 3, n_rods).astype(np.int32)
    return off, group, x4, rbar


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_standalone_broadphase_matches_oracle_predicate(V, seed):
    import torch
    off, group, x4, rbar = _random_rods(seed)
    ref = oracle.broadphase_f32(off, group, x4, rbar)
    t = lambda a: torch.from_numpy(a).cuda()
    got, total = V.broadphase(t(off), t(group), t(x4), t(rbar), max_pairs=4 * len(ref) + 16)
    assert total == len(ref)
    np.testing.assert_array_equal(got, ref)


def test_standalone_broadphase_reports_overflow_count(V):
    import torch
    off, group, x4, rbar = _random_rods(5, n_rods=400, spread=0.2)
    ref = oracle.broadphase_f32(off, group, x4, rbar)
    assert len(ref) > 100
    t = lambda a: torch.from_numpy(a).cuda()
    got, total = V.broadphase(t(off), t(group), t(x4), t(rbar), max_pairs=50)
    assert total == len(ref)
    assert got.shape[0] == 50
    refset = {tuple(p) for p in ref}
    assert all(tuple(p) in refset for p in got)


def test_standalone_broadphase_equals_scene_pairs_on_hair(V):
    import torch
    sc = S.hair(n_rods=3000)
    g = V.Scene(sc)
    g.frame()
    x4, rb = g.predicted()
    scene_pairs = g.pairs()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    got, total = V.broadphase(t(sc.rod_offsets.astype(np.int32)), t(sc.group), t(x4), t(rb),
                              max_pairs=2 * len(scene_pairs) + 16)
    assert total == len(scene_pairs)
    np.testing.assert_array_equal(got, scene_pairs)


def _rods_with_outliers(seed, n_rods=4000, n_long=900, huge=False):
    """Short four-vertex rods, some with a middle segment stretched 5-50x (and
    optionally one segment across the whole domain): the bounding radii then
    have a long tail, so the grid's cell is cut below the largest radius and
    the pills above the cut are paired from their own side."""
    rng = np.random.default_rng(seed)
    off = (np.arange(n_rods + 1) * 4).astype(np.int32)
    nv = 4 * n_rods
    x4 = np.zeros((nv, 4), np.float32)
    base = rng.uniform(-0.5, 0.5, (n_rods, 3))
    d = rng.normal(size=(n_rods, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    steps = np.full((n_rods, 3), 0.01)
    steps[:n_long, 1] *= rng.uniform(5, 50, n_long)
    if huge:
        steps[n_long, 1] = 1.5
    pos = base[:, None, :] + np.concatenate([np.zeros((n_rods, 1)), np.cumsum(steps, 1)], 1)[:, :, None] * d[:, None, :]
    x4[:, :3] = pos.reshape(nv, 3)
    x4[:, 3] = rng.uniform(0.8, 1.2, nv)
    rbar = rng.uniform(0.003, 0.01, nv).astype(np.float32)
    group = np.arange(n_rods, dtype=np.int32)
    return off, group, x4, rbar


@pytest.mark.parametrize("seed,huge", [(0, False), (1, True)])
def test_broadphase_with_oversized_pills_matches_brute_force(V, seed, huge):
    import torch
    off, group, x4, rbar = _rods_with_outliers(seed, huge=huge)
    ref = oracle.broadphase_f32(off, group, x4, rbar, brute=True)
    assert len(ref) > 1000
    t = lambda a: torch.from_numpy(a).cuda()
    got, total = V.broadphase(t(off), t(group), t(x4), t(rbar), max_pairs=2 * len(ref) + 16)
    assert total == len(ref)
    np.testing.assert_array_equal(got, ref)
