"""Serving runtime: continuous batching of many scenes (through the C ABI)."""
import dataclasses

import numpy as np
import pytest

from paper_1906_05260_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SV():
    from paper_1906_05260_gb300 import build
    build.build()
    from paper_1906_05260_gb300 import serving
    return serving


def _frames(srv, sid, n, t0=0.0):
    sc = srv.scenes[sid]
    tks = [srv.submit(sid, t0 + (k + 1) * sc.dt) for k in range(n)]
    return tks


def test_results_identical_alone_and_in_the_mix(SV):
    a = S.muscle_rig(seed=21, n_rods=60, mesh_verts=5000)
    others = [S.muscle_rig(seed=30 + i, n_rods=40 + 30 * i, mesh_verts=3000) for i in range(7)]
    # alone
    srv = SV.Server(8 << 30, max_inflight=64)
    sid = srv.admit(a)
    for tk in _frames(srv, sid, 6):
        st, lat = srv.wait(tk)
        assert st == 0
    alone = srv.state(sid)
    mesh_alone = srv.mesh_out(sid)
    srv.close()
    # in the mix: everything submitted at once, frames of all scenes overlap on the GPU
    srv = SV.Server(8 << 30, max_inflight=64)
    ids = [srv.admit(sc) for sc in [a] + others]
    tks = []
    for k in range(6):
        for i in ids:
            tks.append(srv.submit(i, (k + 1) * a.dt))
    for tk in tks:
        st, lat = srv.wait(tk)
        assert st == 0
    mix = srv.state(ids[0])
    mesh_mix = srv.mesh_out(ids[0])
    stats = srv.stats()
    srv.close()
    for k in ("x4", "v4", "q4", "w4"):
        np.testing.assert_array_equal(alone[k], mix[k])
    np.testing.assert_array_equal(mesh_alone, mesh_mix)
    assert stats["frames"] == 48 and stats["failed"] == 0
    assert stats["steps"] < stats["frames"]  # scenes were stepped together


def test_admission_by_memory_budget(SV):
    from paper_1906_05260_gb300 import viper as V
    a = S.muscle_rig(seed=22, n_rods=80, mesh_verts=20000)
    b = S.muscle_rig(seed=23, n_rods=80, mesh_verts=20000)
    need = V.footprint(a) + 64 * a.mesh.n + 4096
    srv = SV.Server(int(need * 1.5), max_inflight=8)
    ia = srv.admit(a)
    assert ia is not None
    assert srv.admit(b) is None  # does not fit beside a
    for tk in _frames(srv, ia, 2):
        assert srv.wait(tk)[0] == 0
    srv.release(ia)
    ib = srv.admit(b)
    assert ib is not None
    for tk in _frames(srv, ib, 2):
        assert srv.wait(tk)[0] == 0
    srv.close()


def test_a_diverged_scene_does_not_affect_the_others(SV):
    import ctypes as C
    from paper_1906_05260_gb300 import viper as V
    good = S.muscle_rig(seed=24, n_rods=50, mesh_verts=0)
    bad = S.muscle_rig(seed=25, n_rods=50, mesh_verts=0)
    srv = SV.Server(4 << 30, max_inflight=8)
    ig, ib = srv.admit(good), srv.admit(bad)
    st = srv.state(ib)
    x4 = st["x4"].copy()
    x4[3, 0] = np.nan
    h = V.lib().viper_server_scene(srv._h, ib)
    assert V.lib().viper_set_state(C.c_void_p(h), C.c_void_p(x4.ctypes.data), None, None, None) == 0
    res_g, res_b = [], []
    for k in range(4):
        res_g.append(srv.submit(ig, (k + 1) * good.dt))
        res_b.append(srv.submit(ib, (k + 1) * bad.dt))
    assert all(srv.wait(t)[0] == 0 for t in res_g)
    codes = [srv.wait(t)[0] for t in res_b]
    assert V.ENONFINITE in codes
    assert np.isfinite(srv.state(ig)["x4"]).all()
    srv.close()


def test_short_real_time_load(SV):
    temps = SV.scene_templates(seed=5, n=4, rods_lo=40, rods_hi=120, mesh_lo=5000, mesh_hi=20000)
    out = SV.run_load(duration=3.0, rate=4.0, mean_life=2.0, budget=16 << 30, max_inflight=64, seed=5,
                      templates=temps, warm_scenes=6)
    print("short serving load:", out)
    assert out["frames"] > 100
    assert out["failed"] == 0
    assert out["p99_ms"] > 0
