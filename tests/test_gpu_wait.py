"""Bounded device waits running out: the persistent frame kernel's grid barriers.

A test build of the library (libviper_waittest.so) leaves the last CTA's
barrier arrival out and sets a spin limit of 4096 naps, so every barrier wait
of the frame kernel runs out.  The frame must come back as VIPER_ETIMEOUT (the
kernel raised the timeout bit and every CTA returned at its next barrier), and
the CUDA context must stay usable: the regular library then steps the same
scene without error.  Nothing waits without a limit.
"""
import ctypes as C

import pytest

from paper_1906_05260_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1906_05260_gb300 import build
    build.build()
    from paper_1906_05260_gb300 import viper
    return viper


def test_frame_kernel_barrier_wait_runs_out_and_reports_timeout(V):
    import torch
    from paper_1906_05260_gb300 import build
    L = C.CDLL(build.build_wait_test())
    vp = C.c_void_p
    L.viper_scene_create.argtypes = [C.POINTER(V.Desc), C.POINTER(vp)]
    L.viper_set_solver.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    L.viper_step.argtypes = [vp, C.c_float, C.c_int, C.c_int]
    L.viper_sync.argtypes = [vp]
    L.viper_scene_destroy.argtypes = [vp]
    L.viper_scene_destroy.restype = None
    sc = S.muscle_rig(n_rods=24, mesh_verts=0)
    st = torch.cuda.Stream()
    desc, keep = V.make_desc(sc, C.c_void_p(st.cuda_stream))
    h = vp()
    assert L.viper_scene_create(C.byref(desc), C.byref(h)) == 0
    try:
        assert L.viper_set_solver(h, V.SOLVER_FRAME, 4, 256) == 0
        assert L.viper_step(h, sc.dt, sc.substeps, sc.iterations) == 0  # asynchronous: the error comes at sync
        assert L.viper_sync(h) == V.ETIMEOUT
    finally:
        L.viper_scene_destroy(h)
    g = V.Scene(sc, solver=V.SOLVER_FRAME)
    g.frame()
    assert g.sync() == 0
    g.close()
