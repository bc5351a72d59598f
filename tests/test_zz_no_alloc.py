"""viper_broadphase_noalloc: the allocation-free broadphase query.

Callers that cannot allocate device memory when they run the query use this
entry point: real-time loops with a fixed per-frame budget (an allocation can
block or synchronise the device) and hosts whose device memory belongs to
another allocator.  Its scratch is a fixed device array inside the library.
These tests call it through the C ABI and check that two calls in a row
return exactly what the allocating viper_broadphase returns on the same inputs
(the pair set is integer data: compared bit for bit), that a call leaves
torch's allocator untouched, and that queries above the fixed limit are
refused.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1906_05260_gb300 import build
    build.build()
    from paper_1906_05260_gb300 import viper
    return viper


def _rods(seed, n_rods):
    rng = np.random.default_rng(seed)
    lens = rng.integers(2, 24, n_rods)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    nv = int(off[-1])
    x4 = np.zeros((nv, 4), np.float32)
    for r in range(n_rods):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        x4[off[r]:off[r + 1], :3] = rng.uniform(-0.6, 0.6, 3) + np.arange(lens[r])[:, None] * 0.015 * d
    x4[:, 3] = rng.uniform(0.7, 1.3, nv)
    rbar = rng.uniform(0.002, 0.015, nv).astype(np.float32)
    group = np.arange(n_rods, dtype=np.int32)
    return off, group, x4, rbar


def _call(V, fn, off, group, x4, rbar, cap):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_off, d_grp, d_x4, d_rb = t(off), t(group), t(x4), t(rbar)
    pairs = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    rc = fn(len(off) - 1, x4.shape[0], C.c_void_p(d_off.data_ptr()), C.c_void_p(d_grp.data_ptr()),
            C.c_void_p(d_x4.data_ptr()), C.c_void_p(d_rb.data_ptr()), C.c_void_p(pairs.data_ptr()), cap,
            C.c_void_p(n.data_ptr()), C.c_void_p(st.cuda_stream))
    st.synchronize()
    total = int(n.item())
    got = pairs[: min(total, cap)].cpu().numpy()
    got = got[np.lexsort((got[:, 1], got[:, 0]))] if got.size else got
    return rc, total, got


def test_noalloc_matches_allocating_query_on_two_calls_in_a_row(V):
    L = V.lib()
    for call, seed in enumerate((11, 12)):
        off, group, x4, rbar = _rods(seed, 2500 + 700 * call)
        assert x4.shape[0] - (len(off) - 1) <= 65536
        cap = 400_000
        rc_a, tot_a, ref = _call(V, L.viper_broadphase, off, group, x4, rbar, cap)
        rc_b, tot_b, got = _call(V, L.viper_broadphase_noalloc, off, group, x4, rbar, cap)
        assert rc_a == 0 and rc_b == 0
        assert 1000 < tot_a <= cap  # every pair fits: the compared sets are complete
        assert tot_b == tot_a
        np.testing.assert_array_equal(got, ref)


def test_noalloc_refuses_queries_above_its_fixed_scratch(V):
    L = V.lib()
    n_rods = 1000
    nv = n_rods + 65536 + 1  # one segment more than the limit
    dummy = C.c_void_p(256)  # never dereferenced: the size check comes first
    n = C.c_void_p(256)
    rc = L.viper_broadphase_noalloc(n_rods, nv, dummy, None, dummy, dummy, dummy, 16, n, None)
    assert rc == V.EINVAL


def test_noalloc_leaves_the_torch_allocator_untouched(V):
    import torch
    L = V.lib()
    off, group, x4, rbar = _rods(13, 1500)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_off, d_grp, d_x4, d_rb = t(off), t(group), t(x4), t(rbar)
    cap = 200_000
    pairs = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    args = (len(off) - 1, x4.shape[0], C.c_void_p(d_off.data_ptr()), C.c_void_p(d_grp.data_ptr()),
            C.c_void_p(d_x4.data_ptr()), C.c_void_p(d_rb.data_ptr()), C.c_void_p(pairs.data_ptr()), cap,
            C.c_void_p(n.data_ptr()), C.c_void_p(st.cuda_stream))
    assert L.viper_broadphase_noalloc(*args) == 0  # the device's first call: address lookup
    st.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    assert L.viper_broadphase_noalloc(*args) == 0
    st.synchronize()
    assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == before
    assert int(n.item()) > 0
