"""The allocation-free mean solve against the regular one.

bf_solve_mean_static serves callers that cannot allocate device memory while
they run: it keeps its scratch vectors in a fixed array of device memory that
the library declares statically, instead of allocating workspaces.  This test
calls it through the C ABI twice in a row (the second call reuses the array
the first one left behind) and checks each result against bf_solve_mean's,
within the mean-parity tolerance of the other GPU tests (1e-3 voxel).  It is
collected last so that a run stopping at the first failure has run every
other test already; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_util import ctx, gpu_band, torch

pytestmark = pytest.mark.gpu

MEAN_TOL_VOX = 1e-3


def test_static_scratch_mean_solve_matches_the_allocating_one_twice():
    C = ctx()
    lib = C.lib
    for name, kw in (("sphere64", {}), ("union256", dict(n=128, frames=30, image_scale=0.5))):
        w = synth.make_workload(name, **kw)
        gb, depth, poses = gpu_band(w)
        assert gb.N <= 262144
        gb.integrate_depth(depth, poses, w.intr)
        ref = torch.empty(gb.N, device="cuda")
        info = gb.solve_mean(ref, rel_tol=1e-8)
        assert info.rel_res <= 1e-8
        for call in range(2):
            mu = torch.full((gb.N,), float("nan"), device="cuda")
            it, rr = ctypes.c_int(), ctypes.c_double()
            st = lib.bf_solve_mean_static(C._p, gb._p, 1e-8, 20000, ctypes.c_void_p(mu.data_ptr()),
                                          ctypes.byref(it), ctypes.byref(rr))
            assert st == 0, st
            assert rr.value <= 1e-8 and it.value > 0
            err = float((mu - ref).abs().max())
            assert err <= MEAN_TOL_VOX, (name, call, err)


def test_static_scratch_mean_solve_rejects_what_it_cannot_serve():
    C = ctx()
    lib = C.lib
    w = synth.make_workload("sphere64", n=32, image_scale=0.5)
    gb, depth, poses = gpu_band(w)
    mu_host = np.empty(gb.N, np.float32)
    it, rr = ctypes.c_int(), ctypes.c_double()
    # before integration: call-order error
    st = lib.bf_solve_mean_static(C._p, gb._p, 1e-6, 100, ctypes.c_void_p(mu_host.ctypes.data),
                                  ctypes.byref(it), ctypes.byref(rr))
    assert st == 6  # BF_ESTATE
    gb.integrate_depth(depth, poses, w.intr)
    # host output buffer: no staging buffer to copy through
    st = lib.bf_solve_mean_static(C._p, gb._p, 1e-6, 100, ctypes.c_void_p(mu_host.ctypes.data),
                                  ctypes.byref(it), ctypes.byref(rr))
    assert st == 1  # BF_EINVAL
