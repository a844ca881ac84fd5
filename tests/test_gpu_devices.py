"""Device selection: every call that takes a context runs on the context's
device, whichever device the calling thread has current (two contexts on two
GPUs driven from one thread).  Needs two GPUs; skipped on a one-GPU machine."""
import numpy as np
import pytest

import synth
from tests.gpu_util import torch

pytestmark = pytest.mark.gpu


def test_calls_on_one_context_are_unaffected_by_another_device_being_current():
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    from paper_2602_19697_gb300 import bfsdf, build
    build.build()
    w = synth.make_workload("sphere64", n=32, image_scale=0.5)
    results = []
    ctxs = [bfsdf.Context(d, stream=0) for d in (0, 1)]
    for d, C in enumerate(ctxs):
        # the other device is current when this context's calls are made
        torch.cuda.set_device(1 - d)
        b = C.build_band_w(w)            # host arrays: staged by the library on the context's device
        b.integrate_depth(w.depth, w.poses, w.intr)
        mu = np.empty(b.N, np.float32)
        b.solve_mean(mu, rel_tol=1e-8)
        s = np.empty(b.N, np.float32)
        b.estimate_variance(s, K=8, seed=1, rel_tol=1e-6)
        static = torch.empty(b.N, device=f"cuda:{d}")
        st = C.lib.bf_solve_mean_static(C._p, b._p, 1e-8, 20000, bfsdf._ptr(static), None, None)
        assert st == bfsdf.BF_OK
        results.append((mu, s, static.cpu().numpy()))
        b.free()
    np.testing.assert_allclose(results[0][0], results[1][0], rtol=0, atol=1e-5)
    np.testing.assert_allclose(results[0][1], results[1][1], rtol=1e-5)
    np.testing.assert_allclose(results[0][2], results[0][0], rtol=0, atol=1e-4)
    np.testing.assert_allclose(results[1][2], results[1][0], rtol=0, atol=1e-4)
