"""Shared helpers for the GPU parity tests (CUDA path vs oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2602_19697_gb300 import bfsdf, build  # noqa: E402

_ctx = None


def ctx():
    global _ctx
    if _ctx is None:
        if not torch.cuda.is_available():
            pytest.skip("no CUDA device")
        build.build()
        _ctx = bfsdf.Context(0)
    return _ctx


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_band(w):
    c = ctx()
    depth, poses = dev(w.depth), dev(w.poses)
    b = c.build_band_w(w, depth, poses)
    return b, depth, poses


def assert_band_equal(gb, ob):
    assert gb.N == ob.N and gb.NB == ob.NB and gb.n_cand == ob.n_cand
    ex = gb.export_band()
    np.testing.assert_array_equal(ex["brick_dir"], ob.dir)
    np.testing.assert_array_equal(ex["lin"], ob.lin)
    np.testing.assert_array_equal(ex["tsdf"], ob.tsdf)
    np.testing.assert_array_equal(ex["wcount"], ob.wcount)
    np.testing.assert_array_equal(ex["bdry"], ob.bdry)
    np.testing.assert_array_equal(ex["mask"].view(np.uint64), ob.mask)
    return ex
