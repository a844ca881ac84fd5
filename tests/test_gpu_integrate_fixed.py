"""Deterministic observation sums (int64 fixed point) against the oracle and
against themselves.

The fixed-point mode adds each FP32 sample w and w y as an int64 in units of
2^-32, so the totals equal the FP64 sum of the rounded samples exactly and do
not depend on the order of the concurrent updates: repeated integrations give
identical bits.  Against the FP64 oracle the bar is the one of the FP32 path
(the samples themselves are FP32 values); against the FP32 path it is the
FP32 accumulation error.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2602_19697_gb300 import bfsdf
from tests.gpu_util import gpu_band

pytestmark = pytest.mark.gpu

_cache = {}


def case(name):
    if name not in _cache:
        w = (synth.make_workload("union256", n=128, frames=30, image_scale=0.5) if name == "union128"
             else synth.make_workload("sphere64"))
        ob = oracle.build_band_w(w)
        d, hd, _ = oracle.integrate_w(ob, w)
        _cache[name] = dict(w=w, d=d, hd=hd)
    return _cache[name]


@pytest.mark.parametrize("name", ["sphere64", "union128"])
def test_fixed_point_sums_are_reproducible_and_match_the_oracle(name):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr, deterministic=True)
    s1 = gb.export_system()
    scale = np.abs(c["d"]).max()
    np.testing.assert_allclose(s1["d"], c["d"], rtol=1e-4, atol=1e-5 * scale)
    np.testing.assert_allclose(s1["hdata"], c["hd"], rtol=1e-4, atol=2e-5 * np.abs(c["hd"]).max())
    # the same frames again, on the same band after a reset and on a second band: identical bits
    gb.reset_observations()
    gb.integrate_depth(depth, poses, w.intr, deterministic=True)
    s2 = gb.export_system()
    gb2, _, _ = gpu_band(w)
    gb2.integrate_depth(depth, poses, w.intr, deterministic=True)
    s3 = gb2.export_system()
    for k in ("d", "hdata", "qdiag", "rhs"):
        np.testing.assert_array_equal(s1[k], s2[k])
        np.testing.assert_array_equal(s1[k], s3[k])
    # two calls accumulate exactly: the fixed-point sum of the doubled data is twice the single sum
    gb.integrate_depth(depth, poses, w.intr, deterministic=True)
    s4 = gb.export_system()
    np.testing.assert_array_equal(s4["d"], (2.0 * s1["d"].astype(np.float64)).astype(np.float32))
    # the FP32 path agrees within its accumulation error
    gb3, _, _ = gpu_band(w)
    gb3.integrate_depth(depth, poses, w.intr)
    s5 = gb3.export_system()
    np.testing.assert_allclose(s5["d"], s1["d"], rtol=1e-5, atol=1e-6 * scale)
    # FP64 export: the fixed-point totals (rounding them gives the FP32 export), the FP32 sums widened
    d64, h64 = gb2.export_observations_f64()
    np.testing.assert_array_equal(d64.astype(np.float32), s3["d"])
    np.testing.assert_array_equal(h64.astype(np.float32), s3["hdata"])
    np.testing.assert_allclose(d64, c["d"], rtol=1e-5, atol=1e-7 * scale)
    d64f, _ = gb3.export_observations_f64()
    np.testing.assert_array_equal(d64f, s5["d"].astype(np.float64))


def test_one_accumulation_mode_per_band_until_reset():
    c = case("sphere64")
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr, deterministic=True)
    with pytest.raises(bfsdf.BfError):
        gb.integrate_depth(depth, poses, w.intr)
    gb.reset_observations()
    gb.integrate_depth(depth, poses, w.intr)
    with pytest.raises(bfsdf.BfError):
        gb.integrate_depth(depth, poses, w.intr, deterministic=True)
    gb.reset_observations()
    gb.integrate_depth(depth, poses, w.intr, deterministic=True)
    assert np.all(np.isfinite(gb.export_system()["d"]))
