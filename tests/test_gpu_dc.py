"""GPU parity of dual contouring (bf_extract_surface_dc; Sec. 3.8 surface
extraction by "MC or DC") against oracle/dc.py: the same mu (FP32) fed to
both gives the identical triangle list (topology and vertex numbering) and
vertices within FP32 rounding of the FP64 oracle's."""
import numpy as np
import pytest

import oracle
import synth
from oracle import dc
from tests import scenes
from tests.gpu_util import ctx, dev, gpu_band

pytestmark = pytest.mark.gpu


def _check(gb, ob, mu32):
    V, F = gb.extract_surface(dev(mu32), method="dc")
    Vo, Fo, _ = dc.dual_contour(ob, mu32)
    assert len(F) > 100
    np.testing.assert_array_equal(F, Fo)
    np.testing.assert_allclose(V, Vo, rtol=0, atol=1e-6 + 1e-5 * ob.h)
    return V, F


def test_dc_of_an_exact_sphere_sdf():
    s = scenes.hollow_sphere()
    C = ctx()
    gb = C.build_band(dev(s["depth"]), dev(s["poses"]), s["intr"], s["n"], s["h"], s["org"], s["band_vox"],
                      s["trunc_vox"])
    ob = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    mu = ((np.linalg.norm(ob.centres(), axis=1) - s["R"]) / ob.h).astype(np.float32)
    V, F = _check(gb, ob, mu)
    assert np.abs(np.linalg.norm(V, axis=1) - s["R"]).max() <= 0.05 * ob.h


@pytest.mark.parametrize("name", ["sphere64", "union128"])
def test_dc_of_the_posterior_mean(name):
    w = {"sphere64": lambda: synth.make_workload("sphere64"),
         "union128": lambda: synth.make_workload("union256", n=128, frames=30, image_scale=0.5)}[name]()
    r = oracle.solve_all(w, tol=1e-10)
    gb, depth, poses = gpu_band(w)
    mu32 = r["mu"].astype(np.float32)
    _check(gb, r["band"], mu32)
    # marching cubes and dual contouring of the same field: a quad per crossed edge with its four cubes
    Vm, Fm = gb.extract_surface(dev(mu32))
    V, F = gb.extract_surface(dev(mu32), method="dc")
    assert len(F) <= 2 * len(Vm)
