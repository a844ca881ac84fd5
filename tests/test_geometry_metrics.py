"""The geometry metrics (host-side) against closed forms: points on an exact
sphere, a radially offset sphere, an inscribed polyhedron, and the samplers."""
import numpy as np

import synth
from paper_2602_19697_gb300 import geometry


def _sphere_pts(n, r, rng):
    v = rng.standard_normal((n, 3))
    return r * v / np.linalg.norm(v, axis=1, keepdims=True)


def test_sampled_surface_lies_on_the_zero_set_and_covers_it():
    sc = synth.sphere_scene(0.3)
    rng = np.random.default_rng(1)
    pts = geometry.sample_surface(sc.sdf, (-0.5,) * 3, (0.5,) * 3, 5000, rng, band=0.02)
    assert len(pts) == 5000
    np.testing.assert_allclose(np.linalg.norm(pts, axis=1), 0.3, rtol=0, atol=1e-9)
    # directions cover the sphere: every octant is hit
    oct_ = (pts > 0).astype(int) @ np.array([1, 2, 4])
    assert len(np.unique(oct_)) == 8


def test_metrics_of_the_exact_surface_and_of_an_offset_surface():
    sc = synth.sphere_scene(0.3)
    rng = np.random.default_rng(2)
    # 200,000 points on the 1.13 m^2 sphere lie about 2.4 mm apart: nearest-neighbour distances of ~1 mm
    gt = _sphere_pts(20000, 0.3, rng)
    rec = _sphere_pts(200000, 0.3, rng)
    m = geometry.metrics(rec, gt, sc.sdf, tau=0.005)
    assert m["accuracy"] <= 1e-12 and m["precision"] == 1.0
    assert m["completeness"] < 0.002 and m["recall"] > 0.99
    # a sphere offset radially by delta: accuracy = delta exactly, completeness ~ delta, F = 0 below delta
    delta = 0.004
    off = _sphere_pts(200000, 0.3 + delta, rng)
    m = geometry.metrics(off, gt, sc.sdf, tau=0.002)
    np.testing.assert_allclose(m["accuracy"], delta, rtol=1e-9)
    assert delta <= m["completeness"] < delta + 0.002
    assert m["precision"] == 0.0 and m["fscore"] == 0.0
    m = geometry.metrics(off, gt, sc.sdf, tau=0.01)
    assert m["precision"] == 1.0 and m["fscore"] > 0.99


def test_area_weighted_mesh_samples_of_an_octahedron():
    """The octahedron with vertices +-e_i: its 8 faces have equal area, samples lie on the faces (|x|_1 = 1) and
    split evenly among them."""
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float32)
    F = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], np.int32)
    rng = np.random.default_rng(3)
    p = geometry.sample_mesh(V, F, 80000, rng)
    np.testing.assert_allclose(np.abs(p).sum(1), 1.0, rtol=0, atol=1e-6)
    face = (p > 0).astype(int) @ np.array([1, 2, 4])
    counts = np.bincount(face, minlength=8)
    assert counts.min() > 0.9 * 10000 and counts.max() < 1.1 * 10000
