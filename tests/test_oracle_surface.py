"""Pins of the oracle's marching cubes and view scoring (Sec. 3.8 surface
extraction and NBV utility)."""
from collections import Counter

import numpy as np
import pytest

import oracle
import synth
from tests import scenes


def _edges(F):
    return [(a, b) for t in F for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))]


def test_case_polygons_cover_exactly_the_crossed_edges():
    corners = [(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)]
    for cs in range(256):
        tri = oracle.mc_case(cs)
        crossed = set()
        for a in range(3):
            for e in range(4):
                u, v = e & 1, e >> 1
                lo = [0, 0, 0]
                oth = [x for x in range(3) if x != a]
                lo[oth[0]], lo[oth[1]] = u, v
                c0 = lo[0] | lo[1] << 1 | lo[2] << 2
                c1 = c0 | 1 << a
                if ((cs >> c0) & 1) != ((cs >> c1) & 1):
                    crossed.add(4 * a + e)
        assert set(tri.flatten().tolist()) == crossed
        if cs in (0, 255):
            assert len(tri) == 0
        # a polygon of m crossed edges has m - 2 triangles: total = |crossed| - 2 loops
        n_loops = (len(crossed) - len(tri)) / 2
        assert n_loops == int(n_loops) and (len(crossed) == 0 or n_loops >= 1)
        # single inside corner: one triangle, normal pointing away from that corner
        if bin(cs).count("1") == 1:
            c = cs.bit_length() - 1
            assert len(tri) == 1
            pts = []
            for e in tri[0]:
                a, u, v = e >> 2, e & 1, (e >> 1) & 1
                oth = [x for x in range(3) if x != a]
                p = np.zeros(3)
                p[a] = 0.5
                p[oth[0]], p[oth[1]] = u, v
                pts.append(p)
            nrm = np.cross(pts[1] - pts[0], pts[2] - pts[0])
            assert nrm @ (np.mean(pts, 0) - np.array(corners[c])) > 0


def test_sphere_surface_is_a_closed_oriented_genus_zero_mesh():
    s = scenes.hollow_sphere()
    b = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    R, h = s["R"], s["h"]
    mu = ((np.linalg.norm(b.centres(), axis=1) - R) / h).astype(np.float32)   # outside positive
    V, F = oracle.marching_cubes(b, mu)
    E = _edges(F)
    und = Counter(tuple(sorted(e)) for e in E)
    assert set(und.values()) == {2}                           # closed 2-manifold
    assert len(set(E)) == len(E)                              # each directed edge once: oriented
    assert len(V) - len(und) + len(F) == 2                    # Euler characteristic of a sphere
    # vertices on the sphere up to linear-interpolation error h / (8 R) voxels
    assert np.abs(np.linalg.norm(V, axis=1) - R).max() / h <= h / (8 * R) + 1e-6
    # normals point to mu >= 0 (outside)
    v0, v1, v2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    assert np.all(np.einsum("ij,ij->i", nrm, (v0 + v1 + v2) / 3) > 0)
    # every vertex is used and vertices are sorted by (lower voxel, axis)
    assert set(F.flatten().tolist()) == set(range(len(V)))


def test_random_field_mesh_is_watertight_inside_the_grid():
    s = scenes.frontal_plane(n=16, band_vox=20.0, trunc_vox=22.0, W=64, f=60.0)
    b = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    n = s["n"]
    assert b.N == n ** 3
    rng = np.random.default_rng(3)
    ijk = b.ijk()
    mu = np.zeros(b.N)
    for _ in range(12):
        c = rng.uniform(0, n, 3)
        mu += np.exp(-((ijk - c) ** 2).sum(1) / 8.0)
    mu = (0.35 - mu).astype(np.float32)
    V, F = oracle.marching_cubes(b, mu)
    assert len(F) > 500
    E = _edges(F)
    und = Counter(tuple(sorted(e)) for e in E)
    assert set(und.values()) <= {1, 2}
    assert len(set(E)) == len(E)
    g = (V - np.array(s["org"])) / s["h"] - 0.5
    on_face = lambda p: np.any((np.abs(p) < 1e-5) | (np.abs(p - (n - 1)) < 1e-5))
    for e, k in und.items():
        if k == 1:
            assert on_face(g[e[0]]) and on_face(g[e[1]])


@pytest.fixture(scope="module")
def sphere_views():
    w = synth.make_workload("sphere64", noise=False, n=32, image_scale=0.5)
    P = np.concatenate([synth.ring_poses(32, 1.0), np.stack([synth.look_at((0, 0, 1.0)), synth.look_at((0, 0, -1.0))])])
    fx, fy, cx, cy, W, H = w.intr
    w.poses = P.astype(np.float32)
    w.depth = synth.render(w.scene, P, W, H, fx, fy, cx, cy)
    b = oracle.build_band_w(w)
    return w, b


def test_raycast_depth_of_an_exact_sdf_matches_the_rendered_depth(sphere_views):
    w, b = sphere_views
    mu = ((np.linalg.norm(b.centres(), axis=1) - 0.3) / w.h).astype(np.float32)
    pose = synth.look_at((0.9, 0.3, 0.4)).astype(np.float32)
    intr = (70.0, 70.0, 40.0, 30.0, 80, 60)
    Dp = oracle.predict_depth(b, mu, pose, intr)
    Dt = synth.render(synth.sphere_scene(0.3), pose[None].astype(np.float64), 80, 60, 70.0, 70.0, 40.0, 30.0)[0]
    both = (Dp > 0) & (Dt > 0)
    assert both.sum() > 0.9 * (Dt > 0).sum()
    # ignore grazing pixels (the cube/band edge there clips the interpolant)
    C = pose[:, 3].astype(np.float64)
    yy, xx = np.mgrid[0:60, 0:80]
    dc = np.stack([(xx + 0.5 - 40) / 70, (yy + 0.5 - 30) / 70, np.ones_like(xx, float)], -1)
    dw = dc @ pose[:, :3].T.astype(np.float64)
    p = C + Dt[..., None] * dw
    cosi = -np.einsum("ijk,ijk->ij", dw / np.linalg.norm(dw, axis=-1, keepdims=True), p / 0.3)
    sel = both & (cosi > 0.3)
    # trilinear interpolation of |x|-R is exact to O(h^2/R); bisection to h/2^11
    err = np.abs(Dp[sel] - Dt[sel]) * np.linalg.norm(dc[sel], axis=-1)
    assert err.max() <= 0.08 * w.h


def test_view_utility_is_the_diagonal_update_of_the_predicted_observations(sphere_views):
    w, b = sphere_views
    d, hd, _ = oracle.integrate_w(b, w)
    qd, rhs = oracle.assemble(b, d, hd, w.lam, w.lam_b)
    mu, *_ = oracle.pcg(b, w.lam, qd, rhs, tol=1e-12)
    s, *_ = oracle.hutchinson(b, w.lam, qd, 8, 0, tol=1e-10)
    mu32 = mu.astype(np.float32)
    cand = w.cand_poses[:4]
    U, best = oracle.score_views(b, mu32, s, qd, cand, w.cand_intr, w.band_vox, w.sig_a, w.sig_b)
    for v in range(len(cand)):
        Dp = oracle.predict_depth(b, mu32, cand[v], w.cand_intr)
        dd, _, _ = oracle.integrate(b, Dp[None], cand[v:v + 1], w.cand_intr, w.band_vox, w.sig_a, w.sig_b)
        sf = np.maximum(s, 1.0 / qd)
        om = np.abs(mu32.astype(np.float64)) <= 1.0
        ref = np.sum((sf - 1.0 / (1.0 / sf + dd))[om])
        assert abs(U[v] - ref) <= 1e-10 * abs(ref)
    assert best == int(np.argmax(U))


def test_without_prior_the_utility_is_the_exact_variance_reduction(sphere_views):
    """lambda = 0 makes Q diagonal: 1/Q_ii is the exact marginal variance and
    adding a view's precision dd gives exactly 1/(Q_ii + dd_i)."""
    w, b = sphere_views
    d, hd, _ = oracle.integrate_w(b, w)
    qd, rhs = oracle.assemble(b, d, hd, 0.0, 1.0)
    qd = qd + 1e-3
    mu, *_ = oracle.pcg(b, 0.0, qd, rhs, tol=1e-13)
    s, *_ = oracle.hutchinson(b, 0.0, qd, 1, 0, tol=1e-13)
    mu32 = mu.astype(np.float32)
    U, _ = oracle.score_views(b, mu32, s, qd, w.cand_poses[:2], w.cand_intr, w.band_vox, w.sig_a, w.sig_b)
    for v in range(2):
        Dp = oracle.predict_depth(b, mu32, w.cand_poses[v], w.cand_intr)
        dd, _, _ = oracle.integrate(b, Dp[None], w.cand_poses[v:v + 1], w.cand_intr, w.band_vox, w.sig_a, w.sig_b)
        s_after, *_ = oracle.hutchinson(b, 0.0, qd + dd, 1, 0, tol=1e-13)
        om = np.abs(mu32.astype(np.float64)) <= 1.0
        ref = np.sum((1.0 / qd - s_after)[om])
        assert ref > 0
        assert abs(U[v] - ref) <= 1e-9 * ref


def test_view_that_sees_no_band_scores_zero_and_utilities_are_nonnegative():
    w = synth.make_workload("sphere64", n=32, image_scale=0.5)
    r = oracle.solve_all(w, tol=1e-10, K=4)
    b = r["band"]
    mu32 = r["mu"].astype(np.float32)
    away = synth.look_at((1.0, 0.0, 0.0), target=(2.0, 0.0, 0.0))
    cand = np.concatenate([away[None], w.cand_poses[:6]]).astype(np.float32)
    U, best = oracle.score_views(b, mu32, r["s"], r["qdiag"], cand, w.cand_intr, w.band_vox, w.sig_a, w.sig_b)
    assert U[0] == 0.0
    assert np.all(U >= 0) and U.max() > 0 and best == int(np.argmax(U))


def test_exact_utility_without_prior_is_the_closed_form_variance_reduction(sphere_views):
    """lambda = 0: Q diagonal, one Rademacher probe gives diag(Q^-1) exactly (z^2 = 1), so the exact utility is
    sum (1/Q_ii - 1/(Q_ii + dd_i)) over the near-surface voxels, which the diagonal update also equals."""
    w, b = sphere_views
    d, hd, _ = oracle.integrate_w(b, w)
    qd, rhs = oracle.assemble(b, d, hd, 0.0, 1.0)
    qd = qd + 1e-3
    mu, *_ = oracle.pcg(b, 0.0, qd, rhs, tol=1e-13)
    mu32 = mu.astype(np.float32)
    cand = w.cand_poses[:3]
    U, best = oracle.score_views_exact(b, mu32, qd, 0.0, cand, w.cand_intr, w.band_vox, w.sig_a, w.sig_b, K=1,
                                       seed=4, tol=1e-13)
    om = np.abs(mu32.astype(np.float64)) <= 1.0
    s = 1.0 / qd
    Ud, _ = oracle.score_views(b, mu32, s, qd, cand, w.cand_intr, w.band_vox, w.sig_a, w.sig_b)
    for v in range(len(cand)):
        Dp = oracle.predict_depth(b, mu32, cand[v], w.cand_intr)
        dd, _, _ = oracle.integrate(b, Dp[None], cand[v:v + 1], w.cand_intr, w.band_vox, w.sig_a, w.sig_b)
        ref = np.sum((1.0 / qd - 1.0 / (qd + dd))[om])
        assert abs(U[v] - ref) <= 1e-9 * max(ref, 1e-30)
        assert abs(U[v] - Ud[v]) <= 1e-9 * max(ref, 1e-30)
    assert best == int(np.argmax(U))


def test_exact_utility_with_prior_is_positive_and_below_the_prior_variance_sum(sphere_views):
    """With the prior, adding precision can only lower the exact marginal variances (Q' >= Q), so with the same
    probes the estimate drops on average: U > 0 for a view that sees the surface, and U < sum s over the set."""
    w, b = sphere_views
    d, hd, _ = oracle.integrate_w(b, w)
    qd, rhs = oracle.assemble(b, d, hd, w.lam, w.lam_b)
    mu, *_ = oracle.pcg(b, w.lam, qd, rhs, tol=1e-12)
    mu32 = mu.astype(np.float32)
    s, *_ = oracle.hutchinson(b, w.lam, qd, 16, 1, tol=1e-12)
    U, _ = oracle.score_views_exact(b, mu32, qd, w.lam, w.cand_poses[:2], w.cand_intr, w.band_vox, w.sig_a,
                                    w.sig_b, K=16, seed=1, tol=1e-12)
    om = np.abs(mu32.astype(np.float64)) <= 1.0
    assert np.all(U > 0) and np.all(U < np.sum(s[om]))
