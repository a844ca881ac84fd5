"""Pins of the oracle's probe RNG, ray traversal and depth integration
(Sec. 3.5 back-projection, projective SDF, linear rows, noise model; Sec. 3.7
Rademacher probes)."""
import numpy as np

import oracle
import synth
from tests import scenes


def test_splitmix64_published_vectors():
    # SplitMix64 (Steele, Lea & Flood 2014) started from state 0: the first
    # outputs of the reference generator are the mix of k * golden-gamma.
    g = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(g) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * g) % 2 ** 64) == 0x06C45D188009454F


def test_rademacher_probes_are_balanced_and_independent():
    lin = np.arange(1_000_000, dtype=np.int64)
    z0 = oracle.probe(0, 0, lin)
    z1 = oracle.probe(0, 1, lin)
    z0s = oracle.probe(1, 0, lin)
    assert set(np.unique(z0).tolist()) == {-1.0, 1.0}
    for z in (z0, z1, z0s):
        assert abs(z.mean()) < 5e-3            # 5 sigma for 1e6 fair signs
    assert abs(np.mean(z0 * z1)) < 5e-3        # probes uncorrelated
    assert abs(np.mean(z0 * z0s)) < 5e-3       # seeds uncorrelated
    # a pure function of (seed, k, linear index): order independent
    perm = np.random.default_rng(0).permutation(4096)
    np.testing.assert_array_equal(oracle.probe(0, 3, lin[perm]), oracle.probe(0, 3, lin[:4096])[perm])


def _seg_box_overlap(C, r, s0, s1, lo, hi, eps):
    t0, t1 = s0, s1
    for a in range(3):
        if abs(r[a]) < 1e-15:
            if C[a] < lo[a] - eps or C[a] > hi[a] + eps:
                return False
            continue
        u0 = (lo[a] - eps - C[a]) / r[a]
        u1 = (hi[a] + eps - C[a]) / r[a]
        t0, t1 = max(t0, min(u0, u1)), min(t1, max(u0, u1))
    return t0 <= t1


def test_dda_visits_exactly_the_voxels_the_segment_crosses():
    w = synth.make_workload("sphere64", n=32, image_scale=0.5)
    b = oracle.build_band_w(w)
    n, h = w.n, w.h
    org = np.array(w.origin)
    fx, fy, cx, cy, W, H = w.intr
    rng = np.random.default_rng(1)
    tau = w.band_vox * h
    for trial in range(200):
        t = int(rng.integers(w.T))
        px, py = int(rng.integers(W)), int(rng.integers(H))
        D = float(rng.uniform(0.6, 1.2))
        path = oracle.dda_trace(b, w.poses[t], w.intr, px, py, D, w.band_vox)
        assert len(path) > 0
        P = w.poses[t].astype(np.float64)
        dc = np.array([(px + 0.5 - cx) / fx, (py + 0.5 - cy) / fy, 1.0])
        dw = P[:, :3] @ dc
        r = dw / np.linalg.norm(dw)
        C = P[:, 3]
        sp = D * np.linalg.norm(dc)
        s0, s1 = sp - tau, sp + tau
        ijk = [(int(L % n), int((L // n) % n), int(L // (n * n))) for L in path if L >= 0]
        # 6-connected walk, no voxel twice
        for a, c in zip(ijk, ijk[1:]):
            assert sum(abs(x - y) for x, y in zip(a, c)) == 1
        assert len(set(ijk)) == len(ijk)
        # every visited voxel touches the segment
        for v in ijk:
            lo = org + np.array(v) * h
            assert _seg_box_overlap(C, r, s0, s1, lo, lo + h, 1e-5 * h)
        # every segment point lies in a visited voxel (grid interior, away from faces)
        vis = set(ijk)
        for s in np.linspace(s0 + 1e-4 * h, s1 - 1e-4 * h, 400):
            g = (C + s * r - org) / h
            if np.any(g < 0) or np.any(g >= n):
                continue
            fr = g - np.floor(g)
            if np.any(fr < 1e-4) or np.any(fr > 1 - 1e-4):
                continue
            assert tuple(int(x) for x in np.floor(g)) in vis


def test_normal_incidence_samples_equal_the_euclidean_sdf():
    """Camera at the centre of a sphere: every ray meets the surface at normal
    incidence, so the projective sample of a voxel is R - |x| up to the voxel
    centre's offset from the ray: 0 <= y - (R - |x|)/h <= (sqrt(3)/2 h)^2 / (2 |x|) / h."""
    s = scenes.hollow_sphere()
    b = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    d, hd, st = oracle.integrate(b, s["depth"], s["poses"], s["intr"], s["band_vox"], 0.002, 0.0)
    h, R = s["h"], s["R"]
    x = np.linalg.norm(b.centres(), axis=1)
    m = d > 0
    assert m.mean() > 0.9
    y = hd[m] / d[m]
    gt = (R - x[m]) / h
    un = np.abs(gt) <= s["band_vox"] - 0.05          # samples not clamped at +-tau
    bound = (0.75 * h * h) / (2 * x[m]) / h
    err = y - gt
    assert np.all(err[un] >= -1e-9)
    assert np.all(err[un] <= bound[un] + 1e-9)
    # constant sigma: d / w counts observations, an integer
    w = h * h / 0.002 ** 2
    np.testing.assert_allclose(d / w, np.round(d / w), atol=1e-9)
    # clamped voxels see exactly +-tau
    cl = np.abs(gt) > s["band_vox"] + 1.0
    np.testing.assert_allclose(np.abs(y[cl]), s["band_vox"], atol=1e-12)


def test_frontal_plane_weights_follow_the_noise_model():
    s = scenes.frontal_plane()
    b = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    sa, sb, sp = 0.002, 0.004, 0.003
    d1, hd1, _ = oracle.integrate(b, s["depth"], s["poses"], s["intr"], s["band_vox"], sa, sb, sp, 0.0)
    d0, hd0, _ = oracle.integrate(b, s["depth"], s["poses"], s["intr"], s["band_vox"], 1.0, 0.0)
    # every frontal-plane pixel has z-depth 1 m, so w = h^2 / ((a + b)^2 + s_pose^2)
    w = s["h"] ** 2 / ((sa + sb * 1.0) ** 2 + sp ** 2)
    w0 = s["h"] ** 2
    np.testing.assert_allclose(d1 / w, d0 / w0, rtol=1e-5)
    np.testing.assert_allclose(hd1 / d1, hd0 / d0, rtol=1e-12, atol=1e-12)
