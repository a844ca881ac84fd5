"""Pins of the oracle's band builder (Sec. 3.3 TSDF bootstrap and band,
Sec. 3.4 sparse bricks) against closed forms and brute force."""
import numpy as np
import pytest

import oracle
import synth
from tests import scenes


def test_frontal_plane_band_is_the_exact_slab():
    s = scenes.frontal_plane()
    b = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    n, h = s["n"], s["h"]
    c = b.centres()
    dz = c[:, 2] - s["Z0"]
    # closed form: band = voxels with |z - Z0| <= b h  (Z0 is 0.37 h off a centre)
    ks = [k for k in range(n) if abs(s["org"][2] + (k + 0.5) * h - s["Z0"]) <= s["band_vox"] * h]
    assert len(ks) == 6
    assert b.N == n * n * len(ks)
    assert sorted(set(b.ijk()[:, 2].tolist())) == ks
    # TSDF of a frontal plane is exactly the signed distance z - Z0 (FP32 rounding only)
    np.testing.assert_allclose(b.tsdf, dz, atol=2e-6)
    assert np.all(b.wcount > 0)
    # boundary: outermost layers and the grid's side faces
    ijk = b.ijk()
    side = (ijk[:, 0] == 0) | (ijk[:, 0] == n - 1) | (ijk[:, 1] == 0) | (ijk[:, 1] == n - 1)
    outer = (ijk[:, 2] == ks[0]) | (ijk[:, 2] == ks[-1])
    np.testing.assert_array_equal(b.bdry.astype(bool), side | outer)
    exp_deg = 6 - (ijk[:, 0] == 0) - (ijk[:, 0] == n - 1) - (ijk[:, 1] == 0) - (ijk[:, 1] == n - 1) - outer
    np.testing.assert_array_equal(b.deg, exp_deg)


def _brute_force_band(depth, poses, intr, n, h, org, band_vox, trunc_vox):
    """Independent vectorised FP32 TSDF over the WHOLE grid (no candidate
    bricks), numpy float32 ops (each rounded separately, no FMA)."""
    f32 = np.float32
    fx, fy, cx, cy, W, H = [f32(v) for v in intr]
    Wi, Hi = int(intr[4]), int(intr[5])
    i = np.arange(n, dtype=np.float32)
    ax = [f32(org[a]) + (i + f32(0.5)) * f32(h) for a in range(3)]
    X, Y, Z = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
    S = np.zeros(X.shape, np.float32)
    cnt = np.zeros(X.shape, np.int32)
    tauc = f32(trunc_vox) * f32(h)
    beta = f32(band_vox) * f32(h)
    for t in range(depth.shape[0]):
        P = poses[t].astype(np.float32)
        R, C = P[:, :3], P[:, 3]
        dx, dy, dz = X - C[0], Y - C[1], Z - C[2]
        xc = (R[0, 0] * dx + R[1, 0] * dy) + R[2, 0] * dz
        yc = (R[0, 1] * dx + R[1, 1] * dy) + R[2, 1] * dz
        zc = (R[0, 2] * dx + R[1, 2] * dy) + R[2, 2] * dz
        with np.errstate(divide="ignore", invalid="ignore"):
            u = (fx * xc) / zc + cx
            v = (fy * yc) / zc + cy
        vis = (zc > 0) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
        px = np.where(vis, u, 0).astype(np.int64)
        py = np.where(vis, v, 0).astype(np.int64)
        D = depth[t][py.clip(0, Hi - 1), px.clip(0, Wi - 1)]
        ok = vis & (D > 0) & np.isfinite(D)
        sdf = D - zc
        ok &= ~(sdf < -tauc)
        smp = np.minimum(sdf, tauc)
        S = np.where(ok, S + smp, S)
        cnt += ok
    with np.errstate(divide="ignore", invalid="ignore"):
        ts = np.where(cnt > 0, S / cnt.astype(np.float32), 0).astype(np.float32)
    band = (cnt > 0) & (np.abs(ts) <= beta)
    return band, ts, cnt


@pytest.mark.parametrize("case", ["sphere", "union"])
def test_band_matches_whole_grid_brute_force(case):
    if case == "sphere":
        w = synth.make_workload("sphere64", n=32, image_scale=0.5)
    else:
        w = synth.make_workload("union256", n=48, frames=12, image_scale=0.15)
    b = oracle.build_band_w(w)
    band, ts, cnt = _brute_force_band(w.depth, w.poses, w.intr, w.n, w.h, w.origin, w.band_vox, w.trunc_vox)
    n = w.n
    ijk = b.ijk()
    got = np.zeros((n, n, n), bool)
    got[ijk[:, 0], ijk[:, 1], ijk[:, 2]] = True
    assert b.N > 1000
    # the candidate-brick restriction loses no band voxel, and the band is the same set
    np.testing.assert_array_equal(got, band)
    # TSDF values bit-identical under the FP32 specification
    np.testing.assert_array_equal(b.tsdf, ts[ijk[:, 0], ijk[:, 1], ijk[:, 2]])
    np.testing.assert_array_equal(b.wcount, cnt[ijk[:, 0], ijk[:, 1], ijk[:, 2]])


def test_brick_directory_invariants():
    w = synth.make_workload("sphere64")
    b = oracle.build_band_w(w)
    nb = w.n // 8
    ranks = b.dir[b.dir >= 0]
    # ranks are 0..NB-1 in ascending linear brick index
    np.testing.assert_array_equal(ranks, np.arange(b.NB))
    lin_b = np.nonzero(b.dir >= 0)[0]
    np.testing.assert_array_equal(b.bcoord[:, 0] + nb * (b.bcoord[:, 1] + nb * b.bcoord[:, 2]), lin_b)
    pc = np.array([sum(bin(int(x)).count("1") for x in row) for row in b.mask])
    assert pc.sum() == b.N and np.all(pc > 0)
    np.testing.assert_array_equal(np.diff(b.off), pc)
    # compact order: (brick rank, local index) ascending
    ijk = b.ijk()
    brick = b.dir[(ijk[:, 0] >> 3) + nb * ((ijk[:, 1] >> 3) + nb * (ijk[:, 2] >> 3))]
    local = (ijk[:, 0] & 7) + 8 * (ijk[:, 1] & 7) + 64 * (ijk[:, 2] & 7)
    key = brick.astype(np.int64) * 512 + local
    assert np.all(np.diff(key) > 0)
    # band_index round trip
    for v in range(0, b.N, 997):
        assert b.index(*ijk[v]) == v
    # neighbour bricks
    for r in range(b.NB):
        for f in range(6):
            q = b.bcoord[r].copy()
            q[f >> 1] += 1 if f & 1 else -1
            exp = b.dir[q[0] + nb * (q[1] + nb * q[2])] if np.all((q >= 0) & (q < nb)) else -1
            assert b.nbr[r, f] == exp
    # degree / boundary by brute force over the dense band mask
    n = w.n
    m = np.zeros((n + 2, n + 2, n + 2), bool)
    m[ijk[:, 0] + 1, ijk[:, 1] + 1, ijk[:, 2] + 1] = True
    i, j, k = ijk[:, 0] + 1, ijk[:, 1] + 1, ijk[:, 2] + 1
    deg = (m[i - 1, j, k].astype(int) + m[i + 1, j, k] + m[i, j - 1, k] + m[i, j + 1, k] + m[i, j, k - 1] + m[i, j, k + 1])
    np.testing.assert_array_equal(b.deg, deg)
    np.testing.assert_array_equal(b.bdry, (deg < 6).astype(np.uint8))


def test_empty_inputs_give_an_empty_band():
    w = synth.make_workload("sphere64", n=16, image_scale=0.25)
    d = np.zeros_like(w.depth)
    b = oracle.build_band(d, w.poses, w.intr, w.n, w.h, w.origin, w.band_vox, w.trunc_vox)
    assert b.N == 0 and b.NB == 0 and b.n_cand == 0
    d[:] = np.nan
    b = oracle.build_band(d, w.poses, w.intr, w.n, w.h, w.origin, w.band_vox, w.trunc_vox)
    assert b.N == 0
