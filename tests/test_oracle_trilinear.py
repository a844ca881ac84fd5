"""Pins of the trilinear observation rows (oracle/trilinear.py): the weights
against the definition of linear interpolation, a configuration whose samples
fall on voxel centres (where the rows reduce to one non-zero), and the
structure of the resulting precision (symmetric, 27-point, data-term row sums
equal to A^T w, positive definite)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import trilinear


@pytest.fixture(scope="module")
def sphere():
    w = synth.make_workload("sphere64", n=24, image_scale=0.5, frames=12, noise=False)
    b = oracle.build_band_w(w)
    return w, b


def test_weights_are_a_partition_of_unity_and_reproduce_linear_fields(sphere):
    w, b = sphere
    rng = np.random.default_rng(0)
    c = b.centres()
    # points spread around band voxel centres; keep those whose cell lies in the band
    q = c[rng.integers(0, b.N, 4000)] + rng.uniform(-0.5, 0.5, (4000, 3)) * b.h
    idx, wts, used = trilinear.trilinear_rows(b, q)
    assert used.sum() > 1000
    np.testing.assert_allclose(wts[used].sum(1), 1.0, rtol=0, atol=1e-12)
    assert np.all(wts[used] >= 0)
    coef = np.array([0.3, -1.7, 2.2])
    f = c @ coef + 0.4                                         # a linear field at the voxel centres
    interp = np.sum(wts * f[idx], axis=1)
    np.testing.assert_allclose(interp[used], q[used] @ coef + 0.4, rtol=0, atol=1e-10)
    # the corners are the cell's 8 centres, the lowest at floor of the grid coordinate
    g = (q[used] - np.asarray(b.origin)) / b.h - 0.5
    lo = np.floor(g).astype(np.int64)
    ijk = b.ijk()
    for cc in range(8):
        o = np.array([cc & 1, (cc >> 1) & 1, (cc >> 2) & 1])
        np.testing.assert_array_equal(ijk[idx[used, cc]], lo + o)


def test_samples_on_voxel_centres_give_one_nonzero_rows():
    """The central pixel's ray runs along +z through a column of voxel centres and its depth lands on a centre
    (every coordinate a binary fraction): each sample sits on a centre, so each row is e_j with y = -k."""
    n, h, bv = 16, 1.0 / 64, 3.0
    org = (-n * h / 2,) * 3
    i, j, kz = 8, 7, 9                                         # the hit voxel
    C = np.array([org[0] + (i + 0.5) * h, org[1] + (j + 0.5) * h, -1.0])
    zc = org[2] + (kz + 0.5) * h
    pose = np.concatenate([np.eye(3), C[:, None]], 1)[None].astype(np.float32)
    Wd = Hd = 32
    intr = (32.0, 32.0, 16.5, 16.5, Wd, Hd)                   # pixel (16, 16) looks along +z
    plane = np.full((1, Hd, Wd), zc - C[2], np.float32)         # a frontal plane at the hit depth
    b = oracle.build_band(plane, pose, intr, n, h, org, bv, bv + 2)
    one = np.full_like(plane, np.nan)
    one[0, 16, 16] = plane[0, 16, 16]
    q, y, wv = trilinear.samples(one, pose, intr, h, bv, 0.002, 0.0)
    assert len(q) == 7
    np.testing.assert_array_equal(y, -np.arange(-3, 4).astype(np.float64))
    g = (q - np.asarray(org)) / h - 0.5
    np.testing.assert_array_equal(g, np.round(g))
    idx, wts, used = trilinear.trilinear_rows(b, q)
    assert used.all()
    np.testing.assert_array_equal(wts[:, 0], 1.0)
    np.testing.assert_array_equal(wts[:, 1:], 0.0)
    ijk = b.ijk()[idx[:, 0]]
    np.testing.assert_array_equal(ijk[:, 0], i)
    np.testing.assert_array_equal(ijk[:, 1], j)
    np.testing.assert_array_equal(ijk[:, 2], kz + np.arange(-3, 4))


def test_system_structure(sphere):
    w, b = sphere
    Q, hv, d, m = trilinear.system(b, w.depth, w.poses, w.intr, w.band_vox, w.sig_a, w.sig_b, w.lam, w.lam_b)
    assert m > 0 and Q.shape == (b.N, b.N)
    assert abs(Q - Q.T).max() <= 1e-12 * abs(Q).max()
    # couplings only inside the 3 x 3 x 3 neighbourhood
    coo = Q.tocoo()
    ijk = b.ijk()
    assert np.all(np.abs(ijk[coo.row] - ijk[coo.col]).max(1) <= 1)
    # data term: Q - Q0 has row sums A^T w (trilinear weights sum to one)
    bd = b.bdry.astype(np.float64)
    Q0 = oracle.csr(b, w.lam, w.lam * b.deg.astype(np.float64) + w.lam_b * bd)
    import scipy.sparse
    Q0 = scipy.sparse.csr_matrix((Q0[2], Q0[1], Q0[0]), shape=Q.shape)
    np.testing.assert_allclose(np.asarray((Q - Q0).sum(1)).ravel(), d, rtol=1e-12, atol=1e-12 * d.max())
    # positive definite: the solve of Q x = h has a positive energy and a small residual
    import scipy.sparse.linalg
    x = scipy.sparse.linalg.spsolve(Q.tocsc(), hv)
    assert x @ (Q @ x) > 0
    assert np.linalg.norm(Q @ x - hv) <= 1e-8 * np.linalg.norm(hv)
    dense = Q.toarray() if b.N <= 3000 else None
    if dense is not None:
        np.linalg.cholesky(dense)


def test_normal_incidence_mean_is_the_radial_sdf():
    """Cameras at the centre of a sphere: every sample observes the radial SDF (R - |q|)/h exactly, and the
    trilinear interpolation of that field errs by at most h / (4 |x|) voxel (its Hessian has the two tangential
    eigenvalues 1/(|x| h), and a trilinear cell errs by h^2/8 per unit of second derivative along each axis), about
    0.025 voxel here; the posterior mean near the surface stays within that plus the prior's smoothing."""
    import scipy.sparse.linalg
    from tests import scenes
    s = scenes.hollow_sphere()
    b = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    f = (s["R"] - np.linalg.norm(b.centres(), axis=1)) / s["h"]
    near = np.abs(f) <= 1.0
    errs = []
    for lam in (1.0, 0.1):
        Q, hv, d, m = trilinear.system(b, s["depth"], s["poses"], s["intr"], s["band_vox"], 0.002, 0.0, lam, 1.0)
        assert np.all(d[near] > 0)
        mu = scipy.sparse.linalg.spsolve(Q.tocsc(), hv)
        e = np.abs(mu - f)[near]
        assert e.mean() <= 0.03 and e.max() <= 0.15, (lam, e.mean(), e.max())
        errs.append(e.max())
    assert errs[1] <= errs[0]  # less smoothing, closer to the observed field


def test_fp32_rows_follow_the_fp64_definition(sphere):
    """The FP32-specified rows choose the FP64 definition's cell except for samples within FP32 rounding of a cell
    face, and their weights agree to FP32 precision; the same input gives the same bits."""
    w, b = sphere
    q, y, wv = trilinear.samples(w.depth, w.poses, w.intr, b.h, w.band_vox, w.sig_a, w.sig_b)
    idx, wts, used = trilinear.trilinear_rows(b, q)
    idx32, wts32, used32, y32 = trilinear.rows_fp32(b, w.depth, w.poses, w.intr, w.band_vox)
    assert len(idx32) == len(q)
    np.testing.assert_allclose(y32, y, rtol=0, atol=1e-12)
    g = (q - np.asarray(b.origin)) / b.h - 0.5
    near_face = np.any(np.abs(g - np.round(g)) < 1e-4, axis=1)
    same = ~near_face
    assert same.mean() > 0.99
    np.testing.assert_array_equal(used32[same], used[same])
    both = same & used
    np.testing.assert_array_equal(idx32[both], idx[both])
    np.testing.assert_allclose(wts32[both], wts[both], rtol=0, atol=2e-5)
    again = trilinear.rows_fp32(b, w.depth, w.poses, w.intr, w.band_vox)
    np.testing.assert_array_equal(again[0], idx32)
    np.testing.assert_array_equal(again[1], wts32)


def test_posterior_under_trilinear_rows_matches_dense_algebra():
    """Mean and probe estimate of the 27-point system against a dense solve of the same system and probes."""
    w = synth.make_workload("sphere64", n=16, image_scale=0.25, frames=8, noise=False)
    b = oracle.build_band_w(w)
    assert b.N <= 3000
    K, seed = 6, 7
    mu, s = trilinear.posterior(b, w.depth, w.poses, w.intr, w.band_vox, w.sig_a, w.sig_b, w.lam, w.lam_b, K, seed)
    Q, hv, _, _ = trilinear.system(b, w.depth, w.poses, w.intr, w.band_vox, w.sig_a, w.sig_b, w.lam, w.lam_b)
    Qd = Q.toarray()
    np.testing.assert_allclose(mu, np.linalg.solve(Qd, hv), rtol=0, atol=1e-9 * np.abs(mu).max())
    Z = np.stack([oracle.probe(seed, k, b.lin) for k in range(K)], 1)
    ref = np.mean(Z * np.linalg.solve(Qd, Z), axis=1)
    np.testing.assert_allclose(s, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    # and the probe-averaged value bounds: (Q^-1)_ii >= 1/Q_ii holds for the exact diagonal
    Qi = np.linalg.inv(Qd)
    assert np.all(np.diag(Qi) >= 1.0 / np.diag(Qd) * (1 - 1e-12))


def test_system_from_fp32_rows_is_the_fp64_system_up_to_boundary_samples(sphere):
    """The posterior system assembled from the FP32-specified rows (the form the CUDA path reproduces) has the
    structure of the FP64 one (symmetric, 27-point, d = A^T w) and differs from it only by the rows of samples within
    rounding of a cell face: the FP32 and FP64 A^T W A, d and h agree to within the weight of the few rows whose
    decisions differ (each row's weight is w = h^2/sigma^2 <= w_max)."""
    w, b = sphere
    a = dict(band_vox=w.band_vox, sig_a=w.sig_a, sig_b=w.sig_b, lam=w.lam, lam_b=w.lam_b)
    Q64, h64, d64, n64 = trilinear.system(b, w.depth, w.poses, w.intr, **a)
    Q32, h32, d32, n32 = trilinear.system(b, w.depth, w.poses, w.intr, rows="fp32", **a)
    assert abs(n32 - n64) <= 1e-3 * n64
    D = (Q32 - Q32.T).tocoo()
    assert np.abs(D.data).max(initial=0) <= 1e-12 * np.abs(Q32.data).max()
    wmax = float(trilinear.sample_precisions(w.depth, w.band_vox, b.h, w.sig_a, w.sig_b).max())
    diff = (Q32 - Q64).tocoo()
    nbad = np.count_nonzero(np.abs(diff.data) > 1e-4 * np.abs(Q64.data).max())
    assert nbad <= 0.01 * Q64.nnz
    assert np.abs(diff.data).max(initial=0) <= 8 * wmax * max(abs(n32 - n64), 1)
    np.testing.assert_allclose(d32.sum(), d64.sum(), rtol=1e-3)
    ok = np.abs(d32 - d64) <= 1e-4 * d64.max()
    assert ok.mean() >= 0.99
    # row sums of the data term equal A^T w (the FP32 weights of a row sum to one within a few FP32 ulps)
    Q0, _, _, _ = trilinear.system(b, w.depth[:0], w.poses[:0], w.intr, rows="fp32", **a)
    np.testing.assert_allclose(np.asarray((Q32 - Q0).sum(1)).ravel(), d32, rtol=1e-6, atol=1e-9 * d32.max())
