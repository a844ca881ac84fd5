"""Trilinear observation rows (Sec. 3.5: the linear relation y_i ~ a_i^T x whose
row holds the eight trilinear weights of the sample point, one per cell corner) and the posterior
system they give (Sec. 3.6: Q = Q0 + A^T W A, h = A^T W y + b0).

TEST INFRASTRUCTURE: the FP64 reference of the trilinear form of the
observation model (the CUDA path's BF_INTEGRATE_TRILINEAR rows and 27-point
precision are checked against it).  Only tests may use this module.

Readings (where Sec. 3.5 leaves the sample placement open):
  * a valid pixel (depth D > 0 and finite) gives the ray r = R d_c / |d_c|,
    d_c = ((u + 1/2 - cx)/fx, (v + 1/2 - cy)/fy, 1), from the camera centre
    C, hitting p = C + D R d_c at the distance s_p = D |d_c| along the ray;
  * samples sit on the ray at s_k = s_p + k h for the integers k with
    |k| h <= tau (tau = b h, b the band half-width in voxels): 2b + 1 per ray;
  * each sample q_k observes the projective SDF y_k = clamp(<n, q_k - p>,
    -tau, tau)/h with n = -r, i.e. y_k = (s_p - s_k)/h = -k (voxel units);
  * its row a_k holds the trilinear weights of q_k in the cell of the 8 voxel
    centres around it; a sample is used when every corner with a non-zero
    weight is a band voxel (a sample on a centre needs that centre only);
  * precision w = h^2 / sigma^2 with sigma^2 = (sig_a + sig_b D^2)^2 +
    sig_pose^2 + sig_model^2, as for the voxel-binned rows.
The prior is the one of the CUDA path: lambda (deg_j x_j - sum of the band
6-neighbours) + lambda_b on the diagonal of the band boundary, and lambda_b
tsdf_j / h in h.

FP32 specification of the row decisions (`rows_fp32`), for a kernel that must
choose the same cells and weights bit for bit: every operation an IEEE FP32
operation rounded on its own (no fused multiply-add), in this order --
  dx = (u + 0.5 - cx) / fx,  dy = (v + 0.5 - cy) / fy   [((u + 0.5) - cx) / fx]
  nrm = sqrt((dx dx + dy dy) + 1)
  r_i = ((R_i0 dx + R_i1 dy) + R_i2) / nrm
  s = D nrm + k h,  q_i = C_i + s r_i
  g_i = (q_i - o_i) / h - 0.5,  i0_i = floor(g_i),  f_i = g_i - i0_i
  weight of corner c = (w_x w_y) w_z, w = f_i for an upper corner, 1 - f_i for a lower one
and a corner counts when its FP32 weight is not 0.
"""
from __future__ import annotations

import numpy as np


def samples(depth, poses, intr, h, band_vox, sig_a, sig_b, sig_pose=0.0, sig_model=0.0):
    """Sample points q [M,3] (metres), observations y [M] (voxels) and precisions w [M] of all valid pixels."""
    depth = np.asarray(depth, np.float64)
    poses = np.asarray(poses, np.float64)
    fx, fy, cx, cy, W, H = intr
    b = int(np.floor(band_vox + 1e-9))
    ks = np.arange(-b, b + 1, dtype=np.float64)
    qs, ys, ws = [], [], []
    vv, uu = np.mgrid[0:H, 0:W]
    dc = np.stack([(uu + 0.5 - cx) / fx, (vv + 0.5 - cy) / fy, np.ones((H, W))], -1).reshape(-1, 3)
    ndc = np.linalg.norm(dc, axis=1)
    for t in range(depth.shape[0]):
        Dp = depth[t].reshape(-1)
        ok = np.isfinite(Dp) & (Dp > 0)
        if not np.any(ok):
            continue
        Rm, C = poses[t][:, :3], poses[t][:, 3]
        r = (dc[ok] @ Rm.T) / ndc[ok][:, None]
        sp = Dp[ok] * ndc[ok]
        s = sp[:, None] + ks[None, :] * h                       # [P, 2b+1]
        q = C[None, None, :] + s[..., None] * r[:, None, :]
        sig2 = (sig_a + sig_b * Dp[ok] ** 2) ** 2 + sig_pose ** 2 + sig_model ** 2
        w = np.repeat((h * h / sig2)[:, None], ks.size, 1)
        y = np.clip(sp[:, None] - s, -band_vox * h, band_vox * h) / h
        qs.append(q.reshape(-1, 3))
        ys.append(y.reshape(-1))
        ws.append(w.reshape(-1))
    if not qs:
        return np.zeros((0, 3)), np.zeros(0), np.zeros(0)
    return np.concatenate(qs), np.concatenate(ys), np.concatenate(ws)


def compact_map(band) -> np.ndarray:
    """Dense map linear grid index -> compact band index (-1 outside the band)."""
    m = np.full(band.n ** 3, -1, np.int64)
    m[np.asarray(band.lin, np.int64)] = np.arange(band.N)
    return m


def trilinear_rows(band, q, cmap=None):
    """For points q [M,3]: (idx [M,8] compact indices of the cell corners, wts [M,8] trilinear weights, used [M]),
    corner c = (c & 1, (c >> 1) & 1, (c >> 2) & 1) offsets from the cell's lowest centre; a row is used when every
    corner with a non-zero weight is a band voxel (idx of a zero-weight corner outside the band is 0; unused rows
    have idx and wts 0)."""
    n, h = band.n, band.h
    cmap = compact_map(band) if cmap is None else cmap
    g = (np.asarray(q, np.float64) - np.asarray(band.origin, np.float64)) / h - 0.5
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    idx = np.zeros((len(g), 8), np.int64)
    wts = np.zeros((len(g), 8), np.float64)
    used = np.ones(len(g), bool)
    for c in range(8):
        o = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        ii = i0 + o
        wc = np.prod(np.where(o[None, :] == 1, f, 1.0 - f), axis=1)
        inside = np.all((ii >= 0) & (ii < n), axis=1)
        lin = np.where(inside, ii[:, 0] + n * (ii[:, 1] + n * ii[:, 2]), 0)
        j = np.where(inside, cmap[lin], -1)
        used &= (j >= 0) | (wc == 0.0)
        idx[:, c] = np.maximum(j, 0)
        wts[:, c] = wc
    idx[~used] = 0
    wts[~used] = 0.0
    return idx, wts, used


def sample_precisions(depth, band_vox, h, sig_a, sig_b, sig_pose=0.0, sig_model=0.0):
    """w [M] of the samples of ``rows_fp32`` (same order: frames, valid pixels row by row, k), in FP64 from the
    measured depth: h^2 / ((sig_a + sig_b D^2)^2 + sig_pose^2 + sig_model^2)."""
    b = int(np.floor(band_vox + 1e-9))
    out = []
    for Dt in np.asarray(depth, np.float32):
        D = Dt[np.isfinite(Dt) & (Dt > 0)].astype(np.float64)
        sig2 = (sig_a + sig_b * D ** 2) ** 2 + sig_pose ** 2 + sig_model ** 2
        out.append(np.repeat(h * h / sig2, 2 * b + 1))
    return np.concatenate(out) if out else np.zeros(0)


def system(band, depth, poses, intr, band_vox, sig_a, sig_b, lam, lam_b, sig_pose=0.0, sig_model=0.0, rows="fp64"):
    """(Q scipy CSR [N,N], h [N], d [N] = A^T w, number of used samples): the posterior precision and information
    vector with trilinear observation rows.  rows="fp64": cells and weights from the FP64 sample points
    (``samples``, ``trilinear_rows``); rows="fp32": the rows of the FP32 specification (``rows_fp32``), the form a
    kernel reproduces bit for bit (the two differ only for samples within rounding of a cell boundary); the sums
    are FP64 either way."""
    import scipy.sparse

    from . import csr
    if rows == "fp32":
        idx, wts, used, y = rows_fp32(band, depth, poses, intr, band_vox)
        w = sample_precisions(depth, band_vox, band.h, sig_a, sig_b, sig_pose, sig_model)
        wts = wts.astype(np.float64)
    else:
        q, y, w = samples(depth, poses, intr, band.h, band_vox, sig_a, sig_b, sig_pose, sig_model)
        idx, wts, used = trilinear_rows(band, q)
    idx, wts, y, w = idx[used], wts[used], y[used], w[used]
    N = band.N
    # A^T W A: for every row, w a a^T over its 8 x 8 corner pairs
    ri = np.repeat(idx, 8, axis=1).reshape(-1)
    ci = np.tile(idx, (1, 8)).reshape(-1)
    vals = (w[:, None, None] * wts[:, :, None] * wts[:, None, :]).reshape(-1)
    AtWA = scipy.sparse.coo_matrix((vals, (ri, ci)), shape=(N, N)).tocsr()
    d = np.bincount(idx.reshape(-1), weights=(w[:, None] * wts).reshape(-1), minlength=N)
    hd = np.bincount(idx.reshape(-1), weights=(w[:, None] * wts * y[:, None]).reshape(-1), minlength=N)
    bd = np.asarray(band.bdry, np.float64)
    prior_diag = lam * np.asarray(band.deg, np.float64) + lam_b * bd
    indptr, indices, data = csr(band, lam, prior_diag)
    Q0 = scipy.sparse.csr_matrix((data, indices, indptr), shape=(N, N))
    hvec = hd + lam_b * bd * np.asarray(band.tsdf, np.float64) / band.h
    return (Q0 + AtWA).tocsr(), hvec, d, int(used.sum())


def rows_fp32(band, depth, poses, intr, band_vox, cmap=None):
    """The samples' rows under the FP32 specification above: (idx [M,8], wts [M,8] float32, used [M], y [M]),
    samples in the order of ``samples`` (frames, then pixels row by row, then k)."""
    f32 = np.float32
    fx, fy, cx, cy, W, H = (f32(intr[0]), f32(intr[1]), f32(intr[2]), f32(intr[3]), int(intr[4]), int(intr[5]))
    h = f32(band.h)
    org = np.asarray(band.origin, f32)
    n = band.n
    cmap = compact_map(band) if cmap is None else cmap
    b = int(np.floor(band_vox + 1e-9))
    ks = np.arange(-b, b + 1).astype(f32)
    vv, uu = np.mgrid[0:H, 0:W]
    dx = ((uu.astype(f32) + f32(0.5)) - cx) / fx
    dy = ((vv.astype(f32) + f32(0.5)) - cy) / fy
    nrm = np.sqrt((dx * dx + dy * dy) + f32(1.0))
    idxs, wtss, useds, ys = [], [], [], []
    depth = np.asarray(depth, f32)
    poses = np.asarray(poses, f32)
    for t in range(depth.shape[0]):
        Dp = depth[t]
        ok = np.isfinite(Dp) & (Dp > 0)
        if not np.any(ok):
            continue
        Rm, C = poses[t][:, :3], poses[t][:, 3]
        r = [((Rm[i, 0] * dx[ok] + Rm[i, 1] * dy[ok]) + Rm[i, 2]) / nrm[ok] for i in range(3)]
        sp = Dp[ok] * nrm[ok]
        s = sp[:, None] + ks[None, :] * h
        g = np.stack([(((C[i] + s * r[i][:, None]) - org[i]) / h) - f32(0.5) for i in range(3)], -1).reshape(-1, 3)
        i0 = np.floor(g)
        fr = g - i0
        i0 = i0.astype(np.int64)
        M = len(g)
        idx = np.zeros((M, 8), np.int64)
        wts = np.zeros((M, 8), f32)
        used = np.ones(M, bool)
        for c in range(8):
            o = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
            wv = [fr[:, i] if o[i] else f32(1.0) - fr[:, i] for i in range(3)]
            wc = (wv[0] * wv[1]) * wv[2]
            ii = i0 + np.array(o)
            inside = np.all((ii >= 0) & (ii < n), axis=1)
            lin = np.where(inside, ii[:, 0] + n * (ii[:, 1] + n * ii[:, 2]), 0)
            j = np.where(inside, cmap[lin], -1)
            used &= (j >= 0) | (wc == 0)
            idx[:, c] = np.maximum(j, 0)
            wts[:, c] = wc
        idx[~used] = 0
        wts[~used] = 0
        idxs.append(idx)
        wtss.append(wts)
        useds.append(used)
        ys.append(np.repeat(-ks[None, :], len(sp), 0).reshape(-1).astype(np.float64))
    if not idxs:
        return np.zeros((0, 8), np.int64), np.zeros((0, 8), f32), np.zeros(0, bool), np.zeros(0)
    return np.concatenate(idxs), np.concatenate(wtss), np.concatenate(useds), np.concatenate(ys)


def posterior(band, depth, poses, intr, band_vox, sig_a, sig_b, lam, lam_b, K, seed, tol=1e-12, sig_pose=0.0,
              sig_model=0.0, rows="fp64"):
    """(mu [N], s [N]) under trilinear rows: the MAP mean Q mu = h (sparse direct solve) and the K-probe estimate
    s = (1/K) sum_k z_k (.) Q^-1 z_k with the probes of ``oracle.probe`` (block PCG over the K columns); rows as in
    ``system``."""
    import scipy.sparse.linalg

    from . import block_pcg, probe
    Q, hv, _, _ = system(band, depth, poses, intr, band_vox, sig_a, sig_b, lam, lam_b, sig_pose, sig_model, rows)
    mu = scipy.sparse.linalg.spsolve(Q.tocsc(), hv)
    Z = np.stack([probe(seed, k, band.lin) for k in range(K)], 1)
    X, st, _ = block_pcg(band, lam, None, Z, tol=tol, Q=Q)
    if st != 0:
        raise RuntimeError("block PCG did not converge")
    return mu, np.mean(Z * X, axis=1)
