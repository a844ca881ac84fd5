"""GPU parity of the trilinear observation rows and the 27-point precision
(Sec. 3.5 linear row of trilinear weights, one per cell corner; Sec. 3.6 precision and mean
equations; Sec. 3.7 estimator) against oracle/trilinear.py.

Bars: the rows (cells, weights, which samples count) bit-exact against the
oracle's FP32 specification; the 27-point coefficients, d and h within FP32
accumulation error of the oracle's FP64 sums over the same rows; y = Q x
against the oracle's sparse Q; the mean within 1e-3 voxel of the oracle's
direct solve (at rel_tol 1e-8); the probe estimate within 1e-3 relative of
the oracle's with the same probes (at rel_tol 1e-6).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import trilinear
from tests.gpu_util import ctx, dev, gpu_band, torch
from paper_2602_19697_gb300 import bfsdf

pytestmark = pytest.mark.gpu

WORKLOADS = {
    "sphere24": lambda: synth.make_workload("sphere64", n=24, image_scale=0.5, frames=12),
    "union64": lambda: synth.make_workload("union256", n=64, frames=12, image_scale=0.25),
}
_cache = {}


def case(name):
    if name not in _cache:
        w = WORKLOADS[name]()
        ob = oracle.build_band_w(w)
        a = dict(band_vox=w.band_vox, sig_a=w.sig_a, sig_b=w.sig_b, lam=w.lam, lam_b=w.lam_b, sig_pose=w.sig_pose,
                 sig_model=w.sig_model)
        Q, hv, d, nused = trilinear.system(ob, w.depth, w.poses, w.intr, rows="fp32", **a)
        gb, depth, poses = gpu_band(w)
        gb.integrate_depth(depth, poses, w.intr, trilinear=True)
        _cache[name] = dict(w=w, ob=ob, Q=Q.tocsr(), hv=hv, d=d, a=a, gb=gb, depth=depth, poses=poses)
    return _cache[name]


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_rows_are_bit_exact(name):
    c = case(name)
    w, gb = c["w"], c["gb"]
    idx, wts, used = gb.export_trilinear_rows(c["depth"], c["poses"], w.intr)
    i32, w32, u32, _ = trilinear.rows_fp32(c["ob"], w.depth, w.poses, w.intr, w.band_vox)
    ns = 2 * int(np.floor(w.band_vox + 1e-9)) + 1
    valid = np.isfinite(w.depth) & (w.depth > 0)
    sel = np.repeat(valid.reshape(-1), ns)
    assert used.shape == sel.shape and not used[~sel].any()
    np.testing.assert_array_equal(used[sel], u32)
    np.testing.assert_array_equal(wts[sel].view(np.uint32), w32.astype(np.float32).view(np.uint32))
    np.testing.assert_array_equal(idx[sel], i32)
    assert u32.sum() > 1000


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_precision27_and_observations(name):
    c = case(name)
    gb, ob, Q = c["gb"], c["ob"], c["Q"]
    coef = gb.export_precision27().astype(np.float64)
    n = ob.n
    ijk = ob.ijk()
    cmap = trilinear.compact_map(ob)
    scale = np.abs(Q.data).max()
    for o in range(27):
        off = np.array([o % 3 - 1, (o // 3) % 3 - 1, o // 9 - 1])
        nb = ijk + off
        inside = np.all((nb >= 0) & (nb < n), axis=1)
        u = np.where(inside, cmap[np.where(inside, nb[:, 0] + n * (nb[:, 1] + n * nb[:, 2]), 0)], -1)
        ref = np.zeros(ob.N)
        has = u >= 0
        ref[has] = np.asarray(Q[np.arange(ob.N)[has], u[has]]).ravel()
        np.testing.assert_allclose(coef[o], ref, rtol=1e-4, atol=2e-6 * scale, err_msg=f"offset {o}")
    sy = gb.export_system()
    np.testing.assert_allclose(sy["d"], c["d"], rtol=1e-4, atol=2e-6 * c["d"].max())
    np.testing.assert_allclose(sy["rhs"], c["hv"], rtol=1e-4, atol=2e-6 * np.abs(c["hv"]).max())
    np.testing.assert_array_equal(sy["qdiag"], coef[13].astype(np.float32))


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_spmv27_matches_oracle(name):
    c = case(name)
    gb = c["gb"]
    x = np.random.default_rng(3).standard_normal(gb.N).astype(np.float32)
    y = torch.empty(gb.N, device="cuda")
    gb.spmv(dev(x), y)
    ref = c["Q"] @ x.astype(np.float64)
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=0, atol=2e-5 * np.abs(ref).max())


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_mean_and_variance_match_oracle(name):
    import scipy.sparse.linalg
    c = case(name)
    w, gb, ob = c["w"], c["gb"], c["ob"]
    mu_o = scipy.sparse.linalg.spsolve(c["Q"].tocsc(), c["hv"])
    mu = torch.empty(gb.N, device="cuda")
    info = gb.solve_mean(mu, rel_tol=1e-8)
    assert info.rel_res <= 1e-8
    assert np.abs(mu.cpu().numpy() - mu_o).max() <= 1e-3
    K, seed = 12, 4
    Z = np.stack([oracle.probe(seed, k, ob.lin) for k in range(K)], 1)
    X, st, _ = oracle.block_pcg(ob, w.lam, None, Z, tol=1e-12, Q=c["Q"])
    assert st == 0
    s_o = np.mean(Z * X, axis=1)
    s = torch.empty(gb.N, device="cuda")
    iv = gb.estimate_variance(s, K=K, seed=seed, rel_tol=1e-6)
    assert iv.iters >= K
    qd = c["Q"].diagonal()
    rel = np.abs(s.cpu().numpy() - s_o) / np.maximum(np.abs(s_o), 1.0 / qd)
    assert rel.max() <= 1e-3, rel.max()
    # a probe range scaled by 1/K and the rest add up to the same estimate
    p0, p1 = torch.empty(gb.N, device="cuda"), torch.empty(gb.N, device="cuda")
    gb.estimate_variance_range(p0, 0, 5, seed=seed, rel_tol=1e-6, scale=1.0 / K)
    gb.estimate_variance_range(p1, 5, K, seed=seed, rel_tol=1e-6, scale=1.0 / K)
    np.testing.assert_allclose((p0 + p1).cpu().numpy(), s.cpu().numpy(), rtol=1e-4, atol=1e-6 * np.abs(s_o).max())


def test_trilinear_band_state_rules():
    w = WORKLOADS["sphere24"]()
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr, trilinear=True)
    lib, C = gb.ctx.lib, gb.ctx
    # the other kind of rows, and the 7-point-only calls, are refused
    st = lib.bf_integrate_depth(C._p, gb._p, bfsdf._ptr(depth), int(depth.shape[0]), bfsdf._ptr(poses),
                                __import__("ctypes").byref(bfsdf._intr(w.intr)))
    assert st == bfsdf.BF_ESTATE
    X = torch.zeros((gb.N, 8), device="cuda")
    assert lib.bf_spmm(C._p, gb._p, bfsdf._ptr(X), 8, bfsdf._ptr(X)) == bfsdf.BF_ESTATE
    mu = torch.zeros(gb.N, device="cuda")
    assert lib.bf_solve_mean(C._p, gb._p, 1e-6, 100, bfsdf.BF_SOLVE_WARM, bfsdf._ptr(mu), None, None) == \
        bfsdf.BF_EINVAL
    s = torch.zeros(gb.N, device="cuda")
    assert lib.bf_estimate_variance(C._p, gb._p, 8, 0, 1e-6, 100, 16, 0, bfsdf._ptr(s), None) == bfsdf.BF_EINVAL
    # deterministic and trilinear together are refused; after a reset the band takes either kind again
    import ctypes
    st = lib.bf_integrate_depth_ex(C._p, gb._p, bfsdf._ptr(depth), int(depth.shape[0]), bfsdf._ptr(poses),
                                   ctypes.byref(bfsdf._intr(w.intr)), 3)
    assert st == bfsdf.BF_EINVAL
    gb.reset_observations()
    gb.integrate_depth(depth, poses, w.intr)
    assert lib.bf_export_precision27(C._p, gb._p, bfsdf._ptr(torch.zeros(27 * gb.N, device="cuda"))) == \
        bfsdf.BF_ESTATE
