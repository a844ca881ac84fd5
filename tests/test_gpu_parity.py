"""GPU parity of the CUDA path against the oracle, through the C ABI.

Bars: band / directory / mesh topology bit-exact; observation sums within
FP32 accumulation error; mean within 1e-3 voxel of the FP64 oracle solved to
1e-12; variance from identical probe seeds within 1e-3 relative (relative to
max(|s_i|, 1/Q_ii)); view utilities within 1e-3 relative with the same argmax.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import scenes
from tests.gpu_util import assert_band_equal, ctx, dev, gpu_band, torch

pytestmark = pytest.mark.gpu

MEAN_TOL_VOX = 1e-3
VAR_TOL_REL = 1e-3

WORKLOADS = {
    "sphere64": lambda: synth.make_workload("sphere64"),
    "sphere32_small": lambda: synth.make_workload("sphere64", n=32, image_scale=0.5),
    "union128": lambda: synth.make_workload("union256", n=128, frames=30, image_scale=0.5),
    "blob128_b5": lambda: synth.make_workload("blob512", n=128, frames=40, image_scale=0.25, band_vox=5.0),
}

_cache = {}


def case(name):
    if name not in _cache:
        w = WORKLOADS[name]()
        ob = oracle.build_band_w(w)
        d, hd, _ = oracle.integrate_w(ob, w)
        qd, rhs = oracle.assemble(ob, d, hd, w.lam, w.lam_b)
        mu, st, it, rr = oracle.pcg(ob, w.lam, qd, rhs, tol=1e-12)
        assert st == 0
        _cache[name] = dict(w=w, ob=ob, d=d, hd=hd, qd=qd, rhs=rhs, mu=mu)
    return _cache[name]


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_band_is_bit_exact(name):
    c = case(name)
    gb, _, _ = gpu_band(c["w"])
    assert_band_equal(gb, c["ob"])


def test_frontal_plane_and_empty_and_single_brick_bands():
    s = scenes.frontal_plane()
    w = synth.make_workload("sphere64", n=16, image_scale=0.25)
    C = ctx()
    gb = C.build_band(dev(s["depth"]), dev(s["poses"]), s["intr"], s["n"], s["h"], s["org"], s["band_vox"],
                      s["trunc_vox"])
    ob = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"],
                           s["trunc_vox"])
    assert_band_equal(gb, ob)
    empty = np.zeros_like(w.depth)
    gb = C.build_band(dev(empty), dev(w.poses), w.intr, w.n, w.h, w.origin, w.band_vox, w.trunc_vox)
    assert gb.N == 0 and gb.NB == 0
    # a single-brick grid (n = 8) and host (numpy) inputs
    w8 = synth.make_workload("sphere64", n=8, image_scale=0.25)
    gb = C.build_band(w8.depth, w8.poses, w8.intr, 8, w8.h, w8.origin, 2.0, 4.0)
    ob = oracle.build_band(w8.depth, w8.poses, w8.intr, 8, w8.h, w8.origin, 2.0, 4.0)
    assert_band_equal(gb, ob)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_observations_and_system(name):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    sysg = gb.export_system()
    scale = np.abs(c["d"]).max()
    np.testing.assert_allclose(sysg["d"], c["d"], rtol=1e-4, atol=1e-5 * scale)
    np.testing.assert_allclose(sysg["hdata"], c["hd"], rtol=1e-4, atol=2e-5 * np.abs(c["hd"]).max())
    np.testing.assert_allclose(sysg["qdiag"], c["qd"], rtol=1e-4, atol=1e-5 * scale)
    np.testing.assert_allclose(sysg["rhs"], c["rhs"], rtol=1e-4, atol=2e-5 * np.abs(c["rhs"]).max())


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_spmv_matches_oracle(name):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    qd32 = gb.export_system()["qdiag"].astype(np.float64)
    x = np.random.default_rng(0).standard_normal(gb.N).astype(np.float32)
    y = torch.empty(gb.N, device="cuda")
    gb.spmv(dev(x), y)
    ref = oracle.spmv(c["ob"], w.lam, qd32, x.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    # host buffers through the same call
    yh = np.empty(gb.N, np.float32)
    gb.spmv(x, yh)
    np.testing.assert_array_equal(yh, y.cpu().numpy())
    # arrays that do not start on 16 bytes (the kernel without bulk copies): the same bits
    xb = torch.zeros(gb.N + 3, device="cuda")
    yb = torch.full((gb.N + 3,), 7.0, device="cuda")
    for o in (1, 2, 3):
        xb[o:o + gb.N] = dev(x)
        gb.spmv(xb[o:o + gb.N], yb[o:o + gb.N])
        np.testing.assert_array_equal(yb[o:o + gb.N].cpu().numpy(), y.cpu().numpy())
    assert yb[0].item() == 7.0


def test_spmv_bands_with_ragged_runs_and_tails():
    """Runs that start and end inside 16-byte groups, a band size that is not a multiple of 4 (the last brick's
    tail read directly), single-voxel runs: the bulk-copy SpMV against the oracle on small bands."""
    for n, scale, frames, bv in ((16, 0.25, 4, 1.5), (24, 0.25, 6, 2.0), (32, 0.5, 8, 3.0)):
        w = synth.make_workload("sphere64", n=n, image_scale=scale, frames=frames, band_vox=bv)
        ob = oracle.build_band_w(w)
        gb, depth, poses = gpu_band(w)
        gb.integrate_depth(depth, poses, w.intr)
        qd32 = gb.export_system()["qdiag"].astype(np.float64)
        x = np.random.default_rng(n).standard_normal(gb.N).astype(np.float32)
        y = torch.empty(gb.N, device="cuda")
        gb.spmv(dev(x), y)
        ref = oracle.spmv(ob, w.lam, qd32, x.astype(np.float64))
        np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=0, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("name,R", [("sphere32_small", 8), ("union128", 16), ("blob128_b5", 32), ("sphere64", 32)])
def test_spmm_matches_oracle_and_the_single_rhs_spmv(name, R):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    qd32 = gb.export_system()["qdiag"].astype(np.float64)
    X = np.random.default_rng(R).standard_normal((gb.N, R)).astype(np.float32)
    X[:, R - 1] = 0.0  # a zero column
    Y = torch.empty((gb.N, R), device="cuda")
    gb.spmm(dev(X), Y)
    Y = Y.cpu().numpy()
    y1 = torch.empty(gb.N, device="cuda")
    for col in range(R):
        ref = oracle.spmv(c["ob"], w.lam, qd32, X[:, col].astype(np.float64))
        np.testing.assert_allclose(Y[:, col], ref, rtol=0, atol=1e-5 * max(np.abs(ref).max(), 1.0))
        gb.spmv(dev(np.ascontiguousarray(X[:, col])), y1)
        np.testing.assert_allclose(Y[:, col], y1.cpu().numpy(), rtol=1e-6, atol=1e-6 * np.abs(Y[:, col]).max())
    assert np.all(Y[:, R - 1] == 0.0)
    # host buffers through the same call
    Yh = np.empty((gb.N, R), np.float32)
    gb.spmm(X, Yh)
    np.testing.assert_array_equal(Yh, Y)


def test_spmm_argument_checks():
    c = case("sphere32_small")
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    with pytest.raises(Exception):  # before integration
        gb.spmm(torch.zeros((gb.N, 8), device="cuda"), torch.empty((gb.N, 8), device="cuda"))
    gb.integrate_depth(depth, poses, w.intr)
    with pytest.raises(Exception):
        gb.spmm(torch.zeros((gb.N, 12), device="cuda"), torch.empty((gb.N, 12), device="cuda"))
    with pytest.raises(ValueError):
        gb.spmm(torch.zeros((gb.N, 8), device="cuda"), torch.empty((gb.N, 16), device="cuda"))


@pytest.mark.parametrize("name,fp64,tol", [("sphere64", True, 1e-8), ("sphere64", False, 1e-8),
                                           ("union128", False, 1e-8), ("blob128_b5", False, 1e-8),
                                           ("sphere32_small", True, 1e-10), ("sphere32_small", False, 1e-10)])
def test_mean_matches_oracle(name, fp64, tol):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    mu = torch.empty(gb.N, device="cuda")
    info = gb.solve_mean(mu, rel_tol=tol, fp64=fp64)
    assert info.rel_res <= tol and info.iters > 0
    err = np.abs(mu.cpu().numpy() - c["mu"]).max()
    assert err <= MEAN_TOL_VOX, err


@pytest.mark.parametrize("name", ["union128", "blob128_b5"])
def test_mean_at_1e6_is_within_the_residual_error_bound(name):
    """At rel_tol = 1e-6 the error obeys |mu - mu*|_2 <= |h - Q mu|_2 / lambda_min(Q)
    (FP32 storage of mu adds at most 1 ulp per entry)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    mu = torch.empty(gb.N, device="cuda")
    info = gb.solve_mean(mu, rel_tol=1e-6)
    assert info.rel_res <= 1e-6
    m = mu.cpu().numpy().astype(np.float64)
    rp, ci, val = oracle.csr(c["ob"], w.lam, c["qd"])
    Q = sp.csr_matrix((val, ci, rp), shape=(gb.N, gb.N))
    lmin = sla.eigsh(Q, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    r = np.linalg.norm(c["rhs"] - Q @ m)
    e = np.linalg.norm(m - c["mu"])
    ulp = np.linalg.norm(np.abs(c["mu"]) * 2.0 ** -23)
    assert e <= r / lmin * 1.01 + ulp, (e, r / lmin)


def test_solver_edge_cases():
    c = case("sphere32_small")
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    mu = torch.empty(gb.N, device="cuda")
    info = gb.solve_mean(mu, rel_tol=1e-14, max_iter=2, raise_on_fail=False)
    assert info.status == 4 and info.iters == 2          # BF_NOT_CONVERGED, last iterate kept
    # warm start at the oracle solution needs (almost) no iteration
    mu = dev(c["mu"].astype(np.float32))
    info = gb.solve_mean(mu, rel_tol=1e-5, warm=True)
    assert info.iters <= 2
    # host output buffer
    muh = np.empty(gb.N, np.float32)
    gb.solve_mean(muh, rel_tol=1e-8)
    assert np.abs(muh - c["mu"]).max() <= MEAN_TOL_VOX
    # repeated integration accumulates (twice the data = twice d)
    d1 = gb.export_system()["d"]
    gb.integrate_depth(depth, poses, w.intr)
    np.testing.assert_allclose(gb.export_system()["d"], 2 * d1, rtol=1e-5)
    gb.reset_observations()
    assert np.all(gb.export_system()["d"] == 0)
    with pytest.raises(Exception):
        gb.estimate_variance(torch.empty(gb.N, device="cuda"), K=4, rhs_block=12)


@pytest.mark.parametrize("name,K,R", [("sphere32_small", 16, 8), ("sphere32_small", 20, 16),
                                      ("sphere64", 16, 16), ("union128", 8, 32), ("blob128_b5", 8, 8),
                                      ("sphere32_small", 6, 1)])
def test_variance_matches_oracle_for_identical_probes(name, K, R):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    s = torch.empty(gb.N, device="cuda")
    info = gb.estimate_variance(s, K=K, seed=3, rel_tol=1e-7, rhs_block=R)
    so, st, it, _ = oracle.hutchinson(c["ob"], w.lam, c["qd"], K, 3, tol=1e-12)
    rel = np.abs(s.cpu().numpy() - so) / np.maximum(np.abs(so), 1.0 / c["qd"])
    assert rel.max() <= VAR_TOL_REL, rel.max()
    assert info.iters >= K


def test_variance_does_not_depend_on_the_block_width():
    c = case("sphere32_small")
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    out = []
    for R in (8, 16, 32, 1):
        s = torch.empty(gb.N, device="cuda")
        gb.estimate_variance(s, K=32, seed=9, rel_tol=1e-8, rhs_block=R)
        out.append(s.cpu().numpy())
    for o in out[1:]:
        np.testing.assert_allclose(o, out[0], rtol=2e-4, atol=0)


@pytest.mark.parametrize("name", ["sphere64", "union128"])
def test_marching_cubes_topology_is_bit_exact(name):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    mu32 = c["mu"].astype(np.float32)
    V, F = gb.extract_surface(dev(mu32))
    Vo, Fo = oracle.marching_cubes(c["ob"], mu32)
    assert len(F) > 100
    np.testing.assert_array_equal(F, Fo)
    np.testing.assert_allclose(V, Vo, rtol=0, atol=2e-6 + 1e-5 * w.h)


@pytest.mark.parametrize("name", ["sphere32_small", "sphere64"])
def test_view_scores_match_oracle(name):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    so, *_ = oracle.hutchinson(c["ob"], w.lam, c["qd"], 4, 1, tol=1e-10)
    mu32 = c["mu"].astype(np.float32)
    s32 = so.astype(np.float32)
    qd32 = gb.export_system()["qdiag"].astype(np.float64)
    cand = w.cand_poses[:16]
    U, best = gb.score_views(dev(mu32), dev(s32), dev(cand), w.cand_intr)
    Uo, besto = oracle.score_views(c["ob"], mu32, s32.astype(np.float64), qd32, cand, w.cand_intr, w.band_vox,
                                   w.sig_a, w.sig_b, w.sig_pose, w.sig_model)
    assert Uo.max() > 0
    np.testing.assert_allclose(U, Uo, rtol=1e-3, atol=1e-6 * Uo.max())
    assert best == besto or Uo[best] >= Uo[besto] * (1 - 1e-3)


@pytest.mark.parametrize("name,R", [("sphere32_small", 8), ("union128", 0)])
def test_exact_view_utilities_match_oracle(name, R):
    c = case(name)
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    mu32 = c["mu"].astype(np.float32)
    cand = w.cand_poses[:3]
    K, seed = 8, 2
    U, best, iters = gb.score_views_exact(dev(mu32), dev(cand), w.cand_intr, K_probes=K, seed=seed, rel_tol=1e-10,
                                          rhs_block=R)
    Uo, besto = oracle.score_views_exact(c["ob"], mu32, c["qd"], w.lam, cand, w.cand_intr, w.band_vox, w.sig_a,
                                         w.sig_b, K=K, seed=seed, tol=1e-12, sig_pose=w.sig_pose,
                                         sig_model=w.sig_model)
    assert Uo.max() > 0 and iters > 0
    np.testing.assert_allclose(U, Uo, rtol=1e-3, atol=1e-5 * np.abs(Uo).max())
    assert best == besto or Uo[best] >= Uo[besto] * (1 - 1e-3)
    # the band's own diagonal is left as it was
    s1 = torch.empty(gb.N, device="cuda")
    gb.estimate_variance(s1, K=K, seed=seed, rel_tol=1e-10, rhs_block=R)
    so, *_ = oracle.hutchinson(c["ob"], w.lam, c["qd"], K, seed, tol=1e-12)
    rel = np.abs(s1.cpu().numpy() - so) / np.maximum(np.abs(so), 1.0 / c["qd"])
    assert rel.max() <= VAR_TOL_REL


def test_probe_ranges_sum_to_the_full_estimate():
    from paper_2602_19697_gb300.sharding import estimate_variance_sharded, gpu_part_fn
    c = case("sphere32_small")
    w = c["w"]
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    K = 20
    s = torch.empty(gb.N, device="cuda")
    gb.estimate_variance(s, K=K, seed=5, rel_tol=1e-8, rhs_block=8)
    fn = gpu_part_fn(gb, gb.N, K, seed=5, rel_tol=1e-8, rhs_block=8)
    parts = fn(0, 7) + fn(7, 20)          # two "ranks", each part scaled by 1/K in the library
    np.testing.assert_allclose(parts.cpu().numpy(), s.cpu().numpy(), rtol=2e-5, atol=0)
    one = estimate_variance_sharded(fn, K, 0, 1)   # one rank: no collective
    np.testing.assert_allclose(one.cpu().numpy(), s.cpu().numpy(), rtol=2e-5, atol=0)
    # scale = 1 gives the plain sum
    ssum = torch.empty(gb.N, device="cuda")
    gb.estimate_variance_range(ssum, 0, K, seed=5, rel_tol=1e-8, rhs_block=8, scale=1.0)
    np.testing.assert_allclose(ssum.cpu().numpy() / K, s.cpu().numpy(), rtol=2e-5, atol=0)


def test_autotuner_choice_cache_and_library_default(tmp_path, monkeypatch):
    c = case("sphere32_small")
    w = c["w"]
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("BFSDF_TUNE_CACHE", str(path))
    from paper_2602_19697_gb300 import bfsdf
    ctx1 = bfsdf.Context(0)
    depth, poses = dev(w.depth), dev(w.poses)
    b1 = ctx1.build_band_w(w, depth, poses)
    b1.integrate_depth(depth, poses, w.intr)
    R, ms = b1.autotune_rhs_block(64, force=True)
    assert R in (8, 16, 32) and np.all(ms > 0)
    lines = path.read_text().strip().splitlines()
    assert len(lines) == 1 and f'"R": {R}' in lines[0]
    # a second context on the same GPU takes the choice from the file without measuring
    ctx2 = bfsdf.Context(0)
    b2 = ctx2.build_band_w(w, depth, poses)
    b2.integrate_depth(depth, poses, w.intr)
    R2, ms2 = b2.autotune_rhs_block(64)
    assert R2 == R
    np.testing.assert_allclose(ms2, ms, rtol=1e-5)
    assert len(path.read_text().strip().splitlines()) == 1
    # the library's default block width gives the estimate of that width
    s0, sR = torch.empty(b2.N, device="cuda"), torch.empty(b2.N, device="cuda")
    b2.estimate_variance(s0, K=64, seed=2, rel_tol=1e-8, rhs_block=0)
    b2.estimate_variance(sR, K=64, seed=2, rel_tol=1e-8, rhs_block=R)
    np.testing.assert_allclose(s0.cpu().numpy(), sR.cpu().numpy(), rtol=1e-6)
    # a small K never tunes a block wider than it needs
    Rs, mss = b2.autotune_rhs_block(8, force=True)
    assert Rs == 8 and mss[1] == 0 and mss[2] == 0
