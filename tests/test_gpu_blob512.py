"""GPU parity on the 200-frame object sequence at full size.

blob512: spherical-harmonic blob in a 512^3 grid at 2 mm, band +-24 voxels
(N = 7.2 M band voxels in 18.8 k bricks), 200 frames 512x384 on a spiral
with 2 mm pose jitter.  Band bit-exact; the mean solve meets the benchmark
tolerance 1e-6 in the oracle's FP64 system and is within 1e-3 voxel of the
FP64 oracle (solved to 1e-12) at 1e-8; the variance of all 128 probes in the
benchmark's call (bf_estimate_variance, K = 128, rel_tol 1e-6, block width
chosen by the autotuner) within 1e-3 relative of the oracle's 128-probe
estimate at every band voxel, and the probe-sharded form (two probe ranges,
each scaled by 1/K in the library, summed) equal to it; mesh topology
bit-exact; view utilities of a few candidates.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_band_equal, dev, gpu_band, torch

pytestmark = pytest.mark.gpu

K, SEED = 128, 0


@pytest.fixture(scope="module")
def blob():
    w = synth.make_workload("blob512")
    ob = oracle.build_band_w(w)
    d, hd, _ = oracle.integrate_w(ob, w)
    qd, rhs = oracle.assemble(ob, d, hd, w.lam, w.lam_b)
    mu, st, _, _ = oracle.pcg(ob, w.lam, qd, rhs, tol=1e-12)
    assert st == 0
    s, st, _, _ = oracle.hutchinson(ob, w.lam, qd, K, SEED, tol=1e-12)
    assert st == 0
    gb, depth, poses = gpu_band(w)
    gb.integrate_depth(depth, poses, w.intr)
    return dict(w=w, ob=ob, d=d, hd=hd, qd=qd, rhs=rhs, mu=mu, s=s, gb=gb)


def test_blob_band_is_bit_exact(blob):
    assert blob["gb"].N > 5_000_000
    assert_band_equal(blob["gb"], blob["ob"])


def test_blob_system(blob):
    sg = blob["gb"].export_system()
    for k, ref in (("d", blob["d"]), ("hdata", blob["hd"]), ("qdiag", blob["qd"]), ("rhs", blob["rhs"])):
        np.testing.assert_allclose(sg[k], ref, rtol=1e-4, atol=2e-5 * np.abs(ref).max(), err_msg=k)


def test_blob_mean_meets_the_residual_at_1e6_and_the_oracle_at_1e8(blob):
    import scipy.sparse as sp
    gb, w = blob["gb"], blob["w"]
    mu = torch.empty(gb.N, device="cuda")
    info = gb.solve_mean(mu, rel_tol=1e-6)
    assert info.rel_res <= 1e-6
    # the relative residual in the oracle's FP64 system (a 1e-6 residual does not bound the error to
    # 1e-3 voxel on this band: the error parity is checked at 1e-8)
    rp, ci, val = oracle.csr(blob["ob"], w.lam, blob["qd"])
    Q = sp.csr_matrix((val, ci, rp), shape=(gb.N, gb.N))
    m = mu.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(blob["rhs"] - Q @ m) / np.linalg.norm(blob["rhs"])
    assert rel <= 2e-6, rel
    info = gb.solve_mean(mu, rel_tol=1e-8)
    err = np.abs(mu.cpu().numpy().astype(np.float64) - blob["mu"]).max()
    assert err <= 1e-3, err


def test_blob_variance_of_all_probes_in_the_bench_call(blob):
    gb = blob["gb"]
    s = torch.empty(gb.N, device="cuda")
    info = gb.estimate_variance(s, K=K, seed=SEED, rel_tol=1e-6, rhs_block=0)
    assert info.iters >= K
    sv = s.cpu().numpy().astype(np.float64)
    rel = np.abs(sv - blob["s"]) / np.maximum(np.abs(blob["s"]), 1.0 / blob["qd"])
    assert rel.max() <= 1e-3, rel.max()
    # probe-sharded form: two ranges of the same probes, each part scaled by 1/K on the device, summed
    parts = []
    for k0, k1 in ((0, 48), (48, K)):
        p = torch.empty(gb.N, device="cuda")
        gb.estimate_variance_range(p, k0, k1, seed=SEED, rel_tol=1e-6, rhs_block=0, scale=1.0 / K)
        parts.append(p)
    sh = (parts[0] + parts[1]).cpu().numpy().astype(np.float64)
    rel = np.abs(sh - blob["s"]) / np.maximum(np.abs(blob["s"]), 1.0 / blob["qd"])
    assert rel.max() <= 1e-3, rel.max()


def test_blob_marching_cubes_topology(blob):
    mu32 = blob["mu"].astype(np.float32)
    V, F = blob["gb"].extract_surface(dev(mu32))
    Vo, Fo = oracle.marching_cubes(blob["ob"], mu32)
    assert len(F) > 100000
    np.testing.assert_array_equal(F, Fo)
    np.testing.assert_allclose(V, Vo, rtol=0, atol=2e-6 + 1e-5 * blob["w"].h)


def test_blob_view_scores(blob):
    w, gb = blob["w"], blob["gb"]
    mu32 = blob["mu"].astype(np.float32)
    s32 = blob["s"].astype(np.float32)
    qd32 = gb.export_system()["qdiag"].astype(np.float64)
    cand = w.cand_poses[::16]
    U, best = gb.score_views(dev(mu32), dev(s32), dev(cand), w.cand_intr)
    Uo, besto = oracle.score_views(blob["ob"], mu32, s32.astype(np.float64), qd32, cand, w.cand_intr, w.band_vox,
                                   w.sig_a, w.sig_b, w.sig_pose, w.sig_model)
    np.testing.assert_allclose(U, Uo, rtol=1e-3, atol=1e-6 * Uo.max())
    assert best == besto or Uo[best] >= Uo[besto] * (1 - 1e-3)
