"""Pins of the oracle's posterior system and solvers (Sec. 3.6 Q0,
precision and mean equations, PCG; Sec. 3.7 diagonal estimator)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def small():
    w = synth.make_workload("sphere64", n=24, image_scale=0.5, frames=12)
    b = oracle.build_band_w(w)
    d, hd, _ = oracle.integrate_w(b, w)
    qd, rhs = oracle.assemble(b, d, hd, w.lam, w.lam_b)
    return w, b, d, hd, qd, rhs


def test_precision_is_symmetric_with_laplacian_rows_and_spd(small):
    w, b, d, hd, qd, rhs = small
    assert 300 < b.N <= 3500
    Q = oracle.dense_Q(b, w.lam, qd)
    np.testing.assert_array_equal(Q, Q.T)
    # rows of lambda L sum to zero: row sums = lambda_b [dB] + d
    np.testing.assert_allclose(Q.sum(1), w.lam_b * b.bdry + d, rtol=1e-12, atol=1e-12)
    # off-diagonal count = band degree; off-diagonal values -lambda
    off = Q - np.diag(np.diag(Q))
    np.testing.assert_array_equal((off != 0).sum(1), b.deg)
    assert np.all(off[off != 0] == -w.lam)
    assert np.linalg.eigvalsh(Q).min() > 0
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(b.N), rng.standard_normal(b.N)
    qx, qy = oracle.spmv(b, w.lam, qd, x), oracle.spmv(b, w.lam, qd, y)
    assert abs(x @ qy - qx @ y) <= 1e-12 * abs(x @ qy)
    np.testing.assert_allclose(qx, Q @ x, rtol=1e-13, atol=1e-12)
    # anchor term: h = hdata + lambda_b [dB] tsdf / h
    np.testing.assert_allclose(rhs - hd, w.lam_b * b.bdry * b.tsdf.astype(np.float64) / b.h, rtol=0, atol=1e-12 * np.abs(rhs).max())


def test_mean_matches_dense_solve(small):
    w, b, d, hd, qd, rhs = small
    Q = oracle.dense_Q(b, w.lam, qd)
    ref = np.linalg.solve(Q, rhs)
    mu, st, it, rr = oracle.pcg(b, w.lam, qd, rhs, tol=1e-13)
    assert st == 0 and rr <= 1e-13
    np.testing.assert_allclose(mu, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_diagonal_system_is_solved_exactly_in_one_step(small):
    w, b, d, hd, qd, rhs = small
    q = d + 0.5 + b.bdry
    mu, st, it, rr = oracle.pcg(b, 0.0, q, rhs, tol=1e-14)
    assert st == 0 and it == 1
    np.testing.assert_allclose(mu, rhs / q, rtol=1e-14)


def test_pcg_stopping_rule_and_warm_start(small):
    w, b, d, hd, qd, rhs = small
    Q = oracle.dense_Q(b, w.lam, qd)
    for tol in (1e-4, 1e-8):
        mu, st, it, rr = oracle.pcg(b, w.lam, qd, rhs, tol=tol)
        assert st == 0
        true = np.linalg.norm(rhs - Q @ mu) / np.linalg.norm(rhs)
        assert true <= tol and abs(true - rr) <= 1e-12
    # started at the solution, PCG does no iteration
    mu, *_ = oracle.pcg(b, w.lam, qd, rhs, tol=1e-12)
    _, st, it, _ = oracle.pcg(b, w.lam, qd, rhs, tol=1e-8, x0=mu)
    assert st == 0 and it == 0
    # zero right-hand side: x = 0
    x, st, it, rr = oracle.pcg(b, w.lam, qd, np.zeros(b.N), tol=1e-8)
    assert st == 0 and it == 0 and np.all(x == 0)
    # iteration limit reports non-convergence
    _, st, it, _ = oracle.pcg(b, w.lam, qd, rhs, tol=1e-14, max_iter=2)
    assert st == 1 and it == 2


def test_no_prior_gives_the_weighted_mean_of_observations(small):
    """lambda = lambda_b = 0: Q = diag(d), so mu_i = hdata_i / d_i, the
    precision-weighted mean of the samples (observed voxels only)."""
    w, b, d, hd, qd, rhs = small
    q0, r0 = oracle.assemble(b, d, hd, 0.0, 0.0)
    np.testing.assert_array_equal(q0, d)
    m = d > 0
    mu = r0[m] / q0[m]
    np.testing.assert_allclose(mu, hd[m] / d[m], rtol=1e-15)


def test_hutchinson_without_prior_is_exact_for_one_probe(small):
    w, b, d, hd, qd, rhs = small
    q = d + 0.5 * b.bdry + 0.25
    s, st, it, _ = oracle.hutchinson(b, 0.0, q, 1, 0, tol=1e-14)
    assert st == 0
    np.testing.assert_allclose(s, 1.0 / q, rtol=1e-13)


def test_hutchinson_finite_k_definition_and_convergence(small):
    w, b, d, hd, qd, rhs = small
    Q = oracle.dense_Q(b, w.lam, qd)
    Qi = np.linalg.inv(Q)
    K = 16
    s, st, it, U = oracle.hutchinson(b, w.lam, qd, K, 5, tol=1e-13, keep=2)
    assert st == 0
    Z = np.stack([oracle.probe(5, k, b.lin) for k in range(K)])
    exact = np.mean(Z * (Z @ Qi), axis=0)                       # (1/K) sum z (.) Q^-1 z
    np.testing.assert_allclose(s, exact, rtol=0, atol=1e-10 * np.abs(exact).max())
    np.testing.assert_allclose(U[1], Qi @ Z[1], atol=1e-10 * np.abs(U[1]).max())
    # statistical pin against the dense inverse: |s_i - (Q^-1)_ii| <= 4 sd_i for >= 99 %
    K = 1024
    s, st, it, _ = oracle.hutchinson(b, w.lam, qd, K, 11, tol=1e-10)
    off2 = (Qi ** 2).sum(1) - np.diag(Qi) ** 2
    sd = np.sqrt(off2 / K)
    ok = np.abs(s - np.diag(Qi)) <= 4 * sd
    assert ok.mean() >= 0.99
    # Q^-1_ii >= 1 / Q_ii for SPD Q
    assert np.all(np.diag(Qi) >= 1.0 / np.diag(Q) * (1 - 1e-12))
