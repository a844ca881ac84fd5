"""The block PCG oracle (breakdown-free block CG over the probe right-hand
sides) against plain PCG, a dense solve, and the block Krylov property."""
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
    return w, b, qd, rhs


def test_one_column_is_plain_pcg(small):
    w, b, qd, rhs = small
    x, st, it, _ = oracle.pcg(b, w.lam, qd, rhs, tol=1e-10)
    X, st2, it2 = oracle.block_pcg(b, w.lam, qd, rhs, tol=1e-10)
    assert st == 0 and st2 == 0
    assert abs(it2 - it) <= 1
    np.testing.assert_allclose(X[:, 0], x, rtol=0, atol=1e-8 * np.abs(x).max())


def test_block_solution_is_the_dense_solution(small):
    w, b, qd, rhs = small
    indptr, indices, data = oracle.csr(b, w.lam, qd)
    import scipy.sparse
    Q = scipy.sparse.csr_matrix((data, indices, indptr), shape=(b.N, b.N)).toarray()
    Z = np.stack([oracle.probe(3, k, b.lin) for k in range(6)], 1)
    X, st, it = oracle.block_pcg(b, w.lam, qd, Z, tol=1e-12)
    assert st == 0
    np.testing.assert_allclose(X, np.linalg.solve(Q, Z), rtol=0, atol=1e-9 * np.abs(X).max())


def test_block_krylov_needs_no_more_iterations_than_the_slowest_column(small):
    w, b, qd, rhs = small
    K = 8
    Z = np.stack([oracle.probe(5, k, b.lin) for k in range(K)], 1)
    its = []
    for k in range(K):
        _, st, it, _ = oracle.pcg(b, w.lam, qd, Z[:, k], tol=1e-8)
        assert st == 0
        its.append(it)
    X, st, itb = oracle.block_pcg(b, w.lam, qd, Z, tol=1e-8)
    assert st == 0
    assert itb <= max(its) + 1, (itb, its)
    Rres = Z - np.stack([oracle.spmv(b, w.lam, qd, X[:, k]) for k in range(K)], 1)
    assert np.all(np.linalg.norm(Rres, axis=0) <= 1e-8 * np.linalg.norm(Z, axis=0) * 1.0001)


def test_deflated_pcg_solves_the_system_and_removes_the_deflated_eigenvalues():
    """Row f2's deflation evaluation (oracle.deflated_pcg): without a subspace it is plain PCG (same iterations,
    same solution); with W spanning the eigenvectors of the k smallest eigenvalues of M^-1 Q (dense, tiny band) it
    reaches the dense solution and converges no slower, within the CG bound of the deflated condition number
    lambda_max / lambda_{k+1}; Ritz values of a PCG run lie inside the spectrum (interlacing)."""
    import scipy.linalg
    w = synth.make_workload("sphere64", n=16, image_scale=0.25, frames=4)
    b = oracle.build_band_w(w)
    d, hd, _ = oracle.integrate_w(b, w)
    lam = 30.0   # a strong prior spreads the spectrum of M^-1 Q, so deflation has something to remove
    qd, rhs = oracle.assemble(b, d, hd, lam, w.lam_b)
    Q = oracle.dense_Q(b, lam, qd)
    ref = np.linalg.solve(Q, rhs)
    x0, st0, it0 = oracle.deflated_pcg(b, lam, qd, rhs, None, tol=1e-10)
    x1, st1, it1, rr = oracle.pcg(b, lam, qd, rhs, tol=1e-10)
    assert st0 == 0 and it0 == it1
    np.testing.assert_allclose(x0, x1, rtol=0, atol=1e-9 * np.abs(ref).max())
    ev, V = scipy.linalg.eigh(Q, np.diag(np.diag(Q)))   # Q v = mu M v: the spectrum of M^-1 Q
    k = 8
    xk, stk, itk = oracle.deflated_pcg(b, lam, qd, rhs, V[:, :k], tol=1e-10)
    assert stk == 0
    np.testing.assert_allclose(xk, ref, rtol=0, atol=1e-8 * np.abs(ref).max())
    assert itk <= it0
    kappa = ev[-1] / ev[k]
    assert itk <= np.ceil(0.5 * np.sqrt(kappa) * np.log(2.0 / 1e-10)) + 1
    _, _, _, al, be, Zs = oracle.deflated_pcg(b, lam, qd, rhs, None, tol=1e-10, lanczos=True)
    rv, Y = oracle.ritz_vectors(al, be, Zs, 4)
    assert np.all(rv >= ev[0] * (1 - 1e-8)) and np.all(rv <= ev[-1] * (1 + 1e-8))
    assert Y.shape == (b.N, 4)
