"""CPU oracle for the BayesFusion-SDF posterior solve -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
arm may import this package.  The product path (the CUDA library and its
Python binding) never imports, links or runs it, and the two share no code.

The arithmetic lives in ``bfo.c`` (plain C, FP64 for every real-valued
quantity, a fixed FP32 specification for discrete decisions; every function
there cites the section of the paper it restates).  This module compiles it
with gcc and marshals numpy arrays through ctypes; written here in numpy are
``surrogate_judge`` (a per-brick statistic over values the C code returns) and
the evaluations of the next rows' solvers, ``block_pcg`` (block CG over the
probe right-hand sides), ``deflated_pcg`` and ``ritz_vectors`` (deflation of a
probe block's Krylov information from the next block's solves).

Parity status: every function is pinned by the ``-m "not gpu"`` tests against
closed forms, invariants, special cases or brute force (see
tests/test_oracle_*.py); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfo.c")
_SRC_NET = os.path.join(_HERE, "net.c")
_LIB = os.path.join(_HERE, "_bfo.so")
_lib = None

c_i64p = ctypes.POINTER(ctypes.c_int64)
c_dp = ctypes.POINTER(ctypes.c_double)
c_fp = ctypes.POINTER(ctypes.c_float)


class _Band(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nb", ctypes.c_int), ("h", ctypes.c_float),
                ("org", ctypes.c_float * 3), ("N", ctypes.c_int64), ("NB", ctypes.c_int32),
                ("n_cand", ctypes.c_int64),
                ("dir", ctypes.POINTER(ctypes.c_int32)), ("bcoord", ctypes.POINTER(ctypes.c_int32)),
                ("mask", ctypes.POINTER(ctypes.c_uint64)), ("off", c_i64p), ("lin", c_i64p),
                ("tsdf", c_fp), ("wcount", ctypes.POINTER(ctypes.c_int32)),
                ("bdry", ctypes.POINTER(ctypes.c_uint8)), ("deg", ctypes.POINTER(ctypes.c_uint8)),
                ("nbr", ctypes.POINTER(ctypes.c_int32))]


def build(force: bool = False) -> str:
    """Compile the oracle in-tree (gcc, FP contraction off, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_NET))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE", _SRC, _SRC_NET, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    bp = ctypes.POINTER(_Band)
    f, i, d, u64, i64 = ctypes.c_float, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64
    L.bfo_build_band.restype = bp
    L.bfo_build_band.argtypes = [c_fp, i, i, i, c_fp, f, f, f, f, i, f, c_fp, d, d, i]
    L.bfo_band_free.argtypes = [bp]
    L.bfo_band_index.restype = i64
    L.bfo_band_index.argtypes = [bp, i, i, i]
    L.bfo_integrate.argtypes = [bp, c_fp, i, i, i, c_fp, f, f, f, f, d, d, d, d, d, c_dp, c_dp, c_i64p]
    L.bfo_dda_trace.restype = i64
    L.bfo_dda_trace.argtypes = [bp, c_fp, f, f, f, f, i, i, f, d, c_i64p, i64]
    L.bfo_assemble.argtypes = [bp, c_dp, c_dp, d, d, c_dp, c_dp]
    L.bfo_spmv.argtypes = [bp, d, c_dp, c_dp, c_dp]
    L.bfo_csr.restype = i64
    L.bfo_csr.argtypes = [bp, d, c_dp, c_i64p, c_i64p, c_dp]
    L.bfo_pcg.restype = i
    L.bfo_pcg.argtypes = [bp, d, c_dp, c_dp, c_dp, d, i, c_dp, ctypes.POINTER(i), c_dp]
    L.bfo_splitmix64.restype = u64
    L.bfo_splitmix64.argtypes = [u64]
    L.bfo_probe.argtypes = [u64, u64, i64, c_i64p, c_dp]
    L.bfo_hutchinson.restype = i
    L.bfo_hutchinson.argtypes = [bp, d, c_dp, i, u64, d, i, i, c_dp, ctypes.POINTER(i), c_dp, i]
    L.bfo_mc_case.restype = i
    L.bfo_mc_case.argtypes = [i, ctypes.POINTER(ctypes.c_int32)]
    L.bfo_mc.argtypes = [bp, c_fp, c_i64p, ctypes.POINTER(c_dp), c_i64p,
                         ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))]
    L.bfo_free.argtypes = [ctypes.c_void_p]
    L.bfo_predict_depth.argtypes = [bp, c_fp, c_fp, f, f, f, f, i, i, c_fp]
    L.bfo_net_nparams.restype = i64
    L.bfo_net_nparams.argtypes = []
    L.bfo_net_features.argtypes = [bp, c_dp, c_dp]
    L.bfo_net_loss.restype = d
    L.bfo_net_loss.argtypes = [c_dp, i, c_dp, c_dp, c_dp, ctypes.POINTER(ctypes.c_uint8), c_dp, c_dp]
    L.bfo_score_views.restype = i
    L.bfo_score_views.argtypes = [bp, c_fp, c_dp, c_dp, c_fp, i, f, f, f, f, i, i, d, d, d, d, d, d, c_dp]
    _lib = L
    return L


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


@dataclass
class Band:
    """Oracle band: brick directory and compact band arrays (numpy copies)."""
    n: int
    h: float
    origin: tuple
    N: int
    NB: int
    n_cand: int
    dir: np.ndarray       # int32 [nb^3]
    bcoord: np.ndarray    # int32 [NB,3]
    mask: np.ndarray      # uint64 [NB,8]
    off: np.ndarray       # int64 [NB+1]
    lin: np.ndarray       # int64 [N]
    tsdf: np.ndarray      # float32 [N] metres
    wcount: np.ndarray    # int32 [N]
    bdry: np.ndarray      # uint8 [N]
    deg: np.ndarray       # uint8 [N]
    nbr: np.ndarray       # int32 [NB,6]
    _ptr: object = None

    def __del__(self):
        if self._ptr is not None and _lib is not None:
            _lib.bfo_band_free(self._ptr)
            self._ptr = None

    def index(self, i, j, k) -> int:
        return int(_lib.bfo_band_index(self._ptr, i, j, k))

    def ijk(self) -> np.ndarray:
        n = self.n
        L = self.lin
        return np.stack([L % n, (L // n) % n, L // (n * n)], 1)

    def centres(self) -> np.ndarray:
        return np.asarray(self.origin, np.float64) + (self.ijk() + 0.5) * self.h


def build_band(depth, poses, intr, n, h, origin, band_vox, trunc_vox, threads=0) -> Band:
    L = _load()
    depth, poses = _f32(depth), _f32(poses)
    fx, fy, cx, cy, W, H = intr
    T = depth.shape[0]
    org = _f32(origin)
    ptr = L.bfo_build_band(_p(depth, ctypes.c_float), T, H, W, _p(poses, ctypes.c_float), fx, fy, cx, cy,
                           n, h, _p(org, ctypes.c_float), band_vox, trunc_vox, threads)
    b = ptr.contents
    N, NB, nb = b.N, b.NB, b.nb

    def cp(p, cnt, dt):
        return np.ctypeslib.as_array(p, shape=(max(cnt, 1),))[:cnt].astype(dt, copy=True)

    return Band(n=n, h=float(np.float32(h)), origin=tuple(float(v) for v in org), N=N, NB=NB,
                n_cand=b.n_cand, dir=cp(b.dir, nb ** 3, np.int32), bcoord=cp(b.bcoord, 3 * NB, np.int32).reshape(NB, 3),
                mask=cp(b.mask, 8 * NB, np.uint64).reshape(NB, 8), off=cp(b.off, NB + 1, np.int64),
                lin=cp(b.lin, N, np.int64), tsdf=cp(b.tsdf, N, np.float32), wcount=cp(b.wcount, N, np.int32),
                bdry=cp(b.bdry, N, np.uint8), deg=cp(b.deg, N, np.uint8), nbr=cp(b.nbr, 6 * NB, np.int32).reshape(NB, 6),
                _ptr=ptr)


def build_band_w(w, threads=0) -> Band:
    return build_band(w.depth, w.poses, w.intr, w.n, w.h, w.origin, w.band_vox, w.trunc_vox, threads)


def integrate(band: Band, depth, poses, intr, band_vox, sig_a, sig_b, sig_pose=0.0, sig_model=0.0):
    """Returns (d, hdata, stats) in voxel units, FP64."""
    L = _load()
    depth, poses = _f32(depth), _f32(poses)
    fx, fy, cx, cy, W, H = intr
    d = np.zeros(band.N, np.float64)
    hd = np.zeros(band.N, np.float64)
    st = np.zeros(2, np.int64)
    L.bfo_integrate(band._ptr, _p(depth, ctypes.c_float), depth.shape[0], H, W, _p(poses, ctypes.c_float),
                    fx, fy, cx, cy, band_vox, sig_a, sig_b, sig_pose, sig_model, _p(d, ctypes.c_double),
                    _p(hd, ctypes.c_double), _p(st, ctypes.c_int64))
    return d, hd, st


def integrate_w(band, w):
    return integrate(band, w.depth, w.poses, w.intr, w.band_vox, w.sig_a, w.sig_b, w.sig_pose, w.sig_model)


def dda_trace(band: Band, pose, intr, px, py, D, band_vox, cap=4096) -> np.ndarray:
    L = _load()
    pose = _f32(pose)
    fx, fy, cx, cy, W, H = intr
    out = np.empty(cap, np.int64)
    m = L.bfo_dda_trace(band._ptr, _p(pose, ctypes.c_float), fx, fy, cx, cy, px, py, D, band_vox,
                        _p(out, ctypes.c_int64), cap)
    return out[:m].copy()


def assemble(band: Band, d, hd, lam, lam_b):
    L = _load()
    d, hd = _f64(d), _f64(hd)
    qd = np.empty(band.N, np.float64)
    rhs = np.empty(band.N, np.float64)
    L.bfo_assemble(band._ptr, _p(d, ctypes.c_double), _p(hd, ctypes.c_double), lam, lam_b,
                   _p(qd, ctypes.c_double), _p(rhs, ctypes.c_double))
    return qd, rhs


def spmv(band: Band, lam, qdiag, x) -> np.ndarray:
    L = _load()
    qdiag, x = _f64(qdiag), _f64(x)
    y = np.empty(band.N, np.float64)
    L.bfo_spmv(band._ptr, lam, _p(qdiag, ctypes.c_double), _p(x, ctypes.c_double), _p(y, ctypes.c_double))
    return y


def csr(band: Band, lam, qdiag):
    """Q as (indptr, indices, data) numpy arrays."""
    L = _load()
    qdiag = _f64(qdiag)
    nnz = L.bfo_csr(band._ptr, lam, _p(qdiag, ctypes.c_double), None, None, None)
    rp = np.empty(band.N + 1, np.int64)
    ci = np.empty(nnz, np.int64)
    val = np.empty(nnz, np.float64)
    L.bfo_csr(band._ptr, lam, _p(qdiag, ctypes.c_double), _p(rp, ctypes.c_int64), _p(ci, ctypes.c_int64),
              _p(val, ctypes.c_double))
    return rp, ci, val


def dense_Q(band: Band, lam, qdiag) -> np.ndarray:
    rp, ci, val = csr(band, lam, qdiag)
    Q = np.zeros((band.N, band.N))
    for r in range(band.N):
        Q[r, ci[rp[r]:rp[r + 1]]] += val[rp[r]:rp[r + 1]]
    return Q


def pcg(band: Band, lam, qdiag, rhs, tol=1e-12, max_iter=20000, x0=None):
    """Returns (x, status, iters, relres)."""
    L = _load()
    qdiag, rhs = _f64(qdiag), _f64(rhs)
    x = np.empty(band.N, np.float64)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    x0p = _p(_f64(x0), ctypes.c_double) if x0 is not None else None
    if x0 is not None:
        x0 = _f64(x0)
        x0p = _p(x0, ctypes.c_double)
    st = L.bfo_pcg(band._ptr, lam, _p(qdiag, ctypes.c_double), _p(rhs, ctypes.c_double), x0p, tol, max_iter,
                   _p(x, ctypes.c_double), ctypes.byref(it), ctypes.byref(rr))
    return x, st, it.value, rr.value


def splitmix64(x: int) -> int:
    return int(_load().bfo_splitmix64(x))


def probe(seed: int, k: int, lin) -> np.ndarray:
    lin = np.ascontiguousarray(lin, np.int64)
    z = np.empty(len(lin), np.float64)
    _load().bfo_probe(seed, k, len(lin), _p(lin, ctypes.c_int64), _p(z, ctypes.c_double))
    return z


def hutchinson(band: Band, lam, qdiag, K, seed, tol=1e-12, max_iter=20000, k0=0, keep=0):
    """Returns (s, status, total_iters, per_probe_solutions[keep,N])."""
    L = _load()
    qdiag = _f64(qdiag)
    s = np.empty(band.N, np.float64)
    it = ctypes.c_int()
    pp = np.empty((max(keep, 1), band.N), np.float64)
    st = L.bfo_hutchinson(band._ptr, lam, _p(qdiag, ctypes.c_double), K, seed, tol, max_iter, k0,
                          _p(s, ctypes.c_double), ctypes.byref(it), _p(pp, ctypes.c_double), keep)
    return s, st, it.value, pp[:keep]


def mc_case(cs: int) -> np.ndarray:
    tri = np.zeros((16, 3), np.int32)
    m = _load().bfo_mc_case(cs, _p(tri, ctypes.c_int32))
    return tri[:m].copy()


def marching_cubes(band: Band, mu):
    """Returns (verts f64 [V,3] metres, tris int32 [F,3])."""
    L = _load()
    mu = _f32(mu)
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    vp, tp = c_dp(), ctypes.POINTER(ctypes.c_int32)()
    L.bfo_mc(band._ptr, _p(mu, ctypes.c_float), ctypes.byref(nv), ctypes.byref(vp), ctypes.byref(nt),
             ctypes.byref(tp))
    V = np.ctypeslib.as_array(vp, shape=(max(nv.value, 1) * 3,))[:3 * nv.value].reshape(-1, 3).copy()
    F = np.ctypeslib.as_array(tp, shape=(max(nt.value, 1) * 3,))[:3 * nt.value].reshape(-1, 3).copy()
    L.bfo_free(ctypes.cast(vp, ctypes.c_void_p))
    L.bfo_free(ctypes.cast(tp, ctypes.c_void_p))
    return V, F


def predict_depth(band: Band, mu, pose, intr) -> np.ndarray:
    L = _load()
    mu, pose = _f32(mu), _f32(pose)
    fx, fy, cx, cy, W, H = intr
    out = np.empty((H, W), np.float32)
    L.bfo_predict_depth(band._ptr, _p(mu, ctypes.c_float), _p(pose, ctypes.c_float), fx, fy, cx, cy, W, H,
                        _p(out, ctypes.c_float))
    return out


def score_views(band: Band, mu, s, qdiag, cand_poses, cand_intr, band_vox, sig_a, sig_b, sig_pose=0.0,
                sig_model=0.0, eps=1.0):
    """Returns (U f64 [V], best)."""
    L = _load()
    mu, s, qdiag, cand = _f32(mu), _f64(s), _f64(qdiag), _f32(cand_poses)
    fx, fy, cx, cy, W, H = cand_intr
    V = cand.shape[0]
    U = np.zeros(V, np.float64)
    best = L.bfo_score_views(band._ptr, _p(mu, ctypes.c_float), _p(s, ctypes.c_double), _p(qdiag, ctypes.c_double),
                             _p(cand, ctypes.c_float), V, fx, fy, cx, cy, W, H, band_vox, sig_a, sig_b, sig_pose,
                             sig_model, eps, _p(U, ctypes.c_double))
    return U, best


def score_views_exact(band: Band, mu, qdiag, lam, cand_poses, cand_intr, band_vox, sig_a, sig_b, K, seed,
                      tol=1e-12, sig_pose=0.0, sig_model=0.0, eps=1.0):
    """Exact view utilities (the re-solve the NBV equation's s' stands for, Sec. 3.8): per candidate v the
    predicted observations dd_v of its predicted depth (``predict_depth`` then ``integrate``) are added to the
    diagonal of Q and the K-probe estimate is recomputed with the same probes:
    U[v] = sum_{|mu_j| <= eps} (s_j - s'_j).  Returns (U f64 [V], best)."""
    mu32 = _f32(mu)
    qdiag = _f64(qdiag)
    s, st, _, _ = hutchinson(band, lam, qdiag, K, seed, tol=tol)
    if st != 0:
        raise RuntimeError("hutchinson did not converge")
    om = np.abs(mu32.astype(np.float64)) <= eps
    cand = _f32(cand_poses)
    U = np.zeros(cand.shape[0], np.float64)
    for v in range(cand.shape[0]):
        Dp = predict_depth(band, mu32, cand[v], cand_intr)
        dd, _, _ = integrate(band, Dp[None], cand[v:v + 1], cand_intr, band_vox, sig_a, sig_b, sig_pose, sig_model)
        s2, st, _, _ = hutchinson(band, lam, qdiag + dd, K, seed, tol=tol)
        if st != 0:
            raise RuntimeError("hutchinson did not converge")
        U[v] = float(np.sum((s - s2)[om]))
    return U, int(np.argmax(U))


def block_pcg(band: Band, lam, qdiag, B, tol=1e-12, max_iter=20000, rank_tol=1e-10, Q=None):
    """Block PCG with the Jacobi preconditioner for Q X = B (B [N, R]): the R right-hand sides share one block
    Krylov space (O'Leary's block CG) in its breakdown-free form, the direction block kept as an orthonormal basis
    from a rank-revealing QR so that converged or dependent directions drop out.  Per iteration, with P the basis:
        alpha = (P^T Q P)^-1 P^T R,  X += P alpha,  R -= (Q P) alpha,
        Z = M^-1 R,  beta = -(P^T Q P)^-1 (Q P)^T Z,  P = orth(Z + P beta).
    Stops when every column's residual 2-norm is <= tol |b_c|.  Q (a scipy sparse matrix) replaces the 7-point
    precision built from lam and qdiag when given (its diagonal is then the preconditioner).  Returns (X, status,
    iterations), status 0 on convergence, 1 at max_iter."""
    import scipy.linalg
    import scipy.sparse
    if Q is None:
        indptr, indices, data = csr(band, lam, qdiag)
        Q = scipy.sparse.csr_matrix((data, indices, indptr), shape=(band.N, band.N))
    else:
        Q = scipy.sparse.csr_matrix(Q)
        qdiag = Q.diagonal()
    B = np.asarray(B, np.float64)
    if B.ndim == 1:
        B = B[:, None]
    Minv = 1.0 / np.asarray(qdiag, np.float64)
    bn = np.linalg.norm(B, axis=0)

    def orth(Y):
        Qf, Rf, _ = scipy.linalg.qr(Y, mode="economic", pivoting=True)
        d = np.abs(np.diag(Rf))
        keep = d > rank_tol * (d[0] if d.size and d[0] > 0 else 1.0)
        return Qf[:, :int(np.count_nonzero(keep))]

    X = np.zeros_like(B)
    R = B.copy()
    if np.all(np.linalg.norm(R, axis=0) <= tol * bn):
        return X, 0, 0
    P = orth(Minv[:, None] * R)
    for it in range(1, max_iter + 1):
        QP = Q @ P
        G = P.T @ QP
        alpha = np.linalg.solve(G, P.T @ R)
        X += P @ alpha
        R -= QP @ alpha
        if np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            return X, 0, it
        Z = Minv[:, None] * R
        beta = -np.linalg.solve(G, QP.T @ Z)
        P = orth(Z + P @ beta)
        if P.shape[1] == 0:
            return X, 0 if np.all(np.linalg.norm(R, axis=0) <= tol * bn) else 1, it
    return X, 1, max_iter


def _sparse_Q(band, lam, qdiag, Q):
    import scipy.sparse
    if Q is None:
        indptr, indices, data = csr(band, lam, qdiag)
        return scipy.sparse.csr_matrix((data, indices, indptr), shape=(band.N, band.N))
    return scipy.sparse.csr_matrix(Q)


def deflated_pcg(band: Band, lam, qdiag, b, W=None, tol=1e-12, max_iter=20000, Q=None, lanczos=False):
    """Deflated Jacobi PCG (Saad, Yeung, Erhel & Guyomarc'h, 2000) for Q x = b, the evaluation of row f2's
    deflation across probe blocks (Sec. 3.7 needs one solve per probe): the k columns of W span a subspace taken out
    of the iteration -- x0 = W E^-1 W^T b with E = W^T Q W, and every preconditioned residual z = M^-1 r is made
    Q-orthogonal to W, z - W E^-1 (Q W)^T z, before it enters the search direction (M = diag Q).  With W = None
    this is plain PCG.  Stops when |r| <= tol |b|.  Returns (x, status, iters) and, with lanczos=True, also the CG
    coefficients (alphas, betas) and the M-normalised residual directions z_j / sqrt(r_j . z_j) of the run (the
    Lanczos basis from which ``ritz_vectors`` forms Ritz vectors)."""
    Qs = _sparse_Q(band, lam, qdiag, Q)
    Minv = 1.0 / Qs.diagonal()
    b = np.asarray(b, np.float64)
    if W is not None and W.shape[1] > 0:
        QW = Qs @ W
        E = W.T @ QW
        x = W @ np.linalg.solve(E, W.T @ b)
        proj = lambda z: z - W @ np.linalg.solve(E, QW.T @ z)
    else:
        x = np.zeros_like(b)
        proj = lambda z: z
    r = b - Qs @ x
    bn = np.linalg.norm(b)
    z = Minv * r
    rz = float(r @ z)
    p = proj(z)
    als, bes, Zs = [], [], [z / np.sqrt(rz)] if rz > 0 else []
    it, status = 0, 0
    while np.linalg.norm(r) > tol * bn:
        if it >= max_iter:
            status = 1
            break
        q = Qs @ p
        a = rz / float(p @ q)
        x += a * p
        r -= a * q
        it += 1
        z = Minv * r
        rz2 = float(r @ z)
        be = rz2 / rz
        als.append(a)
        bes.append(be)
        if rz2 > 0:
            Zs.append(z / np.sqrt(rz2))
        p = proj(z) + be * p
        rz = rz2
    if lanczos:
        return x, status, it, np.array(als), np.array(bes), Zs
    return x, status, it


def ritz_vectors(alphas, betas, Zs, k):
    """The k smallest Ritz pairs of M^-1 Q from a PCG run's coefficients: the Lanczos tridiagonal has diagonal
    1/alpha_j + beta_{j-1}/alpha_{j-1} and off-diagonal -sqrt(beta_j)/alpha_j; its eigenvectors combine the
    M-normalised residual directions.  Returns (values [k], vectors [N, k])."""
    m = len(alphas)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = -np.sqrt(betas[j]) / alphas[j]
    ev, U = np.linalg.eigh(T)
    V = np.stack(Zs[:m], 1)
    k = min(k, m)
    return ev[:k], V @ U[:, :k]


def solve_all(w, threads=0, tol=1e-12, K=None):
    """Full oracle pipeline for a workload: band, d/h, Q, mu and (optionally) s."""
    b = build_band_w(w, threads)
    d, hd, st = integrate_w(b, w)
    qd, rhs = assemble(b, d, hd, w.lam, w.lam_b)
    mu, status, iters, rr = pcg(b, w.lam, qd, rhs, tol=tol)
    out = dict(band=b, d=d, hd=hd, qdiag=qd, rhs=rhs, mu=mu, iters=iters, relres=rr, status=status)
    if K:
        s, st2, tot, _ = hutchinson(b, w.lam, qd, K, w.seed, tol=tol)
        out.update(s=s, hutch_iters=tot)
    return out


# ------------------------------------------------------------ learned part

def net_nparams() -> int:
    return int(_load().bfo_net_nparams())


def net_features(band: Band, d) -> np.ndarray:
    """[NB,1000,2] input tiles (tsdf/h, log(1+d)) of the band's bricks."""
    d = _f64(d)
    feat = np.empty((band.NB, 1000, 2), np.float64)
    _load().bfo_net_features(band._ptr, _p(d, ctypes.c_double), _p(feat, ctypes.c_double))
    return feat


def net_targets(band: Band, mu, log_s, qdiag=None):
    """Per-brick centre arrays from compact ones: targets [NB,512,2] (mu, log s),
    band mask [NB,512] and log Q_ii [NB,512] (0 where qdiag is None or off the band)."""
    tgt = np.zeros((band.NB, 512, 2), np.float64)
    mask = np.zeros((band.NB, 512), np.uint8)
    lq = np.zeros((band.NB, 512), np.float64)
    brick = np.repeat(np.arange(band.NB), np.diff(band.off))
    ijk = band.ijk()
    loc = (ijk[:, 0] & 7) + 8 * (ijk[:, 1] & 7) + 64 * (ijk[:, 2] & 7)
    tgt[brick, loc, 0] = mu
    tgt[brick, loc, 1] = log_s
    mask[brick, loc] = 1
    if qdiag is not None:
        lq[brick, loc] = np.log(np.asarray(qdiag, np.float64))
    return tgt, mask, lq


def net_loss(params, feat, tgt, mask, lq=None, grad=True):
    """Returns (loss, grad [P] or None, pred [NB,512,2]); lq [NB,512] log Q_ii (default 0)."""
    L = _load()
    params, feat, tgt = _f64(params), _f64(feat), _f64(tgt)
    mask = np.ascontiguousarray(mask, np.uint8)
    NB = feat.shape[0]
    lq = np.zeros((NB, 512)) if lq is None else lq
    lq = _f64(lq)
    g = np.empty(len(params), np.float64) if grad else None
    pred = np.empty((NB, 512, 2), np.float64)
    loss = L.bfo_net_loss(_p(params, ctypes.c_double), NB, _p(feat, ctypes.c_double), _p(lq, ctypes.c_double),
                          _p(tgt, ctypes.c_double), _p(mask, ctypes.c_uint8), _p(g, ctypes.c_double) if grad else None,
                          _p(pred, ctypes.c_double))
    return loss, g, pred


def surrogate_judge(band: Band, log_s_hat, t, qdiag):
    """Acceptance test of the learned variance surrogate, per brick.

    t [K_j, N]: per-probe values t_k = z_k (.) Q^-1 z_k of K_j probes.  With
    s_J = mean_k t_k, se = sample std / sqrt(K_j), f = max(s_J, 1/Q_ii) and
    e = |exp(log_s_hat) - s_J|, a brick is accepted when the median of e/f
    over its voxels is <= 0.10 and max e / (3 se + 0.1 f) <= 1.
    Returns (stat [NB, 2] = (median, max ratio), accepted [NB] uint8)."""
    t = np.asarray(t, np.float64)
    Kj = t.shape[0]
    sJ = t.mean(axis=0)
    se = t.std(axis=0, ddof=1) / math.sqrt(Kj)
    f = np.maximum(sJ, 1.0 / np.asarray(qdiag, np.float64))
    e = np.abs(np.exp(np.asarray(log_s_hat, np.float64)) - sJ)
    stat = np.zeros((band.NB, 2))
    acc = np.zeros(band.NB, np.uint8)
    for b in range(band.NB):
        sl = slice(band.off[b], band.off[b + 1])
        stat[b, 0] = np.median(e[sl] / f[sl])
        stat[b, 1] = np.max(e[sl] / (3.0 * se[sl] + 0.1 * f[sl]))
        acc[b] = stat[b, 0] <= 0.10 and stat[b, 1] <= 1.0
    return stat, acc
