"""Python binding of libbfsdf.so (the C ABI in include/bfsdf.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; their
pointers are passed straight through (the library stages host memory
itself).  If the compiled library is missing this module raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfsdf.so")

BF_OK, BF_EINVAL, BF_ENOMEM, BF_ECUDA, BF_NOT_CONVERGED, BF_BREAKDOWN, BF_ESTATE = range(7)
STATUS_NAMES = {0: "BF_OK", 1: "BF_EINVAL", 2: "BF_ENOMEM", 3: "BF_ECUDA", 4: "BF_NOT_CONVERGED",
                5: "BF_BREAKDOWN", 6: "BF_ESTATE"}
BF_SOLVE_FP64 = 1
BF_SOLVE_WARM = 2

EXPORTED = ["bf_create", "bf_destroy", "bf_last_error", "bf_set_stream", "bf_build_band", "bf_band_free",
            "bf_band_info", "bf_export_band", "bf_integrate_depth", "bf_integrate_depth_ex", "bf_export_observations_f64",
            "bf_reset_observations",
            "bf_export_system",
            "bf_spmv", "bf_spmm", "bf_solve_mean", "bf_estimate_variance", "bf_extract_surface", "bf_get_surface",
            "bf_score_views", "bf_score_views_exact", "bf_solve_mean_static", "bf_estimate_variance_range", "bf_bench_kernel",
            "bf_launch_count", "bf_net_nparams", "bf_net_create", "bf_net_destroy", "bf_net_get_params",
            "bf_net_set_params", "bf_net_forward", "bf_net_train_step", "bf_surrogate_variance",
            "bf_net_bench", "bf_autotune_rhs_block", "bf_export_trilinear_rows", "bf_export_precision27",
            "bf_extract_surface_dc"]
BF_INTEGRATE_DETERMINISTIC = 1
BF_INTEGRATE_TRILINEAR = 2
BF_KERNEL_SPMV = 0
BF_KERNEL_BLOCK_ITER = 1
BF_KERNEL_SPMM = 2
BF_NET_BENCH_FORWARD, BF_NET_BENCH_TRAIN, BF_NET_BENCH_CONV, BF_NET_BENCH_WGRAD, BF_NET_BENCH_CONV_MMA = range(5)
# algorithmic FLOPs of the network per brick tile (10^3 voxels, 27 taps, real channels)
NET_FLOPS_FWD = 2 * 1000 * 27 * (2 * 32 + 32 * 32 + 32 * 32 + 32 * 2)
NET_FLOPS_CONV = 2 * 1000 * 27 * 32 * 32


class BfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("voxel", ctypes.c_float), ("origin", ctypes.c_float * 3)]


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("W", ctypes.c_int), ("H", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("band_vox", ctypes.c_double), ("trunc_vox", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("lambda_b", ctypes.c_double), ("sig_a", ctypes.c_double), ("sig_b", ctypes.c_double),
                ("sig_pose", ctypes.c_double), ("sig_model", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbfsdf.so and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run paper_2602_19697_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    vp, i, d, u, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint, ctypes.c_int64
    pvp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "bf_create": (i, [i, vp, pvp]),
        "bf_destroy": (None, [vp]),
        "bf_last_error": (ctypes.c_char_p, [vp]),
        "bf_set_stream": (i, [vp, vp]),
        "bf_build_band": (i, [vp, vp, i, vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(Grid),
                              ctypes.POINTER(Params), pvp]),
        "bf_band_free": (None, [vp]),
        "bf_band_info": (i, [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(i64)]),
        "bf_export_band": (i, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "bf_integrate_depth": (i, [vp, vp, vp, i, vp, ctypes.POINTER(Intrinsics)]),
        "bf_integrate_depth_ex": (i, [vp, vp, vp, i, vp, ctypes.POINTER(Intrinsics), u]),
        "bf_export_observations_f64": (i, [vp, vp, vp, vp]),
        "bf_reset_observations": (i, [vp, vp]),
        "bf_export_system": (i, [vp, vp, vp, vp, vp, vp]),
        "bf_spmv": (i, [vp, vp, vp, vp]),
        "bf_spmm": (i, [vp, vp, vp, i, vp]),
        "bf_solve_mean": (i, [vp, vp, d, i, u, vp, ctypes.POINTER(i), ctypes.POINTER(d)]),
        "bf_estimate_variance": (i, [vp, vp, i, ctypes.c_uint64, d, i, i, u, vp, ctypes.POINTER(i)]),
        "bf_extract_surface": (i, [vp, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "bf_get_surface": (i, [vp, vp, vp]),
        "bf_extract_surface_dc": (i, [vp, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "bf_score_views": (i, [vp, vp, vp, vp, vp, i, ctypes.POINTER(Intrinsics), d, vp, ctypes.POINTER(i)]),
        "bf_score_views_exact": (i, [vp, vp, vp, vp, i, ctypes.POINTER(Intrinsics), d, i, ctypes.c_uint64, d, i, i,
                                     vp, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "bf_solve_mean_static": (i, [vp, vp, d, i, vp, ctypes.POINTER(i), ctypes.POINTER(d)]),
        "bf_estimate_variance_range": (i, [vp, vp, i, i, d, ctypes.c_uint64, d, i, i, u, vp, ctypes.POINTER(i)]),
        "bf_bench_kernel": (i, [vp, vp, i, i, i, ctypes.POINTER(d)]),
        "bf_launch_count": (i, [ctypes.POINTER(i64)]),
        "bf_net_nparams": (i64, []),
        "bf_net_create": (i, [vp, ctypes.c_uint64, pvp]),
        "bf_net_destroy": (None, [vp]),
        "bf_net_get_params": (i, [vp, vp, vp]),
        "bf_net_set_params": (i, [vp, vp, vp]),
        "bf_net_forward": (i, [vp, vp, vp, vp, vp]),
        "bf_net_train_step": (i, [vp, vp, vp, vp, vp, ctypes.c_float, ctypes.POINTER(d), vp]),
        "bf_surrogate_variance": (i, [vp, vp, vp, i, i, ctypes.c_uint64, d, i, i, u, vp, vp, vp,
                                      ctypes.POINTER(i), ctypes.POINTER(i)]),
        "bf_net_bench": (i, [vp, vp, vp, i, i, ctypes.POINTER(d)]),
        "bf_autotune_rhs_block": (i, [vp, vp, i, i, ctypes.POINTER(i), vp]),
        "bf_export_trilinear_rows": (i, [vp, vp, vp, i, vp, ctypes.POINTER(Intrinsics), vp, vp, vp,
                                         ctypes.POINTER(i64)]),
        "bf_export_precision27": (i, [vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def launch_count() -> int:
    """Kernels the library has run in this process (bf_launch_count)."""
    n = ctypes.c_int64()
    load_library().bf_launch_count(ctypes.byref(n))
    return n.value


def _ptr(a):
    """Raw pointer of a tensor / ndarray (must be contiguous)."""
    if a is None:
        return None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _intr(K) -> Intrinsics:
    fx, fy, cx, cy, W, H = K
    return Intrinsics(float(fx), float(fy), float(cx), float(cy), int(W), int(H))


class Context:
    """bf_ctx: one device and one CUDA stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load_library()
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        self._p = ctypes.c_void_p()
        st = self.lib.bf_create(device, ctypes.c_void_p(stream or 0), ctypes.byref(self._p))
        if st != BF_OK:
            raise BfError(st, "bf_create failed")

    def check(self, st: int, what: str):
        if st != BF_OK:
            raise BfError(st, f"{what}: {self.lib.bf_last_error(self._p).decode()}")

    def set_stream(self, stream):
        self.check(self.lib.bf_set_stream(self._p, ctypes.c_void_p(stream)), "bf_set_stream")

    def close(self):
        if self._p:
            self.lib.bf_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the six calls --------------------------------------------------
    def build_band(self, depth, poses, K, n, voxel, origin, band_vox, trunc_vox, lam=1.0, lam_b=1.0,
                   sig_a=0.0, sig_b=0.0, sig_pose=0.0, sig_model=0.0) -> "Band":
        T = int(depth.shape[0])
        g = Grid(int(n), float(voxel), (ctypes.c_float * 3)(*[float(v) for v in origin]))
        p = Params(band_vox, trunc_vox, lam, lam_b, sig_a, sig_b, sig_pose, sig_model)
        out = ctypes.c_void_p()
        self.check(self.lib.bf_build_band(self._p, _ptr(depth), T, _ptr(poses), ctypes.byref(_intr(K)),
                                          ctypes.byref(g), ctypes.byref(p), ctypes.byref(out)), "bf_build_band")
        return Band(self, out, int(n), float(voxel), tuple(origin))

    def build_band_w(self, w, depth=None, poses=None) -> "Band":
        """build_band for a synth.Workload (depth / poses may be given as device tensors)."""
        return self.build_band(w.depth if depth is None else depth, w.poses if poses is None else poses, w.intr,
                               w.n, w.h, w.origin, w.band_vox, w.trunc_vox, w.lam, w.lam_b, w.sig_a, w.sig_b,
                               w.sig_pose, w.sig_model)


@dataclass
class SolveInfo:
    iters: int
    rel_res: float
    status: int


class Band:
    """bf_band handle with the per-band calls."""

    def __init__(self, ctx: Context, ptr, n, voxel, origin):
        self.ctx, self._p = ctx, ptr
        self.n, self.voxel, self.origin = n, voxel, origin
        N, NB, NC = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        ctx.check(ctx.lib.bf_band_info(ptr, ctypes.byref(N), ctypes.byref(NB), ctypes.byref(NC)), "bf_band_info")
        self.N, self.NB, self.n_cand = N.value, NB.value, NC.value

    def free(self):
        if self._p:
            self.ctx.lib.bf_band_free(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _new(self, dtype, shape, device):
        if device == "numpy":
            return np.empty(shape, dtype=dtype)
        return torch.empty(shape, dtype=dtype, device=device)

    def export_band(self, device="numpy"):
        """dict of lin (int64), tsdf, wcount, bdry, brick_dir, mask (see bf_export_band)."""
        nb = self.n // 8
        tdt = {"i64": np.int64, "f32": np.float32, "i32": np.int32, "u8": np.uint8, "u64": np.uint64}
        if device != "numpy":
            tdt = {"i64": torch.int64, "f32": torch.float32, "i32": torch.int32, "u8": torch.uint8,
                   "u64": torch.int64}
        out = dict(lin=self._new(tdt["i64"], (self.N,), device), tsdf=self._new(tdt["f32"], (self.N,), device),
                   wcount=self._new(tdt["i32"], (self.N,), device), bdry=self._new(tdt["u8"], (self.N,), device),
                   brick_dir=self._new(tdt["i32"], (nb ** 3,), device),
                   mask=self._new(tdt["u64"], (self.NB, 8), device))
        self.ctx.check(self.ctx.lib.bf_export_band(self.ctx._p, self._p, _ptr(out["lin"]), _ptr(out["tsdf"]),
                                                   _ptr(out["wcount"]), _ptr(out["bdry"]), _ptr(out["brick_dir"]),
                                                   _ptr(out["mask"])), "bf_export_band")
        return out

    def integrate_depth(self, depth, poses, K, deterministic=False, trilinear=False):
        """Accumulate the frames' observations; deterministic=True sums them in int64 fixed point;
        trilinear=True uses the trilinear rows (27-point precision)."""
        if trilinear:
            self.ctx.check(self.ctx.lib.bf_integrate_depth_ex(self.ctx._p, self._p, _ptr(depth), int(depth.shape[0]),
                                                              _ptr(poses), ctypes.byref(_intr(K)),
                                                              BF_INTEGRATE_TRILINEAR), "bf_integrate_depth_ex")
            return
        if deterministic:
            self.ctx.check(self.ctx.lib.bf_integrate_depth_ex(self.ctx._p, self._p, _ptr(depth), int(depth.shape[0]),
                                                              _ptr(poses), ctypes.byref(_intr(K)),
                                                              BF_INTEGRATE_DETERMINISTIC), "bf_integrate_depth_ex")
            return
        self.ctx.check(self.ctx.lib.bf_integrate_depth(self.ctx._p, self._p, _ptr(depth), int(depth.shape[0]),
                                                       _ptr(poses), ctypes.byref(_intr(K))), "bf_integrate_depth")

    def export_observations_f64(self):
        """(d, hdata) as FP64 numpy arrays."""
        d, hd = np.empty(self.N, np.float64), np.empty(self.N, np.float64)
        self.ctx.check(self.ctx.lib.bf_export_observations_f64(self.ctx._p, self._p, _ptr(d), _ptr(hd)),
                       "bf_export_observations_f64")
        return d, hd

    def export_trilinear_rows(self, depth, poses, K):
        """(idx [M,8] int32, wts [M,8] float32, used [M] bool) of the frames' trilinear rows
        (bf_export_trilinear_rows), M = T H W (2b + 1) in the order (frame, pixel, k)."""
        M = ctypes.c_int64()
        args = (self.ctx._p, self._p, _ptr(depth), int(depth.shape[0]), _ptr(poses), ctypes.byref(_intr(K)))
        self.ctx.check(self.ctx.lib.bf_export_trilinear_rows(*args, None, None, None, ctypes.byref(M)),
                       "bf_export_trilinear_rows")
        idx = np.empty((M.value, 8), np.int32)
        wts = np.empty((M.value, 8), np.float32)
        used = np.empty(M.value, np.uint8)
        self.ctx.check(self.ctx.lib.bf_export_trilinear_rows(*args, _ptr(idx), _ptr(wts), _ptr(used),
                                                             ctypes.byref(M)), "bf_export_trilinear_rows")
        return idx, wts, used.astype(bool)

    def export_precision27(self):
        """coef [27, N] float32 (bf_export_precision27)."""
        out = np.empty((27, self.N), np.float32)
        self.ctx.check(self.ctx.lib.bf_export_precision27(self.ctx._p, self._p, _ptr(out)), "bf_export_precision27")
        return out

    def reset_observations(self):
        self.ctx.check(self.ctx.lib.bf_reset_observations(self.ctx._p, self._p), "bf_reset_observations")

    def export_system(self, device="numpy"):
        out = {k: self._new(np.float32 if device == "numpy" else torch.float32, (self.N,), device)
               for k in ("d", "hdata", "qdiag", "rhs")}
        self.ctx.check(self.ctx.lib.bf_export_system(self.ctx._p, self._p, _ptr(out["d"]), _ptr(out["hdata"]),
                                                     _ptr(out["qdiag"]), _ptr(out["rhs"])), "bf_export_system")
        return out

    def spmv(self, x, y):
        self.ctx.check(self.ctx.lib.bf_spmv(self.ctx._p, self._p, _ptr(x), _ptr(y)), "bf_spmv")
        return y

    def spmm(self, X, Y):
        """Y = Q X for X, Y of shape [N, R] (R = 8, 16 or 32, rows contiguous)."""
        if X.shape != Y.shape or X.shape[0] != self.N:
            raise ValueError("X and Y must both have shape [N, R]")
        self.ctx.check(self.ctx.lib.bf_spmm(self.ctx._p, self._p, _ptr(X), int(X.shape[1]), _ptr(Y)), "bf_spmm")
        return Y

    def solve_mean(self, mu, rel_tol=1e-6, max_iter=20000, fp64=False, warm=False, raise_on_fail=True):
        it, rr = ctypes.c_int(), ctypes.c_double()
        flags = (BF_SOLVE_FP64 if fp64 else 0) | (BF_SOLVE_WARM if warm else 0)
        st = self.ctx.lib.bf_solve_mean(self.ctx._p, self._p, rel_tol, max_iter, flags, _ptr(mu),
                                        ctypes.byref(it), ctypes.byref(rr))
        if raise_on_fail:
            self.ctx.check(st, "bf_solve_mean")
        return SolveInfo(it.value, rr.value, st)

    def estimate_variance(self, s, K, seed=0, rel_tol=1e-6, max_iter=20000, rhs_block=0, raise_on_fail=True):
        it = ctypes.c_int()
        st = self.ctx.lib.bf_estimate_variance(self.ctx._p, self._p, int(K), int(seed), rel_tol, max_iter,
                                               int(rhs_block), 0, _ptr(s), ctypes.byref(it))
        if raise_on_fail:
            self.ctx.check(st, "bf_estimate_variance")
        return SolveInfo(it.value, 0.0, st)

    def estimate_variance_range(self, s_part, k_begin, k_end, seed=0, rel_tol=1e-6, max_iter=20000, rhs_block=0,
                                scale=1.0):
        """scale x the probe sum over probes [k_begin, k_end) (bf_estimate_variance_range)."""
        it = ctypes.c_int()
        st = self.ctx.lib.bf_estimate_variance_range(self.ctx._p, self._p, int(k_begin), int(k_end), float(scale),
                                                     int(seed), rel_tol, max_iter, int(rhs_block), 0, _ptr(s_part),
                                                     ctypes.byref(it))
        self.ctx.check(st, "bf_estimate_variance_range")
        return SolveInfo(it.value, 0.0, st)

    def surrogate_variance(self, log_s_hat, s, K, K_judge=16, seed=0, rel_tol=1e-6, max_iter=20000, rhs_block=0):
        """diag(Q^-1) with the network's estimate on judge-accepted bricks (bf_surrogate_variance).

        Returns (SolveInfo, accepted [NB] uint8, brick_stat [NB, 2] float64, n_accepted)."""
        it, na = ctypes.c_int(), ctypes.c_int()
        acc = np.zeros(self.NB, np.uint8)
        stat = np.zeros((self.NB, 2), np.float64)
        st = self.ctx.lib.bf_surrogate_variance(self.ctx._p, self._p, _ptr(log_s_hat), int(K), int(K_judge),
                                                int(seed), rel_tol, max_iter, int(rhs_block), 0, _ptr(s),
                                                _ptr(acc), _ptr(stat), ctypes.byref(na), ctypes.byref(it))
        self.ctx.check(st, "bf_surrogate_variance")
        return SolveInfo(it.value, 0.0, st), acc, stat, na.value

    def autotune_rhs_block(self, K: int, force: bool = False):
        """Probe block width chosen by the library's autotuner; returns (R, ms per iteration at 8, 16, 32)."""
        R = ctypes.c_int()
        ms = np.zeros(3, np.float64)
        self.ctx.check(self.ctx.lib.bf_autotune_rhs_block(self.ctx._p, self._p, int(K), int(bool(force)),
                                                          ctypes.byref(R), _ptr(ms)), "bf_autotune_rhs_block")
        return R.value, ms

    def extract_surface(self, mu, device="numpy", method="mc"):
        """(verts [V,3], tris [F,3]) by marching cubes (method="mc") or dual contouring (method="dc")."""
        nv, nt = ctypes.c_int64(), ctypes.c_int64()
        fn = {"mc": self.ctx.lib.bf_extract_surface, "dc": self.ctx.lib.bf_extract_surface_dc}[method]
        self.ctx.check(fn(self.ctx._p, self._p, _ptr(mu), ctypes.byref(nv), ctypes.byref(nt)),
                       "bf_extract_surface" + ("_dc" if method == "dc" else ""))
        V = self._new(np.float32 if device == "numpy" else torch.float32, (nv.value, 3), device)
        F = self._new(np.int32 if device == "numpy" else torch.int32, (nt.value, 3), device)
        self.ctx.check(self.ctx.lib.bf_get_surface(self.ctx._p, _ptr(V) if nv.value else None,
                                                   _ptr(F) if nt.value else None), "bf_get_surface")
        return V, F

    def score_views(self, mu, s, cand_poses, K, eps=1.0):
        V = int(cand_poses.shape[0])
        U = np.zeros(V, np.float64)
        best = ctypes.c_int()
        self.ctx.check(self.ctx.lib.bf_score_views(self.ctx._p, self._p, _ptr(mu), _ptr(s), _ptr(cand_poses), V,
                                                   ctypes.byref(_intr(K)), float(eps), _ptr(U),
                                                   ctypes.byref(best)), "bf_score_views")
        return U, best.value

    def score_views_exact(self, mu, cand_poses, K, eps=1.0, K_probes=16, seed=0, rel_tol=1e-6, max_iter=20000,
                          rhs_block=0):
        """Exact utilities (bf_score_views_exact): returns (U [V] float64, best, total probe iterations)."""
        V = int(cand_poses.shape[0])
        U = np.zeros(V, np.float64)
        best, it = ctypes.c_int(), ctypes.c_int()
        self.ctx.check(self.ctx.lib.bf_score_views_exact(self.ctx._p, self._p, _ptr(mu), _ptr(cand_poses), V,
                                                         ctypes.byref(_intr(K)), float(eps), int(K_probes),
                                                         int(seed), float(rel_tol), int(max_iter), int(rhs_block),
                                                         _ptr(U), ctypes.byref(best), ctypes.byref(it)),
                       "bf_score_views_exact")
        return U, best.value, it.value

    def bench_kernel(self, which: int, R: int = 32, reps: int = 50) -> float:
        """Mean ms per launch of one solver kernel (bf_bench_kernel)."""
        ms = ctypes.c_double()
        self.ctx.check(self.ctx.lib.bf_bench_kernel(self.ctx._p, self._p, int(which), int(R), int(reps),
                                                    ctypes.byref(ms)), "bf_bench_kernel")
        return ms.value


def net_nparams() -> int:
    return int(load_library().bf_net_nparams())


class Net:
    """The learned warm start / variance surrogate network (bf_net_*)."""

    def __init__(self, ctx: Context, seed: int = 0):
        self.ctx = ctx
        p = ctypes.c_void_p()
        ctx.check(ctx.lib.bf_net_create(ctx._p, int(seed), ctypes.byref(p)), "bf_net_create")
        self._p = p
        self.P = net_nparams()

    def close(self):
        if self._p:
            self.ctx.lib.bf_net_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self, out=None):
        out = np.empty(self.P, np.float32) if out is None else out
        self.ctx.check(self.ctx.lib.bf_net_get_params(self.ctx._p, self._p, _ptr(out)), "bf_net_get_params")
        return out

    def set_params(self, params):
        self.ctx.check(self.ctx.lib.bf_net_set_params(self.ctx._p, self._p, _ptr(params)), "bf_net_set_params")

    def forward(self, band: "Band", mu_hat, log_s_hat):
        self.ctx.check(self.ctx.lib.bf_net_forward(self.ctx._p, self._p, band._p, _ptr(mu_hat), _ptr(log_s_hat)),
                       "bf_net_forward")

    def bench(self, band: "Band", which: int, reps: int = 20) -> float:
        """Mean ms per repetition of the network's kernels (bf_net_bench)."""
        ms = ctypes.c_double()
        self.ctx.check(self.ctx.lib.bf_net_bench(self.ctx._p, self._p, band._p, int(which), int(reps),
                                                 ctypes.byref(ms)), "bf_net_bench")
        return ms.value

    def train_step(self, band: "Band", mu, s, lr=1e-3, grad=None) -> float:
        loss = ctypes.c_double()
        self.ctx.check(self.ctx.lib.bf_net_train_step(self.ctx._p, self._p, band._p, _ptr(mu), _ptr(s),
                                                      float(lr), ctypes.byref(loss), _ptr(grad)),
                       "bf_net_train_step")
        return loss.value
