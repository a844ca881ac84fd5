"""Geometry metrics of a reconstructed surface against an analytic scene: a
synthetic analogue of the paper's evaluation (Sec. 4: Chamfer distance,
accuracy, completeness and F-score on the extracted iso-surface, with and
without the TSDF anchor).

  accuracy      mean distance from points sampled on the reconstruction to the
                true surface (|SDF| of the scene)
  completeness  mean distance from points sampled on the true surface to the
                nearest reconstructed sample
  chamfer       (accuracy + completeness) / 2
  precision / recall / F@tau   fractions of reconstruction / true-surface
                samples within tau of the other surface, and their harmonic
                mean

The surface comes from the CUDA library (bf_extract_surface on the posterior
mean); this module samples points and measures distances on the host.
"""
from __future__ import annotations

import json

import numpy as np


def sample_mesh(V: np.ndarray, F: np.ndarray, n: int, rng) -> np.ndarray:
    """n points uniformly distributed over the triangle mesh's area."""
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    if len(F) == 0:
        return np.zeros((0, 3))
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    t = rng.choice(len(F), size=n, p=area / area.sum())
    u, v = rng.random(n), rng.random(n)
    flip = u + v > 1.0
    u[flip], v[flip] = 1.0 - u[flip], 1.0 - v[flip]
    return a[t] + u[:, None] * (b[t] - a[t]) + v[:, None] * (c[t] - a[t])


def sample_surface(sdf, lo, hi, n: int, rng, band: float, iters: int = 8) -> np.ndarray:
    """About n points on the zero set of `sdf` (a callable on [M,3] arrays): points drawn in the box [lo, hi] within
    `band` of the surface, moved along the finite-difference gradient by x - f(x) grad f(x) until |f| < 1e-9."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    pts = []
    got = 0
    eps = 1e-6
    while got < n:
        x = lo + (hi - lo) * rng.random((4 * n, 3))
        x = x[np.abs(sdf(x)) < band]
        for _ in range(iters):
            f = sdf(x)
            g = np.stack([(sdf(x + eps * e) - sdf(x - eps * e)) / (2 * eps) for e in np.eye(3)], 1)
            g /= np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-12)
            x = x - f[:, None] * g
        x = x[np.abs(sdf(x)) < 1e-9]
        pts.append(x)
        got += len(x)
    return np.concatenate(pts)[:n]


def metrics(rec: np.ndarray, gt: np.ndarray, sdf, tau: float) -> dict:
    """Accuracy, completeness, Chamfer distance and precision / recall / F at tau (metres) between reconstruction
    samples rec and true-surface samples gt; the distance of rec to the true surface is |sdf|."""
    from scipy.spatial import cKDTree
    if len(rec) == 0:
        return {"accuracy": float("inf"), "completeness": float("inf"), "chamfer": float("inf"),
                "precision": 0.0, "recall": 0.0, "fscore": 0.0}
    d_rec = np.abs(sdf(rec))
    d_gt, _ = cKDTree(rec).query(gt)
    acc, comp = float(d_rec.mean()), float(d_gt.mean())
    p, r = float(np.mean(d_rec < tau)), float(np.mean(d_gt < tau))
    return {"accuracy": acc, "completeness": comp, "chamfer": 0.5 * (acc + comp), "precision": p, "recall": r,
            "fscore": 0.0 if p + r == 0 else 2 * p * r / (p + r)}


def run(workloads=("sphere64", "union256"), n_pts: int = 200000, tau_vox: float = 1.0, seed: int = 0):
    """For each workload, anchored (lambda_b = 1) and not (lambda_b = 0): posterior mean, marching-cubes surface,
    metrics (tau = tau_vox voxels).  Prints and returns one dict per (workload, anchor)."""
    import torch

    import synth
    from . import bfsdf, build
    build.build()
    ctx = bfsdf.Context(0)
    out = []
    for name in workloads:
        for anchored in (True, False):
            w = synth.make_workload(name)
            w.lam_b = 1.0 if anchored else 0.0
            depth, poses = torch.from_numpy(w.depth).cuda(), torch.from_numpy(w.poses).cuda()
            band = ctx.build_band_w(w, depth, poses)
            band.integrate_depth(depth, poses, w.intr)
            mu = torch.empty(band.N, device="cuda")
            info = band.solve_mean(mu, rel_tol=1e-8, raise_on_fail=False)
            row = {"workload": name, "anchored": anchored, "N_band": band.N, "mean_status": info.status}
            if info.status == 0:
                V, F = band.extract_surface(mu)
                rng = np.random.default_rng(seed)
                rec = sample_mesh(V, F, n_pts, rng)
                ext = 0.5 * w.n * w.h
                gt = sample_surface(w.scene.sdf, (-ext,) * 3, (ext,) * 3, n_pts, rng, band=2 * w.h)
                row.update(triangles=int(len(F)), tau_m=tau_vox * w.h,
                           **metrics(rec, gt, w.scene.sdf, tau_vox * w.h))
            band.free()
            print(json.dumps(row), flush=True)
            out.append(row)
    return out


def main(argv=None) -> None:
    """Print the geometry metrics as JSON lines."""
    import argparse
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--workloads", nargs="+", default=["sphere64", "union256"])
    ap.add_argument("--points", type=int, default=200000)
    ap.add_argument("--tau-vox", type=float, default=1.0)
    a = ap.parse_args(argv)
    run(a.workloads, a.points, a.tau_vox)


if __name__ == "__main__":
    main()
