"""Next-best-view utility against the number of probes, with and without the
TSDF anchor: a synthetic analogue of the paper's NBV utility trends (Sec. 4,
the figure on NBV utility under anchoring configurations).

For each configuration (anchor weight lambda_b = 1, and lambda_b = 0) the band
of a seeded workload is built and integrated once, the mean solved, and for
each probe count K the variance is estimated (Sec. 3.7) and the candidate
views scored (Sec. 3.8): the diagonal-update utility of bf_score_views and,
with --exact, the re-solved utility of bf_score_views_exact.  Every step runs
in the CUDA library; this module only sequences calls and prints one JSON
line per (configuration, K).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def run(workload: str = "sphere64", Ks=(4, 8, 16, 32, 64), candidates: int = 16, exact: bool = False,
        seed: int = 0, rel_tol: float = 1e-8, n=None, frames=None):
    import torch

    import synth
    from . import bfsdf, build

    build.build()
    ctx = bfsdf.Context(0)
    rows = []
    for anchored in (True, False):
        w = synth.make_workload(workload, n=n, frames=frames)
        w.lam_b = 1.0 if anchored else 0.0
        depth, poses = torch.from_numpy(w.depth).cuda(), torch.from_numpy(w.poses).cuda()
        band = ctx.build_band_w(w, depth, poses)
        band.integrate_depth(depth, poses, w.intr)
        mu = torch.empty(band.N, device="cuda")
        info = band.solve_mean(mu, rel_tol=rel_tol, raise_on_fail=False)
        cand = torch.from_numpy(np.ascontiguousarray(w.cand_poses[:candidates])).cuda()
        for K in Ks:
            s = torch.empty(band.N, device="cuda")
            vi = band.estimate_variance(s, K=K, seed=seed, rel_tol=rel_tol, raise_on_fail=False)
            U, best = band.score_views(mu, s, cand, w.cand_intr)
            row = {"workload": workload, "n": w.n, "frames": w.T, "anchored": anchored, "lambda_b": w.lam_b, "K": K, "N_band": band.N,
                   "mean_iters": info.iters, "mean_status": info.status, "variance_status": vi.status,
                   "best": best, "U_best": float(U[best]),
                   "U_mean": float(np.mean(U)), "s_mean": float(s.mean().item())}
            if exact:
                Ue, beste, _ = band.score_views_exact(mu, cand, w.cand_intr, K_probes=K, seed=seed, rel_tol=rel_tol)
                row.update(best_exact=beste, U_best_exact=float(Ue[beste]), U_mean_exact=float(np.mean(Ue)))
            rows.append(row)
            print(json.dumps(row), flush=True)
        band.free()
    return rows


def main(argv=None) -> None:
    """Print the utility trend as JSON lines."""
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--workload", default="sphere64")
    ap.add_argument("--K", type=int, nargs="+", default=[4, 8, 16, 32, 64])
    ap.add_argument("--candidates", type=int, default=16)
    ap.add_argument("--exact", action="store_true", help="also the re-solved utilities (V + 1 estimates per K)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--n", type=int, default=None, help="grid size (the voxel size scales so the scene fits)")
    ap.add_argument("--frames", type=int, default=None, help="number of input views (fewer: sparser coverage)")
    a = ap.parse_args(argv)
    run(a.workload, a.K, a.candidates, a.exact, a.seed, n=a.n, frames=a.frames)


if __name__ == "__main__":
    main()
