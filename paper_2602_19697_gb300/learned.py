"""Training and use of the learned warm start / variance surrogate.

The network itself (features, tensor-core convolutions, loss, backward pass,
Adam, the probe judge) runs in the CUDA library behind ``bf_net_*`` and
``bf_surrogate_variance``; this module only sequences calls.

Training data: seeded sphere instances (radius, centre offset, ring phase
and noise drawn per instance by ``synth.make_workload(..., variant=i)``).
Per instance the targets are the posterior mean solved in FP64 to a tight
tolerance and a many-probe estimate of diag(Q^-1), both from the library's
own solvers.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import bfsdf

try:
    import torch
except ImportError:  # pragma: no cover
    torch = None


@dataclass
class Example:
    band: "bfsdf.Band"
    mu: "torch.Tensor"  # [N] float32, voxels
    s: "torch.Tensor"   # [N] float32, voxels^2
    depth: "torch.Tensor"
    poses: "torch.Tensor"


def make_example(ctx: "bfsdf.Context", w, K: int = 256, mean_tol: float = 1e-10, var_tol: float = 1e-6,
                 seed: int = 12345) -> Example:
    """Band of workload ``w`` with its mean and variance targets (device tensors)."""
    depth = torch.from_numpy(np.ascontiguousarray(w.depth)).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(w.poses)).cuda()
    band = ctx.build_band_w(w, depth, poses)
    band.integrate_depth(depth, poses, w.intr)
    mu = torch.empty(band.N, device="cuda")
    band.solve_mean(mu, rel_tol=mean_tol, fp64=True)
    s = torch.empty(band.N, device="cuda")
    band.estimate_variance(s, K=K, seed=seed, rel_tol=var_tol)
    return Example(band, mu, s, depth, poses)


def train(net: "bfsdf.Net", data: list[Example], epochs: int, lr: float = 1e-3, shuffle_seed: int = 0,
          lr_final: float | None = None) -> list[float]:
    """Adam over the examples, one band per step; returns the mean loss of each epoch.

    With ``lr_final`` the learning rate decays geometrically to it over the run."""
    rng = np.random.default_rng(shuffle_seed)
    hist = []
    nsteps = max(epochs * len(data), 1)
    step = 0
    for _ in range(epochs):
        tot = 0.0
        for i in rng.permutation(len(data)):
            ex = data[i]
            a = lr if lr_final is None else lr * (lr_final / lr) ** (step / nsteps)
            tot += net.train_step(ex.band, ex.mu, ex.s, lr=a)
            step += 1
        hist.append(tot / max(len(data), 1))
    return hist


def evaluate(net: "bfsdf.Net", data: list[Example]) -> float:
    """Mean loss over the examples without updating the network."""
    return float(np.mean([net.train_step(ex.band, ex.mu, ex.s, lr=0.0) for ex in data])) if data else 0.0


def warm_solve(net: "bfsdf.Net", band: "bfsdf.Band", mu, rel_tol: float = 1e-6, fp64: bool = False):
    """Mean solve started from the network's mu_hat; returns (SolveInfo, log_s_hat)."""
    lsh = torch.empty(band.N, device="cuda")
    net.forward(band, mu, lsh)
    info = band.solve_mean(mu, rel_tol=rel_tol, fp64=fp64, warm=True)
    return info, lsh


def surrogate_report(net: "bfsdf.Net", data: list[Example], K: int = 64, K_judge: int = 16, seed: int = 3) -> dict:
    """Judge acceptance and probe iterations of the surrogate against the K-probe estimate, and the warm start's
    relative residual, averaged over the examples."""
    acc, it_s, it_f, r_net, r_tsdf, med = [], [], [], [], [], []
    for ex in data:
        b = ex.band
        mh, lsh = torch.empty(b.N, device="cuda"), torch.empty(b.N, device="cuda")
        net.forward(b, mh, lsh)
        s = torch.empty(b.N, device="cuda")
        info, _, _, na = b.surrogate_variance(lsh, s, K=K, K_judge=K_judge, seed=seed)
        acc.append(na / max(b.NB, 1))
        it_s.append(info.iters)
        it_f.append(b.estimate_variance(torch.empty(b.N, device="cuda"), K=K, seed=seed).iters)
        rel = (lsh.exp() - ex.s).abs() / torch.maximum(ex.s.abs(), torch.full_like(ex.s, 1e-30))
        med.append(rel.median().item())
        rhs = b.export_system()["rhs"].astype(np.float64)
        for x, out in ((mh, r_net), (torch.from_numpy(b.export_band()["tsdf"] / np.float32(b.voxel)).cuda(), r_tsdf)):
            y = torch.empty_like(x)
            b.spmv(x.contiguous(), y)
            out.append(float(np.linalg.norm(rhs - y.cpu().numpy()) / np.linalg.norm(rhs)))
    return {"bricks_accepted": float(np.mean(acc)), "probe_iters_surrogate": float(np.mean(it_s)),
            "probe_iters_full": float(np.mean(it_f)), "median_rel_err_s": float(np.mean(med)),
            "warm_rel_residual": float(np.mean(r_net)), "tsdf_rel_residual": float(np.mean(r_tsdf))}


def main(argv=None) -> None:
    """Train on seeded sphere instances and report on held-out ones (one JSON line)."""
    import argparse
    import json
    import time

    import synth
    from . import build

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--train", type=int, default=50)
    ap.add_argument("--held-out", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    build.build()
    ctx = bfsdf.Context(0)
    train_set = [make_example(ctx, synth.make_workload("sphere64", variant=i)) for i in range(a.train)]
    held = [make_example(ctx, synth.make_workload("sphere64", variant=1000 + i)) for i in range(a.held_out)]
    net = bfsdf.Net(ctx, seed=a.seed)
    t0 = time.perf_counter()
    hist = train(net, train_set, epochs=a.epochs, lr=a.lr)
    torch.cuda.synchronize()
    out = {"train_loss_first_epoch": hist[0], "train_loss_last_epoch": hist[-1],
           "held_out_loss": evaluate(net, held), "train_seconds": time.perf_counter() - t0,
           "steps": a.epochs * a.train}
    out.update(surrogate_report(net, held))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
