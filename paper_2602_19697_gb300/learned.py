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
