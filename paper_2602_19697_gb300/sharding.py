"""Probe sharding of the diagonal estimator across ranks (one GPU per rank).

Probe k is a function of (seed, k, voxel) only (Sec. 3.7 estimator with
counter-based Rademacher probes), so the K probe solves split into contiguous
ranges, one per rank, with no communication until the end: each rank sums
z (.) Q^-1 z over its range and one all-reduce (sum) of the N-vector, divided
by K, gives the estimate every rank would have computed alone.
"""
from __future__ import annotations

from typing import Callable, Tuple

import torch


def probe_range(rank: int, world: int, K: int) -> Tuple[int, int]:
    """Contiguous share [k0, k1) of probes 0..K-1 for `rank` (sizes differ by at most one)."""
    if not (0 <= rank < world) or K < 0:
        raise ValueError("need 0 <= rank < world and K >= 0")
    base, extra = divmod(K, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def combine(partial: torch.Tensor, K: int, group=None) -> torch.Tensor:
    """All-reduce (sum) the per-rank partial sums in place and divide by K."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    partial /= K
    return partial


def estimate_variance_sharded(partial_fn: Callable[[int, int], torch.Tensor], K: int, rank: int, world: int,
                              group=None) -> torch.Tensor:
    """s for K probes: this rank computes partial_fn(k0, k1) = sum over its
    probe range of z (.) Q^-1 z (an [N] tensor; zeros for an empty range),
    then the ranks combine."""
    k0, k1 = probe_range(rank, world, K)
    part = partial_fn(k0, k1)
    return combine(part, K, group)


def gpu_partial_fn(band, N: int, seed: int, rel_tol: float = 1e-6, rhs_block: int = 0, device="cuda"):
    """partial_fn backed by the CUDA library (bf_estimate_variance_range)."""
    def fn(k0: int, k1: int) -> torch.Tensor:
        out = torch.zeros(N, dtype=torch.float32, device=device)
        if k1 > k0:
            band.estimate_variance_range(out, k0, k1, seed=seed, rel_tol=rel_tol, rhs_block=rhs_block)
        return out
    return fn
