"""Probe sharding of the diagonal estimator across ranks (one GPU per rank).

Probe k is a function of (seed, k, voxel) only (Sec. 3.7 estimator with
counter-based Rademacher probes), so the K probe solves split into contiguous
ranges, one per rank, with no communication until the end.  Each rank's part
is (1/K) sum over its range of z (.) Q^-1 z, computed by the library with the
1/K applied on the device (bf_estimate_variance_range with scale = 1/K), and
one all-reduce (sum) of the N-vector gives the estimate every rank would have
computed alone.

Failures: before the data all-reduce the ranks all-reduce (max) a status
word, so when one rank's probe solves fail, that rank re-raises its own
error and every other rank raises ProbeShardError naming it, instead of
summing partial results.  A rank that dies without reaching the status
all-reduce is detected by the process group itself (the peer's connection
closes, or the group's timeout expires) and the others get the backend's
error.
"""
from __future__ import annotations

from typing import Callable, Tuple

import torch


class ProbeShardError(RuntimeError):
    """Another rank's share of the probe solves failed."""

    def __init__(self, rank: int):
        super().__init__(f"probe solves failed on rank {rank}")
        self.rank = rank


def probe_range(rank: int, world: int, K: int) -> Tuple[int, int]:
    """Contiguous share [k0, k1) of probes 0..K-1 for `rank` (sizes differ by at most one)."""
    if not (0 <= rank < world) or K < 0:
        raise ValueError("need 0 <= rank < world and K >= 0")
    base, extra = divmod(K, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def _status_device(group) -> torch.device:
    dist = _dist()
    if dist is not None and dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def check_ranks(failed: bool, rank: int, group=None) -> int:
    """All-reduce (max) of rank + 1 over the ranks that failed; returns the
    highest failed rank, or -1 when every rank succeeded."""
    dist = _dist()
    if dist is None:
        return rank if failed else -1
    flag = torch.tensor([rank + 1 if failed else 0], dtype=torch.int64, device=_status_device(group))
    dist.all_reduce(flag, op=dist.ReduceOp.MAX, group=group)
    return int(flag.item()) - 1


def combine(part: torch.Tensor, group=None) -> torch.Tensor:
    """All-reduce (sum) the per-rank parts in place (each already scaled by 1/K)."""
    dist = _dist()
    if dist is not None:
        dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    return part


def estimate_variance_sharded(part_fn: Callable[[int, int], torch.Tensor], K: int, rank: int, world: int,
                              group=None) -> torch.Tensor:
    """s for K probes: this rank computes part_fn(k0, k1) = (1/K) sum over its
    probe range of z (.) Q^-1 z (an [N] tensor; zeros for an empty range),
    the ranks check each other's status, then sum the parts."""
    k0, k1 = probe_range(rank, world, K)
    err, part = None, None
    try:
        part = part_fn(k0, k1)
    except Exception as e:  # reported to the other ranks before it is re-raised here
        err = e
    bad = check_ranks(err is not None, rank, group)
    if err is not None:
        raise err
    if bad >= 0:
        raise ProbeShardError(bad)
    return combine(part, group)


def gpu_part_fn(band, N: int, K: int, seed: int, rel_tol: float = 1e-6, rhs_block: int = 0, device="cuda"):
    """part_fn backed by the CUDA library: bf_estimate_variance_range with scale = 1/K."""
    def fn(k0: int, k1: int) -> torch.Tensor:
        out = torch.zeros(N, dtype=torch.float32, device=device)
        if k1 > k0:
            band.estimate_variance_range(out, k0, k1, seed=seed, rel_tol=rel_tol, rhs_block=rhs_block,
                                         scale=1.0 / K)
        return out
    return fn
