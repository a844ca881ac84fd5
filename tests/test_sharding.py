"""Probe sharding across ranks: world_size-2 gloo processes on CPU.

Each rank computes the partial probe sum of its range with the oracle (the
stand-in for a rank's GPU), the ranks combine with a real all-reduce, and the
result equals the single-process estimate.  The GPU form of the partial sum
is checked in tests/test_gpu_parity.py.
"""
import os

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2602_19697_gb300.sharding import probe_range


def test_probe_ranges_partition_the_probes():
    for K in (0, 1, 7, 16, 64, 65):
        for world in (1, 2, 3, 8):
            rs = [probe_range(r, world, K) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == K
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        probe_range(2, 2, 4)


def _worker(rank, world, port, K, seed, out_dir):
    import oracle
    import synth
    from paper_2602_19697_gb300.sharding import estimate_variance_sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.make_workload("sphere64", n=24, image_scale=0.5, frames=12)
    b = oracle.build_band_w(w)
    d, hd, _ = oracle.integrate_w(b, w)
    qd, rhs = oracle.assemble(b, d, hd, w.lam, w.lam_b)

    def partial(k0, k1):
        if k1 <= k0:
            return torch.zeros(b.N, dtype=torch.float64)
        s, st, it, _ = oracle.hutchinson(b, w.lam, qd, k1 - k0, seed, tol=1e-12, k0=k0)
        return torch.from_numpy(s * ((k1 - k0) / K))     # this rank's part, scaled by 1/K

    s = estimate_variance_sharded(partial, K, rank, world)
    np.save(os.path.join(out_dir, f"s{rank}.npy"), s.numpy())
    torch.distributed.destroy_process_group()


def test_sharded_estimate_equals_single_process(tmp_path):
    import oracle
    import synth
    K, seed, world = 9, 4, 2
    port = 29500 + (os.getpid() % 1000)
    mp.spawn(_worker, args=(world, port, K, seed, str(tmp_path)), nprocs=world, join=True)
    w = synth.make_workload("sphere64", n=24, image_scale=0.5, frames=12)
    b = oracle.build_band_w(w)
    d, hd, _ = oracle.integrate_w(b, w)
    qd, rhs = oracle.assemble(b, d, hd, w.lam, w.lam_b)
    ref, *_ = oracle.hutchinson(b, w.lam, qd, K, seed, tol=1e-12)
    for r in range(world):
        s = np.load(tmp_path / f"s{r}.npy")
        np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-15)


def _faulty_worker(rank, world, port, out_dir, die):
    import datetime
    import torch.distributed as dist
    from paper_2602_19697_gb300.sharding import estimate_variance_sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))

    def part(k0, k1):
        if rank == 1:
            if die:
                os._exit(3)  # the rank disappears before any collective
            raise RuntimeError("probe solve failed on this rank")
        return torch.ones(4, dtype=torch.float64)

    try:
        estimate_variance_sharded(part, 8, rank, world)
        result = "ok"
    except Exception as e:  # the failing rank's own error, or the error the others receive
        result = type(e).__name__
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(result)
    os._exit(3 if rank == 1 else 0)


def _run_faulty(tmp_path, die):
    world = 2
    port = 29500 + ((os.getpid() + (517 if die else 733)) % 1000)
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_faulty_worker, args=(r, world, port, str(tmp_path), die)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=60)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    assert procs[1].exitcode == 3
    return (tmp_path / "r0.txt").read_text()


def test_a_failed_rank_is_named_to_the_others(tmp_path):
    """Host-injected fault: rank 1's probe solve raises.  It reports the
    failure in the status all-reduce and re-raises its own error; rank 0
    raises ProbeShardError instead of summing a partial result."""
    r0 = _run_faulty(tmp_path, die=False)
    assert (tmp_path / "r1.txt").read_text() == "RuntimeError"
    assert r0 == "ProbeShardError", r0


def test_a_vanished_rank_ends_the_others_collective_with_an_error(tmp_path):
    """Host-injected fault: rank 1 exits before any collective.  Rank 0's
    status all-reduce ends with the process group's error (the peer's
    connection closed, or the 20 s group timeout) instead of hanging."""
    r0 = _run_faulty(tmp_path, die=True)
    assert r0 not in ("ok", "ProbeShardError"), r0
    assert r0 in ("RuntimeError", "DistBackendError", "DistNetworkError"), r0
