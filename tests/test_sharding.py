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
        return torch.from_numpy(s * (k1 - k0))

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


def _faulty_worker(rank, world, port, out_dir):
    import datetime
    import torch.distributed as dist
    from paper_2602_19697_gb300.sharding import estimate_variance_sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))

    def partial(k0, k1):
        if rank == 1:
            raise RuntimeError("probe solve failed on this rank")
        return torch.ones(4, dtype=torch.float64)

    try:
        estimate_variance_sharded(partial, 8, rank, world)
        result = "ok"
    except Exception as e:  # the failing rank's own error, or the collective's on the others
        result = type(e).__name__
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(result)
    if rank == 1:
        os._exit(3)  # the failed rank leaves without joining the all-reduce
    os._exit(0)


def test_a_failed_rank_is_reported_to_the_others_not_waited_for(tmp_path):
    """Host-injected fault: rank 1's probe solve raises and the rank exits; rank 0's all-reduce must end with an
    error (peer gone, or the process group's timeout) instead of hanging."""
    world = 2
    port = 29500 + ((os.getpid() + 517) % 1000)
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_faulty_worker, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    assert procs[1].exitcode == 3
    assert (tmp_path / "r1.txt").read_text() == "RuntimeError"
    r0 = (tmp_path / "r0.txt").read_text()
    assert r0 != "ok", r0
