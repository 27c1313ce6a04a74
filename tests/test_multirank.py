"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): disjoint
orbital ownership per rank, max-over-ranks timing, whole-job throughput, and
the exchange each multi-rank step ends with (bench.sum_over_ranks: the
density and the energy sums over the ranks, the same result on every rank)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle.wavelet as O
    from paper_0904_1543_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        per_rank = 2
        first = bench.rank_first_orbital(rank, per_rank)
        owned = list(range(first, first + per_rank))
        # each rank times a different amount of work; the job takes the max
        ms = [10.0 + rank, 20.0 - rank]
        mx = bench.max_over_ranks(ms, dist, world)
        thr = bench.job_throughput(per_rank, world, 5, mx[0])
        # density of this rank's orbitals, then the sum over ranks
        n = (3, 2, 4)
        V = inputs.gaussian_potential(7, 0, n)
        rho = np.zeros((8, 4, 6))
        for o in owned:
            rho += O.hpsi_local(inputs.orbital(7, o, n), V, 2.0, n)["rho"]
        # the exchange of bench.py's multi-rank step: density and energy sums
        t = torch.from_numpy(rho)
        en = torch.tensor([float(rank + 1), 0.5], dtype=torch.float64)
        bench.sum_over_ranks([t, en], dist, world)
        out[rank] = (owned, mx, thr, t.numpy().copy(), en.numpy().copy())
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    owned0, mx0, thr0, rho0, en0 = out[0]
    owned1, mx1, thr1, rho1, en1 = out[1]
    assert np.array_equal(en0, en1) and list(en0) == [3.0, 1.0]
    assert set(owned0).isdisjoint(owned1)
    assert owned0 + owned1 == [0, 1, 2, 3]
    assert mx0 == mx1 == [11.0, 20.0]
    assert thr0 == thr1 == pytest.approx(2 * 2 * 5 / 11e-3)
    assert np.array_equal(rho0, rho1)
    # the rank sum equals the single-process density of all four orbitals
    import oracle.wavelet as O
    from paper_0904_1543_gb300 import inputs
    n = (3, 2, 4)
    V = inputs.gaussian_potential(7, 0, n)
    ref = sum(O.hpsi_local(inputs.orbital(7, o, n), V, 2.0, n)["rho"] for o in range(4))
    assert np.max(np.abs(rho0 - ref)) < 1e-15
