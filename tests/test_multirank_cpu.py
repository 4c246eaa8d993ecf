"""Multi-rank (gloo, CPU) check of the sharded likelihood path: each rank takes its range
of ordered locations from shard.location_ranges (the split the GPU path uses), evaluates
those terms (here with the oracle, since the CPU has no CUDA library), and the ranks
combine their four result doubles with shard.allreduce_result, the one exchange of the
GPU path.  Every rank must end with the unsplit result within the tolerances; a second
check gathers the per-rank vectors and sums them in rank order on the host."""
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
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2403_07412_gb300 import datagen

    n, m = 1500, 12
    theta = (1.1, 0.07, 1.5, 0.02)
    xy = datagen.uniform_locations(n, 5)
    y = datagen.field_rff(xy, theta, 6, features=256)
    from paper_2403_07412_gb300 import shard

    perm = oracle.order_random(n, 7)
    xo, yo = xy[perm], y[perm]
    i0, i1 = shard.location_ranges(n, world)[rank]
    part = oracle.vecchia_rows(xo, yo, m, theta, rows=np.arange(i0, i1), want_grad=True)
    local = torch.tensor(oracle.compensated_sum(part), dtype=torch.float64)
    gathered = [torch.zeros(4, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, local.clone())
    reduced = shard.allreduce_result(local.clone())
    full_terms = oracle.vecchia_rows(xo, yo, m, theta, want_grad=True)
    full = oracle.compensated_sum(full_terms)
    den = np.abs(full_terms).sum(axis=0)
    in_order = oracle.compensated_sum(np.stack([g.numpy() for g in gathered]))
    q.put((rank, reduced.tolist(), in_order.tolist(), full.tolist(), den.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_location_ranges_partition():
    from paper_2403_07412_gb300 import shard

    for n, parts in ((10, 3), (1_000_000, 8), (7, 7), (3, 5), (0, 2)):
        r = shard.location_ranges(n, parts)
        assert len(r) == parts and r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))
        sizes = [b - a for a, b in r]
        assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_location_split_matches_unsplit(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, reduced, in_order, full, den in results:
        for got in (reduced, in_order):
            assert abs(got[0] - full[0]) <= 1e-9 * den[0], (rank, got, full)
            for k in (1, 2, 3):
                assert abs(got[k] - full[k]) <= 1e-7 * den[k], (rank, k, got, full)
