"""Two-rank (gloo, CPU) check of the sharding arithmetic used when the location range is
split across GPUs: each rank evaluates the terms of a disjoint range of ordered locations,
the per-rank partial sums are gathered, and rank 0 combines them in rank order; the result
must equal the unsplit evaluation within the log-likelihood tolerance."""
import os
import socket

import numpy as np
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
    perm = oracle.order_random(n, 7)
    xo, yo = xy[perm], y[perm]
    bounds = np.linspace(0, n, world + 1).astype(np.int64)
    rows = np.arange(bounds[rank], bounds[rank + 1])
    part = oracle.vecchia_rows(xo, yo, m, theta, rows=rows, want_grad=True)
    local = torch.tensor(oracle.compensated_sum(part), dtype=torch.float64)
    gathered = [torch.zeros(4, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, local)
    if rank == 0:
        combined = oracle.compensated_sum(np.stack([g.numpy() for g in gathered]))
        full_terms = oracle.vecchia_rows(xo, yo, m, theta, want_grad=True)
        full = oracle.compensated_sum(full_terms)
        den = np.abs(full_terms).sum(axis=0)
        q.put((combined.tolist(), full.tolist(), den.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_location_split_matches_unsplit():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    combined, full, den = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert abs(combined[0] - full[0]) <= 1e-9 * den[0]
    for k in (1, 2, 3):
        assert abs(combined[k] - full[k]) <= 1e-7 * den[k]
