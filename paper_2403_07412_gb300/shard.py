"""Splitting one field's likelihood across GPUs (one process per GPU).

The Vecchia log-likelihood is a sum of n independent per-location terms (Sec. V-B,
Algorithm 1), so it shards by contiguous ranges of ordered locations: every rank holds
the same plan (the ordering and conditioning sets; 24 MB of coordinates and data at 1M
locations, plus the neighbour table), evaluates its own range with
``vecchia_loglik_range``, and one all-reduce of the four result doubles
(l, dl/dsigma2, dl/dbeta, dl/dtau2) per theta combines them.  No tile or block moves
between GPUs.  Every output is linear in the per-location sums, so the combined result
equals the single-GPU call up to the order of the floating-point additions.
"""
from __future__ import annotations


def location_ranges(n: int, parts: int):
    """``parts`` contiguous, disjoint ranges [i0, i1) of ordered locations covering [0, n),
    in rank order; sizes differ by at most one location."""
    if n < 0 or parts < 1:
        raise ValueError("n >= 0 and parts >= 1 required")
    base, extra = divmod(n, parts)
    out, i0 = [], 0
    for r in range(parts):
        i1 = i0 + base + (1 if r < extra else 0)
        out.append((i0, i1))
        i0 = i1
    return out


def allreduce_result(t, group=None):
    """Sums a rank's result vector over the process group in place (torch.distributed
    all-reduce: NCCL between GPUs, gloo on CPU).  The only exchange of the sharded path."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def loglik_sharded(plan, y, theta, rank: int, world: int, want_grad: bool = True, out=None, group=None,
                   stream=None):
    """This rank's range of ``plan`` through ``vecchia_loglik_range``, then the all-reduce:
    every rank ends with the whole field's (l[, gradient]) in ``out`` (on the device)."""
    from . import vecchia as V

    i0, i1 = location_ranges(plan.n, world)[rank]
    out = V.vecchia_loglik_range(plan, y, theta, i0, i1, want_grad=want_grad, out=out, stream=stream)
    return allreduce_result(out, group)
