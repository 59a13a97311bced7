"""Column sharding of the signal block over several processes (one GPU each).

The random signals are independent (§3.1: the columns of R are i.i.d.), so
the filtered block Y[:, cols] depends only on R[:, cols]: every rank holds the
whole graph and a slab of columns, and the sweeps need no communication. Two
results combine columns and need one collective each:

* the eigenvalue-count moments (§3.2): mu_m = sum over columns, so the
  per-rank moments are summed (all-reduce of 2p + 1 doubles) before the
  counts and the dichotomy, which every rank then evaluates identically;
* the row normalisation of the features (Eq. (6) rows over all eta
  columns): per-row partial sums of squares are summed (all-reduce of N
  doubles) and every rank scales its own columns.

The functions here are the host-side logic only; the per-rank compute is the
library's (paper_1509_08863_gb300) on CUDA tensors, or any array code in
tests that exercise this logic on CPU ranks.
"""
from __future__ import annotations

import numpy as np

__all__ = ["column_shard", "allreduce_sum", "combine_moments", "normalize_rows_sharded"]


def column_shard(n_sig_total: int, world: int, rank: int):
    """[c0, c1): contiguous, as even as possible, covering every column once."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, rem = divmod(int(n_sig_total), int(world))
    c0 = rank * base + min(rank, rem)
    return c0, c0 + base + (1 if rank < rem else 0)


def allreduce_sum(x, group=None, device=None):
    """Sum a float64 array or tensor over the ranks of `group` (returns the same kind)."""
    import torch
    import torch.distributed as dist

    is_np = isinstance(x, np.ndarray)
    t = torch.as_tensor(x, dtype=torch.float64)
    if device is not None:
        t = t.to(device)
    t = t.contiguous()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy() if is_np else t


def combine_moments(mu_local, group=None, device=None) -> np.ndarray:
    """Moments of the whole block from each rank's moments of its columns."""
    return np.asarray(allreduce_sum(np.asarray(mu_local, dtype=np.float64), group, device))


def normalize_rows_sharded(Y_local, sumsq_fn, scale_fn, group=None):
    """Row-normalise a column shard: sumsq_fn(Y_local) -> per-row partial sums
    (float64, same device as Y_local), summed over ranks, then
    scale_fn(Y_local, total) -> normalised shard."""
    part = sumsq_fn(Y_local)
    total = allreduce_sum(part, group)
    return scale_fn(Y_local, total)
