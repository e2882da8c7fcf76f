"""Batches of independent LPs (argument marshalling and host-side sharding).

A batch is factorised as one block-diagonal system (``ipm_analyse_batch``):
the elimination forest holds one tree per instance, so the level-scheduled
launches of Sec. 4.3 process the fronts of all instances together, while the
pivot floor eps_piv ||K_b||_1 of Sec. 4.5 stays per instance.  Across GPUs
the instances are independent, so they are sharded with no data exchange.
"""
from __future__ import annotations

import numpy as np

from . import IPM_ORD_AMD, ipm_analyse_batch
from .solver import Solver


def lpt_partition(costs, world: int) -> list[list[int]]:
    """Longest-processing-time-first assignment of items to ``world`` bins.

    Deterministic: items by decreasing cost (ties by index) go to the bin
    with the smallest load (ties by bin index).  Returns the item indices of
    every bin in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(costs.size), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    bins: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        b = min(range(world), key=lambda r: (load[r], r))
        bins[b].append(i)
        load[b] += float(costs[i])
    return [sorted(b) for b in bins]


def instance_cost(m: int, n: int, nnz: int) -> float:
    """A-priori work estimate of one instance for load balancing,
    nnz(A) * sqrt(m): it orders the random sparse instances of one family by
    their factorisation work without analysing them."""
    return float(nnz) * float(max(m, 1)) ** 0.5


def shard(lps, rank: int, world: int) -> list[int]:
    """Indices of the instances rank ``rank`` of ``world`` factorises."""
    costs = [instance_cost(lp.m, lp.n, int(lp.colptr[-1])) for lp in lps]
    return lpt_partition(costs, world)[rank]


def shard_sizes(sizes, rank: int, world: int, per_col: int = 5) -> list[int]:
    """The same partition from the instance sizes alone ((m_i, n_i) with
    per_col nonzeros per column), so that a rank generates only its own
    instances."""
    costs = [instance_cost(m, n, per_col * n) for m, n in sizes]
    return lpt_partition(costs, world)[rank]


class BatchSolver(Solver):
    """One context for a list of independent LPs (block-diagonal forest)."""

    def __init__(self, lps, ordering=IPM_ORD_AMD, device=0, **options):
        self.lps = list(lps)
        if not self.lps:
            raise ValueError("empty batch")
        self.ms = np.array([lp.m for lp in self.lps], dtype=np.int32)
        self.ns = np.array([lp.n for lp in self.lps], dtype=np.int32)
        self.m_off = np.concatenate([[0], np.cumsum(self.ms)]).astype(np.int64)
        self.n_off = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)
        colptrs = np.concatenate([np.asarray(lp.colptr, dtype=np.int64) for lp in self.lps])
        rowidxs = np.concatenate([np.asarray(lp.rowidx, dtype=np.int32) for lp in self.lps])
        vals = np.concatenate([np.asarray(lp.vals, dtype=np.float64) for lp in self.lps])
        self._batch = (self.ms, self.ns, colptrs, rowidxs)
        super().__init__(int(self.m_off[-1]), int(self.n_off[-1]), None, None, vals, ordering=ordering,
                         device=device, **options)

    def _analyse(self, m, n, colptr, rowidx, form, ordering, user_perm):
        ms, ns, cps, ris = self._batch
        return ipm_analyse_batch(self.ctx, ms, ns, cps, ris, ordering)

    def concat(self, per_instance):
        """Concatenate per-instance vectors (Theta, r7 or r1) in batch order."""
        return np.concatenate([np.asarray(v, dtype=np.float64) for v in per_instance])

    def split(self, dx, dy):
        """Per-instance (dx_b, dy_b) host arrays of a batch solution."""
        dx = dx.cpu().numpy() if hasattr(dx, "cpu") else np.asarray(dx)
        dy = dy.cpu().numpy() if hasattr(dy, "cpu") else np.asarray(dy)
        return [(dx[self.n_off[b]:self.n_off[b + 1]], dy[self.m_off[b]:self.m_off[b + 1]])
                for b in range(len(self.lps))]
