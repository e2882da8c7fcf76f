"""Seeded generators for the synthetic LP workloads.

Every generator draws from ``numpy.random.default_rng(seed)`` and returns the
constraint matrix A (m x n) in compressed-sparse-column form: 0-based,
row indices sorted inside each column, no duplicates.  The shapes and value
distributions stand in for the paper's Netlib, Mittelmann and PyPSA sets
(Section 5), which are not available here:

* ``random_lp``            -- random sparse LP, k distinct uniform rows per column, N(0,1)
* ``grid_multicommodity``  -- 4-neighbour grid, K commodities, conservation rows
                              (one node row dropped per commodity) plus one joint
                              capacity row per undirected edge, entries +-1
* ``block_angular``        -- independent sparse blocks plus dense linking rows
* ``batched_random``       -- many independent random LPs of log-uniform size
* ``staircase``            -- multi-period LP, each period coupled to the next by
                              identity links

Theta values, right-hand sides and user permutations are drawn here as well so
that both sides of every comparison see identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class LP:
    m: int
    n: int
    colptr: np.ndarray  # int64, n+1
    rowidx: np.ndarray  # int32, nnz
    vals: np.ndarray    # float64, nnz
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])


def _from_coo(m, n, rows, cols, vals, name, meta=None) -> LP:
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((rows, cols))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size:
        dup = (np.diff(cols) == 0) & (np.diff(rows) == 0)
        if dup.any():
            raise ValueError("duplicate entries in generated LP")
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(colptr, cols + 1, 1)
    colptr = np.cumsum(colptr)
    return LP(m, n, colptr, rows.astype(np.int32), vals, name, meta or {})


def random_lp(m: int, n: int, per_col: int, seed: int, name: str = "random") -> LP:
    """``per_col`` distinct rows per column, uniform without replacement, N(0,1)
    values; a row left empty receives one entry in a random column that does
    not already hold it."""
    rng = np.random.default_rng(seed)
    per_col = min(per_col, m)
    rows = np.empty((n, per_col), dtype=np.int64)
    for j in range(n):
        rows[j] = rng.choice(m, size=per_col, replace=False)
    cols = np.repeat(np.arange(n, dtype=np.int64), per_col)
    rows = rows.reshape(-1)
    present = np.zeros(m, dtype=bool)
    present[rows] = True
    extra_r, extra_c = [], []
    for i in np.flatnonzero(~present):
        extra_r.append(int(i))
        extra_c.append(int(rng.integers(n)))
    rows = np.concatenate([rows, np.asarray(extra_r, dtype=np.int64)])
    cols = np.concatenate([cols, np.asarray(extra_c, dtype=np.int64)])
    vals = rng.standard_normal(rows.size)
    return _from_coo(m, n, rows, cols, vals, name, {"per_col": per_col, "seed": seed})


def grid_multicommodity(side: int = 64, commodities: int = 4, seed: int = 1) -> LP:
    """Multicommodity flow on a side x side 4-neighbour grid.

    Columns: one per (commodity, directed arc), +1 at the tail's conservation
    row and -1 at the head's.  Rows: per commodity one conservation row per
    node except node 0 (which would make the rows rank deficient), then one
    joint capacity row per undirected edge summing the 2*commodities flows on
    it with +1.  With side=64 and 4 commodities this gives m = 24,444 and
    n = 64,512.  The seed only matters for the Theta and rhs draws.
    """
    del seed
    nodes = side * side
    edges = []
    for y in range(side):
        for x in range(side):
            v = y * side + x
            if x + 1 < side:
                edges.append((v, v + 1))
            if y + 1 < side:
                edges.append((v, v + side))
    E = len(edges)
    arcs = []
    for e, (u, v) in enumerate(edges):
        arcs.append((u, v, e))
        arcs.append((v, u, e))
    cons_rows = commodities * (nodes - 1)
    m = cons_rows + E
    n = commodities * len(arcs)

    def cons(q, v):
        return -1 if v == 0 else q * (nodes - 1) + (v - 1)

    rows, cols, vals = [], [], []
    j = 0
    for q in range(commodities):
        for (u, v, e) in arcs:
            for r, val in ((cons(q, u), 1.0), (cons(q, v), -1.0), (cons_rows + e, 1.0)):
                if r >= 0:
                    rows.append(r)
                    cols.append(j)
                    vals.append(val)
            j += 1
    return _from_coo(m, n, rows, cols, vals, f"grid{side}x{side}q{commodities}",
                     {"side": side, "commodities": commodities})


def block_angular(blocks: int = 200, bm: int = 150, bn: int = 400, density: float = 0.02,
                  linking: int = 300, seed: int = 1) -> LP:
    """``blocks`` diagonal blocks of bm x bn with Bernoulli(density) N(0,1)
    entries (every column keeps at least one entry) and ``linking`` fully
    dense N(0,1) rows over all columns."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for b in range(blocks):
        mask = rng.random((bm, bn)) < density
        empty = ~mask.any(axis=0)
        if empty.any():
            idx = np.flatnonzero(empty)
            mask[rng.integers(bm, size=idx.size), idx] = True
        r, c = np.nonzero(mask)
        rows.append(r + b * bm)
        cols.append(c + b * bn)
    m = blocks * bm + linking
    n = blocks * bn
    lr = np.repeat(np.arange(blocks * bm, m, dtype=np.int64), n)
    lc = np.tile(np.arange(n, dtype=np.int64), linking)
    rows = np.concatenate(rows + [lr])
    cols = np.concatenate(cols + [lc])
    vals = rng.standard_normal(rows.size)
    return _from_coo(m, n, rows, cols, vals, "block_angular",
                     {"blocks": blocks, "bm": bm, "bn": bn, "linking": linking, "seed": seed})


def batched_sizes(count: int = 512, m_lo: int = 100, m_hi: int = 5000, ratio: float = 2.5,
                  seed: int = 1) -> list[tuple[int, int]]:
    """(m_i, n_i) of the instances of ``batched_random``: m log-uniform in
    [m_lo, m_hi], n = round(ratio*m)."""
    rng = np.random.default_rng(seed)
    ms = np.rint(10.0 ** rng.uniform(np.log10(m_lo), np.log10(m_hi), size=count)).astype(int)
    return [(int(mi), int(round(ratio * mi))) for mi in ms]


def batched_instance(i: int, mi: int, ni: int, per_col: int = 5, seed: int = 1) -> LP:
    """Instance i of ``batched_random`` (its own seed, seed+1+i)."""
    return random_lp(mi, ni, per_col, seed + 1 + i, name=f"batch{i}")


def batched_random(count: int = 512, m_lo: int = 100, m_hi: int = 5000, ratio: float = 2.5,
                   per_col: int = 5, seed: int = 1) -> list[LP]:
    """``count`` independent random LPs with m log-uniform in [m_lo, m_hi],
    n = round(ratio*m), ``per_col`` rows per column; instance i uses seed+1+i."""
    return [batched_instance(i, mi, ni, per_col, seed)
            for i, (mi, ni) in enumerate(batched_sizes(count, m_lo, m_hi, ratio, seed))]


def staircase(periods: int = 50, pm: int = 2000, pn: int = 5000, density: float = 0.002,
              links: int = 500, seed: int = 1) -> LP:
    """Multi-period LP: diagonal blocks pm x pn with Bernoulli(density) N(0,1)
    entries (at least one per row and per column) and, for every period t
    except the last, +1 entries at (row r of period t+1, column r of period t)
    for r < links."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for t in range(periods):
        mask = rng.random((pm, pn)) < density
        er = ~mask.any(axis=1)
        if er.any():
            idx = np.flatnonzero(er)
            mask[idx, rng.integers(pn, size=idx.size)] = True
        ec = ~mask.any(axis=0)
        if ec.any():
            idx = np.flatnonzero(ec)
            mask[rng.integers(pm, size=idx.size), idx] = True
        r, c = np.nonzero(mask)
        rows.append(r + t * pm)
        cols.append(c + t * pn)
        vals.append(rng.standard_normal(r.size))
        if t + 1 < periods:
            lr = np.arange(links) + (t + 1) * pm
            lc = np.arange(links) + t * pn
            rows.append(lr)
            cols.append(lc)
            vals.append(np.ones(links))
    m = periods * pm
    n = periods * pn
    return _from_coo(m, n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                     "staircase", {"periods": periods, "seed": seed})


def feasible_rhs(lp: LP, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """(b, c) making min c^T x, A x = b, x >= 0 feasible and bounded: b = A x0
    and c = A^T y0 + z0 with x0, z0 ~ U[0.5, 2] and y0 ~ N(0, 1), so x0 is
    primal feasible and (y0, z0) dual feasible."""
    rng = np.random.default_rng(seed + 611953)
    x0 = rng.uniform(0.5, 2.0, size=lp.n)
    y0 = rng.standard_normal(lp.m)
    z0 = rng.uniform(0.5, 2.0, size=lp.n)
    cols = np.repeat(np.arange(lp.n), np.diff(lp.colptr))
    b = np.zeros(lp.m)
    np.add.at(b, lp.rowidx, lp.vals * x0[cols])
    c = z0.copy()
    np.add.at(c, cols, lp.vals * y0[lp.rowidx])
    return b, c


def theta_loguniform(n: int, seed: int, lo: float = -8.0, hi: float = 8.0) -> np.ndarray:
    """Theta_j = 10**U[lo, hi]."""
    rng = np.random.default_rng(seed + 7919)
    return 10.0 ** rng.uniform(lo, hi, size=n)


def theta_schedule(n: int, iters: int, seed: int) -> list[np.ndarray]:
    """Theta_j at iteration it = exp(s_it * g_j), g_j ~ U[-ln 1e8, ln 1e8],
    s_it = it/(iters-1): all ones at the first iteration, a 1e-8..1e8 spread
    at the last."""
    rng = np.random.default_rng(seed + 104729)
    g = rng.uniform(-np.log(1e8), np.log(1e8), size=n)
    den = max(iters - 1, 1)
    return [np.exp((it / den) * g) for it in range(iters)]


def rhs_normal(size: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed + 15485863)
    return rng.standard_normal(size)


def random_perm(size: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed + 32452843)
    return rng.permutation(size).astype(np.int32)


def by_name(name: str, seed: int = 1) -> LP:
    """The named workloads at their full sizes."""
    if name == "random_300x800":
        return random_lp(300, 800, 6, seed, name)
    if name == "grid64_q4":
        return grid_multicommodity(64, 4, seed)
    if name == "block_angular":
        return block_angular(seed=seed)
    if name == "staircase":
        return staircase(seed=seed)
    raise KeyError(name)
