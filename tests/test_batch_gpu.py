"""Batches of independent LPs factorised as one block-diagonal forest
(level-scheduled together, Sec. 4.3) against the oracle run on every
instance separately, and against the library run on every instance alone.

Each instance keeps its own pivot floor eps_piv ||K_b||_1 (Sec. 4.5), so its
pivots, lifts and D are bit-identical to a factorisation of that instance on
its own with the same order; the refined solution of the batch meets the
backward-error target on every instance."""
import numpy as np
import pytest

import synth
from oracle import Oracle

pytestmark = pytest.mark.gpu

RHO = DELTA = 1e-8
EPS_PIV = 2.220446049250313e-16


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04370_gb300.build import build

    build()
    import paper_2508_04370_gb300 as p

    return p


def restricted_perm(perm, b, n_off, m_off, Nn):
    """Order of instance b's unknowns (its own numbering: columns, then rows)
    induced by the batch order perm (perm[new] = old)."""
    lo_c, hi_c = n_off[b], n_off[b + 1]
    lo_r, hi_r = Nn + m_off[b], Nn + m_off[b + 1]
    nb = hi_c - lo_c
    out = []
    for o in perm:
        if lo_c <= o < hi_c:
            out.append(o - lo_c)
        elif lo_r <= o < hi_r:
            out.append(nb + o - lo_r)
    return np.array(out, dtype=np.int32)


def make_batch(count, m_lo, m_hi, seed):
    lps = synth.batched_random(count=count, m_lo=m_lo, m_hi=m_hi, seed=seed)
    thetas = [synth.theta_loguniform(lp.n, seed + 7 * i) for i, lp in enumerate(lps)]
    r7s = [synth.rhs_normal(lp.n, seed + 11 * i) for i, lp in enumerate(lps)]
    r1s = [synth.rhs_normal(lp.m, seed + 13 * i + 1) for i, lp in enumerate(lps)]
    return lps, thetas, r7s, r1s


def test_batch_against_oracle_per_instance(pkg):
    lps, thetas, r7s, r1s = make_batch(12, 20, 300, seed=5)
    bs = pkg.BatchSolver(lps)
    bs.factorise(bs.concat(thetas), RHO, DELTA)
    dx, dy = bs.solve(bs.concat(r7s), bs.concat(r1s))
    info = bs.info()
    assert info["nneg"] == bs.N - int(bs.m_off[-1]) and info["npos"] == int(bs.m_off[-1])
    sym = bs.symbolic()
    _, D, dyn = bs.factor()
    perm = sym["perm"]
    Nn = int(bs.n_off[-1])
    parts = bs.split(dx, dy)
    for b, lp in enumerate(lps):
        rp = restricted_perm(perm, b, bs.n_off, bs.m_off, Nn)
        o = Oracle.from_lp(lp)
        o.analyse(rp, amalg_zero_frac=sym["amalg_zero_frac"])
        o.factorise(thetas[b], RHO, DELTA, eps_piv=EPS_PIV)
        ofac = o.factor()
        ox, oy, _ = o.solve(r7s[b], r1s[b], omega_target=1e-12, max_steps=10)
        gx, gy = parts[b]
        w = o.omega_K(thetas[b], RHO, DELTA, r7s[b], r1s[b], gx, gy)
        assert w <= 1e-12, f"instance {b}: omega {w:.3e}"
        ref = np.concatenate([ox, oy])
        err = np.abs(np.concatenate([gx, gy]) - ref).max() / np.abs(ref).max()
        assert err <= 1e-8, f"instance {b}: solution rel err {err:.3e}"
        # this instance's pivots, in the batch order = the oracle's order
        mine = np.array([(n_lo <= o_ < n_hi) or (Nn + m_lo <= o_ < Nn + m_hi)
                         for o_, n_lo, n_hi, m_lo, m_hi in
                         [(o_, bs.n_off[b], bs.n_off[b + 1], bs.m_off[b], bs.m_off[b + 1]) for o_ in perm]])
        Db, dynb = D[mine], dyn[mine]
        assert np.count_nonzero(Db < 0) == lp.n and np.count_nonzero(Db > 0) == lp.m
        mismatch = np.flatnonzero((dynb != 0) != (ofac["dynreg"] != 0))
        assert mismatch.size <= max(2, 0.002 * Db.size), f"instance {b}: lifted sets differ at {mismatch}"
    bs.close()


def test_batch_matches_instances_alone(pkg):
    lps, thetas, r7s, r1s = make_batch(8, 30, 400, seed=9)
    bs = pkg.BatchSolver(lps)
    bs.factorise(bs.concat(thetas), RHO, DELTA)
    sym = bs.symbolic()
    _, D, dyn = bs.factor()
    perm = sym["perm"]
    Nn = int(bs.n_off[-1])
    # value per original unknown of the batch
    Dorig = np.empty_like(D)
    Dorig[perm] = D
    dynorig = np.empty_like(dyn)
    dynorig[perm] = dyn
    nlift = 0
    for b, lp in enumerate(lps):
        rp = restricted_perm(perm, b, bs.n_off, bs.m_off, Nn)
        # the batch's elimination order and amalgamation threshold
        s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_USER, user_perm=rp, amalg_zero_frac=sym["amalg_zero_frac"])
        s.factorise(thetas[b], RHO, DELTA)
        sa = s.symbolic()
        _, Da, dyna = s.factor()
        Dao = np.empty_like(Da)
        Dao[sa["perm"]] = Da
        dao = np.empty_like(dyna)
        dao[sa["perm"]] = dyna
        idx = np.concatenate([np.arange(bs.n_off[b], bs.n_off[b + 1]), Nn + np.arange(bs.m_off[b], bs.m_off[b + 1])])
        assert np.array_equal(Dorig[idx], Dao), f"instance {b}: D differs from the instance alone"
        assert np.array_equal(dynorig[idx], dao), f"instance {b}: lifts differ from the instance alone"
        nlift += int(np.count_nonzero(dao))
        s.close()
    assert nlift > 0  # the per-instance pivot floor was exercised
    bs.close()
