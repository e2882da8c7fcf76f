"""Rows of K longer than 4096 stored entries (a dense row of A): ||K||_1 (the
lift floor eps_piv ||K||_1 of Sec. 4.5) and the residual of refinement sum
such a row with a whole CTA in a fixed order instead of one thread.  The norm
must equal the oracle's to rounding, the factor and refined solution must meet
the parity bar against the oracle."""
import numpy as np
import pytest

import synth
from synth.lp import LP
from test_parity_gpu import check_pair, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04370_gb300.build import build

    build()
    import paper_2508_04370_gb300 as p

    return p


def _with_dense_row(lp, seed):
    # one extra row over every column, N(0,1): its dual column of K holds n + 1 entries
    rng = np.random.default_rng(seed)
    cols = np.repeat(np.arange(lp.n), np.diff(lp.colptr))
    rows = np.concatenate([lp.rowidx.astype(np.int64), np.full(lp.n, lp.m)])
    cols = np.concatenate([cols, np.arange(lp.n)])
    vals = np.concatenate([lp.vals, rng.standard_normal(lp.n)])
    order = np.lexsort((rows, cols))
    colptr = np.zeros(lp.n + 1, dtype=np.int64)
    np.add.at(colptr, cols[order] + 1, 1)
    return LP(lp.m + 1, lp.n, np.cumsum(colptr), rows[order].astype(np.int32), vals[order], "dense_row", {})


def test_dense_row_norm_and_parity(pkg):
    lp = _with_dense_row(synth.random_lp(400, 5000, 3, 7), 8)
    assert np.count_nonzero(lp.rowidx == lp.m - 1) == lp.n > 4096
    theta = synth.theta_loguniform(lp.n, 9)
    r = run_pair(pkg, lp, theta, synth.rhs_normal(lp.n, 10), synth.rhs_normal(lp.m, 11), ordering=pkg.IPM_ORD_AMD)
    # the GPU's ||K||_1 (a CTA-summed dense column) against the oracle's
    assert r["info"]["norm_K1"] == pytest.approx(r["ostats"]["normM1"], rel=1e-13)
    err = check_pair(r, lp)
    assert r["w_gpu"] <= 1e-12
    print(f"dense row: ||K||_1 {r['info']['norm_K1']:.6e} omega {r['w_gpu']:.2e} rel err {err:.2e}")
