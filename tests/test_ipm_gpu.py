"""The interior point driver (Sec. 2-3, 4.7) on feasible, bounded synthetic
LPs: it must reach relative primal/dual residuals and duality gap below 1e-8,
with the optimal objective of an independent simplex/IPM code (SciPy's HiGHS)
to 1e-6, while the factorisations it requests see Theta spreads growing well
past 1e8 and every solve meets the backward-error target."""
import numpy as np
import pytest

import synth

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


def highs_objective(lp, b, c):
    import scipy.sparse as sp
    from scipy.optimize import linprog

    A = sp.csc_matrix((lp.vals, lp.rowidx, lp.colptr), shape=(lp.m, lp.n))
    res = linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("case", ["random_120x300", "random_200x500", "grid16_q4"])
def test_ipm_reaches_optimum(pkg, case):
    from paper_2508_04370_gb300.ipm import solve_lp

    if case.startswith("grid"):
        lp = synth.grid_multicommodity(16, 4)
        ordering = pkg.IPM_ORD_ND
    else:
        m, n = (int(v) for v in case.split("_")[1].split("x"))
        lp = synth.random_lp(m, n, 4, seed=m)
        ordering = pkg.IPM_ORD_AMD
    b, c = synth.feasible_rhs(lp, 7)
    res = solve_lp(lp.m, lp.n, lp.colptr, lp.rowidx, lp.vals, b, c, ordering=ordering, max_iter=80)
    assert res.status == "optimal", res.history[-1]
    ref = highs_objective(lp, b, c)
    assert abs(res.objective - ref) <= 1e-6 * (1.0 + abs(ref)), (res.objective, ref)
    assert np.all(res.x >= 0) and np.all(res.z >= 0)
    spreads = [h["theta_spread"] for h in res.history if "theta_spread" in h]
    assert max(spreads) > 1e8
    assert max(max(h["omega_pred"], h["omega_corr"]) for h in res.history if "omega_pred" in h) <= 1e-12
    print(f"{case}: {res.iterations} iterations, objective {res.objective:.10g} (HiGHS {ref:.10g}), "
          f"final Theta spread {spreads[-1]:.1e}")


def highs_bounded(lp, b, c, lo, up):
    import scipy.sparse as sp
    from scipy.optimize import linprog

    A = sp.csc_matrix((lp.vals, lp.rowidx, lp.colptr), shape=(lp.m, lp.n))
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(z) else z) for a, z in zip(lo, up)]
    res = linprog(c, A_eq=A, b_eq=b, bounds=bounds, method="highs")
    assert res.status == 0
    return res.fun


def test_ipm_bounded_and_free_variables(pkg):
    """Sec. 2.1's bounded formulation: boxed, lower-bounded, upper-bounded and
    free variables (a free variable's diagonal of K is the static
    regularisation alone).  The LP is feasible (x0 strictly inside the bounds,
    b = A x0) and bounded (every column has a finite bound in the direction
    its cost pushes, or is boxed); the optimum must match HiGHS to 1e-6 with
    the paper's termination test at 1e-8, and multiple centrality correctors
    must be taken (accepted only when they lengthen the step); the rule of
    Sec. 4.7 on its own must also reach the optimum."""
    from paper_2508_04370_gb300.ipm import solve_lp

    lp = synth.random_lp(150, 400, 4, seed=11)
    rng = np.random.default_rng(11)
    kind = rng.integers(0, 4, lp.n)  # 0 boxed, 1 lower only, 2 upper only, 3 free
    x0 = rng.uniform(-1.0, 1.0, lp.n)
    lo = np.where((kind == 0) | (kind == 1), x0 - rng.uniform(0.5, 2.0, lp.n), -np.inf)
    up = np.where((kind == 0) | (kind == 2), x0 + rng.uniform(0.5, 2.0, lp.n), np.inf)
    cols = np.repeat(np.arange(lp.n), np.diff(lp.colptr))
    b = np.zeros(lp.m)
    np.add.at(b, lp.rowidx, lp.vals * x0[cols])
    # dual feasible costs: c = A^T y0 + zl - zu with zl > 0 only where lower
    # bounds exist and zu > 0 only where upper bounds exist (free: c_j = (A^T y0)_j)
    y0 = rng.standard_normal(lp.m)
    aty = np.zeros(lp.n)
    np.add.at(aty, cols, lp.vals * y0[lp.rowidx])
    zl = np.where(np.isfinite(lo), rng.uniform(0.1, 1.0, lp.n), 0.0)
    zu = np.where(np.isfinite(up), rng.uniform(0.1, 1.0, lp.n), 0.0)
    c = aty + zl - zu
    # the rule of Sec. 4.7 allows one corrector on an LP this small (a
    # factorisation costs about a solve); up to four are allowed here so that
    # the multiple centrality correctors are exercised
    res = solve_lp(lp.m, lp.n, lp.colptr, lp.rowidx, lp.vals, b, c, lo, up, max_iter=80, correctors=4)
    assert res.status == "optimal", res.history[-1]
    ref = highs_bounded(lp, b, c, lo, up)
    assert abs(res.objective - ref) <= 1e-6 * (1.0 + abs(ref)), (res.objective, ref)
    fin_lo, fin_up = np.isfinite(lo), np.isfinite(up)
    assert np.all(res.x[fin_lo] >= lo[fin_lo] - 1e-7) and np.all(res.x[fin_up] <= up[fin_up] + 1e-7)
    assert sum(h.get("correctors", 0) > 1 for h in res.history) > 0
    assert max(max(h["omega_pred"], h["omega_corr"]) for h in res.history if "omega_pred" in h) <= 1e-12
    print(f"bounded LP: {res.iterations} iterations, objective {res.objective:.10g} (HiGHS {ref:.10g}), "
          f"correctors per iteration {[h.get('correctors') for h in res.history if 'correctors' in h]}")
    rule = solve_lp(lp.m, lp.n, lp.colptr, lp.rowidx, lp.vals, b, c, lo, up, max_iter=80)
    assert rule.status == "optimal" and abs(rule.objective - ref) <= 1e-6 * (1.0 + abs(ref))
    assert all(1 <= h["corrector_limit"] <= 6 for h in rule.history if "corrector_limit" in h)
