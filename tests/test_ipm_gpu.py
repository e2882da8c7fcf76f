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
