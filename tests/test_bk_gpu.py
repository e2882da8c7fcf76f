"""The pivoting mode (Sec. 4.5, the Bunch-Kaufman variation: 1x1 and 2x2
pivots chosen inside each pivot block of a front, pre-swap, lifting) against
the oracle's multifrontal factorisation with the same rule, on the same
order.  The CUDA front kernel evaluates every product and sum of the rule as
written, in the oracle's order, so the pivot sequence (interchanges and block
sizes) must be identical and D, the 2x2 off-diagonals, the lifts and L must
agree to the last bit; the refined solutions must reach omega <= 1e-12 on K
and agree with the oracle's to 1e-8."""
import numpy as np
import pytest

import synth
from oracle import FORM_AS, Oracle
from test_oracle_pins import _bk_case, lp_from_dense

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


def run_bk(pkg, lp, theta, rho, delta, r7, r1, **opts):
    s = pkg.Solver.from_lp(lp, pivoting=1, **opts)
    s.factorise(theta, rho, delta)
    L, D, dyn = s.factor()
    pv = pkg.ipm_get_pivots(s.ctx)
    dx, dy = s.solve(r7, r1)
    info = s.info()
    sym = s.symbolic()
    x = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    o = Oracle.from_lp(lp)
    osym = o.analyse(sym["perm"], amalg_width=opts.get("amalg_width", 16),
                     amalg_zero_frac=sym["amalg_zero_frac"])
    assert np.array_equal(osym["sn_rows"], sym["sn_rows"])
    o.set_pivoting(True)
    o.factorise(theta, rho, delta)
    of, opv = o.factor(), o.pivots()
    ox, oy, _ = o.solve(r7, r1, omega_target=1e-14, max_steps=10)
    ref = np.concatenate([ox, oy])
    w = o.omega_K(theta, rho, delta, r7, r1, x[: lp.n], x[lp.n:])
    s.close()
    return dict(L=L, D=D, dyn=dyn, pv=pv, info=info, x=x, of=of, opv=opv, ref=ref, w=w, ostats=o.stats())


def check_bk(r, lp, bitwise=True):
    assert np.array_equal(r["pv"]["bsize"], r["opv"]["bsize"]), "block sizes differ"
    assert np.array_equal(r["pv"]["lperm"], r["opv"]["lperm"]), "interchanges differ"
    if bitwise:
        for a, b in ((r["D"], r["of"]["D"]), (r["pv"]["Doff"], r["opv"]["Doff"]), (r["dyn"], r["of"]["dynreg"]),
                     (r["L"], r["of"]["L"])):
            assert np.array_equal(a, b)
    assert r["info"]["nneg"] == r["ostats"]["nneg"] and r["info"]["npos"] == r["ostats"]["npos"]
    assert r["w"] <= 1e-12, f"omega {r['w']:.2e}"
    assert np.abs(r["x"] - r["ref"]).max() <= 1e-8 * np.abs(r["ref"]).max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bk_without_regularisation_matches_oracle(pkg, seed):
    """rho = delta = 0 (not quasi-definite): every dual row pairs with its
    matched column in a 2-column front and needs a 2x2 pivot; exactly n
    negative and m positive eigenvalues."""
    rng, A, perm = _bk_case(seed)
    m, n = A.shape
    theta = 10.0 ** rng.uniform(2, 4, n)
    mm, nn, cp, ri, vals = lp_from_dense(A)
    lp = synth.lp.LP(mm, nn, cp, ri, vals)
    r7, r1 = rng.standard_normal(n), rng.standard_normal(m)
    r = run_bk(pkg, lp, theta, 0.0, 0.0, r7, r1, ordering=pkg.IPM_ORD_USER, user_perm=perm, amalg_width=2,
               amalg_zero_frac=0.0)
    assert np.count_nonzero(r["pv"]["bsize"] == 2) == m
    assert r["info"]["nneg"] == n and r["info"]["npos"] == m
    check_bk(r, lp)


def test_bk_quasi_definite_random_lp(pkg):
    """With rho = delta = 1e-8 the pivoting mode still factorises K exactly
    like the oracle's pivoting, on an AMD order with wider fronts."""
    lp = synth.random_lp(150, 400, 4, seed=31)
    theta = synth.theta_loguniform(lp.n, 31, -4.0, 4.0)
    r = run_bk(pkg, lp, theta, 1e-8, 1e-8, synth.rhs_normal(lp.n, 31), synth.rhs_normal(lp.m, 32))
    assert r["info"]["nneg"] == lp.n and r["info"]["npos"] == lp.m
    check_bk(r, lp)


def test_bk_grid_nested_dissection(pkg):
    """A grid LP in nested-dissection order (fronts of a few hundred rows,
    several pivot blocks each)."""
    lp = synth.grid_multicommodity(12, 3)
    theta = synth.theta_loguniform(lp.n, 33, -3.0, 3.0)
    r = run_bk(pkg, lp, theta, 1e-8, 1e-8, synth.rhs_normal(lp.n, 33), synth.rhs_normal(lp.m, 34),
               ordering=pkg.IPM_ORD_ND)
    assert r["info"]["max_front"] > 32
    check_bk(r, lp)


def test_bk_mode_rejects_graphs_and_noalloc(pkg):
    lp = synth.random_lp(20, 50, 3, seed=2)
    s = pkg.Solver.from_lp(lp, pivoting=1)
    s.factorise(synth.theta_loguniform(lp.n, 2), 1e-8, 1e-8)
    z = s._dev(np.zeros(lp.n))
    assert pkg.ipm_graph_capture(s.ctx, z, 1e-8, 1e-8, z, s._dev(np.zeros(lp.m)), z, s._dev(np.zeros(lp.m)),
                                 nsolves=1) == pkg.IPM_ERR_INVALID_ARG
    s.close()
