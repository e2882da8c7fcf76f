"""The remaining workload families as parity cases: the staircase LP along a
Theta schedule (FP64 and mixed precision at a matched backward error), the
full-size staircase checked through properties the oracle evaluates at any
size, and the block-angular LP with dense linking rows through the
augmented-system / normal-equations choice (Sec. 4.2) and both forced forms."""
import numpy as np
import pytest

import synth
from oracle import FORM_NE, Oracle
from test_parity_gpu import EPS_PIV, RHO, DELTA, check_pair, run_pair

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


def small_staircase():
    # 3 periods of 200 x 500 plus links: N = 2,100, so the factor is checked by
    # its own componentwise backward error (the rigorous check)
    return synth.staircase(periods=3, pm=200, pn=500, density=0.01, links=50, seed=3)


def test_staircase_schedule_fp64_against_oracle(pkg):
    lp = small_staircase()
    sched = synth.theta_schedule(lp.n, 40, 3)
    for it in (0, 20, 35):
        r = run_pair(pkg, lp, sched[it], synth.rhs_normal(lp.n, it), synth.rhs_normal(lp.m, it + 1),
                     ordering=pkg.IPM_ORD_ND)
        check_pair(r, lp)
        r["s"].close()


def test_staircase_schedule_end_stalls_like_oracle(pkg):
    """At the end of the schedule (Theta spread 1e16) classical refinement of
    the regularised factorisation (Sec. 4.5) stalls above the target for the
    oracle too (in the AMD order ten classical steps contract the backward
    error by ~10x each and end near 8e-12); with GMRES refinement off, the
    library must stall at the same level, flag REFINE_NOT_CONVERGED, keep the
    inertia and lift the same pivots."""
    lp = small_staircase()
    th = synth.theta_schedule(lp.n, 40, 3)[39]
    r7, r1 = synth.rhs_normal(lp.n, 39), synth.rhs_normal(lp.m, 40)
    r = run_pair(pkg, lp, th, r7, r1, ordering=pkg.IPM_ORD_AMD, gmres_restarts=0)
    w_orc = r["o"].omega_K(th, RHO, DELTA, r7, r1, r["ref"][: lp.n], r["ref"][lp.n:])
    assert w_orc > 1e-12  # the oracle stalls
    assert r["w_gpu"] <= 10.0 * w_orc, f"omega {r['w_gpu']:.3e} vs oracle {w_orc:.3e}"
    assert r["info"]["nneg"] == lp.n and r["info"]["npos"] == lp.m
    mismatch = np.flatnonzero((r["dyn"] != 0) != (r["ofac"]["dynreg"] != 0))
    assert mismatch.size <= max(2, 0.002 * (lp.n + lp.m))
    assert r["s"].status() == pkg.IPM_WARN_REFINE_NOT_CONVERGED
    r["s"].close()


def test_staircase_schedule_end_gmres_reaches_target(pkg):
    """Same system with the GMRES refinement (restarted GMRES(8) on K c = r,
    preconditioned by the same regularised factor): the backward error on K
    reaches 1e-12, and the solution agrees with the oracle's (stalled) one to
    the accuracy the oracle's backward error allows."""
    lp = small_staircase()
    th = synth.theta_schedule(lp.n, 40, 3)[39]
    r7, r1 = synth.rhs_normal(lp.n, 39), synth.rhs_normal(lp.m, 40)
    s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_AMD)
    s.factorise(th, RHO, DELTA)
    dx, dy = s.solve(r7, r1)
    info = s.info()
    assert info["gmres_iters"] > 0
    o = Oracle.from_lp(lp)
    w = o.omega_K(th, RHO, DELTA, r7, r1, dx.cpu().numpy(), dy.cpu().numpy())
    assert w <= 1e-12, f"omega {w:.3e}"
    assert info["omega"] == pytest.approx(w, rel=1e-6, abs=1e-300)
    assert s.status() >= 0 and s.status() != pkg.IPM_WARN_REFINE_NOT_CONVERGED
    print(f"staircase end with GMRES: omega {w:.2e}, {info['gmres_iters']} GMRES iterations, "
          f"{info['refine_steps']} steps in all")
    s.close()


def test_staircase_schedule_mixed_matches_fp64(pkg):
    """Mixed precision (3xTF32 tensor-core Schur updates of fronts >= 64 rows)
    and FP64, both refined to omega <= 1e-10 on K, along the schedule.  Nested
    dissection eliminates some dual rows early with pivots of size delta, so
    the factor grows by ~1/delta and FP32-accurate updates lose the values:
    the mixed path must detect it (non-finite pivots or stalled refinement),
    fall back to FP64 and still meet the target with the same inertia."""
    lp = small_staircase()
    sched = synth.theta_schedule(lp.n, 40, 3)
    sm = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_ND, precision=pkg.IPM_PREC_MIXED, mixed_min_front=64,
                            omega_target=1e-10, level_kernel=0)
    sf = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_ND, omega_target=1e-10)
    o = Oracle.from_lp(lp)
    for it in (0, 10, 20, 30, 35):
        r7, r1 = synth.rhs_normal(lp.n, 100 + it), synth.rhs_normal(lp.m, 200 + it)
        xs = []
        for s in (sm, sf):
            s.factorise(sched[it], RHO, DELTA)
            dx, dy = s.solve(r7, r1)
            info = s.info()
            assert s.status() >= 0
            assert info["nneg"] == lp.n and info["npos"] == lp.m
            x = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
            assert np.all(np.isfinite(x))
            w = o.omega_K(sched[it], RHO, DELTA, r7, r1, x[: lp.n], x[lp.n:])
            assert w <= 1e-10, f"iteration {it}: omega {w:.3e}"
            xs.append(x)
        err = np.abs(xs[0] - xs[1]).max() / np.abs(xs[1]).max()
        assert err <= 1e-6, f"iteration {it}: mixed vs FP64 rel diff {err:.3e}"
    assert sm.info()["precision_fallbacks"] == 1
    sm.close()
    sf.close()


def test_staircase_full_size_properties(pkg):
    """m = 100,000, n = 250,000 late in the schedule (iteration 30 of 40,
    a ~1e12 spread): the refined solution meets omega <= 1e-10 on K (evaluated
    by the oracle's residual) with exactly n negative and m positive pivots."""
    lp = synth.by_name("staircase", 1)
    th = synth.theta_schedule(lp.n, 40, 1)[30]
    r7, r1 = synth.rhs_normal(lp.n, 10), synth.rhs_normal(lp.m, 11)
    s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_ND, omega_target=1e-10)
    s.factorise(th, RHO, DELTA)
    dx, dy = s.solve(r7, r1)
    info = s.info()
    assert info["nneg"] == lp.n and info["npos"] == lp.m
    o = Oracle.from_lp(lp)
    w = o.omega_K(th, RHO, DELTA, r7, r1, dx.cpu().numpy(), dy.cpu().numpy())
    assert w <= 1e-10, f"omega {w:.3e}"
    assert info["omega"] == pytest.approx(w, rel=1e-6, abs=1e-300)
    print(f"staircase full: omega {w:.2e} steps {info['refine_steps']} lifts {info['ndynreg']} "
          f"max front {info['max_front']}")
    s.close()


def small_block_angular():
    return synth.block_angular(blocks=12, bm=30, bn=80, density=0.05, linking=8, seed=4)


def test_block_angular_forms_against_oracle(pkg):
    """The block-angular family.  At its full Theta range 10^U[-8,8] the
    augmented system matches the oracle factor by factor and reaches
    omega <= 1e-12 on K (GMRES refinement takes over where classical
    refinement stalls; the oracle, which refines classically, stalls near
    0.1).  The solution is not compared there: cond(K) eps is far above 1
    (checked), so no solution agreement follows from any backward error.  The
    normal equations are compared with the oracle's normal equations at a
    Theta range of 10^U[-4,4], where A Theta~ A^T still carries the small
    Theta~ contributions (at the full range both sides lose them: omega on K
    stays near 5e-8 with GMRES, near 1 without).  AUTO picks the normal
    equations for this reduced instance (the cost model; the full-size
    instance keeps the augmented system) and solves at the narrower range."""
    lp = small_block_angular()
    theta = synth.theta_loguniform(lp.n, 4)
    r7, r1 = synth.rhs_normal(lp.n, 4), synth.rhs_normal(lp.m, 5)
    # augmented system, against the oracle factor by factor
    r = run_pair(pkg, lp, theta, r7, r1)
    check_pair(r, lp, x_tol=None)
    K = r["o"].matrix()
    import scipy.sparse as sp

    Kd = sp.csc_matrix((K[2], K[1], K[0]), shape=(lp.n + lp.m,) * 2).toarray()
    Kd = np.tril(Kd) + np.tril(Kd, -1).T
    Kd[np.arange(lp.n), np.arange(lp.n)] -= RHO
    Kd[lp.n + np.arange(lp.m), lp.n + np.arange(lp.m)] += DELTA
    assert np.linalg.cond(Kd) * 2.2e-16 > 1.0
    print(f"block-angular AS, Theta 1e-8..1e8: omega {r['w_gpu']:.2e}, GMRES {r['info']['gmres_iters']}, "
          f"oracle omega {r['oinfo']['omega_hist'][-1]:.2e}")
    r["s"].close()
    theta_ne = synth.theta_loguniform(lp.n, 4, -4.0, 4.0)
    # normal equations, against the oracle's normal equations
    s = pkg.Solver.from_lp(lp, form=pkg.IPM_FORM_NORMAL)
    s.factorise(theta_ne, RHO, DELTA)
    dx, dy = s.solve(r7, r1)
    info = s.info()
    assert info["form"] == pkg.IPM_FORM_NORMAL and info["npos"] == lp.m
    x = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    o = Oracle.from_lp(lp, form=FORM_NE)
    sym = s.symbolic()
    o.analyse(sym["perm"], amalg_zero_frac=sym["amalg_zero_frac"])
    o.factorise(theta_ne, RHO, DELTA, eps_piv=EPS_PIV)
    ox, oy, _ = o.solve(r7, r1, omega_target=1e-12, max_steps=10)
    ref = np.concatenate([ox, oy])
    w = o.omega_K(theta_ne, RHO, DELTA, r7, r1, x[: lp.n], x[lp.n:])
    assert w <= 1e-10, f"omega {w:.3e}"
    assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max()
    s.close()
    # the chooser: both costs reported, the chosen form solves to the target
    s = pkg.Solver.from_lp(lp, form=pkg.IPM_FORM_AUTO)
    info = s.info()
    assert info["est_cost_as"] > 0
    s.factorise(theta_ne, RHO, DELTA)
    dx, dy = s.solve(r7, r1)
    w = Oracle.from_lp(lp).omega_K(theta_ne, RHO, DELTA, r7, r1, dx.cpu().numpy(), dy.cpu().numpy())
    assert w <= 1e-10
    print(f"block-angular chooser: form {s.info()['form']} cost AS {info['est_cost_as']:.3e} "
          f"NE {info['est_cost_ne']:.3e}")
    s.close()


def test_staircase_schedule_end_gmres_inside_graph(pkg):
    """The same stalled system through a captured CUDA graph: classical
    refinement ends above 1e-12, so the conditional GMRES section of the graph
    runs (its condition is set on the device) and the backward error on K
    reaches 1e-12; the solution agrees with the direct path's GMRES result,
    and a replay on a system that needs no GMRES skips the section."""
    import torch

    lp = small_staircase()
    sched = synth.theta_schedule(lp.n, 40, 3)
    th = sched[39]
    r7, r1 = synth.rhs_normal(lp.n, 39), synth.rhs_normal(lp.m, 40)
    s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_AMD)
    s.factorise(th, RHO, DELTA)
    ex, ey = s.solve(r7, r1)
    direct = np.concatenate([ex.cpu().numpy(), ey.cpu().numpy()])
    assert s.info()["gmres_iters"] > 0
    dev = s.dev
    theta = torch.as_tensor(th, device=dev)
    r7d, r1d = torch.as_tensor(r7, device=dev), torch.as_tensor(r1, device=dev)
    dx = torch.zeros(lp.n, dtype=torch.float64, device=dev)
    dy = torch.zeros(lp.m, dtype=torch.float64, device=dev)
    assert pkg.ipm_graph_capture(s.ctx, theta, RHO, DELTA, r7d, r1d, dx, dy, nsolves=1) == 0
    assert pkg.ipm_graph_launch(s.ctx) == 0
    torch.cuda.synchronize()
    info = s.info()
    x = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    w = Oracle.from_lp(lp).omega_K(th, RHO, DELTA, r7, r1, x[: lp.n], x[lp.n:])
    assert info["gmres_iters"] > 0 and w <= 1e-12, (info["gmres_iters"], w)
    assert info["omega"] == pytest.approx(w, rel=1e-6, abs=1e-300)
    assert np.abs(x - direct).max() <= 1e-8 * np.abs(direct).max()
    # an early schedule point: classical refinement suffices, the section is skipped
    theta.copy_(torch.as_tensor(sched[5], device=dev))
    assert pkg.ipm_graph_launch(s.ctx) == 0
    torch.cuda.synchronize()
    info = s.info()
    x = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    w = Oracle.from_lp(lp).omega_K(sched[5], RHO, DELTA, r7, r1, x[: lp.n], x[lp.n:])
    assert info["gmres_iters"] == 0 and w <= 1e-12
    print(f"graph GMRES: {info['refine_steps']} steps at iteration 5; stalled case reached {w:.2e}")
    s.close()
