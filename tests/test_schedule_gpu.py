"""Order of the large fronts' 32-column steps (Sec. 4.3, tree-level
parallelism).  In the level order every large front of a tree level steps
through its panels together and the next level waits for the whole level; in
the dependency order a front starts as soon as its children are done, so the
steps follow the longest chain of panels instead of the sum over levels of
each level's widest front.  Both orders apply the same updates to every entry
in the same order, so the factors must agree bit for bit, on the FP64 and the
sliced tensor-core paths, directly and replayed from a captured graph; the
small-front levels that wait for large children (present in both workloads
below) are issued between the steps."""
import numpy as np
import pytest

import synth
from test_parity_gpu import DELTA, RHO

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


def _factor(pkg, lp, th, schedule, **opts):
    # level_kernel=0: the level order runs every large front step by step
    # with the kernels the dependency order uses
    s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_ND, schedule=schedule, level_kernel=0, **opts)
    s.factorise(th, RHO, DELTA)
    fac = s.factor()
    info = s.info()
    return s, fac, info


@pytest.mark.parametrize("prec", ["fp64", "sliced"])
@pytest.mark.parametrize("work", ["staircase4", "grid24"])
def test_dependency_order_equals_level_order(pkg, prec, work):
    lp = synth.staircase(periods=4, seed=1) if work == "staircase4" else synth.grid_multicommodity(24, 4)
    th = synth.theta_loguniform(lp.n, 21)
    opts = {} if prec == "fp64" else dict(precision=pkg.IPM_PREC_SLICED, mixed_min_front=64)
    s1, f1, i1 = _factor(pkg, lp, th, pkg.IPM_SCHED_LEVELS, **opts)
    s2, f2, i2 = _factor(pkg, lp, th, pkg.IPM_SCHED_DEPENDENCY, **opts)
    assert i1["schedule"] == pkg.IPM_SCHED_LEVELS and i2["schedule"] == pkg.IPM_SCHED_DEPENDENCY
    assert i1["steps_levels"] == i2["steps_levels"] and i1["steps_dependency"] == i2["steps_dependency"]
    # no error bits (lifted pivots, status 2, are allowed and must agree)
    assert i1["status"] & ~2 == 0 and i2["status"] == i1["status"] and i1["ndynreg"] == i2["ndynreg"]
    for a, b in zip(f1, f2):
        assert np.array_equal(a, b)
    if prec == "sliced":
        assert i2["mixed_active"] == 1 and i2["flops_tensor"] > 0
    # the same refined solution
    r7, r1 = synth.rhs_normal(lp.n, 22), synth.rhs_normal(lp.m, 23)
    x1 = [t.cpu().numpy() for t in s1.solve(r7, r1)]
    x2 = [t.cpu().numpy() for t in s2.solve(r7, r1)]
    for a, b in zip(x1, x2):
        np.testing.assert_array_equal(a, b)
    assert s2.info()["omega"] <= 1e-12
    print(f"{work} {prec}: steps level order {i2['steps_levels']} dependency order {i2['steps_dependency']}")
    s1.close()
    s2.close()


def test_auto_order_and_graph_replay(pkg):
    """On the 4-period staircase the automatic choice takes the dependency
    order (201 against 270 steps); one IPM iteration replayed from a captured
    graph in that order equals the direct calls in the level order."""
    import torch

    lp = synth.staircase(periods=4, seed=1)
    n, m = lp.n, lp.m
    th = synth.theta_loguniform(n, 31)
    s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_ND, precision=pkg.IPM_PREC_SLICED, mixed_min_front=64)
    dev = s.dev
    r7 = np.concatenate([synth.rhs_normal(n, 32), synth.rhs_normal(n, 33)])
    r1 = np.concatenate([synth.rhs_normal(m, 34), synth.rhs_normal(m, 35)])
    theta = torch.as_tensor(th, device=dev)
    r7d, r1d = torch.as_tensor(r7, device=dev), torch.as_tensor(r1, device=dev)
    dx = torch.zeros(2 * n, dtype=torch.float64, device=dev)
    dy = torch.zeros(2 * m, dtype=torch.float64, device=dev)
    assert pkg.ipm_graph_capture(s.ctx, theta, RHO, DELTA, r7d, r1d, dx, dy, nsolves=2) == 0
    assert pkg.ipm_graph_launch(s.ctx) == 0
    torch.cuda.synchronize()
    info = s.info()
    assert info["schedule"] == pkg.IPM_SCHED_DEPENDENCY
    assert 5 * info["steps_dependency"] <= 4 * info["steps_levels"]
    assert info["omega"] <= 1e-12 and info["mixed_active"] == 1
    gx, gy = dx.cpu().numpy().copy(), dy.cpu().numpy().copy()
    ref, _, _ = _factor(pkg, lp, th, pkg.IPM_SCHED_LEVELS, precision=pkg.IPM_PREC_SLICED, mixed_min_front=64)
    for k in range(2):
        ex, ey = ref.solve(r7[k * n:(k + 1) * n], r1[k * m:(k + 1) * m])
        np.testing.assert_array_equal(gx[k * n:(k + 1) * n], ex.cpu().numpy())
        np.testing.assert_array_equal(gy[k * m:(k + 1) * m], ey.cpu().numpy())
    s.close()
    ref.close()


def test_kernel_trace_matches_kernel_stats(pkg):
    """ipm_kernel_trace lists every profiled launch of a factorisation in issue
    order; its per-class durations sum to what ipm_kernel_stats reports, and
    the critical stream's steps appear in order (no launch on a stream starts
    before the previous one on that stream ended)."""
    lp = synth.staircase(periods=4, seed=1)
    th = synth.theta_loguniform(lp.n, 41)
    s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_ND, precision=pkg.IPM_PREC_SLICED, mixed_min_front=64)
    s.factorise(th, RHO, DELTA)
    pkg.ipm_set_profiling(s.ctx, True)
    pkg.ipm_kernel_stats(s.ctx, reset=True)
    pkg.ipm_kernel_trace(s.ctx)
    s.factorise(th, RHO, DELTA)
    pkg.ipm_set_profiling(s.ctx, False)
    tr = pkg.ipm_kernel_trace(s.ctx)
    ks = pkg.ipm_kernel_stats(s.ctx, reset=True)
    n = tr["count"]
    assert n == len(tr["cls"]) and n == sum(v["launches"] for v in ks.values()) and n > 0
    assert tr["start_ms"][0] == 0.0 and np.all(tr["end_ms"] >= tr["start_ms"])
    assert np.all((tr["cls"] >= 0) & (tr["cls"] < len(pkg.KERNEL_CLASSES)))
    for c, name in enumerate(pkg.KERNEL_CLASSES):
        m = tr["cls"] == c
        assert m.sum() == ks[name]["launches"]
        assert abs(float((tr["end_ms"][m] - tr["start_ms"][m]).sum()) - ks[name]["ms"]) <= 1e-3 * max(1.0, ks[name]["ms"])
    for st in np.unique(tr["stream"]):
        m = tr["stream"] == st
        a, b = tr["start_ms"][m], tr["end_ms"][m]
        assert np.all(a[1:] >= b[:-1] - 1e-3)
    # a second call returns nothing new
    assert pkg.ipm_kernel_trace(s.ctx)["count"] == 0
    s.close()


def test_thin_fronts_block_angular(pkg):
    """A block-angular LP whose fronts are one column plus the dense linking
    rows (k = 1, f ~ 150): the levels outside the level kernel run these
    thin fronts whole, one CTA each, with the per-step bodies in sequence.
    The factor must equal the per-step path's (the dependency order) bit for
    bit and the oracle's to the parity bar."""
    from test_parity_gpu import check_pair, run_pair

    lp = synth.block_angular(blocks=20, bm=60, bn=160, density=0.05, linking=150, seed=5)
    th = synth.theta_loguniform(lp.n, 51)
    s1, f1, i1 = _factor(pkg, lp, th, pkg.IPM_SCHED_LEVELS)
    s2, f2, i2 = _factor(pkg, lp, th, pkg.IPM_SCHED_DEPENDENCY)
    assert i1["nfronts_thin"] > 100, i1["nfronts_thin"]
    assert i1["status"] & ~2 == 0 and i2["status"] == i1["status"]
    for a, b in zip(f1, f2):
        assert np.array_equal(a, b)
    s1.close()
    s2.close()
    r = run_pair(pkg, lp, th, synth.rhs_normal(lp.n, 52), synth.rhs_normal(lp.m, 53), ordering=pkg.IPM_ORD_ND,
                 level_kernel=0, schedule=pkg.IPM_SCHED_LEVELS)
    err = check_pair(r, lp)
    print(f"block-angular thin fronts {i1['nfronts_thin']}: omega {r['w_gpu']:.2e} rel err {err:.2e}")
