"""The sliced tensor-core path (IPM_PREC_SLICED): Schur-complement updates of
large fronts from 7-bit digit slices of the panel operands on the bf16 tensor
cores, exact FP32 accumulation and integer recombination, about as accurate
as FP64 (Sec. 4.4 updates; pivots, lifts, residuals and refinement in FP64).
Unlike the FP32-accurate mixed path it must never fall back to FP64 on these
inputs and must meet the FP64 path's parity bar against the oracle: identical
lift sets, D and L within 1e-10 of the propagated error scale, omega on K
<= 1e-12 and the oracle's solution to 1e-8.  On small systems the dense
reconstruction is checked in its rowwise form (the products are accurate
relative to each row's largest terms, not to each term)."""
import numpy as np
import pytest

import synth
from oracle import Oracle
from test_parity_gpu import DELTA, EPS_PIV, RHO, check_pair, run_pair

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


def _sliced_pair(pkg, lp, theta, seed, ordering, min_front, target=1e-12, level_kernel=0):
    # level_kernel=0: one launch per step on every level, so that every front
    # of at least min_front rows takes the sliced updates (a latency-bound
    # level would otherwise keep the FP64 level kernel)
    r = run_pair(pkg, lp, theta, synth.rhs_normal(lp.n, seed), synth.rhs_normal(lp.m, seed + 1), ordering=ordering,
                 precision=pkg.IPM_PREC_SLICED, mixed_min_front=min_front, omega_target=target,
                 level_kernel=level_kernel)
    info = r["s"].info()
    assert info["flops_tensor"] > 0
    # the digit slices are written by the panel's triangular solve, so the
    # separate slicing class stays empty
    assert r["kstats"]["large_update_tc"]["launches"] > 0 and r["kstats"]["slice"]["launches"] == 0
    assert info["precision_fallbacks"] == 0 and info["mixed_active"] == 1
    return r, info


@pytest.mark.parametrize("order", ["ND", "AMD"])
def test_sliced_updates_grid_match_oracle(pkg, order):
    """Every front of at least 64 rows updated on the tensor cores, Theta
    10^U[-8,8] (a 1e16 spread, where FP32-accurate updates fall back)."""
    lp = synth.grid_multicommodity(24, 4)
    theta = synth.theta_loguniform(lp.n, 9)
    r, info = _sliced_pair(pkg, lp, theta, 9, pkg.IPM_ORD_ND if order == "ND" else pkg.IPM_ORD_AMD, 64)
    err = check_pair(r, lp, rowwise=True)
    print(f"sliced grid24 {order}: omega {r['w_gpu']:.2e} rel err {err:.2e} steps {info['refine_steps']} "
          f"tensor flops {info['flops_tensor']:.3e} of {info['flops_factor']:.3e}")
    r["s"].close()


def test_sliced_updates_large_fronts_ragged(pkg):
    """Dual rows ordered first: one large front with many 32-column panels, a
    ragged last panel and ragged 128-row slice blocks."""
    for (m, n, seed) in ((90, 211, 5), (130, 333, 6)):
        lp = synth.random_lp(m, n, 3, seed=seed)
        theta = synth.theta_loguniform(lp.n, seed, -2.0, 2.0)
        perm = np.concatenate([lp.n + np.arange(lp.m), np.arange(lp.n)]).astype(np.int32)
        r = run_pair(pkg, lp, theta, synth.rhs_normal(lp.n, seed), synth.rhs_normal(lp.m, seed + 1),
                     ordering=pkg.IPM_ORD_USER, user_perm=perm, precision=pkg.IPM_PREC_SLICED, mixed_min_front=64,
                     level_kernel=0)
        info = r["s"].info()
        assert info["max_front"] > 128 and r["kstats"]["large_update_tc"]["launches"] > 0
        assert info["precision_fallbacks"] == 0
        check_pair(r, lp, rowwise=True)
        r["s"].close()


def test_sliced_staircase_schedule_without_fallback(pkg):
    """The staircase along its Theta schedule, where FP32-accurate updates
    cannot be refined at any iteration (pivots of size delta make the factor
    grow by ~1/delta): the sliced updates keep the FP64 path's accuracy, so
    the factor matches the oracle's and refinement reaches 1e-12 without a
    fallback."""
    lp = synth.staircase(periods=3, pm=200, pn=500, density=0.01, links=50, seed=3)
    sched = synth.theta_schedule(lp.n, 40, 3)
    for it in (0, 20, 35):
        r, info = _sliced_pair(pkg, lp, sched[it], it, pkg.IPM_ORD_ND, 64)
        check_pair(r, lp, rowwise=True)
        r["s"].close()


def test_sliced_full_size_grid64_q4(pkg):
    """The grid workload at full size (m = 24,444, n = 64,512) with Theta
    10^U[-8,8]: no fallback, omega <= 1e-12 on K, the oracle's factor and
    solution."""
    lp = synth.by_name("grid64_q4", 1)
    theta = synth.theta_loguniform(lp.n, 1)
    r, info = _sliced_pair(pkg, lp, theta, 1, pkg.IPM_ORD_ND, 256)
    err = check_pair(r, lp, rowwise=True)
    print(f"sliced grid64: omega {r['w_gpu']:.2e} rel err {err:.2e} steps {info['refine_steps']}")
    r["s"].close()


def test_sliced_graph_replay_and_determinism(pkg):
    """The sliced factorisation is deterministic (exact integer sums, every
    entry updated once per panel in panel order): two factorisations agree
    bit for bit, and so does one IPM iteration replayed from a captured CUDA
    graph with the direct calls."""
    import torch

    lp = synth.grid_multicommodity(16, 4)
    n, m = lp.n, lp.m
    s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_ND, precision=pkg.IPM_PREC_SLICED, mixed_min_front=64,
                           level_kernel=0)
    th = synth.theta_loguniform(n, 43)
    s.factorise(th, RHO, DELTA)
    f1 = s.factor()
    s.factorise(th, RHO, DELTA)
    for a, b in zip(f1, s.factor()):
        assert np.array_equal(a, b)
    dev = s.dev
    r7 = np.concatenate([synth.rhs_normal(n, 44), synth.rhs_normal(n, 45)])
    r1 = np.concatenate([synth.rhs_normal(m, 46), synth.rhs_normal(m, 47)])
    theta = torch.as_tensor(th, device=dev)
    r7d, r1d = torch.as_tensor(r7, device=dev), torch.as_tensor(r1, device=dev)
    dx = torch.zeros(2 * n, dtype=torch.float64, device=dev)
    dy = torch.zeros(2 * m, dtype=torch.float64, device=dev)
    assert pkg.ipm_graph_capture(s.ctx, theta, RHO, DELTA, r7d, r1d, dx, dy, nsolves=2) == 0
    assert pkg.ipm_graph_launch(s.ctx) == 0
    torch.cuda.synchronize()
    assert s.info()["omega"] <= 1e-12 and s.info()["mixed_active"] == 1
    gx, gy = dx.cpu().numpy().copy(), dy.cpu().numpy().copy()
    s.factorise(th, RHO, DELTA)
    for k in range(2):
        ex, ey = s.solve(r7[k * n:(k + 1) * n], r1[k * m:(k + 1) * m])
        np.testing.assert_array_equal(gx[k * n:(k + 1) * n], ex.cpu().numpy())
        np.testing.assert_array_equal(gy[k * m:(k + 1) * m], ey.cpu().numpy())
    s.close()
