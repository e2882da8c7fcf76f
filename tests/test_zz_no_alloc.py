"""ipm_solve_noalloc: the allocation-free solve for callers that cannot
allocate device memory at solve time (a host library or callback under a
fixed device-memory budget, or one that must not change the device's
allocation state).  Its output must match ipm_solve's within the parity
tolerance of the solution (|x - x_ref|_inf <= 1e-8 |x_ref|_inf), on two calls
in a row, and ipm_get_info must then report its own backward error; a
tensor-core factor whose refinement stalls is returned with a warning (no
FP64 refactorisation here); a problem that does not fit its fixed work space
must be rejected before anything runs.  This file is collected last on
purpose."""
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


def test_noalloc_solve_matches_solve_twice(pkg):
    import torch

    lp = synth.grid_multicommodity(16, 4)
    theta = synth.theta_loguniform(lp.n, 31)
    r7, r1 = synth.rhs_normal(lp.n, 31), synth.rhs_normal(lp.m, 32)
    s = pkg.Solver.from_lp(lp)
    s.factorise(theta, 1e-8, 1e-8)
    dx, dy = s.solve(r7, r1)
    ref = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    a = s._dev(r7)
    b = s._dev(r1)
    for _ in range(2):
        ox = torch.full((lp.n,), np.nan, dtype=torch.float64, device=s.dev)
        oy = torch.full((lp.m,), np.nan, dtype=torch.float64, device=s.dev)
        rc = pkg.ipm_solve_noalloc(s.ctx, a, b, ox, oy)
        assert rc >= 0, rc
        torch.cuda.synchronize()
        x = np.concatenate([ox.cpu().numpy(), oy.cpu().numpy()])
        assert np.all(np.isfinite(x))
        assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max()
        info = s.info()
        assert info["omega"] <= 1e-12 and info["gmres_iters"] == 0
        assert info["omega_hist"][info["refine_steps"]] == pytest.approx(info["omega"], rel=0, abs=info["omega"])
    s.close()


def test_noalloc_reports_a_stalled_tensor_core_factor(pkg):
    """FP32-accurate tensor-core updates cannot be refined on this staircase
    (pivots of size delta make the factor grow by ~1/delta): ipm_solve would
    factorise again in FP64; the allocation-free solve does not, and says so
    in its return code (or reports the non-finite pivots)."""
    import torch

    lp = synth.staircase(periods=3, pm=200, pn=500, density=0.01, links=50, seed=3)
    theta = synth.theta_schedule(lp.n, 40, 3)[20]
    s = pkg.Solver.from_lp(lp, ordering=pkg.IPM_ORD_ND, precision=pkg.IPM_PREC_MIXED, mixed_min_front=64,
                           omega_target=1e-10, level_kernel=0)
    s.factorise(theta, 1e-8, 1e-8)
    ox = torch.empty(lp.n, dtype=torch.float64, device=s.dev)
    oy = torch.empty(lp.m, dtype=torch.float64, device=s.dev)
    rc = pkg.ipm_solve_noalloc(s.ctx, s._dev(synth.rhs_normal(lp.n, 1)), s._dev(synth.rhs_normal(lp.m, 2)), ox, oy)
    assert rc in (pkg.IPM_WARN_REFINE_NOT_CONVERGED, pkg.IPM_ERR_NONFINITE), rc
    info = s.info()
    assert info["mixed_active"] == 1 and info["precision_fallbacks"] == 0
    assert not (info["omega"] <= 1e-10)
    s.close()


def test_noalloc_rejects_problems_beyond_its_work_space(pkg):
    # 7 N + sum f > 2^21 doubles: N = 330,000 unknowns with one entry per column
    m, n = 110000, 220000
    colptr = np.arange(n + 1, dtype=np.int64)
    rowidx = (np.arange(n) % m).astype(np.int32)
    rowidx_sorted = rowidx  # one entry per column: sorted trivially
    ctx = pkg.ipm_create()
    assert pkg.ipm_analyse(ctx, m, n, colptr, rowidx_sorted) == 0
    rc = pkg.ipm_solve_noalloc(ctx, 0, 0, 0, 0, stream=0)
    assert rc == pkg.IPM_ERR_SCRATCH_TOO_SMALL
    pkg.ipm_destroy(ctx)
