"""The pivot reciprocal of the factorisation (every column of L is the
pivot column scaled by it, Sec. 4.4-4.5) against CUDA's correctly rounded
1.0 / x: within one unit in the last place on log-uniform samples over the
whole range where the fast path applies, and equal to the division outside
it (range edges, subnormals, zeros, infinities, NaN), for both signs."""
import numpy as np
import pytest

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


def _run(pkg, x):
    import torch

    xd = torch.as_tensor(x, device="cuda")
    r = torch.empty_like(xd)
    q = torch.empty_like(xd)
    assert pkg.ipm_test_recip_pivot(xd, r, q) == 0
    torch.cuda.synchronize()
    return r.cpu().numpy(), q.cpu().numpy()


def test_recip_pivot_within_one_ulp(pkg):
    rng = np.random.default_rng(5)
    e = rng.uniform(-999.0, 999.0, 1 << 20)
    x = np.ldexp(rng.uniform(1.0, 2.0, e.size), np.floor(e).astype(np.int64))
    x[::2] *= -1.0
    r, q = _run(pkg, x)
    assert np.array_equal(q, 1.0 / x)  # CUDA's division is correctly rounded
    ulp = np.spacing(np.abs(q))
    err = np.abs(r - q) / ulp
    assert np.all(err <= 1.0), f"max {err.max():.2f} ulp"
    print(f"recip_pivot: max {err.max():.2f} ulp, exact on {np.mean(err == 0):.4f} of the samples")


def test_recip_pivot_range_edges(pkg):
    tiny = np.finfo(np.float64).tiny
    edges = [2.0 ** -1000, np.nextafter(2.0 ** -1000, 0.0), np.nextafter(2.0 ** -1000, 1.0),
             2.0 ** 1000, np.nextafter(2.0 ** 1000, np.inf), np.nextafter(2.0 ** 1000, 0.0),
             tiny, tiny / 8.0, 5e-324, np.finfo(np.float64).max, 1.0, 2.0, 0.5, 3.0, 1.0 / 3.0,
             np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 0.0, np.inf]
    x = np.array(edges + [-v for v in edges] + [np.nan])
    r, q = _run(pkg, x)
    out = (np.abs(x) < 2.0 ** -1000) | (np.abs(x) > 2.0 ** 1000) | ~np.isfinite(x)
    assert np.array_equal(r[out], q[out], equal_nan=True)
    fin = ~out
    assert np.all(np.abs(r[fin] - q[fin]) <= np.spacing(np.abs(q[fin])))
    assert np.all(r[x == 1.0] == 1.0) and np.all(r[x == 0.5] == 2.0)
