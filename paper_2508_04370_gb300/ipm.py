"""Primal-dual interior point driver for standard-form LPs

    min c^T x   subject to   A x = b,  x >= 0,

built on this library's factorisation and solves (Zanetti & Gondzio,
arXiv 2508.04370, Sec. 2-3 and 4.7).  Each iteration forms Theta = X Z^-1,
factorises the regularised augmented system K = [[-(Theta^-1 + rho I), A^T],
[A, delta I]] once, and solves it twice: the Mehrotra predictor and one
corrector (Sec. 4.7: the first corrector always pays).  With the static
regularisation the directions are those of the primal-dual proximal method
the paper's regularisation comes from: the proximal terms vanish at the
current iterate, so the right-hand sides are the plain Newton ones,

    A dx = b - A x,   A^T dy + dz = c - A^T y - z,   Z dx + X dz = sigma mu e - X Z e,

and eliminating dz = X^-1 (r_c - Z dx) gives K [dx; dy] = [r_d - X^-1 r_c; r_p].
The factorise/solve work runs in the library's kernels; the driver's vector
updates are torch operations on the same device.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import IPM_ORD_AMD
from .solver import Solver


@dataclass
class IPMResult:
    status: str                 # "optimal" or "max_iter"
    iterations: int
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    objective: float
    history: list = field(default_factory=list)  # per iteration: residuals, mu, steps, solve omegas


def _csr_of_csc(m, n, colptr, rowidx, vals):
    colptr = np.asarray(colptr, dtype=np.int64)
    rowidx = np.asarray(rowidx, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    counts = np.bincount(rowidx, minlength=m)
    crow = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    order = np.argsort(rowidx, kind="stable")
    return crow, cols[order], vals[order]


def _step_to_boundary(torch, v, dv):
    neg = dv < 0
    if not bool(neg.any()):
        return 1.0
    return float(torch.clamp((-v[neg] / dv[neg]).min(), max=1.0))


def solve_lp(m, n, colptr, rowidx, vals, b, c, *, tol=1e-8, max_iter=100, rho=1e-8, delta=1e-8,
             ordering=IPM_ORD_AMD, device=0, step_factor=0.995, **options) -> IPMResult:
    """Solve min c^T x, A x = b, x >= 0 (A m x n in CSC, 0-based) to relative
    primal and dual residuals and duality gap below tol."""
    import torch

    dev = torch.device("cuda", int(device))
    solver = Solver(m, n, colptr, rowidx, vals, ordering=ordering, device=device, **options)
    crow, cols, avals = _csr_of_csc(m, n, colptr, rowidx, vals)
    A = torch.sparse_csr_tensor(torch.as_tensor(crow), torch.as_tensor(cols), torch.as_tensor(avals),
                                size=(m, n), dtype=torch.float64).to(dev)
    tcrow, tcols, tvals = _csr_of_csc(n, m, *_csc_of_transpose(m, n, colptr, rowidx, vals))
    At = torch.sparse_csr_tensor(torch.as_tensor(tcrow), torch.as_tensor(tcols), torch.as_tensor(tvals),
                                 size=(n, m), dtype=torch.float64).to(dev)
    b = torch.as_tensor(np.asarray(b, dtype=np.float64), device=dev)
    c = torch.as_tensor(np.asarray(c, dtype=np.float64), device=dev)
    x = torch.ones(n, dtype=torch.float64, device=dev)
    z = torch.ones(n, dtype=torch.float64, device=dev)
    y = torch.zeros(m, dtype=torch.float64, device=dev)
    nb, nc = 1.0 + float(torch.linalg.norm(b)), 1.0 + float(torch.linalg.norm(c))
    hist = []
    status = "max_iter"
    it = 0
    try:
        for it in range(max_iter + 1):
            rp = b - A @ x
            rd = c - At @ y - z
            mu = float(x @ z) / n
            pobj, dobj = float(c @ x), float(b @ y)
            rec = {"iter": it, "pres": float(torch.linalg.norm(rp)) / nb, "dres": float(torch.linalg.norm(rd)) / nc,
                   "gap": abs(pobj - dobj) / (1.0 + abs(pobj)), "mu": mu, "pobj": pobj}
            if max(rec["pres"], rec["dres"], rec["gap"]) < tol:
                hist.append(rec)
                status = "optimal"
                break
            if it == max_iter:
                hist.append(rec)
                break
            solver.factorise(x / z, rho, delta)
            # predictor (affine scaling): r_c = -X Z e
            rc = -x * z
            dx, dy = solver.solve(rd - rc / x, rp)
            dz = (rc - z * dx) / x
            w_pred = solver.info()["omega"]
            ap = _step_to_boundary(torch, x, dx)
            ad = _step_to_boundary(torch, z, dz)
            mu_aff = float((x + ap * dx) @ (z + ad * dz)) / n
            sigma = (mu_aff / mu) ** 3
            # corrector: r_c = sigma mu e - X Z e - dX_aff dZ_aff e
            rc = sigma * mu - x * z - dx * dz
            dx, dy = solver.solve(rd - rc / x, rp)
            dz = (rc - z * dx) / x
            w_corr = solver.info()["omega"]
            ap = min(1.0, step_factor * _step_to_boundary(torch, x, dx))
            ad = min(1.0, step_factor * _step_to_boundary(torch, z, dz))
            x = x + ap * dx
            y = y + ad * dy
            z = z + ad * dz
            rec.update({"sigma": sigma, "alpha_p": ap, "alpha_d": ad, "omega_pred": w_pred, "omega_corr": w_corr,
                        "theta_spread": float((x / z).max() / (x / z).min())})
            hist.append(rec)
    finally:
        solver.close()
    return IPMResult(status, it, x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy(), float(c @ x), hist)


def _csc_of_transpose(m, n, colptr, rowidx, vals):
    """CSC of A^T (n x m) from the CSC of A, i.e. the CSR of A reinterpreted."""
    crow, cols, avals = _csr_of_csc(m, n, colptr, rowidx, vals)
    return crow, cols, avals
