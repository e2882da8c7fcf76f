"""Primal-dual interior point driver for LPs with bounds

    min c^T x   subject to   A x = b,   l <= x <= u   (entries of l, u may be infinite),

built on this library's factorisation and solves (Zanetti & Gondzio,
arXiv 2508.04370, Sec. 2-3 and 4.7).  Every iteration forms
Theta^-1 = Z^l (X^l)^-1 + Z^u (X^u)^-1 (a free variable contributes nothing:
its diagonal of K is the static regularisation -rho alone), factorises the
regularised augmented system K = [[-(Theta^-1 + rho I), A^T], [A, delta I]]
once, and solves it 1 + k times: the predictor, Mehrotra's corrector and up
to k - 1 multiple centrality correctors (Colombo and Gondzio), k from the
rule of Sec. 4.7,

    (1 + k)(1 + f/2) E_s ~= E_f alpha_F,

read with measured times: E_s alpha_s and E_f alpha_f are the measured time
of one solve pass (forward and backward through L) and of one
factorisation, so k = T_f / ((1 + f/2) T_s) - 1, lifted to at least 1 and
capped; f is the mean number of refinement steps per solve of the previous
iteration.  With the static regularisation the directions are those of the
primal-dual proximal method the regularisation comes from: the proximal
terms vanish at the current iterate, so the right-hand sides are the plain
Newton ones of Sec. 2.1,

    r1 = b - A x,  r2 = l - x + x^l,  r3 = u - x - x^u,  r4 = c - A^T y - z^l + z^u,
    r5 = sigma mu e - X^l Z^l e,  r6 = sigma mu e - X^u Z^u e,
    r7 = r4 - (X^l)^-1 (r5 + Z^l r2) + (X^u)^-1 (r6 - Z^u r3),

K [dx; dy] = [r7; r1], and dx^l = dx - r2, dx^u = r3 - dx,
dz^l = (X^l)^-1 (r5 - Z^l dx^l), dz^u = (X^u)^-1 (r6 - Z^u dx^u).
Termination is the paper's (Sec. 2.2): primal and dual infeasibility and the
relative primal-dual gap below tol.  The factorise/solve work runs in the
library's kernels; the driver's vector updates are torch operations on the
same device.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import IPM_ORD_AMD
from .solver import Solver

THETA_FREE = 1e30  # Theta of a free variable (Theta^-1 = 0 up to rounding): K's diagonal is -rho


@dataclass
class IPMResult:
    status: str                 # "optimal" or "max_iter"
    iterations: int
    x: np.ndarray
    y: np.ndarray
    zl: np.ndarray
    zu: np.ndarray
    objective: float
    history: list = field(default_factory=list)  # per iteration: residuals, mu, steps, correctors, solve omegas

    @property
    def z(self):
        """Reduced costs z^l - z^u."""
        return self.zl - self.zu


def corrector_count(t_factor, t_solve, refine_steps, k_max):
    """The number of correctors k of Sec. 4.7: (1 + k)(1 + f/2) solves take about
    the time of one factorisation, k >= 1 (the first corrector always pays)
    and k <= k_max."""
    if t_solve <= 0.0:
        return 1
    k = int(np.floor(t_factor / ((1.0 + refine_steps / 2.0) * t_solve) - 1.0))
    return max(1, min(k_max, k))


def _csr_of_csc(m, n, colptr, rowidx, vals):
    colptr = np.asarray(colptr, dtype=np.int64)
    rowidx = np.asarray(rowidx, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    counts = np.bincount(rowidx, minlength=m)
    crow = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    order = np.argsort(rowidx, kind="stable")
    return crow, cols[order], vals[order]


def _step_to_boundary(torch, v, dv, mask):
    """Largest alpha in (0, 1] with v + alpha dv >= 0 on the mask."""
    neg = mask & (dv < 0)
    if not bool(neg.any()):
        return 1.0
    return float(torch.clamp((-v[neg] / dv[neg]).min(), max=1.0))


class _Problem:
    """Device copies of the data and the bounded-variable bookkeeping."""

    def __init__(self, torch, dev, m, n, colptr, rowidx, vals, b, c, lower, upper):
        self.t = torch
        crow, cols, avals = _csr_of_csc(m, n, colptr, rowidx, vals)
        self.A = torch.sparse_csr_tensor(torch.as_tensor(crow), torch.as_tensor(cols), torch.as_tensor(avals),
                                         size=(m, n), dtype=torch.float64).to(dev)
        tcrow, tcols, tvals = _csr_of_csc(n, m, crow, cols, avals)
        self.At = torch.sparse_csr_tensor(torch.as_tensor(tcrow), torch.as_tensor(tcols), torch.as_tensor(tvals),
                                          size=(n, m), dtype=torch.float64).to(dev)
        f64 = dict(dtype=torch.float64, device=dev)
        self.b = torch.as_tensor(np.asarray(b, dtype=np.float64), **f64)
        self.c = torch.as_tensor(np.asarray(c, dtype=np.float64), **f64)
        lo = np.full(n, 0.0) if lower is None else np.asarray(lower, dtype=np.float64)
        up = np.full(n, np.inf) if upper is None else np.asarray(upper, dtype=np.float64)
        self.L = torch.as_tensor(np.isfinite(lo), device=dev)
        self.U = torch.as_tensor(np.isfinite(up), device=dev)
        self.l = torch.as_tensor(np.where(np.isfinite(lo), lo, 0.0), **f64)
        self.u = torch.as_tensor(np.where(np.isfinite(up), up, 0.0), **f64)
        self.nbound = int(self.L.sum()) + int(self.U.sum())
        self.scale_p = 1.0 + max(float(np.abs(b).max()) if len(b) else 0.0,
                                 float(np.abs(lo[np.isfinite(lo)]).max()) if np.isfinite(lo).any() else 0.0,
                                 float(np.abs(up[np.isfinite(up)]).max()) if np.isfinite(up).any() else 0.0)
        self.scale_d = 1.0 + (float(np.abs(c).max()) if len(c) else 0.0)

    def masked(self, v, mask):
        return self.t.where(mask, v, self.t.zeros_like(v))


def solve_lp(m, n, colptr, rowidx, vals, b, c, lower=None, upper=None, *, tol=1e-8, max_iter=100, rho=1e-8,
             delta=1e-8, ordering=IPM_ORD_AMD, device=0, step_factor=0.995, max_correctors=6, correctors=None,
             mcc_step=0.1, mcc_gain=0.1, beta_min=0.1, beta_max=10.0, **options) -> IPMResult:
    """Solve min c^T x, A x = b, lower <= x <= upper (A m x n in CSC, 0-based;
    lower defaults to 0 and upper to +inf: standard form) to the paper's
    termination test with tau_feas = tau_opt = tol.  correctors: None takes
    the number of correctors per iteration from the rule of Sec. 4.7 (at most
    max_correctors); an integer fixes it."""
    import torch

    dev = torch.device("cuda", int(device))
    solver = Solver(m, n, colptr, rowidx, vals, ordering=ordering, device=device, **options)
    P = _Problem(torch, dev, m, n, colptr, rowidx, vals, b, c, lower, upper)
    L, U = P.L, P.U
    one = torch.ones(n, dtype=torch.float64, device=dev)
    # starting point: boxed variables at the middle, one-sided ones one unit
    # inside their bound, free ones at 0; unit bound duals
    x = torch.where(L & U, 0.5 * (P.l + P.u), torch.where(L, P.l + 1.0, torch.where(U, P.u - 1.0, 0.0 * one)))
    xl = P.masked(x - P.l, L)
    xu = P.masked(P.u - x, U)
    boxed_narrow = L & U & (P.u - P.l < 2.0)
    xl = torch.where(boxed_narrow, 0.5 * (P.u - P.l), xl)
    xu = torch.where(boxed_narrow, 0.5 * (P.u - P.l), xu)
    zl = P.masked(one, L)
    zu = P.masked(one, U)
    y = torch.zeros(m, dtype=torch.float64, device=dev)
    hist = []
    status = "max_iter"
    it = 0
    f_prev = 1.0
    k_rule = 1

    def recover(dx, r2, r3, r5, r6):
        dxl = P.masked(dx - r2, L)
        dxu = P.masked(r3 - dx, U)
        dzl = P.masked((r5 - zl * dxl) / torch.where(L, xl, one), L)
        dzu = P.masked((r6 - zu * dxu) / torch.where(U, xu, one), U)
        return dxl, dxu, dzl, dzu

    def steps(dxl, dxu, dzl, dzu):
        ap = min(_step_to_boundary(torch, xl, dxl, L), _step_to_boundary(torch, xu, dxu, U))
        ad = min(_step_to_boundary(torch, zl, dzl, L), _step_to_boundary(torch, zu, dzu, U))
        return ap, ad

    def newton(r1, r2, r3, r4, r5, r6):
        r7 = (r4 - P.masked((r5 + zl * r2) / torch.where(L, xl, one), L)
              + P.masked((r6 - zu * r3) / torch.where(U, xu, one), U))
        t0 = time.perf_counter()
        dx, dy = solver.solve(r7, r1)
        torch.cuda.synchronize()
        info = solver.info()
        return dx, dy, info, time.perf_counter() - t0

    try:
        for it in range(max_iter + 1):
            r1 = P.b - P.A @ x
            r2 = P.masked(P.l - x + xl, L)
            r3 = P.masked(P.u - x - xu, U)
            r4 = P.c - P.At @ y - zl + zu
            mu = (float(xl @ zl) + float(xu @ zu)) / max(P.nbound, 1)
            fp = float(P.c @ x)
            fd = float(P.b @ y) + float(P.l @ zl) - float(P.u @ zu)
            pinf = max(float(r1.abs().max()) if m else 0.0, float(r2.abs().max()), float(r3.abs().max()))
            rec = {"iter": it, "pres": pinf / P.scale_p, "dres": float(r4.abs().max()) / P.scale_d,
                   "gap": abs(fp - fd) / (1.0 + 0.5 * abs(fp + fd)), "mu": mu, "pobj": fp}
            if max(rec["pres"], rec["dres"], rec["gap"]) < tol:
                hist.append(rec)
                status = "optimal"
                break
            if it == max_iter:
                hist.append(rec)
                break
            theta_inv = P.masked(zl / torch.where(L, xl, one), L) + P.masked(zu / torch.where(U, xu, one), U)
            theta = torch.where(theta_inv > 1.0 / THETA_FREE, 1.0 / theta_inv, THETA_FREE * one)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            solver.factorise(theta, rho, delta)
            torch.cuda.synchronize()
            t_factor = time.perf_counter() - t0
            # predictor (affine scaling, sigma = 0)
            r5 = P.masked(-xl * zl, L)
            r6 = P.masked(-xu * zu, U)
            dx, dy, info, t_pred = newton(r1, r2, r3, r4, r5, r6)
            omegas = [info["omega"]]
            fsteps = [info["refine_steps"]]
            dxl, dxu, dzl, dzu = recover(dx, r2, r3, r5, r6)
            ap, ad = steps(dxl, dxu, dzl, dzu)
            mu_aff = (float((xl + ap * dxl) @ (zl + ad * dzl)) + float((xu + ap * dxu) @ (zu + ad * dzu))) / max(
                P.nbound, 1)
            sigma = (mu_aff / mu) ** 3 if mu > 0 else 0.0
            # Mehrotra's corrector (the first corrector, always taken)
            r5 = P.masked(sigma * mu - xl * zl - dxl * dzl, L)
            r6 = P.masked(sigma * mu - xu * zu - dxu * dzu, U)
            dx, dy, info, _ = newton(r1, r2, r3, r4, r5, r6)
            omegas.append(info["omega"])
            fsteps.append(info["refine_steps"])
            dxl, dxu, dzl, dzu = recover(dx, r2, r3, r5, r6)
            ap, ad = steps(dxl, dxu, dzl, dzu)
            # number of correctors this iteration may afford (Sec. 4.7)
            # (one solve pass: the predictor's time over its 1 + refinement solves)
            k_rule = (corrector_count(t_factor, t_pred / (1.0 + fsteps[0]), f_prev, max_correctors)
                      if correctors is None else max(1, int(correctors)))
            used = 1
            # multiple centrality correctors (Colombo and Gondzio): aim at the
            # point of an enlarged step, move its complementarity products
            # outlying [beta_min, beta_max] sigma mu back into that interval
            for _ in range(k_rule - 1):
                if min(ap, ad) >= 1.0:
                    break
                tp, td = min(1.0, ap + mcc_step), min(1.0, ad + mcc_step)
                vl = P.masked((xl + tp * dxl) * (zl + td * dzl), L)
                vu = P.masked((xu + tp * dxu) * (zu + td * dzu), U)
                lo_t, hi_t = beta_min * sigma * mu, beta_max * sigma * mu
                tl = torch.clamp(lo_t - vl, min=0.0) + torch.clamp(hi_t - vl, max=0.0).clamp(min=-hi_t)
                tu = torch.clamp(lo_t - vu, min=0.0) + torch.clamp(hi_t - vu, max=0.0).clamp(min=-hi_t)
                cr5, cr6 = P.masked(tl, L), P.masked(tu, U)
                zero_n = torch.zeros(n, dtype=torch.float64, device=dev)
                zero_m = torch.zeros(m, dtype=torch.float64, device=dev)
                cdx, cdy, info, _ = newton(zero_m, zero_n, zero_n, zero_n, cr5, cr6)
                omegas.append(info["omega"])
                fsteps.append(info["refine_steps"])
                c_xl, c_xu, c_zl, c_zu = recover(cdx, zero_n, zero_n, cr5, cr6)
                n_xl, n_xu, n_zl, n_zu = dxl + c_xl, dxu + c_xu, dzl + c_zl, dzu + c_zu
                nap, nad = steps(n_xl, n_xu, n_zl, n_zu)
                if nap + nad < ap + ad + mcc_gain * mcc_step:
                    break  # not worth it: keep the previous direction
                dx, dy = dx + cdx, dy + cdy
                dxl, dxu, dzl, dzu = n_xl, n_xu, n_zl, n_zu
                ap, ad = nap, nad
                used += 1
            f_prev = float(np.mean(fsteps))
            ap = min(1.0, step_factor * ap)
            ad = min(1.0, step_factor * ad)
            x = x + ap * dx
            xl = xl + ap * dxl
            xu = xu + ap * dxu
            y = y + ad * dy
            zl = zl + ad * dzl
            zu = zu + ad * dzu
            rec.update({"sigma": sigma, "alpha_p": ap, "alpha_d": ad, "omega_pred": omegas[0],
                        "omega_corr": max(omegas[1:]), "correctors": used, "corrector_limit": k_rule,
                        "t_factor": t_factor, "theta_spread": float(theta.max() / theta.min())})
            hist.append(rec)
    finally:
        solver.close()
    return IPMResult(status, it, x.cpu().numpy(), y.cpu().numpy(), zl.cpu().numpy(), zu.cpu().numpy(),
                     float(P.c @ x), hist)
