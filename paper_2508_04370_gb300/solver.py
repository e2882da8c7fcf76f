"""Convenience owner of one ipm context (argument marshalling only).

Device buffers are torch CUDA tensors; every numeric step runs in the CUDA
library behind include/ipm_mf.h.
"""
from __future__ import annotations

import numpy as np

from . import (IPM_FORM_AUGMENTED, IPM_ORD_AMD, ipm_analyse, ipm_autotune, ipm_create, ipm_default_options,
               ipm_destroy, ipm_factorise, ipm_get_factor, ipm_get_info, ipm_get_symbolic, ipm_iterate_host, ipm_load_analysis,
               ipm_save_analysis, ipm_set_values, ipm_solve, ipm_sync_status)


class Solver:
    """Analyse once (pattern of A), then factorise(theta) and solve(r7, r1)
    as many times as needed (one IPM iteration each)."""

    def __init__(self, m, n, colptr, rowidx, vals, form=IPM_FORM_AUGMENTED, ordering=IPM_ORD_AMD, user_perm=None,
                 device=0, **options):
        import torch

        self.torch = torch
        self.m, self.n = int(m), int(n)
        self.opt = ipm_default_options()
        self.opt.device = int(device)
        for k, v in options.items():
            if not hasattr(self.opt, k):
                raise KeyError(k)
            setattr(self.opt, k, v)
        self.ctx = ipm_create(self.opt)
        rc = self._analyse(m, n, colptr, rowidx, form, ordering, user_perm)
        if rc:
            ipm_destroy(self.ctx)
            self.ctx = None
            raise ValueError(f"ipm_analyse failed ({rc})")
        self.dev = torch.device("cuda", int(device))
        self.Ax = torch.as_tensor(np.ascontiguousarray(vals, dtype=np.float64), device=self.dev)
        rc = ipm_set_values(self.ctx, self.Ax)
        if rc:
            raise RuntimeError(f"ipm_set_values failed ({rc})")
        self.N = self.n + self.m

    def _analyse(self, m, n, colptr, rowidx, form, ordering, user_perm):
        path = getattr(self, "_load_path", None)
        if path is not None:
            rc = ipm_load_analysis(self.ctx, path)
            if rc == 0:
                _, info = ipm_get_info(self.ctx)
                self.m, self.n = int(info.m), int(info.n)
            return rc
        return ipm_analyse(self.ctx, m, n, colptr, rowidx, form, ordering, user_perm)

    @classmethod
    def from_lp(cls, lp, **kw):
        return cls(lp.m, lp.n, lp.colptr, lp.rowidx, lp.vals, **kw)

    @classmethod
    def from_analysis(cls, path, vals, device=0, **options):
        """A solver whose analysis is read from a file written by
        save_analysis (the pattern of A is in the file; vals are A's values
        in its CSC order)."""
        s = cls.__new__(cls)
        s._load_path = str(path)
        s.__init__(0, 0, None, None, vals, device=device, **options)
        return s

    def save_analysis(self, path):
        rc = ipm_save_analysis(self.ctx, str(path))
        if rc:
            raise RuntimeError(f"ipm_save_analysis failed ({rc})")

    def factorise(self, theta, rho, delta):
        theta = self._dev(theta)
        rc = ipm_factorise(self.ctx, theta, rho, delta)
        if rc < 0:
            raise RuntimeError(f"ipm_factorise failed ({rc})")
        self._theta = theta
        return rc

    def autotune(self, theta, rho, delta, reps=3):
        """Pick the factorisation's launch shapes by timing this problem
        (see ipm_autotune); returns the choices."""
        theta = self._dev(theta)
        rc = ipm_autotune(self.ctx, theta, rho, delta, reps)
        if rc < 0:
            raise RuntimeError(f"ipm_autotune failed ({rc})")
        self._theta = theta
        i = self.info()
        return {"small_threads": i["tune_small_threads"], "level_ratio": i["tune_level_ratio"],
                "level_ctas_per_sm": i["tune_level_ctas_per_sm"], "ms": i["tune_ms"]}

    def solve(self, r7, r1):
        r7 = self._dev(r7)
        r1 = self._dev(r1)
        dx = self.torch.empty(self.n, dtype=self.torch.float64, device=self.dev)
        dy = self.torch.empty(self.m, dtype=self.torch.float64, device=self.dev)
        rc = ipm_solve(self.ctx, r7, r1, dx, dy)
        if rc < 0:
            raise RuntimeError(f"ipm_solve failed ({rc})")
        return dx, dy

    def iterate_host(self, theta, rho, delta, r7, r1):
        dx = np.empty(self.n, np.float64)
        dy = np.empty(self.m, np.float64)
        rc = ipm_iterate_host(self.ctx, np.ascontiguousarray(theta, np.float64), rho, delta,
                              np.ascontiguousarray(r7, np.float64), np.ascontiguousarray(r1, np.float64), dx, dy)
        return rc, dx, dy

    def status(self):
        return ipm_sync_status(self.ctx)

    def info(self):
        rc, info = ipm_get_info(self.ctx)
        d = info.as_dict()
        d["rc"] = rc
        return d

    def symbolic(self):
        return ipm_get_symbolic(self.ctx)

    def factor(self):
        return ipm_get_factor(self.ctx)

    def _dev(self, x):
        t = self.torch
        if isinstance(x, t.Tensor):
            return x.to(device=self.dev, dtype=t.float64).contiguous()
        return t.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device=self.dev)

    def close(self):
        if self.ctx is not None:
            ipm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
