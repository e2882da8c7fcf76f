"""ctypes wrapper of the C oracle (ipm_oracle.c).

Test infrastructure: plain double-precision CPU code written from the paper
(Sections 3-4), used to check the GPU library.  Nothing in the product path
imports this module.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ipm_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libipm_oracle.so")

FORM_AS = 1
FORM_NE = 2

_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (portable flags only)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-w", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ct.CDLL(build_oracle())
    P = ct.c_void_p
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [ct.c_int, ct.c_int, i64p, i32p, f64p, ct.c_int]
    lib.orc_destroy.argtypes = [P]
    lib.orc_N.argtypes = [P]
    lib.orc_N.restype = ct.c_int
    lib.orc_analyse.argtypes = [P, P, ct.c_int, ct.c_int, ct.c_double]
    lib.orc_analyse.restype = ct.c_int
    lib.orc_nsuper.argtypes = [P]
    lib.orc_nsuper.restype = ct.c_int
    lib.orc_nrows_total.argtypes = [P]
    lib.orc_nrows_total.restype = ct.c_int64
    lib.orc_nnzL_stored.argtypes = [P]
    lib.orc_nnzL_stored.restype = ct.c_int64
    lib.orc_get_symbolic.argtypes = [P, i32p, i32p, i64p, i32p, i32p, i64p, i32p]
    lib.orc_factorise.argtypes = [P, f64p, ct.c_double, ct.c_double, ct.c_double]
    lib.orc_factorise.restype = ct.c_int
    lib.orc_get_factor.argtypes = [P, f64p, f64p, f64p, i64p]
    lib.orc_dense_ldlt_bk.argtypes = [ct.c_int, ct.c_int, f64p, ct.c_double, ct.c_double, i32p, f64p, f64p, i32p,
                                      f64p]
    lib.orc_dense_ldlt_bk.restype = ct.c_int
    lib.orc_front_ldlt_bk.argtypes = [ct.c_int, ct.c_int, ct.c_int, f64p, ct.c_double, ct.c_double, i32p, f64p, f64p,
                                      i32p, f64p]
    lib.orc_front_ldlt_bk.restype = ct.c_int
    lib.orc_dense_solve_bk.argtypes = [ct.c_int, f64p, f64p, f64p, i32p, i32p, f64p, f64p]
    lib.orc_dense_solve_bk.restype = ct.c_int
    lib.orc_set_pivoting.argtypes = [P, ct.c_int]
    lib.orc_get_pivots.argtypes = [P, i32p, f64p, i32p]
    lib.orc_get_stats.argtypes = [P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                  ct.POINTER(ct.c_double)]
    lib.orc_solve.argtypes = [P, f64p, f64p, f64p, f64p, f64p, ct.c_double, ct.c_int]
    lib.orc_solve.restype = ct.c_int
    lib.orc_refine_record.argtypes = [P, f64p, ct.POINTER(ct.c_double)]
    lib.orc_refine_record.restype = ct.c_int
    lib.orc_omega_K.argtypes = [P, f64p, ct.c_double, ct.c_double, f64p, f64p, f64p, f64p]
    lib.orc_omega_K.restype = ct.c_double
    lib.orc_front_factor.argtypes = [ct.c_int, ct.c_int, ct.c_int, f64p, i32p, f64p, ct.c_double, f64p, f64p]
    lib.orc_front_factor.restype = ct.c_int
    lib.orc_backward_error.argtypes = [ct.c_int, f64p, f64p, f64p, f64p, f64p]
    lib.orc_backward_error.restype = ct.c_double
    lib.orc_get_matrix.argtypes = [P, i64p, i32p, f64p]
    lib.orc_nnzM.argtypes = [P]
    lib.orc_nnzM.restype = ct.c_int64
    _lib = lib
    return lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Oracle:
    """One matrix pattern: analyse once, factorise and solve many times."""

    def __init__(self, m, n, colptr, rowidx, vals, form=FORM_AS):
        lib = _load()
        self.m, self.n, self.form = int(m), int(n), int(form)
        self._keep = (_c(colptr, np.int64), _c(rowidx, np.int32), _c(vals, np.float64))
        self.h = lib.orc_create(self.m, self.n, *self._keep, self.form)
        if not self.h:
            raise ValueError("oracle rejected the matrix")
        self.N = lib.orc_N(self.h)
        self.lib = lib

    @classmethod
    def from_lp(cls, lp, form=FORM_AS):
        return cls(lp.m, lp.n, lp.colptr, lp.rowidx, lp.vals, form)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def analyse(self, perm=None, nb=32, amalg_width=16, amalg_zero_frac=0.1):
        p = None
        if perm is not None:
            self._perm_in = _c(perm, np.int32)
            if self._perm_in.size != self.N:
                raise ValueError("permutation size")
            p = self._perm_in.ctypes.data_as(ct.c_void_p)
        rc = self.lib.orc_analyse(self.h, p, int(nb), int(amalg_width), float(amalg_zero_frac))
        if rc:
            raise ValueError(f"oracle analyse failed ({rc})")
        return self.symbolic()

    def symbolic(self):
        N, ns = self.N, self.lib.orc_nsuper(self.h)
        nr = self.lib.orc_nrows_total(self.h)
        out = dict(perm=np.empty(N, np.int32), parent=np.empty(N, np.int32), colcount=np.empty(N, np.int64),
                   sn_start=np.empty(ns + 1, np.int32), sn_parent=np.empty(ns, np.int32),
                   sn_rptr=np.empty(ns + 1, np.int64), sn_rows=np.empty(nr, np.int32))
        self.lib.orc_get_symbolic(self.h, out["perm"], out["parent"], out["colcount"], out["sn_start"],
                                  out["sn_parent"], out["sn_rptr"], out["sn_rows"])
        return out

    def set_pivoting(self, bk):
        """True: factorise every front with the Bunch-Kaufman variation of
        Sec. 4.5 (1x1 and 2x2 pivots, interchanges among its fully-summed
        columns); False: 1x1 pivots with the Prop. 3 bound."""
        self.lib.orc_set_pivoting(self.h, 1 if bk else 0)

    def pivots(self):
        """Per factorisation position: the local index the front moved there
        (lperm), D(p+1, p) of a 2x2 block starting at p (Doff) and the block
        size at a block's first position (bsize: 1, 2, or 0 at a 2x2 block's
        second position)."""
        N = self.N
        lp, do, bs = np.empty(N, np.int32), np.empty(N, np.float64), np.empty(N, np.int32)
        self.lib.orc_get_pivots(self.h, lp, do, bs)
        return dict(lperm=lp, Doff=do, bsize=bs)

    def factorise(self, theta, rho, delta, eps_piv=2.220446049250313e-16):
        rc = self.lib.orc_factorise(self.h, _c(theta, np.float64), float(rho), float(delta), float(eps_piv))
        self.theta = _c(theta, np.float64)
        self.rho, self.delta = float(rho), float(delta)
        return rc

    def factor(self):
        ns = self.lib.orc_nsuper(self.h)
        nl = self.lib.orc_nnzL_stored(self.h)
        L = np.empty(nl, np.float64)
        D = np.empty(self.N, np.float64)
        dyn = np.empty(self.N, np.float64)
        lptr = np.empty(ns + 1, np.int64)
        self.lib.orc_get_factor(self.h, L, D, dyn, lptr)
        return dict(L=L, D=D, dynreg=dyn, lptr=lptr)

    def stats(self):
        a, b, c = ct.c_int(), ct.c_int(), ct.c_int()
        d = ct.c_double()
        self.lib.orc_get_stats(self.h, ct.byref(a), ct.byref(b), ct.byref(c), ct.byref(d))
        return dict(ndyn=a.value, npos=b.value, nneg=c.value, normM1=d.value)

    def solve(self, r7, r1, omega_target=1e-12, max_steps=2):
        dx = np.empty(self.n, np.float64)
        dy = np.empty(self.m, np.float64)
        self.lib.orc_solve(self.h, self.theta, _c(r7, np.float64), _c(r1, np.float64), dx, dy,
                           float(omega_target), int(max_steps))
        hist = np.empty(65, np.float64)
        wk = ct.c_double()
        steps = self.lib.orc_refine_record(self.h, hist, ct.byref(wk))
        return dx, dy, dict(steps=steps, omega_hist=hist[: steps + 1].copy(), omega_K=wk.value)

    def omega_K(self, theta, rho, delta, r7, r1, dx, dy):
        return self.lib.orc_omega_K(self.h, _c(theta, np.float64), float(rho), float(delta), _c(r7, np.float64),
                                    _c(r1, np.float64), _c(dx, np.float64), _c(dy, np.float64))

    def nnz_lower(self):
        """Stored entries of the lower part of the matrix (K, or A A^T for the
        normal equations), diagonal included."""
        return int(self.lib.orc_nnzM(self.h))

    def nnzL_stored(self):
        """Entries of the supernodal L as stored: f_s x k_s per supernode."""
        return int(self.lib.orc_nnzL_stored(self.h))

    def nnzL(self):
        """Entries of L in the supernodal structure, unit diagonal included:
        supernode s holds k_s columns whose j-th (from 0) has f_s - j rows, so
        sum over s of k f - k (k - 1) / 2."""
        sym = self.symbolic()
        k = np.diff(sym["sn_start"]).astype(np.int64)
        f = np.diff(sym["sn_rptr"]).astype(np.int64)
        return int(np.sum(k * f - k * (k - 1) // 2))

    def front_flops(self):
        """sum over supernodes of sum_{i=1..k} (f-i)(f-i+3), from the symbolic
        result (the flop count of the blocked partial LDL^T of every front)."""
        sym = self.symbolic()
        k = np.diff(sym["sn_start"]).astype(np.int64)
        f = np.diff(sym["sn_rptr"]).astype(np.int64)
        total = 0.0
        for fs, ks in zip(f.tolist(), k.tolist()):
            i = np.arange(1, ks + 1, dtype=np.float64)
            total += float(np.sum((fs - i) * (fs - i + 3)))
        return total

    def matrix(self):
        nz = self.lib.orc_nnzM(self.h)
        cp = np.empty(self.N + 1, np.int64)
        ri = np.empty(nz, np.int32)
        x = np.empty(nz, np.float64)
        self.lib.orc_get_matrix(self.h, cp, ri, x)
        return cp, ri, x


def choose_form(lp, perm_as, perm_ne, az_as=0.1, az_ne=0.1, flop_rate=1.0e12, bandwidth=6.7e12, solves=3):
    """Choice between the augmented system and the normal equations (Sec. 4.2:
    the augmented system is the default, the normal equations are taken when
    they are cheaper; the paper leaves the measure open).  Reading: the
    per-iteration cost of a form is its front flops at flop_rate plus `solves`
    solves, each reading L twice (8 bytes per entry of the supernodal
    structure, Oracle.nnzL) at bandwidth;
    forming A Theta~ A^T adds 2 flops per contributor pair (one pair per column
    j of A and pair of its rows i <= r).  In order:
      1. symbolic analysis of K in the order perm_as;
      2. the normal equations are abandoned, cost -1, when the lower part of
         A A^T (diagonal included) holds more entries than L of step 1;
      3. otherwise symbolic analysis of A A^T in the order perm_ne;
      4. the form with the smaller cost wins, ties to the augmented system.
    The orders are inputs (ordering parity is not pinned); az_* are the
    amalgamation thresholds the symbolic analyses use.
    Returns (form, cost_as, cost_ne, nnz_ne_lower)."""
    oa = Oracle.from_lp(lp, FORM_AS)
    oa.analyse(perm_as, amalg_zero_frac=az_as)
    nnzl_as = oa.nnzL()
    cost_as = oa.front_flops() / flop_rate + solves * 2.0 * nnzl_as * 8.0 / bandwidth
    on = Oracle.from_lp(lp, FORM_NE)
    nnz_ne = on.nnz_lower()
    if nnz_ne > nnzl_as:
        return FORM_AS, cost_as, -1.0, nnz_ne
    on.analyse(perm_ne, amalg_zero_frac=az_ne)
    counts = np.diff(np.asarray(lp.colptr, dtype=np.int64)).astype(np.float64)
    pairs = float(np.sum(counts * (counts + 1.0) / 2.0))
    cost_ne = (on.front_flops() + 2.0 * pairs) / flop_rate + solves * 2.0 * on.nnzL() * 8.0 / bandwidth
    return (FORM_NE if cost_ne < cost_as else FORM_AS), cost_as, cost_ne, nnz_ne


def front_factor(F, k, signs, sreg, b1, nb=32):
    """Run the oracle's dense front factorisation (Sec. 4.4-4.5) on a full
    symmetric matrix F (f x f).  Returns (F_out, D, dynreg, rc)."""
    lib = _load()
    F = np.array(F, dtype=np.float64, order="F")
    f = F.shape[0]
    buf = np.ascontiguousarray(F.T.reshape(-1))  # column-major flat
    D = np.zeros(max(k, 1), np.float64)
    dyn = np.zeros(max(k, 1), np.float64)
    rc = lib.orc_front_factor(int(f), int(k), int(nb), buf, _c(signs, np.int32), _c(sreg, np.float64),
                              float(b1), D, dyn)
    out = buf.reshape(f, f).T.copy()
    return out, D[:k], dyn[:k], rc


def backward_error(r, ad, ae, f, d):
    lib = _load()
    return lib.orc_backward_error(int(len(r)), _c(r, np.float64), _c(ad, np.float64), _c(ae, np.float64),
                                  _c(f, np.float64), _c(d, np.float64))


BK_ALPHA = (1.0 + 17.0 ** 0.5) / 8.0  # the usual Bunch-Kaufman threshold (Sec. 4.5)


def dense_ldlt_bk(A, nb, b1, alpha=BK_ALPHA):
    """LDL^T of the dense symmetric matrix A with the pivoting of Sec. 4.5
    (a Bunch-Kaufman variation restricted to pivot blocks of nb columns, with
    a pre-swap and pivot lifting to magnitude b1).  Returns a dict with L
    (unit lower triangular), D and Doff (the block diagonal: Doff[k] =
    D(k+1, k) of a 2x2 block), bsize (1 or 2 at a block's first column, 0 at
    the second), perm (perm[new] = old), lift and rc, so that
    A[perm][:, perm] + diag(lift) = L Dblock L^T."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    F = np.asfortranarray(A).ravel(order="F").copy()
    perm = np.zeros(n, np.int32)
    D = np.zeros(n)
    Doff = np.zeros(n)
    bsize = np.zeros(n, np.int32)
    lift = np.zeros(n)
    rc = _load().orc_dense_ldlt_bk(n, int(nb), F, float(b1), float(alpha), perm, D, Doff, bsize, lift)
    M = F.reshape((n, n), order="F")
    L = np.tril(M, -1) + np.eye(n)
    Dblock = np.diag(D) + np.diag(Doff[:-1], -1) + np.diag(Doff[:-1], 1) if n > 1 else np.diag(D)
    return dict(L=L, D=D, Doff=Doff, Dblock=Dblock, bsize=bsize, perm=perm, lift=lift, rc=rc)


def dense_solve_bk(fac, b):
    """Solve with a factorisation from dense_ldlt_bk: x with
    P^T (L D L^T) P x = b, i.e. A x = b when nothing was lifted."""
    n = fac["L"].shape[0]
    Lf = np.asfortranarray(fac["L"]).ravel(order="F").copy()
    x = np.zeros(n)
    rc = _load().orc_dense_solve_bk(n, Lf, np.ascontiguousarray(fac["D"]), np.ascontiguousarray(fac["Doff"]),
                                    np.ascontiguousarray(fac["bsize"]), np.ascontiguousarray(fac["perm"]),
                                    np.ascontiguousarray(b, dtype=np.float64), x)
    if rc:
        raise RuntimeError(f"orc_dense_solve_bk failed ({rc})")
    return x


def front_ldlt_bk(A, k, nb, b1, alpha=BK_ALPHA):
    """Partial factorisation of a dense front with k fully-summed columns and
    the pivoting of Sec. 4.5: as dense_ldlt_bk on the first k columns, with
    S (the Schur complement of the trailing block) in the result."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    F = np.asfortranarray(A).ravel(order="F").copy()
    perm = np.zeros(n, np.int32)
    D = np.zeros(n)
    Doff = np.zeros(n)
    bsize = np.zeros(n, np.int32)
    lift = np.zeros(n)
    rc = _load().orc_front_ldlt_bk(n, int(k), int(nb), F, float(b1), float(alpha), perm, D, Doff, bsize, lift)
    M = F.reshape((n, n), order="F")
    L = np.tril(M[:, :k], -1)
    L[np.arange(k), np.arange(k)] = 1.0
    Dk = np.diag(D[:k]) + (np.diag(Doff[: k - 1], -1) + np.diag(Doff[: k - 1], 1) if k > 1 else 0.0)
    S = np.tril(M[k:, k:]) + np.tril(M[k:, k:], -1).T
    return dict(L=L, Dblock=Dk, D=D, Doff=Doff, bsize=bsize, perm=perm, lift=lift, S=S, rc=rc)
