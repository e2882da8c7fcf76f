"""Pins for the CPU oracle: facts fixed by the paper and by mathematics,
independent of the oracle's own code.

* hand-worked pivot-rule cases (Sec. 4.5, Prop. 3)         -> golden/pivot_rule_cases.json
* hand-worked symbolic cases (Sec. 4.1-4.3)                -> golden/symbolic_cases.json
* hand-worked backward-error cases (Sec. 4.5)              -> golden/backward_error_cases.json
* closed forms for A = I (Eq. augsys / Eq. normeq with Eq. regul_matrix)
* exact rational LDL^T on tiny systems (Python fractions)
* symbolic structure from a numpy Cholesky of a random SPD matrix on the pattern
* dense reconstruction, dense solve, inertia (Props. 1-2) against numpy / LAPACK
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import FORM_AS, FORM_NE, Oracle, backward_error, front_factor


# ----------------------------------------------------------------- helpers

def lp_from_dense(A):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    C = sp.csc_matrix(A)
    C.sort_indices()
    return m, n, C.indptr.astype(np.int64), C.indices.astype(np.int32), C.data.astype(np.float64)


def K_dense(A, theta, rho, delta):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    K = np.zeros((n + m, n + m))
    K[:n, :n] = np.diag(-(1.0 / theta + rho))
    K[n:, :n] = A
    K[:n, n:] = A.T
    K[n:, n:] = delta * np.eye(m)
    return K


def dense_L(orc_sym, fac, N):
    L = np.zeros((N, N))
    ns = len(orc_sym["sn_parent"])
    for s in range(ns):
        c0, c1 = orc_sym["sn_start"][s], orc_sym["sn_start"][s + 1]
        k = c1 - c0
        R = orc_sym["sn_rows"][orc_sym["sn_rptr"][s]:orc_sym["sn_rptr"][s + 1]]
        f = len(R)
        blk = fac["L"][fac["lptr"][s]:fac["lptr"][s + 1]].reshape(k, f).T
        for jj in range(k):
            L[R, c0 + jj] = blk[:, jj]
    return L


def load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as fh:
        return json.load(fh)


# ------------------------------------------------------- pivot rule cases

def test_pivot_rule_hand_cases(golden_dir):
    data = load(golden_dir, "pivot_rule_cases.json")
    for case in data["cases"]:
        F = np.array(case["F"])
        Fo, D, dyn, rc = front_factor(F, case["k"], case["signs"], case["sreg"], case["b1"])
        assert rc == 0, case["name"]
        np.testing.assert_allclose(D, case["D"], rtol=1e-13, atol=0, err_msg=case["name"])
        np.testing.assert_allclose(dyn, case["dynreg"], rtol=1e-12, atol=1e-15, err_msg=case["name"])
        L = np.tril(Fo, -1) + np.eye(F.shape[0])
        np.testing.assert_allclose(L, np.array(case["L"], dtype=float), rtol=1e-13, atol=1e-15,
                                   err_msg=case["name"])


def test_prop3_bound_holds_for_every_accepted_pivot():
    """Prop. 3: after a pivot is accepted, every later same-sign diagonal in
    its block that was correctly signed keeps its sign.  Checked on random
    symmetric blocks by recomputing the partially eliminated matrix densely."""
    rng = np.random.default_rng(5)
    fired = 0
    for trial in range(40):
        f = 12
        signs = rng.choice([-1, 1], size=f)
        B = rng.standard_normal((f, f))
        F = 0.6 * (B + B.T) / 2
        F[np.arange(f), np.arange(f)] = signs * rng.uniform(0.05, 1.5, size=f)
        # a few diagonals pushed towards zero or past it
        bad = rng.choice(f, size=3, replace=False)
        F[bad, bad] = signs[bad] * rng.uniform(-0.2, 0.01, size=3)
        sreg = np.full(f, 1e-3)
        Fo, D, dyn, rc = front_factor(F, f, signs, sreg, 0.05, nb=4)
        L = np.tril(Fo, -1) + np.eye(f)
        # reconstruct the matrix actually factorised: F + diag(s*sreg + dyn)
        Freg = F + np.diag(signs * sreg + dyn)
        scale = np.abs(L) @ np.diag(np.abs(D)) @ np.abs(L).T
        scale += np.diag(np.abs(np.diag(F)) + sreg + np.abs(dyn))  # rounding of F_pp + s*sreg + dyn
        assert np.all(np.abs(L @ np.diag(D) @ L.T - Freg) <= 1e-13 * scale + 1e-300)
        # signs of the pivots are the expected ones
        assert np.all(np.sign(D) == signs)
        fired += int(np.count_nonzero(dyn))
        # Prop. 3 inside each block of 4: after eliminating p, diagonal j>p of the
        # same block with the same sign and correct sign before keeps it
        S = F.copy()
        acc = np.abs(np.diag(F)).copy()  # magnitude of everything summed into each diagonal
        for p in range(f):
            blk_end = (p // 4 + 1) * 4
            S[p, p] += signs[p] * sreg[p] + dyn[p]  # both terms enter at pivot time
            before = np.diag(S).copy()
            col = S[:, p].copy()
            upd = np.outer(col, col) / S[p, p]
            S = S - upd
            acc += np.abs(np.diag(upd))
            for j in range(p + 1, min(blk_end, f)):
                # only diagonals that are clearly correctly signed (not a rounding-level
                # zero left by an earlier pivot lifted exactly to its bound)
                if signs[j] == signs[p] and signs[j] * before[j] > 1e-8 * acc[j]:
                    tol = 1e-8 * acc[j]
                    assert signs[j] * S[j, j] >= -tol, (trial, p, j)
    assert fired > 10


# ---------------------------------------------------------- backward error

def test_backward_error_hand_cases(golden_dir):
    data = load(golden_dir, "backward_error_cases.json")
    for case in data["cases"]:
        M = np.array(case["M"], dtype=float)
        d = np.array(case["d"], dtype=float)
        f = np.array(case["f"], dtype=float)
        r = f - M @ d
        ad = np.abs(M) @ np.abs(d)
        ae = np.abs(M).sum(axis=1)
        w = backward_error(r, ad, ae, f, d)
        assert w == pytest.approx(case["omega"], rel=1e-12, abs=1e-300), case["name"]


def test_backward_error_nonfinite_solution():
    # a solution with a NaN component has no finite backward error, whichever
    # component it poisons (Sec. 4.5: omega bounds the relative perturbation)
    M = np.array([[2.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 4.0]])
    f = np.array([1.0, -2.0, 0.5])
    for bad in range(3):
        d = np.linalg.solve(M, f)
        assert backward_error(f - M @ d, np.abs(M) @ np.abs(d), np.abs(M).sum(axis=1), f, d) < 1e-15
        d[bad] = np.nan
        r = f - M @ d
        w = backward_error(r, np.abs(M) @ np.abs(d), np.abs(M).sum(axis=1), f, d)
        assert w == np.inf


# -------------------------------------------------------------- symbolic

def _tridiag_ne(m):
    A = np.zeros((m, m - 1))
    for i in range(m - 1):
        A[i, i] = 1.0
        A[i + 1, i] = 1.0
    return A


def _arrow_ne(m):
    A = np.zeros((m, m - 1))
    for i in range(m - 1):
        A[i, i] = 1.0
        A[m - 1, i] = 1.0
    return A


def test_symbolic_hand_cases(golden_dir):
    data = load(golden_dir, "symbolic_cases.json")
    cases = {c["kind"]: c for c in data["cases"]}
    # tridiagonal: chain
    m = cases["ne_path"]["m"]
    o = Oracle(*lp_from_dense(_tridiag_ne(m)), form=FORM_NE)
    s = o.analyse(np.arange(m))
    assert list(s["parent"]) == list(range(1, m)) + [-1]
    assert list(s["colcount"]) == [2] * (m - 1) + [1]
    assert list(s["sn_start"]) == cases["ne_path"]["sn_start"]
    o2 = Oracle(*lp_from_dense(_tridiag_ne(m)), form=FORM_NE)
    s2 = o2.analyse(np.arange(m), amalg_width=1, amalg_zero_frac=0.0)
    assert list(s2["sn_start"]) == list(range(0, m - 1)) + [m]
    # arrowhead: star
    m = cases["ne_arrow"]["m"]
    o = Oracle(*lp_from_dense(_arrow_ne(m)), form=FORM_NE)
    s = o.analyse(np.arange(m))
    assert list(s["parent"]) == [m - 1] * (m - 1) + [-1]
    assert list(s["colcount"]) == [2] * (m - 1) + [1]
    assert list(s["sn_start"]) == cases["ne_arrow"]["sn_start"]
    # identity A, interleaved
    n = cases["as_identity"]["n"]
    o = Oracle(*lp_from_dense(np.eye(n)), form=FORM_AS)
    perm = np.ravel(np.column_stack([np.arange(n), n + np.arange(n)])).astype(np.int32)
    s = o.analyse(perm)
    assert list(s["perm"]) == list(perm)
    assert list(s["parent"]) == [v for j in range(n) for v in (2 * j + 1, -1)]
    assert list(s["colcount"]) == [2, 1] * n
    assert list(s["sn_start"]) == list(range(0, 2 * n + 1, 2))
    # two overlapping dense columns: the zero-fraction rule decides the merge
    c = cases["ne_two_blocks"]
    m = c["m"]
    A = np.zeros((m, 2))
    A[:19, 0] = 1.0
    A[10:, 1] = 1.0
    o = Oracle(*lp_from_dense(A), form=FORM_NE)
    s = o.analyse(np.arange(m))
    assert list(s["colcount"]) == [19 - j for j in range(10)] + [20 - j for j in range(10, 20)]
    assert list(s["sn_start"]) == c["sn_start"]
    o = Oracle(*lp_from_dense(A), form=FORM_NE)
    s = o.analyse(np.arange(m), amalg_zero_frac=0.04)
    assert list(s["sn_start"]) == c["sn_start_4pct"]


def _structure_from_cholesky(Mpat_dense, rng):
    """Structure of L from a numeric Cholesky of an SPD matrix with the given
    pattern (no cancellation for generic random values)."""
    N = Mpat_dense.shape[0]
    V = rng.uniform(0.5, 1.0, size=(N, N))
    V = (V + V.T) / 2 * Mpat_dense
    np.fill_diagonal(V, 0.0)
    V += np.diag(np.abs(V).sum(axis=1) + 1.0)
    L = np.linalg.cholesky(V)
    nzL = L != 0.0
    parent = np.full(N, -1)
    colcount = np.zeros(N, dtype=int)
    for j in range(N):
        rows = np.flatnonzero(nzL[j + 1:, j]) + j + 1
        parent[j] = rows[0] if rows.size else -1
        colcount[j] = rows.size + 1
    return parent, colcount, nzL


@pytest.mark.parametrize("form", [FORM_AS, FORM_NE])
def test_symbolic_against_numeric_cholesky(form):
    rng = np.random.default_rng(11)
    for trial in range(6):
        lp = synth.random_lp(14 + trial, 30 + 2 * trial, 3, seed=100 + trial)
        o = Oracle.from_lp(lp, form=form)
        N = o.N
        s = o.analyse(synth.random_perm(N, trial))
        cp, ri, _ = o.matrix()
        pat = np.zeros((N, N), dtype=bool)
        for j in range(N):
            for p in range(cp[j], cp[j + 1]):
                pat[ri[p], j] = pat[j, ri[p]] = True
        P = s["perm"]
        parent, colcount, nzL = _structure_from_cholesky(pat[np.ix_(P, P)].astype(float), rng)
        assert np.array_equal(s["parent"], parent)
        assert np.array_equal(s["colcount"], colcount)
        # postorder: every parent comes after its children, and subtrees are contiguous
        assert np.all((s["parent"] == -1) | (s["parent"] > np.arange(N)))
        # supernodes: contiguous columns, rows sorted, first k rows are the columns
        for t in range(len(s["sn_parent"])):
            c0, c1 = s["sn_start"][t], s["sn_start"][t + 1]
            R = s["sn_rows"][s["sn_rptr"][t]:s["sn_rptr"][t + 1]]
            assert list(R[: c1 - c0]) == list(range(c0, c1))
            assert np.all(np.diff(R) > 0)
            # the front rows are exactly the union of its columns' structures
            union = set()
            for j in range(c0, c1):
                union |= set(np.flatnonzero(nzL[:, j]).tolist())
            assert set(R.tolist()) == union


# ----------------------------------------------------------- closed forms

def test_closed_form_identity_augmented():
    n = 10
    theta = 10.0 ** np.linspace(-3, 3, n)
    rho, delta = 1e-6, 2e-6
    o = Oracle(*lp_from_dense(np.eye(n)), form=FORM_AS)
    perm = np.ravel(np.column_stack([np.arange(n), n + np.arange(n)])).astype(np.int32)
    s = o.analyse(perm)
    assert o.factorise(theta, rho, delta, eps_piv=0.0) == 0
    fac = o.factor()
    D = fac["D"]
    dx = -(1.0 / theta + rho)
    dy = delta + 1.0 / (1.0 / theta + rho)
    np.testing.assert_allclose(D[0::2], dx, rtol=4e-16)
    np.testing.assert_allclose(D[1::2], dy, rtol=4e-16)
    L = dense_L(s, fac, 2 * n)
    for j in range(n):
        assert L[2 * j + 1, 2 * j] == pytest.approx(1.0 / dx[j], rel=4e-16)
    assert np.all(fac["dynreg"] == 0.0)


def test_closed_form_identity_normal_equations():
    n = 10
    theta = 10.0 ** np.linspace(-4, 4, n)
    rho, delta = 1e-6, 3e-6
    o = Oracle(*lp_from_dense(np.eye(n)), form=FORM_NE)
    o.analyse(None)
    assert o.factorise(theta, rho, delta, eps_piv=0.0) == 0
    D = o.factor()["D"]
    np.testing.assert_allclose(D, 1.0 / (1.0 / theta + rho) + delta, rtol=4e-16)


# ------------------------------------------------------- exact arithmetic

def _exact_ldlt(M):
    N = len(M)
    A = [row[:] for row in M]
    L = [[Fraction(int(i == j)) for j in range(N)] for i in range(N)]
    D = [Fraction(0)] * N
    for p in range(N):
        D[p] = A[p][p]
        for i in range(p + 1, N):
            L[i][p] = A[i][p] / D[p]
        for i in range(p + 1, N):
            for j in range(p + 1, i + 1):
                A[i][j] -= L[i][p] * D[p] * L[j][p]
                A[j][i] = A[i][j]
    return L, D


def test_exact_rational_ldlt():
    rng = np.random.default_rng(3)
    for trial in range(5):
        m, n = 3, 5
        Aint = rng.integers(-3, 4, size=(m, n))
        Aint[rng.random((m, n)) < 0.4] = 0
        for j in range(n):
            if not Aint[:, j].any():
                Aint[rng.integers(m), j] = 1
        for i in range(m):
            if not Aint[i].any():
                Aint[i, rng.integers(n)] = 2
        theta_fr = [Fraction(2) ** int(e) for e in rng.integers(-6, 7, size=n)]
        rho = Fraction(1, 2 ** 10)
        delta = Fraction(1, 2 ** 11)
        N = n + m
        K = [[Fraction(0)] * N for _ in range(N)]
        for j in range(n):
            K[j][j] = -(1 / theta_fr[j] + rho)
        for i in range(m):
            K[n + i][n + i] = delta
            for j in range(n):
                K[n + i][j] = K[j][n + i] = Fraction(int(Aint[i, j]))
        o = Oracle(*lp_from_dense(Aint.astype(float)), form=FORM_AS)
        s = o.analyse(synth.random_perm(N, 50 + trial))
        P = s["perm"]
        KP = [[K[P[i]][P[j]] for j in range(N)] for i in range(N)]
        Le, De = _exact_ldlt(KP)
        theta = np.array([float(t) for t in theta_fr])
        assert o.factorise(theta, float(rho), float(delta), eps_piv=0.0) == 0
        fac = o.factor()
        assert np.all(fac["dynreg"] == 0.0)
        Lx = np.array([[float(v) for v in row] for row in Le])
        Dx = np.array([float(v) for v in De])
        eps = 2.220446049250313e-16
        Lo = dense_L(s, fac, N)
        Do = fac["D"]
        # (1) backward stability against the exact matrix: |L D L^T - P K P^T| <= c eps |L||D||L^T|
        KPx = np.array([[float(v) for v in row] for row in KP])
        So = np.abs(Lo) @ np.diag(np.abs(Do)) @ np.abs(Lo).T
        assert np.all(np.abs(Lo @ np.diag(Do) @ Lo.T - KPx) <= 32 * eps * So), trial
        # (2) forward agreement with the exact factors; the leading blocks have
        # condition numbers up to ~1e5 here, so 1e-8 of the |L||D||L^T| scale
        # still fails on any dropped term or sign
        S = np.abs(Lx) @ np.diag(np.abs(Dx)) @ np.abs(Lx).T
        assert np.all(np.abs(Do - Dx) <= 1e-8 * np.diag(S)), trial
        tolL = 1e-8 * (S / np.abs(Dx)[None, :] + np.abs(Lx))
        assert np.all(np.abs(Lo - Lx) <= tolL), trial
        # structural zeros are exact zeros
        assert np.all(Lo[Lx == 0] == 0.0)


# ---------------------------------------------- dense brute force, inertia

@pytest.mark.parametrize("form", [FORM_AS, FORM_NE])
def test_dense_reconstruction_and_solve(form):
    for trial in range(3):
        lp = synth.random_lp(40, 100, 4, seed=200 + trial)
        theta = synth.theta_loguniform(lp.n, trial, -1.0, 1.0)
        rho, delta = 1e-8, 1e-8
        o = Oracle.from_lp(lp, form=form)
        s = o.analyse(synth.random_perm(o.N, trial))
        assert o.factorise(theta, rho, delta, eps_piv=1e-14) == 0
        fac = o.factor()
        N = o.N
        A = sp.csc_matrix((lp.vals, lp.rowidx, lp.colptr), shape=(lp.m, lp.n)).toarray()
        K = K_dense(A, theta, rho, delta)
        if form == FORM_AS:
            M = K.copy()
        else:
            tt = 1.0 / (1.0 / theta + rho)
            M = A @ np.diag(tt) @ A.T + delta * np.eye(lp.m)
        P = s["perm"]
        Mp = M[np.ix_(P, P)] + np.diag(fac["dynreg"])
        L = dense_L(s, fac, N)
        R = L @ np.diag(fac["D"]) @ L.T
        scale = np.abs(L) @ np.diag(np.abs(fac["D"])) @ np.abs(L).T
        assert np.all(np.abs(R - Mp) <= 1e-13 * scale + 1e-300)
        # inertia: n negative and m positive pivots (AS), m positive (NE)
        if form == FORM_AS:
            assert (fac["D"] < 0).sum() == lp.n and (fac["D"] > 0).sum() == lp.m
            ev = np.linalg.eigvalsh(K)
            assert (ev < 0).sum() == lp.n
        else:
            assert (fac["D"] > 0).sum() == lp.m
        # solve against LAPACK on the well-conditioned system
        r7 = synth.rhs_normal(lp.n, trial)
        r1 = synth.rhs_normal(lp.m, trial + 9)
        dx, dy, info = o.solve(r7, r1, omega_target=1e-14, max_steps=5)
        x = np.linalg.solve(K, np.concatenate([r7, r1]))
        np.testing.assert_allclose(np.concatenate([dx, dy]), x, rtol=1e-9, atol=1e-9 * np.abs(x).max())
        assert info["omega_K"] < 1e-13


def test_refinement_reaches_target_on_ill_conditioned_theta():
    lp = synth.by_name("random_300x800", 1)
    theta = synth.theta_loguniform(lp.n, 1)
    o = Oracle.from_lp(lp)
    o.analyse(synth.random_perm(o.N, 1))
    o.factorise(theta, 1e-8, 1e-8, eps_piv=1e-14)
    r7 = synth.rhs_normal(lp.n, 1)
    r1 = synth.rhs_normal(lp.m, 2)
    dx, dy, info = o.solve(r7, r1, omega_target=1e-12, max_steps=10)
    assert info["omega_hist"][-1] <= 1e-12
    assert info["omega_K"] <= 1e-12
    # every accepted refinement step at least halves omega
    h = info["omega_hist"]
    assert np.all(h[1:] <= 0.5 * h[:-1])
    # the oracle's omega equals a direct evaluation of the formula
    w = o.omega_K(theta, 1e-8, 1e-8, r7, r1, dx, dy)
    assert w == info["omega_K"]


def test_normal_equations_match_augmented_system():
    lp = synth.random_lp(60, 150, 4, seed=7)
    theta = synth.theta_loguniform(lp.n, 7, -2.0, 2.0)
    r7 = synth.rhs_normal(lp.n, 3)
    r1 = synth.rhs_normal(lp.m, 4)
    res = {}
    for form in (FORM_AS, FORM_NE):
        o = Oracle.from_lp(lp, form=form)
        o.analyse(synth.random_perm(o.N, 1))
        o.factorise(theta, 1e-8, 1e-8, eps_piv=1e-14)
        res[form] = o.solve(r7, r1, omega_target=1e-14, max_steps=5)
        assert res[form][2]["omega_K"] < 1e-12
    x1 = np.concatenate(res[FORM_AS][:2])
    x2 = np.concatenate(res[FORM_NE][:2])
    np.testing.assert_allclose(x1, x2, rtol=1e-8, atol=1e-8 * np.abs(x1).max())


def test_deterministic_bitwise():
    lp = synth.by_name("random_300x800", 2)
    theta = synth.theta_loguniform(lp.n, 2)
    outs = []
    for _ in range(2):
        o = Oracle.from_lp(lp)
        o.analyse(synth.random_perm(o.N, 2))
        o.factorise(theta, 1e-8, 1e-8)
        outs.append(o.factor())
    for key in ("L", "D", "dynreg"):
        assert np.array_equal(outs[0][key], outs[1][key])


def test_rejects_bad_input():
    lp = synth.random_lp(5, 8, 2, seed=1)
    o = Oracle.from_lp(lp)
    with pytest.raises(ValueError):
        o.analyse(np.zeros(o.N, dtype=np.int32))  # not a permutation
    o.analyse(None)
    theta = np.ones(lp.n)
    theta[3] = np.nan
    assert o.factorise(theta, 1e-8, 1e-8) != 0
    bad = lp.rowidx.copy()
    bad[0] = lp.m + 3
    with pytest.raises(ValueError):
        Oracle(lp.m, lp.n, lp.colptr, bad, lp.vals)


# --------------------------------------------- Bunch-Kaufman pivoting (dense)
# Sec. 4.5: the variation of Bunch-Kaufman pivoting inside pivot blocks, with a
# pre-swap and pivot lifting.  Pinned by the factorisation identity (checked by
# numpy products), Sylvester's law of inertia, the element-growth bound of
# Bunch-Kaufman, and hand-worked cases.

def _bk_residual(A, r):
    P = r["perm"]
    R = r["L"] @ r["Dblock"] @ r["L"].T - (A[np.ix_(P, P)] + np.diag(r["lift"]))
    return np.abs(R).max() / max(np.abs(A).max(), 1e-300)


@pytest.mark.parametrize("n,nb", [(1, 1), (2, 2), (13, 4), (40, 8), (40, 40), (33, 32), (50, 7)])
def test_bk_factor_identity_and_permutation(n, nb):
    from oracle.oracle import dense_ldlt_bk

    rng = np.random.default_rng(100 + n + nb)
    A = rng.standard_normal((n, n))
    A = A + A.T
    r = dense_ldlt_bk(A, nb, 0.0)
    assert r["rc"] == 0
    assert np.array_equal(np.sort(r["perm"]), np.arange(n))
    assert _bk_residual(A, r) <= 1e-12
    # blocks: a 2x2 block's second column carries 0, and the block sizes tile n
    assert r["bsize"].sum() == n
    for k in np.flatnonzero(r["bsize"] == 2):
        assert r["bsize"][k + 1] == 0 and (k // nb) == ((k + 1) // nb)  # a 2x2 block stays inside its pivot block
    # pivots are exchanged only within their pivot block
    assert all(r["perm"][k] // nb == k // nb for k in range(n))
    r2 = dense_ldlt_bk(A, nb, 0.0)
    assert all(np.array_equal(r[key], r2[key]) for key in ("L", "D", "Doff", "perm", "bsize"))


def test_bk_needs_a_2x2_pivot():
    """[[0, 1], [1, 0]] has no usable 1x1 pivot: the whole matrix is one 2x2
    block of D and L is the identity."""
    from oracle.oracle import dense_ldlt_bk

    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    r = dense_ldlt_bk(A, 2, 0.0)
    assert r["rc"] == 0 and list(r["bsize"]) == [2, 0]
    assert np.array_equal(r["Dblock"], A) and np.array_equal(r["L"], np.eye(2))


def test_bk_inertia_and_growth():
    """Sylvester: the block diagonal D has the inertia of A.  With one pivot
    block (the classical setting) every entry of L is bounded by the
    Bunch-Kaufman growth bound 1 / (1 - alpha) (1 / alpha for 1x1 pivots)."""
    from oracle.oracle import BK_ALPHA, dense_ldlt_bk

    rng = np.random.default_rng(7)
    for trial in range(5):
        n = 30 + 3 * trial
        A = rng.standard_normal((n, n))
        A = A + A.T + np.diag(rng.standard_normal(n) * (10.0 if trial % 2 else 0.01))
        for nb in (n, 8):
            r = dense_ldlt_bk(A, nb, 0.0)
            ev_a = np.linalg.eigvalsh(A)
            ev_d = np.linalg.eigvalsh(r["Dblock"])
            assert (ev_a > 0).sum() == (ev_d > 0).sum() and (ev_a < 0).sum() == (ev_d < 0).sum()
        r = dense_ldlt_bk(A, n, 0.0)
        assert np.abs(np.tril(r["L"], -1)).max() <= 1.0 / (1.0 - BK_ALPHA) + 1e-12


def test_bk_pre_swap_and_no_pivoting_cases():
    """The pre-swap moves the largest diagonal of the block to the pivot
    position; a diagonally dominant matrix then needs 1x1 pivots only.  With
    blocks of one column nothing can be exchanged: plain LDL^T."""
    from oracle.oracle import dense_ldlt_bk

    rng = np.random.default_rng(3)
    n = 6
    A = 0.01 * rng.standard_normal((n, n))
    A = A + A.T + np.diag([2.0, -3.0, 1.5, 9.0, -4.0, 2.5])
    r = dense_ldlt_bk(A, n, 0.0)
    assert r["perm"][0] == 3 and np.all(r["bsize"] == 1)
    assert _bk_residual(A, r) <= 1e-14
    B = rng.standard_normal((n, n))
    B = B + B.T + 6.0 * np.eye(n)
    r = dense_ldlt_bk(B, 1, 0.0)
    assert np.array_equal(r["perm"], np.arange(n)) and np.all(r["bsize"] == 1)
    assert _bk_residual(B, r) <= 1e-13


def test_bk_lift_keeps_the_sign():
    """A pivot whose magnitude and column are below b1 is lifted to
    magnitude b1 with the sign of M_pp; the larger diagonal goes first."""
    from oracle.oracle import dense_ldlt_bk

    A = np.array([[-1e-20, 0.0], [0.0, 1.0]])
    r = dense_ldlt_bk(A, 2, 1e-10)
    assert list(r["perm"]) == [1, 0]
    assert r["D"][0] == 1.0 and r["D"][1] == -1e-10
    assert r["lift"][1] == -1e-10 - (-1e-20) and r["lift"][0] == 0.0


def test_bk_decision_rule_hand_cases():
    """Hand-worked 3 x 3 blocks (alpha = (1 + sqrt 17) / 8 = 0.640):
    M = [[a, g, 0], [g, b, h], [0, h, c]] with a the largest diagonal, so
    p = 0, r = 1, gamma_p = |g|, gamma_r = max(|g|, |h|).
      a = .5, g = 1, h = 2: |a| < alpha |g|, but |a| gamma_r = 1 >= alpha g^2
        -> 1x1 pivot at p;
      a = .5, g = 1, h = .5: |a| gamma_r = .5 < alpha, |b| = .1 < alpha gamma_r
        -> 2x2 pivot (0, 1);
      a = .7, g = 1: |a| >= alpha |g| -> 1x1 pivot at p."""
    from oracle.oracle import dense_ldlt_bk

    def block(a, g, h, b=0.1, c=0.1):
        return np.array([[a, g, 0.0], [g, b, h], [0.0, h, c]])

    r = dense_ldlt_bk(block(0.5, 1.0, 2.0), 3, 0.0)
    assert r["perm"][0] == 0 and r["bsize"][0] == 1
    r = dense_ldlt_bk(block(0.5, 1.0, 0.5), 3, 0.0)
    assert list(r["perm"][:2]) == [0, 1] and r["bsize"][0] == 2
    assert r["Dblock"][1, 0] == 1.0 and r["D"][0] == 0.5 and r["D"][1] == 0.1
    r = dense_ldlt_bk(block(0.7, 1.0, 0.5), 3, 0.0)
    assert r["perm"][0] == 0 and r["bsize"][0] == 1
    for M in (block(0.5, 1.0, 2.0), block(0.5, 1.0, 0.5), block(0.7, 1.0, 0.5)):
        assert _bk_residual(M, dense_ldlt_bk(M, 3, 0.0)) <= 1e-15


def test_bk_solve_against_lapack():
    """The solve with a pivoted factorisation (P b, forward with L, 1x1 and
    2x2 blocks of D, backward with L^T, P^T) agrees with LAPACK's solve of
    the original matrix on random indefinite systems, including blocks that
    force 2x2 pivots."""
    from oracle.oracle import dense_ldlt_bk, dense_solve_bk

    rng = np.random.default_rng(11)
    for n, nb in ((2, 2), (25, 8), (40, 40), (37, 5)):
        A = rng.standard_normal((n, n))
        A = A + A.T
        if n == 2:
            A = np.array([[0.0, 1.0], [1.0, 0.0]])
        fac = dense_ldlt_bk(A, nb, 0.0)
        assert np.all(fac["lift"] == 0.0)
        b = rng.standard_normal(n)
        x = dense_solve_bk(fac, b)
        ref = np.linalg.solve(A, b)
        cond = np.linalg.cond(A)
        assert np.abs(x - ref).max() <= 1e-13 * cond * max(1.0, np.abs(ref).max()), (n, nb)
        assert np.abs(A @ x - b).max() <= 1e-12 * np.abs(A).max() * max(1.0, np.abs(x).max())


def test_bk_front_partial_factorisation():
    """A front with k fully-summed columns: only they are interchanged (the
    contribution rows keep their order), P A P^T + diag(lift) equals
    [L1; L2] D [L1; L2]^T plus the Schur complement S in the trailing block,
    and S equals A22 - A21 A11^-1 A12 of the permuted matrix (LAPACK)."""
    from oracle.oracle import front_ldlt_bk

    rng = np.random.default_rng(21)
    for f, k, nb in ((20, 8, 4), (37, 32, 32), (30, 13, 8), (12, 0, 4), (9, 9, 3)):
        A = rng.standard_normal((f, f))
        A = A + A.T
        r = front_ldlt_bk(A, k, nb, 0.0)
        assert r["rc"] == 0
        P = r["perm"]
        assert np.array_equal(P[k:], np.arange(k, f)) and np.array_equal(np.sort(P[:k]), np.arange(k))
        Ap = A[np.ix_(P, P)] + np.diag(r["lift"])
        R = r["L"] @ r["Dblock"] @ r["L"].T
        R[k:, k:] += r["S"]
        assert np.abs(R - Ap).max() <= 1e-12 * np.abs(A).max()
        if 0 < k < f:
            S = Ap[k:, k:] - Ap[k:, :k] @ np.linalg.solve(Ap[:k, :k], Ap[:k, k:])
            assert np.abs(S - r["S"]).max() <= 1e-10 * max(1.0, np.abs(S).max()) * np.linalg.cond(Ap[:k, :k])


# ------------------------------------------------- ||K||_1 (lift floor)

def _norm1_cases():
    rng = np.random.default_rng(17)
    A = rng.standard_normal((7, 12)) * (rng.random((7, 12)) < 0.4)
    A[np.arange(7), rng.integers(12, size=7)] = rng.standard_normal(7)
    A[rng.integers(7, size=12), np.arange(12)] = rng.standard_normal(12)
    # moderate Theta and more entries per row than per column, so that the
    # largest column sum is a dual column made of mirrored entries
    theta = 10.0 ** rng.uniform(0, 1, 12)
    return A, theta


def test_norm1_reg_against_dense_max_column_sum():
    """The lift floor eps_piv ||K||_1 (Sec. 4.5) uses the maximum absolute
    column sum of the regularised matrix, K with rho and delta for the
    augmented system and A Theta~ A^T + delta I for the normal equations.
    Pinned against numpy's matrix 1-norm of the dense matrices; a planted
    mistake (a column sum of the stored lower part only, without the mirrored
    entries, or without the static terms) differs from the pin on these
    cases."""
    A, theta = _norm1_cases()
    m, n = A.shape
    rho, delta = 0.3, 0.7  # large enough for the static terms to move the norm
    K = K_dense(A, theta, rho, delta)
    o = Oracle(*lp_from_dense(A), form=FORM_AS)
    o.analyse(None)
    o.factorise(theta, rho, delta)
    got = o.stats()["normM1"]
    want = np.linalg.norm(K, 1)
    assert got == pytest.approx(want, rel=1e-14)
    # the pin is sensitive to the plausible mistakes
    assert abs(np.abs(np.tril(K)).sum(0).max() - want) > 1e-6 * want
    K0 = K_dense(A, theta, 0.0, 0.0)
    assert abs(np.linalg.norm(K0, 1) - want) > 1e-6 * want
    # normal equations
    tt = 1.0 / (1.0 / theta + rho)
    M = A @ np.diag(tt) @ A.T + delta * np.eye(m)
    on = Oracle(*lp_from_dense(A), form=FORM_NE)
    on.analyse(None)
    on.factorise(theta, rho, delta)
    assert on.stats()["normM1"] == pytest.approx(np.linalg.norm(M, 1), rel=1e-13)
    assert abs(np.abs(np.tril(M)).sum(0).max() - np.linalg.norm(M, 1)) > 1e-6 * np.linalg.norm(M, 1)


# ------------------------------------------------------ AS / NE chooser

def test_chooser_closed_form_identity():
    """A = I (m = n): K in the interleaved order (x_j, y_j) gives n separate
    2 x 2 supernodes (f = k = 2: 3 entries of L and 4 flops each), A A^T is
    diagonal (1 entry, 0 flops per supernode, one contributor pair per
    column), so cost_AS = 4n/P + 3*2*3n*8/B and cost_NE = 2n/P + 3*2*n*8/B and
    the normal equations win."""
    from oracle import choose_form

    n = 9
    lp = synth.lp.LP(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))
    perm = np.ravel(np.column_stack([np.arange(n), n + np.arange(n)])).astype(np.int32)
    P, B = 1.0e12, 6.7e12
    form, cas, cne, nne = choose_form(lp, perm, np.arange(n, dtype=np.int32), 0.0, 0.0, P, B)
    assert nne == n
    assert cas == pytest.approx(4 * n / P + 3 * 2 * 3 * n * 8 / B, rel=1e-14)
    assert cne == pytest.approx(2 * n / P + 3 * 2 * n * 8 / B, rel=1e-14)
    assert form == FORM_NE


def test_chooser_abandons_dense_normal_equations():
    """One dense column makes A A^T dense: its lower part (m(m+1)/2 entries)
    exceeds L of the augmented system in an order that eliminates the dense
    column last, so the normal equations are abandoned (cost -1) and the
    augmented system is kept."""
    from oracle import choose_form

    m, n = 30, 40
    rows = [np.array([j % m]) for j in range(n)] + [np.arange(m)]
    cp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    ri = np.concatenate(rows).astype(np.int32)
    lp = synth.lp.LP(m, n + 1, cp, ri, np.ones(len(ri)))
    # the sparse columns first, then the rows, the dense column last: no fill
    perm = np.concatenate([np.arange(n), n + 1 + np.arange(m), [n]]).astype(np.int32)
    form, cas, cne, nne = choose_form(lp, perm, np.arange(m, dtype=np.int32))
    assert nne == m * (m + 1) // 2
    assert form == FORM_AS and cne == -1.0 and cas > 0


# ---------------------------------------- multifrontal Bunch-Kaufman (Sec. 4.5)

def _bk_dense_factor(o, sym):
    """The multifrontal BK factor as dense matrices in the final order (the
    factorisation order composed with every front's interchanges): returns
    (q, L, Dblk) with K[perm][:, perm][q][:, q] + diag(lift) = L Dblk L^T."""
    N = o.N
    fac = o.factor()
    pv = o.pivots()
    q = np.arange(N)
    for s in range(len(sym["sn_parent"])):
        c0, c1 = sym["sn_start"][s], sym["sn_start"][s + 1]
        q[c0:c1] = c0 + pv["lperm"][c0:c1]
    qinv = np.empty(N, np.int64)
    qinv[q] = np.arange(N)
    L = np.zeros((N, N))
    for s in range(len(sym["sn_parent"])):
        c0, c1 = sym["sn_start"][s], sym["sn_start"][s + 1]
        k = c1 - c0
        R = sym["sn_rows"][sym["sn_rptr"][s]:sym["sn_rptr"][s + 1]]
        f = len(R)
        blk = fac["L"][fac["lptr"][s]:fac["lptr"][s + 1]].reshape(k, f).T
        rows = np.concatenate([np.arange(c0, c1), qinv[R[k:]]])
        L[np.ix_(rows, np.arange(c0, c1))] = blk
    Dblk = np.diag(fac["D"])
    for p in np.flatnonzero(pv["bsize"] == 2):
        Dblk[p + 1, p] = Dblk[p, p + 1] = pv["Doff"][p]
    return q, L, Dblk, fac, pv


def _bk_case(seed):
    """A (m x n): row i has one large entry a_i in its matched column
    cols[i] and random entries only in the other (unmatched) columns, so the
    pairs (y_i, x_cols[i]) are independent subtrees; the order is y_0,
    x_cols[0], y_1, x_cols[1], ..., then the unmatched columns.  Each pair is
    one front whose pivot block [[0, a_i], [a_i, -1/theta]] needs a 2x2 pivot
    when 1/theta < alpha |a_i|; eliminating it adds A_ir^T A_ir / (theta a_i^2)
    to the unmatched columns' block, which stays negative definite."""
    rng = np.random.default_rng(seed)
    m, n = 12 + 3 * seed, 30 + 5 * seed
    cols = rng.permutation(n)[:m]
    rest = np.setdiff1d(np.arange(n), cols)
    A = np.zeros((m, n))
    A[np.arange(m), cols] = rng.standard_normal(m) + 3.0
    R = rng.standard_normal((m, rest.size)) * (rng.random((m, rest.size)) < 0.25)
    R[rng.integers(m, size=rest.size), np.arange(rest.size)] += rng.standard_normal(rest.size)
    A[:, rest] = R
    perm = np.concatenate([np.ravel(np.column_stack([n + np.arange(m), cols])), rest]).astype(np.int32)
    return rng, A, perm


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_multifrontal_bk_without_regularisation(seed):
    """rho = delta = 0: K = [[-Theta^-1, A^T], [A, 0]] is not quasi-definite
    (zero dual diagonal).  The multifrontal factorisation with the
    Bunch-Kaufman variation of Sec. 4.5 must reproduce the permuted matrix
    (dense reconstruction to 1e-13 of the entries' scale), take 2x2 pivots
    (Theta of 1e2..1e4 makes -1/theta_j small against the off-diagonal a:
    |M_pp| < alpha gamma_p and |M_rr| = 0), give exactly n negative and m
    positive eigenvalues (Sylvester: A has full row rank), and solve K x = f
    like LAPACK."""
    rng, A, perm = _bk_case(seed)
    m, n = A.shape
    theta = 10.0 ** rng.uniform(2, 4, n)
    o = Oracle(*lp_from_dense(A), form=FORM_AS)
    # every dual row with its matched column as one 2-column front (no wider
    # amalgamation): the pivoting of Sec. 4.5 searches only a front's
    # fully-summed columns, so a front whose own block is singular at
    # rho = delta = 0 would need a lift (and grow) instead of a delayed pivot
    sym = o.analyse(perm, amalg_width=2, amalg_zero_frac=0.0)
    assert np.all(np.diff(sym["sn_start"])[:m] == 2)
    o.set_pivoting(True)
    assert o.factorise(theta, 0.0, 0.0) == 0
    q, L, Dblk, fac, pv = _bk_dense_factor(o, sym)
    K = K_dense(A, theta, 0.0, 0.0)
    Kq = K[np.ix_(sym["perm"], sym["perm"])][np.ix_(q, q)] + np.diag(fac["dynreg"])
    err = np.abs(L @ Dblk @ L.T - Kq).max()
    assert err <= 1e-13 * np.abs(L).max() ** 2 * np.abs(Dblk).max(), err
    assert np.count_nonzero(pv["bsize"] == 2) == m and np.all(fac["dynreg"] == 0.0)
    st = o.stats()
    assert st["nneg"] == n and st["npos"] == m
    b = rng.standard_normal(n + m)
    dx, dy, info = o.solve(b[:n], b[n:], omega_target=1e-14, max_steps=5)
    ref = np.linalg.solve(K, b)
    x = np.concatenate([dx, dy])
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    # the same matrix without pivoting needs a lift at every zero pivot
    o.set_pivoting(False)
    o.factorise(theta, 0.0, 0.0)
    assert o.stats()["ndyn"] > 0


def test_multifrontal_bk_equals_plain_solution_when_quasi_definite():
    """With rho, delta > 0 both pivoting modes factorise the same regularised
    K (possibly with different pivot orders): the refined solutions agree."""
    rng = np.random.default_rng(7)
    lp = synth.random_lp(40, 100, 4, seed=7)
    theta = synth.theta_loguniform(lp.n, 7, -3.0, 3.0)
    r7, r1 = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    out = []
    for bk in (False, True):
        o = Oracle.from_lp(lp)
        o.analyse(None)
        o.set_pivoting(bk)
        o.factorise(theta, 1e-6, 1e-6)
        dx, dy, info = o.solve(r7, r1, omega_target=1e-14, max_steps=10)
        out.append(np.concatenate([dx, dy]))
        assert o.stats()["nneg"] == lp.n and o.stats()["npos"] == lp.m
    assert np.abs(out[0] - out[1]).max() <= 1e-10 * np.abs(out[0]).max()
