"""CPU tests of the library's host side: the shared library loads and exports
every symbol include/ipm_mf.h declares, and the symbolic analysis (Sec.
4.2-4.3) is bit-exact with the oracle's by-definition symbolic analysis for
the same fill-reducing order.  No GPU call is made here."""
import ctypes as ct

import numpy as np
import pytest

import synth
from oracle import FORM_AS, Oracle


@pytest.fixture(scope="module")
def lib():
    from paper_2508_04370_gb300.build import build

    build()
    import paper_2508_04370_gb300 as pkg

    return pkg


def test_exports_every_declared_symbol(lib):
    names = lib.declared_symbols()
    assert len(names) >= 17
    so = lib.library()
    for name in names:
        assert hasattr(so, name), name


def _analyse(lib, lp, ordering, perm=None):
    ctx = lib.ipm_create()
    rc = lib.ipm_analyse(ctx, lp.m, lp.n, lp.colptr, lp.rowidx, lib.IPM_FORM_AUGMENTED, ordering, perm)
    return ctx, rc


def _compare_with_oracle(lib, ctx, lp):
    sym = lib.ipm_get_symbolic(ctx)
    o = Oracle.from_lp(lp, form=FORM_AS)
    s = o.analyse(sym["perm"], amalg_zero_frac=sym["amalg_zero_frac"])
    assert np.array_equal(s["perm"], sym["perm"])
    assert np.array_equal(s["parent"], sym["etree"])
    assert np.array_equal(s["colcount"], sym["colcount"])
    assert np.array_equal(s["sn_start"], sym["snode_ptr"])
    assert np.array_equal(s["sn_parent"], sym["sn_parent"])
    assert np.array_equal(s["sn_rptr"], sym["sn_rptr"])
    assert np.array_equal(s["sn_rows"], sym["sn_rows"])
    return sym


@pytest.mark.parametrize("ordering", [0, 1, 3])
def test_symbolic_bit_exact_random(lib, ordering):
    for seed in range(3):
        lp = synth.random_lp(60 + 20 * seed, 150 + 40 * seed, 4, seed=seed)
        ctx, rc = _analyse(lib, lp, ordering)
        assert rc == 0
        _compare_with_oracle(lib, ctx, lp)
        lib.ipm_destroy(ctx)


def test_symbolic_bit_exact_user_perm(lib):
    lp = synth.random_lp(50, 120, 4, seed=9)
    perm = synth.random_perm(lp.m + lp.n, 9)
    ctx, rc = _analyse(lib, lp, lib.IPM_ORD_USER, perm)
    assert rc == 0
    sym = lib.ipm_get_symbolic(ctx)
    # both sides compose the same user order with the same postorder
    o = Oracle.from_lp(lp)
    s = o.analyse(perm, amalg_zero_frac=sym["amalg_zero_frac"])
    assert np.array_equal(s["perm"], sym["perm"])
    _compare_with_oracle(lib, ctx, lp)
    lib.ipm_destroy(ctx)


def test_symbolic_bit_exact_config1_and_grid(lib):
    for lp, ordering in ((synth.by_name("random_300x800"), 0), (synth.grid_multicommodity(12, 2), 0),
                         (synth.grid_multicommodity(12, 2), 1)):
        ctx, rc = _analyse(lib, lp, ordering)
        assert rc == 0
        _compare_with_oracle(lib, ctx, lp)
        lib.ipm_destroy(ctx)


def test_amd_fill_beats_natural_order(lib):
    lp = synth.grid_multicommodity(16, 2)
    nnz = {}
    for ordering in (0, 1, 3):
        ctx, rc = _analyse(lib, lp, ordering)
        assert rc == 0
        rc, info = lib.ipm_get_info(ctx)
        nnz[ordering] = info.nnz_L
        lib.ipm_destroy(ctx)
    assert nnz[0] < nnz[3] / 3
    assert nnz[1] < nnz[3] / 3


def test_batch_analysis_is_block_diagonal_lp(lib):
    lps = [synth.random_lp(20 + 5 * i, 50 + 9 * i, 3, seed=40 + i) for i in range(4)]
    ctx = lib.ipm_create()
    rc = lib.ipm_analyse_batch(ctx, [lp.m for lp in lps], [lp.n for lp in lps],
                               np.concatenate([lp.colptr for lp in lps]),
                               np.concatenate([lp.rowidx for lp in lps]), lib.IPM_ORD_AMD)
    assert rc == 0
    # the same block-diagonal LP assembled here
    m = sum(lp.m for lp in lps)
    n = sum(lp.n for lp in lps)
    cols, rows = [], []
    ro = co = 0
    for lp in lps:
        for j in range(lp.n):
            for p in range(lp.colptr[j], lp.colptr[j + 1]):
                rows.append(ro + lp.rowidx[p])
                cols.append(co + j)
        ro += lp.m
        co += lp.n
    big = synth.lp._from_coo(m, n, rows, cols, np.ones(len(rows)), "blockdiag")
    ctx2, rc = _analyse(lib, big, lib.IPM_ORD_AMD)
    assert rc == 0
    a, b = lib.ipm_get_symbolic(ctx), lib.ipm_get_symbolic(ctx2)
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    _compare_with_oracle(lib, ctx, big)
    lib.ipm_destroy(ctx)
    lib.ipm_destroy(ctx2)


def test_rejects_malformed_input(lib):
    lp = synth.random_lp(10, 20, 3, seed=1)
    ctx = lib.ipm_create()
    bad = lp.rowidx.copy()
    bad[0] = lp.m
    assert lib.ipm_analyse(ctx, lp.m, lp.n, lp.colptr, bad) == lib.IPM_ERR_INVALID_ARG
    unsorted = lp.rowidx.copy()
    unsorted[0], unsorted[1] = unsorted[1], unsorted[0]
    assert lib.ipm_analyse(ctx, lp.m, lp.n, lp.colptr, unsorted) == lib.IPM_ERR_INVALID_ARG
    perm = np.zeros(lp.m + lp.n, np.int32)
    assert lib.ipm_analyse(ctx, lp.m, lp.n, lp.colptr, lp.rowidx, 1, lib.IPM_ORD_USER, perm) == lib.IPM_ERR_INVALID_ARG
    # calls before analysis
    assert lib.ipm_factorise(ctx, 0, 1e-8, 1e-8, stream=0) == lib.IPM_ERR_NOT_ANALYSED
    lib.ipm_destroy(ctx)
    opt = lib.ipm_default_options()
    opt.nb = 48
    with pytest.raises(RuntimeError):
        lib.ipm_create(opt)


def test_edge_patterns(lib):
    # no constraints, one empty column, a single column
    for m, n, cp, ri in ((0, 5, np.zeros(6, np.int64), np.zeros(0, np.int32)),
                         (3, 4, np.array([0, 1, 1, 3, 4]), np.array([0, 1, 2, 2])),
                         (1, 1, np.array([0, 1]), np.array([0]))):
        ctx = lib.ipm_create()
        rc = lib.ipm_analyse(ctx, m, n, cp, ri)
        assert rc == 0
        lp = synth.lp.LP(m, n, np.asarray(cp, np.int64), np.asarray(ri, np.int32), np.ones(len(ri)))
        _compare_with_oracle(lib, ctx, lp)
        lib.ipm_destroy(ctx)


def test_normal_equations_symbolic_bit_exact(lib):
    from oracle import FORM_NE

    for seed in range(3):
        lp = synth.random_lp(50 + 10 * seed, 140, 3, seed=60 + seed)
        ctx = lib.ipm_create()
        assert lib.ipm_analyse(ctx, lp.m, lp.n, lp.colptr, lp.rowidx, lib.IPM_FORM_NORMAL, lib.IPM_ORD_AMD) == 0
        sym = lib.ipm_get_symbolic(ctx)
        o = Oracle.from_lp(lp, form=FORM_NE)
        s = o.analyse(sym["perm"], amalg_zero_frac=sym["amalg_zero_frac"])
        for a, b in (("parent", "etree"), ("colcount", "colcount"), ("sn_start", "snode_ptr"),
                     ("sn_parent", "sn_parent"), ("sn_rows", "sn_rows")):
            assert np.array_equal(s[a], sym[b]), a
        lib.ipm_destroy(ctx)


def _chooser_against_oracle(lib, lp, ordering):
    """The library's AUTO choice and both modelled costs against the oracle's
    restatement of the chooser (oracle.choose_form), given the orders the
    library computes for each form (ordering parity is not pinned)."""
    from oracle import FORM_NE, choose_form

    syms = {}
    for form in (lib.IPM_FORM_AUGMENTED, lib.IPM_FORM_NORMAL):
        ctx = lib.ipm_create()
        rc = lib.ipm_analyse(ctx, lp.m, lp.n, lp.colptr, lp.rowidx, form, ordering)
        syms[form] = lib.ipm_get_symbolic(ctx) if rc == 0 else None
        lib.ipm_destroy(ctx)
    sa, sn = syms[lib.IPM_FORM_AUGMENTED], syms[lib.IPM_FORM_NORMAL]
    pn = sn["perm"] if sn is not None else np.arange(lp.m, dtype=np.int32)
    azn = sn["amalg_zero_frac"] if sn is not None else 0.1
    oform, ocas, ocne, onne = choose_form(lp, sa["perm"], pn, sa["amalg_zero_frac"], azn)
    ctx = lib.ipm_create()
    assert lib.ipm_analyse(ctx, lp.m, lp.n, lp.colptr, lp.rowidx, lib.IPM_FORM_AUTO, ordering) == 0
    rc, info = lib.ipm_get_info(ctx)
    lib.ipm_destroy(ctx)
    assert info.est_cost_as == pytest.approx(ocas, rel=1e-12)
    if ocne < 0:
        assert info.est_cost_ne == -1.0 and info.nnz_ne_seen > info.nnz_L
    else:
        assert info.est_cost_ne == pytest.approx(ocne, rel=1e-12)
        assert info.nnz_ne_seen == onne
    assert info.form == (lib.IPM_FORM_NORMAL if oform == FORM_NE else lib.IPM_FORM_AUGMENTED)
    return info


def test_form_chooser(lib):
    """Sec. 4.2: the library's choice between the augmented system and the
    normal equations equals the oracle's restatement of it: a dense column
    makes A A^T dense, so forming the normal equations is abandoned once they
    hold more entries than L of the augmented system; sparse LPs compare the
    two modelled costs; the reduced block-angular LP with dense linking rows
    (the family where the paper weighs the two forms)."""
    lp = synth.random_lp(400, 1000, 3, seed=5)
    cp = np.concatenate([lp.colptr, [lp.colptr[-1] + lp.m]]).astype(np.int64)
    ri = np.concatenate([lp.rowidx, np.arange(lp.m, dtype=np.int32)])
    dense = synth.lp.LP(lp.m, lp.n + 1, cp, ri, np.ones(len(ri)))
    info = _chooser_against_oracle(lib, dense, lib.IPM_ORD_AMD)
    assert info.form == lib.IPM_FORM_AUGMENTED and info.est_cost_ne == -1.0
    _chooser_against_oracle(lib, lp, lib.IPM_ORD_AMD)
    _chooser_against_oracle(lib, synth.random_lp(300, 800, 2, seed=6), lib.IPM_ORD_ND)
    _chooser_against_oracle(lib, synth.block_angular(blocks=12, bm=30, bn=80, density=0.05, linking=8, seed=4),
                            lib.IPM_ORD_AMD)


def test_analysis_checkpoint_roundtrip(tmp_path):
    """The analysis written by ipm_save_analysis and read back into a fresh
    context gives the same symbolic results and statistics; truncated or
    foreign files are rejected and leave the context unchanged."""
    import paper_2508_04370_gb300 as L

    for name, form, ordering in (("grid", L.IPM_FORM_AUGMENTED, L.IPM_ORD_ND),
                                 ("ne", L.IPM_FORM_NORMAL, L.IPM_ORD_AMD)):
        lp = synth.grid_multicommodity(12, 3) if name == "grid" else synth.random_lp(80, 200, 4, seed=3)
        a = L.ipm_create(L.ipm_default_options())
        assert L.ipm_save_analysis(a, str(tmp_path / "none.plan")) == L.IPM_ERR_NOT_ANALYSED
        assert L.ipm_analyse(a, lp.m, lp.n, lp.colptr, lp.rowidx, form, ordering) == 0
        path = tmp_path / f"{name}.plan"
        assert L.ipm_save_analysis(a, str(path)) == 0
        b = L.ipm_create(L.ipm_default_options())
        assert L.ipm_load_analysis(b, str(path)) == 0
        sa, sb = L.ipm_get_symbolic(a), L.ipm_get_symbolic(b)
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), k
        ia, ib = L.ipm_get_info(a)[1].as_dict(), L.ipm_get_info(b)[1].as_dict()
        for k in ("form", "nsuper", "nlevels", "max_front", "nnz_L", "flops_factor", "nnz_K_lower"):
            assert ia[k] == ib[k], k
        data = path.read_bytes()
        bad = tmp_path / "bad.plan"
        for blob in (data[: len(data) // 2], b"NOTAPLAN" + data[8:], data + b"x"):
            bad.write_bytes(blob)
            assert L.ipm_load_analysis(b, str(bad)) == L.IPM_ERR_INVALID_ARG
        assert L.ipm_get_info(b)[1].as_dict()["nsuper"] == ia["nsuper"]  # unchanged
        assert L.ipm_load_analysis(b, str(tmp_path / "missing.plan")) == L.IPM_ERR_INVALID_ARG
        L.ipm_destroy(a)
        L.ipm_destroy(b)


def test_launch_shapes_validation(lib):
    """ipm_set_launch_shapes accepts the autotuner's widths (or 0 for the
    default) and a non-negative level ratio, ipm_set_level_ctas 0 to 64 CTAs
    per SM, and both reject anything else without touching the GPU;
    ipm_autotune needs values first."""
    ctx = lib.ipm_create()
    assert lib.ipm_set_launch_shapes(ctx, [32, 128, 256], 1.0) == 0
    assert lib.ipm_set_launch_shapes(ctx, [0, 0, 0]) == 0
    assert lib.ipm_set_launch_shapes(ctx, None, 0.0) == 0
    assert lib.ipm_set_launch_shapes(ctx, [48, 64, 128]) == lib.IPM_ERR_INVALID_ARG
    assert lib.ipm_set_launch_shapes(ctx, [32, 64, 512]) == lib.IPM_ERR_INVALID_ARG
    assert lib.ipm_set_launch_shapes(ctx, None, float("nan")) == lib.IPM_ERR_INVALID_ARG
    for per_sm in (0, 1, 2, 64):
        assert lib.ipm_set_level_ctas(ctx, per_sm) == 0
    assert lib.ipm_set_level_ctas(ctx, -1) == lib.IPM_ERR_INVALID_ARG
    assert lib.ipm_set_level_ctas(ctx, 65) == lib.IPM_ERR_INVALID_ARG
    rc, info = lib.ipm_get_info(ctx)
    assert info.tune_level_ctas_per_sm == 0  # no device state yet
    assert lib.ipm_autotune(ctx, None, 1e-8, 1e-8, 1, stream=0) == lib.IPM_ERR_NOT_ANALYSED
    lib.ipm_destroy(ctx)


def test_nested_dissection_deterministic_with_bounded_fill(lib):
    """Nested dissection (the better of ratio-scored level cuts and
    multilevel separators, each refined by vertex Fiduccia-Mattheyses moves)
    is deterministic although its candidates run on worker threads, gives a
    permutation, and on a grid LP fills within 30% of AMD and far below the
    natural order."""
    lp = synth.grid_multicommodity(24, 3)
    perms, nnz = [], {}
    for ordering in (1, 1, 0, 3):
        ctx, rc = _analyse(lib, lp, ordering)
        assert rc == 0
        rc, info = lib.ipm_get_info(ctx)
        nnz[ordering] = info.nnz_L
        if ordering == 1:
            perms.append(lib.ipm_get_symbolic(ctx)["perm"])
        lib.ipm_destroy(ctx)
    assert np.array_equal(perms[0], perms[1])
    assert np.array_equal(np.sort(perms[0]), np.arange(lp.m + lp.n))
    assert nnz[1] < 1.3 * nnz[0]
    assert nnz[1] < nnz[3] / 3


def test_amalgamation_threshold_chosen_by_model(lib):
    """With amalg_zero_frac < 0 (the default) the analysis takes 0.1 or 0.2,
    whichever gives the smaller modelled factorisation time (front flops at
    1 TFLOP/s + 60 us per tree level): a grid LP, whose extra levels cost more
    than the extra flops, gets 0.2; a random LP with equal level counts and a
    staircase whose flops dominate keep 0.1.  The partition equals the one
    the explicit threshold gives, and the oracle reproduces it bit for bit
    with the reported value."""
    cases = ((synth.grid_multicommodity(24, 3), lib.IPM_ORD_ND, 0.2, True),
             (synth.random_lp(300, 800, 6, seed=1), lib.IPM_ORD_AMD, 0.1, True),
             (synth.staircase(periods=2, seed=1), lib.IPM_ORD_ND, 0.1, False))  # oracle analysis: ~10 s
    for lp, ordering, want, with_oracle in cases:
        syms = {}
        for az in (-1.0, want):
            opt = lib.ipm_default_options()
            opt.amalg_zero_frac = az
            ctx = lib.ipm_create(opt)
            assert lib.ipm_analyse(ctx, lp.m, lp.n, lp.colptr, lp.rowidx, lib.IPM_FORM_AUGMENTED, ordering) == 0
            rc, info = lib.ipm_get_info(ctx)
            assert info.amalg_zero_frac == want
            syms[az] = lib.ipm_get_symbolic(ctx)
            lib.ipm_destroy(ctx)
        for key in ("perm", "snode_ptr", "sn_parent", "sn_rptr", "sn_rows"):
            assert np.array_equal(syms[-1.0][key], syms[want][key]), key
        if with_oracle:
            o = Oracle.from_lp(lp, form=FORM_AS)
            s = o.analyse(syms[-1.0]["perm"], amalg_zero_frac=syms[-1.0]["amalg_zero_frac"])
            assert np.array_equal(s["sn_start"], syms[-1.0]["snode_ptr"])


def test_corrector_count_rule():
    """Sec. 4.7: (1 + k)(1 + f/2) solves should take about one factorisation;
    k is lifted to 1 and capped."""
    from paper_2508_04370_gb300.ipm import corrector_count

    # T_f = 10 solves, f = 2: (1 + k) 2 = 10 -> k = 4
    assert corrector_count(10.0, 1.0, 2, 6) == 4
    # f = 0: 1 + k = 10 -> k = 9, capped at 6
    assert corrector_count(10.0, 1.0, 0, 6) == 6
    # a factorisation cheaper than two solves: still one corrector
    assert corrector_count(1.0, 1.0, 1, 6) == 1
    assert corrector_count(1.0, 0.0, 1, 6) == 1
