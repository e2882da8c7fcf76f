/*
 * Reference oracle for the regularised multifrontal LDL^T of the interior
 * point method of Zanetti & Gondzio (arXiv 2508.04370).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is plain, slow, single-threaded C in
 * double precision.  It shares no code, header, table or helper with the
 * CUDA library, and only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  Every step follows the paper:
 *
 *   matrix to factorise ......... Eq. (augsys) and Eq. (normeq) with the
 *                                  regularisation of Eq. (regul_matrix), Sec. 3.2
 *   symbolic analysis ........... Sec. 4.1-4.3: elimination tree, column
 *                                  counts, supernodes and amalgamation, written
 *                                  from the textbook definitions
 *   numeric factorisation ....... Sec. 4.1 (multifrontal, children summed in a
 *                                  fixed order), Sec. 4.4 (blocked dense
 *                                  factorisation of each front: left-looking
 *                                  update of the block, factorisation kernel on
 *                                  the diagonal block, triangular solve for the
 *                                  rows below), Sec. 4.5 (static and dynamic
 *                                  regularisation, Prop. 3 sign bound)
 *   solve ....................... Sec. 4: forward with L, diagonal D, backward
 *                                  with L^T
 *   iterative refinement ........ Sec. 4.5, with the component-wise backward
 *                                  error of Arioli, Demmel and Duff
 *
 * Readings of the paper where it is silent or ambiguous (all of them are
 * options passed in, so tests can vary them):
 *   - static regularisation rho (primal, sign -1) and delta (dual, sign +1)
 *     is added to the pivot after it has been computed (Sec. 4.5); the
 *     matrix used for residuals contains rho and delta on its diagonal;
 *   - dynamic regularisation lifts a pivot to sign s_p * max(s_p*d, b) with
 *     b = max(eps_piv * ||K||_1, b2), b2 the Prop. 3 bound over the remaining
 *     fully-summed columns of the current pivot block that carry the same
 *     expected sign and a correctly signed diagonal; the same formula is used
 *     for both signs; 2x2 pivots and swaps are never used because the
 *     regularised matrix is quasi-definite (Sec. 4.6);
 *   - supernode amalgamation (Sec. 4.1 cites Ashcraft-Grimes without a rule):
 *     bottom-up in postorder, the child that ends right before the parent is
 *     merged into it when the merged width is at most amalg_width or when the
 *     explicit zeros of the merged supernode are at most amalg_zero_frac of
 *     its stored entries;
 *   - the small-denominator threshold of the backward error is
 *     tau_i = 1000 N eps (||M_i||_1-row * ||d||_inf + |f_i|).
 *
 * Pivoting for matrices that are not quasi-definite (Sec. 4.5, the variation
 * of Bunch-Kaufman pivoting), as a dense kernel of its own
 * (orc_dense_ldlt_bk); the multifrontal path above does not call it.
 * Readings: the search covers only the rows and columns of the current pivot
 * block that are not yet eliminated; gamma_r is the largest off-diagonal
 * magnitude of row/column r there; the pre-swap puts the remaining block
 * diagonal of largest magnitude (first on ties) at the pivot position before
 * each pivot is chosen; a lifted pivot keeps the sign of M_pp (+ for 0).
 *
 * Parity unpinned: the fill-reducing ordering itself (taken as an input).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FORM_AS 1
#define ORC_FORM_NE 2

#define ORC_OK 0
/* element count for an allocation that may be empty */
#define NZ(x) ((size_t)((x) > 0 ? (x) : 1))
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NONFINITE (-5)

typedef struct orc {
    /* problem: A is m x n, CSC, 0-based, sorted, no duplicates */
    int m, n, form, N;
    int64_t *Acp;
    int32_t *Ari;
    double *Ax;
    /* A in CSR for row-wise access (NE formation, residuals) */
    int64_t *Arp;
    int32_t *Aci;
    double *Arx;
    /* lower pattern (with diagonal) of the matrix M to factorise, original
       numbering, CSC: column j lists rows i >= j in increasing order */
    int64_t *Mcp;
    int32_t *Mri;
    double *Mx; /* values of M (AS: -1/theta on primal diagonal, 0 on dual
                   diagonal, A entries; NE: A Theta~ A^T) */
    /* symbolic on the factorisation order */
    int32_t *perm;  /* perm[new] = old */
    int32_t *iperm; /* iperm[old] = new */
    int32_t *parent;
    int64_t *colcount;
    int64_t *Lsp;   /* column structure S_j (rows > j), CSC */
    int32_t *Lsi;
    int nsuper;
    int32_t *sn_start; /* nsuper+1 */
    int32_t *sn_parent;
    int64_t *sn_rptr; /* nsuper+1 */
    int32_t *sn_rows; /* front row lists, sorted, first k are the columns */
    /* numeric */
    int64_t *sn_lptr; /* offsets into Lval, per supernode f*k column-major */
    double *Lval;
    double *D;
    double *dynreg;
    double *theta_t; /* NE: Theta~ = 1/(1/theta + rho) */
    double rho, delta, eps_piv, normM1;
    int nb;
    /* pivoting of Sec. 4.5 (Bunch-Kaufman variation, 1x1 and 2x2 pivots) per
       front instead of the 1x1 pivots with the Prop. 3 bound */
    int bk;
    int32_t *lperm;  /* per position c0 + t of a supernode: the local index moved to t */
    double *Doff;    /* D(p+1, p) of a 2x2 block starting at p, else 0 */
    int32_t *bsize;  /* 1 or 2 at a block's first position, 0 at the second */
    int ndyn, npos, nneg;
    int status;
    /* refinement record */
    int refine_steps;
    double omega_hist[64];
    double omega_K;
} orc;

/* ------------------------------------------------------------------ utils */

static void *xmalloc(size_t bytes) {
    void *p = malloc(bytes ? bytes : 1);
    return p;
}
static void *xcalloc(size_t count, size_t size) {
    void *p = calloc(count ? count : 1, size ? size : 1);
    return p;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void orc_destroy(orc *o);

static void free_symbolic(orc *o) {
    free(o->perm); free(o->iperm); free(o->parent); free(o->colcount);
    free(o->Lsp); free(o->Lsi); free(o->sn_start); free(o->sn_parent);
    free(o->sn_rptr); free(o->sn_rows); free(o->sn_lptr); free(o->Lval);
    free(o->D); free(o->dynreg);
    free(o->lperm); free(o->Doff); free(o->bsize);
    o->lperm = NULL; o->Doff = NULL; o->bsize = NULL;
    o->perm = o->iperm = o->parent = NULL; o->colcount = NULL;
    o->Lsp = NULL; o->Lsi = NULL; o->sn_start = o->sn_parent = NULL;
    o->sn_rptr = NULL; o->sn_rows = NULL; o->sn_lptr = NULL; o->Lval = NULL;
    o->D = o->dynreg = NULL;
}

/* --------------------------------------------------------- problem set-up */

/* Build CSR of A and the lower pattern of M.
 * AS (Eq. augsys): unknowns [x (n); y (m)]; M = [[-Theta^-1, A^T], [A, 0]];
 *   column j < n holds the diagonal and rows n+i for each a_ij.
 *   column n+i holds only its diagonal.
 * NE (Eq. normeq): M = A Theta A^T over the m rows of A; column i holds rows
 *   i' >= i that share a column of A with row i. */
orc *orc_create(int m, int n, const int64_t *colptr, const int32_t *rowidx,
                const double *vals, int form) {
    if (m < 0 || n < 0 || (form != ORC_FORM_AS && form != ORC_FORM_NE)) return NULL;
    orc *o = (orc *)xcalloc(1, sizeof(orc));
    o->m = m; o->n = n; o->form = form;
    o->N = (form == ORC_FORM_AS) ? n + m : m;
    int64_t nnz = colptr[n];
    o->Acp = (int64_t *)xmalloc(sizeof(int64_t) * (n + 1));
    o->Ari = (int32_t *)xmalloc(sizeof(int32_t) * NZ(nnz));
    o->Ax = (double *)xmalloc(sizeof(double) * NZ(nnz));
    memcpy(o->Acp, colptr, sizeof(int64_t) * (n + 1));
    memcpy(o->Ari, rowidx, sizeof(int32_t) * (size_t)nnz);
    if (vals) memcpy(o->Ax, vals, sizeof(double) * (size_t)nnz);
    else for (int64_t p = 0; p < nnz; p++) o->Ax[p] = 1.0;
    /* validate */
    for (int j = 0; j < n; j++) {
        if (colptr[j + 1] < colptr[j]) { orc_destroy(o); return NULL; }
        for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
            if (rowidx[p] < 0 || rowidx[p] >= m) { orc_destroy(o); return NULL; }
            if (p > colptr[j] && rowidx[p] <= rowidx[p - 1]) { orc_destroy(o); return NULL; }
        }
    }
    /* CSR */
    o->Arp = (int64_t *)xcalloc(m + 1, sizeof(int64_t));
    o->Aci = (int32_t *)xmalloc(sizeof(int32_t) * NZ(nnz));
    o->Arx = (double *)xmalloc(sizeof(double) * NZ(nnz));
    for (int64_t p = 0; p < nnz; p++) o->Arp[o->Ari[p] + 1]++;
    for (int i = 0; i < m; i++) o->Arp[i + 1] += o->Arp[i];
    int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * (m + 1));
    memcpy(fill, o->Arp, sizeof(int64_t) * (m + 1));
    for (int j = 0; j < n; j++)
        for (int64_t p = o->Acp[j]; p < o->Acp[j + 1]; p++) {
            int i = o->Ari[p];
            o->Aci[fill[i]] = j;
            o->Arx[fill[i]] = o->Ax[p];
            fill[i]++;
        }
    free(fill);
    /* lower pattern of M */
    int N = o->N;
    if (form == ORC_FORM_AS) {
        o->Mcp = (int64_t *)xmalloc(sizeof(int64_t) * (N + 1));
        o->Mri = (int32_t *)xmalloc(sizeof(int32_t) * (nnz + N));
        int64_t q = 0;
        for (int j = 0; j < n; j++) {
            o->Mcp[j] = q;
            o->Mri[q++] = j;
            for (int64_t p = o->Acp[j]; p < o->Acp[j + 1]; p++) o->Mri[q++] = n + o->Ari[p];
        }
        for (int i = 0; i < m; i++) { o->Mcp[n + i] = q; o->Mri[q++] = n + i; }
        o->Mcp[N] = q;
    } else {
        /* column i of the lower part of A A^T: union over columns j of A
           containing row i of the rows i' >= i of column j */
        int32_t *mark = (int32_t *)xmalloc(sizeof(int32_t) * NZ(m));
        for (int i = 0; i < m; i++) mark[i] = -1;
        int64_t cap = 16 + 2 * nnz, q = 0;
        int32_t *rows = (int32_t *)xmalloc(sizeof(int32_t) * cap);
        o->Mcp = (int64_t *)xmalloc(sizeof(int64_t) * (N + 1));
        for (int i = 0; i < m; i++) {
            o->Mcp[i] = q;
            int64_t start = q;
            if (q + 1 > cap) { cap *= 2; rows = (int32_t *)realloc(rows, sizeof(int32_t) * cap); }
            rows[q++] = i; mark[i] = i;
            for (int64_t p = o->Arp[i]; p < o->Arp[i + 1]; p++) {
                int j = o->Aci[p];
                for (int64_t r = o->Acp[j]; r < o->Acp[j + 1]; r++) {
                    int ii = o->Ari[r];
                    if (ii > i && mark[ii] != i) {
                        mark[ii] = i;
                        if (q + 1 > cap) { cap *= 2; rows = (int32_t *)realloc(rows, sizeof(int32_t) * cap); }
                        rows[q++] = ii;
                    }
                }
            }
            qsort(rows + start, (size_t)(q - start), sizeof(int32_t), cmp_i32);
        }
        o->Mcp[N] = q;
        o->Mri = rows;
        free(mark);
    }
    o->Mx = (double *)xcalloc((size_t)o->Mcp[N], sizeof(double));
    o->nb = 32;
    return o;
}

void orc_destroy(orc *o) {
    if (!o) return;
    free_symbolic(o);
    free(o->Acp); free(o->Ari); free(o->Ax); free(o->Arp); free(o->Aci); free(o->Arx);
    free(o->Mcp); free(o->Mri); free(o->Mx); free(o->theta_t);
    free(o);
}

int orc_N(const orc *o) { return o->N; }
int64_t orc_nnzM(const orc *o) { return o->Mcp[o->N]; }

/* ------------------------------------------------------------- symbolic */

/* Lower pattern of B = P M P^T: for every stored (i, j) of M's lower part the
 * entry lands at column min(iperm i, iperm j), row max(...).  Output columns
 * are sorted and include the diagonal. */
static void permuted_lower(const orc *o, const int32_t *iperm, int64_t **bp_out, int32_t **bi_out) {
    int N = o->N;
    int64_t nz = o->Mcp[N];
    int64_t *bp = (int64_t *)xcalloc(N + 1, sizeof(int64_t));
    int32_t *bi = (int32_t *)xmalloc(sizeof(int32_t) * NZ(nz));
    for (int j = 0; j < N; j++)
        for (int64_t p = o->Mcp[j]; p < o->Mcp[j + 1]; p++) {
            int a = iperm[o->Mri[p]], b = iperm[j];
            int c = a < b ? a : b;
            bp[c + 1]++;
        }
    for (int j = 0; j < N; j++) bp[j + 1] += bp[j];
    int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * (N + 1));
    memcpy(fill, bp, sizeof(int64_t) * (N + 1));
    for (int j = 0; j < N; j++)
        for (int64_t p = o->Mcp[j]; p < o->Mcp[j + 1]; p++) {
            int a = iperm[o->Mri[p]], b = iperm[j];
            int c = a < b ? a : b, r = a < b ? b : a;
            bi[fill[c]++] = r;
        }
    free(fill);
    for (int j = 0; j < N; j++) qsort(bi + bp[j], (size_t)(bp[j + 1] - bp[j]), sizeof(int32_t), cmp_i32);
    *bp_out = bp;
    *bi_out = bi;
}

/* Lower part of B = P M P^T in CSC (new numbering) together with, for each
 * stored entry, its position in M's value array. */
static void permuted_lower_src(const orc *o, int64_t **bp_out, int32_t **bi_out, int64_t **src_out) {
    int N = o->N;
    int64_t nz = o->Mcp[N];
    int64_t *bp = (int64_t *)xcalloc(N + 1, sizeof(int64_t));
    int32_t *bi = (int32_t *)xmalloc(sizeof(int32_t) * NZ(nz));
    int64_t *src = (int64_t *)xmalloc(sizeof(int64_t) * NZ(nz));
    for (int j = 0; j < N; j++)
        for (int64_t p = o->Mcp[j]; p < o->Mcp[j + 1]; p++) {
            int a = o->iperm[o->Mri[p]], b = o->iperm[j];
            bp[(a < b ? a : b) + 1]++;
        }
    for (int j = 0; j < N; j++) bp[j + 1] += bp[j];
    int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * (N + 1));
    memcpy(fill, bp, sizeof(int64_t) * (N + 1));
    for (int j = 0; j < N; j++)
        for (int64_t p = o->Mcp[j]; p < o->Mcp[j + 1]; p++) {
            int a = o->iperm[o->Mri[p]], b = o->iperm[j];
            int c = a < b ? a : b, r = a < b ? b : a;
            bi[fill[c]] = r;
            src[fill[c]] = p;
            fill[c]++;
        }
    free(fill);
    *bp_out = bp;
    *bi_out = bi;
    *src_out = src;
}

/* Symbolic elimination by definition.  With S_j the row structure of column j
 * of L strictly below the diagonal:
 *     S_j = { i > j : B_ij != 0 }  U  U_{k < j, j in S_k} ( S_k  n  {i > j} )
 *     parent(j) = min S_j  (-1 when S_j is empty)
 *     colcount(j) = |S_j| + 1
 * Every earlier column whose structure contains j contributes; no tree
 * shortcut is used. */
static int symbolic_by_definition(orc *o, const int32_t *perm) {
    int N = o->N;
    int32_t *iperm = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    for (int i = 0; i < N; i++) iperm[i] = -1;
    for (int i = 0; i < N; i++) {
        if (perm[i] < 0 || perm[i] >= N || iperm[perm[i]] != -1) { free(iperm); return ORC_ERR_ARG; }
        iperm[perm[i]] = i;
    }
    int64_t *bp; int32_t *bi;
    permuted_lower(o, iperm, &bp, &bi);
    /* lists of k with j in S_k, filled as columns are finished */
    int64_t *lcnt = (int64_t *)xcalloc(N + 1, sizeof(int64_t));
    int32_t **lists = (int32_t **)xcalloc(N ? N : 1, sizeof(int32_t *));
    int64_t *lcap = (int64_t *)xcalloc(N ? N : 1, sizeof(int64_t));
    int32_t *mark = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    for (int i = 0; i < N; i++) mark[i] = -1;
    int64_t cap = 1024, used = 0;
    int32_t *Si = (int32_t *)xmalloc(sizeof(int32_t) * cap);
    int64_t *Sp = (int64_t *)xcalloc(N + 1, sizeof(int64_t));
    int32_t *tmp = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    for (int j = 0; j < N; j++) {
        int cnt = 0;
        mark[j] = j;
        for (int64_t p = bp[j]; p < bp[j + 1]; p++) {
            int i = bi[p];
            if (i > j && mark[i] != j) { mark[i] = j; tmp[cnt++] = i; }
        }
        for (int64_t t = 0; t < lcnt[j]; t++) {
            int k = lists[j][t];
            for (int64_t p = Sp[k]; p < Sp[k + 1]; p++) {
                int i = Si[p];
                if (i > j && mark[i] != j) { mark[i] = j; tmp[cnt++] = i; }
            }
        }
        qsort(tmp, (size_t)cnt, sizeof(int32_t), cmp_i32);
        if (used + cnt > cap) {
            while (used + cnt > cap) cap *= 2;
            Si = (int32_t *)realloc(Si, sizeof(int32_t) * cap);
        }
        memcpy(Si + used, tmp, sizeof(int32_t) * cnt);
        used += cnt;
        Sp[j + 1] = used;
        for (int t = 0; t < cnt; t++) {
            int i = tmp[t];
            if (lcnt[i] + 1 > lcap[i]) {
                lcap[i] = lcap[i] ? 2 * lcap[i] : 4;
                lists[i] = (int32_t *)realloc(lists[i], sizeof(int32_t) * lcap[i]);
            }
            lists[i][lcnt[i]++] = j;
        }
        free(lists[j]);
        lists[j] = NULL;
    }
    free(lists); free(lcap); free(lcnt); free(mark); free(tmp); free(bp); free(bi);
    free(o->perm); free(o->iperm); free(o->parent); free(o->colcount); free(o->Lsp); free(o->Lsi);
    o->perm = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    memcpy(o->perm, perm, sizeof(int32_t) * N);
    o->iperm = iperm;
    o->Lsp = Sp;
    o->Lsi = Si;
    o->parent = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    o->colcount = (int64_t *)xmalloc(sizeof(int64_t) * NZ(N));
    for (int j = 0; j < N; j++) {
        o->parent[j] = (Sp[j + 1] > Sp[j]) ? Si[Sp[j]] : -1;
        o->colcount[j] = Sp[j + 1] - Sp[j] + 1;
    }
    return ORC_OK;
}

/* Postorder of the elimination forest: depth-first, children visited in
 * ascending index, roots in ascending index; post[t] is the t-th finished
 * node. */
static void postorder(int N, const int32_t *parent, int32_t *post) {
    int32_t *head = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    int32_t *next = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    int32_t *stack = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    for (int j = 0; j < N; j++) head[j] = -1;
    /* children lists in ascending order: insert in descending order at head */
    for (int j = N - 1; j >= 0; j--)
        if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = j; }
    int t = 0;
    for (int r = 0; r < N; r++) {
        if (parent[r] != -1) continue;
        int top = 0;
        stack[top++] = r;
        while (top > 0) {
            int v = stack[top - 1];
            int c = head[v];
            if (c == -1) {
                top--;
                post[t++] = v;
            } else {
                head[v] = next[c];
                stack[top++] = c;
            }
        }
    }
    free(head); free(next); free(stack);
}

/* Full analysis for a given fill-reducing order perm_in (perm[new] = old):
 * symbolic on perm_in, postorder of its tree, symbolic again on the composed
 * order, then fundamental supernodes and amalgamation. */
int orc_analyse(orc *o, const int32_t *perm_in, int nb, int amalg_width, double amalg_zero_frac) {
    int N = o->N;
    if (nb < 1) return ORC_ERR_ARG;
    free_symbolic(o);
    o->nb = nb;
    int32_t *p0 = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    if (perm_in) memcpy(p0, perm_in, sizeof(int32_t) * N);
    else for (int i = 0; i < N; i++) p0[i] = i;
    int rc = symbolic_by_definition(o, p0);
    if (rc) { free(p0); return rc; }
    int32_t *post = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    postorder(N, o->parent, post);
    int32_t *p1 = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    for (int t = 0; t < N; t++) p1[t] = p0[post[t]];
    free(post); free(p0);
    rc = symbolic_by_definition(o, p1);
    free(p1);
    if (rc) return rc;

    /* fundamental supernodes: column j+1 joins the supernode of j when
       parent(j) = j+1, j is the only child of j+1 and
       colcount(j) = colcount(j+1) + 1 */
    int32_t *nchild = (int32_t *)xcalloc(N ? N : 1, sizeof(int32_t));
    for (int j = 0; j < N; j++) if (o->parent[j] >= 0) nchild[o->parent[j]]++;
    int32_t *start = (int32_t *)xmalloc(sizeof(int32_t) * (N + 1));
    int ns = 0;
    for (int j = 0; j < N; j++) {
        int joins = (j > 0) && o->parent[j - 1] == j && nchild[j] == 1 &&
                    o->colcount[j - 1] == o->colcount[j] + 1;
        if (!joins) start[ns++] = j;
    }
    start[ns] = N;
    free(nchild);

    /* amalgamation, bottom-up: for supernode p (in increasing order) try to
       absorb the supernode c that ends right before p while c is a child of p */
    int64_t *true_nnz = (int64_t *)xmalloc(sizeof(int64_t) * NZ(ns));
    int64_t *fsz = (int64_t *)xmalloc(sizeof(int64_t) * NZ(ns));
    for (int s = 0; s < ns; s++) {
        int64_t z = 0;
        for (int j = start[s]; j < start[s + 1]; j++) z += o->colcount[j];
        true_nnz[s] = z;
        fsz[s] = o->colcount[start[s]]; /* fundamental: first column holds all rows */
    }
    /* a stack of finished supernodes: [st_start, st_end) ranges */
    int32_t *st_s = (int32_t *)xmalloc(sizeof(int32_t) * (ns + 1));
    int32_t *st_e = (int32_t *)xmalloc(sizeof(int32_t) * (ns + 1));
    int64_t *st_nnz = (int64_t *)xmalloc(sizeof(int64_t) * (ns + 1));
    int64_t *st_f = (int64_t *)xmalloc(sizeof(int64_t) * (ns + 1));
    int top = 0;
    for (int s = 0; s < ns; s++) {
        int ps = start[s], pe = start[s + 1];
        int64_t pn = true_nnz[s], pf = fsz[s];
        while (top > 0) {
            int cs = st_s[top - 1], ce = st_e[top - 1];
            if (ce != ps) break;
            int par = o->parent[ce - 1];
            if (!(par >= ps && par < pe)) break;
            int64_t kc = ce - cs, kp = pe - ps;
            int64_t k = kc + kp, f = kc + pf;
            int64_t total = k * f - k * (k - 1) / 2;
            int64_t zeros = total - (st_nnz[top - 1] + pn);
            int merge = (k <= amalg_width) || ((double)zeros <= amalg_zero_frac * (double)total);
            if (!merge) break;
            ps = cs; pn += st_nnz[top - 1]; pf = f;
            top--;
        }
        st_s[top] = ps; st_e[top] = pe; st_nnz[top] = pn; st_f[top] = pf;
        top++;
    }
    o->nsuper = top;
    o->sn_start = (int32_t *)xmalloc(sizeof(int32_t) * (top + 1));
    for (int s = 0; s < top; s++) o->sn_start[s] = st_s[s];
    o->sn_start[top] = N;
    free(st_s); free(st_e); free(st_nnz); free(st_f); free(true_nnz); free(fsz); free(start);

    /* supernode parents and front rows: R_s = U_{j in cols(s)} ({j} U S_j) */
    int32_t *col2sn = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    for (int s = 0; s < o->nsuper; s++)
        for (int j = o->sn_start[s]; j < o->sn_start[s + 1]; j++) col2sn[j] = s;
    o->sn_parent = (int32_t *)xmalloc(sizeof(int32_t) * (o->nsuper ? o->nsuper : 1));
    o->sn_rptr = (int64_t *)xcalloc(o->nsuper + 1, sizeof(int64_t));
    int32_t *mark = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    for (int i = 0; i < N; i++) mark[i] = -1;
    int64_t cap = 1024, used = 0;
    int32_t *rows = (int32_t *)xmalloc(sizeof(int32_t) * cap);
    int32_t *tmp = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    for (int s = 0; s < o->nsuper; s++) {
        int cnt = 0;
        for (int j = o->sn_start[s]; j < o->sn_start[s + 1]; j++) {
            if (mark[j] != s) { mark[j] = s; tmp[cnt++] = j; }
            for (int64_t p = o->Lsp[j]; p < o->Lsp[j + 1]; p++) {
                int i = o->Lsi[p];
                if (mark[i] != s) { mark[i] = s; tmp[cnt++] = i; }
            }
        }
        qsort(tmp, (size_t)cnt, sizeof(int32_t), cmp_i32);
        if (used + cnt > cap) { while (used + cnt > cap) cap *= 2; rows = (int32_t *)realloc(rows, sizeof(int32_t) * cap); }
        memcpy(rows + used, tmp, sizeof(int32_t) * cnt);
        used += cnt;
        o->sn_rptr[s + 1] = used;
        int last = o->sn_start[s + 1] - 1;
        o->sn_parent[s] = o->parent[last] >= 0 ? col2sn[o->parent[last]] : -1;
    }
    o->sn_rows = rows;
    free(mark); free(tmp); free(col2sn);

    /* factor storage */
    o->sn_lptr = (int64_t *)xcalloc(o->nsuper + 1, sizeof(int64_t));
    for (int s = 0; s < o->nsuper; s++) {
        int64_t k = o->sn_start[s + 1] - o->sn_start[s];
        int64_t f = o->sn_rptr[s + 1] - o->sn_rptr[s];
        o->sn_lptr[s + 1] = o->sn_lptr[s] + f * k;
    }
    o->Lval = (double *)xcalloc((size_t)o->sn_lptr[o->nsuper], sizeof(double));
    o->D = (double *)xcalloc(N ? N : 1, sizeof(double));
    o->dynreg = (double *)xcalloc(N ? N : 1, sizeof(double));
    o->lperm = (int32_t *)xcalloc(N ? N : 1, sizeof(int32_t));
    o->Doff = (double *)xcalloc(N ? N : 1, sizeof(double));
    o->bsize = (int32_t *)xcalloc(N ? N : 1, sizeof(int32_t));
    return ORC_OK;
}

int orc_nsuper(const orc *o) { return o->nsuper; }
int64_t orc_nrows_total(const orc *o) { return o->sn_rptr ? o->sn_rptr[o->nsuper] : 0; }
int64_t orc_nnzL_stored(const orc *o) { return o->sn_lptr ? o->sn_lptr[o->nsuper] : 0; }

void orc_get_symbolic(const orc *o, int32_t *perm, int32_t *parent, int64_t *colcount,
                      int32_t *sn_start, int32_t *sn_parent, int64_t *sn_rptr, int32_t *sn_rows) {
    int N = o->N;
    if (perm) memcpy(perm, o->perm, sizeof(int32_t) * N);
    if (parent) memcpy(parent, o->parent, sizeof(int32_t) * N);
    if (colcount) memcpy(colcount, o->colcount, sizeof(int64_t) * N);
    if (sn_start) memcpy(sn_start, o->sn_start, sizeof(int32_t) * (o->nsuper + 1));
    if (sn_parent) memcpy(sn_parent, o->sn_parent, sizeof(int32_t) * o->nsuper);
    if (sn_rptr) memcpy(sn_rptr, o->sn_rptr, sizeof(int64_t) * (o->nsuper + 1));
    if (sn_rows) memcpy(sn_rows, o->sn_rows, sizeof(int32_t) * o->sn_rptr[o->nsuper]);
}

/* ------------------------------------------------------ matrix values */

/* Values of M in original numbering (Eq. augsys / Eq. normeq):
 *   AS: M_jj = -1/theta_j (primal), M_{n+i,n+i} = 0 (dual), A entries;
 *       rho and delta are added at the pivot and in the residual matrix.
 *   NE: M = A Theta~ A^T with Theta~_j = 1/(1/theta_j + rho); delta is
 *       added at the pivot and in the residual matrix. */
static int set_values(orc *o, const double *theta) {
    int n = o->n, m = o->m, N = o->N;
    for (int j = 0; j < n; j++)
        if (!(theta[j] > 0.0) || !isfinite(theta[j])) return ORC_ERR_NONFINITE;
    if (o->form == ORC_FORM_AS) {
        for (int j = 0; j < n; j++) {
            int64_t q = o->Mcp[j];
            o->Mx[q] = -1.0 / theta[j];
            int64_t t = q + 1;
            for (int64_t p = o->Acp[j]; p < o->Acp[j + 1]; p++) o->Mx[t++] = o->Ax[p];
        }
        for (int i = 0; i < m; i++) o->Mx[o->Mcp[n + i]] = 0.0;
    } else {
        free(o->theta_t);
        o->theta_t = (double *)xmalloc(sizeof(double) * NZ(n));
        for (int j = 0; j < n; j++) o->theta_t[j] = 1.0 / (1.0 / theta[j] + o->rho);
        /* M_{i' i} = sum_j a_{i' j} theta~_j a_{i j}, j ascending over row i */
        double *acc = (double *)xcalloc(m ? m : 1, sizeof(double));
        for (int i = 0; i < N; i++) {
            for (int64_t q = o->Mcp[i]; q < o->Mcp[i + 1]; q++) acc[o->Mri[q]] = 0.0;
            for (int64_t p = o->Arp[i]; p < o->Arp[i + 1]; p++) {
                int j = o->Aci[p];
                double w = o->Arx[p] * o->theta_t[j];
                for (int64_t r = o->Acp[j]; r < o->Acp[j + 1]; r++) {
                    int ii = o->Ari[r];
                    if (ii >= i) acc[ii] += o->Ax[r] * w;
                }
            }
            for (int64_t q = o->Mcp[i]; q < o->Mcp[i + 1]; q++) o->Mx[q] = acc[o->Mri[q]];
        }
        free(acc);
    }
    return ORC_OK;
}

/* sign s_j of original unknown j: -1 for the primal block, +1 for the dual
 * block (Sec. 4.5); the normal equations are positive definite. */
static int sign_of(const orc *o, int j) {
    if (o->form == ORC_FORM_NE) return 1;
    return j < o->n ? -1 : 1;
}
static double static_of(const orc *o, int j) {
    if (o->form == ORC_FORM_NE) return o->delta;
    return j < o->n ? o->rho : o->delta;
}

/* ||M_reg||_1: maximum absolute column sum of the regularised matrix. */
static double norm1_reg(const orc *o) {
    int N = o->N;
    double *cs = (double *)xcalloc(N ? N : 1, sizeof(double));
    for (int j = 0; j < N; j++)
        for (int64_t p = o->Mcp[j]; p < o->Mcp[j + 1]; p++) {
            int i = o->Mri[p];
            double v = o->Mx[p];
            if (i == j) {
                v += sign_of(o, j) * static_of(o, j);
                cs[j] += fabs(v);
            } else {
                cs[j] += fabs(v);
                cs[i] += fabs(v);
            }
        }
    double mx = 0.0;
    for (int j = 0; j < N; j++) if (cs[j] > mx) mx = cs[j];
    free(cs);
    return mx;
}

/* ----------------------------------------------------- dense front work */

/* Blocked LDL^T of the k fully-summed columns of one dense front (Sec. 4.4),
 * followed by the Schur complement of the remaining f-k rows.
 *   F     f x f, column-major, lower triangle used; on exit the first k
 *         columns hold L (unit diagonal implied) and the trailing block holds
 *         the Schur complement F22 - L21 D L21^T.
 *   sgn   expected sign of each of the f rows (+1 / -1)
 *   sreg  static regularisation of each of the first k rows
 *   b1    eps_piv * ||M||_1
 * For each pivot block B_D of nb columns:
 *   (a) left-looking update of B_D and of the rows below it (B_P) by every
 *       earlier block:  F(i, j) -= sum_q L(i,q) d_q L(j,q)
 *   (b) factorisation kernel on B_D with static and dynamic regularisation
 *   (c) triangular solve for B_P:  B_P <- B_P L_BD^-T D^-1
 * Returns ORC_OK or ORC_ERR_NONFINITE. */
int orc_front_factor(int f, int k, int nb, double *F, const int *sgn, const double *sreg, double b1,
                     double *D, double *dynreg) {
    if (f < 0 || k < 0 || k > f || nb < 1) return ORC_ERR_ARG;
#define FE(i, j) F[(int64_t)(j) * f + (i)]
    int rc = ORC_OK;
    for (int b0 = 0; b0 < k; b0 += nb) {
        int b1c = b0 + nb < k ? b0 + nb : k;
        /* (a) updates from the blocks to the left */
        for (int a0 = 0; a0 < b0; a0 += nb) {
            int a1 = a0 + nb;
            for (int j = b0; j < b1c; j++)
                for (int i = j; i < f; i++) {
                    double s = 0.0;
                    for (int q = a0; q < a1; q++) s += FE(i, q) * D[q] * FE(j, q);
                    FE(i, j) -= s;
                }
        }
        /* (b) factorisation kernel on the diagonal block */
        for (int p = b0; p < b1c; p++) {
            double d = FE(p, p);
            int s = sgn[p];
            d += s * sreg[p];
            double b2 = 0.0;
            for (int j = p + 1; j < b1c; j++) {
                if (sgn[j] != s) continue;
                double fjj = FE(j, j);
                if (!(s * fjj > 0.0)) continue;
                double fjp = FE(j, p);
                double v = fjp * fjp / fabs(fjj);
                if (v > b2) b2 = v;
            }
            double bnd = b1 > b2 ? b1 : b2;
            double sd = s * d;
            double dn = s * (sd > bnd ? sd : bnd);
            if (!isfinite(d) || !isfinite(dn)) rc = ORC_ERR_NONFINITE;
            D[p] = dn;
            dynreg[p] = dn - d;
            for (int j = p + 1; j < b1c; j++) FE(j, p) = FE(j, p) / dn;
            for (int j = p + 1; j < b1c; j++)
                for (int i = j; i < b1c; i++) FE(i, j) -= FE(i, p) * dn * FE(j, p);
        }
        /* (c) rows below the diagonal block */
        for (int i = b1c; i < f; i++)
            for (int p = b0; p < b1c; p++) {
                double t = FE(i, p);
                for (int q = b0; q < p; q++) t -= FE(i, q) * D[q] * FE(p, q);
                FE(i, p) = t / D[p];
            }
    }
    /* Schur complement of the front */
    for (int j = k; j < f; j++)
        for (int i = j; i < f; i++) {
            double s = 0.0;
            for (int q = 0; q < k; q++) s += FE(i, q) * D[q] * FE(j, q);
            FE(i, j) -= s;
        }
#undef FE
    return rc;
}

/* ------------------------------------------------------ multifrontal */

int orc_front_ldlt_bk(int n, int k, int nb, double *A, double b1, double alpha, int32_t *perm, double *D,
                      double *Doff, int32_t *bsize, double *lift);

/* Select the pivoting of a front: 0 = 1x1 pivots with static and dynamic
 * regularisation (Sec. 4.4-4.5, Prop. 3); 1 = the Bunch-Kaufman variation of
 * Sec. 4.5 (1x1 and 2x2 pivots chosen within each pivot block, pre-swap,
 * lifting) through orc_front_ldlt_bk, for matrices that are not
 * quasi-definite.  Reading: the static terms s_p sigma_p enter the diagonal
 * of the fully-summed columns before the front is factorised (the matrix
 * factorised is K with rho and delta, as in mode 0); the interchanges stay
 * among the fully-summed columns, so the symbolic structure is unchanged. */
void orc_set_pivoting(orc *o, int bk) { o->bk = bk ? 1 : 0; }

int orc_factorise(orc *o, const double *theta, double rho, double delta, double eps_piv) {
    if (!o->sn_start) return ORC_ERR_ARG;
    o->rho = rho; o->delta = delta; o->eps_piv = eps_piv;
    int rc = set_values(o, theta);
    if (rc) { o->status = rc; return rc; }
    int N = o->N, ns = o->nsuper;
    o->normM1 = norm1_reg(o);
    double b1 = eps_piv * o->normM1;
    /* children of each supernode in ascending order */
    int32_t *chead = (int32_t *)xmalloc(sizeof(int32_t) * NZ(ns));
    int32_t *cnext = (int32_t *)xmalloc(sizeof(int32_t) * NZ(ns));
    for (int s = 0; s < ns; s++) chead[s] = -1;
    for (int s = ns - 1; s >= 0; s--)
        if (o->sn_parent[s] >= 0) { cnext[s] = chead[o->sn_parent[s]]; chead[o->sn_parent[s]] = s; }
    int64_t *bp; int32_t *bi; int64_t *bsrc;
    permuted_lower_src(o, &bp, &bi, &bsrc);
    double **cb = (double **)xcalloc(ns ? ns : 1, sizeof(double *));
    int32_t *loc = (int32_t *)xmalloc(sizeof(int32_t) * NZ(N));
    int status = ORC_OK;
    o->ndyn = o->npos = o->nneg = 0;
    for (int s = 0; s < ns; s++) {
        int c0 = o->sn_start[s], k = o->sn_start[s + 1] - c0;
        int64_t r0 = o->sn_rptr[s];
        int f = (int)(o->sn_rptr[s + 1] - r0);
        const int32_t *R = o->sn_rows + r0;
        for (int t = 0; t < f; t++) loc[R[t]] = t;
        double *F = (double *)xcalloc((size_t)f * f, sizeof(double));
        /* original entries of the columns of this supernode: column j of the
           lower part of B = P M P^T, i >= j */
        for (int jj = 0; jj < k; jj++) {
            int jn = c0 + jj;
            for (int64_t p = bp[jn]; p < bp[jn + 1]; p++)
                F[(int64_t)jj * f + loc[bi[p]]] += o->Mx[bsrc[p]];
        }
        /* children contribution blocks, ascending child index */
        for (int c = chead[s]; c != -1; c = cnext[c]) {
            int kc = o->sn_start[c + 1] - o->sn_start[c];
            int64_t rc0 = o->sn_rptr[c];
            int fc = (int)(o->sn_rptr[c + 1] - rc0);
            int cc = fc - kc;
            const int32_t *Rc = o->sn_rows + rc0 + kc;
            for (int jj = 0; jj < cc; jj++)
                for (int ii = jj; ii < cc; ii++)
                    F[(int64_t)loc[Rc[jj]] * f + loc[Rc[ii]]] += cb[c][(int64_t)jj * cc + ii];
            free(cb[c]);
            cb[c] = NULL;
        }
        /* dense factorisation */
        int *sg = (int *)xmalloc(sizeof(int) * NZ(f));
        double *sr = (double *)xmalloc(sizeof(double) * NZ(f));
        for (int t = 0; t < f; t++) {
            sg[t] = sign_of(o, o->perm[R[t]]);
            sr[t] = static_of(o, o->perm[R[t]]);
        }
        int frc;
        if (!o->bk) {
            frc = orc_front_factor(f, k, o->nb, F, sg, sr, b1, o->D + c0, o->dynreg + c0);
        } else {
            /* static terms on the fully-summed diagonal, both triangles for the
               symmetric interchanges, then the pivoted partial factorisation */
            for (int t = 0; t < k; t++) F[(int64_t)t * f + t] += sg[t] * sr[t];
            for (int j = 0; j < f; j++)
                for (int i = j + 1; i < f; i++) F[(int64_t)i * f + j] = F[(int64_t)j * f + i];
            int32_t *lp = (int32_t *)xmalloc(sizeof(int32_t) * NZ(f));
            double *Df = (double *)xmalloc(sizeof(double) * NZ(f));
            double *Of = (double *)xmalloc(sizeof(double) * NZ(f));
            int32_t *Bf = (int32_t *)xmalloc(sizeof(int32_t) * NZ(f));
            double *lf = (double *)xmalloc(sizeof(double) * NZ(f));
            frc = orc_front_ldlt_bk(f, k, o->nb, F, b1, 1.0 / 8.0 + sqrt(17.0) / 8.0, lp, Df, Of, Bf, lf);
            for (int t = 0; t < k; t++) {
                o->lperm[c0 + t] = lp[t];
                o->D[c0 + t] = Df[t];
                o->Doff[c0 + t] = Of[t];
                o->bsize[c0 + t] = Bf[t];
                o->dynreg[c0 + t] = lf[t];
            }
            free(lp); free(Df); free(Of); free(Bf); free(lf);
        }
        if (frc && !status) status = frc;
        free(sg); free(sr);
        /* store L and keep the contribution block for the parent */
        double *L = o->Lval + o->sn_lptr[s];
        for (int jj = 0; jj < k; jj++)
            for (int ii = 0; ii < f; ii++)
                L[(int64_t)jj * f + ii] = (ii > jj) ? F[(int64_t)jj * f + ii] : (ii == jj ? 1.0 : 0.0);
        int cc = f - k;
        if (cc > 0) {
            cb[s] = (double *)xmalloc(sizeof(double) * (size_t)cc * cc);
            for (int jj = 0; jj < cc; jj++)
                for (int ii = 0; ii < cc; ii++)
                    cb[s][(int64_t)jj * cc + ii] = F[(int64_t)(k + jj) * f + (k + ii)];
        }
        free(F);
    }
    for (int s = 0; s < ns; s++) free(cb[s]);
    free(cb); free(loc); free(chead); free(cnext); free(bp); free(bi); free(bsrc);
    for (int j = 0; j < N; j++) {
        if (o->dynreg[j] != 0.0) o->ndyn++;
        if (o->bk && o->bsize[j] == 2) {
            /* a 2x2 block: one positive and one negative eigenvalue when its
               determinant is negative, else both of the sign of its trace */
            const double det = o->D[j] * o->D[j + 1] - o->Doff[j] * o->Doff[j];
            if (det < 0) { o->npos++; o->nneg++; }
            else if (det > 0) { if (o->D[j] + o->D[j + 1] > 0) o->npos += 2; else o->nneg += 2; }
            if (o->dynreg[j + 1] != 0.0) o->ndyn++;
            j++;
            continue;
        }
        if (o->D[j] > 0) o->npos++;
        else if (o->D[j] < 0) o->nneg++;
    }
    o->status = status;
    return status;
}

void orc_get_factor(const orc *o, double *Lval, double *D, double *dynreg, int64_t *sn_lptr) {
    if (Lval) memcpy(Lval, o->Lval, sizeof(double) * o->sn_lptr[o->nsuper]);
    if (D) memcpy(D, o->D, sizeof(double) * o->N);
    if (dynreg) memcpy(dynreg, o->dynreg, sizeof(double) * o->N);
    if (sn_lptr) memcpy(sn_lptr, o->sn_lptr, sizeof(int64_t) * (o->nsuper + 1));
}

void orc_get_pivots(const orc *o, int32_t *lperm, double *Doff, int32_t *bsize) {
    if (lperm) memcpy(lperm, o->lperm, sizeof(int32_t) * o->N);
    if (Doff) memcpy(Doff, o->Doff, sizeof(double) * o->N);
    if (bsize) memcpy(bsize, o->bsize, sizeof(int32_t) * o->N);
}

void orc_get_stats(const orc *o, int *ndyn, int *npos, int *nneg, double *normM1) {
    if (ndyn) *ndyn = o->ndyn;
    if (npos) *npos = o->npos;
    if (nneg) *nneg = o->nneg;
    if (normM1) *normM1 = o->normM1;
}

/* ------------------------------------------------------------- solves */

/* x <- (P^T L D L^T P)^-1 x in original numbering (Sec. 4: forward with L,
 * diagonal D, backward with L^T). */
static void ldlt_solve(const orc *o, double *x) {
    int N = o->N;
    double *y = (double *)xmalloc(sizeof(double) * NZ(N));
    for (int i = 0; i < N; i++) y[i] = x[o->perm[i]];
    double *tmp = (double *)xmalloc(sizeof(double) * NZ(N));
    for (int s = 0; s < o->nsuper; s++) {
        int c0 = o->sn_start[s], k = o->sn_start[s + 1] - c0;
        int f = (int)(o->sn_rptr[s + 1] - o->sn_rptr[s]);
        const int32_t *R = o->sn_rows + o->sn_rptr[s];
        const double *L = o->Lval + o->sn_lptr[s];
        if (o->bk) {
            /* the front's interchanges: position t holds local index lperm[t] */
            for (int t = 0; t < k; t++) tmp[t] = y[c0 + o->lperm[c0 + t]];
            for (int t = 0; t < k; t++) y[c0 + t] = tmp[t];
        }
        for (int jj = 0; jj < k; jj++) {
            double yj = y[c0 + jj];
            for (int ii = jj + 1; ii < f; ii++) y[R[ii]] -= L[(int64_t)jj * f + ii] * yj;
        }
    }
    for (int i = 0; i < N; i++) {
        if (o->bk && o->bsize[i] == 2) {
            /* 2x2 block of D: the inverse of [e11 e21; e21 e22] */
            const double e11 = o->D[i], e21 = o->Doff[i], e22 = o->D[i + 1];
            const double det = e11 * e22 - e21 * e21;
            const double y0 = y[i], y1 = y[i + 1];
            y[i] = (e22 * y0 - e21 * y1) / det;
            y[i + 1] = (e11 * y1 - e21 * y0) / det;
            i++;
            continue;
        }
        y[i] /= o->D[i];
    }
    for (int s = o->nsuper - 1; s >= 0; s--) {
        int c0 = o->sn_start[s], k = o->sn_start[s + 1] - c0;
        int f = (int)(o->sn_rptr[s + 1] - o->sn_rptr[s]);
        const int32_t *R = o->sn_rows + o->sn_rptr[s];
        const double *L = o->Lval + o->sn_lptr[s];
        for (int jj = k - 1; jj >= 0; jj--) {
            double t = y[c0 + jj];
            for (int ii = jj + 1; ii < f; ii++) t -= L[(int64_t)jj * f + ii] * y[R[ii]];
            y[c0 + jj] = t;
        }
        if (o->bk) {
            for (int t = 0; t < k; t++) tmp[t] = y[c0 + t];
            for (int t = 0; t < k; t++) y[c0 + o->lperm[c0 + t]] = tmp[t];
        }
    }
    for (int i = 0; i < N; i++) x[o->perm[i]] = y[i];
    free(y);
    free(tmp);
}

/* ---------------------------------------------------- residual, error */

/* Products with the regularised augmented matrix K = [[-(Theta^-1+rho I), A^T],
 * [A, delta I]] (Eq. regul_matrix), original numbering.
 *   r  = f - K d            (when r != NULL)
 *   ad = |K| |d|            (when ad != NULL)
 *   ae = |K| e              (when ae != NULL) */
static void k_products(const orc *o, const double *theta, const double *d, const double *f,
                       double *r, double *ad, double *ae) {
    int n = o->n, m = o->m;
    for (int j = 0; j < n; j++) {
        double dg = -(1.0 / theta[j] + o->rho);
        double s = dg * d[j], sa = fabs(dg) * fabs(d[j]), se = fabs(dg);
        for (int64_t p = o->Acp[j]; p < o->Acp[j + 1]; p++) {
            double a = o->Ax[p];
            double v = d[n + o->Ari[p]];
            s += a * v; sa += fabs(a) * fabs(v); se += fabs(a);
        }
        if (r) r[j] = f[j] - s;
        if (ad) ad[j] = sa;
        if (ae) ae[j] = se;
    }
    for (int i = 0; i < m; i++) {
        double s = o->delta * d[n + i], sa = o->delta * fabs(d[n + i]), se = o->delta;
        for (int64_t p = o->Arp[i]; p < o->Arp[i + 1]; p++) {
            double a = o->Arx[p];
            double v = d[o->Aci[p]];
            s += a * v; sa += fabs(a) * fabs(v); se += fabs(a);
        }
        if (r) r[n + i] = f[n + i] - s;
        if (ad) ad[n + i] = sa;
        if (ae) ae[n + i] = se;
    }
}

/* Same products with the regularised normal-equations matrix
 * A Theta~ A^T + delta I (explicitly formed lower part Mx). */
static void ne_products(const orc *o, const double *d, const double *f, double *r, double *ad, double *ae) {
    int N = o->N;
    double *s = (double *)xcalloc(N ? N : 1, sizeof(double));
    double *sa = (double *)xcalloc(N ? N : 1, sizeof(double));
    double *se = (double *)xcalloc(N ? N : 1, sizeof(double));
    for (int j = 0; j < N; j++)
        for (int64_t p = o->Mcp[j]; p < o->Mcp[j + 1]; p++) {
            int i = o->Mri[p];
            double v = o->Mx[p];
            if (i == j) {
                v += o->delta;
                s[j] += v * d[j]; sa[j] += fabs(v) * fabs(d[j]); se[j] += fabs(v);
            } else {
                s[i] += v * d[j]; sa[i] += fabs(v) * fabs(d[j]); se[i] += fabs(v);
                s[j] += v * d[i]; sa[j] += fabs(v) * fabs(d[i]); se[j] += fabs(v);
            }
        }
    for (int i = 0; i < N; i++) {
        if (r) r[i] = f[i] - s[i];
        if (ad) ad[i] = sa[i];
        if (ae) ae[i] = se[i];
    }
    free(s); free(sa); free(se);
}

/* Component-wise backward error of Arioli, Demmel and Duff (Sec. 4.5):
 *   omega = max_i |f - M d|_i / (|M||d| + |f|)_i,
 * where a denominator not larger than tau_i = 1000 N eps (||M_i||_1 ||d||_inf
 * + |f_i|) is replaced by (|M||d| + ||d||_inf |M| e)_i.  A component whose
 * residual or denominator is NaN makes omega infinite. */
double orc_backward_error(int N, const double *r, const double *ad, const double *ae,
                          const double *f, const double *d) {
    double dinf = 0.0;
    for (int i = 0; i < N; i++) if (fabs(d[i]) > dinf) dinf = fabs(d[i]);
    const double eps = 2.220446049250313e-16;
    double w = 0.0;
    for (int i = 0; i < N; i++) {
        double den = ad[i] + fabs(f[i]);
        double tau = 1000.0 * N * eps * (ae[i] * dinf + fabs(f[i]));
        if (den <= tau) den = ad[i] + dinf * ae[i];
        double num = fabs(r[i]);
        double wi;
        if (isnan(num) || isnan(den)) wi = INFINITY; /* a non-finite residual is no backward error */
        else if (den > 0.0) wi = num / den;
        else wi = (num > 0.0) ? INFINITY : 0.0;
        if (wi > w || isnan(wi)) w = wi;
    }
    return w;
}

/* Iterative refinement (Sec. 4.5): d = M^-1 f, then repeat
 * r = f - M d, d <- d + M^-1 r, until omega <= target, max_steps
 * corrections were made, or omega fails to halve; the iterate with the
 * smallest omega is returned.
 * AS: M is K; f = [r7; r1]; out = [dx; dy].
 * NE: M is A Theta~ A^T + delta I; f = r8 = r1 + A Theta~ r7; dx recovered as
 *     Theta~ (A^T dy - r7).  The returned omega_K is measured on K. */
int orc_solve(orc *o, const double *theta, const double *r7, const double *r1, double *dx, double *dy,
              double omega_target, int max_steps) {
    int n = o->n, m = o->m, N = o->N;
    double *f = (double *)xmalloc(sizeof(double) * NZ(N));
    if (o->form == ORC_FORM_AS) {
        memcpy(f, r7, sizeof(double) * n);
        memcpy(f + n, r1, sizeof(double) * m);
    } else {
        for (int i = 0; i < m; i++) {
            double s = r1[i];
            for (int64_t p = o->Arp[i]; p < o->Arp[i + 1]; p++) {
                int j = o->Aci[p];
                s += o->Arx[p] * (o->theta_t[j] * r7[j]);
            }
            f[i] = s;
        }
    }
    double *d = (double *)xmalloc(sizeof(double) * NZ(N));
    double *best = (double *)xmalloc(sizeof(double) * NZ(N));
    double *r = (double *)xmalloc(sizeof(double) * NZ(N));
    double *ad = (double *)xmalloc(sizeof(double) * NZ(N));
    double *ae = (double *)xmalloc(sizeof(double) * NZ(N));
    memcpy(d, f, sizeof(double) * N);
    ldlt_solve(o, d);
    if (o->form == ORC_FORM_AS) k_products(o, theta, d, f, r, ad, ae);
    else ne_products(o, d, f, r, ad, ae);
    double w = orc_backward_error(N, r, ad, ae, f, d);
    double wbest = w;
    memcpy(best, d, sizeof(double) * N);
    int steps = 0;
    o->omega_hist[0] = w;
    while (wbest > omega_target && steps < max_steps && steps < 63) {
        ldlt_solve(o, r);
        for (int i = 0; i < N; i++) d[i] += r[i];
        steps++;
        if (o->form == ORC_FORM_AS) k_products(o, theta, d, f, r, ad, ae);
        else ne_products(o, d, f, r, ad, ae);
        w = orc_backward_error(N, r, ad, ae, f, d);
        o->omega_hist[steps] = w;
        int halved = w <= 0.5 * wbest;
        if (w < wbest) { wbest = w; memcpy(best, d, sizeof(double) * N); }
        if (!halved) break;
    }
    o->refine_steps = steps;
    if (o->form == ORC_FORM_AS) {
        memcpy(dx, best, sizeof(double) * n);
        memcpy(dy, best + n, sizeof(double) * m);
    } else {
        memcpy(dy, best, sizeof(double) * m);
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int64_t p = o->Acp[j]; p < o->Acp[j + 1]; p++) s += o->Ax[p] * dy[o->Ari[p]];
            dx[j] = o->theta_t[j] * (s - r7[j]);
        }
    }
    /* omega on K for (dx, dy) */
    {
        int NK = n + m;
        double *fk = (double *)xmalloc(sizeof(double) * NZ(NK));
        double *dk = (double *)xmalloc(sizeof(double) * NZ(NK));
        double *rk = (double *)xmalloc(sizeof(double) * NZ(NK));
        double *adk = (double *)xmalloc(sizeof(double) * NZ(NK));
        double *aek = (double *)xmalloc(sizeof(double) * NZ(NK));
        memcpy(fk, r7, sizeof(double) * n); memcpy(fk + n, r1, sizeof(double) * m);
        memcpy(dk, dx, sizeof(double) * n); memcpy(dk + n, dy, sizeof(double) * m);
        k_products(o, theta, dk, fk, rk, adk, aek);
        o->omega_K = orc_backward_error(NK, rk, adk, aek, fk, dk);
        free(fk); free(dk); free(rk); free(adk); free(aek);
    }
    free(f); free(d); free(best); free(r); free(ad); free(ae);
    return ORC_OK;
}

int orc_refine_record(const orc *o, double *hist, double *omega_K) {
    if (hist) for (int i = 0; i <= o->refine_steps; i++) hist[i] = o->omega_hist[i];
    if (omega_K) *omega_K = o->omega_K;
    return o->refine_steps;
}

/* Backward error of a given (dx, dy) for K (exposed for tests). */
double orc_omega_K(orc *o, const double *theta, double rho, double delta,
                   const double *r7, const double *r1, const double *dx, const double *dy) {
    int n = o->n, m = o->m, NK = n + m;
    double save_r = o->rho, save_d = o->delta;
    o->rho = rho; o->delta = delta;
    double *fk = (double *)xmalloc(sizeof(double) * NZ(NK));
    double *dk = (double *)xmalloc(sizeof(double) * NZ(NK));
    double *rk = (double *)xmalloc(sizeof(double) * NZ(NK));
    double *adk = (double *)xmalloc(sizeof(double) * NZ(NK));
    double *aek = (double *)xmalloc(sizeof(double) * NZ(NK));
    memcpy(fk, r7, sizeof(double) * n); memcpy(fk + n, r1, sizeof(double) * m);
    memcpy(dk, dx, sizeof(double) * n); memcpy(dk + n, dy, sizeof(double) * m);
    k_products(o, theta, dk, fk, rk, adk, aek);
    double w = orc_backward_error(NK, rk, adk, aek, fk, dk);
    free(fk); free(dk); free(rk); free(adk); free(aek);
    o->rho = save_r; o->delta = save_d;
    return w;
}

/* Values of M in original numbering (lower part, CSC over Mcp/Mri). */
void orc_get_matrix(const orc *o, int64_t *Mcp, int32_t *Mri, double *Mx) {
    if (Mcp) memcpy(Mcp, o->Mcp, sizeof(int64_t) * (o->N + 1));
    if (Mri) memcpy(Mri, o->Mri, sizeof(int32_t) * o->Mcp[o->N]);
    if (Mx) memcpy(Mx, o->Mx, sizeof(double) * o->Mcp[o->N]);
}

/* ------------------------------------------- Bunch-Kaufman pivoting (dense) */

/* Symmetric interchange of rows/columns a and b of the n x n matrix A
 * (column-major, both triangles kept) and of perm. */
static void bk_swap(int n, double *A, int32_t *perm, int a, int b) {
    if (a == b) return;
#define AE(i, j) A[(int64_t)(j) * n + (i)]
    for (int i = 0; i < n; i++) {
        double t = AE(i, a);
        AE(i, a) = AE(i, b);
        AE(i, b) = t;
    }
    for (int j = 0; j < n; j++) {
        double t = AE(a, j);
        AE(a, j) = AE(b, j);
        AE(b, j) = t;
    }
#undef AE
    int32_t t = perm[a];
    perm[a] = perm[b];
    perm[b] = t;
}

/* LDL^T with the pivoting of Sec. 4.5 of the n x n symmetric matrix A
 * (column-major, both triangles), in pivot blocks of nb columns; only the
 * entries of the current block that are not yet eliminated take part in the
 * pivot search, as the paper restricts it to the diagonal block B_D.  For
 * each pivot position p of the block:
 *   pre-swap   the remaining block diagonal of largest magnitude moves to p;
 *   gamma_p    = |M_rp|, the largest magnitude below the pivot in the block;
 *   lift       if max(|M_pp|, gamma_p) <= b1, the pivot becomes
 *              sign(M_pp) b1 (a 1x1 pivot; lift[p] = new - old);
 *   1x1 at p   if |M_pp| >= alpha gamma_p, or |M_pp| gamma_r >= alpha gamma_p^2
 *              (gamma_r the largest off-diagonal magnitude of row r);
 *   1x1 at r   if |M_rr| >= alpha gamma_r (r interchanged with p);
 *   2x2 (p, r) otherwise (r interchanged with p + 1).
 * (With the pre-swap, |M_rr| <= |M_pp| < alpha gamma_p <= alpha gamma_r
 * whenever the third test is reached, so it never fires; it is kept as the
 * paper states the rule.)
 * Every pivot eliminates its columns from all rows below (a right-looking
 * update of the whole trailing matrix).  On return
 *   P A P^T + diag(lift) = L D L^T,  P e_k = e_{perm[k]} (perm[new] = old),
 * with L unit lower triangular in the strict lower triangle of A, D[k] the
 * diagonal of D, Doff[k] = D(k+1, k) for the first column of a 2x2 block
 * (else 0) and bsize[k] = 1 or 2 for the first column of a block, 0 for the
 * second.  orc_front_ldlt_bk eliminates only the first k columns, as in a
 * front with k fully-summed columns: only they are interchanged, and the
 * trailing (n-k) x (n-k) block ends as the Schur complement (D, bsize, lift
 * are zero there, the identity holds with L's trailing block and that Schur
 * complement in D's place).  Returns ORC_OK, ORC_ERR_ARG or
 * ORC_ERR_NONFINITE. */
int orc_front_ldlt_bk(int n, int k, int nb, double *A, double b1, double alpha, int32_t *perm, double *D,
                      double *Doff, int32_t *bsize, double *lift) {
    if (n < 0 || k < 0 || k > n || nb < 1 || !(b1 >= 0.0) || !(alpha > 0.0 && alpha < 1.0)) return ORC_ERR_ARG;
#define AE(i, j) A[(int64_t)(j) * n + (i)]
    for (int k = 0; k < n; k++) {
        perm[k] = k;
        D[k] = Doff[k] = lift[k] = 0.0;
        bsize[k] = 0;
    }
    int rc = ORC_OK;
    for (int b0 = 0; b0 < k; b0 += nb) {
        const int b1c = b0 + nb < k ? b0 + nb : k;
        int p = b0;
        while (p < b1c) {
            /* pre-swap: the largest remaining block diagonal to position p */
            int q = p;
            for (int t = p + 1; t < b1c; t++)
                if (fabs(AE(t, t)) > fabs(AE(q, q))) q = t;
            bk_swap(n, A, perm, p, q);
            /* gamma_p and r within the block */
            int r = -1;
            double gp = 0.0;
            for (int i = p + 1; i < b1c; i++)
                if (fabs(AE(i, p)) > gp) {
                    gp = fabs(AE(i, p));
                    r = i;
                }
            const double app = AE(p, p);
            int two = 0;
            if ((fabs(app) > gp ? fabs(app) : gp) <= b1) {
                const double dn = app < 0.0 ? -b1 : b1;
                lift[p] = dn - app;
                AE(p, p) = dn;
            } else if (fabs(app) < alpha * gp) {
                double gr = 0.0;
                for (int i = p; i < b1c; i++)
                    if (i != r && fabs(AE(i, r)) > gr) gr = fabs(AE(i, r));
                if (fabs(app) * gr >= alpha * gp * gp) {
                    /* 1x1 at p */
                } else if (fabs(AE(r, r)) >= alpha * gr) {
                    bk_swap(n, A, perm, p, r);
                } else {
                    bk_swap(n, A, perm, p + 1, r);
                    two = 1;
                }
            }
            if (!two) {
                const double d = AE(p, p);
                D[p] = d;
                bsize[p] = 1;
                if (!isfinite(d) || d == 0.0) rc = ORC_ERR_NONFINITE;
                for (int i = p + 1; i < n; i++) AE(i, p) /= d;
                for (int j = p + 1; j < n; j++)
                    for (int i = j; i < n; i++) {
                        AE(i, j) -= AE(i, p) * d * AE(j, p);
                        AE(j, i) = AE(i, j);
                    }
                for (int i = p + 1; i < n; i++) AE(p, i) = 0.0;  /* upper part of L's column: unused */
                p += 1;
            } else {
                const double e11 = AE(p, p), e21 = AE(p + 1, p), e22 = AE(p + 1, p + 1);
                const double det = e11 * e22 - e21 * e21;
                D[p] = e11;
                D[p + 1] = e22;
                Doff[p] = e21;
                bsize[p] = 2;
                if (!isfinite(det) || det == 0.0) rc = ORC_ERR_NONFINITE;
                /* [l_ip, l_ip+1] = [a_ip, a_ip+1] E^-1 for every row below the block pair */
                for (int i = p + 2; i < n; i++) {
                    const double x = AE(i, p), y = AE(i, p + 1);
                    AE(i, p) = (x * e22 - y * e21) / det;
                    AE(i, p + 1) = (y * e11 - x * e21) / det;
                }
                /* A_ij -= [l_ip l_ip+1] E [l_jp l_jp+1]^T */
                for (int j = p + 2; j < n; j++) {
                    const double wj0 = e11 * AE(j, p) + e21 * AE(j, p + 1);
                    const double wj1 = e21 * AE(j, p) + e22 * AE(j, p + 1);
                    for (int i = j; i < n; i++) {
                        AE(i, j) -= AE(i, p) * wj0 + AE(i, p + 1) * wj1;
                        AE(j, i) = AE(i, j);
                    }
                }
                AE(p + 1, p) = 0.0;  /* L is unit lower triangular: the 2x2 block lives in D */
                for (int i = p + 1; i < n; i++) AE(p, i) = 0.0;
                for (int i = p + 2; i < n; i++) AE(p + 1, i) = 0.0;
                p += 2;
            }
        }
    }
#undef AE
    return rc;
}

int orc_dense_ldlt_bk(int n, int nb, double *A, double b1, double alpha, int32_t *perm, double *D, double *Doff,
                      int32_t *bsize, double *lift) {
    return orc_front_ldlt_bk(n, n, nb, A, b1, alpha, perm, D, Doff, bsize, lift);
}

/* Solve A x = b with a factorisation from orc_dense_ldlt_bk (lift zero, or
 * the lifted matrix P^T (P A P^T + diag(lift)) P is the one solved):
 *   y = P b;  L z = y (forward);  D w = z (1x1 divisions, 2x2 blocks by
 *   their inverse);  L^T v = w (backward);  x = P^T v.
 * Lf holds L in its strict lower triangle (n x n, column-major). */
int orc_dense_solve_bk(int n, const double *Lf, const double *D, const double *Doff, const int32_t *bsize,
                       const int32_t *perm, const double *b, double *x) {
    if (n < 0) return ORC_ERR_ARG;
    double *v = (double *)xmalloc(NZ(n) * sizeof(double));
    for (int k = 0; k < n; k++) v[k] = b[perm[k]];
    for (int j = 0; j < n; j++)
        for (int i = j + 1; i < n; i++) v[i] -= Lf[(int64_t)j * n + i] * v[j];
    for (int k = 0; k < n;) {
        if (bsize[k] == 2) {
            const double e11 = D[k], e21 = Doff[k], e22 = D[k + 1];
            const double det = e11 * e22 - e21 * e21;
            const double y0 = v[k], y1 = v[k + 1];
            v[k] = (e22 * y0 - e21 * y1) / det;
            v[k + 1] = (e11 * y1 - e21 * y0) / det;
            k += 2;
        } else {
            v[k] /= D[k];
            k += 1;
        }
    }
    for (int j = n - 1; j >= 0; j--)
        for (int i = j + 1; i < n; i++) v[j] -= Lf[(int64_t)j * n + i] * v[i];
    for (int k = 0; k < n; k++) x[perm[k]] = v[k];
    free(v);
    return ORC_OK;
}
