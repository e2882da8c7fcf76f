// Symbolic analysis on the host, done once per pattern (Sec. 4.2-4.3 of
// Zanetti & Gondzio, arXiv 2508.04370):
//   pattern of K (Eq. augsys) or of A A^T (Eq. normeq)
//   -> fill-reducing order (AMD / nested dissection / user / natural)
//   -> elimination tree (Liu's algorithm with path compression)
//   -> postorder (depth first, children in ascending order)
//   -> column counts (row-subtree traversal)
//   -> fundamental supernodes and amalgamation (Sec. 4.1)
//   -> front row lists, extend-add maps, original-entry maps, tree levels and
//      the device layout of the fronts.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <numeric>

#include "ipm_plan.h"

namespace ipm {

namespace {

constexpr int kErrInvalid = -1;

// Lower pattern (with diagonal) of the matrix to factorise, original numbering,
// CSC: column j holds rows i >= j.  AS: [[D, A^T], [A, D]]; NE: A A^T.
void lower_pattern(const Plan &P, std::vector<int64_t> &cp, std::vector<int32_t> &ri) {
    const int32_t m = P.m, n = P.n;
    if (P.form == 1) {
        const int32_t N = n + m;
        cp.assign(N + 1, 0);
        ri.clear();
        ri.reserve(P.Acp[n] + N);
        for (int32_t j = 0; j < n; j++) {
            cp[j] = (int64_t)ri.size();
            ri.push_back(j);
            for (int64_t p = P.Acp[j]; p < P.Acp[j + 1]; p++) ri.push_back(n + P.Ari[p]);
        }
        for (int32_t i = 0; i < m; i++) {
            cp[n + i] = (int64_t)ri.size();
            ri.push_back(n + i);
        }
        cp[N] = (int64_t)ri.size();
    } else {
        // rows of A in CSR
        std::vector<int64_t> rp(m + 1, 0);
        std::vector<int32_t> rc(P.Acp[n]);
        for (int64_t p = 0; p < P.Acp[n]; p++) rp[P.Ari[p] + 1]++;
        for (int32_t i = 0; i < m; i++) rp[i + 1] += rp[i];
        std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
        for (int32_t j = 0; j < n; j++)
            for (int64_t p = P.Acp[j]; p < P.Acp[j + 1]; p++) rc[fill[P.Ari[p]]++] = j;
        std::vector<int32_t> mark(m, -1);
        cp.assign(m + 1, 0);
        ri.clear();
        for (int32_t i = 0; i < m; i++) {
            cp[i] = (int64_t)ri.size();
            size_t start = ri.size();
            ri.push_back(i);
            mark[i] = i;
            for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
                int32_t j = rc[p];
                for (int64_t q = P.Acp[j]; q < P.Acp[j + 1]; q++) {
                    int32_t r = P.Ari[q];
                    if (r > i && mark[r] != i) {
                        mark[r] = i;
                        ri.push_back(r);
                    }
                }
            }
            std::sort(ri.begin() + start, ri.end());
        }
        cp[m] = (int64_t)ri.size();
    }
}

Graph symmetric_graph(int32_t N, const std::vector<int64_t> &cp, const std::vector<int32_t> &ri) {
    Graph g;
    g.N = N;
    g.ptr.assign(N + 1, 0);
    for (int32_t j = 0; j < N; j++)
        for (int64_t p = cp[j]; p < cp[j + 1]; p++)
            if (ri[p] != j) {
                g.ptr[j + 1]++;
                g.ptr[ri[p] + 1]++;
            }
    for (int32_t j = 0; j < N; j++) g.ptr[j + 1] += g.ptr[j];
    g.adj.resize(g.ptr[N]);
    std::vector<int64_t> fill(g.ptr.begin(), g.ptr.end() - 1);
    for (int32_t j = 0; j < N; j++)
        for (int64_t p = cp[j]; p < cp[j + 1]; p++)
            if (ri[p] != j) {
                g.adj[fill[j]++] = ri[p];
                g.adj[fill[ri[p]]++] = j;
            }
    return g;
}

// Elimination tree of P M P^T (Liu): parent[i] for new indices.
std::vector<int32_t> etree(const Graph &g, const std::vector<int32_t> &perm, const std::vector<int32_t> &iperm) {
    const int32_t N = g.N;
    std::vector<int32_t> parent(N, -1), anc(N, -1);
    for (int32_t i = 0; i < N; i++) {
        int32_t io = perm[i];
        for (int64_t p = g.ptr[io]; p < g.ptr[io + 1]; p++) {
            int32_t k = iperm[g.adj[p]];
            if (k >= i) continue;
            int32_t r = k;
            while (anc[r] != -1 && anc[r] != i) {
                int32_t t = anc[r];
                anc[r] = i;
                r = t;
            }
            if (anc[r] == -1) {
                anc[r] = i;
                parent[r] = i;
            }
        }
    }
    return parent;
}

// Postorder: depth first, children ascending, roots ascending.
std::vector<int32_t> postorder(const std::vector<int32_t> &parent) {
    const int32_t N = (int32_t)parent.size();
    std::vector<int32_t> head(N, -1), next(N, -1), post;
    post.reserve(N);
    for (int32_t j = N - 1; j >= 0; j--)
        if (parent[j] >= 0) {
            next[j] = head[parent[j]];
            head[parent[j]] = j;
        }
    std::vector<int32_t> stack;
    for (int32_t r = 0; r < N; r++) {
        if (parent[r] != -1) continue;
        stack.push_back(r);
        while (!stack.empty()) {
            int32_t v = stack.back();
            int32_t c = head[v];
            if (c == -1) {
                stack.pop_back();
                post.push_back(v);
            } else {
                head[v] = next[c];
                stack.push_back(c);
            }
        }
    }
    return post;
}

double front_flops(int64_t f, int64_t k) {
    // sum_{i=1..k} (f-i)(f-i+3)
    double s = 0.0;
    for (int64_t i = 1; i <= k; i++) s += (double)(f - i) * (double)(f - i + 3);
    return s;
}

}  // namespace

int64_t count_ne_lower(int32_t m, int32_t n, const int64_t *colptr, const int32_t *rowidx, int64_t limit) {
    std::vector<int64_t> rp(m + 1, 0);
    std::vector<int32_t> rc(colptr[n]);
    for (int64_t p = 0; p < colptr[n]; p++) rp[rowidx[p] + 1]++;
    for (int32_t i = 0; i < m; i++) rp[i + 1] += rp[i];
    std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
    for (int32_t j = 0; j < n; j++)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) rc[fill[rowidx[p]]++] = j;
    std::vector<int32_t> mark(m, -1);
    int64_t total = 0;
    for (int32_t i = 0; i < m; i++) {
        mark[i] = i;
        total++;
        for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
            const int32_t j = rc[p];
            for (int64_t q = colptr[j]; q < colptr[j + 1]; q++) {
                const int32_t r = rowidx[q];
                if (r > i && mark[r] != i) {
                    mark[r] = i;
                    if (++total > limit) return limit + 1;
                }
            }
        }
    }
    return total;
}

int analyse(Plan &P, int32_t m, int32_t n, const int64_t *colptr, const int32_t *rowidx, int32_t form,
            int32_t ordering, const int32_t *user_perm, const AnalyseOptions &opt, std::string &err) {
    auto t0 = std::chrono::steady_clock::now();
    if (m < 0 || n < 0 || !colptr || (colptr[n] > 0 && !rowidx)) {
        err = "bad sizes or null pattern";
        return kErrInvalid;
    }
    if (colptr[0] != 0) {
        err = "colptr[0] must be 0";
        return kErrInvalid;
    }
    for (int32_t j = 0; j < n; j++) {
        if (colptr[j + 1] < colptr[j]) {
            err = "colptr not monotone";
            return kErrInvalid;
        }
        for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
            if (rowidx[p] < 0 || rowidx[p] >= m) {
                err = "row index out of range";
                return kErrInvalid;
            }
            if (p > colptr[j] && rowidx[p] <= rowidx[p - 1]) {
                err = "rows not sorted or duplicated";
                return kErrInvalid;
            }
        }
    }
    if (form != 1 && form != 2) {
        err = "form must be augmented (1) or normal (2) here";
        return kErrInvalid;
    }
    P = Plan();
    P.m = m;
    P.n = n;
    P.form = form;
    P.ordering = ordering;
    P.Acp.assign(colptr, colptr + n + 1);
    P.Ari.assign(rowidx, rowidx + colptr[n]);
    const int32_t N = form == 1 ? n + m : m;
    P.N = N;

    std::vector<int64_t> lcp;
    std::vector<int32_t> lri;
    lower_pattern(P, lcp, lri);
    P.nnzK_lower = lcp[N];
    if (form == 2) {
        // contributor pairs of every lower entry (r, i) of A A^T, ascending j
        if ((int64_t)P.Acp[n] > INT32_MAX) {
            err = "too many entries in A for the normal equations";
            return kErrInvalid;
        }
        std::vector<int64_t> rp(m + 1, 0);
        std::vector<int32_t> rc(P.Acp[n]), rpos(P.Acp[n]);
        for (int64_t p = 0; p < P.Acp[n]; p++) rp[P.Ari[p] + 1]++;
        for (int32_t i = 0; i < m; i++) rp[i + 1] += rp[i];
        {
            std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
            for (int32_t j = 0; j < n; j++)
                for (int64_t p = P.Acp[j]; p < P.Acp[j + 1]; p++) {
                    rc[fill[P.Ari[p]]] = j;
                    rpos[fill[P.Ari[p]]++] = (int32_t)p;
                }
        }
        std::vector<int64_t> cnt(lcp[N] + 1, 0);
        std::vector<int64_t> pos(m, -1);
        int64_t total = 0;
        for (int pass = 0; pass < 2; pass++) {
            if (pass == 1) {
                for (int64_t e = 0; e < lcp[N]; e++) cnt[e + 1] += cnt[e];
                total = cnt[lcp[N]];
                if (total > kMaxNePairs) {
                    err = "normal equations too expensive to form (pair limit)";
                    return kErrInvalid;
                }
                P.ne_ta.resize(total);
                P.ne_tb.resize(total);
                P.ne_tj.resize(total);
            }
            std::vector<int64_t> fillc;
            if (pass == 1) fillc.assign(cnt.begin(), cnt.end() - 1);
            for (int32_t i = 0; i < m; i++) {
                for (int64_t q = lcp[i]; q < lcp[i + 1]; q++) pos[lri[q]] = q;
                for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
                    const int32_t j = rc[p];
                    const int32_t aij = rpos[p];
                    for (int64_t t = P.Acp[j]; t < P.Acp[j + 1]; t++) {
                        const int32_t r = P.Ari[t];
                        if (r < i) continue;
                        const int64_t e = pos[r];
                        if (pass == 0) cnt[e + 1]++;
                        else {
                            const int64_t w = fillc[e]++;
                            P.ne_ta[w] = (int32_t)t;
                            P.ne_tb[w] = aij;
                            P.ne_tj[w] = j;
                        }
                    }
                }
            }
        }
        P.ne_tptr.assign(cnt.begin(), cnt.end());
        P.ne_cp = lcp;
        P.ne_ri = lri;
    }
    Graph g = symmetric_graph(N, lcp, lri);

    // ----- ordering
    std::vector<int32_t> perm0;
    switch (ordering) {
        case 0: perm0 = order_amd(g, opt.dense_row_factor); break;
        case 1: perm0 = order_nd(g, opt.nd_leaf, opt.dense_row_factor); break;
        case 2: {
            if (!user_perm) {
                err = "user permutation missing";
                return kErrInvalid;
            }
            perm0.assign(user_perm, user_perm + N);
            break;
        }
        case 3:
            perm0.resize(N);
            std::iota(perm0.begin(), perm0.end(), 0);
            break;
        default: err = "unknown ordering"; return kErrInvalid;
    }
    if ((int32_t)perm0.size() != N) {
        err = "ordering produced a wrong size";
        return kErrInvalid;
    }
    std::vector<int32_t> iperm0(N, -1);
    for (int32_t i = 0; i < N; i++) {
        if (perm0[i] < 0 || perm0[i] >= N || iperm0[perm0[i]] != -1) {
            err = "not a permutation";
            return kErrInvalid;
        }
        iperm0[perm0[i]] = i;
    }

    // ----- elimination tree and postorder
    std::vector<int32_t> parent0 = etree(g, perm0, iperm0);
    std::vector<int32_t> post = postorder(parent0);
    std::vector<int32_t> ipost(N);
    for (int32_t t = 0; t < N; t++) ipost[post[t]] = t;
    P.perm.resize(N);
    P.iperm.resize(N);
    P.parent.resize(N);
    for (int32_t t = 0; t < N; t++) {
        P.perm[t] = perm0[post[t]];
        P.iperm[P.perm[t]] = t;
        int32_t pa = parent0[post[t]];
        P.parent[t] = pa >= 0 ? ipost[pa] : -1;
    }

    // ----- column counts: every row i's subtree {k : L_ik != 0}
    P.colcount.assign(N, 1);
    {
        std::vector<int32_t> mark(N, -1);
        for (int32_t i = 0; i < N; i++) {
            mark[i] = i;
            int32_t io = P.perm[i];
            for (int64_t p = g.ptr[io]; p < g.ptr[io + 1]; p++) {
                int32_t k = P.iperm[g.adj[p]];
                if (k >= i) continue;
                while (mark[k] != i) {
                    P.colcount[k]++;
                    mark[k] = i;
                    k = P.parent[k];
                }
            }
        }
    }

    // ----- fundamental supernodes
    std::vector<int32_t> nchild(N, 0);
    for (int32_t j = 0; j < N; j++)
        if (P.parent[j] >= 0) nchild[P.parent[j]]++;
    std::vector<int32_t> fstart;
    for (int32_t j = 0; j < N; j++) {
        bool joins = j > 0 && P.parent[j - 1] == j && nchild[j] == 1 && P.colcount[j - 1] == P.colcount[j] + 1;
        if (!joins) fstart.push_back(j);
    }
    fstart.push_back(N);
    const int32_t nf = (int32_t)fstart.size() - 1;

    // ----- amalgamation: bottom-up; absorb the supernode ending right before
    // p while it is a child of p and (merged width <= amalg_width or its
    // explicit zeros <= zero_frac of its stored entries)
    struct Open {
        int32_t s, e;
        int64_t nnz, f;
    };
    auto amalgamate = [&](double zero_frac) {
        std::vector<Open> st;
        st.reserve(nf);
        for (int32_t t = 0; t < nf; t++) {
            int32_t ps = fstart[t], pe = fstart[t + 1];
            int64_t pnnz = 0;
            for (int32_t j = ps; j < pe; j++) pnnz += P.colcount[j];
            int64_t pf = P.colcount[ps];
            while (!st.empty()) {
                const Open &c = st.back();
                if (c.e != ps) break;
                int32_t par = P.parent[c.e - 1];
                if (!(par >= ps && par < pe)) break;
                int64_t k = (int64_t)(c.e - c.s) + (pe - ps);
                int64_t f = (int64_t)(c.e - c.s) + pf;
                int64_t total = k * f - k * (k - 1) / 2;
                int64_t zeros = total - (c.nnz + pnnz);
                bool merge = k <= opt.amalg_width || (double)zeros <= zero_frac * (double)total;
                if (!merge) break;
                ps = c.s;
                pnnz += c.nnz;
                pf = f;
                st.pop_back();
            }
            st.push_back({ps, pe, pnnz, pf});
        }
        return st;
    };
    // A negative threshold chooses between 0.1 and 0.2 by a model of the
    // factorisation time: front flops at 1 TFLOP/s (the FP64 update rate)
    // plus 60 us per tree level (the latency of one level's launches and
    // pivot chains).  More amalgamation trades flops for fewer, larger
    // supernodes and fewer levels; the model keeps it where the levels, not
    // the flops, dominate.
    std::vector<Open> st;
    if (opt.amalg_zero_frac >= 0) {
        st = amalgamate(opt.amalg_zero_frac);
        P.amalg_zero_frac = opt.amalg_zero_frac;
    } else {
        double best_t = 0.0;
        std::vector<int32_t> c2s(N), height;
        for (double zf : {0.1, 0.2}) {
            std::vector<Open> cand = amalgamate(zf);
            const int32_t nc = (int32_t)cand.size();
            double flops = 0.0;
            height.assign(nc, 0);
            int32_t levels = 0;
            for (int32_t t = 0; t < nc; t++)
                for (int32_t j = cand[t].s; j < cand[t].e; j++) c2s[j] = t;
            for (int32_t t = 0; t < nc; t++) {
                const double k = cand[t].e - cand[t].s, f = (double)cand[t].f;
                // sum_{i=1..k} (f-i)(f-i+3) with u = f-i running over f-k .. f-1
                const double a = f - k, b = f - 1;
                const double su = (b * (b + 1) - (a - 1) * a) / 2.0;
                const double su2 = (b * (b + 1) * (2 * b + 1) - (a - 1) * a * (2 * a - 1)) / 6.0;
                flops += su2 + 3.0 * su;
                levels = std::max(levels, height[t] + 1);
                const int32_t pc = P.parent[cand[t].e - 1];
                if (pc >= 0) height[c2s[pc]] = std::max(height[c2s[pc]], height[t] + 1);
            }
            const double tm = flops / 1e12 + 60e-6 * levels;
            if (st.empty() || tm < best_t) {
                best_t = tm;
                st.swap(cand);
                P.amalg_zero_frac = zf;
            }
        }
    }
    const int32_t ns = (int32_t)st.size();
    P.nsuper = ns;
    P.sn_start.resize(ns + 1);
    for (int32_t s = 0; s < ns; s++) P.sn_start[s] = st[s].s;
    P.sn_start[ns] = N;
    std::vector<int32_t> col2sn(N);
    for (int32_t s = 0; s < ns; s++)
        for (int32_t j = P.sn_start[s]; j < P.sn_start[s + 1]; j++) col2sn[j] = s;
    P.sn_parent.resize(ns);
    for (int32_t s = 0; s < ns; s++) {
        int32_t last = P.sn_start[s + 1] - 1;
        P.sn_parent[s] = P.parent[last] >= 0 ? col2sn[P.parent[last]] : -1;
    }
    // children lists, ascending
    P.child_ptr.assign(ns + 1, 0);
    for (int32_t s = 0; s < ns; s++)
        if (P.sn_parent[s] >= 0) P.child_ptr[P.sn_parent[s] + 1]++;
    for (int32_t s = 0; s < ns; s++) P.child_ptr[s + 1] += P.child_ptr[s];
    P.child_list.resize(P.child_ptr[ns]);
    {
        std::vector<int32_t> fill(P.child_ptr.begin(), P.child_ptr.end() - 1);
        for (int32_t s = 0; s < ns; s++)
            if (P.sn_parent[s] >= 0) P.child_list[fill[P.sn_parent[s]]++] = s;
    }

    // ----- front rows: R_s = cols(s) U {A-pattern rows of cols(s)} U
    //       U_{children c} (R_c \ cols(c))
    P.sn_rptr.assign(ns + 1, 0);
    P.sn_rows.clear();
    {
        std::vector<int32_t> mark(N, -1), tmp;
        for (int32_t s = 0; s < ns; s++) {
            const int32_t c0 = P.sn_start[s], c1 = P.sn_start[s + 1];
            tmp.clear();
            for (int32_t j = c0; j < c1; j++) {
                mark[j] = s;
                tmp.push_back(j);
            }
            for (int32_t j = c0; j < c1; j++) {
                int32_t jo = P.perm[j];
                for (int64_t p = g.ptr[jo]; p < g.ptr[jo + 1]; p++) {
                    int32_t i = P.iperm[g.adj[p]];
                    if (i > j && mark[i] != s) {
                        mark[i] = s;
                        tmp.push_back(i);
                    }
                }
            }
            for (int32_t q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
                int32_t c = P.child_list[q];
                int32_t kc = P.sn_start[c + 1] - P.sn_start[c];
                for (int64_t p = P.sn_rptr[c] + kc; p < P.sn_rptr[c + 1]; p++) {
                    int32_t i = P.sn_rows[p];
                    if (mark[i] != s) {
                        mark[i] = s;
                        tmp.push_back(i);
                    }
                }
            }
            std::sort(tmp.begin(), tmp.end());
            P.sn_rows.insert(P.sn_rows.end(), tmp.begin(), tmp.end());
            P.sn_rptr[s + 1] = (int64_t)P.sn_rows.size();
        }
    }

    // ----- per-supernode layout, statistics
    P.sn_k.resize(ns);
    P.sn_f.resize(ns);
    P.sn_ld.resize(ns);
    P.sn_off.resize(ns + 1);
    P.sn_level.assign(ns, 0);
    P.upd_off.resize(ns + 1);
    int64_t off = 0, uoff = 0;
    for (int32_t s = 0; s < ns; s++) {
        int32_t k = P.sn_start[s + 1] - P.sn_start[s];
        int32_t f = (int32_t)(P.sn_rptr[s + 1] - P.sn_rptr[s]);
        int32_t ld = (f + 3) & ~3;
        P.sn_k[s] = k;
        P.sn_f[s] = f;
        P.sn_ld[s] = ld;
        P.sn_off[s] = off;
        off += (int64_t)ld * f;
        P.upd_off[s] = uoff;
        uoff += f;
        P.nnzL += (int64_t)k * f - (int64_t)k * (k - 1) / 2;
        P.flops += front_flops(f, k);
        P.max_f = std::max(P.max_f, f);
        P.max_k = std::max(P.max_k, k);
        for (int32_t q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++)
            P.sn_level[s] = std::max(P.sn_level[s], P.sn_level[P.child_list[q]] + 1);
    }
    P.sn_off[ns] = off;
    P.front_doubles = off;
    P.upd_off[ns] = uoff;
    P.upd_total = uoff;

    // ----- extend-add maps: contribution rows of s -> local rows of parent
    P.map_off.assign(ns + 1, 0);
    P.relmap.clear();
    {
        std::vector<int32_t> pos(N, -1);
        for (int32_t s = 0; s < ns; s++) {
            int32_t pa = P.sn_parent[s];
            int32_t k = P.sn_k[s], f = P.sn_f[s];
            P.map_off[s] = (int64_t)P.relmap.size();
            if (pa < 0 || f == k) continue;
            for (int64_t p = P.sn_rptr[pa]; p < P.sn_rptr[pa + 1]; p++) pos[P.sn_rows[p]] = (int32_t)(p - P.sn_rptr[pa]);
            for (int64_t p = P.sn_rptr[s] + k; p < P.sn_rptr[s + 1]; p++) {
                int32_t r = pos[P.sn_rows[p]];
                if (r < 0) {
                    err = "internal: contribution row missing from parent front";
                    return kErrInvalid;
                }
                P.relmap.push_back(r);
            }
            for (int64_t p = P.sn_rptr[pa]; p < P.sn_rptr[pa + 1]; p++) pos[P.sn_rows[p]] = -1;
        }
        P.map_off[ns] = (int64_t)P.relmap.size();
    }

    // ----- original entries: for every stored lower entry of P M P^T, the
    // front of its column's supernode and the local offset col*ld + row
    P.sign.resize(N);
    for (int32_t i = 0; i < N; i++) P.sign[i] = (form == 1 && P.perm[i] < n) ? -1 : 1;
    {
        // value source of each lower entry in original numbering:
        //   AS: diagonal of primal j -> -1-j; dual diagonal -> none; A entry -> its index
        //   NE: index of the lower entry of M (filled by the formation kernel)
        struct Ent {
            int32_t s, row, col;
            int64_t src;
        };
        std::vector<Ent> ents;
        ents.reserve(lcp[N]);
        for (int32_t jo = 0; jo < N; jo++) {
            for (int64_t p = lcp[jo]; p < lcp[jo + 1]; p++) {
                int32_t io = lri[p];
                int64_t src;
                if (form == 1) {
                    if (io == jo) {
                        if (jo >= n) continue;  // dual diagonal: zero until delta at the pivot
                        src = -1 - (int64_t)jo;
                    } else {
                        src = P.Acp[jo] + (p - lcp[jo] - 1);  // column jo < n holds [diag, A rows]
                    }
                } else {
                    src = p;
                }
                int32_t a = P.iperm[io], b = P.iperm[jo];
                int32_t col = std::min(a, b), row = std::max(a, b);
                ents.push_back({col2sn[col], row, col, src});
            }
        }
        std::stable_sort(ents.begin(), ents.end(), [](const Ent &x, const Ent &y) { return x.s < y.s; });
        P.orig_ptr.assign(ns + 1, 0);
        for (const Ent &e : ents) P.orig_ptr[e.s + 1]++;
        for (int32_t s = 0; s < ns; s++) P.orig_ptr[s + 1] += P.orig_ptr[s];
        P.orig_dst.resize(ents.size());
        P.orig_src.resize(ents.size());
        std::vector<int32_t> lrow(N, -1);
        int32_t cur = -1;
        for (size_t t = 0; t < ents.size(); t++) {
            const Ent &e = ents[t];
            if (e.s != cur) {
                if (cur >= 0)
                    for (int64_t p = P.sn_rptr[cur]; p < P.sn_rptr[cur + 1]; p++) lrow[P.sn_rows[p]] = -1;
                for (int64_t p = P.sn_rptr[e.s]; p < P.sn_rptr[e.s + 1]; p++)
                    lrow[P.sn_rows[p]] = (int32_t)(p - P.sn_rptr[e.s]);
                cur = e.s;
            }
            int32_t lr = lrow[e.row], lc = e.col - P.sn_start[e.s];
            if (lr < 0 || lc < 0 || lc >= P.sn_k[e.s]) {
                err = "internal: original entry outside its front";
                return kErrInvalid;
            }
            int64_t dst = (int64_t)lc * P.sn_ld[e.s] + lr;
            if (dst > INT32_MAX) {
                err = "front too large for 32-bit local offsets";
                return kErrInvalid;
            }
            P.orig_dst[t] = (int32_t)dst;
            P.orig_src[t] = e.src;
        }
        // each supernode's entries by destination (column-major), so that a
        // range of front columns owns a contiguous range of entries
        std::vector<std::pair<int32_t, int64_t>> tmp;
        for (int32_t s = 0; s < ns; s++) {
            tmp.clear();
            for (int64_t t = P.orig_ptr[s]; t < P.orig_ptr[s + 1]; t++) tmp.emplace_back(P.orig_dst[t], P.orig_src[t]);
            std::sort(tmp.begin(), tmp.end());
            for (size_t u = 0; u < tmp.size(); u++) {
                P.orig_dst[P.orig_ptr[s] + u] = tmp[u].first;
                P.orig_src[P.orig_ptr[s] + u] = tmp[u].second;
            }
        }
    }

    // ----- levels and size classes
    P.nlevels = 0;
    for (int32_t s = 0; s < ns; s++) P.nlevels = std::max(P.nlevels, P.sn_level[s] + 1);
    P.lvl_small_ptr.assign(P.nlevels + 1, 0);
    P.lvl_large_ptr.assign(P.nlevels + 1, 0);
    // small or large path per front (see kPromoteBelow)
    P.sn_large.assign(ns, 0);
    {
        std::vector<int32_t> mid(P.nlevels, 0);
        for (int32_t s = 0; s < ns; s++)
            if (P.sn_f[s] > kPromoteMin && P.sn_f[s] <= kSmallFrontMax) mid[P.sn_level[s]]++;
        for (int32_t s = 0; s < ns; s++) {
            const int32_t f = P.sn_f[s];
            P.sn_large[s] = (f > kSmallFrontMax || (f > kPromoteMin && mid[P.sn_level[s]] < kPromoteBelow)) ? 1 : 0;
        }
    }
    for (int32_t s = 0; s < ns; s++) {
        if (!P.sn_large[s]) P.lvl_small_ptr[P.sn_level[s] + 1]++;
        else P.lvl_large_ptr[P.sn_level[s] + 1]++;
    }
    for (int32_t l = 0; l < P.nlevels; l++) {
        P.lvl_small_ptr[l + 1] += P.lvl_small_ptr[l];
        P.lvl_large_ptr[l + 1] += P.lvl_large_ptr[l];
    }
    P.lvl_small.resize(P.lvl_small_ptr[P.nlevels]);
    P.lvl_large.resize(P.lvl_large_ptr[P.nlevels]);
    {
        std::vector<int32_t> fs(P.lvl_small_ptr.begin(), P.lvl_small_ptr.end() - 1);
        std::vector<int32_t> fl(P.lvl_large_ptr.begin(), P.lvl_large_ptr.end() - 1);
        for (int32_t s = 0; s < ns; s++) {
            if (!P.sn_large[s]) P.lvl_small[fs[P.sn_level[s]]++] = s;
            else P.lvl_large[fl[P.sn_level[s]]++] = s;
        }
    }
    P.nsmall = (int32_t)P.lvl_small.size();
    P.nlarge = (int32_t)P.lvl_large.size();

    if (opt.verbose) {
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        std::fprintf(stderr,
                     "[ipm analyse] N=%d nsuper=%d levels=%d small=%d large=%d max_f=%d max_k=%d nnzL=%lld "
                     "flops=%.3e fronts=%.1f MB (%.1f ms)\n",
                     N, ns, P.nlevels, P.nsmall, P.nlarge, P.max_f, P.max_k, (long long)P.nnzL, P.flops,
                     P.front_doubles * 8.0 / 1e6, ms);
    }
    return 0;
}

}  // namespace ipm
