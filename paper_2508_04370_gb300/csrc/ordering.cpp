// Fill-reducing orderings for the symbolic analysis (Sec. 4.2).
//
// order_amd: approximate minimum degree on a quotient graph, after Amestoy,
//   Davis and Duff (SIAM J. Matrix Anal. Appl. 17, 1996): variables and
//   elements, the approximate external degree bound
//       d_i <- min( n_left - |i|,  d_i + |L_p \ i|,  |A_i \ i| + |L_p \ i| + sum_{e in E_i \ p} |L_e \ L_p| ),
//   aggressive element absorption (|L_e \ L_p| = 0), supervariable detection
//   by hashing, and dense rows (degree > max(16, f*sqrt(N))) ordered last.
// order_nd: nested dissection by recursive vertex separators taken from
//   breadth-first level structures rooted at a pseudo-peripheral vertex;
//   subgraphs below the leaf size are ordered with order_amd.  The paper uses
//   Metis (Sec. 4.2); this is a self-contained replacement.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "ipm_plan.h"

namespace ipm {
namespace {

enum Kind : int8_t { VAR = 0, MERGED = 1, ELEM = 2, DEAD = 3, DENSE = 4 };

struct Amd {
    int32_t N;
    std::vector<std::vector<int32_t>> A, E, Le;
    std::vector<int8_t> kind;
    std::vector<int32_t> nv, deg, head, nxt, prv, mnext, mlast;
    std::vector<int32_t> mark, wval, wtouch;
    int32_t tag = 0, mindeg = 0;

    void bucket_insert(int32_t i) {
        int32_t d = deg[i];
        nxt[i] = head[d];
        prv[i] = -1;
        if (head[d] >= 0) prv[head[d]] = i;
        head[d] = i;
        if (d < mindeg) mindeg = d;
    }
    void bucket_remove(int32_t i) {
        if (prv[i] >= 0) nxt[prv[i]] = nxt[i];
        else head[deg[i]] = nxt[i];
        if (nxt[i] >= 0) prv[nxt[i]] = prv[i];
        nxt[i] = prv[i] = -1;
    }
    int32_t next_tag() {
        if (++tag == INT32_MAX) {
            std::fill(mark.begin(), mark.end(), 0);
            tag = 1;
        }
        return tag;
    }
};

}  // namespace

std::vector<int32_t> order_amd(const Graph &g, double dense_factor) {
    Amd s;
    const int32_t N = g.N;
    s.N = N;
    std::vector<int32_t> order;
    order.reserve(N);
    if (N == 0) return order;
    s.A.resize(N);
    s.E.resize(N);
    s.Le.resize(N);
    s.kind.assign(N, VAR);
    s.nv.assign(N, 1);
    s.deg.assign(N, 0);
    s.head.assign(N + 1, -1);
    s.nxt.assign(N, -1);
    s.prv.assign(N, -1);
    s.mnext.assign(N, -1);
    s.mlast.resize(N);
    std::iota(s.mlast.begin(), s.mlast.end(), 0);
    s.mark.assign(N, 0);
    s.wval.assign(N, 0);
    s.wtouch.assign(N, 0);

    const double thr = std::max(16.0, dense_factor * std::sqrt((double)N));
    int32_t ndense = 0;
    for (int32_t i = 0; i < N; i++) {
        int64_t d = g.ptr[i + 1] - g.ptr[i];
        if (dense_factor > 0 && (double)d > thr) {
            s.kind[i] = DENSE;
            ndense++;
        }
    }
    for (int32_t i = 0; i < N; i++) {
        if (s.kind[i] != VAR) continue;
        auto &a = s.A[i];
        for (int64_t p = g.ptr[i]; p < g.ptr[i + 1]; p++) {
            int32_t j = g.adj[p];
            if (j != i && s.kind[j] == VAR) a.push_back(j);
        }
        s.deg[i] = (int32_t)a.size();
    }
    s.mindeg = N;
    for (int32_t i = N - 1; i >= 0; i--)
        if (s.kind[i] == VAR) s.bucket_insert(i);

    const int32_t nvar = N - ndense;
    int32_t nel = 0;
    std::vector<int32_t> Lp, keys;
    std::vector<int64_t> hash;
    std::vector<int32_t> touched;
    int32_t wstamp = 0;
    while (nel < nvar) {
        while (s.mindeg <= N && s.head[s.mindeg] < 0) s.mindeg++;
        int32_t p = s.head[s.mindeg];
        s.bucket_remove(p);
        const int32_t tg = s.next_tag();
        s.mark[p] = tg;
        Lp.clear();
        int64_t degLp = 0;
        for (int32_t e : s.E[p]) {
            if (s.kind[e] != ELEM) continue;
            for (int32_t i : s.Le[e])
                if (s.kind[i] == VAR && s.mark[i] != tg) {
                    s.mark[i] = tg;
                    Lp.push_back(i);
                    degLp += s.nv[i];
                }
            s.kind[e] = DEAD;
            std::vector<int32_t>().swap(s.Le[e]);
        }
        for (int32_t i : s.A[p])
            if (s.kind[i] == VAR && s.mark[i] != tg) {
                s.mark[i] = tg;
                Lp.push_back(i);
                degLp += s.nv[i];
            }
        std::vector<int32_t>().swap(s.E[p]);
        std::vector<int32_t>().swap(s.A[p]);
        s.kind[p] = ELEM;
        for (int32_t v = p; v >= 0; v = s.mnext[v]) order.push_back(v);
        nel += s.nv[p];
        for (int32_t i : Lp) s.bucket_remove(i);

        // |L_e \ L_p| for every element adjacent to L_p
        if (++wstamp == INT32_MAX) {
            std::fill(s.wtouch.begin(), s.wtouch.end(), 0);
            wstamp = 1;
        }
        touched.clear();
        for (int32_t i : Lp)
            for (int32_t e : s.E[i]) {
                if (s.kind[e] != ELEM) continue;
                if (s.wtouch[e] != wstamp) {
                    s.wtouch[e] = wstamp;
                    int32_t w = 0;
                    for (int32_t j : s.Le[e])
                        if (s.kind[j] == VAR) w += s.nv[j];
                    s.wval[e] = w;
                    touched.push_back(e);
                }
                s.wval[e] -= s.nv[i];
            }
        const int32_t nleft = nvar - nel;
        for (int32_t i : Lp) {
            auto &Ei = s.E[i];
            int64_t sumw = 0;
            size_t w = 0;
            for (int32_t e : Ei) {
                if (s.kind[e] != ELEM) continue;
                if (s.wval[e] == 0) {  // L_e is inside L_p: absorb
                    s.kind[e] = DEAD;
                    std::vector<int32_t>().swap(s.Le[e]);
                    continue;
                }
                Ei[w++] = e;
                sumw += s.wval[e];
            }
            Ei.resize(w);
            Ei.push_back(p);
            auto &Ai = s.A[i];
            int64_t suma = 0;
            w = 0;
            for (int32_t j : Ai)
                if (s.kind[j] == VAR && s.mark[j] != tg) {
                    Ai[w++] = j;
                    suma += s.nv[j];
                }
            Ai.resize(w);
            int64_t ext = degLp - s.nv[i];
            int64_t d = std::min<int64_t>((int64_t)s.deg[i] + ext, suma + ext + sumw);
            d = std::min<int64_t>(d, (int64_t)nleft - s.nv[i]);
            s.deg[i] = (int32_t)std::max<int64_t>(d, 0);
        }
        // supervariables: identical element and variable lists
        if (Lp.size() > 1) {
            hash.resize(Lp.size());
            keys.resize(Lp.size());
            for (size_t t = 0; t < Lp.size(); t++) {
                int32_t i = Lp[t];
                int64_t h = 0;
                for (int32_t e : s.E[i]) h += e;
                for (int32_t j : s.A[i]) h += j;
                hash[t] = h;
                keys[t] = (int32_t)t;
            }
            std::sort(keys.begin(), keys.end(), [&](int32_t a, int32_t b) {
                if (hash[a] != hash[b]) return hash[a] < hash[b];
                return Lp[a] < Lp[b];
            });
            for (size_t a = 0; a < keys.size(); a++) {
                int32_t i = Lp[keys[a]];
                if (s.kind[i] != VAR) continue;
                bool sorted_i = false;
                for (size_t b = a + 1; b < keys.size() && hash[keys[b]] == hash[keys[a]]; b++) {
                    int32_t j = Lp[keys[b]];
                    if (s.kind[j] != VAR) continue;
                    if (s.E[i].size() != s.E[j].size() || s.A[i].size() != s.A[j].size()) continue;
                    if (!sorted_i) {
                        std::sort(s.E[i].begin(), s.E[i].end());
                        std::sort(s.A[i].begin(), s.A[i].end());
                        sorted_i = true;
                    }
                    std::sort(s.E[j].begin(), s.E[j].end());
                    std::sort(s.A[j].begin(), s.A[j].end());
                    if (s.E[i] != s.E[j] || s.A[i] != s.A[j]) continue;
                    // merge j into i
                    s.deg[i] -= s.nv[j];
                    if (s.deg[i] < 0) s.deg[i] = 0;
                    s.nv[i] += s.nv[j];
                    s.nv[j] = 0;
                    s.kind[j] = MERGED;
                    s.mnext[s.mlast[i]] = j;
                    s.mlast[i] = s.mlast[j];
                    std::vector<int32_t>().swap(s.E[j]);
                    std::vector<int32_t>().swap(s.A[j]);
                }
            }
        }
        auto &Lep = s.Le[p];
        Lep.clear();
        for (int32_t i : Lp)
            if (s.kind[i] == VAR) {
                Lep.push_back(i);
                if (s.deg[i] > N) s.deg[i] = N;
                s.bucket_insert(i);
            }
    }
    for (int32_t i = 0; i < N; i++)
        if (s.kind[i] == DENSE) order.push_back(i);
    return order;
}

namespace {

struct Sub {
    std::vector<int32_t> verts;  // global ids
};

// Induced subgraph on `verts` (global ids); loc must map global -> local for
// members (stamped with `stamp`).
Graph induced(const Graph &g, const std::vector<int32_t> &verts, std::vector<int32_t> &loc,
              std::vector<int32_t> &stampv, int32_t stamp) {
    Graph h;
    h.N = (int32_t)verts.size();
    for (int32_t t = 0; t < h.N; t++) {
        loc[verts[t]] = t;
        stampv[verts[t]] = stamp;
    }
    h.ptr.assign(h.N + 1, 0);
    for (int32_t t = 0; t < h.N; t++) {
        int32_t v = verts[t];
        for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; p++)
            if (stampv[g.adj[p]] == stamp) h.adj.push_back(loc[g.adj[p]]);
        h.ptr[t + 1] = (int64_t)h.adj.size();
    }
    return h;
}

// BFS levels from `root` over local graph h restricted to active vertices.
int32_t bfs_levels(const Graph &h, int32_t root, std::vector<int32_t> &level, std::vector<int32_t> &queue) {
    std::fill(level.begin(), level.end(), -1);
    queue.clear();
    queue.push_back(root);
    level[root] = 0;
    int32_t maxl = 0;
    for (size_t q = 0; q < queue.size(); q++) {
        int32_t v = queue[q];
        for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++) {
            int32_t u = h.adj[p];
            if (level[u] < 0) {
                level[u] = level[v] + 1;
                maxl = std::max(maxl, level[u]);
                queue.push_back(u);
            }
        }
    }
    return maxl;
}

}  // namespace

std::vector<int32_t> order_nd(const Graph &g, int32_t leaf, double dense_factor) {
    const int32_t N = g.N;
    std::vector<int32_t> order;
    order.reserve(N);
    if (N == 0) return order;
    leaf = std::max<int32_t>(leaf, 8);
    // dense vertices go last, as in order_amd
    const double thr = std::max(16.0, dense_factor * std::sqrt((double)N));
    std::vector<int32_t> dense, rest;
    for (int32_t i = 0; i < N; i++) {
        int64_t d = g.ptr[i + 1] - g.ptr[i];
        if (dense_factor > 0 && (double)d > thr) dense.push_back(i);
        else rest.push_back(i);
    }
    std::vector<int32_t> loc(N, -1), stampv(N, 0);
    int32_t stamp = 0;
    // explicit work stack: entries are either a vertex set to dissect or a
    // separator to emit after its two halves
    struct Item {
        std::vector<int32_t> verts;
        bool emit;
    };
    std::vector<Item> stack;
    stack.push_back({rest, false});
    std::vector<int32_t> level, queue, comp;
    while (!stack.empty()) {
        Item it = std::move(stack.back());
        stack.pop_back();
        if (it.emit) {
            for (int32_t v : it.verts) order.push_back(v);
            continue;
        }
        auto &vs = it.verts;
        if (vs.empty()) continue;
        ++stamp;
        Graph h = induced(g, vs, loc, stampv, stamp);
        const int32_t n = h.N;
        if (n <= leaf) {
            std::vector<int32_t> o = order_amd(h, 0.0);
            for (int32_t t : o) order.push_back(vs[t]);
            continue;
        }
        level.assign(n, -1);
        // connected components
        comp.assign(n, -1);
        int32_t ncomp = 0;
        std::vector<int32_t> csize;
        for (int32_t r = 0; r < n; r++) {
            if (comp[r] >= 0) continue;
            queue.clear();
            queue.push_back(r);
            comp[r] = ncomp;
            for (size_t q = 0; q < queue.size(); q++) {
                int32_t v = queue[q];
                for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++)
                    if (comp[h.adj[p]] < 0) {
                        comp[h.adj[p]] = ncomp;
                        queue.push_back(h.adj[p]);
                    }
            }
            csize.push_back((int32_t)queue.size());
            ncomp++;
        }
        if (ncomp > 1) {
            // independent components: dissect each separately (pushed in
            // reverse so that the lowest component is ordered first)
            std::vector<std::vector<int32_t>> parts(ncomp);
            for (int32_t t = 0; t < n; t++) parts[comp[t]].push_back(vs[t]);
            for (int32_t c = ncomp - 1; c >= 0; c--) stack.push_back({std::move(parts[c]), false});
            continue;
        }
        // pseudo-peripheral root
        int32_t root = 0;
        for (int32_t t = 1; t < n; t++)
            if (h.ptr[t + 1] - h.ptr[t] < h.ptr[root + 1] - h.ptr[root]) root = t;
        int32_t ecc = bfs_levels(h, root, level, queue);
        for (int iter = 0; iter < 6; iter++) {
            int32_t best = -1;
            for (int32_t t = 0; t < n; t++)
                if (level[t] == ecc && (best < 0 || h.ptr[t + 1] - h.ptr[t] < h.ptr[best + 1] - h.ptr[best])) best = t;
            std::vector<int32_t> lv2(n);
            int32_t e2 = bfs_levels(h, best, lv2, queue);
            if (e2 <= ecc) break;
            root = best;
            ecc = e2;
            level.swap(lv2);
        }
        if (ecc < 2) {
            std::vector<int32_t> o = order_amd(h, 0.0);
            for (int32_t t : o) order.push_back(vs[t]);
            continue;
        }
        std::vector<int64_t> cnt(ecc + 2, 0);
        for (int32_t t = 0; t < n; t++) cnt[level[t]]++;
        // candidate separators: vertices of level l adjacent to level l+1
        // ("low side") or of level l+1 adjacent to level l ("high side")
        std::vector<int64_t> lo_sep(ecc + 1, 0), hi_sep(ecc + 1, 0);
        {
            std::vector<int8_t> adj_up(n, 0), adj_dn(n, 0);
            for (int32_t v = 0; v < n; v++)
                for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++) {
                    int32_t u = h.adj[p];
                    if (level[u] == level[v] + 1) adj_up[v] = 1;
                    if (level[u] == level[v] - 1) adj_dn[v] = 1;
                }
            for (int32_t v = 0; v < n; v++) {
                if (adj_up[v]) lo_sep[level[v]]++;
                if (adj_dn[v] && level[v] >= 1) hi_sep[level[v] - 1]++;
            }
        }
        double best_score = 1e300;
        int32_t best_l = -1, best_side = 0;
        int64_t below = 0;
        for (int32_t l = 0; l < ecc; l++) {
            // split between level l and l+1
            int64_t left = below + cnt[l];  // levels <= l
            int64_t right = n - left;
            below += cnt[l];
            for (int side = 0; side < 2; side++) {
                int64_t sep = side == 0 ? lo_sep[l] : hi_sep[l];
                int64_t a = side == 0 ? left - sep : left;
                int64_t b = side == 0 ? right : right - sep;
                if (a <= 0 || b <= 0) continue;
                double mn = (double)std::min(a, b), mx = (double)std::max(a, b);
                if (mn < 0.2 * (double)n) continue;
                double score = (double)sep * (1.0 + 0.5 * (mx - mn) / (double)n);
                if (score < best_score) {
                    best_score = score;
                    best_l = l;
                    best_side = side;
                }
            }
        }
        if (best_l < 0) {
            std::vector<int32_t> o = order_amd(h, 0.0);
            for (int32_t t : o) order.push_back(vs[t]);
            continue;
        }
        std::vector<int32_t> P1, P2, S;
        for (int32_t v = 0; v < n; v++) {
            int32_t lv = level[v];
            bool in_sep = false;
            if (best_side == 0 && lv == best_l) {
                for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++)
                    if (level[h.adj[p]] == lv + 1) { in_sep = true; break; }
            } else if (best_side == 1 && lv == best_l + 1) {
                for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++)
                    if (level[h.adj[p]] == lv - 1) { in_sep = true; break; }
            }
            if (in_sep) S.push_back(vs[v]);
            else if (lv <= best_l) P1.push_back(vs[v]);
            else P2.push_back(vs[v]);
        }
        // order: P1, P2, then the separator
        stack.push_back({std::move(S), true});
        stack.push_back({std::move(P2), false});
        stack.push_back({std::move(P1), false});
    }
    for (int32_t v : dense) order.push_back(v);
    return order;
}

}  // namespace ipm
