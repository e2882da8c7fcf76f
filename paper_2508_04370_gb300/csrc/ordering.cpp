// Fill-reducing orderings for the symbolic analysis (Sec. 4.2).
//
// order_amd: approximate minimum degree on a quotient graph, after Amestoy,
//   Davis and Duff (SIAM J. Matrix Anal. Appl. 17, 1996): variables and
//   elements, the approximate external degree bound
//       d_i <- min( n_left - |i|,  d_i + |L_p \ i|,  |A_i \ i| + |L_p \ i| + sum_{e in E_i \ p} |L_e \ L_p| ),
//   aggressive element absorption (|L_e \ L_p| = 0), supervariable detection
//   by hashing, and dense rows (degree > max(16, f*sqrt(N))) ordered last.
// order_nd: nested dissection by recursive vertex separators; each subgraph
//   takes the best (separator / side x side) of a separator from
//   breadth-first level structures and multilevel separators (heavy-edge
//   coarsening, separators grown on the coarsest graph, vertex
//   Fiduccia-Mattheyses refinement on the way back), computed on worker
//   threads; subgraphs below the leaf size are ordered with order_amd.  The
//   subsets left after the first dissection steps are dissected on worker
//   threads; the order does not depend on them.  The paper uses Metis
//   (Sec. 4.2); this is a self-contained replacement.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <system_error>
#include <thread>
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

// Smallest vertex separator for a given edge cut: the cut edges form a
// bipartite graph between the boundary vertices of the two sides, and its
// minimum vertex cover (Konig's theorem: from a maximum matching, the
// unmatched low-side vertices and everything reachable from them by
// alternating paths, Z; cover = (low \ Z) + (high intersect Z)) separates
// the sides with the fewest vertices.  side[v]: 1 or 2 for every vertex.
// Returns the cover as part[] (0 for cover vertices, else the side).
int64_t cover_separator(const Graph &h, const std::vector<int8_t> &side, std::vector<int8_t> &part) {
    const int32_t n = h.N;
    part.assign(side.begin(), side.end());
    // boundary vertices and their cut edges
    std::vector<int32_t> lows, idx(n, -1);
    for (int32_t v = 0; v < n; v++) {
        if (side[v] != 1) continue;
        for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++)
            if (side[h.adj[p]] == 2) {
                idx[v] = (int32_t)lows.size();
                lows.push_back(v);
                break;
            }
    }
    std::vector<int32_t> mate_hi(n, -1), mate_lo(lows.size(), -1), seen(n, -1);
    // augmenting paths by iterative depth-first search (Kuhn): frame t holds a
    // low vertex and its next edge; via[t] is the high vertex leading from
    // frame t to frame t+1 (matched to frame t+1's low vertex)
    struct Frame {
        int32_t li;
        int64_t pos;
    };
    std::vector<Frame> frames;
    std::vector<int32_t> via;
    for (int32_t i = 0; i < (int32_t)lows.size(); i++) {
        frames.assign(1, {i, h.ptr[lows[i]]});
        via.clear();
        while (!frames.empty()) {
            Frame &fr = frames.back();
            const int32_t v = lows[fr.li];
            if (fr.pos >= h.ptr[v + 1]) {  // dead end
                frames.pop_back();
                if (!via.empty()) via.pop_back();
                continue;
            }
            const int32_t u = h.adj[fr.pos++];
            if (side[u] != 2 || seen[u] == i) continue;
            seen[u] = i;
            if (mate_hi[u] < 0) {  // free: flip the path
                via.push_back(u);
                for (size_t t = 0; t < frames.size(); t++) {
                    mate_lo[frames[t].li] = via[t];
                    mate_hi[via[t]] = frames[t].li;
                }
                break;
            }
            via.push_back(u);
            frames.push_back({mate_hi[u], h.ptr[lows[mate_hi[u]]]});
        }
    }
    // Konig: alternating reachability from unmatched low vertices
    std::vector<char> zl(lows.size(), 0), zh(n, 0);
    std::vector<int32_t> q;
    for (int32_t i = 0; i < (int32_t)lows.size(); i++)
        if (mate_lo[i] < 0) {
            zl[i] = 1;
            q.push_back(i);
        }
    for (size_t t = 0; t < q.size(); t++) {
        const int32_t v = lows[q[t]];
        for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++) {
            const int32_t u = h.adj[p];
            if (side[u] != 2 || zh[u]) continue;
            zh[u] = 1;
            const int32_t m = mate_hi[u];
            if (m >= 0 && !zl[m]) {
                zl[m] = 1;
                q.push_back(m);
            }
        }
    }
    int64_t size = 0;
    for (int32_t i = 0; i < (int32_t)lows.size(); i++)
        if (!zl[i]) {
            part[lows[i]] = 0;
            size++;
        }
    for (int32_t u = 0; u < n; u++)
        if (zh[u] && side[u] == 2) {
            part[u] = 0;
            size++;
        }
    return size;
}

// Vertex-separator refinement (Fiduccia-Mattheyses moves on a vertex
// separator, the node-based refinement of multilevel nested dissection):
// moving a separator vertex v into side a pulls its neighbours on the other
// side b into the separator, so the separator changes by w(N(v) on b) - w(v)
// (w = 1 without vertex weights; with weights vw, the number of vertices a
// coarse vertex stands for).  A pass repeatedly makes the best admissible
// move (each vertex moves out of the separator at most once per pass; moves
// that do not shrink the separator are allowed), then rolls back to the
// smallest separator it saw; it gives up after min(max(n/100, 15), 100) moves
// without a new best.  The weight of each vertex's neighbours on either side
// is kept up to date, so a move costs its neighbours' degrees.  part[v]: 0
// separator, 1 or 2 a side.  The larger side stays within max(its initial
// share, 60%) of both sides.
void refine_separator(const Graph &h, std::vector<int8_t> &part, int max_passes,
                      const std::vector<int32_t> *vw = nullptr) {
    const int32_t n = h.N;
    auto wt = [&](int32_t v) -> int64_t { return vw ? (*vw)[v] : 1; };
    int64_t cnt[3] = {0, 0, 0};
    for (int32_t v = 0; v < n; v++) cnt[part[v]] += wt(v);
    const double share = std::max(0.6, (double)std::max(cnt[1], cnt[2]) / (double)std::max<int64_t>(1, cnt[1] + cnt[2]));
    const size_t patience = (size_t)std::min<int64_t>(std::max<int64_t>(n / 100, 15), 100);
    struct Mv {
        int32_t v;
        int8_t from, to;
    };
    struct Cand {
        int64_t gain;
        int32_t v;
        int8_t side;
        bool operator<(const Cand &o) const { return gain < o.gain || (gain == o.gain && v > o.v); }
    };
    std::vector<char> locked(n);
    std::vector<int64_t> conn(2 * (size_t)n);  // conn[2v + s - 1]: weight of v's neighbours on side s
    std::vector<Mv> log;
    std::vector<Cand> heap;
    auto gain_of = [&](int32_t v, int8_t a) { return wt(v) - conn[2 * (size_t)v + (2 - a)]; };
    auto push = [&](int32_t v) {
        if (part[v] != 0 || locked[v]) return;
        for (int8_t a = 1; a <= 2; a++) {
            heap.push_back({gain_of(v, a), v, a});
            std::push_heap(heap.begin(), heap.end());
        }
    };
    for (int pass = 0; pass < max_passes; pass++) {
        std::fill(locked.begin(), locked.end(), 0);
        std::fill(conn.begin(), conn.end(), 0);
        for (int32_t v = 0; v < n; v++)
            for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++) {
                const int8_t s = part[h.adj[p]];
                if (s) conn[2 * (size_t)v + s - 1] += wt(h.adj[p]);
            }
        log.clear();
        heap.clear();
        for (int32_t v = 0; v < n; v++)
            if (part[v] == 0) push(v);
        const int64_t start_sep = cnt[0];
        int64_t best_sep = cnt[0];
        size_t best_len = 0;
        while (!heap.empty()) {
            std::pop_heap(heap.begin(), heap.end());
            const Cand c = heap.back();
            heap.pop_back();
            if (part[c.v] != 0 || locked[c.v] || gain_of(c.v, c.side) != c.gain) continue;  // stale
            const int8_t a = c.side, b = (int8_t)(3 - a);
            const int64_t ca = cnt[a] + wt(c.v), cb = cnt[b] - conn[2 * (size_t)c.v + b - 1];
            if (cb <= 0 || (double)std::max(ca, cb) > share * (double)(ca + cb)) continue;
            part[c.v] = a;
            locked[c.v] = 1;
            cnt[0] -= wt(c.v);
            cnt[a] += wt(c.v);
            log.push_back({c.v, 0, a});
            for (int64_t p = h.ptr[c.v]; p < h.ptr[c.v + 1]; p++) {
                const int32_t u = h.adj[p];
                conn[2 * (size_t)u + a - 1] += wt(c.v);
                push(u);  // a separator neighbour now pulls more when it moves to b
            }
            for (int64_t p = h.ptr[c.v]; p < h.ptr[c.v + 1]; p++) {
                const int32_t u = h.adj[p];
                if (part[u] != b) continue;
                part[u] = 0;  // pulled into the separator
                cnt[b] -= wt(u);
                cnt[0] += wt(u);
                log.push_back({u, b, 0});
                for (int64_t q = h.ptr[u]; q < h.ptr[u + 1]; q++) {
                    const int32_t z = h.adj[q];
                    conn[2 * (size_t)z + b - 1] -= wt(u);
                    push(z);
                }
                push(u);
            }
            if (cnt[0] < best_sep) {
                best_sep = cnt[0];
                best_len = log.size();
            }
            if (log.size() > best_len + patience) break;  // long enough without improvement
        }
        for (size_t t = log.size(); t > best_len; t--) {
            const Mv &m = log[t - 1];
            cnt[m.to] -= wt(m.v);
            cnt[m.from] += wt(m.v);
            part[m.v] = m.from;
        }
        if (best_sep >= start_sep) break;
    }
}

// Level-structure separator: breadth-first levels from a pseudo-peripheral
// vertex; the few most promising cuts between consecutive levels get their
// optimal vertex separator (cover_separator), the best by separator /
// (side x side) is refined.  h must be connected with more than one level.
bool level_separator(const Graph &h, std::vector<int8_t> &part, std::vector<int32_t> &level,
                     std::vector<int32_t> &queue) {
    const int32_t n = h.N;
    level.assign(n, -1);
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
    if (ecc < 2) return false;
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
    // candidate cuts between level l and l+1 with both sides at least 20% of
    // the vertices; the cheap one-sided separator estimates rank them and
    // the best few get their optimal vertex separator (minimum cover of
    // the cut edges)
    std::vector<std::pair<double, int32_t>> cands;
    int64_t below = 0;
    for (int32_t l = 0; l < ecc; l++) {
        const int64_t left = below + cnt[l], right = n - left;
        below += cnt[l];
        const int64_t sep = std::min(lo_sep[l], hi_sep[l]);
        if (std::min(left, right) - sep < (int64_t)(0.2 * n)) continue;
        cands.push_back({(double)sep / ((double)(left - sep) * (double)(right - sep) + 1.0), l});
    }
    if (cands.empty()) return false;
    std::sort(cands.begin(), cands.end());
    if (cands.size() > 6) cands.resize(6);
    std::vector<int8_t> trial, sidev(n);
    part.clear();
    double best_score = 1e300;
    for (const auto &cd : cands) {
        const int32_t l = cd.second;
        for (int32_t v = 0; v < n; v++) sidev[v] = level[v] <= l ? 1 : 2;
        const int64_t sep = cover_separator(h, sidev, trial);
        int64_t c1 = 0;
        for (int32_t v = 0; v < n; v++) c1 += trial[v] == 1;
        const int64_t c2 = n - sep - c1;
        if (c1 <= 0 || c2 <= 0) continue;
        const double score = (double)sep / ((double)c1 * (double)c2);
        if (score < best_score) {
            best_score = score;
            part.swap(trial);
        }
    }
    if (part.empty()) return false;
    refine_separator(h, part, 8);
    return true;
}

// separator / (side x side) of a partition (0 separator, 1 or 2 a side);
// +inf when a side is empty
double separator_ratio(const std::vector<int8_t> &part) {
    int64_t c[3] = {0, 0, 0};
    for (int8_t p : part) c[p]++;
    if (c[1] == 0 || c[2] == 0) return 1e300;
    return (double)c[0] / ((double)c[1] * (double)c[2]);
}

// splitmix64: deterministic visit orders and seeds
uint64_t next_random(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One level of the multilevel scheme: a graph with edge weights (parallel to
// g.adj: how many finer edges an edge stands for) and vertex weights (how many
// original vertices a vertex stands for); cmap sends a vertex to its vertex
// on the next coarser level.
struct MLevel {
    Graph g;
    std::vector<int32_t> ew, vw, cmap;
};

// Heavy-edge matching: vertices in a shuffled order are paired with the
// unmatched neighbour across their heaviest edge (ties: the lighter
// neighbour), keeping coarse vertex weights <= max_vw; pairs and unmatched
// vertices become the coarse vertices, parallel edges merge with summed
// weights.  Returns false when the graph shrinks by less than 10%.
bool coarsen(MLevel &f, MLevel &c, int64_t max_vw, uint64_t &rng) {
    const int32_t n = f.g.N;
    std::vector<int32_t> order(n), mate(n, -1);
    std::iota(order.begin(), order.end(), 0);
    for (int32_t i = n - 1; i > 0; i--) std::swap(order[i], order[(int32_t)(next_random(rng) % (uint64_t)(i + 1))]);
    for (int32_t v : order) {
        if (mate[v] >= 0) continue;
        int32_t best = -1;
        for (int64_t p = f.g.ptr[v]; p < f.g.ptr[v + 1]; p++) {
            const int32_t u = f.g.adj[p];
            if (mate[u] >= 0 || u == v || (int64_t)f.vw[v] + f.vw[u] > max_vw) continue;
            if (best < 0 || f.ew[p] > f.ew[best] || (f.ew[p] == f.ew[best] && f.vw[u] < f.vw[f.g.adj[best]])) best = (int32_t)p;
        }
        if (best >= 0) {
            mate[v] = f.g.adj[best];
            mate[f.g.adj[best]] = v;
        } else {
            mate[v] = v;
        }
    }
    f.cmap.assign(n, -1);
    int32_t nc = 0;
    for (int32_t v = 0; v < n; v++)
        if (f.cmap[v] < 0) {
            f.cmap[v] = nc;
            f.cmap[mate[v]] = nc;
            nc++;
        }
    if ((double)nc > 0.9 * (double)n) return false;
    c.g.N = nc;
    c.g.ptr.assign(nc + 1, 0);
    c.g.adj.clear();
    c.ew.clear();
    c.vw.assign(nc, 0);
    std::vector<int64_t> pos(nc, -1);
    for (int32_t v = 0; v < n; v++) {
        if (mate[v] < v) continue;  // the pair is built from its lower vertex, in coarse order
        const int32_t cv = f.cmap[v];
        const int64_t start = (int64_t)c.g.adj.size();
        for (int t = 0; t < (mate[v] == v ? 1 : 2); t++) {
            const int32_t w = t == 0 ? v : mate[v];
            c.vw[cv] += f.vw[w];
            for (int64_t p = f.g.ptr[w]; p < f.g.ptr[w + 1]; p++) {
                const int32_t cu = f.cmap[f.g.adj[p]];
                if (cu == cv) continue;
                if (pos[cu] >= start) {
                    c.ew[pos[cu]] += f.ew[p];
                } else {
                    pos[cu] = (int64_t)c.g.adj.size();
                    c.g.adj.push_back(cu);
                    c.ew.push_back(f.ew[p]);
                }
            }
        }
        c.g.ptr[cv + 1] = (int64_t)c.g.adj.size();
    }
    return true;
}

// Multilevel vertex separator of a connected graph h (the scheme of
// multilevel nested dissection): coarsen by heavy-edge matching to about 100
// vertices; on the coarsest graph grow breadth-first regions of half the
// weight from several seeds, take the minimum vertex cover of each region's
// cut edges and refine it by weighted moves, keeping the best by separator /
// (side x side); project it back level by level (a coarse separator stays a
// separator) with weighted refinement at each level.  run seeds the shuffles.
bool multilevel_separator(const Graph &h, std::vector<int8_t> &part, int run) {
    const int32_t n = h.N;
    if (n < 16) return false;
    std::vector<MLevel> lv(1);
    lv[0].g = h;
    lv[0].ew.assign(h.adj.size(), 1);
    lv[0].vw.assign(n, 1);
    constexpr int32_t kCoarsest = 100;
    const int64_t max_vw = std::max<int64_t>(1, (int64_t)(1.5 * (double)n / kCoarsest));
    uint64_t rng = 0x243F6A8885A308D3ull ^ (uint64_t)n ^ ((uint64_t)run << 40);
    while (lv.back().g.N > kCoarsest && lv.size() < 40) {
        MLevel c;
        if (!coarsen(lv.back(), c, max_vw, rng)) break;
        lv.push_back(std::move(c));
    }
    // initial separators on the coarsest graph
    const MLevel &C = lv.back();
    const int32_t nc = C.g.N;
    int64_t total = 0;
    for (int32_t w : C.vw) total += w;
    std::vector<int8_t> best, side(nc), trial;
    double best_score = 1e300;
    std::vector<int32_t> level(nc), queue;
    constexpr int kTrials = 8;
    for (int t = 0; t < kTrials; t++) {
        int32_t seed;
        if (t == 0) {  // far end of a breadth-first search from vertex 0
            bfs_levels(C.g, 0, level, queue);
            seed = queue.back();
        } else {
            seed = (int32_t)(next_random(rng) % (uint64_t)nc);
        }
        std::fill(side.begin(), side.end(), 2);
        bfs_levels(C.g, seed, level, queue);
        int64_t w1 = 0;
        for (size_t q = 0; q < queue.size() && 2 * w1 < total; q++) {
            side[queue[q]] = 1;
            w1 += C.vw[queue[q]];
        }
        if (w1 == 0 || w1 >= total) continue;
        cover_separator(C.g, side, trial);
        refine_separator(C.g, trial, 8, &C.vw);
        int64_t c[3] = {0, 0, 0};
        for (int32_t v = 0; v < nc; v++) c[trial[v]] += C.vw[v];
        if (c[1] == 0 || c[2] == 0) continue;
        const double score = (double)c[0] / ((double)c[1] * (double)c[2]);
        if (score < best_score) {
            best_score = score;
            best.swap(trial);
        }
    }
    if (best.empty()) return false;
    // project back with refinement
    for (int l = (int)lv.size() - 2; l >= 0; l--) {
        const MLevel &F = lv[l];
        std::vector<int8_t> fp(F.g.N);
        for (int32_t v = 0; v < F.g.N; v++) fp[v] = best[F.cmap[v]];
        refine_separator(F.g, fp, 8, &F.vw);
        best.swap(fp);
    }
    int64_t c1 = 0, c2 = 0;
    for (int8_t p : best) {
        c1 += p == 1;
        c2 += p == 2;
    }
    if (c1 == 0 || c2 == 0) return false;
    part.swap(best);
    return true;
}
}  // namespace

namespace {

// Per-thread scratch of the dissection: global -> local maps of the induced
// subgraphs and the breadth-first buffers.
struct NdScratch {
    std::vector<int32_t> loc, stampv, level, queue, comp;
    int32_t stamp = 0;
    explicit NdScratch(int32_t N) : loc(N, -1), stampv(N, 0) {}
};

// One dissection step on the vertex set vs (global ids of g).  Either vs is
// ordered outright (a leaf, or a subgraph without a separator: order_amd),
// or it splits into parts to dissect in turn, in order, followed by the
// separator (connected components have none).
struct NdStep {
    bool ordered = false;
    std::vector<int32_t> order;
    std::vector<std::vector<int32_t>> parts;
    bool has_sep = false;
    std::vector<int32_t> sep;
};

NdStep nd_step(const Graph &g, const std::vector<int32_t> &vs, int32_t leaf, NdScratch &w) {
    NdStep out;
    Graph h = induced(g, vs, w.loc, w.stampv, ++w.stamp);
    const int32_t n = h.N;
    auto by_amd = [&]() {
        out.ordered = true;
        for (int32_t t : order_amd(h, 0.0)) out.order.push_back(vs[t]);
        return out;
    };
    if (n <= leaf) return by_amd();
    // connected components: dissected separately, lowest first
    w.comp.assign(n, -1);
    int32_t ncomp = 0;
    for (int32_t r = 0; r < n; r++) {
        if (w.comp[r] >= 0) continue;
        w.queue.clear();
        w.queue.push_back(r);
        w.comp[r] = ncomp;
        for (size_t q = 0; q < w.queue.size(); q++) {
            int32_t v = w.queue[q];
            for (int64_t p = h.ptr[v]; p < h.ptr[v + 1]; p++)
                if (w.comp[h.adj[p]] < 0) {
                    w.comp[h.adj[p]] = ncomp;
                    w.queue.push_back(h.adj[p]);
                }
        }
        ncomp++;
    }
    if (ncomp > 1) {
        out.parts.assign(ncomp, {});
        for (int32_t t = 0; t < n; t++) out.parts[w.comp[t]].push_back(vs[t]);
        return out;
    }
    // the level-structure separator and multilevel ones from differently
    // shuffled coarsenings (three above 5000 vertices, on their own
    // threads): the best ratio wins, ties to the earlier candidate
    const int runs = n > 5000 ? 3 : 1;
    std::vector<std::vector<int8_t>> mpart(runs);
    std::vector<char> mok(runs, 0);
    std::vector<std::thread> workers;
    if (runs > 1) {
        try {
            for (int r = 0; r < runs; r++)
                workers.emplace_back([&h, &mpart, &mok, r] {
                    try {  // a run that cannot allocate is dropped, not fatal
                        mok[r] = multilevel_separator(h, mpart[r], r);
                    } catch (...) {
                        mok[r] = 0;
                    }
                });
        } catch (const std::system_error &) {
            for (auto &t : workers) t.join();
            workers.clear();
            std::fill(mok.begin(), mok.end(), 0);
            for (int r = 0; r < runs; r++) mok[r] = multilevel_separator(h, mpart[r], r);
        }
    } else {
        mok[0] = multilevel_separator(h, mpart[0], 0);
    }
    w.level.assign(n, -1);
    std::vector<int8_t> part;
    double best_ratio = level_separator(h, part, w.level, w.queue) ? separator_ratio(part) : 1e300;
    for (auto &t : workers) t.join();
    for (int r = 0; r < runs; r++)
        if (mok[r] && separator_ratio(mpart[r]) < best_ratio) {
            best_ratio = separator_ratio(mpart[r]);
            part.swap(mpart[r]);
        }
    if (part.empty()) return by_amd();
    // order: P1, P2, then the separator
    out.parts.assign(2, {});
    out.has_sep = true;
    for (int32_t v = 0; v < n; v++) (part[v] == 0 ? out.sep : out.parts[part[v] - 1]).push_back(vs[v]);
    return out;
}

// Nested dissection of vs, appended to order: depth first with an explicit
// stack (a part's whole subtree before the next part, each separator after
// its parts).
void nd_serial(const Graph &g, std::vector<int32_t> vs, int32_t leaf, NdScratch &w, std::vector<int32_t> &order) {
    struct Item {
        std::vector<int32_t> verts;
        bool emit;
    };
    std::vector<Item> stack;
    stack.push_back({std::move(vs), false});
    while (!stack.empty()) {
        Item it = std::move(stack.back());
        stack.pop_back();
        if (it.emit) {
            order.insert(order.end(), it.verts.begin(), it.verts.end());
            continue;
        }
        if (it.verts.empty()) continue;
        NdStep st = nd_step(g, it.verts, leaf, w);
        if (st.ordered) {
            order.insert(order.end(), st.order.begin(), st.order.end());
            continue;
        }
        if (st.has_sep) stack.push_back({std::move(st.sep), true});
        for (size_t c = st.parts.size(); c-- > 0;) stack.push_back({std::move(st.parts[c]), false});
    }
}

// The first kNdTopLevels steps run here and leave a list of tasks in output
// order (sets still to dissect, or vertices already in their final order);
// the sets then run on worker threads.  Each set's order is a function of the
// set alone, so the result is the serial one whatever the threads do.
constexpr int kNdTopLevels = 3;
constexpr size_t kNdParallelMin = 20000;

struct NdTask {
    std::vector<int32_t> verts;
    bool done;  // verts already ordered (a separator, or a set ordered outright)
};

void nd_expand(const Graph &g, std::vector<int32_t> vs, int32_t leaf, int depth, NdScratch &w,
               std::vector<NdTask> &tasks) {
    if (vs.empty()) return;
    if (depth == 0 || vs.size() < kNdParallelMin) {
        tasks.push_back({std::move(vs), false});
        return;
    }
    NdStep st = nd_step(g, vs, leaf, w);
    if (st.ordered) {
        tasks.push_back({std::move(st.order), true});
        return;
    }
    for (auto &part : st.parts) nd_expand(g, std::move(part), leaf, depth - 1, w, tasks);
    if (st.has_sep) tasks.push_back({std::move(st.sep), true});
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
    NdScratch main_w(N);
    std::vector<NdTask> tasks;
    nd_expand(g, std::move(rest), leaf, kNdTopLevels, main_w, tasks);
    std::vector<std::vector<int32_t>> sub(tasks.size());
    std::vector<std::thread> workers;
    std::vector<size_t> serial;
    for (size_t t = 0; t < tasks.size(); t++) {
        if (tasks[t].done) continue;
        bool started = false;
        if (tasks[t].verts.size() >= kNdParallelMin / 4) {
            try {
                workers.emplace_back([&g, &tasks, &sub, t, leaf, N] {
                    try {
                        NdScratch w(N);
                        nd_serial(g, tasks[t].verts, leaf, w, sub[t]);
                    } catch (...) {
                        sub[t].clear();  // redone serially below
                    }
                });
                started = true;
            } catch (const std::system_error &) {
            }
        }
        if (!started) serial.push_back(t);
    }
    for (size_t t : serial) nd_serial(g, tasks[t].verts, leaf, main_w, sub[t]);
    for (auto &th : workers) th.join();
    for (size_t t = 0; t < tasks.size(); t++) {
        if (tasks[t].done) {
            order.insert(order.end(), tasks[t].verts.begin(), tasks[t].verts.end());
            continue;
        }
        if (sub[t].size() != tasks[t].verts.size()) {  // a worker failed: redo here
            sub[t].clear();
            nd_serial(g, tasks[t].verts, leaf, main_w, sub[t]);
        }
        order.insert(order.end(), sub[t].begin(), sub[t].end());
    }
    for (int32_t v : dense) order.push_back(v);
    return order;
}

}  // namespace ipm
