// Host-side analysis results shared by the library's host and device code.
// Everything here is computed once per pattern by analyse.cpp (Sec. 4.2-4.3 of
// Zanetti & Gondzio, arXiv 2508.04370) and uploaded to the device.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ipm {

// Symmetric adjacency (no diagonal) of an N x N pattern, CSR.
struct Graph {
    int32_t N = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
};

// Orderings (ordering.cpp).  All return perm with perm[new] = old.
std::vector<int32_t> order_amd(const Graph &g, double dense_factor);
std::vector<int32_t> order_nd(const Graph &g, int32_t leaf, double dense_factor);

// Front size classes.
constexpr int32_t kSmallFrontMax = 128;  // fronts with f <= this can run fully in shared memory
// A level with fewer than kPromoteBelow fronts of f in (kPromoteMin, kSmallFrontMax]
// sends them to the multi-CTA large-front path: one SM per such front would
// leave most of the GPU idle while it works through the front's flops.
constexpr int32_t kPromoteMin = 64;
constexpr int32_t kPromoteBelow = 152;

struct Plan {
    // problem
    int32_t m = 0, n = 0, N = 0, form = 1, ordering = 0;
    std::vector<int64_t> Acp;  // CSC of A as given
    std::vector<int32_t> Ari;
    // batch bookkeeping (empty for a single LP): instance of every unknown,
    // indexed in the factorisation order
    int32_t batch_count = 0;
    std::vector<int32_t> inst;

    // symbolic, factorisation order
    std::vector<int32_t> perm, iperm, parent;
    std::vector<int64_t> colcount;
    int32_t nsuper = 0;
    std::vector<int32_t> sn_start, sn_parent;
    std::vector<int64_t> sn_rptr;
    std::vector<int32_t> sn_rows;  // global (new) row indices, sorted, first k = columns

    // per-supernode numeric layout
    std::vector<int32_t> sn_k, sn_f, sn_ld, sn_level;
    std::vector<int64_t> sn_off;      // offset of the f x ld slab in the front arena (doubles)
    int64_t front_doubles = 0;
    std::vector<int32_t> child_ptr, child_list;  // children, ascending
    std::vector<int64_t> map_off;     // this supernode's contribution rows -> parent local rows
    std::vector<int32_t> relmap;
    std::vector<int64_t> orig_ptr;    // original entries: per supernode
    std::vector<int32_t> orig_dst;    // local offset col*ld + row
    std::vector<int64_t> orig_src;    // >= 0: value index; < 0: -1-j primal diagonal of column j
    std::vector<int32_t> sign;        // expected pivot sign per new index (-1 primal / +1 dual)

    // levels (leaves first); supernodes of a level split into small / large
    int32_t nlevels = 0;
    std::vector<int32_t> lvl_small_ptr, lvl_small;  // small fronts per level
    std::vector<int32_t> lvl_large_ptr, lvl_large;  // large fronts per level
    std::vector<int8_t> sn_large;                    // 1: the front runs on the large-front path

    // solve buffers: per supernode offset of its contribution vector (length f-k)
    std::vector<int64_t> upd_off;
    int64_t upd_total = 0;

    // statistics
    int64_t nnzL = 0, nnzK_lower = 0;
    double flops = 0.0;
    double amalg_zero_frac = 0.0;  // the amalgamation threshold used (chosen when the option is < 0)
    int32_t max_f = 0, max_k = 0;
    int32_t nsmall = 0, nlarge = 0;

    // normal equations: lower entries of M = A Theta~ A^T in original
    // numbering (CSC, rows >= column) and, for each entry (r, i), the A-entry
    // pairs (a_rj, a_ij) contributing to it, in ascending column j
    std::vector<int64_t> ne_cp;
    std::vector<int32_t> ne_ri;
    std::vector<int64_t> ne_tptr;     // per NE entry: range in ne_ta/ne_tb/ne_tj
    std::vector<int32_t> ne_ta, ne_tb;  // A value indices of a_rj and a_ij
    std::vector<int32_t> ne_tj;         // the column j
    // chooser record
    double est_as = 0.0, est_ne = 0.0;
    int64_t nnz_ne_seen = 0;
};

// Largest number of (a_rj, a_ij) pairs the normal equations may need; a
// pattern beyond it is not formed (dense rows of A make A A^T expensive).
constexpr int64_t kMaxNePairs = int64_t(1) << 28;

// Entries of the lower part of A A^T (with diagonal), counting stops once it
// exceeds `limit` (returns limit + 1 then).
int64_t count_ne_lower(int32_t m, int32_t n, const int64_t *colptr, const int32_t *rowidx, int64_t limit);

struct AnalyseOptions {
    int32_t nb = 32;
    int32_t amalg_width = 16;
    double amalg_zero_frac = 0.05;  // < 0: choose 0.1 or 0.2 by the modelled factorisation time
    int32_t nd_leaf = 128;
    double dense_row_factor = 10.0;
    int32_t verbose = 0;
};

// Analysis checkpoint (analysis_io.cpp): 0 on success, -1 with err set.
int plan_save(const Plan &plan, const std::string &path, std::string &err);
int plan_load(Plan &plan, const std::string &path, std::string &err);

// Returns 0 or a negative IPM error code; fills plan.
int analyse(Plan &plan, int32_t m, int32_t n, const int64_t *colptr, const int32_t *rowidx, int32_t form,
            int32_t ordering, const int32_t *user_perm, const AnalyseOptions &opt, std::string &err);

}  // namespace ipm
