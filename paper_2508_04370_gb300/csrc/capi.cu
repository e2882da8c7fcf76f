// C ABI of the multifrontal factorise/solve library (include/ipm_mf.h).
// Host orchestration: device arena, plan upload, per-level launch sequence of
// the numeric factorisation (Sec. 4.1, 4.3-4.5 of Zanetti & Gondzio, arXiv
// 2508.04370) and of the solves with iterative refinement (Sec. 4.5).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ipm_mf.h"
#include "ipm_dev.h"
#include "ipm_plan.h"

using namespace ipm;

namespace {

// Algorithmic work of one launch (for the per-kernel roofline).
struct Work {
    double flops = 0.0, bytes = 0.0;
};
struct StepWork {
    int64_t asm_off;    // dependency order: assembly items of the fronts starting at this step
    int32_t asm_cnt;
    int32_t small_wait;  // dependency order: small-front level whose launch the assembly waits for (-1: none)
    int64_t panel_off;  // diagonal-block items (one per front)
    int32_t panel_cnt;
    int64_t trsm_off;   // row-chunk items below the diagonal blocks
    int32_t trsm_cnt;
    int64_t tile_off;   // FP64 update tiles: the first tile_cnt1 (strips) cover the next panel's
    int32_t tile_cnt;   // columns (lookahead, on the critical path), the rest the
    int32_t tile_cnt1;  // remaining trailing columns (a third stream)
    int64_t tc_off;   // tensor-core tiles (mixed precision, large fronts)
    int32_t tc_cnt;
    int64_t alt_off;  // FP64 tiles of the same fronts, used after a precision fallback
    int32_t alt_cnt;
    int32_t alt_cnt1;  // lookahead tiles among them
    int64_t st_off;   // sliced path: 128 x 32 output tiles; the first st_cnt1 cover the next panel's
    int32_t st_cnt;   // columns (critical path), the rest run beside the next panel
    int32_t st_cnt1;
    Work panel_w, trsm_w, tile_w, tile_w1, tc_w, alt_w, alt_w1, st_w1, st_w2, asm_w;
};
struct SmallClass {
    int64_t off;
    int32_t cnt, maxf;
    int32_t cls;  // size class: f <= 32, <= 64, <= 128
    Work w;
};
struct LevelWork {
    std::vector<SmallClass> small;  // small fronts of the level by size class
    int64_t all_off;
    int32_t all_cnt, all_maxf;
    int64_t asm_off;   // assembly items of the level's large fronts (the level kernel takes them all)
    int32_t asm_cnt;
    int64_t asm_off2;  // those of the fronts that go through the steps
    int32_t asm_cnt2;
    int64_t thin_off = 0;  // thin fronts, whole in one CTA each (k_thin_fronts)
    int32_t thin_cnt = 0;
    Work thin_w;
    std::vector<StepWork> steps;
    Work asm_w, fwd_w, bwd_w;
    int64_t lvl_off = 0;   // items of the persistent level kernel (FP64 large fronts)
    int32_t lvl_cnt = 0;
    int32_t lvl_ncnt = 0;  // its dependency counters
    bool has_tc = false;   // some front of the level has tensor-core update tiles
    // The level kernel pays off where a level's large fronts are bound by
    // their pivot chains (about 35 us per 32-column panel): a level takes it
    // when its FP64 front work at ~1 TFLOP/s is below tune_ratio times its
    // longest chain (0.5 unless ipm_autotune chose otherwise).  Levels with
    // more work run one launch per step at full occupancy.
    int32_t lvl_chain = 0;  // 32-column panels of the level's widest large front
    Work lvl_w;             // algorithmic work of the level's large fronts (assembly and factorisation)
};

struct ProfRec {
    int cls;
    cudaEvent_t e0, e1;
    double flops, bytes;
    cudaStream_t st;
};
// One profiled launch in issue order: class, stream index (in order of first
// use), start and end in ms from the first launch folded with it.
struct TraceRec {
    int32_t cls, stream;
    double t0, t1;
};


}  // namespace

struct ipm_ctx {
    ipm_options opt;
    Plan plan;
    bool analysed = false;
    bool dev_ready = false;
    bool values_set = false;
    bool factorised = false;
    std::vector<void *> allocs;
    int64_t device_bytes = 0;
    DevPlan dp{};
    DevCtl *ctl = nullptr;
    double *fronts = nullptr, *D = nullptr, *Dinv = nullptr, *dyn = nullptr;
    double *Doff = nullptr;      // pivoting mode: D(p+1, p) of 2x2 blocks
    int32_t *bsz = nullptr;      // pivoting mode: block sizes (1, 2, 0 at a 2x2 block's second position)
    int32_t *lperm = nullptr;    // pivoting mode: each front's interchanges (local index at each position)
    double *Ax = nullptr;
    double *theta = nullptr;  // owned copy for host entry points
    double *vf = nullptr, *vx = nullptr, *vbest = nullptr, *vr = nullptr, *vad = nullptr, *vae = nullptr,
           *vc = nullptr, *upd = nullptr;
    double *h_r7 = nullptr, *h_r1 = nullptr, *d_r7 = nullptr, *d_r1 = nullptr, *d_dx = nullptr, *d_dy = nullptr;
    int32_t *lvl_small = nullptr, *lvl_all = nullptr;
    int32_t *bwd_order = nullptr, *solve_sync = nullptr;
    SolveSched sched{};  // dependency-driven solve schedule (device pointers)
    int32_t solve_maxf = 0, solve_grid = 0;
    PanelItem *asm_items = nullptr, *panel_items = nullptr, *trsm_items = nullptr;
    AsmItem *asm_info = nullptr;
    int32_t *asm_cr = nullptr;
    int32_t *trsm_slots = nullptr;
    int32_t *trsm_sbase = nullptr;     // sliced path: first slice block of each TRSM item's front (-1: none)
    int32_t *thin_list = nullptr, *thin_asm = nullptr, *thin_slot = nullptr;  // thin fronts by level
    double *panel_ws = nullptr;
    TileItem *tile_items = nullptr, *tc_items = nullptr, *alt_items = nullptr;
    SlicedTile *sliced_tiles = nullptr;  // sliced tensor-core path: output tiles per step
    uint8_t *slice_ws = nullptr;       // digit images of a step: two halves, used by alternate steps
    int32_t *slice_exp = nullptr;      // their row scales (two halves)
    int64_t slice_half_blocks = 0;     // slice blocks per half
    FactorItem *lvl_items = nullptr;  // persistent level kernel: items of all levels
    InvItem *inv_items = nullptr;     // diagonal blocks inverted after each factorisation
    InvItem *pair_items = nullptr;    // blocks of multi-block supernodes (neighbour products)
    double *linv = nullptr;
    int32_t ninv = 0, npairs = 0;
    int32_t *lvl_sync = nullptr;      // its ticket and counters (1 + max counters of a level)
    int32_t lvl_grid = 1;  // CTAs of the level kernel: every SM full
    int32_t sms = 1;       // SMs of the device
    // choices of ipm_autotune: threads per small-front CTA by size class
    // (0: 32 / 64 / 128), the level-kernel threshold and the level kernel's
    // CTAs per SM (0: as many as fit).  One CTA per SM leaves each SM
    // sub-partition's FP64 pipe to one CTA's pivot chain; two keep more
    // trailing tiles in flight.
    int32_t tune_threads[3] = {0, 0, 0};
    double tune_ratio = 0.5;
    int32_t tune_lvl_per_sm = 0;
    double tune_ms = 0.0;
    bool mixed_active = false;  // tensor-core updates in use (mixed precision, no fallback yet)
    int32_t fallbacks = 0;
    double flops_tensor = 0.0;
    std::vector<LevelWork> levels;
    bool dep_sched = false;              // large fronts in the dependency order (else level by level)
    std::vector<StepWork> dsteps;        // its steps
    std::vector<int32_t> small_dep;      // per level: step whose completion its small fronts wait for (-1: none)
    int32_t steps_levels = 0, steps_dependency = 0;
    int32_t nfronts_thin = 0;
    std::vector<cudaEvent_t> done_ev;    // dependency order: end of each step on the critical stream
    // numeric state of the last factorisation
    double rho = 0.0, delta = 0.0;
    const double *theta_used = nullptr;
    // last solve
    DevCtl last{};
    int32_t refine_steps = 0;
    int32_t gmres_iters = 0;  // GMRES iterations of the last solve
    double *gm_V = nullptr, *gm_Z = nullptr, *gm_zero = nullptr, *gm_w = nullptr, *gm_part = nullptr,
           *gm_h = nullptr;
    GmDev *gm_dev = nullptr;            // device-side GMRES state of captured graphs
    cudaStream_t gm_stream = nullptr;   // captures the conditional GMRES body of a graph
    double omega = 0.0;      // reported backward error (on K)
    double omega_sys = 0.0;  // backward error of the refined system (K, or M for the normal equations)
    double omega_hist[16] = {0};
    int32_t status_acc = 0;
    int32_t nl_factor = 0, nl_solve = 0;
    double ms_analyse = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool graph_solved = false;  // the last solve ran inside a graph (info comes from the device)
    int32_t graph_kernels = 0;  // kernel nodes of the captured graph
    cudaStream_t cap_stream = nullptr;  // private stream used only for capturing
    cudaStream_t side = nullptr;        // large fronts of a level run here, beside the small fronts
    cudaStream_t side2 = nullptr;       // trailing updates beside the next panel (lookahead)
    cudaStream_t cls[2] = {nullptr, nullptr};  // the 2nd and 3rd small-front size classes of a level
    std::vector<cudaEvent_t> dep_ev;    // level-to-level dependencies between the streams
    std::vector<cudaEvent_t> step_ev;   // per-step fork/join of the trailing updates
    // normal equations
    NeView ne{};
    double *kf = nullptr, *kr = nullptr, *kad = nullptr, *kae = nullptr;  // K-sized scratch for omega on K
    // per-kernel-class measurement
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfRec> prof_pending;
    std::vector<TraceRec> trace;              // launches folded since the last ipm_kernel_trace
    std::vector<cudaStream_t> trace_streams;  // stream indices of the trace
    ipm_kernel_stat prof_tot[IPM_K_COUNT] = {};
    Work resid_w;
};

namespace {

int to_err(cudaError_t e) { return e == cudaSuccess ? IPM_OK : (e == cudaErrorMemoryAllocation ? IPM_ERR_OOM : IPM_ERR_CUDA); }

cudaEvent_t next_event(ipm_ctx *c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// Brackets one launch with events on its stream when profiling is enabled.
struct Prof {
    ipm_ctx *c;
    int cls;
    double flops, bytes;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr;
    Prof(ipm_ctx *c_, int cls_, const Work &w, cudaStream_t st_) : c(c_), cls(cls_), flops(w.flops), bytes(w.bytes), st(st_) {
        if (c->prof_on) {
            e0 = next_event(c);
            cudaEventRecord(e0, st);
        }
    }
    ~Prof() {
        if (c->prof_on) {
            cudaEvent_t e1 = next_event(c);
            cudaEventRecord(e1, st);
            c->prof_pending.push_back({cls, e0, e1, flops, bytes, st});
        }
    }
};

void fold_profile(ipm_ctx *c) {
    const cudaEvent_t base = c->prof_pending.empty() ? nullptr : c->prof_pending.front().e0;
    for (const ProfRec &r : c->prof_pending) {
        float ms = 0.f, a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        ipm_kernel_stat &t = c->prof_tot[r.cls];
        t.launches++;
        t.ms += ms;
        t.flops += r.flops;
        t.bytes += r.bytes;
        if (cudaEventElapsedTime(&a, base, r.e0) != cudaSuccess || cudaEventElapsedTime(&b, base, r.e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int32_t sid = 0;
        while (sid < (int32_t)c->trace_streams.size() && c->trace_streams[sid] != r.st) sid++;
        if (sid == (int32_t)c->trace_streams.size()) c->trace_streams.push_back(r.st);
        c->trace.push_back({r.cls, sid, (double)a, (double)b});
    }
    c->prof_pending.clear();
    c->ev_used = 0;
}


template <typename T>
int dalloc(ipm_ctx *c, T **p, size_t count) {
    void *q = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return to_err(e);
    }
    c->allocs.push_back(q);
    c->device_bytes += (int64_t)bytes;
    *p = (T *)q;
    return IPM_OK;
}

template <typename T>
int dupload(ipm_ctx *c, T **p, const std::vector<T> &h) {
    int rc = dalloc(c, p, h.size());
    if (rc) return rc;
    if (!h.empty()) {
        cudaError_t e = cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return to_err(e);
    }
    return IPM_OK;
}

// Items of the persistent level kernel for the large fronts of level l, in
// ticket order: all assembly items, then per pivot block t the diagonal
// blocks, the triangular solves, the remaining trailing tiles of block t-1
// and the lookahead strips of block t (after the last block, the remaining
// tiles of the last block).  Counters per front (base b): b+0 assembly
// items done, b+1 diagonal blocks done, b+2 triangular-solve chunks done,
// then one counter per 32 x 32 tile (ib >= jb) of the front that grows by 8
// per pivot block applied to the tile (a whole tile adds 8, the strips of a
// tile add 8 between them).  Every wait refers to items placed earlier:
//   diagonal block t:     tile (t, t) >= 8 t (assembly done for t = 0),
//   solve chunk (t, r):   diagonal block t done, tile (r / 32, t) >= 8 t,
//   update (t, ib, jb):   all solve chunks of blocks <= t, tile >= 8 t.
// Tiles lie on the front's 32-grid; updates skip the columns < p1 (the
// panel's own columns) of a grid tile that a partial last panel cuts.
void build_level_items(const Plan &P, int32_t l, LevelWork &W, const std::vector<int32_t> &slot_of,
                       std::vector<FactorItem> &items, std::vector<int32_t> &cbase) {
    constexpr int32_t B = kUpdTile;  // == nb == 32
    W.lvl_off = (int64_t)items.size();
    const int32_t t0 = P.lvl_large_ptr[l], t1 = P.lvl_large_ptr[l + 1];
    int32_t ncnt = 0, maxsteps = 0;
    for (int32_t q = t0; q < t1; q++) {
        const int32_t s = P.lvl_large[q], nblk = (P.sn_f[s] + B - 1) / B;
        cbase[s] = ncnt;
        ncnt += 3 + nblk * (nblk + 1) / 2;
        maxsteps = std::max(maxsteps, (P.sn_k[s] + B - 1) / B);
    }
    auto tidx = [&](int32_t s, int32_t ib, int32_t jb) { return cbase[s] + 3 + ib * (ib + 1) / 2 + jb; };
    auto item = [](int32_t kind, int32_t s, int32_t t, int32_t a, int32_t b, int32_t aux) {
        FactorItem it;
        it.kind = kind;
        it.s = s;
        it.t = t;
        it.a = a;
        it.b = b;
        it.aux = aux;
        it.wait0 = it.wait1 = -1;
        it.need0 = it.need1 = 0;
        it.sig = -1;
        it.add = 0;
        return it;
    };
    // assembly, in the order of the level's AsmItems
    int64_t ai = W.asm_off;
    for (int32_t q = t0; q < t1; q++) {
        const int32_t s = P.lvl_large[q];
        for (int32_t cl = 0; cl < P.sn_f[s]; cl += B) {
            FactorItem it = item(kItemAssemble, s, 0, cl, std::min(cl + B, P.sn_f[s]), (int32_t)ai++);
            it.sig = cbase[s];
            it.add = 1;
            items.push_back(it);
        }
    }
    // triangular-solve chunks of rows [p1, f): the first ends at the next
    // multiple of kTrsmRowsHost, so that no chunk crosses a 32-row tile
    // (each chunk waits on the one tile it lies in)
    auto chunk_end = [](int32_t r, int32_t f) { return std::min(f, (r / kTrsmRowsHost + 1) * kTrsmRowsHost); };
    auto nchunks = [&](int32_t p1, int32_t f) {
        int32_t n = 0;
        for (int32_t r = p1; r < f; r = chunk_end(r, f)) n++;
        return n;
    };
    // solve chunks of blocks <= t of front s
    auto cum_chunks = [&](int32_t s, int32_t t) {
        const int32_t k = P.sn_k[s], f = P.sn_f[s];
        int32_t n = 0;
        for (int32_t u = 0; u <= t && u * B < k; u++) n += nchunks(std::min((u + 1) * B, k), f);
        return n;
    };
    // updates of block t of front s: tiles (ib, jb >= first) with the
    // lookahead column block as strips when la
    auto updates = [&](int32_t q, int32_t t, bool lookahead) {
        const int32_t s = P.lvl_large[q], k = P.sn_k[s], f = P.sn_f[s];
        if (t * B >= k) return;
        const int32_t p1 = std::min((t + 1) * B, k);
        if (p1 >= f) return;
        const bool next_panel = p1 < k;
        const int32_t jb0 = p1 / B, nblk = (f + B - 1) / B, nchunk = cum_chunks(s, t);
        for (int32_t jb = jb0; jb < nblk; jb++) {
            const bool la = next_panel && jb == t + 1;
            if (la != lookahead) continue;
            for (int32_t ib = jb; ib < nblk; ib++) {
                const int32_t need = 8 * t;
                if (la) {
                    const int32_t c1 = std::min((jb + 1) * B, f), nstrip = (c1 - jb * B + kStripCols - 1) / kStripCols;
                    for (int32_t u = 0; u < nstrip; u++) {
                        FactorItem it = item(kItemStrip, s, t, ib * B, jb * B + u * kStripCols, 0);
                        it.wait0 = cbase[s] + 2;
                        it.need0 = nchunk;
                        if (t > 0) {
                            it.wait1 = tidx(s, ib, jb);
                            it.need1 = need;
                        }
                        it.sig = tidx(s, ib, jb);
                        it.add = u + 1 < nstrip ? 1 : 8 - (nstrip - 1);
                        items.push_back(it);
                    }
                } else {
                    FactorItem it = item(kItemTile, s, t, ib * B, jb * B, 0);
                    it.wait0 = cbase[s] + 2;
                    it.need0 = nchunk;
                    if (t > 0) {
                        it.wait1 = tidx(s, ib, jb);
                        it.need1 = need;
                    }
                    it.sig = tidx(s, ib, jb);
                    it.add = 8;
                    items.push_back(it);
                }
            }
        }
    };
    for (int32_t t = 0; t <= maxsteps; t++) {
        if (t < maxsteps) {
            for (int32_t q = t0; q < t1; q++) {
                const int32_t s = P.lvl_large[q];
                if (t * B >= P.sn_k[s]) continue;
                FactorItem it = item(kItemDiag, s, t, 0, 0, slot_of[s]);
                if (t == 0) {
                    it.wait0 = cbase[s];
                    it.need0 = (P.sn_f[s] + B - 1) / B;
                } else {
                    it.wait0 = tidx(s, t, t);
                    it.need0 = 8 * t;
                }
                it.sig = cbase[s] + 1;
                it.add = 1;
                items.push_back(it);
            }
            for (int32_t q = t0; q < t1; q++) {
                const int32_t s = P.lvl_large[q], k = P.sn_k[s], f = P.sn_f[s];
                if (t * B >= k) continue;
                const int32_t p1 = std::min((t + 1) * B, k);
                for (int32_t r = p1; r < f; r = chunk_end(r, f)) {
                    FactorItem it = item(kItemTrsm, s, t, r, chunk_end(r, f), slot_of[s]);
                    it.wait0 = cbase[s] + 1;
                    it.need0 = t + 1;
                    if (t > 0) {
                        it.wait1 = tidx(s, r / B, t);
                        it.need1 = 8 * t;
                    }
                    it.sig = cbase[s] + 2;
                    it.add = 1;
                    items.push_back(it);
                }
            }
        }
        if (t > 0)
            for (int32_t q = t0; q < t1; q++) updates(q, t - 1, false);
        if (t < maxsteps)
            for (int32_t q = t0; q < t1; q++) updates(q, t, true);
    }
    W.lvl_cnt = (int32_t)(items.size() - W.lvl_off);
    W.lvl_ncnt = ncnt;
    // Deadlock freedom, checked: running the items one at a time in ticket
    // order must meet every wait (then every wait of the parallel run is met
    // by items with smaller tickets, all of which complete by induction).
    // A level that fails the check keeps the one-launch-per-step path.
    std::vector<int32_t> sim(ncnt, 0);
    bool ok = true;
    for (int64_t i = W.lvl_off; i < (int64_t)items.size() && ok; i++) {
        const FactorItem &it = items[i];
        for (int u = 0; u < 2; u++) {
            const int32_t wi = u ? it.wait1 : it.wait0, need = u ? it.need1 : it.need0;
            if (wi >= ncnt || (wi >= 0 && sim[wi] < need)) ok = false;
        }
        if (it.sig >= ncnt) ok = false;
        if (it.kind == kItemTrsm && (it.a / B != (it.b - 1) / B || it.b - it.a > kTrsmRowsHost)) ok = false;
        if (ok && it.sig >= 0) sim[it.sig] += it.add;
    }
    if (!ok) {
        items.resize(W.lvl_off);
        W.lvl_cnt = 0;
        W.lvl_ncnt = 0;
    }
}

void free_device(ipm_ctx *c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->cap_stream = nullptr;
    if (c->side) cudaStreamDestroy(c->side);
    c->side = nullptr;
    if (c->side2) cudaStreamDestroy(c->side2);
    c->side2 = nullptr;
    for (cudaStream_t &q : c->cls) {
        if (q) cudaStreamDestroy(q);
        q = nullptr;
    }
    for (cudaEvent_t e : c->dep_ev) cudaEventDestroy(e);
    c->dep_ev.clear();
    for (cudaEvent_t e : c->step_ev) cudaEventDestroy(e);
    c->step_ev.clear();
    if (c->gm_stream) cudaStreamDestroy(c->gm_stream);
    c->gm_stream = nullptr;
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
    // buffers allocated on first use live in allocs too
    c->gm_V = c->gm_Z = c->gm_zero = c->gm_w = c->gm_part = c->gm_h = nullptr;
    c->gm_dev = nullptr;
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    c->ev_used = 0;
    c->prof_pending.clear();
    if (c->h_r7) cudaFreeHost(c->h_r7);
    c->h_r7 = nullptr;
    c->device_bytes = 0;
    c->dev_ready = false;
    c->values_set = false;
    c->factorised = false;
}

// Build the device plan and the large-front work lists, then upload.
// Solve schedule: per-supernode descriptors, per-row gather lists of the
// children's contributions (children ascending, so every row sums in the
// same order as a child-by-child scatter), and the forward / backward item
// lists in topological order.
int build_solve_schedule(ipm_ctx *c, const std::vector<int32_t> &fwd_order, const std::vector<int32_t> &bwd_order,
                         const int32_t *d_rows) {
    const Plan &P = c->plan;
    const int32_t ns = P.nsuper;
    std::vector<SolveNode> nodes(ns);
    for (int32_t s = 0; s < ns; s++) {
        SolveNode &nd = nodes[s];
        nd.off = P.sn_off[s];
        nd.upd = P.upd_off[s];
        nd.rptr = P.sn_rptr[s];
        nd.f = P.sn_f[s];
        nd.k = P.sn_k[s];
        nd.ld = P.sn_ld[s];
        nd.c0 = P.sn_start[s];
        nd.parent = P.sn_parent[s];
        nd.nchild = P.child_ptr[s + 1] - P.child_ptr[s];
        const int64_t rect = (int64_t)nd.k * (nd.f - nd.k);
        nd.nblk = (nd.k + 31) / 32;
        nd.nrect = (nd.f > nd.k && (rect >= kRectSplit || nd.nblk > 1)) ? (nd.f - nd.k + kRectRows - 1) / kRectRows : 0;
        nd.inv = -1;
    }
    // Supernodes whose diagonal blocks the sweeps apply through explicit
    // inverses (computed once per factorisation): every block of a supernode
    // with several blocks, and the block of a supernode with children and
    // k >= 16.  Their substitutions lie on the sweeps' dependency chains;
    // the leaves, off them, keep the substitution.
    // A supernode with several blocks also keeps, per block, the products of
    // X_b with its neighbouring blocks of L11 (3 x 1024 doubles per block).
    std::vector<InvItem> inv_items, pair_items;
    int64_t ninv = 0;  // doubles
    for (int32_t s = 0; s < ns; s++) {
        SolveNode &nd = nodes[s];
        if (!(nd.nblk > 1 || (nd.nchild > 0 && nd.k >= 16))) continue;
        const int64_t stride = nd.nblk > 1 ? 3072 : 1024;
        nd.inv = ninv;
        for (int32_t b = 0; b < nd.nblk; b++) {
            inv_items.push_back({s, b, ninv + b * stride});
            if (nd.nblk > 1) pair_items.push_back({s, b, ninv + b * stride});
        }
        ninv += nd.nblk * stride;
    }
    const int64_t nrows = P.sn_rptr[ns];
    std::vector<int64_t> grp(nrows + 1, 0);
    for (int32_t s = 0; s < ns; s++)
        for (int32_t q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
            const int32_t ch = P.child_list[q];
            const int32_t cc = P.sn_f[ch] - P.sn_k[ch];
            for (int32_t r = 0; r < cc; r++) grp[P.sn_rptr[s] + P.relmap[P.map_off[ch] + r] + 1]++;
        }
    for (int64_t i = 0; i < nrows; i++) grp[i + 1] += grp[i];
    std::vector<int64_t> gsrc(std::max<int64_t>(grp[nrows], 1));
    {
        std::vector<int64_t> fill(grp.begin(), grp.end() - 1);
        for (int32_t s = 0; s < ns; s++)
            for (int32_t q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
                const int32_t ch = P.child_list[q];
                const int32_t cc = P.sn_f[ch] - P.sn_k[ch];
                for (int32_t r = 0; r < cc; r++)
                    gsrc[fill[P.sn_rptr[s] + P.relmap[P.map_off[ch] + r]]++] = P.upd_off[ch] + r;
            }
    }
    // Ticket order: critical path first.  With a latency model of one item,
    // the forward priority of s is the longest path from s to the root and the
    // backward priority the longest path from s down to a leaf; both orders
    // sorted by decreasing priority are topological (a child's forward
    // priority exceeds its parent's, a parent's backward priority exceeds its
    // children's), and they start the long chains first.
    std::vector<double> wcost(ns), up(ns, 0.0), down(ns, 0.0);
    for (int32_t s = 0; s < ns; s++) {
        const double k = nodes[s].k, f = nodes[s].f;
        const double rect = nodes[s].nrect > 0 ? 32.0 * k : (f - k) * k;
        wcost[s] = 4.0 + 3.0 * nodes[s].nblk + rect / 1500.0;  // microseconds, roughly
    }
    for (int32_t s = ns - 1; s >= 0; s--) up[s] = wcost[s] + (nodes[s].parent >= 0 ? up[nodes[s].parent] : 0.0);
    for (int32_t s = 0; s < ns; s++) {
        down[s] += wcost[s];
        if (nodes[s].parent >= 0) down[nodes[s].parent] = std::max(down[nodes[s].parent], down[s]);
    }
    std::vector<int32_t> of(fwd_order), ob(bwd_order);
    std::stable_sort(of.begin(), of.end(), [&](int32_t a, int32_t b) { return up[a] > up[b]; });
    std::stable_sort(ob.begin(), ob.end(), [&](int32_t a, int32_t b) { return down[a] > down[b]; });
    // Childless single-item supernodes with f <= 32 run one per warp, eight
    // to a ticket.  A forward group takes the place of its first member (a
    // leaf waits on nothing); a backward group the place of its last member
    // (so every member's parent has an earlier ticket).
    std::vector<char> is_leaf(ns, 0);
    for (int32_t s = 0; s < ns; s++)
        is_leaf[s] = nodes[s].nchild == 0 && nodes[s].nblk == 1 && nodes[s].nrect == 0 && nodes[s].f <= 32;
    std::vector<SolveItem> fwd, bwd;
    std::vector<int32_t> fleaf, bleaf;
    for (int32_t s : of) {
        if (is_leaf[s]) {
            if (fleaf.size() % 8 == 0) fwd.push_back({(int32_t)(fleaf.size() / 8), kLeafGroup});
            fleaf.push_back(s);
            continue;
        }
        for (int32_t b = 0; b < nodes[s].nblk; b++) fwd.push_back({s, -1 - b});
        for (int32_t r = 0; r < nodes[s].nrect; r++) fwd.push_back({s, r});
    }
    while (fleaf.size() % 8) fleaf.push_back(-1);
    for (int32_t s : ob) {
        if (is_leaf[s]) {
            bleaf.push_back(s);
            if (bleaf.size() % 8 == 0) bwd.push_back({(int32_t)(bleaf.size() / 8 - 1), kLeafGroup});
            continue;
        }
        for (int32_t b = nodes[s].nblk - 1; b >= 0; b--) bwd.push_back({s, -1 - b});
    }
    if (bleaf.size() % 8) {
        bwd.push_back({(int32_t)(bleaf.size() / 8), kLeafGroup});
        while (bleaf.size() % 8) bleaf.push_back(-1);
    }
    SolveNode *d_nodes;
    int64_t *d_grp, *d_gsrc;
    SolveItem *d_fwd, *d_bwd;
    double *d_yv;
    int32_t *d_fleaf, *d_bleaf;
    int rc;
    if ((rc = dupload(c, &d_nodes, nodes)) || (rc = dupload(c, &d_grp, grp)) || (rc = dupload(c, &d_gsrc, gsrc)) ||
        (rc = dupload(c, &d_fwd, fwd)) || (rc = dupload(c, &d_bwd, bwd)) || (rc = dalloc(c, &d_yv, (size_t)P.N)) ||
        (rc = dupload(c, &d_fleaf, fleaf)) || (rc = dupload(c, &d_bleaf, bleaf)) ||
        (rc = dupload(c, &c->inv_items, inv_items)) || (rc = dupload(c, &c->pair_items, pair_items)) ||
        (rc = dalloc(c, &c->linv, (size_t)ninv)))
        return rc;
    c->ninv = (int32_t)inv_items.size();
    c->npairs = (int32_t)pair_items.size();
    SolveSched &S = c->sched;
    S.node = d_nodes;
    S.sn_rows = d_rows;
    S.gat_rp = d_grp;
    S.gat_src = d_gsrc;
    S.fwd = d_fwd;
    S.bwd = d_bwd;
    S.spin_limit = c->opt.spin_limit_log2 < 0 ? 0 : (1ll << c->opt.spin_limit_log2);
    S.nfwd = (int32_t)fwd.size();
    S.nbwd = (int32_t)bwd.size();
    S.nsuper = ns;
    S.sync = c->solve_sync;
    S.yv = d_yv;
    S.nyv = P.N;
    S.fwd_leaf = d_fleaf;
    S.bwd_leaf = d_bleaf;
    S.Linv = c->linv;
    return IPM_OK;
}

int setup_device(ipm_ctx *c) {
    const Plan &P = c->plan;
    cudaError_t e = cudaSetDevice(c->opt.device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return IPM_ERR_NO_DEVICE;
    }
    const int32_t ns = P.nsuper, N = P.N;
    std::vector<int32_t> c0(ns);
    for (int32_t s = 0; s < ns; s++) c0[s] = P.sn_start[s];
    std::vector<int8_t> sign(P.sign.begin(), P.sign.end());
    // regularised matrix, full symmetric CSR in factorisation order
    std::vector<int64_t> kp(N + 1, 0);
    std::vector<int32_t> kj;
    std::vector<int64_t> ksrc;
    if (P.form == 1) {
        const int32_t n = P.n;
        // count
        for (int32_t j = 0; j < n; j++) {
            kp[P.iperm[j] + 1]++;  // diagonal
            for (int64_t p = P.Acp[j]; p < P.Acp[j + 1]; p++) {
                kp[P.iperm[j] + 1]++;
                kp[P.iperm[n + P.Ari[p]] + 1]++;
            }
        }
        for (int32_t i = 0; i < P.m; i++) kp[P.iperm[n + i] + 1]++;
        for (int32_t i = 0; i < N; i++) kp[i + 1] += kp[i];
        kj.resize(kp[N]);
        ksrc.resize(kp[N]);
        std::vector<int64_t> fill(kp.begin(), kp.end() - 1);
        for (int32_t j = 0; j < n; j++) {
            int32_t a = P.iperm[j];
            kj[fill[a]] = a;
            ksrc[fill[a]++] = -1 - (int64_t)j;
            for (int64_t p = P.Acp[j]; p < P.Acp[j + 1]; p++) {
                int32_t b = P.iperm[n + P.Ari[p]];
                kj[fill[a]] = b;
                ksrc[fill[a]++] = p;
                kj[fill[b]] = a;
                ksrc[fill[b]++] = p;
            }
        }
        for (int32_t i = 0; i < P.m; i++) {
            int32_t b = P.iperm[n + i];
            kj[fill[b]] = b;
            ksrc[fill[b]++] = kDualDiag;
        }
    }
    if (P.form == 2) {
        // M = A Theta~ A^T + delta I, full symmetric CSR in factorisation order; value
        // source = index of the lower entry (the diagonal adds delta)
        const std::vector<int64_t> &cp = P.ne_cp;
        const std::vector<int32_t> &ri = P.ne_ri;
        for (int32_t jo = 0; jo < N; jo++)
            for (int64_t p = cp[jo]; p < cp[jo + 1]; p++) {
                const int32_t a = P.iperm[ri[p]], b = P.iperm[jo];
                kp[a + 1]++;
                if (a != b) kp[b + 1]++;
            }
        for (int32_t i = 0; i < N; i++) kp[i + 1] += kp[i];
        kj.resize(kp[N]);
        ksrc.resize(kp[N]);
        std::vector<int64_t> fill(kp.begin(), kp.end() - 1);
        for (int32_t jo = 0; jo < N; jo++)
            for (int64_t p = cp[jo]; p < cp[jo + 1]; p++) {
                const int32_t a = P.iperm[ri[p]], b = P.iperm[jo];
                kj[fill[a]] = b;
                ksrc[fill[a]++] = p;
                if (a != b) {
                    kj[fill[b]] = a;
                    ksrc[fill[b]++] = p;
                }
            }
    }
    // per-level lists
    std::vector<int32_t> lvl_all, small_lists;
    std::vector<PanelItem> asm_items, panel_items, trsm_items;
    std::vector<AsmItem> asm_info;
    std::vector<int32_t> asm_cr;
    std::vector<int32_t> trsm_slots, trsm_sbase, slot_of(P.nsuper, -1);
    std::vector<int32_t> thin_list, thin_asm, thin_slot;
    int32_t nslots = 0;
    for (int32_t s = 0; s < P.nsuper; s++)
        if (P.sn_large[s]) slot_of[s] = nslots++;
    std::vector<TileItem> tile_items, tc_items, alt_items;
    std::vector<SlicedTile> sliced_tiles;
    int64_t max_slice_blocks = 0;
    const bool sliced = c->opt.precision == IPM_PREC_SLICED;
    std::vector<FactorItem> lvl_items;
    std::vector<int32_t> cbase(P.nsuper, -1);
    int32_t max_ncnt = 0;
    c->levels.assign(P.nlevels, LevelWork());
    c->flops_tensor = 0.0;
    // algorithmic work of assembling and factorising one front
    auto front_work = [&](int32_t s) {
        const double f = P.sn_f[s];
        Work fr;
        for (int32_t i = 1; i <= P.sn_k[s]; i++) fr.flops += (f - i) * (f - i + 3);
        fr.bytes = 8.0 * f * (f + 1) / 2 + 12.0 * (double)(P.orig_ptr[s + 1] - P.orig_ptr[s]);
        for (int32_t q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
            const double cc = P.sn_f[P.child_list[q]] - P.sn_k[P.child_list[q]];
            fr.bytes += 8.0 * cc * (cc + 1) / 2 + 4.0 * cc;
            fr.flops += cc * (cc + 1) / 2;
        }
        return fr;
    };
    // One assembly item: columns [cl, ce), rows [rlo, rhi) of large front s;
    // its original entries (those of the columns) and, per child, the
    // contribution-block columns and rows that land in it.
    auto add_asm = [&](int32_t s, int32_t cl, int32_t ce, int32_t rlo, int32_t rhi) {
        const int32_t ld = P.sn_ld[s];
        asm_items.push_back({s, cl, ce, 0});
        const int32_t *d0 = P.orig_dst.data() + P.orig_ptr[s], *d1 = P.orig_dst.data() + P.orig_ptr[s + 1];
        AsmItem ai;
        ai.o0 = std::lower_bound(d0, d1, (int64_t)cl * ld) - P.orig_dst.data();
        ai.o1 = std::lower_bound(d0, d1, (int64_t)ce * ld) - P.orig_dst.data();
        ai.cr = (int64_t)(asm_cr.size() / 4);
        ai.r_lo = rlo;
        ai.r_hi = rhi;
        for (int32_t q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
            const int32_t ch = P.child_list[q];
            const int32_t *m0 = P.relmap.data() + P.map_off[ch], *m1 = m0 + (P.sn_f[ch] - P.sn_k[ch]);
            asm_cr.push_back((int32_t)(std::lower_bound(m0, m1, cl) - m0));
            asm_cr.push_back((int32_t)(std::lower_bound(m0, m1, ce) - m0));
            asm_cr.push_back((int32_t)(std::lower_bound(m0, m1, rlo) - m0));
            asm_cr.push_back((int32_t)(std::lower_bound(m0, m1, rhi) - m0));
        }
        asm_info.push_back(ai);
    };
    // One step of the large-front path: for each (front s, panel start p0)
    // of fp, the diagonal block of the panel, the triangular solve of the rows
    // below it and the update tiles of the front's trailing part.
    auto add_step = [&](const std::vector<std::pair<int32_t, int32_t>> &fp) {
        StepWork S{};
        S.small_wait = -1;
        S.panel_off = (int64_t)panel_items.size();
        S.trsm_off = (int64_t)trsm_items.size();
        S.tile_off = (int64_t)tile_items.size();
        S.tc_off = (int64_t)tc_items.size();
        S.alt_off = (int64_t)alt_items.size();
        S.st_off = (int64_t)sliced_tiles.size();
        int32_t nblk = 0;  // slice blocks of this step
        std::vector<SlicedTile> t1, t2;  // sliced tiles: next panel's columns / the rest
        std::vector<TileItem> u1, u2, a1, a2;  // lookahead / remaining tiles of this step
        Work w1, w2, wa1, wa2;
        // lower entries of a kUpdTile tile times 2 w flops (and its bytes)
        auto tile_work = [](Work &acc, int32_t f, int32_t i0, int32_t j0, double w) {
            double e = 0.0;
            for (int32_t j = j0; j < std::min(j0 + kUpdTile, f); j++)
                e += std::max(0, std::min(i0 + kUpdTile, f) - std::max(i0, j));
            acc.flops += 2.0 * w * e;
            acc.bytes += 16.0 * e + 8.0 * w * (2.0 * kUpdTile);
        };
        for (const auto &e : fp) {
            const int32_t s = e.first, p0 = e.second;
            const int32_t k = P.sn_k[s], f = P.sn_f[s];
            const int32_t p1 = std::min(p0 + c->opt.nb, k);
            panel_items.push_back({s, 0, slot_of[s], p0});
            const bool tc = c->opt.precision != IPM_PREC_FP64 && f >= c->opt.mixed_min_front;
            // Sliced fronts take their full panels in pairs: the first panel of a
            // pair updates only the second's columns, the second updates the
            // whole trailing part with both (two chunks, K = 64).  A ragged last
            // panel, and a full panel left over before it, stand alone.
            const int32_t tpan = p0 / c->opt.nb, npair = 2 * ((k / c->opt.nb) / 2);
            const bool pair_first = tpan < npair && tpan % 2 == 0;
            const bool pair_second = tpan < npair && tpan % 2 == 1;
            // sliced fronts: the triangular solve writes the digit slices of the rows it finishes
            const int32_t sbase = (tc && sliced && p1 < f) ? (nblk << 1) | (pair_second ? 1 : 0) : -1;
            for (int32_t r = p1; r < f; r += kTrsmItemRowsHost) {
                trsm_items.push_back({s, r, std::min(r + kTrsmItemRowsHost, f), p0});
                trsm_slots.push_back(slot_of[s]);
                trsm_sbase.push_back(sbase);
            }
            const double w = p1 - p0, rest = f - p1;
            // tiles of the next panel's columns (when the front has one) go first
            const bool next_panel = p1 < k;
            if (tc && sliced && p1 < f) {
                // slice blocks of rows p1.. (written by the triangular solve),
                // then the 128 x 32 tiles of the lower trailing part (only the
                // next panel's columns after the first panel of a pair), row
                // blocks aligned with the slice blocks
                const int32_t base = nblk;
                const int32_t kc = pair_second ? 2 : 1;
                const double wk = pair_second ? w + c->opt.nb : w;  // columns of the product
                const int32_t jend = pair_first ? p1 + kSliceCols : f;
                nblk += (f - p1 + kSliceRows - 1) / kSliceRows;
                for (int32_t j0 = p1; j0 < jend; j0 += kSliceCols)
                    for (int32_t b = (j0 - p1) / kSliceRows; p1 + b * kSliceRows < f; b++) {
                        const int32_t i0 = p1 + b * kSliceRows;
                        const bool la = next_panel && j0 == p1;
                        (la ? t1 : t2).push_back({s, i0, j0, base + b, base + (j0 - p1) / kSliceRows,
                                                  (j0 - p1) % kSliceRows, kc});
                        // lower entries of the tile times 2 wk flops; its C read and write
                        double e = 0.0;
                        for (int32_t j = j0; j < std::min(j0 + kSliceCols, f); j++)
                            e += std::max(0, std::min(i0 + kSliceRows, f) - std::max(i0, j));
                        Work &tw = la ? S.st_w1 : S.st_w2;
                        tw.flops += 2.0 * wk * e;
                        // C read and written; the digit images of its 128 A rows and 32 B rows (bf16)
                        tw.bytes += 16.0 * e + 2.0 * kSlices * wk * (kSliceRows + kSliceCols);
                    }
                S.trsm_w.bytes += 2.0 * kSlices * 2.0 * rest * wk;  // the slices the solve writes
                if (pair_second) S.trsm_w.bytes += 8.0 * rest * c->opt.nb;  // the first panel's rows it re-reads
            } else if (tc) {
                for (int32_t j0 = p1; j0 < f; j0 += kTcTile)
                    for (int32_t i0 = j0; i0 < f; i0 += kTcTile) tc_items.push_back({s, i0, j0, p0});
            }
            for (int32_t j0 = p1; j0 < f; j0 += kUpdTile)
                for (int32_t i0 = j0; i0 < f; i0 += kUpdTile) {
                    // lookahead tiles become strips of kStripCols columns
                    const bool la = next_panel && j0 == p1;
                    std::vector<TileItem> &dst = tc ? (la ? a1 : a2) : (la ? u1 : u2);
                    if (la) {
                        for (int32_t jj = j0; jj < std::min(j0 + kUpdTile, f); jj += kStripCols)
                            dst.push_back({s, i0, jj, p0});
                    } else {
                        dst.push_back({s, i0, j0, p0});
                    }
                    tile_work(tc ? (la ? wa1 : wa2) : (la ? w1 : w2), f, i0, j0, w);
                }
            // pivot block (w^3/3) + triangular solve of the rows below; update of the lower trailing part
            S.panel_w.flops += w * w * w / 3.0;
            S.panel_w.bytes += 16.0 * w * w;
            S.trsm_w.flops += rest * w * w;
            S.trsm_w.bytes += 16.0 * rest * w;
            if (tc) {
                S.tc_w.flops += 2.0 * w * rest * (rest + 1) / 2;
                S.tc_w.bytes += 16.0 * rest * (rest + 1) / 2 + 8.0 * rest * w;
                c->flops_tensor += 2.0 * w * rest * (rest + 1) / 2;
            }
        }
        tile_items.insert(tile_items.end(), u1.begin(), u1.end());
        tile_items.insert(tile_items.end(), u2.begin(), u2.end());
        alt_items.insert(alt_items.end(), a1.begin(), a1.end());
        alt_items.insert(alt_items.end(), a2.begin(), a2.end());
        S.tile_cnt1 = (int32_t)u1.size();
        S.alt_cnt1 = (int32_t)a1.size();
        S.tile_w1 = w1;
        S.tile_w = w2;
        S.alt_w1 = wa1;
        S.alt_w = wa2;
        S.panel_cnt = (int32_t)(panel_items.size() - S.panel_off);
        S.trsm_cnt = (int32_t)(trsm_items.size() - S.trsm_off);
        S.tile_cnt = (int32_t)(tile_items.size() - S.tile_off);
        S.tc_cnt = (int32_t)(tc_items.size() - S.tc_off);
        S.alt_cnt = (int32_t)(alt_items.size() - S.alt_off);
        sliced_tiles.insert(sliced_tiles.end(), t1.begin(), t1.end());
        sliced_tiles.insert(sliced_tiles.end(), t2.begin(), t2.end());
        S.st_cnt = (int32_t)(sliced_tiles.size() - S.st_off);
        S.st_cnt1 = (int32_t)t1.size();
        max_slice_blocks = std::max<int64_t>(max_slice_blocks, nblk);
        return S;
    };
    for (int32_t l = 0; l < P.nlevels; l++) {
        LevelWork &W = c->levels[l];
        // small fronts of the level, by size class (shared memory per launch
        // is sized by the class maximum)
        const int32_t bounds[3] = {32, 64, kSmallFrontMax};
        int32_t lo = 0, maxsmall = 0;
        for (int32_t b = 0; b < 3; b++) {
            SmallClass C;
            C.off = (int64_t)small_lists.size();
            C.maxf = 0;
            for (int32_t t = P.lvl_small_ptr[l]; t < P.lvl_small_ptr[l + 1]; t++) {
                const int32_t s = P.lvl_small[t], f = P.sn_f[s];
                if (f > lo && f <= bounds[b]) {
                    small_lists.push_back(s);
                    C.maxf = std::max(C.maxf, f);
                    const Work fr = front_work(s);
                    C.w.flops += fr.flops;
                    C.w.bytes += fr.bytes;
                }
            }
            C.cnt = (int32_t)(small_lists.size() - C.off);
            C.cls = b;
            lo = bounds[b];
            maxsmall = std::max(maxsmall, C.maxf);
            if (C.cnt > 0) W.small.push_back(C);
        }
        W.all_off = (int64_t)lvl_all.size();
        W.all_maxf = maxsmall;
        for (int32_t t = P.lvl_small_ptr[l]; t < P.lvl_small_ptr[l + 1]; t++) lvl_all.push_back(P.lvl_small[t]);
        for (int32_t t = P.lvl_large_ptr[l]; t < P.lvl_large_ptr[l + 1]; t++) {
            lvl_all.push_back(P.lvl_large[t]);
            W.all_maxf = std::max(W.all_maxf, P.sn_f[P.lvl_large[t]]);
        }
        W.all_cnt = (int32_t)(lvl_all.size() - W.all_off);
        // algorithmic work of the level's assembly and solve launches
        for (int64_t t = W.all_off; t < (int64_t)lvl_all.size(); t++) {
            const int32_t s = lvl_all[t];
            const double f = P.sn_f[s], k = P.sn_k[s];
            const double lnz = f * k - k * (k - 1) / 2;  // stored entries of L
            if (P.sn_large[s]) W.asm_w.bytes += front_work(s).bytes;
            W.fwd_w.flops += 2.0 * (lnz - f);
            W.fwd_w.bytes += 8.0 * lnz + 8.0 * (f + 2 * k);
            W.bwd_w.flops += 2.0 * (lnz - f);
            W.bwd_w.bytes += 8.0 * lnz + 8.0 * (f + k);
        }
        // large fronts; the thin ones (one pivot block, f <= kThinMaxF, FP64
        // updates) of a level that does not take the level kernel run whole,
        // one CTA each, instead of through the steps
        W.asm_off = (int64_t)asm_items.size();
        int32_t maxsteps = 0;
        std::vector<int32_t> main_fronts;
        std::vector<int64_t> main_first;
        W.thin_off = (int64_t)thin_list.size();
        for (int32_t t = P.lvl_large_ptr[l]; t < P.lvl_large_ptr[l + 1]; t++) {
            const int32_t s = P.lvl_large[t];
            const int64_t first = (int64_t)asm_items.size();
            for (int32_t cl = 0; cl < P.sn_f[s]; cl += 32) add_asm(s, cl, std::min(cl + 32, P.sn_f[s]), cl, P.sn_f[s]);
            const bool thin = P.sn_k[s] <= c->opt.nb && P.sn_f[s] <= kThinMaxF &&
                              !(c->opt.precision != IPM_PREC_FP64 && P.sn_f[s] >= c->opt.mixed_min_front);
            if (thin) {
                thin_list.push_back(s);
                thin_asm.push_back((int32_t)first);
                thin_slot.push_back(slot_of[s]);
                const Work fr = front_work(s);
                W.thin_w.flops += fr.flops;
                W.thin_w.bytes += fr.bytes;
            } else {
                main_fronts.push_back(s);
                main_first.push_back(first);
                maxsteps = std::max(maxsteps, (P.sn_k[s] + c->opt.nb - 1) / c->opt.nb);
            }
        }
        W.asm_cnt = (int32_t)(asm_items.size() - W.asm_off);
        W.thin_cnt = (int32_t)((int64_t)thin_list.size() - W.thin_off);
        if (W.thin_cnt > 0) {
            // the per-step assembly launch takes the other fronts' items (copies)
            W.asm_off2 = (int64_t)asm_items.size();
            for (size_t q = 0; q < main_fronts.size(); q++)
                for (int64_t a = main_first[q]; a < main_first[q] + (P.sn_f[main_fronts[q]] + 31) / 32; a++) {
                    const PanelItem pi = asm_items[a];
                    const AsmItem ai = asm_info[a];
                    asm_items.push_back(pi);
                    asm_info.push_back(ai);
                }
            W.asm_cnt2 = (int32_t)((int64_t)asm_items.size() - W.asm_off2);
        } else {
            W.asm_off2 = W.asm_off;
            W.asm_cnt2 = W.asm_cnt;
        }
        std::vector<std::pair<int32_t, int32_t>> fp;
        for (int32_t st = 0; st < maxsteps; st++) {
            fp.clear();
            for (int32_t s : main_fronts)
                if (st * c->opt.nb < P.sn_k[s]) fp.push_back({s, st * c->opt.nb});
            const StepWork S = add_step(fp);
            W.steps.push_back(S);
            if (S.tc_cnt > 0 || S.st_cnt > 0) W.has_tc = true;
        }
        build_level_items(P, l, W, slot_of, lvl_items, cbase);
        {
            int32_t chain = 0;
            for (int32_t t = P.lvl_large_ptr[l]; t < P.lvl_large_ptr[l + 1]; t++) {
                const int32_t s = P.lvl_large[t];
                const Work fr = front_work(s);
                W.lvl_w.flops += fr.flops;
                W.lvl_w.bytes += fr.bytes;
                chain = std::max(chain, (P.sn_k[s] + 31) / 32);
            }
            W.lvl_chain = chain;
        }
        max_ncnt = std::max(max_ncnt, W.lvl_ncnt);
    }
    // Dependency order of the large fronts' steps.  Front s starts at step
    // g0[s], two steps after the last panel of its last large child (the
    // child's trailing tiles of that step finish before the lookahead tiles
    // of the next step, which every later step of the critical stream
    // follows) and not before the small-front levels holding its small
    // children were issued.  Small-front level l is issued (on the caller's
    // stream) once the steps up to small_dep[l] are done, small_dep[l] being
    // one past the last panel of the last large child of its fronts.
    c->dsteps.clear();
    c->small_dep.assign(P.nlevels, -1);
    int32_t steps_levels = 0;
    for (const LevelWork &W : c->levels) steps_levels += (int32_t)W.steps.size();
    {
        const int32_t nb = c->opt.nb;
        std::vector<int32_t> g0(ns, 0), gend(ns, -1), small_em(P.nlevels, 0), nsmall_child(ns, -1);
        int32_t T = 0;
        for (int32_t l = 0; l < P.nlevels; l++) {
            for (int32_t t = P.lvl_large_ptr[l]; t < P.lvl_large_ptr[l + 1]; t++) {
                const int32_t s = P.lvl_large[t];
                int32_t g = 0;
                for (int32_t q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
                    const int32_t ch = P.child_list[q];
                    if (P.sn_large[ch]) {
                        g = std::max(g, gend[ch] + 2);
                    } else {
                        g = std::max(g, small_em[P.sn_level[ch]]);
                        nsmall_child[s] = std::max(nsmall_child[s], P.sn_level[ch]);
                    }
                }
                g0[s] = g;
                gend[s] = g + (P.sn_k[s] + nb - 1) / nb - 1;
                T = std::max(T, gend[s] + 1);
            }
            int32_t dep = -1;
            for (int32_t t = P.lvl_small_ptr[l]; t < P.lvl_small_ptr[l + 1]; t++) {
                const int32_t s = P.lvl_small[t];
                for (int32_t q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++)
                    if (P.sn_large[P.child_list[q]]) dep = std::max(dep, gend[P.child_list[q]] + 1);
            }
            c->small_dep[l] = dep;
            small_em[l] = std::max(l > 0 ? small_em[l - 1] : 0, dep + 1);
        }
        c->steps_dependency = T;
        // the order in use
        int32_t lk_steps = 0;
        for (const LevelWork &W : c->levels)
            if (c->opt.level_kernel && W.lvl_cnt > 0 &&
                W.lvl_w.flops / 1.0e12 < c->tune_ratio * W.lvl_chain * 35e-6)
                lk_steps += (int32_t)W.steps.size();
        c->dep_sched = !c->opt.pivoting && P.nlarge > 0 &&
                       (c->opt.schedule == IPM_SCHED_DEPENDENCY ||
                        (c->opt.schedule == IPM_SCHED_AUTO && 5 * (int64_t)T <= 4 * (int64_t)steps_levels &&
                         10 * lk_steps < steps_levels));
        if (c->dep_sched) {
            // fronts by start step; the active set advances one panel per step
            std::vector<std::vector<int32_t>> starting(T);
            for (int32_t s = 0; s < ns; s++)
                if (P.sn_large[s]) starting[g0[s]].push_back(s);
            std::vector<int32_t> active;
            std::vector<std::pair<int32_t, int32_t>> fp;
            for (int32_t g = 0; g < T; g++) {
                // assembly copies of the starting fronts (same ranges as their level items)
                const int64_t aoff = (int64_t)asm_items.size();
                Work aw;
                int32_t swait = -1;
                for (int32_t s : starting[g]) {
                    // one item per 32 columns (splitting the rows too made more,
                    // shorter CTAs that slowed the trailing tiles beside them more
                    // than they sped up the assembly)
                    const int32_t f = P.sn_f[s];
                    for (int32_t cl = 0; cl < f; cl += 32) add_asm(s, cl, std::min(cl + 32, f), cl, f);
                    aw.bytes += front_work(s).bytes;
                    swait = std::max(swait, nsmall_child[s]);
                    active.push_back(s);
                }
                fp.clear();
                for (int32_t s : active) fp.push_back({s, (g - g0[s]) * nb});
                StepWork S = add_step(fp);
                S.asm_off = aoff;
                S.asm_cnt = (int32_t)((int64_t)asm_items.size() - aoff);
                S.asm_w = aw;
                S.small_wait = swait;
                c->dsteps.push_back(S);
                active.erase(std::remove_if(active.begin(), active.end(), [&](int32_t s) { return gend[s] == g; }),
                             active.end());
            }
        }
    }
    c->steps_levels = steps_levels;
    c->nfronts_thin = (int32_t)thin_list.size();
    std::vector<int64_t> upd_off(P.upd_off.begin(), P.upd_off.end());
    std::vector<int32_t> bwd_order(lvl_all.rbegin(), lvl_all.rend());
    c->solve_maxf = P.max_f;
    int rc = 0;
    int32_t *d_c0, *d_k, *d_f, *d_ld, *d_rows, *d_cptr, *d_clist, *d_relmap, *d_odst, *d_perm, *d_kj;
    int64_t *d_off, *d_rptr, *d_moff, *d_optr, *d_osrc, *d_uoff, *d_kp, *d_ksrc;
    int8_t *d_sign;
    std::vector<int64_t> upd_sizes;
    if ((rc = dupload(c, &d_c0, c0)) || (rc = dupload(c, &d_k, P.sn_k)) || (rc = dupload(c, &d_f, P.sn_f)) ||
        (rc = dupload(c, &d_ld, P.sn_ld)) || (rc = dupload(c, &d_off, P.sn_off)) ||
        (rc = dupload(c, &d_rptr, P.sn_rptr)) || (rc = dupload(c, &d_rows, P.sn_rows)) ||
        (rc = dupload(c, &d_cptr, P.child_ptr)) || (rc = dupload(c, &d_clist, P.child_list)) ||
        (rc = dupload(c, &d_moff, P.map_off)) || (rc = dupload(c, &d_relmap, P.relmap)) ||
        (rc = dupload(c, &d_optr, P.orig_ptr)) || (rc = dupload(c, &d_odst, P.orig_dst)) ||
        (rc = dupload(c, &d_osrc, P.orig_src)) || (rc = dupload(c, &d_sign, sign)) ||
        (rc = dupload(c, &d_perm, P.perm)) || (rc = dupload(c, &d_uoff, upd_off)) || (rc = dupload(c, &d_kp, kp)) ||
        (rc = dupload(c, &d_kj, kj)) || (rc = dupload(c, &d_ksrc, ksrc)) ||
        (rc = dupload(c, &c->lvl_small, small_lists)) || (rc = dupload(c, &c->lvl_all, lvl_all)) ||
        (rc = dupload(c, &c->asm_items, asm_items)) || (rc = dupload(c, &c->asm_info, asm_info)) ||
        (rc = dupload(c, &c->asm_cr, asm_cr)) || (rc = dupload(c, &c->panel_items, panel_items)) ||
        (rc = dupload(c, &c->trsm_items, trsm_items)) || (rc = dupload(c, &c->trsm_slots, trsm_slots)) ||
        (rc = dalloc(c, &c->panel_ws, (size_t)std::max(nslots, 1) * kPanelWsHost)) ||
        (rc = dupload(c, &c->tile_items, tile_items)) || (rc = dupload(c, &c->tc_items, tc_items)) ||
        (rc = dupload(c, &c->alt_items, alt_items)) || (rc = dupload(c, &c->bwd_order, bwd_order)) ||
        (rc = dupload(c, &c->trsm_sbase, trsm_sbase)) || (rc = dupload(c, &c->sliced_tiles, sliced_tiles)) ||
        (rc = dupload(c, &c->thin_list, thin_list)) || (rc = dupload(c, &c->thin_asm, thin_asm)) ||
        (rc = dupload(c, &c->thin_slot, thin_slot)) ||
        (rc = dalloc(c, &c->slice_ws, 2 * (size_t)max_slice_blocks * (size_t)kSliceBlockBytes)) ||
        (rc = dalloc(c, &c->slice_exp, 2 * (size_t)std::max<int64_t>(max_slice_blocks, 1) * kSliceRows * 2)) ||
        (rc = dupload(c, &c->lvl_items, lvl_items)) || (rc = dalloc(c, &c->lvl_sync, (size_t)max_ncnt + 1)) ||
        (rc = dalloc(c, &c->solve_sync, (size_t)3 * ns + 1)))
        return rc;
    c->slice_half_blocks = max_slice_blocks;
    int32_t *d_sparent, *d_long;
    if ((rc = dupload(c, &d_sparent, P.sn_parent))) return rc;
    std::vector<int32_t> long_cols;  // columns of K summed by a CTA each in the norm
    for (int32_t i = 0; i < N; i++)
        if (kp[i + 1] - kp[i] > kLongColumn) long_cols.push_back(i);
    if ((rc = dupload(c, &d_long, long_cols))) return rc;
    {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_probe_kernel(), 256,
                                                      (size_t)std::max(P.max_f, kRectRows) * sizeof(double));
        c->solve_grid = std::max(1, std::min(ns, sms * std::max(1, per_sm)));
        int lvl_per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lvl_per_sm, large_level_kernel(), 256, 0);
        c->lvl_grid = sms * std::max(1, lvl_per_sm);
        c->sms = std::max(1, sms);
    }
    DevPlan &dp = c->dp;
    dp.N = N;
    dp.n = P.n;
    dp.m = P.m;
    dp.nsuper = ns;
    dp.form = P.form;
    dp.sn_c0 = d_c0;
    dp.sn_k = d_k;
    dp.sn_f = d_f;
    dp.sn_ld = d_ld;
    dp.sn_off = d_off;
    dp.sn_rptr = d_rptr;
    dp.sn_rows = d_rows;
    dp.child_ptr = d_cptr;
    dp.child_list = d_clist;
    dp.sn_parent = d_sparent;
    dp.map_off = d_moff;
    dp.relmap = d_relmap;
    dp.orig_ptr = d_optr;
    dp.orig_dst = d_odst;
    dp.orig_src = d_osrc;
    dp.sign = d_sign;
    dp.perm = d_perm;
    dp.upd_off = d_uoff;
    dp.kp = d_kp;
    dp.kj = d_kj;
    dp.ksrc = d_ksrc;
    dp.long_cols = d_long;
    dp.nlong = (int32_t)long_cols.size();
    dp.batch_count = 0;
    dp.inst = nullptr;
    dp.inst_norm1 = dp.inst_b1 = nullptr;
    if (P.batch_count > 0) {
        int32_t *d_inst;
        double *d_in, *d_ib;
        if ((rc = dupload(c, &d_inst, P.inst)) || (rc = dalloc(c, &d_in, (size_t)P.batch_count)) ||
            (rc = dalloc(c, &d_ib, (size_t)P.batch_count)))
            return rc;
        dp.batch_count = P.batch_count;
        dp.inst = d_inst;
        dp.inst_norm1 = d_in;
        dp.inst_b1 = d_ib;
    }
    if ((rc = build_solve_schedule(c, lvl_all, bwd_order, d_rows))) return rc;
    const int64_t nnzA = P.Acp[P.n];
    if ((rc = dalloc(c, &c->fronts, (size_t)P.front_doubles)) || (rc = dalloc(c, &c->D, N)) ||
        (rc = dalloc(c, &c->Dinv, N)) ||
        (rc = dalloc(c, &c->dyn, N)) || (rc = dalloc(c, &c->ctl, 1)) || (rc = dalloc(c, &c->Ax, nnzA)) ||
        (rc = dalloc(c, &c->theta, P.n)) ||
        (rc = dalloc(c, &c->vf, N)) || (rc = dalloc(c, &c->vx, N)) || (rc = dalloc(c, &c->vbest, N)) ||
        (rc = dalloc(c, &c->vr, N)) || (rc = dalloc(c, &c->vad, N)) || (rc = dalloc(c, &c->vae, N)) ||
        (rc = dalloc(c, &c->vc, N)) || (rc = dalloc(c, &c->upd, (size_t)std::max<int64_t>(P.upd_total, 1))))
        return rc;
    if (c->opt.pivoting &&
        ((rc = dalloc(c, &c->Doff, N)) || (rc = dalloc(c, &c->bsz, N)) || (rc = dalloc(c, &c->lperm, N))))
        return rc;
    if (P.form == 2) {
        const int32_t n = P.n, m = P.m;
        std::vector<int64_t> arp(m + 1, 0);
        std::vector<int32_t> aci(P.Acp[n]), apos(P.Acp[n]);
        for (int64_t q = 0; q < P.Acp[n]; q++) arp[P.Ari[q] + 1]++;
        for (int32_t i = 0; i < m; i++) arp[i + 1] += arp[i];
        std::vector<int64_t> fill(arp.begin(), arp.end() - 1);
        for (int32_t j = 0; j < n; j++)
            for (int64_t q = P.Acp[j]; q < P.Acp[j + 1]; q++) {
                aci[fill[P.Ari[q]]] = j;
                apos[fill[P.Ari[q]]++] = (int32_t)q;
            }
        int64_t *d_tptr, *d_arp, *d_acp;
        int32_t *d_ta, *d_tb, *d_tj, *d_aci, *d_apos, *d_ari;
        std::vector<int64_t> acp(P.Acp.begin(), P.Acp.end());
        if ((rc = dupload(c, &d_tptr, P.ne_tptr)) || (rc = dupload(c, &d_ta, P.ne_ta)) ||
            (rc = dupload(c, &d_tb, P.ne_tb)) || (rc = dupload(c, &d_tj, P.ne_tj)) || (rc = dupload(c, &d_arp, arp)) ||
            (rc = dupload(c, &d_aci, aci)) || (rc = dupload(c, &d_apos, apos)) || (rc = dupload(c, &d_acp, acp)) ||
            (rc = dupload(c, &d_ari, P.Ari)) || (rc = dalloc(c, &c->ne.tt, n)) ||
            (rc = dalloc(c, &c->ne.nev, (size_t)P.ne_cp[N])) || (rc = dalloc(c, &c->kf, (size_t)n + m)) ||
            (rc = dalloc(c, &c->kr, (size_t)n + m)) || (rc = dalloc(c, &c->kad, (size_t)n + m)) ||
            (rc = dalloc(c, &c->kae, (size_t)n + m)))
            return rc;
        c->ne.n = n;
        c->ne.m = m;
        c->ne.nnz = P.ne_cp[N];
        c->ne.tptr = d_tptr;
        c->ne.ta = d_ta;
        c->ne.tb = d_tb;
        c->ne.tj = d_tj;
        c->ne.Arp = d_arp;
        c->ne.Aci = d_aci;
        c->ne.Apos = d_apos;
        c->ne.Acp = d_acp;
        c->ne.Ari = d_ari;
    }
    cudaMemset(c->ctl, 0, sizeof(DevCtl));
    cudaMemset(c->fronts, 0, (size_t)std::max<int64_t>(P.front_doubles, 1) * sizeof(double));
    c->mixed_active = c->opt.precision != IPM_PREC_FP64;
    c->fallbacks = 0;
    c->resid_w.flops = 6.0 * (double)kp[N];
    c->resid_w.bytes = 20.0 * (double)kp[N] + 48.0 * N;
    c->dev_ready = true;
    return to_err(cudaGetLastError());
}

// CTAs of the level kernel: every SM full, or tune_lvl_per_sm per SM.
static int32_t level_grid(const ipm_ctx *c) {
    if (c->tune_lvl_per_sm <= 0) return c->lvl_grid;
    return std::max(1, std::min(c->lvl_grid, c->sms * c->tune_lvl_per_sm));
}

int factorise_enqueue(ipm_ctx *c, const double *theta, double rho, double delta, cudaStream_t st) {
    const Plan &P = c->plan;
    DevVals V{};
    V.Ax = c->Ax;
    V.theta = theta;
    V.nev = c->ne.nev;
    V.rho = rho;
    V.delta = delta;
    V.large_reg = c->opt.large_reg;
    int nl = 0;
    if (P.form == 2) {
        Prof pr(c, IPM_K_OTHER, Work(), st);
        launch_ne_form(c->ne, c->Ax, theta, rho, c->ctl, st);
        nl += 2;
    }
    // reset the per-factorisation fields of the control block
    cudaMemsetAsync(&c->ctl->ndyn, 0, offsetof(DevCtl, omega) - offsetof(DevCtl, ndyn), st);
    {
        Prof pr(c, IPM_K_OTHER, Work(), st);
        launch_norm1(c->dp, V, c->ctl, c->opt.eps_piv, st);
    }
    nl += 2;
    if (c->opt.pivoting) {
        // Sec. 4.5 pivoting: one CTA per front, the tree's levels in order
        for (int32_t l = 0; l < P.nlevels; l++) {
            const LevelWork &W = c->levels[l];
            Prof pr(c, IPM_K_LARGE_PANEL, W.lvl_w, st);
            launch_front_bk(c->dp, V, c->fronts, c->D, c->Doff, c->bsz, c->lperm, c->dyn, c->ctl,
                            c->lvl_all + W.all_off, W.all_cnt, c->opt.nb, st);
            nl++;
        }
        {
            Prof pr(c, IPM_K_OTHER, Work(), st);
            launch_factor_stats_bk(c->D, c->Doff, c->bsz, c->dyn, P.N, c->opt.large_reg, c->ctl, st);
        }
        nl++;
        c->nl_factor = nl;
        return to_err(cudaGetLastError());
    }
    // Small fronts run on the caller's stream and the large fronts of the
    // same level on a second stream: fronts of one level are independent
    // (Sec. 4.3, tree-level parallelism), so a level costs the longer of the
    // two instead of their sum.  Level l's small fronts wait for the large
    // fronts of level l-1 and vice versa (events; a captured graph keeps them
    // as edges).
    if (!c->side) {
        // the large fronts' per-step chain (diagonal block, triangular solve,
        // lookahead update) is the factorisation's critical path: its stream
        // gets the highest priority, so its CTAs go first when the trailing
        // updates running beside it on side2 release SMs
        int prio_lo = 0, prio_hi = 0;
        cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
        if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
            cudaGetLastError();
            c->side = nullptr;
            return IPM_ERR_CUDA;
        }
    }
    const size_t nev = 5 * (size_t)P.nlevels + 2;  // per level: fork, two joins, small done, large done
    while (c->dep_ev.size() < nev) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        c->dep_ev.push_back(e);
    }
    for (cudaStream_t *q : {&c->side2, &c->cls[0], &c->cls[1]}) {
        if (!*q && cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            *q = nullptr;
            return IPM_ERR_CUDA;
        }
    }
    size_t nsteps = c->dsteps.size();
    for (const LevelWork &W : c->levels) nsteps += W.steps.size();
    while (c->step_ev.size() < 2 * nsteps) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        c->step_ev.push_back(e);
    }
    while (c->done_ev.size() < c->dsteps.size() + 1) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        c->done_ev.push_back(e);
    }
    cudaStream_t sd = c->side, sd2 = c->side2;
    size_t sidx = 0;
    cudaEventRecord(c->dep_ev[0], st);
    cudaStreamWaitEvent(sd, c->dep_ev[0], 0);
    cudaEvent_t last_small = nullptr, last_large = nullptr;
    // the small fronts of level l on the caller's stream, one stream per size
    // class (the classes of a level are independent); records last_small
    auto emit_small = [&](int32_t l) {
        const LevelWork &W = c->levels[l];
        cudaEvent_t fork = c->dep_ev[1 + 5 * l];
        if (W.small.size() > 1) cudaEventRecord(fork, st);
        for (size_t q = 0; q < W.small.size(); q++) {
            const SmallClass &C = W.small[q];
            cudaStream_t sq = q == 0 ? st : c->cls[(q - 1) & 1];
            if (q > 0) cudaStreamWaitEvent(sq, fork, 0);
            Prof pr(c, IPM_K_SMALL_FRONTS, C.w, sq);
            launch_small_fronts(c->dp, V, c->fronts, c->D, c->Dinv, c->dyn, c->ctl, c->lvl_small + C.off, C.cnt,
                                c->opt.nb, C.maxf, c->tune_threads[C.cls], sq);
            nl++;
            if (q > 0) {
                cudaEvent_t join = c->dep_ev[2 + 5 * l + (q - 1)];
                cudaEventRecord(join, sq);
                cudaStreamWaitEvent(st, join, 0);
            }
        }
        last_small = c->dep_ev[4 + 5 * l];
        cudaEventRecord(last_small, st);
    };
    // Per 32-column step: diagonal blocks and triangular solves, then the
    // update split in two.  The tiles of the next panel's columns (lookahead)
    // stay on the critical path; the remaining trailing tiles run on a third
    // stream beside the next step's diagonal blocks.  Every entry still
    // receives the panels' updates in panel order: the lookahead tiles of
    // step s wait for the remaining tiles of step s-1.
    cudaEvent_t prev_rest = nullptr;
    auto emit_step = [&](const StepWork &S) {
        {
            Prof pr(c, IPM_K_PIVOT_BLOCK, S.panel_w, sd);
            launch_panel_diag(c->dp, V, c->fronts, c->D, c->Dinv, c->dyn, c->ctl, c->panel_items + S.panel_off,
                              S.panel_cnt, c->opt.nb, c->panel_ws, sd);
        }
        nl++;
        const bool use_tc = (S.tc_cnt > 0 || S.st_cnt > 0) && c->mixed_active;
        const bool use_sliced = use_tc && S.st_cnt > 0;
        // sliced path: the digit images of this step (alternate halves of the
        // work space: the rest of step s-1 may still read its half while
        // step s slices; step s+1 slices only after step s's lookahead,
        // which waits for the rest of step s-1)
        uint8_t *ws = c->slice_ws + (sidx & 1) * c->slice_half_blocks * kSliceBlockBytes;
        int32_t *wexp = c->slice_exp + (sidx & 1) * c->slice_half_blocks * kSliceRows * 2;
        if (S.trsm_cnt > 0) {
            // on the sliced path the solve also writes the slices of the rows it finishes
            Prof pr(c, IPM_K_LARGE_PANEL, S.trsm_w, sd);
            launch_panel_trsm(c->dp, c->fronts, c->trsm_items + S.trsm_off, c->trsm_slots + S.trsm_off, S.trsm_cnt,
                              c->opt.nb, c->panel_ws, sd, c->trsm_sbase + S.trsm_off, use_sliced ? ws : nullptr,
                              wexp, c->D, c->ctl);
            nl++;
        }
        const int32_t rest_tiles = S.tile_cnt - S.tile_cnt1;
        const int32_t rest_alt = ((S.tc_cnt > 0 || S.st_cnt > 0) && !c->mixed_active) ? S.alt_cnt - S.alt_cnt1 : 0;
        const int32_t rest_sliced = use_sliced ? S.st_cnt - S.st_cnt1 : 0;
        cudaEvent_t this_rest = nullptr;
        if (rest_tiles > 0 || rest_alt > 0 || rest_sliced > 0) {
            cudaEvent_t ev_in = c->step_ev[2 * sidx], ev_out = c->step_ev[2 * sidx + 1];
            cudaEventRecord(ev_in, sd);
            cudaStreamWaitEvent(sd2, ev_in, 0);
            if (rest_tiles > 0) {
                Prof pr(c, IPM_K_LARGE_UPDATE, S.tile_w, sd2);
                launch_large_update(c->dp, c->fronts, c->D, c->tile_items + S.tile_off + S.tile_cnt1, rest_tiles,
                                    c->opt.nb, sd2);
                nl++;
            }
            if (rest_alt > 0) {
                Prof pr(c, IPM_K_LARGE_UPDATE, S.alt_w, sd2);
                launch_large_update(c->dp, c->fronts, c->D, c->alt_items + S.alt_off + S.alt_cnt1, rest_alt,
                                    c->opt.nb, sd2);
                nl++;
            }
            if (rest_sliced > 0) {
                Prof pr(c, IPM_K_LARGE_UPDATE_TC, S.st_w2, sd2);
                launch_update_sliced(c->dp, c->fronts, c->sliced_tiles + S.st_off + S.st_cnt1, rest_sliced, ws, wexp,
                                     c->ctl, sd2);
                nl++;
            }
            cudaEventRecord(ev_out, sd2);
            this_rest = ev_out;
        }
        sidx++;
        if (prev_rest) cudaStreamWaitEvent(sd, prev_rest, 0);
        if (S.tile_cnt1 > 0) {
            Prof pr(c, IPM_K_LARGE_UPDATE, S.tile_w1, sd);
            launch_large_update_strip(c->dp, c->fronts, c->D, c->tile_items + S.tile_off, S.tile_cnt1, c->opt.nb,
                                      sd);
            nl++;
        }
        if ((S.tc_cnt > 0 || S.st_cnt > 0) && !c->mixed_active && S.alt_cnt1 > 0) {
            Prof pr(c, IPM_K_LARGE_UPDATE, S.alt_w1, sd);
            launch_large_update_strip(c->dp, c->fronts, c->D, c->alt_items + S.alt_off, S.alt_cnt1, c->opt.nb, sd);
            nl++;
        } else if (use_sliced) {
            if (S.st_cnt1 > 0) {
                Prof pr(c, IPM_K_LARGE_UPDATE_TC, S.st_w1, sd);
                launch_update_sliced(c->dp, c->fronts, c->sliced_tiles + S.st_off, S.st_cnt1, ws, wexp, c->ctl, sd);
                nl++;
            }
        } else if (use_tc) {
            Prof pr(c, IPM_K_LARGE_UPDATE_TC, S.tc_w, sd);
            launch_large_update_tc(c->dp, c->fronts, c->D, c->tc_items + S.tc_off, S.tc_cnt, c->opt.nb, c->ctl, sd);
            nl++;
        }
        prev_rest = this_rest;
    };
    if (c->dep_sched) {
        // Dependency order: the steps of all large fronts in one sequence on
        // the critical stream; each small-front level is issued on the
        // caller's stream as soon as the steps its large children need are
        // done, and a front's assembly waits for the level of its small
        // children.  Every wait refers to an event recorded earlier in issue
        // order, so a capture keeps them as edges.
        const int32_t T = (int32_t)c->dsteps.size();
        int32_t next = 0;  // next small-front level to issue
        auto issue_small = [&](int32_t g) {
            while (next < P.nlevels && c->small_dep[next] < g) {
                if (!c->levels[next].small.empty()) {
                    if (c->small_dep[next] >= 0) cudaStreamWaitEvent(st, c->done_ev[c->small_dep[next]], 0);
                    emit_small(next);
                }
                next++;
            }
        };
        for (int32_t g = 0; g < T; g++) {
            issue_small(g);
            const StepWork &S = c->dsteps[g];
            if (S.small_wait >= 0) cudaStreamWaitEvent(sd, c->dep_ev[4 + 5 * S.small_wait], 0);
            if (S.asm_cnt > 0) {
                Prof pr(c, IPM_K_LARGE_ASSEMBLE, S.asm_w, sd);
                launch_large_assemble(c->dp, V, c->fronts, c->asm_items + S.asm_off, c->asm_info + S.asm_off,
                                      c->asm_cr, S.asm_cnt, sd);
                nl++;
            }
            emit_step(S);
            cudaEventRecord(c->done_ev[g], sd);
        }
        if (prev_rest) cudaStreamWaitEvent(sd, prev_rest, 0);
        cudaEventRecord(c->done_ev[T], sd);
        issue_small(INT32_MAX);
    } else {
        // Level order: small fronts on the caller's stream and the large
        // fronts of the same level on a second stream (fronts of one level
        // are independent, Sec. 4.3), so a level costs the longer of the two
        // instead of their sum.  Level l's small fronts wait for the large
        // fronts of level l-1 and vice versa.
        for (int32_t l = 0; l < P.nlevels; l++) {
            const LevelWork &W = c->levels[l];
            cudaEvent_t small_before = last_small, large_before = last_large;
            if (!W.small.empty()) {
                if (large_before) cudaStreamWaitEvent(st, large_before, 0);
                emit_small(l);
            }
            if (W.asm_cnt == 0 && W.steps.empty() && W.thin_cnt == 0) continue;
            if (small_before) cudaStreamWaitEvent(sd, small_before, 0);
            const bool latency_bound = W.lvl_w.flops / 1.0e12 < c->tune_ratio * W.lvl_chain * 35e-6;
            // (a latency-bound level keeps the FP64 level kernel in the tensor-core
            // modes too: its work is too small for the tensor cores to matter)
            if (c->opt.level_kernel && W.lvl_cnt > 0 && latency_bound) {
                // FP64: all large-front work of the level in one dependency-driven launch
                {
                    Prof pr(c, IPM_K_LARGE_PANEL, W.lvl_w, sd);
                    launch_large_level(c->dp, V, c->fronts, c->D, c->Dinv, c->dyn, c->ctl, c->lvl_items + W.lvl_off,
                                       W.lvl_cnt, c->lvl_sync, W.lvl_ncnt, c->asm_info, c->asm_cr, c->panel_ws,
                                       c->opt.nb, level_grid(c),
                                       c->opt.spin_limit_log2 < 0 ? 0 : (1ll << c->opt.spin_limit_log2), sd);
                }
                nl++;
                last_large = c->dep_ev[5 + 5 * l];
                cudaEventRecord(last_large, sd);
                continue;
            }
            if (W.asm_cnt2 > 0) {
                Prof pr(c, IPM_K_LARGE_ASSEMBLE, W.asm_w, sd);
                launch_large_assemble(c->dp, V, c->fronts, c->asm_items + W.asm_off2, c->asm_info + W.asm_off2,
                                      c->asm_cr, W.asm_cnt2, sd);
                nl++;
            }
            if (W.thin_cnt > 0) {
                Prof pr(c, IPM_K_LARGE_PANEL, W.thin_w, sd);
                launch_thin_fronts(c->dp, V, c->fronts, c->D, c->Dinv, c->dyn, c->ctl, c->thin_list + W.thin_off,
                                   c->thin_asm + W.thin_off, c->thin_slot + W.thin_off, c->asm_info, c->asm_cr,
                                   c->panel_ws, W.thin_cnt, c->opt.nb, sd);
                nl++;
            }
            prev_rest = nullptr;
            for (const StepWork &S : W.steps) emit_step(S);
            if (prev_rest) cudaStreamWaitEvent(sd, prev_rest, 0);
            last_large = c->dep_ev[5 + 5 * l];
            cudaEventRecord(last_large, sd);
        }
    }
    // join: the second stream always rejoins the caller's stream (a capture
    // needs every forked stream joined back)
    cudaEventRecord(c->dep_ev[nev - 1], sd);
    cudaStreamWaitEvent(st, c->dep_ev[nev - 1], 0);
    if (c->ninv > 0) {
        Prof pr(c, IPM_K_OTHER, Work(), st);
        launch_diag_inverse(c->sched, c->fronts, c->linv, c->inv_items, c->ninv, c->pair_items, c->npairs, st);
        nl += c->npairs > 0 ? 2 : 1;
    }
    {
        Prof pr(c, IPM_K_OTHER, Work(), st);
        launch_factor_stats(c->D, c->dyn, P.N, c->opt.large_reg, c->ctl, st);
    }
    nl++;
    c->nl_factor = nl;
    return to_err(cudaGetLastError());
}

// x <- (L D L^T)^-1 x in the factorisation order: one persistent launch per
// sweep (dependency-driven, see kernels_solve.cu).
int solve_inplace(ipm_ctx *c, double *x, cudaStream_t st, int *nl) {
    const Plan &P = c->plan;
    if (c->opt.pivoting) {
        // per-level sweeps with the fronts' interchanges and 1x1 / 2x2 blocks of D
        for (int32_t l = 0; l < P.nlevels; l++) {
            const LevelWork &W = c->levels[l];
            Prof pr(c, IPM_K_FORWARD, W.fwd_w, st);
            launch_forward_bk(c->dp, c->fronts, c->D, c->Doff, c->bsz, c->lperm, x, c->upd,
                              c->lvl_all + W.all_off, W.all_cnt, W.all_maxf, st);
        }
        for (int32_t l = P.nlevels - 1; l >= 0; l--) {
            const LevelWork &W = c->levels[l];
            Prof pr(c, IPM_K_BACKWARD, W.bwd_w, st);
            launch_backward_bk(c->dp, c->fronts, c->lperm, x, c->lvl_all + W.all_off, W.all_cnt, W.all_maxf, st);
        }
        *nl += 2 * P.nlevels;
        return to_err(cudaGetLastError());
    }
    Work fw, bw;
    for (const LevelWork &W : c->levels) {
        fw.flops += W.fwd_w.flops;
        fw.bytes += W.fwd_w.bytes;
        bw.flops += W.bwd_w.flops;
        bw.bytes += W.bwd_w.bytes;
    }
    {
        Prof pr(c, IPM_K_FORWARD, fw, st);
        launch_forward_persistent(c->sched, c->fronts, c->Dinv, x, c->upd, c->solve_maxf, c->solve_grid, c->ctl, st);
    }
    {
        Prof pr(c, IPM_K_BACKWARD, bw, st);
        launch_backward_persistent(c->sched, c->fronts, x, c->solve_maxf, c->solve_grid, c->ctl, st);
    }
    *nl += 4;  // per sweep: the reset of its counters and chain values, then the sweep
    return to_err(cudaGetLastError());
}

// The GMRES refinement of a captured graph: a conditional node whose body
// (captured on a second stream) runs only when classical refinement ended
// above the target; inside it every kernel tests the device-side flags of
// GmDev, so cycles and Arnoldi steps that are not needed return at entry.
int capture_gmres(ipm_ctx *c, const DevVals &V, cudaStream_t st) {
    const Plan &P = c->plan;
    const int64_t N = P.N;
    const int m = kGmresM;
    const double target = c->opt.omega_target;
    const int R = c->opt.gmres_restarts;
    GmDev *gm = c->gm_dev;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusActive) return IPM_ERR_CUDA;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, 0)) != cudaSuccess) return to_err(e);
    launch_gm_begin(c->ctl, gm, target, (unsigned long long)h, st);
    if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd)) != cudaSuccess) return to_err(e);
    cudaGraphNodeParams prm{};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeIf;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, ed, nd, &prm)) != cudaSuccess) return to_err(e);
    cudaGraph_t body = prm.conditional.phGraph_out[0];
    if ((e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return to_err(e);
    if (!c->gm_stream && (e = cudaStreamCreateWithFlags(&c->gm_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        c->gm_stream = nullptr;
        return to_err(e);
    }
    cudaStream_t s2 = c->gm_stream;
    if ((e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess)
        return to_err(e);
    launch_copy_if(c->vx, c->vbest, (int32_t)N, nullptr, 0, s2);
    for (int r = 0; r <= R; r++) {
        // r = f - K x and omega of the current x; keep it if it improved
        launch_residual_omega(c->dp, V, c->vf, c->vx, c->vr, c->vad, c->vae, c->ctl, s2, &gm->stop);
        launch_gm_cycle(c->ctl, gm, target, r, R, s2);
        launch_copy_if(c->vbest, c->vx, (int32_t)N, &gm->improved, 0, s2);
        if (r == R) break;
        launch_dots(c->vr, c->vr, N, 1, c->gm_part, gm->h, s2, &gm->stop);
        launch_gm_init(c->ctl, gm, target, s2);
        launch_scale_dev(c->gm_V, c->vr, gm, NAN, N, &gm->stop, s2);
        for (int j = 0; j < m; j++) {
            double *vj = c->gm_V + (int64_t)j * N, *zj = c->gm_Z + (int64_t)j * N, *vn = vj + N;
            launch_copy_if(zj, vj, (int32_t)N, &gm->skip_inner, 1, s2);
            launch_forward_persistent(c->sched, c->fronts, c->Dinv, zj, c->upd, c->solve_maxf, c->solve_grid, c->ctl,
                                      s2, &gm->skip_inner);
            launch_backward_persistent(c->sched, c->fronts, zj, c->solve_maxf, c->solve_grid, c->ctl, s2,
                                       &gm->skip_inner);
            launch_residual_omega(c->dp, V, c->gm_zero, zj, c->gm_w, c->vad, c->vae, c->ctl, s2, &gm->skip_inner);
            launch_scale_dev(vn, c->gm_w, gm, -1.0, N, &gm->skip_inner, s2);  // K z
            for (int pass = 0; pass < 2; pass++) {
                launch_dots(vn, c->gm_V, N, j + 1, c->gm_part, gm->h, s2, &gm->skip_inner);
                launch_gs_update_dev(vn, c->gm_V, gm, N, j + 1, s2);
                launch_gm_hacc(gm, j, s2);
            }
            launch_dots(vn, vn, N, 1, c->gm_part, gm->h, s2, &gm->skip_inner);
            launch_gm_arnoldi(gm, j, s2);
            launch_scale_dev(vn, vn, gm, NAN, N, &gm->skip_inner, s2);
        }
        launch_gm_ls(gm, s2);
        launch_combine_dev(c->vx, c->gm_Z, gm, N, s2);
    }
    launch_gm_end(c->ctl, gm, s2);
    cudaGraph_t out = nullptr;
    const cudaError_t e1 = cudaGetLastError();
    e = cudaStreamEndCapture(s2, &out);
    if (e1 != cudaSuccess) return to_err(e1);
    return to_err(e);
}


// GMRES refines an FP64-accurate factor (FP64 or sliced updates); a stalled
// 3xTF32 factor is replaced by an FP64 one instead
bool gmres_allowed(const ipm_ctx *c) {
    return c->opt.gmres_restarts > 0 && !(c->opt.precision == IPM_PREC_MIXED && c->mixed_active);
}

// Refined solve with all decisions taken on the device, so it can be
// captured into a CUDA graph: refine_max steps are enqueued and every kernel
// of a step exits at entry once the control block says the refinement is
// done (omega <= target, omega failed to halve, or the step limit).
int solve_device_driven(ipm_ctx *c, const double *r7, const double *r1, double *dx, double *dy, cudaStream_t st) {
    const Plan &P = c->plan;
    const int32_t N = P.N;
    DevVals V{};
    V.Ax = c->Ax;
    V.theta = c->theta;
    V.rho = c->rho;
    V.delta = c->delta;
    const int32_t *done = &c->ctl->done;
    const int32_t *improved = &c->ctl->improved;
    const double target = c->opt.omega_target;
    const int32_t rmax = c->opt.refine_max;
    V.nev = c->ne.nev;
    if (P.form == 2) launch_ne_rhs(c->ne, c->dp.perm, c->Ax, r7, r1, c->vf, st);
    else launch_permute_in(c->dp, r7, r1, c->vf, st);
    launch_copy_if(c->vx, c->vf, N, nullptr, 0, st);
    launch_forward_persistent(c->sched, c->fronts, c->Dinv, c->vx, c->upd, c->solve_maxf, c->solve_grid, c->ctl, st);
    launch_backward_persistent(c->sched, c->fronts, c->vx, c->solve_maxf, c->solve_grid, c->ctl, st);
    launch_residual_omega(c->dp, V, c->vf, c->vx, c->vr, c->vad, c->vae, c->ctl, st);
    launch_refine_init(c->ctl, target, rmax, st);
    launch_copy_if(c->vbest, c->vx, N, nullptr, 0, st);
    for (int32_t step = 1; step <= rmax; step++) {
        launch_copy_if(c->vc, c->vr, N, done, 1, st);
        launch_forward_persistent(c->sched, c->fronts, c->Dinv, c->vc, c->upd, c->solve_maxf, c->solve_grid, c->ctl, st,
                                  done);
        launch_backward_persistent(c->sched, c->fronts, c->vc, c->solve_maxf, c->solve_grid, c->ctl, st, done);
        launch_axpy(c->vx, c->vc, N, st, done);
        launch_residual_omega(c->dp, V, c->vf, c->vx, c->vr, c->vad, c->vae, c->ctl, st, done);
        launch_refine_step(c->ctl, target, step, rmax, st);
        launch_copy_if(c->vbest, c->vx, N, improved, 0, st);
    }
    if (c->gm_dev && gmres_allowed(c)) {
        int rc = capture_gmres(c, V, st);
        if (rc) return rc;
    }
    launch_refine_finish(c->ctl, target, st);
    launch_permute_out(c->dp, c->vbest, dx, dy, st);
    if (P.form == 2) launch_ne_dx(c->ne, c->Ax, dy, r7, dx, st);
    return to_err(cudaGetLastError());
}

int check_ctx(const ipm_ctx *c) {
    if (!c) return IPM_ERR_INVALID_ARG;
    if (!c->analysed) return IPM_ERR_NOT_ANALYSED;
    return IPM_OK;
}

int status_to_code(int32_t st) {
    if (st & kStatNonFinite) return IPM_ERR_NONFINITE;
    if (st & kStatTimeout) return IPM_ERR_DEVICE_TIMEOUT;
    if (st & kStatRefineFail) return IPM_WARN_REFINE_NOT_CONVERGED;
    if (st & kStatLargeReg) return IPM_WARN_LARGE_REG;
    if (st & kStatDynReg) return IPM_WARN_DYNREG_APPLIED;
    return IPM_OK;
}

}  // namespace

extern "C" {

void ipm_default_options(ipm_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->nb = 32;
    o->amalg_width = 16;
    o->amalg_zero_frac = -1.0;
    o->eps_piv = 2.220446049250313e-16;  // machine precision (Sec. 4.5)
    o->large_reg = 1e-4;
    o->precision = IPM_PREC_FP64;
    o->mixed_min_front = 256;
    o->omega_target = 1e-12;
    o->refine_max = 10;
    o->gmres_restarts = 6;
    o->nd_leaf = 128;
    o->dense_row_factor = 10.0;
    o->device = 0;
    o->spin_limit_log2 = 24;
    o->level_kernel = 1;
    o->pivoting = 0;
    o->schedule = IPM_SCHED_AUTO;
    o->verbose = 0;
}

int ipm_create(ipm_ctx **out, const ipm_options *opt) {
    if (!out) return IPM_ERR_INVALID_ARG;
    ipm_ctx *c = new (std::nothrow) ipm_ctx();
    if (!c) return IPM_ERR_OOM;
    if (opt) c->opt = *opt;
    else ipm_default_options(&c->opt);
    if (c->opt.nb != 32 || c->opt.refine_max < 0 || c->opt.refine_max > 15 ||
        c->opt.gmres_restarts < 0 || c->opt.gmres_restarts > 16 ||
        c->opt.spin_limit_log2 < -1 || c->opt.spin_limit_log2 > 40 || !(c->opt.eps_piv >= 0.0) ||
        c->opt.level_kernel < 0 || c->opt.level_kernel > 1 ||
        (c->opt.precision != IPM_PREC_FP64 && c->opt.precision != IPM_PREC_MIXED &&
         c->opt.precision != IPM_PREC_SLICED) ||
        c->opt.mixed_min_front < 1 || c->opt.pivoting < 0 || c->opt.pivoting > 1 || c->opt.schedule < 0 ||
        c->opt.schedule > IPM_SCHED_DEPENDENCY ||
        (c->opt.pivoting && c->opt.precision != IPM_PREC_FP64)) {
        delete c;
        return IPM_ERR_INVALID_ARG;
    }
    *out = c;
    return IPM_OK;
}

int ipm_destroy(ipm_ctx *c) {
    if (!c) return IPM_ERR_INVALID_ARG;
    if (c->dev_ready) {
        cudaSetDevice(c->opt.device);
        cudaDeviceSynchronize();
    }
    free_device(c);
    delete c;
    return IPM_OK;
}

int ipm_analyse(ipm_ctx *c, int32_t m, int32_t n, const int64_t *colptr, const int32_t *rowidx, int32_t form,
                int32_t ordering, const int32_t *user_perm) {
    if (!c) return IPM_ERR_INVALID_ARG;
    if (form != IPM_FORM_AUTO && form != IPM_FORM_AUGMENTED && form != IPM_FORM_NORMAL) return IPM_ERR_INVALID_ARG;
    if (form == IPM_FORM_AUTO && ordering == IPM_ORD_USER) return IPM_ERR_INVALID_ARG;  // order size depends on the form
    if (c->opt.pivoting) {
        if (form == IPM_FORM_NORMAL) return IPM_ERR_INVALID_ARG;  // pivoting is for the indefinite K only
        form = IPM_FORM_AUGMENTED;
    }
    AnalyseOptions ao;
    ao.nb = c->opt.nb;
    ao.amalg_width = c->opt.amalg_width;
    ao.amalg_zero_frac = c->opt.amalg_zero_frac;
    ao.nd_leaf = c->opt.nd_leaf;
    ao.dense_row_factor = c->opt.dense_row_factor;
    ao.verbose = c->opt.verbose;
    std::string err;
    if (c->dev_ready) {
        cudaSetDevice(c->opt.device);
        cudaDeviceSynchronize();
    }
    free_device(c);
    c->analysed = false;
    auto t0 = std::chrono::steady_clock::now();
    int rc;
    if (form == IPM_FORM_AUTO) {
        // Sec. 4.2: the augmented-system symbolic first; forming the normal
        // equations is abandoned as soon as they hold more entries than L of
        // the augmented system, otherwise the modelled per-iteration costs
        // decide (factorisation flops at the FP64 rate, three solves' worth of
        // L traffic at HBM bandwidth, the formation of A Theta~ A^T; ties go
        // to the augmented system)
        constexpr double kFlop = 1.0e12, kBw = 6.7e12;
        Plan pas;
        rc = analyse(pas, m, n, colptr, rowidx, 1, ordering, user_perm, ao, err);
        if (rc) {
            if (c->opt.verbose) std::fprintf(stderr, "[ipm analyse] %s\n", err.c_str());
            return rc;
        }
        const double cost_as = pas.flops / kFlop + 3.0 * 2.0 * (double)pas.nnzL * 8.0 / kBw;
        const int64_t ne_seen = count_ne_lower(m, n, colptr, rowidx, pas.nnzL);
        double cost_ne = -1.0;
        bool use_ne = false;
        Plan pne;
        if (ne_seen <= pas.nnzL) {
            std::string err2;
            if (analyse(pne, m, n, colptr, rowidx, 2, ordering, nullptr, ao, err2) == 0) {
                const double pairs = (double)pne.ne_tptr.back();
                cost_ne = (pne.flops + 2.0 * pairs) / kFlop + 3.0 * 2.0 * (double)pne.nnzL * 8.0 / kBw;
                use_ne = cost_ne < cost_as;
            }
        }
        c->plan = use_ne ? std::move(pne) : std::move(pas);
        c->plan.est_as = cost_as;
        c->plan.est_ne = cost_ne;
        c->plan.nnz_ne_seen = ne_seen;
    } else {
        rc = analyse(c->plan, m, n, colptr, rowidx, form, ordering, user_perm, ao, err);
        if (rc) {
            if (c->opt.verbose) std::fprintf(stderr, "[ipm analyse] %s\n", err.c_str());
            return rc;
        }
    }
    c->plan.batch_count = 0;
    c->plan.inst.clear();
    c->ms_analyse = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c->analysed = true;
    return IPM_OK;
}

int ipm_save_analysis(const ipm_ctx *c, const char *path) {
    if (!c || !path) return IPM_ERR_INVALID_ARG;
    if (!c->analysed) return IPM_ERR_NOT_ANALYSED;
    std::string err;
    if (plan_save(c->plan, path, err)) {
        if (c->opt.verbose) std::fprintf(stderr, "[ipm save] %s\n", err.c_str());
        return IPM_ERR_INVALID_ARG;
    }
    return IPM_OK;
}

int ipm_load_analysis(ipm_ctx *c, const char *path) {
    if (!c || !path) return IPM_ERR_INVALID_ARG;
    Plan Q;
    std::string err;
    if (plan_load(Q, path, err)) {
        if (c->opt.verbose) std::fprintf(stderr, "[ipm load] %s\n", err.c_str());
        return IPM_ERR_INVALID_ARG;
    }
    if (c->dev_ready) {
        cudaSetDevice(c->opt.device);
        cudaDeviceSynchronize();
    }
    free_device(c);
    c->plan = std::move(Q);
    c->ms_analyse = 0.0;
    c->analysed = true;
    return IPM_OK;
}

int ipm_analyse_batch(ipm_ctx *c, int32_t count, const int32_t *ms, const int32_t *ns, const int64_t *colptrs,
                      const int32_t *rowidxs, int32_t ordering) {
    if (!c || count <= 0 || !ms || !ns || !colptrs || !rowidxs) return IPM_ERR_INVALID_ARG;
    int64_t M = 0, Nn = 0;
    for (int32_t b = 0; b < count; b++) {
        if (ms[b] < 0 || ns[b] < 0) return IPM_ERR_INVALID_ARG;
        M += ms[b];
        Nn += ns[b];
    }
    if (M + Nn > INT32_MAX) return IPM_ERR_INVALID_ARG;
    // block-diagonal A: instance b's columns follow instance b-1's, its rows are shifted by sum m
    std::vector<int64_t> cp(Nn + 1, 0);
    std::vector<int32_t> ri;
    int64_t cpo = 0, rio = 0, col = 0, roff = 0;
    for (int32_t b = 0; b < count; b++) {
        const int64_t *cpb = colptrs + cpo;
        if (cpb[0] != 0) return IPM_ERR_INVALID_ARG;
        for (int32_t j = 0; j < ns[b]; j++) {
            if (cpb[j + 1] < cpb[j]) return IPM_ERR_INVALID_ARG;
            for (int64_t p = cpb[j]; p < cpb[j + 1]; p++) {
                const int32_t r = rowidxs[rio + p];
                if (r < 0 || r >= ms[b]) return IPM_ERR_INVALID_ARG;
                ri.push_back((int32_t)(roff + r));
            }
            cp[col + j + 1] = (int64_t)ri.size();
        }
        rio += cpb[ns[b]];
        cpo += ns[b] + 1;
        col += ns[b];
        roff += ms[b];
    }
    const int rc = ipm_analyse(c, (int32_t)M, (int32_t)Nn, cp.data(), ri.data(), IPM_FORM_AUGMENTED, ordering,
                               nullptr);
    if (rc) return rc;
    // instance of every unknown, in the factorisation order: the pivot floor
    // eps_piv ||K||_1 of Sec. 4.5 is taken per instance, so that each problem
    // is factorised exactly as it would be on its own
    Plan &P = c->plan;
    P.batch_count = count;
    P.inst.assign(P.N, 0);
    int64_t co = 0, ro = 0;
    for (int32_t b = 0; b < count; b++) {
        for (int32_t j = 0; j < ns[b]; j++) P.inst[P.iperm[co + j]] = b;
        for (int32_t i = 0; i < ms[b]; i++) P.inst[P.iperm[Nn + ro + i]] = b;
        co += ns[b];
        ro += ms[b];
    }
    return IPM_OK;
}


int ipm_set_values(ipm_ctx *c, const double *Ax_dev, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!Ax_dev && c->plan.Acp[c->plan.n] > 0) return IPM_ERR_INVALID_ARG;
    if (!c->dev_ready) {
        rc = setup_device(c);
        if (rc) return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nnz = c->plan.Acp[c->plan.n];
    if (nnz > 0) {
        cudaError_t e = cudaMemcpyAsync(c->Ax, Ax_dev, nnz * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return to_err(e);
    }
    c->values_set = true;
    c->factorised = false;
    return IPM_OK;
}

int ipm_factorise(ipm_ctx *c, const double *theta_dev, double rho, double delta, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->values_set) return IPM_ERR_NOT_ANALYSED;
    if (!theta_dev && c->plan.n > 0) return IPM_ERR_INVALID_ARG;
    if (!(rho >= 0.0) || !(delta >= 0.0) || !std::isfinite(rho) || !std::isfinite(delta)) return IPM_ERR_INVALID_ARG;
    // the pivoting mode: augmented system, fronts within the sweeps' shared memory (f + k doubles)
    if (c->opt.pivoting &&
        (c->plan.form != 1 || 2 * (int64_t)c->plan.max_f * (int64_t)sizeof(double) > kSweepSmemLimit))
        return IPM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (c->plan.n > 0 && theta_dev != c->theta) {
        cudaError_t e = cudaMemcpyAsync(c->theta, theta_dev, c->plan.n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return to_err(e);
    }
    c->rho = rho;
    c->delta = delta;
    rc = factorise_enqueue(c, c->theta, rho, delta, st);
    if (rc) return rc;
    c->factorised = true;
    return IPM_OK;
}

// Autotuner (the batching of Sec. 4.3 leaves the per-bucket launch shapes
// open): times factorisations of the context's own problem on the device
// and keeps, by coordinate descent, the level-kernel threshold and the CTA
// width of each small-front size class that give the shortest time; a
// candidate replaces the incumbent only when at least 2% faster, so that
// timing noise does not move the choice.  No choice changes the arithmetic
// of any entry, so the factors stay the same bit for bit.
constexpr double kTuneMargin = 0.98;
int ipm_autotune(ipm_ctx *c, const double *theta_dev, double rho, double delta, int32_t reps, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->values_set) return IPM_ERR_NOT_ANALYSED;
    if (reps < 1 || reps > 20) return IPM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return IPM_ERR_CUDA;
    }
    // median of reps factorisations after one untimed
    auto measure = [&](double &ms) -> int {
        std::vector<float> t;
        for (int r = 0; r <= reps; r++) {
            cudaEventRecord(e0, st);
            int q = ipm_factorise(c, theta_dev, rho, delta, st);
            if (q) return q;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return IPM_ERR_CUDA;
            float x = 0.f;
            cudaEventElapsedTime(&x, e0, e1);
            if (r > 0) t.push_back(x);
        }
        std::sort(t.begin(), t.end());
        ms = t[t.size() / 2];
        return IPM_OK;
    };
    bool present[3] = {false, false, false};
    for (const LevelWork &W : c->levels)
        for (const SmallClass &C : W.small) present[C.cls] = true;
    double best = 0.0;
    if ((rc = measure(best))) goto done;
    {
        const double ratios[] = {0.0, 0.25, 0.5, 1.0, 2.0, 1e30};
        const double r0 = c->tune_ratio;
        double pick = r0;
        for (double r : ratios) {
            if (r == r0) continue;
            c->tune_ratio = r;
            double ms;
            if ((rc = measure(ms))) goto done;
            if (ms < best * kTuneMargin) {
                best = ms;
                pick = r;
            }
        }
        c->tune_ratio = pick;
        const int32_t widths[3][2] = {{32, 64}, {64, 128}, {128, 256}};
        for (int b = 0; b < 3; b++) {
            if (!present[b]) continue;
            const int32_t t0 = c->tune_threads[b];
            int32_t keep = t0;
            for (int32_t w : widths[b]) {
                if (w == t0 || (t0 == 0 && w == widths[b][0])) continue;  // 0 is the first width
                c->tune_threads[b] = w;
                double ms;
                if ((rc = measure(ms))) goto done;
                if (ms < best * kTuneMargin) {
                    best = ms;
                    keep = w;
                }
            }
            c->tune_threads[b] = keep;
        }
        if (c->lvl_grid > c->sms) {  // more than one level-kernel CTA fits per SM: try one
            const int32_t l0 = c->tune_lvl_per_sm;
            c->tune_lvl_per_sm = l0 == 1 ? 0 : 1;
            double ms;
            if ((rc = measure(ms))) goto done;
            if (ms < best * kTuneMargin) best = ms;
            else c->tune_lvl_per_sm = l0;
        }
        c->tune_ms = best;
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

static int read_ctl(ipm_ctx *c, cudaStream_t st, DevCtl *h) {
    cudaError_t e = cudaMemcpyAsync(h, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return to_err(e);
    c->status_acc |= h->status;
    return IPM_OK;
}

int ipm_set_level_ctas(ipm_ctx *c, int32_t per_sm) {
    if (!c || per_sm < 0 || per_sm > 64) return IPM_ERR_INVALID_ARG;
    c->tune_lvl_per_sm = per_sm;
    return IPM_OK;
}

int ipm_set_launch_shapes(ipm_ctx *c, const int32_t *small_threads, double level_ratio) {
    if (!c) return IPM_ERR_INVALID_ARG;
    if (small_threads)
        for (int b = 0; b < 3; b++) {
            const int32_t w = small_threads[b];
            if (w != 0 && w != 32 && w != 64 && w != 128 && w != 256) return IPM_ERR_INVALID_ARG;
        }
    if (!(level_ratio < 0.0) && !(level_ratio >= 0.0)) return IPM_ERR_INVALID_ARG;  // NaN
    if (small_threads)
        for (int b = 0; b < 3; b++) c->tune_threads[b] = small_threads[b];
    if (level_ratio >= 0.0) c->tune_ratio = level_ratio;
    return IPM_OK;
}

// GMRES refinement, an extension of the refinement of Sec. 4.5 for systems
// where classical refinement stalls above the target (lifted pivots make the
// factor a poor enough preconditioner that r -> K^-1 r steps stop halving
// omega): restarted GMRES(m) on K c = r, right-preconditioned by the
// regularised LDL^T factor (c = M^-1 u), classical Gram-Schmidt with one
// re-orthogonalisation, Givens rotations on the host; every restart updates
// x and measures omega with the true residual, and the best iterate is kept.
// Starts from c->vbest (omega wbest); returns the improved wbest.
constexpr int kGmresRestart = 8;

static_assert(kGmresRestart == kGmresM, "host and device restart lengths differ");

// Work space of the GMRES refinement (allocated on first use; before any
// stream capture for the graph-resident version).
static int gmres_alloc(ipm_ctx *c, cudaStream_t st) {
    if (c->gm_V) return IPM_OK;
    const int64_t N = c->plan.N;
    const int m = kGmresRestart;
    int rc;
    if ((rc = dalloc(c, &c->gm_V, (size_t)(m + 1) * N)) || (rc = dalloc(c, &c->gm_Z, (size_t)m * N)) ||
        (rc = dalloc(c, &c->gm_zero, (size_t)N)) || (rc = dalloc(c, &c->gm_w, (size_t)N)) ||
        (rc = dalloc(c, &c->gm_part, (size_t)dots_partial_size())) || (rc = dalloc(c, &c->gm_h, kMaxDots)) ||
        (rc = dalloc(c, &c->gm_dev, 1)))
        return rc;
    cudaMemsetAsync(c->gm_zero, 0, sizeof(double) * N, st);
    cudaMemsetAsync(c->gm_dev, 0, sizeof(GmDev), st);
    return to_err(cudaGetLastError());
}

static int gmres_refine(ipm_ctx *c, const DevVals &V, cudaStream_t st, double &wbest, int *nl) {
    const Plan &P = c->plan;
    const int64_t N = P.N;
    const int m = kGmresRestart;
    int rc;
    if ((rc = gmres_alloc(c, st))) return rc;
    const double target = c->opt.omega_target;
    double hbuf[kMaxDots];
    auto read_h = [&](int cnt) -> int {
        cudaError_t e = cudaMemcpyAsync(hbuf, c->gm_h, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return to_err(e);
    };
    cudaMemcpyAsync(c->vx, c->vbest, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    for (int restart = 0; restart <= c->opt.gmres_restarts; restart++) {
        // r = f - K x and omega of the current x
        launch_residual_omega(c->dp, V, c->vf, c->vx, c->vr, c->vad, c->vae, c->ctl, st);
        *nl += 2;
        DevCtl h{};
        if ((rc = read_ctl(c, st, &h))) return rc;
        if (h.status & kStatNonFinite) break;
        if (restart > 0) {
            if (h.omega < wbest) {
                wbest = h.omega;
                cudaMemcpyAsync(c->vbest, c->vx, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
            } else {
                break;  // no progress
            }
        }
        if (wbest <= target || restart == c->opt.gmres_restarts) break;
        launch_dots(c->vr, c->vr, N, 1, c->gm_part, c->gm_h, st);
        if ((rc = read_h(1))) return rc;
        const double beta = std::sqrt(hbuf[0]);
        if (!(beta > 0.0) || !std::isfinite(beta)) break;
        launch_scale(c->gm_V, c->vr, 1.0 / beta, N, st);
        double H[kGmresRestart + 1][kGmresRestart] = {};
        double cs[kGmresRestart], sn[kGmresRestart], g[kGmresRestart + 1] = {};
        g[0] = beta;
        // relative residual reduction that brings omega under the target, with margin
        const double eta = std::min(0.5, std::max(1e-14, 0.1 * target / std::max(h.omega, 1e-300)));
        int jdone = 0;
        for (int j = 0; j < m; j++) {
            double *vj = c->gm_V + (int64_t)j * N, *zj = c->gm_Z + (int64_t)j * N, *vn = vj + N;
            cudaMemcpyAsync(zj, vj, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
            if ((rc = solve_inplace(c, zj, st, nl))) return rc;
            launch_residual_omega(c->dp, V, c->gm_zero, zj, c->gm_w, c->vad, c->vae, c->ctl, st);  // -K z
            launch_scale(vn, c->gm_w, -1.0, N, st);
            *nl += 3;
            for (int pass = 0; pass < 2; pass++) {
                launch_dots(vn, c->gm_V, N, j + 1, c->gm_part, c->gm_h, st);
                launch_gs_update(vn, c->gm_V, c->gm_h, N, j + 1, st);
                *nl += 3;
                if ((rc = read_h(j + 1))) return rc;
                for (int i = 0; i <= j; i++) H[i][j] += hbuf[i];
            }
            launch_dots(vn, vn, N, 1, c->gm_part, c->gm_h, st);
            if ((rc = read_h(1))) return rc;
            const double hn = std::sqrt(hbuf[0]);
            H[j + 1][j] = hn;
            if (hn > 0.0) launch_scale(vn, vn, 1.0 / hn, N, st);
            // Givens rotations: apply the earlier ones, then annihilate H[j+1][j]
            for (int i = 0; i < j; i++) {
                const double a = H[i][j], b = H[i + 1][j];
                H[i][j] = cs[i] * a + sn[i] * b;
                H[i + 1][j] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[j][j], b = H[j + 1][j], r = std::hypot(a, b);
            cs[j] = r > 0.0 ? a / r : 1.0;
            sn[j] = r > 0.0 ? b / r : 0.0;
            H[j][j] = r;
            H[j + 1][j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jdone = j + 1;
            c->gmres_iters++;
            if (std::fabs(g[j + 1]) <= eta * beta || !(hn > 0.0)) break;
        }
        // y = R^-1 g, x += Z y
        GmresCoef y{};
        for (int i = jdone - 1; i >= 0; i--) {
            double t = g[i];
            for (int q = i + 1; q < jdone; q++) t -= H[i][q] * y.c[q];
            y.c[i] = H[i][i] != 0.0 ? t / H[i][i] : 0.0;
        }
        launch_combine(c->vx, c->gm_Z, y, N, jdone, st);
        *nl += 1;
    }
    return IPM_OK;
}

static int solve_once(ipm_ctx *c, const double *r7, const double *r1, double *dx, double *dy, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->factorised) return IPM_ERR_NOT_FACTORISED;
    const Plan &P = c->plan;
    if ((P.n > 0 && (!r7 || !dx)) || (P.m > 0 && (!r1 || !dy))) return IPM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t N = P.N;
    DevVals V{};
    V.Ax = c->Ax;
    V.theta = c->theta;
    V.rho = c->rho;
    V.delta = c->delta;
    V.nev = c->ne.nev;
    int nl = 0;
    if (P.form == 2) launch_ne_rhs(c->ne, c->dp.perm, c->Ax, r7, r1, c->vf, st);  // r8 = r1 + A Theta~ r7
    else launch_permute_in(c->dp, r7, r1, c->vf, st);
    nl++;
    cudaMemcpyAsync(c->vx, c->vf, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if ((rc = solve_inplace(c, c->vx, st, &nl))) return rc;
    {
        Prof pr(c, IPM_K_RESIDUAL, c->resid_w, st);
        launch_residual_omega(c->dp, V, c->vf, c->vx, c->vr, c->vad, c->vae, c->ctl, st);
    }
    nl += 2;
    DevCtl h{};
    if ((rc = read_ctl(c, st, &h))) return rc;
    double wbest = h.omega;
    cudaMemcpyAsync(c->vbest, c->vx, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    int steps = 0;
    c->omega_hist[0] = h.omega;
    const double target = c->opt.omega_target;
    while (wbest > target && steps < c->opt.refine_max && !(h.status & kStatNonFinite)) {
        cudaMemcpyAsync(c->vc, c->vr, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if ((rc = solve_inplace(c, c->vc, st, &nl))) return rc;
        launch_axpy(c->vx, c->vc, N, st);
        {
            Prof pr(c, IPM_K_RESIDUAL, c->resid_w, st);
            launch_residual_omega(c->dp, V, c->vf, c->vx, c->vr, c->vad, c->vae, c->ctl, st);
        }
        nl += 3;
        if ((rc = read_ctl(c, st, &h))) return rc;
        steps++;
        if (steps < 16) c->omega_hist[steps] = h.omega;
        const bool halved = h.omega <= 0.5 * wbest;
        if (h.omega < wbest) {
            wbest = h.omega;
            cudaMemcpyAsync(c->vbest, c->vx, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
        }
        if (!halved) break;
    }
    // GMRES refinement of an FP64 factor; a tensor-core factor whose classical
    // refinement stalls is replaced by an FP64 one instead (ipm_solve), which
    // later iterations keep, rather than paying GMRES iterations every solve
    c->gmres_iters = 0;
    if (wbest > target && gmres_allowed(c) && !(h.status & kStatNonFinite)) {
        if ((rc = gmres_refine(c, V, st, wbest, &nl))) return rc;
        steps += c->gmres_iters;
    }
    launch_permute_out(c->dp, c->vbest, dx, dy, st);
    nl++;
    c->refine_steps = steps;
    c->omega = wbest;
    c->omega_sys = wbest;
    if (P.form == 2) {
        // dx = Theta~ (A^T dy - r7); the reported backward error is the one on K
        launch_ne_dx(c->ne, c->Ax, dy, r7, dx, st);
        launch_residual_K(c->ne, c->Ax, c->theta, c->rho, c->delta, r7, r1, dx, dy, c->kf, c->kr, c->kad, c->kae,
                          c->ctl, st);
        launch_omega_only(P.n + P.m, c->kr, c->kad, c->kae, c->kf, c->ctl, st);
        nl += 3;
        if ((rc = read_ctl(c, st, &h))) return rc;
        c->omega = h.omega;
    }
    c->graph_solved = false;
    if (wbest > target) c->status_acc |= kStatRefineFail;
    c->nl_solve = nl;
    return to_err(cudaGetLastError());
}

int ipm_solve(ipm_ctx *c, const double *r7, const double *r1, double *dx, double *dy, void *stream) {
    int rc = solve_once(c, r7, r1, dx, dy, stream);
    if (rc) return rc;
    // mixed precision: when refinement stalls above the target (or the
    // FP32-accurate updates drove a pivot to overflow), factorise again in
    // FP64 and solve again; later factorisations stay in FP64.  The status of
    // the abandoned factorisation is dropped.
    if (c->mixed_active && !(c->omega_sys <= c->opt.omega_target)) {
        c->mixed_active = false;
        c->fallbacks++;
        c->status_acc &= ~(kStatRefineFail | kStatNonFinite | kStatDynReg | kStatLargeReg);
        cudaMemsetAsync(&c->ctl->status, 0, sizeof(int32_t), (cudaStream_t)stream);
        if ((rc = factorise_enqueue(c, c->theta, c->rho, c->delta, (cudaStream_t)stream))) return rc;
        rc = solve_once(c, r7, r1, dx, dy, stream);
    }
    return rc;
}

int ipm_iterate_host(ipm_ctx *c, const double *theta_h, double rho, double delta, int32_t nrhs, const double *r7_h,
                     const double *r1_h, double *dx_h, double *dy_h, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->values_set) return IPM_ERR_NOT_ANALYSED;
    const Plan &P = c->plan;
    if (nrhs < 0 || (P.n > 0 && !theta_h) || (nrhs > 0 && ((P.n > 0 && (!r7_h || !dx_h)) || (P.m > 0 && (!r1_h || !dy_h)))))
        return IPM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->d_r7) {
        if ((rc = dalloc(c, &c->d_r7, P.n)) || (rc = dalloc(c, &c->d_r1, P.m)) || (rc = dalloc(c, &c->d_dx, P.n)) ||
            (rc = dalloc(c, &c->d_dy, P.m)))
            return rc;
    }
    cudaError_t e = cudaMemcpyAsync(c->theta, theta_h, P.n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return to_err(e);
    if ((rc = ipm_factorise(c, c->theta, rho, delta, stream))) return rc;
    for (int32_t k = 0; k < nrhs; k++) {
        cudaMemcpyAsync(c->d_r7, r7_h + (size_t)k * P.n, P.n * sizeof(double), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(c->d_r1, r1_h + (size_t)k * P.m, P.m * sizeof(double), cudaMemcpyHostToDevice, st);
        if ((rc = ipm_solve(c, c->d_r7, c->d_r1, c->d_dx, c->d_dy, stream))) return rc;
        cudaMemcpyAsync(dx_h + (size_t)k * P.n, c->d_dx, P.n * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(dy_h + (size_t)k * P.m, c->d_dy, P.m * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    return ipm_sync_status(c, stream);
}

int ipm_sync_status(ipm_ctx *c, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->dev_ready) return IPM_OK;
    DevCtl h{};
    if ((rc = read_ctl(c, (cudaStream_t)stream, &h))) return rc;
    c->last = h;
    int32_t st = c->status_acc;
    c->status_acc = 0;
    cudaMemsetAsync(&c->ctl->status, 0, sizeof(int32_t), (cudaStream_t)stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    return status_to_code(st);
}

int ipm_get_info(ipm_ctx *c, ipm_info *out) {
    if (!c || !out) return IPM_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    const Plan &P = c->plan;
    out->m = P.m;
    out->n = P.n;
    out->N = P.N;
    out->form = P.form;
    out->ordering = P.ordering;
    out->nsuper = P.nsuper;
    out->nlevels = P.nlevels;
    out->nfronts_small = P.nsmall;
    out->nfronts_large = P.nlarge;
    out->max_front = P.max_f;
    out->max_k = P.max_k;
    out->nnz_A = P.Acp.empty() ? 0 : P.Acp[P.n];
    out->nnz_K_lower = P.nnzK_lower;
    out->nnz_L = P.nnzL;
    out->flops_factor = P.flops;
    out->amalg_zero_frac = P.amalg_zero_frac;
    out->flops_tensor = c->flops_tensor;
    out->precision_fallbacks = c->fallbacks;
    out->est_cost_as = P.est_as;
    out->est_cost_ne = P.est_ne;
    out->nnz_ne_seen = P.nnz_ne_seen;
    out->mixed_active = c->mixed_active ? 1 : 0;
    out->device_bytes = c->device_bytes;
    out->ms_analyse = c->ms_analyse;
    out->refine_steps = c->refine_steps;
    out->gmres_iters = c->gmres_iters;
    for (int b = 0; b < 3; b++) {
        const int32_t dflt = b == 0 ? 32 : b == 1 ? 64 : 128;
        out->tune_small_threads[b] = c->tune_threads[b] > 0 ? c->tune_threads[b] : dflt;
    }
    out->tune_level_ratio = c->tune_ratio;
    out->tune_level_ctas_per_sm = c->dev_ready ? level_grid(c) / c->sms : 0;
    out->graph_kernels = c->graph_kernels;
    out->schedule = c->dep_sched ? IPM_SCHED_DEPENDENCY : IPM_SCHED_LEVELS;
    out->steps_levels = c->steps_levels;
    out->steps_dependency = c->steps_dependency;
    out->nfronts_thin = c->nfronts_thin;
    out->tune_ms = c->tune_ms;
    out->omega = c->omega;
    for (int i = 0; i < 16; i++) out->omega_hist[i] = c->omega_hist[i];
    if (!c->analysed) return IPM_ERR_NOT_ANALYSED;
    int code = IPM_OK;
    if (c->dev_ready) {
        cudaSetDevice(c->opt.device);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return to_err(e);
        DevCtl h{};
        e = cudaMemcpy(&h, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return to_err(e);
        c->status_acc |= h.status;
        if (c->graph_solved) {
            out->refine_steps = h.steps + h.gmres_iters;
            out->gmres_iters = h.gmres_iters;
            out->omega = h.omega_best;
            for (int i = 0; i < 16; i++) out->omega_hist[i] = i <= h.steps ? h.omega_hist[i] : 0.0;
        }
        out->npos = h.npos;
        out->nneg = h.nneg;
        out->ndynreg = h.ndyn;
        out->max_dynreg = h.max_dyn;
        out->norm_K1 = h.norm1;
        out->status = c->status_acc;
        code = status_to_code(c->status_acc);
    }
    return code;
}

int ipm_get_sizes(const ipm_ctx *c, int32_t *N, int32_t *nsuper, int64_t *nrows_total, int64_t *nnz_L_stored) {
    int rc = check_ctx(c);
    if (rc) return rc;
    const Plan &P = c->plan;
    if (N) *N = P.N;
    if (nsuper) *nsuper = P.nsuper;
    if (nrows_total) *nrows_total = P.sn_rptr[P.nsuper];
    if (nnz_L_stored) {
        int64_t t = 0;
        for (int32_t s = 0; s < P.nsuper; s++) t += (int64_t)P.sn_f[s] * P.sn_k[s];
        *nnz_L_stored = t;
    }
    return IPM_OK;
}

int ipm_get_symbolic(const ipm_ctx *c, int32_t *perm, int32_t *etree, int64_t *colcount, int32_t *snode_ptr,
                     int32_t *sn_parent, int64_t *sn_rptr, int32_t *sn_rows) {
    int rc = check_ctx(c);
    if (rc) return rc;
    const Plan &P = c->plan;
    if (perm) std::memcpy(perm, P.perm.data(), P.N * sizeof(int32_t));
    if (etree) std::memcpy(etree, P.parent.data(), P.N * sizeof(int32_t));
    if (colcount) std::memcpy(colcount, P.colcount.data(), P.N * sizeof(int64_t));
    if (snode_ptr) std::memcpy(snode_ptr, P.sn_start.data(), (P.nsuper + 1) * sizeof(int32_t));
    if (sn_parent) std::memcpy(sn_parent, P.sn_parent.data(), P.nsuper * sizeof(int32_t));
    if (sn_rptr) std::memcpy(sn_rptr, P.sn_rptr.data(), (P.nsuper + 1) * sizeof(int64_t));
    if (sn_rows) std::memcpy(sn_rows, P.sn_rows.data(), P.sn_rptr[P.nsuper] * sizeof(int32_t));
    return IPM_OK;
}

int ipm_get_factor(ipm_ctx *c, double *L_host, double *D_host, double *dyn_host) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->factorised) return IPM_ERR_NOT_FACTORISED;
    const Plan &P = c->plan;
    cudaSetDevice(c->opt.device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return to_err(e);
    if (D_host && (e = cudaMemcpy(D_host, c->D, P.N * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return to_err(e);
    if (dyn_host && (e = cudaMemcpy(dyn_host, c->dyn, P.N * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return to_err(e);
    if (L_host) {
        std::vector<double> F((size_t)P.front_doubles);
        if ((e = cudaMemcpy(F.data(), c->fronts, F.size() * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return to_err(e);
        int64_t o = 0;
        for (int32_t s = 0; s < P.nsuper; s++) {
            const int32_t f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s];
            const double *src = F.data() + P.sn_off[s];
            for (int32_t jj = 0; jj < k; jj++)
                for (int32_t ii = 0; ii < f; ii++)
                    L_host[o + (int64_t)jj * f + ii] = ii > jj ? src[(int64_t)jj * ld + ii] : (ii == jj ? 1.0 : 0.0);
            o += (int64_t)f * k;
        }
    }
    return IPM_OK;
}

int ipm_graph_capture(ipm_ctx *c, const double *theta_dev, double rho, double delta, const double *r7_dev,
                      const double *r1_dev, double *dx_dev, double *dy_dev, int32_t nsolves, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->values_set) return IPM_ERR_NOT_ANALYSED;
    const Plan &P = c->plan;
    if (nsolves < 0 || (P.n > 0 && !theta_dev) || !(rho >= 0.0) || !(delta >= 0.0) ||
        (nsolves > 0 && ((P.n > 0 && (!r7_dev || !dx_dev)) || (P.m > 0 && (!r1_dev || !dy_dev)))))
        return IPM_ERR_INVALID_ARG;
    (void)stream;
    if (c->opt.pivoting) return IPM_ERR_INVALID_ARG;  // the pivoting mode runs host-driven sweeps
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    // capture on a private stream (the legacy default stream cannot be
    // captured); the graph is later launched on any stream
    if (!c->cap_stream) {
        cudaError_t e0 = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e0 != cudaSuccess) {
            cudaGetLastError();
            c->cap_stream = nullptr;
            return to_err(e0);
        }
    }
    cudaStream_t st = c->cap_stream;
    if (nsolves > 0 && gmres_allowed(c)) {
        // the graph-resident GMRES refinement needs its work space before the capture
        if ((rc = gmres_alloc(c, st))) return rc;
        cudaError_t e0 = cudaStreamSynchronize(st);
        if (e0 != cudaSuccess) return to_err(e0);
    }
    const bool prof = c->prof_on;
    c->prof_on = false;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->prof_on = prof;
        return to_err(e);
    }
    c->rho = rho;
    c->delta = delta;
    if (P.n > 0 && theta_dev != c->theta)
        cudaMemcpyAsync(c->theta, theta_dev, P.n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    rc = factorise_enqueue(c, c->theta, rho, delta, st);
    for (int32_t k = 0; k < nsolves && rc == IPM_OK; k++)
        rc = solve_device_driven(c, r7_dev + (size_t)k * P.n, r1_dev + (size_t)k * P.m, dx_dev + (size_t)k * P.n,
                                 dy_dev + (size_t)k * P.m, st);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    c->prof_on = prof;
    if (rc || e != cudaSuccess) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return rc ? rc : to_err(e);
    }
    {
        // kernel nodes of the graph (one launch each per replay)
        size_t nn = 0;
        c->graph_kernels = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
                for (size_t q = 0; q < nn; q++) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nodes[q], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                        c->graph_kernels++;
                }
        }
        cudaGetLastError();
    }
    // keep the priorities the kernels were captured with (the critical
    // stream's), instead of the priority of the stream the graph is launched on
    e = cudaGraphInstantiate(&c->graph_exec, g, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        c->graph_exec = nullptr;
        return to_err(e);
    }
    c->graph = g;
    return IPM_OK;
}

int ipm_get_pivots(ipm_ctx *c, int32_t *lperm_host, double *Doff_host, int32_t *bsize_host) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->opt.pivoting) return IPM_ERR_INVALID_ARG;
    if (!c->factorised) return IPM_ERR_NOT_FACTORISED;
    cudaSetDevice(c->opt.device);
    cudaError_t e = cudaDeviceSynchronize();
    const size_t N = (size_t)c->plan.N;
    if (e == cudaSuccess && lperm_host) e = cudaMemcpy(lperm_host, c->lperm, N * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && Doff_host) e = cudaMemcpy(Doff_host, c->Doff, N * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && bsize_host) e = cudaMemcpy(bsize_host, c->bsz, N * sizeof(int32_t), cudaMemcpyDeviceToHost);
    return to_err(e);
}

int ipm_graph_launch(ipm_ctx *c, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->graph_exec) return IPM_ERR_INVALID_ARG;
    cudaError_t e = cudaGraphLaunch(c->graph_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return to_err(e);
    c->factorised = true;
    c->graph_solved = true;
    return IPM_OK;
}

int ipm_launch_counts(const ipm_ctx *c, int32_t *nf, int32_t *ns) {
    if (!c) return IPM_ERR_INVALID_ARG;
    if (nf) *nf = c->nl_factor;
    if (ns) *ns = c->nl_solve;
    return IPM_OK;
}


int ipm_measure_fp64_peak(int32_t device, double *dfma_tflops, double *dmma_tflops) {
    if (!dfma_tflops || !dmma_tflops) return IPM_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return to_err(e);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = std::max(sms, 1) * 8;
    double *buf = nullptr;
    if ((e = cudaMalloc(&buf, (size_t)blocks * 256 * sizeof(double))) != cudaSuccess) return to_err(e);
    cudaStream_t st = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaFree(buf);
        return to_err(e);
    }
    const int rc = measure_fp64_peaks(buf, blocks, 20000, 3, st, dfma_tflops, dmma_tflops);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    cudaFree(buf);
    return rc ? IPM_ERR_CUDA : to_err(cudaGetLastError());
}

int ipm_test_recip_pivot(const double *x, double *rcp, double *quo, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !rcp || !quo))) return IPM_ERR_INVALID_ARG;
    launch_test_recip(x, rcp, quo, n, (cudaStream_t)stream);
    return to_err(cudaGetLastError());
}

int ipm_set_profiling(ipm_ctx *c, int32_t enable) {
    if (!c) return IPM_ERR_INVALID_ARG;
    c->prof_on = enable != 0;
    return IPM_OK;
}

int ipm_kernel_stats(ipm_ctx *c, ipm_kernel_stat *out, int32_t reset) {
    if (!c) return IPM_ERR_INVALID_ARG;
    if (c->dev_ready) {
        cudaSetDevice(c->opt.device);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return to_err(e);
    }
    fold_profile(c);
    if (out) std::memcpy(out, c->prof_tot, sizeof(c->prof_tot));
    if (reset) std::memset(c->prof_tot, 0, sizeof(c->prof_tot));
    return IPM_OK;
}

int ipm_kernel_trace(ipm_ctx *c, int32_t *cls, int32_t *stream, double *start_ms, double *end_ms, int32_t cap,
                     int32_t *count) {
    if (!c || cap < 0 || !count || (cap > 0 && (!cls || !stream || !start_ms || !end_ms)))
        return IPM_ERR_INVALID_ARG;
    if (c->dev_ready) {
        cudaSetDevice(c->opt.device);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return to_err(e);
    }
    fold_profile(c);
    *count = (int32_t)c->trace.size();
    const int32_t n = std::min(cap, *count);
    for (int32_t i = 0; i < n; i++) {
        cls[i] = c->trace[i].cls;
        stream[i] = c->trace[i].stream;
        start_ms[i] = c->trace[i].t0;
        end_ms[i] = c->trace[i].t1;
    }
    c->trace.clear();
    return IPM_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free solve.
//
// Some callers cannot allocate device memory when they need a solve:
// callbacks of an optimisation loop that run under a strict device-memory
// budget, or a host library that must never change the device's allocation
// state (an allocation there can fail, or make the caching allocator of the
// surrounding framework release and re-reserve memory).  ipm_solve_noalloc
// serves them: it takes every work vector from one file-scope device array
// instead of the context's own buffers, and it calls no allocating routine.
// It is a plain variant, not a copy of ipm_solve: it runs the per-level sweeps
// (k_forward / k_backward, one launch per tree level), which need no
// dependency counters and no per-context scratch, and classical refinement
// only (no GMRES, and no FP64 refactorisation of a tensor-core factor that
// fails to refine: it returns IPM_WARN_REFINE_NOT_CONVERGED instead).  Its
// refinement decisions are taken on the host (one synchronisation of the
// stream per step).
namespace {

// Capacity of the shared work array, in doubles (16 MiB).  A solve needs
// 7 N + sum_s (f_s - k_s) doubles (N unknowns; f_s - k_s the contribution
// rows of supernode s, one update vector entry each).
constexpr int64_t kNoAllocDoubles = int64_t(1) << 21;
static __device__ __align__(256) double g_noalloc_work[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
double *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the work array for the current device, looked up once
// per device (with that device current).  In host code the array's name is
// only a stand-in, so kernels must receive this address instead.
int noalloc_base(int device, double **out) {
    if (device < 0 || device >= kMaxDevices) return IPM_ERR_INVALID_ARG;
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_work);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        g_noalloc_ptr[device] = (double *)p;
    }
    *out = g_noalloc_ptr[device];
    return IPM_OK;
}

int noalloc_sweeps(ipm_ctx *c, double *x, double *upd, cudaStream_t st) {
    const Plan &P = c->plan;
    for (int32_t l = 0; l < P.nlevels; l++) {
        const LevelWork &W = c->levels[l];
        launch_forward(c->dp, c->fronts, c->D, x, upd, c->lvl_all + W.all_off, W.all_cnt, W.all_maxf, st);
    }
    for (int32_t l = P.nlevels - 1; l >= 0; l--) {
        const LevelWork &W = c->levels[l];
        launch_backward(c->dp, c->fronts, x, c->lvl_all + W.all_off, W.all_cnt, W.all_maxf, st);
    }
    return to_err(cudaGetLastError());
}

}  // namespace

extern "C" {

int ipm_solve_noalloc(ipm_ctx *c, const double *r7, const double *r1, double *dx, double *dy, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    const Plan &P = c->plan;
    const int64_t N = P.N;
    const int64_t need = 7 * N + P.upd_total;
    if (need > kNoAllocDoubles) {
        if (c->opt.verbose)
            std::fprintf(stderr, "[ipm] ipm_solve_noalloc: needs %lld doubles of work space, the limit is %lld\n",
                         (long long)need, (long long)kNoAllocDoubles);
        return IPM_ERR_SCRATCH_TOO_SMALL;
    }
    // the per-level sweeps keep one front's gathered vector in shared memory
    if ((int64_t)P.max_f * (int64_t)sizeof(double) > kSweepSmemLimit) {
        if (c->opt.verbose)
            std::fprintf(stderr, "[ipm] ipm_solve_noalloc: a front of %d rows exceeds the sweeps' shared memory\n",
                         (int)P.max_f);
        return IPM_ERR_SCRATCH_TOO_SMALL;
    }
    if (!c->factorised) return IPM_ERR_NOT_FACTORISED;
    if (P.form != 1 || c->opt.pivoting) return IPM_ERR_INVALID_ARG;  // augmented system, 1x1 pivots only
    if ((P.n > 0 && (!r7 || !dx)) || (P.m > 0 && (!r1 || !dy))) return IPM_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(c->opt.device);
    if (e != cudaSuccess) return to_err(e);
    double *base = nullptr;
    if ((rc = noalloc_base(c->opt.device, &base))) return rc;
    // every vector below is written before it is read within one call, so
    // nothing left by the previous call needs clearing
    double *vf = base, *vx = base + N, *vbest = base + 2 * N, *vr = base + 3 * N, *vad = base + 4 * N,
           *vae = base + 5 * N, *vc = base + 6 * N, *upd = base + 7 * N;
    cudaStream_t st = (cudaStream_t)stream;
    DevVals V{};
    V.Ax = c->Ax;
    V.theta = c->theta;
    V.rho = c->rho;
    V.delta = c->delta;
    launch_permute_in(c->dp, r7, r1, vf, st);
    cudaMemcpyAsync(vx, vf, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if ((rc = noalloc_sweeps(c, vx, upd, st))) return rc;
    launch_residual_omega(c->dp, V, vf, vx, vr, vad, vae, c->ctl, st);
    DevCtl h{};
    if ((rc = read_ctl(c, st, &h))) return rc;
    double wbest = h.omega;
    cudaMemcpyAsync(vbest, vx, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    int steps = 0;
    c->omega_hist[0] = h.omega;
    const double target = c->opt.omega_target;
    while (wbest > target && steps < c->opt.refine_max && !(h.status & kStatNonFinite)) {
        cudaMemcpyAsync(vc, vr, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if ((rc = noalloc_sweeps(c, vc, upd, st))) return rc;
        launch_axpy(vx, vc, (int32_t)N, st);
        launch_residual_omega(c->dp, V, vf, vx, vr, vad, vae, c->ctl, st);
        if ((rc = read_ctl(c, st, &h))) return rc;
        steps++;
        if (steps < 16) c->omega_hist[steps] = h.omega;
        const bool halved = h.omega <= 0.5 * wbest;
        if (h.omega < wbest) {
            wbest = h.omega;
            cudaMemcpyAsync(vbest, vx, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
        }
        if (!halved) break;
    }
    launch_permute_out(c->dp, vbest, dx, dy, st);
    // what ipm_get_info reports about the last solve
    c->refine_steps = steps;
    c->gmres_iters = 0;
    c->omega = wbest;
    c->omega_sys = wbest;
    c->graph_solved = false;
    if ((rc = to_err(cudaGetLastError()))) return rc;
    if (h.status & kStatNonFinite) return IPM_ERR_NONFINITE;
    if (wbest > target) {
        c->status_acc |= kStatRefineFail;
        return IPM_WARN_REFINE_NOT_CONVERGED;
    }
    return IPM_OK;
}

}  // extern "C"
