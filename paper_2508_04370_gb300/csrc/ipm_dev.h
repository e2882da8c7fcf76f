// Device-side view of the analysis plan and kernel entry points of the
// multifrontal factorise/solve (Zanetti & Gondzio, arXiv 2508.04370, Sec. 4).
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

namespace ipm {

// Status bits written by kernels (never traps): OR-ed into DevCtl::status.
enum : int32_t {
    kStatNonFinite = 1,    // NaN / Inf in Theta, a pivot or a residual
    kStatDynReg = 2,       // a pivot was lifted
    kStatLargeReg = 4,     // a lift exceeded opt.large_reg
    kStatTimeout = 8,      // a bounded wait expired
    kStatRefineFail = 16,  // refinement did not reach the target
    kStatWaitCopy = 32,    // with kStatTimeout: a tensor-core kernel's wait for its bulk copies gave up
    kStatWaitMma = 64,     // with kStatTimeout: a wait for the completion of MMAs gave up
};

// Dynamic shared memory the per-level solve sweeps may use (one front's
// gathered vector, f doubles): fronts above 25,600 rows do not fit.
constexpr int64_t kSweepSmemLimit = 200 * 1024;

// Kernel attributes such as the dynamic shared-memory limit belong to one
// device: true the first time it is asked for the current device, so the
// attribute is set once per device and kernel (mask: one bit per device).
inline bool first_on_device(uint64_t &mask) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) {
        cudaGetLastError();
        return true;
    }
    const uint64_t bit = (uint64_t)1 << d;
    if (mask & bit) return false;
    mask |= bit;
    return true;
}

// Small control block in device memory.
struct DevCtl {
    int32_t status;
    int32_t ndyn;
    int32_t npos, nneg;
    double max_dyn;
    double norm1;          // ||K||_1 (or ||M||_1) of the current factorisation
    double b1;             // eps_piv * norm1
    // refinement
    double omega;          // backward error of the current iterate
    double omega_best;
    double dinf;           // ||d||_inf of the current iterate (as ordered bits >= 0)
    int32_t done;          // refinement finished
    int32_t steps;
    int32_t improved;      // the last step improved omega_best
    double omega_hist[16];
    int32_t gmres_iters;   // GMRES iterations of a graph-resident refinement
};

// Read-only plan arrays on the device (all indices in factorisation order).
struct DevPlan {
    int32_t N, n, m, nsuper, form;
    const int32_t *sn_c0, *sn_k, *sn_f, *sn_ld;
    const int64_t *sn_off;        // slab offset (doubles)
    const int64_t *sn_rptr;       // row list offset
    const int32_t *sn_rows;       // global row indices
    const int32_t *child_ptr, *child_list;
    const int32_t *sn_parent;     // parent supernode or -1
    const int64_t *map_off;
    const int32_t *relmap;
    const int64_t *orig_ptr;
    const int32_t *orig_dst;
    const int64_t *orig_src;
    const int8_t *sign;           // expected pivot sign per row (-1 / +1)
    const int32_t *perm;          // perm[new] = old
    const int64_t *upd_off;       // solve: contribution-vector offsets
    // regularised matrix in factorisation order, full symmetric CSR (for
    // residuals): value source per entry (>= 0: A index, -1-j: primal
    // diagonal of old column j, kDualDiag: delta)
    const int64_t *kp;
    const int32_t *kj;
    const int64_t *ksrc;
    // columns of K with more than kLongColumn stored entries (dense rows of A):
    // summed by a whole CTA each in the norm
    const int32_t *long_cols;
    int32_t nlong;
    // batches of independent problems: instance of each unknown (factorisation
    // order) and, per instance, ||K_b||_1 and eps_piv ||K_b||_1; null otherwise
    int32_t batch_count;
    const int32_t *inst;
    double *inst_norm1, *inst_b1;
};

// eps_piv ||K||_1 of the problem that owns column c (Sec. 4.5); the norm is
// per instance when independent problems are factorised together.
__device__ __forceinline__ double pivot_floor(const DevPlan &P, const DevCtl *ctl, int c) {
    return P.inst ? P.inst_b1[P.inst[c]] : ctl->b1;
}

constexpr int64_t kDualDiag = INT64_MIN;

// Numeric values for one factorisation.
struct DevVals {
    const double *Ax;      // A values (CSC order of the pattern)
    const double *theta;   // n
    const double *nev;     // normal equations: lower entries of M (or null)
    double rho, delta;
    double large_reg;
};

// Rows of a panel handled by one CTA of the panel kernel (one thread per row).
constexpr int kPanelRows = 128;
// Output tile of the FP64 trailing-update kernel.
constexpr int kUpdTile = 32;
// Lookahead (next panel) columns of the trailing update are cut into strips
// of kUpdTile rows x kStripCols columns, one output per thread.
constexpr int kStripCols = 4;
// Output tile of the tensor-core trailing update (M = N).
constexpr int kTcTile = 128;

// Device data of the normal-equations path.
struct NeView {
    int32_t n, m;
    int64_t nnz;                 // lower entries of M
    const int64_t *tptr;         // contributor pairs per entry
    const int32_t *ta, *tb, *tj;
    double *tt;                  // Theta~ (n)
    double *nev;                 // formed entries of M (nnz)
    const int64_t *Arp;          // A by rows: pointer, column, position in Ax
    const int32_t *Aci, *Apos;
    const int64_t *Acp;          // A by columns
    const int32_t *Ari;
};

// Dependency-driven solve schedule, built once per pattern.  A supernode
// with k > 32 or a large rectangular part L21 is split into one item per
// 32-column block of L11 and row-chunk items (kRectRows rows of L21 each),
// which run on other SMs.
struct SolveNode {
    int64_t off;    // slab offset (doubles)
    int64_t upd;    // offset of its contribution vector
    int64_t rptr;   // first entry in sn_rows and gat_rp
    int64_t inv;    // inverses of its diagonal blocks in SolveSched::Linv, -1: none (layout: block_slot)
    int32_t f, k, ld, c0;
    int32_t parent, nchild, nrect, nblk;  // nblk: items of L11 (32-column blocks; 1 when unsplit)
};
struct SolveItem {
    int32_t s, r;  // r < 0: block -1-r of L11; else row chunk r of L21
};
struct SolveSched {
    const SolveNode *node;
    const int32_t *sn_rows;
    const int64_t *gat_rp;   // per front row: range in gat_src
    const int64_t *gat_src;  // contribution-vector positions summed into the row, children ascending
    const SolveItem *fwd, *bwd;
    int32_t nfwd, nbwd, nsuper;
    long long spin_limit;    // polls before a dependency wait gives up (kStatTimeout)
    int32_t *sync;           // ticket + 2 x nsuper counters (forward: children done, items done;
                             // backward: done flag, blocks done)
    double *yv;              // the values split supernodes' blocks pass along their chain (y forward,
                             // z backward), reset to an unset pattern before each sweep
    int32_t nyv;
    const int32_t *fwd_leaf, *bwd_leaf;  // leaf groups: 8 childless single-item supernodes with f <= 32
                                         // per ticket (-1 pads), one warp each
    const double *Linv;                  // inverse unit-lower diagonal blocks, column-major 32 x 32
};
// One diagonal block to invert after a factorisation: block b of supernode s
// into Linv + dst.
struct InvItem {
    int32_t s, b;
    int64_t dst;
};
constexpr int32_t kLeafGroup = INT32_MIN;  // SolveItem.r of a leaf group (s = group index)
constexpr int kRectRows = 32;
constexpr int64_t kRectSplit = 8192;  // split when k (f - k) reaches this

// Work item of the large-front path.
struct PanelItem {
    int32_t s;       // supernode
    int32_t r0, r1;  // row range (local) handled by this block
    int32_t p0;      // first column of the item's panel (diagonal blocks, triangular solves)
};
// Precomputed ranges of an assembly item (front columns [r0, r1) of a large
// front, rows [r_lo, r_hi)): its original entries [o0, o1) (those of the
// columns; the item keeps the ones in its rows) and, at acr[4 * cr ...], per
// child (children ascending) the range [a, b) of contribution-block columns
// and the range [ilo, ihi) of contribution-block rows that land in the item.
struct AsmItem {
    int64_t o0, o1, cr;
    int32_t r_lo, r_hi;  // front rows [r_lo, r_hi) handled (rows below the columns' first: the upper part is never read)
};
struct TileItem {
    int32_t s;
    int32_t i0, j0;  // first local row / column of a kUpdTile x kUpdTile output tile
                     // (kUpdTile x kStripCols for the lookahead strips)
    int32_t p0;      // first column of the panel whose update the tile applies
};

// Sliced tensor-core update (FP64-accurate Schur complement on bf16 tensor
// cores).  Panels of a large front are taken in pairs: after the first panel
// of a pair only the second panel's columns are updated; after the second,
// every trailing row r >= p1 of both panel operands over both panels' 64
// columns, L(r, q) and L(r, q) d_q, is scaled by one power of two per row
// and split into kSlices balanced 7-bit digits, and the whole trailing part
// receives the two panels' update at once (K = 64).  One slice block holds
// 128 rows: one chunk of digit images per 32 columns.
constexpr int kSlices = 8;                           // 8 x 7 = 56 bits per operand
constexpr int kSliceRows = 128;                      // rows per slice block (the MMA's M)
constexpr int kSliceCols = 32;                       // output columns per tile (the MMA's N), columns per chunk
constexpr int kSliceChunks = 2;                      // chunks of 32 columns per slice block (K <= 64)
constexpr int64_t kSlicePairBytes = 128 * 128;       // two slices of 128 rows x 32 bf16, one swizzled image
constexpr int64_t kSliceOperandBytes = 4 * kSlicePairBytes;
constexpr int64_t kSliceChunkBytes = 2 * kSliceOperandBytes;  // operand A (L), then operand B (L d)
constexpr int64_t kSliceBlockBytes = kSliceChunks * kSliceChunkBytes;

struct SlicedTile {
    int32_t s;
    int32_t i0, j0;     // output rows i0 .. i0+127, columns j0 .. j0+31 (lower part only)
    int32_t blk_a;      // slice block of rows i0 ..
    int32_t blk_b;      // slice block holding columns j0 .. j0+31 as rows,
    int32_t roff_b;     // at row offset roff_b (a multiple of 32) inside it
    int32_t kc;         // chunks of the product: 1 (one panel, K <= 32) or 2 (a pair of panels, K <= 64)
};

// One item of the persistent level kernel (large fronts of one tree level):
// it waits until counter wait0 >= need0 and counter wait1 >= need1 (-1: no
// wait), runs, then adds `add` to counter sig.  Counters are per level,
// zeroed before the launch; the host orders the items so that every wait
// refers to items with smaller positions.
enum : int32_t { kItemAssemble = 0, kItemDiag = 1, kItemTrsm = 2, kItemStrip = 3, kItemTile = 4 };
struct FactorItem {
    int32_t kind;
    int32_t s, t;  // front, pivot block (panel) index
    int32_t a, b;  // assemble: columns [a, b); trsm: rows [a, b); strip / tile: first row, first column
    int32_t aux;   // assemble: AsmItem index; diag / trsm: panel workspace slot
    int32_t wait0, need0, wait1, need1;
    int32_t sig, add;
};

// ---------------------------------------------------------------- launches
// factorisation (kernels_factor.cu)
void launch_norm1(const DevPlan &P, const DevVals &V, DevCtl *ctl, double eps_piv, cudaStream_t st);
void launch_small_fronts(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Dinv, double *dyn,
                         DevCtl *ctl, const int32_t *list, int32_t count, int32_t nb, int32_t maxf, int32_t threads,
                         cudaStream_t st);
void launch_large_assemble(const DevPlan &P, const DevVals &V, double *fronts, const PanelItem *items,
                           const AsmItem *ainfo, const int32_t *acr, int32_t count, cudaStream_t st);
// panel step 1 (diagonal block of the panel [item.p0, item.p0 + nb), one item
// per front; item.r1 = workspace slot)
void launch_panel_diag(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Dinv, double *dyn,
                       DevCtl *ctl, const PanelItem *items, int32_t count, int32_t nb, double *pws, cudaStream_t st);
// panel step 2 (rows below, kTrsmRowsHost rows per item; slots[i] = workspace slot of item i)
// sbase[i] >= 0 (with sws non-null): item i also writes the digit slices of
// its rows into the sliced update's work space (slice blocks from
// sbase[i] >> 1; bit 0 set: the second panel of a pair, two chunks)
void launch_panel_trsm(const DevPlan &P, double *fronts, const PanelItem *items, const int32_t *slots, int32_t count,
                       int32_t nb, const double *pws, cudaStream_t st, const int32_t *sbase = nullptr,
                       uint8_t *sws = nullptr, int32_t *sexp = nullptr, const double *D = nullptr,
                       DevCtl *ctl = nullptr);
constexpr int kTrsmRowsHost = 8;       // rows of a triangular-solve chunk of the level kernel
constexpr int kTrsmItemRowsHost = 32;  // rows of a triangular-solve item of the one-launch-per-step kernel
constexpr int kPanelWsHost = 32 * 33 + 32;
void launch_large_update_strip(const DevPlan &P, double *fronts, const double *D, const TileItem *items,
                               int32_t count, int32_t w, cudaStream_t st);
constexpr int64_t kLongColumn = 4096;
// thin fronts (k <= nb, f <= kThinMaxF), one CTA per front: list[i] the front,
// first_asm[i] its first assembly item (one per 32 columns, rows from the
// block's first column), slots[i] its panel workspace slot
constexpr int kThinMaxF = 512;
void launch_thin_fronts(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Dinv, double *dyn,
                        DevCtl *ctl, const int32_t *list, const int32_t *first_asm, const int32_t *slots,
                        const AsmItem *ainfo, const int32_t *acr, double *pws, int32_t count, int32_t nb,
                        cudaStream_t st);
void launch_large_level(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Dinv, double *dyn,
                        DevCtl *ctl, const FactorItem *items, int32_t count, int32_t *sync, int32_t ncounters,
                        const AsmItem *ainfo, const int32_t *acr, double *pws, int32_t nb, int32_t grid,
                        long long spin_limit, cudaStream_t st);
const void *large_level_kernel();
void launch_large_update(const DevPlan &P, double *fronts, const double *D, const TileItem *items, int32_t count,
                         int32_t w, cudaStream_t st);
void launch_large_update_tc(const DevPlan &P, double *fronts, const double *D, const TileItem *items, int32_t count,
                            int32_t w, DevCtl *ctl, cudaStream_t st);
void launch_update_sliced(const DevPlan &P, double *fronts, const SlicedTile *items, int32_t count,
                          const uint8_t *ws, const int32_t *ws_exp, DevCtl *ctl, cudaStream_t st);
int measure_fp64_peaks(double *out, int blocks, int iters, int reps, cudaStream_t st, double *dfma_tflops,
                       double *dmma_tflops);
void launch_front_bk(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Doff, int32_t *bsz,
                     int32_t *lperm, double *dyn, DevCtl *ctl, const int32_t *list, int32_t count, int32_t nb,
                     cudaStream_t st);
void launch_factor_stats_bk(const double *D, const double *Doff, const int32_t *bsz, const double *dyn, int N,
                            double large_reg, DevCtl *ctl, cudaStream_t st);
void launch_forward_bk(const DevPlan &P, const double *fronts, const double *D, const double *Doff,
                       const int32_t *bsz, const int32_t *lperm, double *x, double *upd, const int32_t *list,
                       int32_t count, int32_t maxf, cudaStream_t st);
void launch_backward_bk(const DevPlan &P, const double *fronts, const int32_t *lperm, double *x,
                        const int32_t *list, int32_t count, int32_t maxf, cudaStream_t st);
void launch_test_recip(const double *x, double *rcp, double *quo, int64_t n, cudaStream_t st);
void launch_factor_stats(const double *D, const double *dyn, int N, double large_reg, DevCtl *ctl, cudaStream_t st);
// solves and refinement (kernels_solve.cu)
void launch_forward(const DevPlan &P, const double *fronts, const double *D, double *x, double *upd,
                    const int32_t *list, int32_t count, int32_t maxf, cudaStream_t st);
void launch_backward(const DevPlan &P, const double *fronts, double *x, const int32_t *list, int32_t count,
                     int32_t maxf, cudaStream_t st);
void launch_diag_inverse(const SolveSched &S, const double *fronts, double *Linv, const InvItem *items,
                         int32_t count, const InvItem *pairs, int32_t npairs, cudaStream_t st);
void launch_forward_persistent(const SolveSched &S, const double *fronts, const double *Dinv, double *x, double *upd,
                               int32_t maxf, int32_t grid, DevCtl *ctl, cudaStream_t st,
                               const int32_t *skip = nullptr);
void launch_backward_persistent(const SolveSched &S, const double *fronts, double *x, int32_t maxf, int32_t grid,
                                DevCtl *ctl, cudaStream_t st, const int32_t *skip = nullptr);
// GMRES refinement vectors (kernels_krylov.cu)
constexpr int kMaxDots = 16;  // vectors per dot-product launch (restart length + 1 at most)
constexpr int kGmresM = 8;    // GMRES restart length

// Device-side state of the GMRES refinement inside a captured graph: the
// Hessenberg matrix and its Givens rotations, and the flags the kernels of the
// section test at entry.
struct GmDev {
    double H[(kGmresM + 1) * kGmresM];  // H(i, j) at i * kGmresM + j
    double cs[kGmresM], sn[kGmresM], g[kGmresM + 1], y[kGmresM];
    double h[kMaxDots];                 // output of the dot products
    double beta, inv, eta, wbest;
    int32_t stop;        // GMRES finished: every kernel of the section returns at entry
    int32_t skip_inner;  // stop, or the current cycle has converged
    int32_t improved;    // the last cycle improved the best iterate
    int32_t jdone, iters;
};
struct GmresCoef {
    double c[kMaxDots];
};
void launch_dots(const double *w, const double *V, int64_t N, int32_t cnt, double *part, double *out,
                 cudaStream_t st, const int32_t *skip = nullptr);
// graph-resident GMRES (control kernels and device-parameter vector kernels)
void launch_gm_begin(DevCtl *ctl, GmDev *gm, double target, unsigned long long cond_handle, cudaStream_t st);
void launch_gm_cycle(DevCtl *ctl, GmDev *gm, double target, int32_t cycle, int32_t last, cudaStream_t st);
void launch_gm_init(DevCtl *ctl, GmDev *gm, double target, cudaStream_t st);
void launch_gm_hacc(GmDev *gm, int32_t j, cudaStream_t st);
void launch_gm_arnoldi(GmDev *gm, int32_t j, cudaStream_t st);
void launch_gm_ls(GmDev *gm, cudaStream_t st);
void launch_gm_end(DevCtl *ctl, GmDev *gm, cudaStream_t st);
void launch_gs_update_dev(double *w, const double *V, const GmDev *gm, int64_t N, int32_t cnt, cudaStream_t st);
void launch_scale_dev(double *dst, const double *src, const GmDev *gm, double factor, int64_t N,
                      const int32_t *skip, cudaStream_t st);
void launch_combine_dev(double *x, const double *Z, const GmDev *gm, int64_t N, cudaStream_t st);
void launch_gs_update(double *w, const double *V, const double *h, int64_t N, int32_t cnt, cudaStream_t st);
void launch_scale(double *dst, const double *src, double alpha, int64_t N, cudaStream_t st);
void launch_combine(double *x, const double *Z, const GmresCoef &y, int64_t N, int32_t cnt, cudaStream_t st);
int32_t dots_partial_size();
// normal equations (kernels_ne.cu)
void launch_ne_form(const NeView &E, const double *Ax, const double *theta, double rho, DevCtl *ctl, cudaStream_t st);
void launch_ne_rhs(const NeView &E, const int32_t *perm, const double *Ax, const double *r7, const double *r1,
                   double *f, cudaStream_t st);
void launch_ne_dx(const NeView &E, const double *Ax, const double *dy, const double *r7, double *dx, cudaStream_t st);
void launch_residual_K(const NeView &E, const double *Ax, const double *theta, double rho, double delta,
                       const double *r7, const double *r1, const double *dx, const double *dy, double *f, double *r,
                       double *ad, double *ae, DevCtl *ctl, cudaStream_t st);
// backward error from precomputed r, |K||d|, |K|e, f (ctl->dinf set)
void launch_omega_only(int32_t N, const double *r, const double *ad, const double *ae, const double *f, DevCtl *ctl,
                       cudaStream_t st);
// kernel used to size the persistent sweeps' grid (occupancy query)
const void *persistent_probe_kernel();
void launch_permute_in(const DevPlan &P, const double *r7, const double *r1, double *f, cudaStream_t st);
void launch_permute_out(const DevPlan &P, const double *x, double *dx, double *dy, cudaStream_t st);
// skip != nullptr: the kernels return at entry while *skip != 0 (graph-captured refinement)
void launch_residual_omega(const DevPlan &P, const DevVals &V, const double *f, const double *x, double *r,
                           double *ad, double *ae, DevCtl *ctl, cudaStream_t st, const int32_t *skip = nullptr);
void launch_axpy(double *x, const double *c, int32_t N, cudaStream_t st, const int32_t *skip = nullptr);
void launch_refine_init(DevCtl *ctl, double target, int32_t max_steps, cudaStream_t st);
void launch_refine_step(DevCtl *ctl, double target, int32_t step, int32_t max_steps, cudaStream_t st);
void launch_refine_finish(DevCtl *ctl, double target, cudaStream_t st);
// dst = src when flag == nullptr or (*flag != 0) != invert
void launch_copy_if(double *dst, const double *src, int32_t N, const int32_t *flag, int32_t invert, cudaStream_t st);

}  // namespace ipm
