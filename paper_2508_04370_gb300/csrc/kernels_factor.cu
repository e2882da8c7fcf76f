// Numeric multifrontal factorisation kernels (Zanetti & Gondzio,
// arXiv 2508.04370, Sec. 4.1, 4.4, 4.5), FP64.
//
// Every front s owns a resident f x f slab (column-major, leading dimension
// ld) in one device arena.  After its factorisation the first k columns hold
// L (strictly lower part; D on the diagonal) and the trailing (f-k) x (f-k)
// lower block holds the contribution block (Schur complement) that the
// parent pulls during its own assembly (the strict upper part of a small
// front's slab holds scratch and is never read).  Children are always summed
// in ascending order, original entries first, so results do not depend on
// scheduling (Sec. 4.3, determinism).
//
// Kernels: k_small_fronts (a whole front of f <= 128 in shared memory, one
// CTA per front); the large-front bodies (assembly, diagonal block,
// triangular solve, lookahead strip, trailing tile), run either one launch
// per kind and pivot block or as items of the persistent level kernel
// k_large_level; k_norm1 / k_set_b1 (||K||_1 and the lift floor) and
// k_factor_stats (inertia, lifts).  The tensor-core trailing update is in
// kernels_tc.cu.
//
// Pivot rule (Sec. 4.5, Prop. 3), applied to pivot p of the current pivot
// block [b0, b1) of nb fully-summed columns:
//   d   = F_pp + s_p * sigma_p          (static term after the pivot is computed)
//   b2  = max over j in (p, b1) with s_j = s_p and s_j F_jj > 0 of F_jp^2 / |F_jj|
//   d  <- s_p * max(s_p d, max(eps_piv ||K||_1, b2))
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "ipm_dev.h"
#include "sliced_common.cuh"

namespace ipm {

namespace {

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double orig_value(const DevPlan &P, const DevVals &V, int64_t src) {
    if (src >= 0) return P.form == 1 ? V.Ax[src] : V.nev[src];
    const int64_t j = -1 - src;
    return -1.0 / V.theta[j];
}

// Pivot decision of Sec. 4.5 / Prop. 3 for pivot p of the block [0, w) held
// column-major in shared memory (one full warp, w <= 32):
//   d   = F_pp + s_p sigma_p          (static term after the pivot is computed)
//   b2  = max over j in (p, w) with s_j = s_p and s_j F_jj > 0 of F_jp^2 / |F_jj|
//   d  <- s_p max(s_p d, max(eps_piv ||K||_1, b2)).
// Every FP64 instruction costs this GPU about 64 cycles per warp whatever
// the number of active lanes, while integer instructions cost a few, so the
// common case is decided with integer arithmetic on the IEEE bit patterns:
// for non-negative doubles the bit pattern orders like the value, and
// bits(x) / 2^52 - 1023 is a lower bound of log2(x) that is within 0.0861 of
// it for normal x (and an upper-bound-preserving one for subnormal x).  A
// candidate j is screened out when 2 log2|F_jp| < log2|F_jj| + log2(t) - 0.0278
// with t = max(s_p d, eps_piv ||K||_1), which proves F_jp^2 / |F_jj| < t even
// after rounding, so b2 cannot change the pivot.  If any candidate survives
// the screen (rare: in exact arithmetic the same-sign block is definite and
// b2 <= |d|), the bound is evaluated exactly as written above.  Either way the
// result equals the plain evaluation of the rule.  Lane 0 records D, the
// lift and the status and returns the pivot and its reciprocal through
// shared memory.
constexpr long long kSignBit = (long long)0x8000000000000000ull;
constexpr long long kAbsMask = 0x7fffffffffffffffll;
constexpr long long kInfBits = 0x7ff0000000000000ll;
constexpr long long kBias = 0x3ff0000000000000ll;    // bits(1.0)
constexpr long long kScreen = 0x0003333333333333ll;  // 0.2 * 2^52
constexpr long long kTiny = 0x2000000000000000ll;    // bits(2^-511): squares stay normal above it
constexpr long long kHuge = 0x5fe0000000000000ll;    // bits(2^511): squares stay finite below it

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// 1 / x for a pivot: the hardware estimate (relative error below 2^-20 for
// normal x) refined by one third-order Newton-Raphson step for the
// reciprocal, r' = r (1 + e + e^2) with e = 1 - x r, whose error is about
// e^3 < 2^-60, below the rounding of the final fused multiply-add (so the
// result is within about half an ulp).  Three dependent FMAs instead of a
// full division on the pivot chain.  Outside [2^-1000, 2^1000] in magnitude
// (never the case for a pivot above the floor eps ||K||_1 of a sensible K)
// it divides.
__device__ __forceinline__ double recip_pivot(double x) {
    const long long a = __double_as_longlong(x) & 0x7fffffffffffffffll;
    if (a < 0x0170000000000000ll || a > 0x7e70000000000000ll) return 1.0 / x;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// x > b for a non-negative, non-NaN b, with IEEE semantics (NaN > b is false).
__device__ __forceinline__ bool gt_nonneg(long long xb, long long bb) {
    return xb >= 0 && xb <= kInfBits && xb > bb;
}

// The exact evaluation of the rule for the lanes the integer screen could
// not settle (maybe).  For non-negative values the rule only takes maxima,
// so it runs on bit patterns: the result is max(s_p d, b1, b2) and a lane
// can change it only if its F_jp^2 / |F_jj| exceeds t = max(s_p d, b1).  A
// second screen decides that without dividing: with a = fl(F_jp^2) and
// b = fl(t |F_jj|), bits(a) < bits(b) - 16 gives a < b (1 - 2^-49) and so
// fl(a / |F_jj|) < t (for lanes inside the first screen's ranges, where no
// product over- or underflows in a way that could mislead it).  Only the
// lanes left over divide, as the rule is written.  Returns the bits of the
// signed pivot.
__device__ __forceinline__ long long pivot_exact_bits(bool maybe, bool screenable, double c, double g, long long tb,
                                                      long long sdb, long long b1b, int sp) {
    bool need = false;
    if (maybe) {
        need = true;
        if (screenable) {
            const long long a = dbits(c * c), b = dbits(__longlong_as_double(tb) * fabs(g));
            need = !(a < b - 16);
        }
    }
    long long b2b = 0;
    if (__any_sync(0xffffffffu, need)) {
        if (need) b2b = dbits(c * c / fabs(g));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, b2b, o);
            if (ov > b2b) b2b = ov;
        }
    }
    const long long bndb = b1b > b2b ? b1b : b2b;            // max(b1, b2), both >= 0
    const long long res = gt_nonneg(sdb, bndb) ? sdb : bndb;  // s_p d > bnd ? s_p d : bnd
    return sp < 0 ? res ^ kSignBit : res;
}

__device__ __forceinline__ void pivot_warp(const double *Fd, int LDD, int p, int w, const int8_t *sgn, double rho,
                                           double delta, double b1floor, double *dstat, double *piv_out) {
    const int lane = threadIdx.x & 31;
    const int sp = sgn[p];
    const double d = Fd[p * LDD + p] + (sp < 0 ? -rho : delta);
    const long long db = dbits(d);
    const long long sdb = sp < 0 ? db ^ kSignBit : db;  // bits of s_p d
    const long long b1b = dbits(b1floor);
    const long long tb = gt_nonneg(sdb, b1b) ? sdb : b1b;  // bits of t = max(s_p d, b1)
    const bool t_ok = tb > 0x000fffffffffffffll && tb < kInfBits;  // t normal and finite
    bool maybe = false, screenable = false;
    double c = 0.0, g = 0.0;
    const int j = p + 1 + lane;
    if (j < w && sgn[j] == sp) {
        g = Fd[j * LDD + j];
        const long long jb = dbits(g);
        const long long ja = jb & kAbsMask;
        const bool cand = ja != 0 && ja <= kInfBits && ((jb < 0) == (sp < 0));  // s_j F_jj > 0
        if (cand) {
            c = Fd[p * LDD + j];
            const long long ab = dbits(c) & kAbsMask;
            if (ab != 0) {
                screenable = t_ok && ab >= kTiny && ab < kHuge && ja > 0x000fffffffffffffll && ja < kInfBits;
                maybe = !screenable || 2 * (ab - kBias) >= (ja - kBias) + (tb - kBias) - kScreen;
            }
        }
    }
    // the common-case pivot and its reciprocal, started before the vote so
    // that the reciprocal's latency overlaps the screen
    const long long dnb_fast = sp < 0 ? tb ^ kSignBit : tb;
    const double rinv_fast = recip_pivot(__longlong_as_double(dnb_fast));
    long long dnb = dnb_fast;
    if (__any_sync(0xffffffffu, maybe)) dnb = pivot_exact_bits(maybe, screenable, c, g, tb, sdb, b1b, sp);
    if (lane == 0) {
        const double dn = __longlong_as_double(dnb);
        dstat[p] = d;  // the lift dn - d and the status are formed off the chain
        piv_out[0] = dn;
        piv_out[1] = dnb == dnb_fast ? rinv_fast : recip_pivot(dn);
    }
}

// Named barriers, the id chosen by parity so that it stays an immediate:
// sync/arrive on barrier base + (parity & 1) with kCount threads.
template <int kBase, int kCount = 128>
__device__ __forceinline__ void bar_sync_parity(int parity) {
    if (parity & 1) asm volatile("bar.sync %0, %1;" ::"n"(kBase + 1), "n"(kCount) : "memory");
    else asm volatile("bar.sync %0, %1;" ::"n"(kBase), "n"(kCount) : "memory");
}
template <int kBase, int kCount = 128>
__device__ __forceinline__ void bar_arrive_parity(int parity) {
    if (parity & 1) asm volatile("bar.arrive %0, %1;" ::"n"(kBase + 1), "n"(kCount) : "memory");
    else asm volatile("bar.arrive %0, %1;" ::"n"(kBase), "n"(kCount) : "memory");
}

// ------------------------------------------------------------ small fronts
// One CTA per front, the whole front in shared memory.  FP64 is scarce on
// this GPU (about 0.4 FP64 FMA per clock per SM sub-partition), so every
// pivot's work is spread over all warps: warp 0 decides the pivot
// (pivot_warp), all threads scale the pivot column with one reciprocal and
// apply the rank-1 update to the rest of the pivot block's columns (all rows
// below, which also performs the triangular solve of the rows under the
// block); after each block of 32 pivots all threads apply the block to the
// trailing lower part.
template <int NT>
__global__ void __launch_bounds__(NT) k_small_fronts(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                      double *__restrict__ Dg, double *__restrict__ Dig,
                                                      double *__restrict__ dyng,
                                                      DevCtl *ctl, const int32_t *__restrict__ list, int nb) {
    extern __shared__ double smem[];
    __shared__ double wcol[128];  // fronts up to 128 rows use this kernel
    __shared__ double dq[32];
    __shared__ double dsm[32];  // statically regularised pivots of the block, before any lift
    __shared__ double piv[2];
    __shared__ int8_t sg[128];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    double *F = smem;  // ld * f
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
    const int sz = ld * f;
    for (int t = tid; t < sz; t += NT) F[t] = 0.0;
    __syncthreads();
    for (int64_t q = P.orig_ptr[s] + tid; q < P.orig_ptr[s + 1]; q += NT)
        F[P.orig_dst[q]] = orig_value(P, V, P.orig_src[q]);
    __syncthreads();
    for (int q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
        const int c = P.child_list[q];
        const int kc = P.sn_k[c], ldc = P.sn_ld[c];
        const int cc = P.sn_f[c] - kc;
        const double *CB = fronts + P.sn_off[c] + (int64_t)kc * ldc + kc;
        const int32_t *map = P.relmap + P.map_off[c];
        for (int t = tid; t < cc * cc; t += NT) {
            const int jj = t / cc, ii = t - jj * cc;
            if (ii >= jj) F[map[jj] * ld + map[ii]] += CB[(int64_t)jj * ldc + ii];
        }
        __syncthreads();
    }
    for (int t = tid; t < k; t += NT) sg[t] = P.sign[c0 + t];
    __syncthreads();
    const int8_t *sgn = sg;
    const double b1floor = pivot_floor(P, ctl, c0);
    for (int b0 = 0; b0 < k; b0 += nb) {
        const int b1 = min(b0 + nb, k), w = b1 - b0;
        double *Fb = F + b0 * ld + b0;
        for (int p = 0; p < w; p++) {
            if (warp == 0) pivot_warp(Fb, ld, p, w, sgn + b0, V.rho, V.delta, b1floor, dsm, piv);
            __syncthreads();
            const double dn = piv[0], rinv = piv[1];
            const int pc = b0 + p;  // front column of the pivot
            for (int i = pc + 1 + tid; i < f; i += NT) {
                const double v = F[pc * ld + i];
                wcol[i] = v;
                F[pc * ld + i] = v * rinv;
            }
            if (tid == 0) {
                F[pc * ld + pc] = dn;
                dq[p] = dn;
                Dig[c0 + pc] = rinv;
            }
            __syncthreads();
            // rank-1 update of the block's remaining columns, all rows below
            for (int j = pc + 1 + warp; j < b0 + w; j += NW) {
                const double wj = wcol[j];
                for (int i = j + lane; i < f; i += 32) F[j * ld + i] -= F[pc * ld + i] * wj;
            }
            __syncthreads();
        }
        // the block's pivots, lifts and status (dq and dsm are rewritten only
        // after the barriers of the trailing update)
        if (tid < w) {
            const double dn = dq[tid], d = dsm[tid];
            const long long db = dbits(d), dnb = dbits(dn);
            Dg[c0 + b0 + tid] = dn;
            dyng[c0 + b0 + tid] = dnb == db ? 0.0 : dn - d;
            const bool fin = (db & kAbsMask) < kInfBits && (dnb & kAbsMask) < kInfBits && (dnb & kAbsMask) != 0;
            if (!fin) atomicOr(&ctl->status, kStatNonFinite);
        }
        // trailing update of columns [b1, f) by the block's pivots:
        // W_jq = L_jq d_q is formed once into the unused upper triangle
        // (row b0 + q of column j), then each entry takes one FMA per pivot
        for (int t = tid; t < w * (f - b1); t += NT) {
            const int q = t % w, j = b1 + t / w;
            F[j * ld + b0 + q] = F[(b0 + q) * ld + j] * dq[q];
        }
        __syncthreads();
        for (int j = b1 + warp; j < f; j += NW) {
            for (int i = j + lane; i < f; i += 32) {
                double acc = 0.0;
                for (int q = 0; q < w; q++) acc += F[(b0 + q) * ld + i] * F[j * ld + b0 + q];
                F[j * ld + i] -= acc;
            }
        }
        __syncthreads();
    }
    double *out = fronts + P.sn_off[s];
    for (int t = tid; t < sz; t += NT) out[t] = F[t];
}

// -------------------------------------------------------------- large fronts
// The work on a large front is cut into items (Sec. 4.4: per pivot block of
// nb = 32 columns, the diagonal block, the triangular solve of the rows below
// it and the trailing update), each written once as a CTA-wide body (256
// threads call it; bodies that need fewer leave the others idle).  The
// bodies serve both the one-launch-per-step kernels and the persistent
// level kernel below.  Front data are read through L2 (ld.global.cg)
// because in the persistent kernel other CTAs of the same launch wrote
// them.  All bodies share one shared-memory pool sized for the largest.
constexpr int kBodyThreads = 256;
constexpr int kPoolDoubles = 2 * 32 * 33 + 32;  // a 32 x 32 update tile's two operands; L_11, 1/d and a 32 x 33 tile

// Assembly of columns [c_lo, c_hi), rows [ai.r_lo, ai.r_hi) of front s into
// its slab in global memory: zero the block, place the original entries (a
// precomputed contiguous range of the columns' entries, filtered by row),
// then add the children's contribution-block entries that land in the block
// (column and row ranges precomputed per child), children in ascending order.
// Rows above the block's first column (the upper part) are never read and
// are not written.  Child descriptors are staged in shared memory 64 at a
// time.
constexpr int kAsmBatch = 8;  // contribution-block rows per lane per round of the extend-add

__device__ __forceinline__ void body_assemble(const DevPlan &P, const DevVals &V, double *__restrict__ fronts, int s,
                                              int c_lo, int c_hi, const AsmItem &ai, const int32_t *__restrict__ acr,
                                              double *pool) {
    constexpr int NT = kBodyThreads;
    int32_t *ch_a = reinterpret_cast<int32_t *>(pool), *ch_b = ch_a + 64, *ch_ldc = ch_b + 64;
    int32_t *ch_ilo = ch_ldc + 64, *ch_ihi = ch_ilo + 64;
    int64_t *ch_cb = reinterpret_cast<int64_t *>(ch_ihi + 64), *ch_map = ch_cb + 64;
    const int ld = P.sn_ld[s];
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncol = c_hi - c_lo, r_lo = ai.r_lo, r_hi = ai.r_hi;
    for (int c = 0; c < ncol; c++)
        for (int r = r_lo + tid; r < r_hi; r += NT) F[(int64_t)(c_lo + c) * ld + r] = 0.0;
    __syncthreads();
    for (int64_t q = ai.o0 + tid; q < ai.o1; q += NT) {
        const int32_t d = P.orig_dst[q];
        const int r = d % ld;
        if (r >= r_lo && r < r_hi) F[d] = orig_value(P, V, P.orig_src[q]);
    }
    const int q0 = P.child_ptr[s], nch = P.child_ptr[s + 1] - q0;
    for (int base = 0; base < nch; base += 64) {
        __syncthreads();
        if (tid < 64 && base + tid < nch) {
            const int c = P.child_list[q0 + base + tid];
            const int kc = P.sn_k[c], ldc = P.sn_ld[c];
            const int32_t *e = acr + 4 * (ai.cr + base + tid);
            ch_a[tid] = e[0];
            ch_b[tid] = e[1];
            ch_ilo[tid] = e[2];
            ch_ihi[tid] = e[3];
            ch_ldc[tid] = ldc;
            ch_cb[tid] = P.sn_off[c] + (int64_t)kc * ldc + kc;
            ch_map[tid] = P.map_off[c];
        }
        __syncthreads();
        const int nu = min(64, nch - base);
        for (int u = 0; u < nu; u++) {
            const int a = ch_a[u], b = ch_b[u], ilo = ch_ilo[u], ihi = ch_ihi[u];
            if (a >= b || ilo >= ihi) continue;  // uniform over the CTA
            const int ldc = ch_ldc[u];
            const double *CB = fronts + ch_cb[u];
            const int32_t *map = P.relmap + ch_map[u];
            for (int jj = a + warp; jj < b; jj += NT / 32) {
                double *Fj = F + (int64_t)map[jj] * ld;
                const double *CBj = CB + (int64_t)jj * ldc;
                // kAsmBatch rows per lane per round, every load issued before
                // any store: the entries one child adds to are distinct, so
                // the batch's loads are independent of its stores (the child
                // block and the front never overlap), and each entry still
                // receives its children's terms in ascending child order
                for (int i0 = max(jj, ilo) + lane; i0 < ihi; i0 += 32 * kAsmBatch) {
                    int32_t mi[kAsmBatch];
                    double cv[kAsmBatch], fv[kAsmBatch];
#pragma unroll
                    for (int t = 0; t < kAsmBatch; t++) {
                        const int ii = i0 + 32 * t;
                        mi[t] = ii < ihi ? __ldg(map + ii) : -1;
                        cv[t] = ii < ihi ? __ldcg(CBj + ii) : 0.0;
                    }
#pragma unroll
                    for (int t = 0; t < kAsmBatch; t++) fv[t] = mi[t] >= 0 ? Fj[mi[t]] : 0.0;
#pragma unroll
                    for (int t = 0; t < kAsmBatch; t++)
                        if (mi[t] >= 0) Fj[mi[t]] = fv[t] + cv[t];
                }
            }
            __syncthreads();
        }
    }
}

// The nb x nb diagonal block of panel [p0, p0 + nb) of front s as a
// pipeline over the pivots spread over the SM's four sub-partitions (each
// FP64 instruction holds its sub-partition's FP64 pipe for tens of cycles,
// so the pivot chain is kept to as few FP64 instructions as possible on one
// of them).  Warp 0 owns the pivot chain: lane j keeps c = F_jp of the
// current pivot column, g = F_jj and gs = F_jj + s_j sigma_j (the static
// term) up to date; per pivot it screens the Prop. 3 candidates, scales the
// column (l_jp = F_jp / d_p, keeping the unscaled w_jp = F_jp), publishes p,
// and brings gs (first, for the next pivot), c and g to pivot p + 1.  Warp 5
// forms the reciprocal of each pivot's common case (the pivot or the lift
// floor, whichever is larger) from d, handed over through shared memory, while
// warp 0 screens; warp 0 recomputes it only when the exact rule moves the
// pivot.  Warps 2, 3, 6 and 7 apply pivot p to the strictly lower entries
// of columns >= p + 2 while warp 0 already works on pivot p + 1, which needs
// only column p + 1 and the diagonal; each of their threads holds up to four
// of these entries in registers for the whole block and stores one when its
// column has received its last update here.  Named barriers alternate by
// pivot parity (1-2 pivot published, 3-4 columns updated, 5-6 d ready, 7-8
// reciprocal ready), so no side runs more than one pivot ahead.  Every value
// is formed by the same operations as in a single warp, so the factor does
// not depend on the split.  The factorised block goes back to the slab (L
// strictly below the diagonal, D on it) together with D, 1/D and the lifts,
// and the panel workspace ws receives the rows of L_11 (row-major,
// ws[q * 33 + q'] = L_qq') and 1 / d_q for the triangular solve below.
constexpr int kPanelWs = 32 * 33 + 32;  // doubles of panel workspace per large front

__device__ __forceinline__ void body_diag(const DevPlan &P, const DevVals &V, double *__restrict__ fronts,
                                          double *__restrict__ Dg, double *__restrict__ Dig,
                                          double *__restrict__ dyng, DevCtl *ctl, int s, int p0, int nb,
                                          double *__restrict__ ws, double *pool) {
    // warp 0 (SM sub-partition 0) carries the chain, warp 5 (sub-partition 1)
    // forms each pivot's reciprocal, warps 2, 3, 6 and 7 (sub-partitions 2
    // and 3) apply the pivots to the later columns
    constexpr int LDD = 33, NU = 128, kOwn = 4;  // 4 x 128 >= 435 entries
    constexpr int kBarPub = 1, kBarUpd = 3, kBarD = 5, kBarR = 7;
    constexpr int kPubCount = 32 + NU;  // warp 0 and the update warps
    double *Fd = pool;                          // 32 x 33, column-major
    double(*wsv)[32] = reinterpret_cast<double(*)[32]>(pool + 32 * 33);  // [2][32]
    double *Dtmp = pool + 32 * 33 + 64, *dstat = Dtmp + 32, *rtmp = dstat + 32;
    int8_t *sg = reinterpret_cast<int8_t *>(rtmp + 32);
    double *shd = rtmp + 32 + 4, *shr = shd + 2;  // pivot d and its reciprocal, by pivot parity
    const int k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    const int w = min(p0 + nb, k) - p0;
    if (w <= 0) return;  // uniform over the CTA
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        // all loads in flight before the shared-memory stores
        constexpr int U = 32 * 32 / kBodyThreads;
        double v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = tid + u * kBodyThreads, jj = t >> 5, ii = t & 31;
            v[u] = (jj < w && ii < w && ii >= jj) ? __ldcg(F + (int64_t)(p0 + jj) * ld + (p0 + ii)) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = tid + u * kBodyThreads;
            Fd[(t >> 5) * LDD + (t & 31)] = v[u];
        }
    }
    if (tid < 32) sg[tid] = tid < w ? P.sign[c0 + p0 + tid] : (int8_t)0;
    __syncthreads();
    if (warp == 0) {
        const double b1floor = pivot_floor(P, ctl, c0);
        const long long b1b = dbits(b1floor);
        const int sl = sg[lane];
        double g = lane < w ? Fd[lane * LDD + lane] : 0.0;   // F_jj of row j = lane
        double gs = g + (sl < 0 ? -V.rho : V.delta);
        double c = (lane > 0 && lane < w) ? Fd[lane] : 0.0;  // column 0
        double my_dn = 0.0, my_d = 0.0, my_r = 0.0;          // lane p keeps pivot p's values
        double d = __shfl_sync(0xffffffffu, gs, 0);
        if (lane == 0) shd[0] = d;
        __syncwarp();
        bar_arrive_parity<kBarD, 64>(0);
        for (int p = 0; p < w; p++) {
            const int sp = __shfl_sync(0xffffffffu, sl, p);
            // the Prop. 3 screen (on IEEE bit patterns) while warp 5 forms the
            // reciprocal of the common-case pivot
            const long long db = dbits(d);
            const long long sdb = sp < 0 ? db ^ kSignBit : db;
            const long long tb = gt_nonneg(sdb, b1b) ? sdb : b1b;
            const bool t_ok = tb > 0x000fffffffffffffll && tb < kInfBits;
            bool maybe = false, screenable = false;
            if (lane > p && lane < w && sl == sp) {
                const long long jb = dbits(g);
                const long long ja = jb & kAbsMask;
                const bool cand = ja != 0 && ja <= kInfBits && ((jb < 0) == (sp < 0));
                if (cand) {
                    const long long ab = dbits(c) & kAbsMask;
                    if (ab != 0) {
                        screenable = t_ok && ab >= kTiny && ab < kHuge && ja > 0x000fffffffffffffll && ja < kInfBits;
                        maybe = !screenable || 2 * (ab - kBias) >= (ja - kBias) + (tb - kBias) - kScreen;
                    }
                }
            }
            const long long dnb_fast = sp < 0 ? tb ^ kSignBit : tb;
            const bool any = __any_sync(0xffffffffu, maybe);
            bar_sync_parity<kBarR, 64>(p);
            double rinv = shr[p & 1];
            long long dnb = dnb_fast;
            if (any) {
                dnb = pivot_exact_bits(maybe, screenable, c, g, tb, sdb, b1b, sp);
                if (dnb != dnb_fast) rinv = recip_pivot(__longlong_as_double(dnb));
            }
            const double dn = __longlong_as_double(dnb);
            if (lane == p) {
                my_dn = dn;
                my_d = d;
                my_r = rinv;
            }
            const bool below = lane > p && lane < w;
            const double l = below ? c * rinv : 0.0;
            if (below) {
                Fd[p * LDD + lane] = l;
                wsv[p & 1][lane] = c;
            }
            __syncwarp();
            bar_arrive_parity<kBarPub, kPubCount>(p);
            if (p + 1 < w) {
                if (p >= 1) bar_sync_parity<kBarUpd, kPubCount>(p + 1);  // pivot p-1 applied to columns >= p+1
                const double wn = __shfl_sync(0xffffffffu, c, p + 1);  // w_{p+1,p}, unscaled
                const double fv = (lane > p + 1 && lane < w) ? Fd[(p + 1) * LDD + lane] : 0.0;
                // the next pivot first, so that its reciprocal starts early
                gs -= l * c;
                d = __shfl_sync(0xffffffffu, gs, p + 1);
                if (lane == 0) shd[(p + 1) & 1] = d;
                __syncwarp();
                bar_arrive_parity<kBarD, 64>(p + 1);
                const double cn = fv - l * wn;
                g -= l * c;
                c = lane > p + 1 ? cn : 0.0;
            }
        }
        // the pivots' values, off the chain (read only after the CTA barrier)
        if (lane < w) {
            Fd[lane * LDD + lane] = my_dn;
            Dtmp[lane] = my_dn;
            dstat[lane] = my_d;
            rtmp[lane] = my_r;
            const long long db = dbits(my_d), dnb = dbits(my_dn);
            const bool fin = (db & kAbsMask) < kInfBits && (dnb & kAbsMask) < kInfBits && (dnb & kAbsMask) != 0;
            if (!fin) atomicOr(&ctl->status, kStatNonFinite);
        }
    } else if (warp == 5) {
        // the reciprocal of each pivot's common case: the larger (as bit
        // patterns) of s_p d and the lift floor, with the sign s_p
        const long long b1b = dbits(pivot_floor(P, ctl, c0));
        for (int p = 0; p < w; p++) {
            const int sp = sg[p];
            bar_sync_parity<kBarD, 64>(p);
            const long long db = dbits(shd[p & 1]);
            const long long sdb = sp < 0 ? db ^ kSignBit : db;
            const long long tb = gt_nonneg(sdb, b1b) ? sdb : b1b;
            const double r = recip_pivot(__longlong_as_double(sp < 0 ? tb ^ kSignBit : tb));
            if (lane == 0) shr[p & 1] = r;
            __syncwarp();
            bar_arrive_parity<kBarR, 64>(p);
        }
    } else if (warp == 2 || warp == 3 || warp == 6 || warp == 7) {
        // this thread owns the strictly lower entries e = ut + 128 t of columns
        // >= 2, enumerated last column first: e = r (r + 1) / 2 + c  ->
        // column w-2-r, row w-1-r+c (0 <= c <= r)
        const int ut = ((warp & 3) - 2 + 2 * (warp >> 2)) * 32 + lane;
        const int nall = w >= 3 ? (w - 3) * (w - 2) / 2 : 0;
        int jo[kOwn], io[kOwn];
        double vo[kOwn];
#pragma unroll
        for (int t = 0; t < kOwn; t++) {
            const int e = ut + NU * t;
            jo[t] = 0;
            io[t] = 0;
            vo[t] = 0.0;
            if (e < nall) {
                int r = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                while ((r + 1) * (r + 2) / 2 <= e) r++;
                while (r * (r + 1) / 2 > e) r--;
                jo[t] = w - 2 - r;
                io[t] = w - 1 - r + (e - r * (r + 1) / 2);
                vo[t] = Fd[jo[t] * LDD + io[t]];
            }
        }
        for (int q = 0; q < w; q++) {
            bar_sync_parity<kBarPub, kPubCount>(q);
            const int m = w - 3 - q;  // columns >= q + 2 have m (m + 1) / 2 such entries
            const int ne = m > 0 ? m * (m + 1) / 2 : 0;
            double lq[kOwn], wq[kOwn];
#pragma unroll
            for (int t = 0; t < kOwn; t++) {
                const bool on = ut + NU * t < ne;
                lq[t] = on ? Fd[q * LDD + io[t]] : 0.0;
                wq[t] = on ? wsv[q & 1][jo[t]] : 0.0;
            }
#pragma unroll
            for (int t = 0; t < kOwn; t++) {
                if (ut + NU * t < ne) {
                    vo[t] -= lq[t] * wq[t];
                    if (jo[t] == q + 2) Fd[jo[t] * LDD + io[t]] = vo[t];
                }
            }
            if (q <= w - 3) bar_arrive_parity<kBarUpd, kPubCount>(q);
        }
    }
    __syncthreads();
    for (int t = tid; t < 32 * 32; t += kBodyThreads) {
        const int jj = t >> 5, ii = t & 31;
        const bool in = jj < w && ii < w;
        if (in && ii >= jj) F[(int64_t)(p0 + jj) * ld + (p0 + ii)] = Fd[jj * LDD + ii];
        ws[ii * 33 + jj] = (in && ii > jj) ? Fd[jj * LDD + ii] : 0.0;  // L(row ii, column jj), row-major
    }
    if (tid < 32) {
        const int t = tid;
        ws[32 * 33 + t] = t < w ? rtmp[t] : 0.0;
        if (t < w) {
            const double dn = Dtmp[t], d = dstat[t];
            Dg[c0 + p0 + t] = dn;
            Dig[c0 + p0 + t] = rtmp[t];
            dyng[c0 + p0 + t] = dbits(dn) == dbits(d) ? 0.0 : dn - d;
        }
    }
}

// Rows [r0, r1) below the diagonal block of panel [p0, p0 + nb), one warp
// per row with one lane per pivot column q.  With u_iq = l_iq d_q the rows
// satisfy
//   u_iq = F_iq - sum_{q' < q} u_iq' L_qq',   l_iq = u_iq / d_q,
// so step q' broadcasts the finished u_iq' and every lane q > q' applies one
// FMA: 32 dependent steps per row instead of 528 per thread when a thread
// owns a whole row.  An item holds up to kTrsmItemRows rows (chunks of the
// level kernel hold kTrsmRows); warp w solves rows w, w + 8, w + 16 and
// w + 24 together, four independent chains on the same L_11, so a CTA costs
// about one chain's latency.
constexpr int kTrsmRows = 8;
constexpr int kTrsmItemRows = 32;
static_assert(kTrsmRows == kTrsmRowsHost && kTrsmItemRows == kTrsmItemRowsHost, "host and device row chunks differ");
static_assert(32 * kTrsmRows == kBodyThreads, "one warp per row");

// Where the triangular solve of a sliced front writes the digit slices of the
// rows it finishes (ws == nullptr: no slicing): block base + (row - p1) / 128,
// row (row - p1) % 128 of the step's work space.  pair = 0: one chunk, this
// panel's columns; pair = 1 (the second panel of a pair): two chunks with one
// row scale, the previous panel's 32 columns (final since the last step)
// and this panel's.
struct SliceOut {
    uint8_t *ws;
    int32_t *exps;
    int32_t base;
    int32_t pair;
    int32_t p1;
    const double *D;
    DevCtl *ctl;
};

template <int RW>  // rows per warp, solved together: items of up to 8 RW rows
__device__ __forceinline__ void body_trsm(const DevPlan &P, double *__restrict__ fronts, int s, int r0, int r1,
                                          int p0, int nb, const double *__restrict__ ws, double *pool,
                                          const SliceOut so = SliceOut{nullptr, nullptr, 0, 0, 0, nullptr, nullptr}) {
    constexpr int kRows = kTrsmRows * RW;
    constexpr int TP = kRows + 1;  // padded row count of the tile
    double *Wd = pool;                             // 32 x 33 + 32
    double(*T)[TP] = reinterpret_cast<double(*)[TP]>(pool + 32 * 33 + 32);  // [32 columns][rows]
    const int k = P.sn_k[s], ld = P.sn_ld[s];
    const int w = min(p0 + nb, k) - p0;
    const int nr = r1 - r0;  // <= kRows
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        // all loads in flight before the shared-memory stores
        constexpr int U = (32 * 33 + 32 + kBodyThreads - 1) / kBodyThreads;
        constexpr int V = 32 * kRows / kBodyThreads;
        double v[U], tv[V];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = tid + u * kBodyThreads;
            v[u] = t < 32 * 33 + 32 ? __ldcg(ws + t) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < V; u++) {
            const int t = tid + u * kBodyThreads, q = t / kRows, r = t % kRows;
            tv[u] = (q < w && r < nr) ? __ldcg(F + (int64_t)(p0 + q) * ld + r0 + r) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = tid + u * kBodyThreads;
            if (t < 32 * 33 + 32) Wd[t] = v[u];
        }
#pragma unroll
        for (int u = 0; u < V; u++) {
            const int t = tid + u * kBodyThreads;
            T[t / kRows][t % kRows] = tv[u];
        }
    }
    __syncthreads();
    if (warp < nr) {
        // rows warp, warp + 8, ... : RW independent chains share L_11 in registers
        double Lr[32];
#pragma unroll
        for (int c = 0; c < 32; c++) Lr[c] = Wd[lane * 33 + c];
        double t[RW];
#pragma unroll
        for (int j = 0; j < RW; j++) t[j] = T[lane][warp + kTrsmRows * j];
#pragma unroll
        for (int c = 0; c < 31; c++) {
#pragma unroll
            for (int j = 0; j < RW; j++) {
                const double u = __shfl_sync(0xffffffffu, t[j], c);
                if (lane > c) t[j] -= u * Lr[c];
            }
        }
        const double dinv = Wd[32 * 33 + lane];
#pragma unroll
        for (int j = 0; j < RW; j++) {
            const int rr = warp + kTrsmRows * j;
            if (rr >= nr) break;  // uniform over the warp
            const double lv = t[j] * dinv;
            T[lane][rr] = lv;
            if (so.ws) {
                // the finished row, sliced for the tensor-core update
                const int row = r0 + rr;
                const int c0 = P.sn_c0[s];
                const double dq = lane < w ? so.D[c0 + p0 + lane] : 0.0;
                const double lq = lane < w ? lv : 0.0;
                const int blk = so.base + (row - so.p1) / kSliceRows;
                uint8_t *bp = so.ws + (int64_t)blk * kSliceBlockBytes;
                int32_t *ep = so.exps + (int64_t)blk * kSliceRows * 2;
                bool bad;
                if (so.pair) {
                    // the previous panel (always 32 columns) as chunk 0, this one as chunk 1
                    const double l2[2] = {__ldcg(F + (int64_t)(p0 - 32 + lane) * ld + row), lq};
                    const double d2[2] = {so.D[c0 + p0 - 32 + lane], dq};
                    bad = sliced::slice_row_warp<2>(l2, d2, bp, ep, (row - so.p1) % kSliceRows);
                } else {
                    const double l1[1] = {lq}, d1[1] = {dq};
                    bad = sliced::slice_row_warp<1>(l1, d1, bp, ep, (row - so.p1) % kSliceRows);
                }
                if (bad && lane == 0) atomicOr(&so.ctl->status, kStatNonFinite);
            }
        }
    }
    __syncthreads();
    for (int t = tid; t < 32 * kRows; t += kBodyThreads) {
        const int q = t / kRows, r = t % kRows;
        if (q < w && r < nr) F[(int64_t)(p0 + q) * ld + r0 + r] = T[q][r];
    }
}

// Trailing update of the lower part of columns [p1, f) by the panel
// [p0, p0+w): C(i, j) -= sum_q L(i,q) d_q L(j,q), one kUpdTile x kUpdTile
// tile at (i0, j0), 16 x 16 threads with 2 x 2 outputs each.  FP64 runs at
// about 2 FMA per clock per SM on this GPU, so tiles are small (32 x 32) to
// put every SM to work.
__device__ __forceinline__ void body_tile(const DevPlan &P, double *__restrict__ fronts,
                                          const double *__restrict__ Dg, int s, int i0, int j0, int p0, int w,
                                          double *pool) {
    constexpr int T = kUpdTile;
    static_assert(T == 32, "16 x 16 threads, 2 x 2 outputs");
    double(*As)[T + 1] = reinterpret_cast<double(*)[T + 1]>(pool);
    double(*Bs)[T + 1] = reinterpret_cast<double(*)[T + 1]>(pool + 32 * (T + 1));
    const int f = P.sn_f[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    w = min(w, P.sn_k[s] - p0);  // ragged last panel
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    // this thread's 2 x 2 outputs of the tile (lower part, columns from the
    // panel's end), fetched with the operands: their latency overlaps the
    // operand loads instead of following the products
    double cv[2][2];
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const int j = j0 + ty + 16 * b;
#pragma unroll
        for (int a = 0; a < 2; a++) {
            const int i = i0 + tx + 16 * a;
            cv[a][b] = (j < f && j >= p0 + w && i < f && i >= j) ? __ldcg(F + (int64_t)j * ld + i) : 0.0;
        }
    }
    {
        // all loads in flight before the shared-memory stores
        constexpr int U = 32 * T / kBodyThreads;
        double va[U], vb[U], vd[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = tid + u * kBodyThreads, q = t / T, r = t % T;
            const int i = i0 + r, j = j0 + r;
            const bool qa = q < w;
            va[u] = (qa && i < f) ? __ldcg(F + (int64_t)(p0 + q) * ld + i) : 0.0;
            vb[u] = (qa && j < f) ? __ldcg(F + (int64_t)(p0 + q) * ld + j) : 0.0;
            vd[u] = qa ? __ldcg(Dg + c0 + p0 + q) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = tid + u * kBodyThreads, q = t / T, r = t % T;
            As[q][r] = va[u];
            Bs[q][r] = vb[u] * vd[u];
        }
    }
    __syncthreads();
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int q = 0; q < w; q++) {
        const double a0 = As[q][tx], a1 = As[q][tx + 16];
        const double b0 = Bs[q][ty], b1 = Bs[q][ty + 16];
        acc[0][0] += a0 * b0;
        acc[1][0] += a1 * b0;
        acc[0][1] += a0 * b1;
        acc[1][1] += a1 * b1;
    }
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const int j = j0 + ty + 16 * b;
        if (j >= f || j < p0 + w) continue;  // a grid tile cut by a partial last panel
#pragma unroll
        for (int a = 0; a < 2; a++) {
            const int i = i0 + tx + 16 * a;
            if (i < f && i >= j) F[(int64_t)j * ld + i] = cv[a][b] - acc[a][b];
        }
    }
}

// The same update for the next panel's columns, which lie on the critical
// path: a strip of kUpdTile rows x kStripCols columns at (i0, j0), one
// output per thread on threads 0..32 kStripCols - 1, summed over the panel's
// pivots in the same order as body_tile (so the results are identical).  A
// whole 32 x 32 tile is 32k FP64 FMAs, about 8 us on one SM of this GPU;
// strips spread those few tiles over eight times as many SMs.
__device__ __forceinline__ void body_strip(const DevPlan &P, double *__restrict__ fronts,
                                           const double *__restrict__ Dg, int s, int i0, int j0, int p0, int w,
                                           double *pool) {
    constexpr int T = kUpdTile, C = kStripCols;
    static_assert(T == 32 && 32 * C <= kBodyThreads, "one row per lane, one column per warp");
    double(*As)[T + 1] = reinterpret_cast<double(*)[T + 1]>(pool);
    double(*Bs)[C] = reinterpret_cast<double(*)[C]>(pool + 32 * (T + 1));
    const int f = P.sn_f[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    w = min(w, P.sn_k[s] - p0);
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x;
    {
        // all loads in flight before the shared-memory stores
        constexpr int U = 32 * T / kBodyThreads;
        double va[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = tid + u * kBodyThreads, q = t / T, r = t % T;
            va[u] = (q < w && i0 + r < f) ? __ldcg(F + (int64_t)(p0 + q) * ld + i0 + r) : 0.0;
        }
        double vb = 0.0, vd = 0.0;
        const int q = tid / C, cc = tid % C, j = j0 + cc;
        if (tid < 32 * C && q < w && j < f) {
            vb = __ldcg(F + (int64_t)(p0 + q) * ld + j);
            vd = __ldcg(Dg + c0 + p0 + q);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = tid + u * kBodyThreads;
            As[t / T][t % T] = va[u];
        }
        if (tid < 32 * C) Bs[q][cc] = vb * vd;
    }
    __syncthreads();
    const int r = tid & 31, cc = tid >> 5;
    const int i = i0 + r, j = j0 + cc;
    if (cc < C && i < f && j < f && i >= j && j >= p0 + w) {
        double acc = 0.0;
        for (int q = 0; q < w; q++) acc += As[q][r] * Bs[q][cc];
        double *e = F + (int64_t)j * ld + i;
        *e = __ldcg(e) - acc;
    }
}

// One launch per step: one item per CTA.
__global__ void __launch_bounds__(kBodyThreads) k_large_assemble(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                                  const PanelItem *__restrict__ items,
                                                                  const AsmItem *__restrict__ ainfo,
                                                                  const int32_t *__restrict__ acr) {
    __shared__ double pool[kPoolDoubles];
    const PanelItem it = items[blockIdx.x];
    body_assemble(P, V, fronts, it.s, it.r0, it.r1, ainfo[blockIdx.x], acr, pool);
}

__global__ void __launch_bounds__(kBodyThreads) k_panel_diag(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                              double *__restrict__ Dg, double *__restrict__ Dig,
                                                              double *__restrict__ dyng, DevCtl *ctl,
                                                              const PanelItem *__restrict__ items, int nb,
                                                              double *__restrict__ pws) {
    __shared__ double pool[kPoolDoubles];
    const PanelItem it = items[blockIdx.x];
    body_diag(P, V, fronts, Dg, Dig, dyng, ctl, it.s, it.p0, nb, pws + (int64_t)it.r1 * kPanelWs, pool);
}

__global__ void __launch_bounds__(kBodyThreads) k_panel_trsm(DevPlan P, double *__restrict__ fronts,
                                                              const PanelItem *__restrict__ items,
                                                              const int32_t *slots, int nb,
                                                              const double *__restrict__ pws,
                                                              const int32_t *__restrict__ sbase, uint8_t *sws,
                                                              int32_t *sexp, const double *__restrict__ Dg,
                                                              DevCtl *ctl) {
    __shared__ double pool[kPoolDoubles];
    const PanelItem it = items[blockIdx.x];
    SliceOut so{nullptr, nullptr, 0, 0, 0, nullptr, nullptr};
    if (sws && sbase[blockIdx.x] >= 0)
        so = SliceOut{sws, sexp, sbase[blockIdx.x] >> 1, sbase[blockIdx.x] & 1, min(it.p0 + nb, P.sn_k[it.s]), Dg,
                      ctl};
    body_trsm<kTrsmItemRows / kTrsmRows>(P, fronts, it.s, it.r0, it.r1, it.p0, nb,
                                         pws + (int64_t)slots[blockIdx.x] * kPanelWs, pool, so);
}

__global__ void __launch_bounds__(kBodyThreads) k_large_update(DevPlan P, double *__restrict__ fronts,
                                                                const double *__restrict__ Dg,
                                                                const TileItem *__restrict__ items, int w) {
    __shared__ double pool[kPoolDoubles];
    const TileItem it = items[blockIdx.x];
    body_tile(P, fronts, Dg, it.s, it.i0, it.j0, it.p0, w, pool);
}

__global__ void __launch_bounds__(kBodyThreads) k_large_update_strip(DevPlan P, double *__restrict__ fronts,
                                                                        const double *__restrict__ Dg,
                                                                        const TileItem *__restrict__ items, int w) {
    __shared__ double pool[kPoolDoubles];
    const TileItem it = items[blockIdx.x];
    body_strip(P, fronts, Dg, it.s, it.i0, it.j0, it.p0, w, pool);
}

// A thin front (one pivot block, k <= nb, f <= kThinMaxF) whole in one CTA:
// the same bodies as the one-launch-per-step kernels, called in sequence
// (assembly by 32-column blocks, the diagonal block, the triangular solve in
// 32-row items, the trailing 32 x 32 tiles), so the front's values are
// those of the per-step path bit for bit; a level of many such fronts costs
// one launch instead of one per body and item.
__global__ void __launch_bounds__(kBodyThreads, 3) k_thin_fronts(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                               double *__restrict__ Dg, double *__restrict__ Dig,
                                                               double *__restrict__ dyng, DevCtl *ctl,
                                                               const int32_t *__restrict__ list,
                                                               const int32_t *__restrict__ first_asm,
                                                               const int32_t *__restrict__ slots,
                                                               const AsmItem *__restrict__ ainfo,
                                                               const int32_t *__restrict__ acr, double *__restrict__ pws,
                                                               int nb) {
    __shared__ double pool[kPoolDoubles];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s];
    const int64_t a0 = first_asm[blockIdx.x];
    for (int cl = 0, a = 0; cl < f; cl += 32, a++) {
        body_assemble(P, V, fronts, s, cl, min(cl + 32, f), ainfo[a0 + a], acr, pool);
        __syncthreads();
    }
    double *ws = pws + (int64_t)slots[blockIdx.x] * kPanelWs;
    body_diag(P, V, fronts, Dg, Dig, dyng, ctl, s, 0, nb, ws, pool);
    __syncthreads();
    // (one row per warp: the light variant keeps three CTAs per SM; these
    // fronts' solves are short, k <= 32 columns)
    for (int r0 = k; r0 < f; r0 += kTrsmRows) {
        body_trsm<1>(P, fronts, s, r0, min(r0 + kTrsmRows, f), 0, nb, ws, pool);
        __syncthreads();
    }
    for (int j0 = k; j0 < f; j0 += kUpdTile)
        for (int i0 = j0; i0 < f; i0 += kUpdTile) {
            body_tile(P, fronts, Dg, s, i0, j0, 0, nb, pool);
            __syncthreads();
        }
}

// Persistent level kernel: all large-front items of one tree level in one
// launch.  CTAs take tickets in the host's order, wait (thread 0, bounded
// spin on acquire loads) until the item's counters reach their thresholds,
// run the item's body, and add the item's increment to its completion
// counter (release: every thread fences its writes before the barrier).
// Every item waits only on items with smaller tickets, which were taken by
// running CTAs, so the launch completes whatever the grid size.  A wait
// that runs out sets kStatTimeout and the item proceeds (its results are
// then wrong, but the launch still ends).
__device__ __forceinline__ int ld_acquire_i32(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Once some wait of the launch has given up, the others stop at their next
// check of the status word, so a failed launch ends after one wait limit.
__device__ __forceinline__ void wait_counter(const int32_t *cnt, int need, DevCtl *ctl, long long limit) {
    long long spins = 0;
    while (ld_acquire_i32(cnt) < need) {
        if (++spins > limit) {
            atomicOr(&ctl->status, kStatTimeout);
            break;
        }
        if ((spins & 1023) == 0 && (*(volatile int32_t *)&ctl->status & kStatTimeout)) break;
        __nanosleep(64);
    }
}

__global__ void __launch_bounds__(kBodyThreads) k_large_level(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                               double *__restrict__ Dg, double *__restrict__ Dig,
                                                               double *__restrict__ dyng, DevCtl *ctl,
                                                               const FactorItem *__restrict__ items, int nitems,
                                                               int32_t *sync, const AsmItem *__restrict__ ainfo,
                                                               const int32_t *__restrict__ acr,
                                                               double *__restrict__ pws, int nb, long long limit) {
    __shared__ double pool[kPoolDoubles];
    __shared__ FactorItem sh_it;
    int32_t *cnt = sync + 1;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const int t = atomicAdd(sync, 1);
            FactorItem a;
            a.kind = -1;
            if (t < nitems) a = items[t];
            sh_it = a;
        }
        __syncthreads();
        const FactorItem it = sh_it;
        __syncthreads();
        if (it.kind < 0) break;
        if (tid == 0) {
            if (it.wait0 >= 0) wait_counter(cnt + it.wait0, it.need0, ctl, limit);
            if (it.wait1 >= 0) wait_counter(cnt + it.wait1, it.need1, ctl, limit);
        }
        __syncthreads();
        switch (it.kind) {
            case kItemAssemble: body_assemble(P, V, fronts, it.s, it.a, it.b, ainfo[it.aux], acr, pool); break;
            case kItemDiag:
                body_diag(P, V, fronts, Dg, Dig, dyng, ctl, it.s, it.t * nb, nb, pws + (int64_t)it.aux * kPanelWs,
                          pool);
                break;
            case kItemTrsm:
                body_trsm<1>(P, fronts, it.s, it.a, it.b, it.t * nb, nb, pws + (int64_t)it.aux * kPanelWs, pool);
                break;
            case kItemStrip: body_strip(P, fronts, Dg, it.s, it.a, it.b, it.t * nb, nb, pool); break;
            default: body_tile(P, fronts, Dg, it.s, it.a, it.b, it.t * nb, nb, pool); break;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0 && it.sig >= 0) atomicAdd(cnt + it.sig, it.add);
    }
}

// ||K||_1 of the regularised augmented matrix (maximum absolute row sum of
// the symmetric matrix, fixed summation order per row); also checks that
// Theta is positive and finite.
// |K_pi| of stored entry p of column i (with the static terms)
__device__ __forceinline__ double kabs(const DevPlan &P, const DevVals &V, int i, int64_t p, bool &bad) {
    const int64_t src = P.ksrc[p];
    double val;
    if (P.form == 2) val = V.nev[src] + (P.kj[p] == i ? V.delta : 0.0);
    else if (src >= 0) val = V.Ax[src];
    else if (src == kDualDiag) val = V.delta;
    else {
        const double th = V.theta[-1 - src];
        if (!(th > 0.0) || !isfinite(th)) bad = true;
        val = 1.0 / th + V.rho;
    }
    return fabs(val);
}

// ||K||_1: column sums in entry order, one thread per column; columns longer
// than kLongColumn are left to k_norm1_long (a thread alone on a dense row of
// A would take milliseconds)
__global__ void k_norm1(DevPlan P, DevVals V, DevCtl *ctl) {
    double mx = 0.0;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
        if (P.kp[i + 1] - P.kp[i] > kLongColumn) continue;
        double sum = 0.0;
        for (int64_t p = P.kp[i]; p < P.kp[i + 1]; p++) sum += kabs(P, V, i, p, bad);
        mx = fmax(mx, sum);
        if (P.inst) atomicMax((unsigned long long *)&P.inst_norm1[P.inst[i]], (unsigned long long)__double_as_longlong(sum));
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&ctl->norm1, (unsigned long long)__double_as_longlong(mx));
    if (bad) atomicOr(&ctl->status, kStatNonFinite);
}

// One long column per CTA: thread t sums the t-th of 256 contiguous runs in
// entry order, then the runs' sums are added pairwise in a fixed tree (a
// deterministic order, not the sequential one).
__global__ void __launch_bounds__(256) k_norm1_long(DevPlan P, DevVals V, DevCtl *ctl) {
    __shared__ double part[256];
    const int i = P.long_cols[blockIdx.x];
    const int64_t p0 = P.kp[i], n = P.kp[i + 1] - p0;
    const int64_t run = (n + 255) / 256;
    const int64_t a = p0 + run * threadIdx.x, b = min(a + run, p0 + n);
    bool bad = false;
    double sum = 0.0;
    for (int64_t p = a; p < b; p++) sum += kabs(P, V, i, p, bad);
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax((unsigned long long *)&ctl->norm1, (unsigned long long)__double_as_longlong(part[0]));
        if (P.inst)
            atomicMax((unsigned long long *)&P.inst_norm1[P.inst[i]], (unsigned long long)__double_as_longlong(part[0]));
    }
    if (bad) atomicOr(&ctl->status, kStatNonFinite);
}

__global__ void k_set_b1(DevPlan P, DevCtl *ctl, double eps_piv) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->b1 = eps_piv * ctl->norm1;
    if (P.inst)
        for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.batch_count; b += gridDim.x * blockDim.x)
            P.inst_b1[b] = eps_piv * P.inst_norm1[b];
}

// Statistics of the factorisation: inertia, number and size of lifts.
__global__ void k_factor_stats(const double *__restrict__ D, const double *__restrict__ dyn, int N, double large_reg,
                               DevCtl *ctl) {
    int npos = 0, nneg = 0, ndyn = 0;
    double mx = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const double d = D[j];
        npos += d > 0.0;
        nneg += d < 0.0;
        const double a = fabs(dyn[j]);
        ndyn += a != 0.0;
        mx = fmax(mx, a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        npos += __shfl_xor_sync(0xffffffffu, npos, o);
        nneg += __shfl_xor_sync(0xffffffffu, nneg, o);
        ndyn += __shfl_xor_sync(0xffffffffu, ndyn, o);
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ctl->npos, npos);
        atomicAdd(&ctl->nneg, nneg);
        atomicAdd(&ctl->ndyn, ndyn);
        atomicMax((unsigned long long *)&ctl->max_dyn, (unsigned long long)__double_as_longlong(mx));
        if (ndyn) atomicOr(&ctl->status, kStatDynReg);
        if (mx > large_reg) atomicOr(&ctl->status, kStatLargeReg);
    }
}

// ---------------------------------------------------------------------------
// Pivoting of Sec. 4.5 (the Bunch-Kaufman variation) for matrices that are not
// quasi-definite: one CTA per front assembles it (original entries, then the
// children's contribution blocks in ascending order), adds the static terms
// to its fully-summed diagonal and factorises its k fully-summed columns in
// pivot blocks of nb columns, with 1x1 and 2x2 pivots chosen inside the
// block: pre-swap of the largest remaining block diagonal, gamma_p = the
// largest magnitude below the pivot in the block (row r), a lift of the pivot
// to sign(M_pp) eps_piv ||K||_1 when max(|M_pp|, gamma_p) is not above it,
// else a 1x1 pivot at p when |M_pp| >= alpha gamma_p or
// |M_pp| gamma_r >= alpha gamma_p^2, a 1x1 pivot at r when
// |M_rr| >= alpha gamma_r, otherwise the 2x2 pivot (p, r).  Interchanges stay
// among the fully-summed columns, so the structure of the front is unchanged;
// every pivot updates the whole trailing part of the front (the contribution
// block included).  Each product and sum is rounded as written (no fused
// multiply-add), so the arithmetic is that of a plain evaluation of the rule.
// The front lives in its slab (lower triangle); a symmetric interchange of
// positions a < b moves entries of the lower triangle only.
constexpr int kBkThreads = 256;

__device__ void bk_swap(double *F, int ld, int f, int a, int b, int32_t *lperm) {
    if (a == b) return;
#define FE(i, j) F[(int64_t)(j) * ld + (i)]
    for (int i = threadIdx.x; i < f; i += kBkThreads) {
        if (i < a) {
            const double t = FE(a, i);
            FE(a, i) = FE(b, i);
            FE(b, i) = t;
        } else if (i == a) {
            const double t = FE(a, a);
            FE(a, a) = FE(b, b);
            FE(b, b) = t;
        } else if (i < b) {
            const double t = FE(i, a);
            FE(i, a) = FE(b, i);
            FE(b, i) = t;
        } else if (i > b) {
            const double t = FE(i, a);
            FE(i, a) = FE(i, b);
            FE(i, b) = t;
        }
    }
    if (threadIdx.x == 0) {
        const int32_t t = lperm[a];
        lperm[a] = lperm[b];
        lperm[b] = t;
    }
#undef FE
}

// argmax over lanes of v (first index on ties, -1 when every v is 0 and zero_is_none)
__device__ __forceinline__ int warp_argmax_first(double v, int idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    return idx;
}

__global__ void __launch_bounds__(kBkThreads) k_front_bk(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                         double *__restrict__ D, double *__restrict__ Doff,
                                                         int32_t *__restrict__ bsz, int32_t *__restrict__ lperm,
                                                         double *__restrict__ dyn, DevCtl *ctl,
                                                         const int32_t *__restrict__ list, int nb, double alpha) {
    __shared__ int sh_q, sh_two, sh_swap_a, sh_swap_b;
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#define FE(i, j) F[(int64_t)(j) * ld + (i)]
    // assembly, in the order of the plain multifrontal method
    for (int64_t t = tid; t < (int64_t)f * ld; t += kBkThreads) F[t] = 0.0;
    __syncthreads();
    for (int64_t q = P.orig_ptr[s] + tid; q < P.orig_ptr[s + 1]; q += kBkThreads)
        F[P.orig_dst[q]] = orig_value(P, V, P.orig_src[q]);
    __syncthreads();
    for (int q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
        const int c = P.child_list[q];
        const int kc = P.sn_k[c], ldc = P.sn_ld[c], cc = P.sn_f[c] - kc;
        const double *CB = fronts + P.sn_off[c] + (int64_t)kc * ldc + kc;
        const int32_t *map = P.relmap + P.map_off[c];
        for (int jj = warp; jj < cc; jj += kBkThreads / 32)
            for (int ii = jj + lane; ii < cc; ii += 32)
                F[(int64_t)map[jj] * ld + map[ii]] += CB[(int64_t)jj * ldc + ii];
        __syncthreads();
    }
    // static terms on the fully-summed diagonal; interchanges start from the identity
    for (int t = tid; t < k; t += kBkThreads) {
        const int sg = P.sign[c0 + t];
        const double sigma = sg < 0 ? V.rho : V.delta;
        FE(t, t) = __dadd_rn(FE(t, t), (double)sg * sigma);
        lperm[c0 + t] = t;
        Doff[c0 + t] = 0.0;
        dyn[c0 + t] = 0.0;
    }
    __syncthreads();
    const double b1 = ctl->b1;
    int32_t *lp = lperm + c0;
    for (int b0 = 0; b0 < k; b0 += nb) {
        const int b1c = min(b0 + nb, k);
        int p = b0;
        while (p < b1c) {
            // pre-swap: the largest remaining block diagonal to position p
            if (warp == 0) {
                const int t = p + lane;
                const double v = t < b1c ? fabs(FE(t, t)) : -1.0;
                const int q = warp_argmax_first(v, t < b1c ? t : 0x7fffffff);
                if (lane == 0) sh_q = q;
            }
            __syncthreads();
            bk_swap(F, ld, f, p, sh_q, lp);
            __syncthreads();
            // gamma_p and r within the block; the pivot decision
            if (warp == 0) {
                const int i = p + 1 + lane;
                const double v = i < b1c ? fabs(FE(i, p)) : -1.0;
                const int r0 = warp_argmax_first(v, i < b1c ? i : 0x7fffffff);
                const double gp_all = __shfl_sync(0xffffffffu, v, (r0 - p - 1) & 31);
                if (lane == 0) {
                    const double gp = (r0 < b1c && gp_all > 0.0) ? gp_all : 0.0;
                    const int r = gp > 0.0 ? r0 : -1;
                    const double app = FE(p, p);
                    int two = 0, sa = -1, sb = -1;
                    if ((fabs(app) > gp ? fabs(app) : gp) <= b1) {
                        const double dn = app < 0.0 ? -b1 : b1;
                        dyn[c0 + p] = __dsub_rn(dn, app);
                        FE(p, p) = dn;
                    } else if (fabs(app) < __dmul_rn(alpha, gp)) {
                        double gr = 0.0;
                        for (int t = p; t < b1c; t++) {
                            if (t == r) continue;
                            const double a = t < r ? fabs(FE(r, t)) : fabs(FE(t, r));
                            if (a > gr) gr = a;
                        }
                        if (__dmul_rn(fabs(app), gr) >= __dmul_rn(__dmul_rn(alpha, gp), gp)) {
                            // 1x1 at p
                        } else if (fabs(FE(r, r)) >= __dmul_rn(alpha, gr)) {
                            sa = p;
                            sb = r;
                        } else {
                            sa = p + 1;
                            sb = r;
                            two = 1;
                        }
                    }
                    sh_two = two;
                    sh_swap_a = sa;
                    sh_swap_b = sb;
                }
            }
            __syncthreads();
            if (sh_swap_a >= 0) {
                bk_swap(F, ld, f, sh_swap_a, sh_swap_b, lp);
                __syncthreads();
            }
            if (!sh_two) {
                const double d = FE(p, p);
                if (tid == 0) {
                    D[c0 + p] = d;
                    bsz[c0 + p] = 1;
                    if (!isfinite(d) || d == 0.0) atomicOr(&ctl->status, kStatNonFinite);
                }
                for (int i = p + 1 + tid; i < f; i += kBkThreads) FE(i, p) = __ddiv_rn(FE(i, p), d);
                __syncthreads();
                for (int j = p + 1 + warp; j < f; j += kBkThreads / 32) {
                    const double ljp = FE(j, p);
                    for (int i = j + lane; i < f; i += 32)
                        FE(i, j) = __dsub_rn(FE(i, j), __dmul_rn(__dmul_rn(FE(i, p), d), ljp));
                }
                __syncthreads();
                p += 1;
            } else {
                const double e11 = FE(p, p), e21 = FE(p + 1, p), e22 = FE(p + 1, p + 1);
                const double det = __dsub_rn(__dmul_rn(e11, e22), __dmul_rn(e21, e21));
                if (tid == 0) {
                    D[c0 + p] = e11;
                    D[c0 + p + 1] = e22;
                    Doff[c0 + p] = e21;
                    bsz[c0 + p] = 2;
                    bsz[c0 + p + 1] = 0;
                    if (!isfinite(det) || det == 0.0) atomicOr(&ctl->status, kStatNonFinite);
                }
                for (int i = p + 2 + tid; i < f; i += kBkThreads) {
                    const double x = FE(i, p), y = FE(i, p + 1);
                    FE(i, p) = __ddiv_rn(__dsub_rn(__dmul_rn(x, e22), __dmul_rn(y, e21)), det);
                    FE(i, p + 1) = __ddiv_rn(__dsub_rn(__dmul_rn(y, e11), __dmul_rn(x, e21)), det);
                }
                __syncthreads();
                for (int j = p + 2 + warp; j < f; j += kBkThreads / 32) {
                    const double l0 = FE(j, p), l1 = FE(j, p + 1);
                    const double w0 = __dadd_rn(__dmul_rn(e11, l0), __dmul_rn(e21, l1));
                    const double w1 = __dadd_rn(__dmul_rn(e21, l0), __dmul_rn(e22, l1));
                    for (int i = j + lane; i < f; i += 32)
                        FE(i, j) = __dsub_rn(FE(i, j), __dadd_rn(__dmul_rn(FE(i, p), w0), __dmul_rn(FE(i, p + 1), w1)));
                }
                __syncthreads();
                if (tid == 0) FE(p + 1, p) = 0.0;  // L is unit lower triangular: the 2x2 block lives in D
                __syncthreads();
                p += 2;
            }
        }
    }
#undef FE
}

// Inertia and lift statistics of a factorisation with 1x1 and 2x2 blocks: a
// 2x2 block holds one positive and one negative eigenvalue when its
// determinant is negative, else two of the sign of its trace.
__global__ void k_factor_stats_bk(const double *__restrict__ D, const double *__restrict__ Doff,
                                  const int32_t *__restrict__ bsz, const double *__restrict__ dyn, int N,
                                  double large_reg, DevCtl *ctl) {
    int npos = 0, nneg = 0, ndyn = 0;
    double mx = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const double a = fabs(dyn[j]);
        ndyn += a != 0.0;
        mx = fmax(mx, a);
        if (bsz[j] == 2) {
            const double det = __dsub_rn(__dmul_rn(D[j], D[j + 1]), __dmul_rn(Doff[j], Doff[j]));
            if (det < 0.0) {
                npos++;
                nneg++;
            } else if (det > 0.0) {
                if (__dadd_rn(D[j], D[j + 1]) > 0.0) npos += 2;
                else nneg += 2;
            }
        } else if (bsz[j] == 1) {
            npos += D[j] > 0.0;
            nneg += D[j] < 0.0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        npos += __shfl_xor_sync(0xffffffffu, npos, o);
        nneg += __shfl_xor_sync(0xffffffffu, nneg, o);
        ndyn += __shfl_xor_sync(0xffffffffu, ndyn, o);
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ctl->npos, npos);
        atomicAdd(&ctl->nneg, nneg);
        atomicAdd(&ctl->ndyn, ndyn);
        atomicMax((unsigned long long *)&ctl->max_dyn, (unsigned long long)__double_as_longlong(mx));
        if (ndyn) atomicOr(&ctl->status, kStatDynReg);
        if (mx > large_reg) atomicOr(&ctl->status, kStatLargeReg);
    }
}

}  // namespace

void launch_small_fronts(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Dinv, double *dyn,
                         DevCtl *ctl, const int32_t *list, int32_t count, int32_t nb, int32_t maxf, int32_t threads,
                         cudaStream_t st) {
    if (count <= 0) return;
    const int ldmax = (maxf + 3) & ~3;
    const size_t smem = (size_t)ldmax * maxf * sizeof(double);
    static uint64_t attr = 0;
    if (first_on_device(attr)) {
        cudaFuncSetAttribute(k_small_fronts<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_small_fronts<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_small_fronts<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_small_fronts<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    // default: one warp per front up to f = 32, two up to 64, four beyond;
    // the autotuner may choose any of 32, 64, 128, 256 (same arithmetic per
    // entry whatever the width)
    if (threads <= 0) threads = maxf <= 32 ? 32 : maxf <= 64 ? 64 : 128;
    switch (threads) {
        case 32: k_small_fronts<32><<<count, 32, smem, st>>>(P, V, fronts, D, Dinv, dyn, ctl, list, nb); break;
        case 64: k_small_fronts<64><<<count, 64, smem, st>>>(P, V, fronts, D, Dinv, dyn, ctl, list, nb); break;
        case 256: k_small_fronts<256><<<count, 256, smem, st>>>(P, V, fronts, D, Dinv, dyn, ctl, list, nb); break;
        default: k_small_fronts<128><<<count, 128, smem, st>>>(P, V, fronts, D, Dinv, dyn, ctl, list, nb); break;
    }
}

void launch_large_assemble(const DevPlan &P, const DevVals &V, double *fronts, const PanelItem *items,
                           const AsmItem *ainfo, const int32_t *acr, int32_t count, cudaStream_t st) {
    if (count <= 0) return;
    k_large_assemble<<<count, kBodyThreads, 0, st>>>(P, V, fronts, items, ainfo, acr);
}

void launch_panel_diag(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Dinv, double *dyn,
                       DevCtl *ctl,
                       const PanelItem *items, int32_t count, int32_t nb, double *pws, cudaStream_t st) {
    if (count <= 0) return;
    k_panel_diag<<<count, kBodyThreads, 0, st>>>(P, V, fronts, D, Dinv, dyn, ctl, items, nb, pws);
}

void launch_panel_trsm(const DevPlan &P, double *fronts, const PanelItem *items, const int32_t *slots, int32_t count,
                       int32_t nb, const double *pws, cudaStream_t st, const int32_t *sbase,
                       uint8_t *sws, int32_t *sexp, const double *D, DevCtl *ctl) {
    if (count <= 0) return;
    k_panel_trsm<<<count, kBodyThreads, 0, st>>>(P, fronts, items, slots, nb, pws, sbase, sws, sexp, D, ctl);
}

void launch_large_update(const DevPlan &P, double *fronts, const double *D, const TileItem *items, int32_t count,
                         int32_t w, cudaStream_t st) {
    if (count <= 0) return;
    k_large_update<<<count, kBodyThreads, 0, st>>>(P, fronts, D, items, w);
}

void launch_large_update_strip(const DevPlan &P, double *fronts, const double *D, const TileItem *items,
                               int32_t count, int32_t w, cudaStream_t st) {
    if (count <= 0) return;
    k_large_update_strip<<<count, kBodyThreads, 0, st>>>(P, fronts, D, items, w);
}

void launch_thin_fronts(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Dinv, double *dyn,
                        DevCtl *ctl, const int32_t *list, const int32_t *first_asm, const int32_t *slots,
                        const AsmItem *ainfo, const int32_t *acr, double *pws, int32_t count, int32_t nb,
                        cudaStream_t st) {
    if (count <= 0) return;
    k_thin_fronts<<<count, kBodyThreads, 0, st>>>(P, V, fronts, D, Dinv, dyn, ctl, list, first_asm, slots, ainfo, acr,
                                                   pws, nb);
}

void launch_large_level(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Dinv, double *dyn,
                        DevCtl *ctl, const FactorItem *items, int32_t count, int32_t *sync, int32_t ncounters,
                        const AsmItem *ainfo, const int32_t *acr, double *pws, int32_t nb, int32_t grid,
                        long long spin_limit, cudaStream_t st) {
    if (count <= 0) return;
    cudaMemsetAsync(sync, 0, sizeof(int32_t) * (size_t)(ncounters + 1), st);
    k_large_level<<<grid < count ? grid : count, kBodyThreads, 0, st>>>(P, V, fronts, D, Dinv, dyn, ctl, items, count,
                                                                        sync, ainfo, acr, pws, nb, spin_limit);
}

const void *large_level_kernel() { return reinterpret_cast<const void *>(k_large_level); }

// The pivot reciprocal of the factorisation beside CUDA's correctly rounded
// division, element by element (a test hook: the factorisation scales every
// column of L by this reciprocal, Sec. 4.4-4.5).
__global__ void k_test_recip(const double *__restrict__ x, double *__restrict__ rcp, double *__restrict__ quo,
                             int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        rcp[i] = recip_pivot(v);
        quo[i] = 1.0 / v;
    }
}

void launch_front_bk(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *Doff, int32_t *bsz,
                     int32_t *lperm, double *dyn, DevCtl *ctl, const int32_t *list, int32_t count, int32_t nb,
                     cudaStream_t st) {
    if (count <= 0) return;
    k_front_bk<<<count, kBkThreads, 0, st>>>(P, V, fronts, D, Doff, bsz, lperm, dyn, ctl, list, nb,
                                            0.125 + 0.125 * sqrt(17.0));
}

void launch_factor_stats_bk(const double *D, const double *Doff, const int32_t *bsz, const double *dyn, int N,
                            double large_reg, DevCtl *ctl, cudaStream_t st) {
    k_factor_stats_bk<<<152, 256, 0, st>>>(D, Doff, bsz, dyn, N, large_reg, ctl);
}

void launch_test_recip(const double *x, double *rcp, double *quo, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t blocks = (n + 255) / 256;
    k_test_recip<<<(int)(blocks < 1216 ? blocks : 1216), 256, 0, st>>>(x, rcp, quo, n);
}

void launch_norm1(const DevPlan &P, const DevVals &V, DevCtl *ctl, double eps_piv, cudaStream_t st) {
    const int grid = (P.N + 255) / 256 < 608 ? (P.N + 255) / 256 : 608;
    if (P.inst) cudaMemsetAsync(P.inst_norm1, 0, sizeof(double) * P.batch_count, st);
    k_norm1<<<grid > 0 ? grid : 1, 256, 0, st>>>(P, V, ctl);
    if (P.nlong > 0) k_norm1_long<<<P.nlong, 256, 0, st>>>(P, V, ctl);
    k_set_b1<<<P.inst ? (P.batch_count + 255) / 256 : 1, 256, 0, st>>>(P, ctl, eps_piv);
}

void launch_factor_stats(const double *D, const double *dyn, int N, double large_reg, DevCtl *ctl, cudaStream_t st) {
    k_factor_stats<<<152, 256, 0, st>>>(D, dyn, N, large_reg, ctl);
}

}  // namespace ipm
