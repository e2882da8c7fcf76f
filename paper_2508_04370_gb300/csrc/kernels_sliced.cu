// FP64-accurate Schur-complement updates of large fronts on the bf16 tensor
// cores (the dgemm updates of Sec. 4.4, with FP64 pivots, regularisation and
// refinement unchanged).
//
// The regularised augmented systems of an IPM grow by about 1/delta when a
// dual row is eliminated with a pivot of size delta (and by more at wide
// Theta spreads), so FP32-accurate updates leave errors that refinement
// cannot remove.  These kernels keep the product accurate to about 2^-54 of
// the largest operand entry of each row, like an FP64 product, by exact
// integer arithmetic on the tensor cores (the splitting idea of Ozaki et
// al.):
//
//  1. k_slice_panel: after a 32-column panel [p0, p1), every trailing row r
//     of the two panel operands a_rq = L(r, q) 2^h_q and
//     b_rq = L(r, q) d_q 2^-h_q (h_q = floor(log2 |d_q| / 2): an exact
//     balancing of each column, so that a_rq^2 and b_rq^2 are both within a
//     factor 4 of L(r, q)^2 |d_q|, whatever the spread of the pivots) gets a
//     power-of-two scale 2^E_r with |entries| < 2^E_r and is rounded to the
//     56-bit integers X_rq = rint(a_rq 2^(56 - E_r)), written as eight
//     balanced base-2^7 digits X = sum_t x_t 2^(7 (7 - t)), |x_t| <= 64
//     (|x_0| <= 128), each exactly a bf16.  The digits go to a work space in
//     the 128-byte-swizzled K-major image the tensor cores read.
//  2. k_update_sliced: one CTA per 128 x 32 output tile; the digit images
//     arrive by bulk copies (TMA), one thread issues the 36 digit products
//     with t + u <= 7 (72 tcgen05.mma.kind::f16, K = 16) into eight TMEM
//     accumulators S_d, d = t + u.  Digit products are at most 2^14 and a
//     panel has at most 32 columns, so every S_d is an integer below 2^22
//     and FP32 accumulation is exact.  The epilogue forms
//     hi = sum_{d<4} S_d 2^(7 (3 - d)) and lo = sum_{d>=4} S_d 2^(7 (7 - d))
//     exactly in integers, the product
//     sum_q a_iq b_jq ~= 2^(E_i + E_j - 63) (hi 2^28 + lo)
//     as a double built from the integer's bits (one rounding), and
//     subtracts it from the FP64 entry: one FP64 instruction per entry.
// Error per entry: operand rounding 2^-57 and the dropped digit products
// (t + u >= 8) below 2^-55, relative to 2^(E_i + E_j) per column of the
// panel, that is about 2^-52 sqrt(max_q L_iq^2 |d_q| max_q L_jq^2 |d_q|);
// FP64 GEMM's is 2^-53 of each |L_iq d_q L_jq|, summed.  Without the
// balancing a panel mixing pivots of size delta and of size 1/delta pairs
// the largest a of one column with the largest b of another, and the
// factorisation of a matrix with that much growth diverges.
#include <cuda_runtime.h>

#include <cstdint>

#include "ipm_dev.h"
#include "tc_common.cuh"

namespace ipm {

namespace {

constexpr long long kSlicePolls = 1ll << 24;  // bounded waits on copies and MMAs (~1 s)
constexpr int kNoScale = -1100;                // row scale of an all-zero row: every digit is 0

// Byte offset of the 16-byte chunk c (0..7) of row r in a 128-byte-swizzled
// K-major image (eight rows form a 1024-byte atom).
__device__ __forceinline__ uint32_t swz_chunk(int r, int c) {
    return (uint32_t)r * 128u + ((((uint32_t)c) ^ ((uint32_t)r & 7u)) << 4);
}

// Biased exponent field of a double given as bits.
__device__ __forceinline__ int biased_exp(long long b) { return (int)((b >> 52) & 0x7ff); }

// rint(v 2^h 2^(56 - E)) for |v 2^h| < 2^E, from the bits of v (subnormal
// v give 0).
__device__ __forceinline__ long long fixed56(double v, int h, int E) {
    const long long b = __double_as_longlong(v);
    const int eb = biased_exp(b);
    if (eb == 0 || eb == 0x7ff) return 0;
    const long long m = (b & 0x000fffffffffffffll) | 0x0010000000000000ll;
    // v 2^h = m 2^(eb + h - 1075); sh <= 3 because eb + h <= E + 1022
    const int sh = eb + h - 1019 - E;
    long long x;
    if (sh >= 0) x = m << sh;
    else if (sh >= -62) x = (m + (1ll << (-sh - 1))) >> (-sh);
    else x = 0;
    return b < 0 ? -x : x;
}

// Eight balanced base-2^7 digits of x (|x| <= 2^56): x = sum_t d[t] 2^(7 (7 - t)).
// In 32-bit arithmetic: the low 28 bits give digits 7..4 and a carry of 0 or
// 1 into the high part, which gives digits 3..0.
__device__ __forceinline__ void digits8(long long x, int *d) {
    int lo = (int)(x & 0x0fffffff);
    int hi = (int)(x >> 28);
#pragma unroll
    for (int t = 7; t >= 4; t--) {
        const int dg = ((lo + 64) & 127) - 64;
        d[t] = dg;
        lo = (lo - dg) >> 7;
    }
    hi += lo;
#pragma unroll
    for (int t = 3; t >= 1; t--) {
        const int dg = ((hi + 64) & 127) - 64;
        d[t] = dg;
        hi = (hi - dg) >> 7;
    }
    d[0] = hi;
}

__device__ __forceinline__ uint32_t bf16_bits(int v) {
    // every |v| <= 256 is exact in bf16: the high half of the float
    return __float_as_uint((float)v) >> 16;
}

// One 128-row slice block per CTA: thread (r, op) takes row r of operand op
// (op 0: a_rq = L(r, q) 2^h_q, op 1: b_rq = L(r, q) d_q 2^-h_q) and writes its
// digit images and row scale.
__global__ void __launch_bounds__(256) k_slice_panel(DevPlan P, const double *__restrict__ fronts,
                                                     const double *__restrict__ Dg,
                                                     const SliceItem *__restrict__ items, int p0, int w,
                                                     uint8_t *__restrict__ ws, int32_t *__restrict__ ws_exp,
                                                     DevCtl *ctl) {
    const SliceItem it = items[blockIdx.x];
    const int s = it.s;
    const int f = P.sn_f[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    w = min(w, P.sn_k[s] - p0);
    const double *F = fronts + P.sn_off[s];
    const int r = threadIdx.x, op = threadIdx.y;
    const int row = it.r0 + r;
    const bool valid = row < f;
    double v[kSliceCols];
    int sh[kSliceCols];
    // largest biased exponent of a nonzero normal entry after the column
    // shifts; kNoExp: none
    constexpr int kNoExp = -100000;
    int emax = kNoExp;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < kSliceCols; q++) {
        const double dq = q < w ? Dg[c0 + p0 + q] : 0.0;
        const int ed = biased_exp(__double_as_longlong(dq));
        const int h = ed == 0 ? 0 : ((ed - 1023) >> 1);  // floor(log2 |d_q| / 2)
        const double l = (valid && q < w) ? F[(int64_t)(p0 + q) * ld + row] : 0.0;
        v[q] = op == 0 ? l : l * dq;
        sh[q] = op == 0 ? h : -h;
        const int e = biased_exp(__double_as_longlong(v[q]));
        bad |= e == 0x7ff;
        if (e != 0) emax = max(emax, e + sh[q]);
    }
    if (bad) atomicOr(&ctl->status, kStatNonFinite);
    // |v 2^shift| < 2^E with E = (largest shifted biased exponent) - 1022
    const int E = (emax == kNoExp || bad) ? kNoScale : emax - 1022;
    ws_exp[((int64_t)it.blk * kSliceRows + r) * 2 + op] = E;
    uint8_t *img = ws + (int64_t)it.blk * kSliceBlockBytes + op * kSliceOperandBytes;
#pragma unroll
    for (int qg = 0; qg < kSliceCols / 8; qg++) {
        // 8 columns x 8 slices: one 16-byte chunk per slice
        uint32_t pk[kSlices][4];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            int d[kSlices];
            digits8(E == kNoScale ? 0 : fixed56(v[qg * 8 + j], sh[qg * 8 + j], E), d);
#pragma unroll
            for (int t = 0; t < kSlices; t++) {
                const uint32_t hb = bf16_bits(d[t]);
                if (j & 1) pk[t][j >> 1] |= hb << 16;
                else pk[t][j >> 1] = hb;
            }
        }
#pragma unroll
        for (int t = 0; t < kSlices; t++) {
            // slice t sits in pair image t/2, K bytes (t%2)*64 .. +63 of each row
            const int chunk = (t & 1) * 4 + qg;
            uint4 *dst = (uint4 *)(img + (t >> 1) * kSlicePairBytes + swz_chunk(r, chunk));
            *dst = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
        }
    }
}

// t 2^e as a double (round half up to 53 bits), built with integer
// operations; t != 0.  Leaves the normal range only through ldexp.
__device__ __forceinline__ double int_scaled(long long t, int e) {
    const unsigned long long a = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << lz;  // bit 63 set
    unsigned long long mant = (n >> 11) + ((n >> 10) & 1ull);
    int ex = 63 - lz;  // a in [2^ex, 2^(ex + 1))
    if (mant >> 53) {
        mant >>= 1;
        ex++;
    }
    const int field = ex + e + 1023;  // t 2^e = mant 2^(ex - 52 + e)
    if (field <= 0 || field >= 2047) return ldexp((double)t, e);
    return __longlong_as_double((long long)(((unsigned long long)(t < 0) << 63) |
                                            ((unsigned long long)field << 52) | (mant & 0x000fffffffffffffull)));
}

// Exact integer value of an FP32 accumulator holding an integer below 2^22.
__device__ __forceinline__ int acc_int(uint32_t bits) {
    return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}

constexpr int kSlicedSmem = 4 * (int)kSlicePairBytes + 4 * 4096 + 1024;  // A (128 rows), B (32 rows), alignment

// One CTA (8 warps) per 128 x 32 output tile of the lower trailing part:
//     C(i, j) -= sum_q L(i, q) d_q L(j, q),   i >= j,  over the panel's columns q.
// Warps w and w + 4 read the same 32 TMEM lanes (rows) and split the tile's
// columns, 16 each, so the epilogue runs on twice the threads.
constexpr int kSlicedThreads = 256;
__global__ void __launch_bounds__(kSlicedThreads, 2) k_update_sliced(DevPlan P, double *__restrict__ fronts,
                                                       const SlicedTile *__restrict__ items,
                                                       const uint8_t *__restrict__ ws,
                                                       const int32_t *__restrict__ ws_exp, DevCtl *ctl) {
    extern __shared__ uint8_t sl_raw[];
    uint8_t *A = (uint8_t *)(((uintptr_t)sl_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *B = A + 4 * kSlicePairBytes;
    __shared__ uint64_t bar_load, bar_mma;
    __shared__ uint32_t tbase;
    __shared__ int32_t eb_col[kSliceCols];
    const SlicedTile it = items[blockIdx.x];
    const int s = it.s;
    const int f = P.sn_f[s], ld = P.sn_ld[s];
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&tbase, 256);  // 8 accumulators x 32 columns
    if (tid == 0) {
        tc::mbar_init(&bar_load, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
    }
    if (tid < kSliceCols) eb_col[tid] = ws_exp[((int64_t)it.blk_b * kSliceRows + it.roff_b + tid) * 2 + 1];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tbase;
    const uint8_t *srcA = ws + (int64_t)it.blk_a * kSliceBlockBytes;
    const uint8_t *srcB = ws + (int64_t)it.blk_b * kSliceBlockBytes + kSliceOperandBytes;
    if (tid == 0) {
        tc::mbar_expect_tx(&bar_load, (uint32_t)(4 * kSlicePairBytes + 4 * 4096));
        tc::bulk_g2s(A, srcA, (uint32_t)(4 * kSlicePairBytes), &bar_load);
#pragma unroll
        for (int pr = 0; pr < 4; pr++)
            tc::bulk_g2s(B + pr * 4096, srcB + pr * kSlicePairBytes + it.roff_b * 128, 4096, &bar_load);
    }
    bool ok = tc::mbar_wait(&bar_load, 0, kSlicePolls);
    if (!ok) {
        if (lane == 0) atomicOr(&ctl->status, kStatTimeout);
        tc::mbar_wait(&bar_load, 0, kSlicePolls);  // let the copies in flight land before the CTA exits
    }
    if (ok && tid == 0) {
        tc::fence_after_sync();
        constexpr uint32_t id = tc::idesc_bf16(kSliceRows, kSliceCols);
        const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
#pragma unroll
        for (int d = 0; d < kSlices; d++)
#pragma unroll
            for (int t = 0; t <= d; t++) {
                const int u = d - t;
#pragma unroll
                for (int kk = 0; kk < 2; kk++) {
                    const uint64_t ad = tc::smem_desc(a0 + (t >> 1) * (uint32_t)kSlicePairBytes + (t & 1) * 64 + kk * 32);
                    const uint64_t bd = tc::smem_desc(b0 + (u >> 1) * 4096u + (u & 1) * 64 + kk * 32);
                    tc::mma_bf16(tmem + (uint32_t)(d * kSliceCols), ad, bd, id, (t > 0 || kk > 0) ? 1u : 0u);
                }
            }
        tc::commit_to(&bar_mma);
    }
    // the tile's FP64 entries of this thread's row and column half, fetched
    // while the copies and the MMAs run (independent loads; lower part only)
    constexpr int kHalf = kSliceCols / 2;
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane;
    const int row = it.i0 + r;
    const int cbase = half * kHalf;
    double cv[kHalf];
    uint32_t live = 0;  // bit c: entry (row, j0 + cbase + c) exists and is updated
#pragma unroll
    for (int c = 0; c < kHalf; c++) {
        const int col = it.j0 + cbase + c;
        const bool v = row < f && col < f && row >= col;
        live |= (uint32_t)v << c;
        cv[c] = v ? F[(int64_t)col * ld + row] : 0.0;
    }
    if (ok) {
        ok = tc::mbar_wait(&bar_mma, 0, kSlicePolls);
        if (!ok) {
            if (lane == 0) atomicOr(&ctl->status, kStatTimeout);
            tc::mbar_wait(&bar_mma, 0, kSlicePolls);  // the MMAs must finish before TMEM is freed
        }
    }
    tc::fence_after_sync();
    if (ok) {
        const int Ea = ws_exp[((int64_t)it.blk_a * kSliceRows + r) * 2 + 0];
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
        for (int c8 = 0; c8 < kHalf / 8; c8++) {
            // S_0..S_3 first (hi), then S_4..S_7 (lo), to keep the registers low
            uint32_t v[4][8];
            long long hi[8];
#pragma unroll
            for (int d = 0; d < 4; d++)
                tc::tmem_ld8(lane_base + (uint32_t)(d * kSliceCols + cbase + c8 * 8), v[d]);
            tc::tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 8; c++)
                // hi = S0 2^21 + S1 2^14 + S2 2^7 + S3 (|hi| < 2^41)
                hi[c] = ((long long)(acc_int(v[0][c]) * 128 + acc_int(v[1][c])) << 14) +
                        (acc_int(v[2][c]) * 128 + acc_int(v[3][c]));
#pragma unroll
            for (int d = 0; d < 4; d++)
                tc::tmem_ld8(lane_base + (uint32_t)((d + 4) * kSliceCols + cbase + c8 * 8), v[d]);
            tc::tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const long long lo = ((long long)(acc_int(v[0][c]) * 128 + acc_int(v[1][c])) << 14) +
                                     (acc_int(v[2][c]) * 128 + acc_int(v[3][c]));
                // T = hi 2^28 + lo, kept as T 2^-8 (|.| < 2^61): the bits dropped
                // are far below the truncation of the digit products with t + u >= 8
                const long long tq = (hi[c] << 20) + (lo >> 8);
                if (tq != 0 && ((live >> (c8 * 8 + c)) & 1u))
                    cv[c8 * 8 + c] -= int_scaled(tq, Ea + eb_col[cbase + c8 * 8 + c] - 55);
            }
        }
#pragma unroll
        for (int c = 0; c < kHalf; c++)
            if ((live >> c) & 1u) F[(int64_t)(it.j0 + cbase + c) * ld + row] = cv[c];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace

void launch_slice_panel(const DevPlan &P, const double *fronts, const double *D, const SliceItem *items,
                        int32_t count, int32_t p0, int32_t w, uint8_t *ws, int32_t *ws_exp, DevCtl *ctl,
                        cudaStream_t st) {
    if (count <= 0) return;
    k_slice_panel<<<count, dim3(kSliceRows, 2), 0, st>>>(P, fronts, D, items, p0, w, ws, ws_exp, ctl);
}

void launch_update_sliced(const DevPlan &P, double *fronts, const SlicedTile *items, int32_t count,
                          const uint8_t *ws, const int32_t *ws_exp, DevCtl *ctl, cudaStream_t st) {
    if (count <= 0) return;
    static uint64_t attr = 0;
    if (first_on_device(attr))
        cudaFuncSetAttribute(k_update_sliced, cudaFuncAttributeMaxDynamicSharedMemorySize, kSlicedSmem);
    k_update_sliced<<<count, kSlicedThreads, kSlicedSmem, st>>>(P, fronts, items, ws, ws_exp, ctl);
}

}  // namespace ipm
