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
//  1. slicing, in the panel's triangular solve (k_panel_trsm holds each
//     finished row of L in one warp).  Panels are taken in pairs: after the
//     first panel of a pair only the second panel's 32 columns are updated
//     (one chunk); after the second panel the whole trailing part receives
//     both panels' update at once (two chunks, K = 64), which halves the
//     read-modify-write passes over the trailing part and the epilogue work
//     per panel.  Every trailing row r of the two panel operands
//     a_rq = L(r, q) 2^h_q and b_rq = L(r, q) d_q 2^-h_q over the chunks'
//     columns (h_q = floor(log2 |d_q| / 2): an exact balancing of each
//     column, so that a_rq^2 and b_rq^2 are both within a factor 4 of
//     L(r, q)^2 |d_q|, whatever the spread of the pivots) gets one
//     power-of-two scale 2^E_r with |entries| < 2^E_r and is rounded to the
//     56-bit integers X_rq = rint(a_rq 2^(56 - E_r)), written as eight
//     balanced base-2^7 digits X = sum_t x_t 2^(7 (7 - t)), |x_t| <= 64
//     (|x_0| <= 128), each exactly a bf16.  The digits go to a work space in
//     the 128-byte-swizzled K-major image the tensor cores read, one image
//     set per chunk.
//  2. k_update_sliced: one CTA per 128 x 32 output tile; per chunk the digit
//     images arrive by bulk copies (TMA) and one thread issues the 36 digit
//     products with t + u <= 7 (72 tcgen05.mma.kind::f16, K = 16) into eight
//     TMEM accumulators S_d, d = t + u, kept across the chunks.  For a
//     given d at most two products involve x_0 or y_0 (up to 128 x 64) and
//     the others are at most 64 x 64, so |S_d| <= 40960 K <= 2^21.4 for
//     K <= 64 and FP32 accumulation is exact.  The epilogue forms
//     hi = sum_{d<4} S_d 2^(7 (3 - d)) and lo = sum_{d>=4} S_d 2^(7 (7 - d))
//     exactly in integers, the product
//     sum_q a_iq b_jq ~= 2^(E_i + E_j - 63) (hi 2^28 + lo)
//     as a double built from the integer's bits (one rounding), and
//     subtracts it from the FP64 entry: one FP64 instruction per entry.
// Error per entry: operand rounding 2^-57 and the dropped digit products
// (t + u >= 8) below 2^-55, relative to 2^(E_i + E_j) per column of the
// chunks, that is about 2^-52 sqrt(max_q L_iq^2 |d_q| max_q L_jq^2 |d_q|);
// FP64 GEMM's is 2^-53 of each |L_iq d_q L_jq|, summed.  Without the
// balancing a panel mixing pivots of size delta and of size 1/delta pairs
// the largest a of one column with the largest b of another, and the
// factorisation of a matrix with that much growth diverges.
#include <cuda_runtime.h>

#include <cstdint>

#include "ipm_dev.h"
#include "tc_common.cuh"
#include "sliced_common.cuh"

namespace ipm {

using namespace sliced;

namespace {


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
    __shared__ uint64_t bar_load, bar_mid, bar_mma;
    __shared__ uint32_t tbase;
    __shared__ int32_t eb_col[kSliceCols];
    const SlicedTile it = items[blockIdx.x];
    const int s = it.s;
    const int f = P.sn_f[s], ld = P.sn_ld[s];
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // One thread streams the kc chunks (32 columns of the panel pair each)
    // through the one buffer: copy, 72 MMAs into the same accumulators, wait
    // for them before the next copy.  bar_mma completes once every MMA it
    // issued has (also after a failed wait, so that TMEM is never freed
    // under running MMAs).
    auto chunk_copy = [&](int ch) {
        const uint8_t *srcA = ws + (int64_t)it.blk_a * kSliceBlockBytes + ch * kSliceChunkBytes;
        const uint8_t *srcB = ws + (int64_t)it.blk_b * kSliceBlockBytes + ch * kSliceChunkBytes + kSliceOperandBytes;
        tc::mbar_expect_tx(&bar_load, (uint32_t)(4 * kSlicePairBytes + 4 * 4096));
        tc::bulk_g2s(A, srcA, (uint32_t)(4 * kSlicePairBytes), &bar_load);
#pragma unroll
        for (int pr = 0; pr < 4; pr++)
            tc::bulk_g2s(B + pr * 4096, srcB + pr * kSlicePairBytes + it.roff_b * 128, 4096, &bar_load);
    };
    auto chunk_mma = [&](int ch, uint32_t acc) {
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
                    tc::mma_bf16(acc + (uint32_t)(d * kSliceCols), ad, bd, id, (ch > 0 || t > 0 || kk > 0) ? 1u : 0u);
                }
            }
    };
    const int kc = it.kc;
    // the first chunk's copy goes out before anything else the tile waits
    // for (TMEM, the column scales)
    if (tid == 0) {
        tc::mbar_init(&bar_load, 1);
        tc::mbar_init(&bar_mid, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
        chunk_copy(0);
    }
    if (warp == 0) tc::tmem_alloc(&tbase, 256);  // 8 accumulators x 32 columns
    if (tid < kSliceCols) eb_col[tid] = ws_exp[((int64_t)it.blk_b * kSliceRows + it.roff_b + tid) * 2 + 1];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tbase;
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
    const int Ea = ws_exp[((int64_t)it.blk_a * kSliceRows + r) * 2 + 0];  // the row's scale
    if (tid == 0) {
        bool lead_ok = true;  // every copy and MMA of the tile issued
        if (tc::mbar_wait(&bar_load, 0)) {
            chunk_mma(0, tmem);
        } else {
            atomicOr(&ctl->status, kStatTimeout | kStatWaitCopy);
            tc::mbar_wait(&bar_load, 0);  // let the copies in flight land before the CTA exits
            lead_ok = false;
        }
        for (int ch = 1; ch < kc && lead_ok; ch++) {
            // the buffer is free once the previous chunk's MMAs are done
            tc::commit_to(&bar_mid);
            if (!tc::mbar_wait(&bar_mid, (ch - 1) & 1)) {
                atomicOr(&ctl->status, kStatTimeout | kStatWaitMma);
                lead_ok = false;
                break;
            }
            chunk_copy(ch);
            if (!tc::mbar_wait(&bar_load, ch & 1)) {
                atomicOr(&ctl->status, kStatTimeout | kStatWaitCopy);
                tc::mbar_wait(&bar_load, ch & 1);
                lead_ok = false;
                break;
            }
            chunk_mma(ch, tmem);
        }
        tc::commit_to(&bar_mma);
    }
    bool ok = tc::mbar_wait(&bar_mma, 0);
    if (!ok) {
        atomicOr(&ctl->status, kStatTimeout | kStatWaitMma);
        tc::mbar_wait(&bar_mma, 0);  // the MMAs must finish before TMEM is freed
    }
    ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the TMEM loads below are warp-collective
    tc::fence_after_sync();
    if (ok) {
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
                // hi = S0 2^21 + S1 2^14 + S2 2^7 + S3 (|hi| < 2^42)
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
                // T = hi 2^28 + lo, kept as T 2^-8 (|.| < 2^62): the bits dropped
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

void launch_update_sliced(const DevPlan &P, double *fronts, const SlicedTile *items, int32_t count,
                          const uint8_t *ws, const int32_t *ws_exp, DevCtl *ctl, cudaStream_t st) {
    if (count <= 0) return;
    static uint64_t attr = 0;
    if (first_on_device(attr))
        cudaFuncSetAttribute(k_update_sliced, cudaFuncAttributeMaxDynamicSharedMemorySize, kSlicedSmem);
    k_update_sliced<<<count, kSlicedThreads, kSlicedSmem, st>>>(P, fronts, items, ws, ws_exp, ctl);
}


}  // namespace ipm
