// Digit slicing of the sliced tensor-core updates (done by the panel's
// triangular solve for the rows it finishes): a row
// of an operand scaled by 2^-E (|entries| < 2^E) becomes 56-bit integers
// written as eight balanced base-2^7 digits, each exactly a bf16, in the
// 128-byte-swizzled K-major image the tensor cores read.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "ipm_dev.h"

namespace ipm {
namespace sliced {

constexpr int kNoScale = -1100;  // row scale of an all-zero row: every digit is 0
constexpr int kNoExp = -100000;  // no nonzero normal entry seen

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

// One row r of both operands sliced by one warp over NC chunks of 32
// columns: lane q holds L(r, q) and d_q of chunk c in l[c], dq[c] (both 0
// beyond the panel).  Writes the row's digits at row rr of chunk c of the
// slice block `blk` (operand A: L 2^h_q, operand B: L d_q 2^-h_q,
// h_q = floor(log2 |d_q| / 2)), one row scale per operand over all NC
// chunks at exps[2 rr + op]; returns true when an entry is not finite (its
// row is then sliced as zero).
template <int NC>
__device__ __forceinline__ bool slice_row_warp(const double (&l)[NC], const double (&dq)[NC], uint8_t *blk,
                                               int32_t *exps, int rr) {
    const int lane = threadIdx.x & 31;
    double v[NC][2];
    int sh[NC][2];
#pragma unroll
    for (int c = 0; c < NC; c++) {
        const int ed = biased_exp(__double_as_longlong(dq[c]));
        const int h = ed == 0 ? 0 : ((ed - 1023) >> 1);
        v[c][0] = l[c];
        v[c][1] = l[c] * dq[c];
        sh[c][0] = h;
        sh[c][1] = -h;
    }
    int E[2];
    bool bad = false;
#pragma unroll
    for (int op = 0; op < 2; op++) {
        int m = kNoExp;
#pragma unroll
        for (int c = 0; c < NC; c++) {
            const int e = biased_exp(__double_as_longlong(v[c][op]));
            bad |= e == 0x7ff;
            if (e != 0) m = max(m, e + sh[c][op]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        E[op] = m;
    }
    bad = __any_sync(0xffffffffu, bad);
#pragma unroll
    for (int op = 0; op < 2; op++) {
        E[op] = (E[op] == kNoExp || bad) ? kNoScale : E[op] - 1022;
        if (lane == 0) exps[2 * rr + op] = E[op];
#pragma unroll
        for (int c = 0; c < NC; c++) {
            int d[8];
            digits8(E[op] == kNoScale ? 0 : fixed56(v[c][op], sh[c][op], E[op]), d);
            uint8_t *img = blk + c * kSliceChunkBytes + op * kSliceOperandBytes;
#pragma unroll
            for (int t = 0; t < 8; t++) {
                // pack lanes 8k .. 8k+7 (columns) into one 16-byte chunk held by lane 8k
                const uint32_t hb = bf16_bits(d[t]);
                const uint32_t pair = hb | (__shfl_down_sync(0xffffffffu, hb, 1) << 16);
                const uint32_t w1 = __shfl_down_sync(0xffffffffu, pair, 2);
                const uint32_t w2 = __shfl_down_sync(0xffffffffu, pair, 4);
                const uint32_t w3 = __shfl_down_sync(0xffffffffu, pair, 6);
                if ((lane & 7) == 0) {
                    const int chunk = (t & 1) * 4 + (lane >> 3);
                    *(uint4 *)(img + (t >> 1) * kSlicePairBytes + swz_chunk(rr, chunk)) =
                        make_uint4(pair, w1, w2, w3);
                }
            }
        }
    }
    return bad;
}

}  // namespace sliced
}  // namespace ipm
