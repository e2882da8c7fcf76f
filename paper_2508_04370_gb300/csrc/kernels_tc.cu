// Mixed-precision trailing (Schur-complement) update on the Blackwell tensor
// cores: the FP32 Schur updates of large fronts (Sec. 4.4 dgemm updates, here
// with FP64 pivots, regularisation and refinement kept in FP64).
//
// One CTA (4 warps) updates one 128 x 128 tile of the lower trailing part of
// a front after a 32-column panel [p0, p0+w):
//     C(i, j) -= sum_q L(i, q) * (d_q L(j, q)),   i >= j.
// The FP64 operands are read from the front slab, rounded to FP32 and split
// into tf32 hi + lo parts (3xTF32: hi*hi + hi*lo + lo*hi, FP32 accumulation),
// stored in 128-byte-swizzled K-major shared-memory tiles, multiplied by 12
// tcgen05.mma (kind::tf32, M = N = 128, K = 8) issued by one thread into a
// 128-column TMEM accumulator, and the accumulator is subtracted from the
// FP64 tile in the epilogue (tcgen05.ld, 32 lanes per warp).
#include <cuda_runtime.h>

#include <cstdint>

#include "ipm_dev.h"
#include "tc_common.cuh"

namespace ipm {

namespace {

constexpr int kTcSmem = 4 * 16384 + 1024;    // four 128 x 32 fp32 tiles + alignment

__global__ void __launch_bounds__(128) k_large_update_tc(DevPlan P, double *__restrict__ fronts,
                                                         const double *__restrict__ Dg,
                                                         const TileItem *__restrict__ items, int w,
                                                         DevCtl *ctl) {
    extern __shared__ uint8_t tc_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *Ahi = base, *Alo = base + 16384, *Bhi = base + 32768, *Blo = base + 49152;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    const TileItem it = items[blockIdx.x];
    const int s = it.s, p0 = it.p0;
    const int f = P.sn_f[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    w = min(w, P.sn_k[s] - p0);
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&tbase, 128);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    // thread r stages row r of A (rows i0 + r) and of B (rows j0 + r)
    const int i = it.i0 + tid, j = it.j0 + tid;
#pragma unroll 8
    for (int q = 0; q < 32; q++) {
        const bool qa = q < w;
        const double a = (qa && i < f) ? F[(int64_t)(p0 + q) * ld + i] : 0.0;
        const double b = (qa && j < f) ? F[(int64_t)(p0 + q) * ld + j] * Dg[c0 + p0 + q] : 0.0;
        const float af = (float)a, bf = (float)b;
        const float ah = tc::to_tf32(af), bh = tc::to_tf32(bf);
        const uint32_t o = tc::swz_offset(tid, q);
        *(float *)(Ahi + o) = ah;
        *(float *)(Alo + o) = tc::to_tf32(af - ah);
        *(float *)(Bhi + o) = bh;
        *(float *)(Blo + o) = tc::to_tf32(bf - bh);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tbase;
    if (tid == 0) {
        constexpr uint32_t id = tc::idesc_tf32(128, 128);
        const uint32_t ah0 = tc::smem_u32(Ahi), al0 = tc::smem_u32(Alo);
        const uint32_t bh0 = tc::smem_u32(Bhi), bl0 = tc::smem_u32(Blo);
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            const uint64_t ah = tc::smem_desc(ah0 + kk * 32), al = tc::smem_desc(al0 + kk * 32);
            const uint64_t bh = tc::smem_desc(bh0 + kk * 32), bl = tc::smem_desc(bl0 + kk * 32);
            tc::mma_tf32(tmem, ah, bh, id, kk > 0);
            tc::mma_tf32(tmem, ah, bl, id, 1);
            tc::mma_tf32(tmem, al, bh, id, 1);
        }
        tc::commit_to(&mbar);
    }
    bool ok = tc::mbar_wait(&mbar, 0);
    if (!ok) {
        atomicOr(&ctl->status, kStatTimeout | kStatWaitMma);
        tc::mbar_wait(&mbar, 0);  // the MMAs must finish before TMEM is freed
    }
    ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the TMEM loads below are warp-collective
    tc::fence_after_sync();
    if (ok) {
        const int row = it.i0 + warp * 32 + lane;
#pragma unroll 1
        for (int ch = 0; ch < 4; ch++) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), v);
            if (row < f) {
#pragma unroll
                for (int c = 0; c < 32; c++) {
                    const int col = it.j0 + ch * 32 + c;
                    if (col < f && row >= col) F[(int64_t)col * ld + row] -= (double)v[c];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

}  // namespace

void launch_large_update_tc(const DevPlan &P, double *fronts, const double *D, const TileItem *items, int32_t count,
                            int32_t w, DevCtl *ctl, cudaStream_t st) {
    if (count <= 0) return;
    static uint64_t attr = 0;
    if (first_on_device(attr)) {
        cudaFuncSetAttribute(k_large_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    }
    k_large_update_tc<<<count, 128, kTcSmem, st>>>(P, fronts, D, items, w, ctl);
}

}  // namespace ipm
