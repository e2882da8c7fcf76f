// FP64 peak microbenchmarks: the denominators of the FP64 rooflines (the
// pivot blocks, triangular solves and FP64 trailing updates of Sec. 4.4 run
// on these units).  Both kernels keep every SM busy with independent chains
// and write one value per thread so that nothing is optimised away.
//   k_peak_dfma: DFMA chains (8 independent accumulators per thread).
//   k_peak_dmma: mma.sync.m8n8k4.f64 chains (the FP64 tensor instruction),
//                4 independent accumulator tiles per warp.
#include <cuda_runtime.h>

#include <cstdint>

#include "ipm_dev.h"

namespace ipm {

namespace {

constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(256) k_peak_dfma(double *out, int iters, double a, double b) {
    double acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) acc[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kPeakChains; c++) acc[c] = fma(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dmma(double *out, int iters, double a, double b) {
    // per lane: A fragment 1 double, B fragment 1 double, C/D fragment 2 doubles
    double c[4][2];
#pragma unroll
    for (int t = 0; t < 4; t++) c[t][0] = c[t][1] = (double)(threadIdx.x + t);
    const double av = a + threadIdx.x * 1e-9, bv = b;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int t = 0; t < 4; t++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[t][0]), "+d"(c[t][1])
                         : "d"(av), "d"(bv));
    }
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < 4; t++) s += c[t][0] + c[t][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// Runs each kernel once untimed and `reps` times timed (CUDA events on
// `st`); returns the best TFLOP/s of each (2 flops per FMA; an m8n8k4 MMA is
// 256 FMAs per warp).  out must hold blocks * 256 doubles.
int measure_fp64_peaks(double *out, int blocks, int iters, int reps, cudaStream_t st, double *dfma_tflops,
                       double *dmma_tflops) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1;
    }
    double best[2] = {0.0, 0.0};
    for (int k = 0; k < 2; k++) {
        for (int r = 0; r <= reps; r++) {
            cudaEventRecord(e0, st);
            if (k == 0) k_peak_dfma<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-7);
            else k_peak_dmma<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-7);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double threads = (double)blocks * 256.0;
            const double flops = k == 0 ? threads * iters * kPeakChains * 2.0
                                        : (threads / 32.0) * iters * 4.0 * 256.0 * 2.0;
            if (r > 0 && ms > 0.f) best[k] = best[k] > flops / (ms * 1e-3) / 1e12 ? best[k] : flops / (ms * 1e-3) / 1e12;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *dfma_tflops = best[0];
    *dmma_tflops = best[1];
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm
