// Vector kernels of the GMRES refinement (an extension of the refinement of
// Sec. 4.5: restarted, right-preconditioned GMRES on K c = r with the
// regularised LDL^T factor as preconditioner, used when classical
// refinement stalls above the backward-error target).  Reductions are
// deterministic: a fixed grid writes per-block partial sums, which one block
// adds in block order.
#include <cuda_runtime.h>

#include <cstdint>

#include "ipm_dev.h"

namespace ipm {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 304;  // 2 per SM of a 152-SM part; fixed for determinism

// part[b * kMaxDots + i] = sum over block b's slice of w * V_i (i < cnt)
__global__ void __launch_bounds__(kThreads) k_dots(const double *__restrict__ w, const double *__restrict__ V,
                                                   int64_t N, int cnt, double *__restrict__ part) {
    __shared__ double red[kThreads / 32][kMaxDots];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc[kMaxDots];
#pragma unroll
    for (int i = 0; i < kMaxDots; i++) acc[i] = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)kThreads + tid; t < N; t += (int64_t)kBlocks * kThreads) {
        const double wt = w[t];
#pragma unroll
        for (int i = 0; i < kMaxDots; i++)
            if (i < cnt) acc[i] += wt * V[(int64_t)i * N + t];
    }
#pragma unroll
    for (int i = 0; i < kMaxDots; i++) {
        double v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (tid < kMaxDots) {
        double v = 0.0;
        for (int q = 0; q < kThreads / 32; q++) v += red[q][tid];
        part[blockIdx.x * kMaxDots + tid] = v;
    }
}

__global__ void k_dots_final(const double *__restrict__ part, int cnt, double *__restrict__ out) {
    const int i = threadIdx.x;
    if (i < cnt) {
        double v = 0.0;
        for (int b = 0; b < kBlocks; b++) v += part[b * kMaxDots + i];
        out[i] = v;
    }
}

// w -= sum_i h_i V_i
__global__ void k_gs_update(double *__restrict__ w, const double *__restrict__ V, const double *__restrict__ h,
                            int64_t N, int cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        double s = w[t];
        for (int i = 0; i < cnt; i++) s -= h[i] * V[(int64_t)i * N + t];
        w[t] = s;
    }
}

// dst = alpha * src
__global__ void k_scale(double *__restrict__ dst, const double *__restrict__ src, double alpha, int64_t N) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = alpha * src[t];
}

// x += sum_j y_j Z_j
__global__ void k_combine(double *__restrict__ x, const double *__restrict__ Z, GmresCoef y, int64_t N, int cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        double s = x[t];
        for (int j = 0; j < cnt; j++) s += y.c[j] * Z[(int64_t)j * N + t];
        x[t] = s;
    }
}

inline int grid_for(int64_t n) {
    const int64_t g = (n + kThreads - 1) / kThreads;
    return (int)(g < 1 ? 1 : (g > 1216 ? 1216 : g));
}

}  // namespace

void launch_dots(const double *w, const double *V, int64_t N, int32_t cnt, double *part, double *out,
                 cudaStream_t st) {
    k_dots<<<kBlocks, kThreads, 0, st>>>(w, V, N, cnt, part);
    k_dots_final<<<1, 32, 0, st>>>(part, cnt, out);
}

void launch_gs_update(double *w, const double *V, const double *h, int64_t N, int32_t cnt, cudaStream_t st) {
    k_gs_update<<<grid_for(N), kThreads, 0, st>>>(w, V, h, N, cnt);
}

void launch_scale(double *dst, const double *src, double alpha, int64_t N, cudaStream_t st) {
    k_scale<<<grid_for(N), kThreads, 0, st>>>(dst, src, alpha, N);
}

void launch_combine(double *x, const double *Z, const GmresCoef &y, int64_t N, int32_t cnt, cudaStream_t st) {
    k_combine<<<grid_for(N), kThreads, 0, st>>>(x, Z, y, N, cnt);
}

int32_t dots_partial_size() { return kBlocks * kMaxDots; }

}  // namespace ipm
