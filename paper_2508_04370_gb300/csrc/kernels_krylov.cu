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
                                                   int64_t N, int cnt, double *__restrict__ part,
                                                   const int32_t *skip) {
    if (skip && *skip) return;
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

__global__ void k_dots_final(const double *__restrict__ part, int cnt, double *__restrict__ out,
                             const int32_t *skip) {
    if (skip && *skip) return;
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
                 cudaStream_t st, const int32_t *skip) {
    k_dots<<<kBlocks, kThreads, 0, st>>>(w, V, N, cnt, part, skip);
    k_dots_final<<<1, 32, 0, st>>>(part, cnt, out, skip);
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


// ---------------------------------------------------------------------------
// GMRES refinement inside a captured CUDA graph.  The host-driven version
// (gmres_refine) reads the dot products and solves the small least-squares
// problem on the host; here one thread does that work on the device (GmDev)
// and every vector kernel of the section returns at entry once the flags say
// so.  The whole section sits in a conditional graph node that runs only
// when classical refinement ended above the target (k_gm_begin sets it).

namespace {

__global__ void k_gm_begin(DevCtl *ctl, GmDev *gm, double target, cudaGraphConditionalHandle handle) {
    const double wb = ctl->omega_best;
    const bool run = wb > target && !(ctl->status & kStatNonFinite);
    gm->wbest = wb;
    gm->stop = run ? 0 : 1;
    gm->skip_inner = gm->stop;
    gm->improved = 0;
    gm->iters = 0;
    ctl->gmres_iters = 0;
    cudaGraphSetConditional(handle, run ? 1u : 0u);
}

// after r = f - K x and omega(x): keep x when it improved, decide whether to go on
__global__ void k_gm_cycle(DevCtl *ctl, GmDev *gm, double target, int cycle, int last) {
    if (gm->stop) {
        gm->improved = 0;
        return;
    }
    const double w = ctl->omega;
    int improved = 0;
    if (cycle > 0) {
        if (w < gm->wbest) {
            gm->wbest = w;
            improved = 1;
            ctl->omega_best = w;
        } else {
            gm->stop = 1;  // no progress
        }
    }
    if (gm->wbest <= target || cycle == last || (ctl->status & kStatNonFinite)) gm->stop = 1;
    gm->improved = improved;
    gm->skip_inner = gm->stop;
}

// beta = ||r||, V_0 = r / beta; reset the Hessenberg matrix of the cycle
__global__ void k_gm_init(DevCtl *ctl, GmDev *gm, double target) {
    if (gm->stop) return;
    const double beta = sqrt(gm->h[0]);
    if (!(beta > 0.0) || !isfinite(beta)) {
        gm->stop = 1;
        gm->skip_inner = 1;
        return;
    }
    gm->beta = beta;
    gm->inv = 1.0 / beta;
    for (int i = 0; i < (kGmresM + 1) * kGmresM; i++) gm->H[i] = 0.0;
    for (int i = 0; i <= kGmresM; i++) gm->g[i] = 0.0;
    gm->g[0] = beta;
    // relative residual reduction that brings omega under the target, with margin
    gm->eta = fmin(0.5, fmax(1e-14, 0.1 * target / fmax(ctl->omega, 1e-300)));
    gm->jdone = 0;
    gm->skip_inner = 0;
}

// H(i, j) += h_i (one classical Gram-Schmidt pass)
__global__ void k_gm_hacc(GmDev *gm, int j) {
    if (gm->skip_inner) return;
    for (int i = 0; i <= j; i++) gm->H[i * kGmresM + j] += gm->h[i];
}

// H(j+1, j) = ||v||, the Givens rotations, the convergence test of the cycle
__global__ void k_gm_arnoldi(GmDev *gm, int j) {
    if (gm->skip_inner) return;
    const double hn = sqrt(gm->h[0]);
    double *H = gm->H;
    H[(j + 1) * kGmresM + j] = hn;
    gm->inv = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; i++) {
        const double a = H[i * kGmresM + j], b = H[(i + 1) * kGmresM + j];
        H[i * kGmresM + j] = gm->cs[i] * a + gm->sn[i] * b;
        H[(i + 1) * kGmresM + j] = -gm->sn[i] * a + gm->cs[i] * b;
    }
    const double a = H[j * kGmresM + j], b = H[(j + 1) * kGmresM + j], r = hypot(a, b);
    gm->cs[j] = r > 0.0 ? a / r : 1.0;
    gm->sn[j] = r > 0.0 ? b / r : 0.0;
    H[j * kGmresM + j] = r;
    H[(j + 1) * kGmresM + j] = 0.0;
    gm->g[j + 1] = -gm->sn[j] * gm->g[j];
    gm->g[j] = gm->cs[j] * gm->g[j];
    gm->jdone = j + 1;
    gm->iters++;
    if (fabs(gm->g[j + 1]) <= gm->eta * gm->beta || !(hn > 0.0)) gm->skip_inner = 1;
}

// y = R^-1 g over the cycle's jdone columns
__global__ void k_gm_ls(GmDev *gm) {
    if (gm->stop) return;
    const int n = gm->jdone;
    for (int i = n - 1; i >= 0; i--) {
        double t = gm->g[i];
        for (int q = i + 1; q < n; q++) t -= gm->H[i * kGmresM + q] * gm->y[q];
        const double d = gm->H[i * kGmresM + i];
        gm->y[i] = d != 0.0 ? t / d : 0.0;
    }
}

__global__ void k_gm_end(DevCtl *ctl, GmDev *gm) { ctl->gmres_iters = gm->iters; }

// w -= sum_i h_i V_i with h on the device (skipped with the cycle)
__global__ void k_gs_update_dev(double *__restrict__ w, const double *__restrict__ V, const GmDev *gm, int64_t N,
                                int cnt) {
    if (gm->skip_inner) return;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        double s = w[t];
        for (int i = 0; i < cnt; i++) s -= gm->h[i] * V[(int64_t)i * N + t];
        w[t] = s;
    }
}

// dst = factor * gm->inv * src (factor * src when factor carries its own scale: use_inv = 0)
__global__ void k_scale_dev(double *__restrict__ dst, const double *__restrict__ src, const GmDev *gm, double factor,
                            int64_t N, const int32_t *skip) {
    if (skip && *skip) return;
    const double a = isnan(factor) ? gm->inv : factor;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = a * src[t];
}

// x += sum_j y_j Z_j over the cycle's jdone vectors
__global__ void k_combine_dev(double *__restrict__ x, const double *__restrict__ Z, const GmDev *gm, int64_t N) {
    if (gm->stop) return;
    const int cnt = gm->jdone;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        double s = x[t];
        for (int j = 0; j < cnt; j++) s += gm->y[j] * Z[(int64_t)j * N + t];
        x[t] = s;
    }
}

}  // namespace

void launch_gm_begin(DevCtl *ctl, GmDev *gm, double target, unsigned long long cond_handle, cudaStream_t st) {
    k_gm_begin<<<1, 1, 0, st>>>(ctl, gm, target, (cudaGraphConditionalHandle)cond_handle);
}
void launch_gm_cycle(DevCtl *ctl, GmDev *gm, double target, int32_t cycle, int32_t last, cudaStream_t st) {
    k_gm_cycle<<<1, 1, 0, st>>>(ctl, gm, target, cycle, last);
}
void launch_gm_init(DevCtl *ctl, GmDev *gm, double target, cudaStream_t st) { k_gm_init<<<1, 1, 0, st>>>(ctl, gm, target); }
void launch_gm_hacc(GmDev *gm, int32_t j, cudaStream_t st) { k_gm_hacc<<<1, 1, 0, st>>>(gm, j); }
void launch_gm_arnoldi(GmDev *gm, int32_t j, cudaStream_t st) { k_gm_arnoldi<<<1, 1, 0, st>>>(gm, j); }
void launch_gm_ls(GmDev *gm, cudaStream_t st) { k_gm_ls<<<1, 1, 0, st>>>(gm); }
void launch_gm_end(DevCtl *ctl, GmDev *gm, cudaStream_t st) { k_gm_end<<<1, 1, 0, st>>>(ctl, gm); }
void launch_gs_update_dev(double *w, const double *V, const GmDev *gm, int64_t N, int32_t cnt, cudaStream_t st) {
    k_gs_update_dev<<<grid_for(N), kThreads, 0, st>>>(w, V, gm, N, cnt);
}
void launch_scale_dev(double *dst, const double *src, const GmDev *gm, double factor, int64_t N,
                      const int32_t *skip, cudaStream_t st) {
    k_scale_dev<<<grid_for(N), kThreads, 0, st>>>(dst, src, gm, factor, N, skip);
}
void launch_combine_dev(double *x, const double *Z, const GmDev *gm, int64_t N, cudaStream_t st) {
    k_combine_dev<<<grid_for(N), kThreads, 0, st>>>(x, Z, gm, N);
}

}  // namespace ipm
