// Solve and refinement kernels (Zanetti & Gondzio, arXiv 2508.04370, Sec. 4:
// forward solve with L, diagonal solve with D, backward solve with L^T;
// Sec. 4.5: residual of the regularised matrix and the component-wise
// backward error of Arioli, Demmel and Duff used to stop the refinement).
//
// All vectors are kept in the factorisation order.  The forward sweep is
// multifrontal: each supernode pulls the contribution vectors of its
// children (ascending order) into its local vector, eliminates its k
// columns and leaves a contribution vector of length f-k for its parent.
// The backward sweep gathers the already final values of the ancestors.
#include <cuda_runtime.h>

#include <cstdint>

#include "ipm_dev.h"

namespace ipm {

namespace {

constexpr int kSolveThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Forward: L y = b on the supernodes of one level, then y <- D^-1 y.
__global__ void __launch_bounds__(kSolveThreads) k_forward(DevPlan P, const double *__restrict__ fronts,
                                                            const double *__restrict__ D, double *__restrict__ x,
                                                            double *__restrict__ upd,
                                                            const int32_t *__restrict__ list) {
    extern __shared__ double v[];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    const double *L = fronts + P.sn_off[s];
    const int tid = threadIdx.x;
    for (int t = tid; t < f; t += kSolveThreads) v[t] = t < k ? x[c0 + t] : 0.0;
    __syncthreads();
    for (int q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
        const int c = P.child_list[q];
        const int cc = P.sn_f[c] - P.sn_k[c];
        const double *u = upd + P.upd_off[c];
        const int32_t *map = P.relmap + P.map_off[c];
        for (int t = tid; t < cc; t += kSolveThreads) v[map[t]] += u[t];
        __syncthreads();
    }
    const int lane = tid & 31, warp = tid >> 5;
    // column-oriented elimination in blocks of 32 columns: warp 0 solves the
    // 32 x 32 triangle, then all threads update the rows below the block
    for (int b0 = 0; b0 < k; b0 += 32) {
        const int b1 = min(b0 + 32, k);
        if (warp == 0) {
            for (int j = b0; j < b1; j++) {
                const double yj = v[j];
                __syncwarp();
                const int i = j + 1 + lane;
                if (i < b1) v[i] -= L[(int64_t)j * ld + i] * yj;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = b1 + tid; i < f; i += kSolveThreads) {
            double acc = 0.0;
            for (int j = b0; j < b1; j++) acc += L[(int64_t)j * ld + i] * v[j];
            v[i] -= acc;
        }
        __syncthreads();
    }
    (void)warp;
    for (int t = tid; t < f; t += kSolveThreads) {
        if (t < k) x[c0 + t] = v[t] / D[c0 + t];
        else upd[P.upd_off[s] + (t - k)] = v[t];
    }
}

// Backward: L^T z = y on the supernodes of one level (ancestors are final).
__global__ void __launch_bounds__(kSolveThreads) k_backward(DevPlan P, const double *__restrict__ fronts,
                                                             double *__restrict__ x,
                                                             const int32_t *__restrict__ list) {
    extern __shared__ double z[];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    const double *L = fronts + P.sn_off[s];
    const int32_t *rows = P.sn_rows + P.sn_rptr[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < f; t += kSolveThreads) z[t] = t < k ? x[c0 + t] : x[rows[t]];
    __syncthreads();
    // blocks of 32 columns from the last: the rows below the block are final
    const int nblk = (k + 31) / 32;
    for (int bb = nblk - 1; bb >= 0; bb--) {
        const int b0 = bb * 32, b1 = min(b0 + 32, k);
        // z_j -= sum_{i >= b1} L(i, j) z_i  for j in the block (one warp per column)
        for (int j = b0 + warp; j < b1; j += kSolveThreads / 32) {
            double acc = 0.0;
            for (int i = b1 + lane; i < f; i += 32) acc += L[(int64_t)j * ld + i] * z[i];
            acc = warp_sum(acc);
            if (lane == 0) z[j] -= acc;
        }
        __syncthreads();
        if (warp == 0) {
            for (int j = b1 - 1; j >= b0; j--) {
                double acc = 0.0;
                const int i = j + 1 + lane;
                if (i < b1) acc = L[(int64_t)j * ld + i] * z[i];
                acc = warp_sum(acc);
                if (lane == 0) z[j] -= acc;
                __syncwarp();
            }
        }
        __syncthreads();
    }
    for (int t = tid; t < k; t += kSolveThreads) x[c0 + t] = z[t];
}

// f (factorisation order) from [r7; r1] (original order).
__global__ void k_permute_in(const int32_t *__restrict__ perm, int N, int n, const double *__restrict__ r7,
                             const double *__restrict__ r1, double *__restrict__ f, int form) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int o = perm[i];
        f[i] = form == 1 ? (o < n ? r7[o] : r1[o - n]) : r1[o];
    }
}
__global__ void k_permute_out(const int32_t *__restrict__ perm, int N, int n, const double *__restrict__ x,
                              double *__restrict__ dx, double *__restrict__ dy) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int o = perm[i];
        if (o < n) dx[o] = x[i];
        else dy[o - n] = x[i];
    }
}

// r = f - K x, ad = |K||x|, ae = |K|e in the factorisation order; also the
// running max of |x| (ctl->dinf, as ordered bits of a non-negative double).
__global__ void k_residual(DevPlan P, DevVals V, const double *__restrict__ f, const double *__restrict__ x,
                           double *__restrict__ r, double *__restrict__ ad, double *__restrict__ ae, DevCtl *ctl) {
    double xm = 0.0;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
        double s = 0.0, sa = 0.0, se = 0.0;
        for (int64_t p = P.kp[i]; p < P.kp[i + 1]; p++) {
            const int64_t src = P.ksrc[p];
            double val;
            if (src >= 0) val = V.Ax[src];
            else if (src == kDualDiag) val = V.delta;
            else val = -(1.0 / V.theta[-1 - src] + V.rho);
            const double xj = x[P.kj[p]];
            s += val * xj;
            sa += fabs(val) * fabs(xj);
            se += fabs(val);
        }
        const double ri = f[i] - s;
        if (!isfinite(ri)) bad = true;
        r[i] = ri;
        ad[i] = sa;
        ae[i] = se;
        xm = fmax(xm, fabs(x[i]));
    }
    xm = warp_max(xm);
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&ctl->dinf, (unsigned long long)__double_as_longlong(xm));
    if (bad) atomicOr(&ctl->status, kStatNonFinite);
}

// omega = max_i |r_i| / den_i, den_i = (|K||x| + |f|)_i, replaced by
// (|K||x| + ||x||_inf |K|e)_i when den_i <= 1000 N eps (ae_i ||x||_inf + |f_i|).
__global__ void k_omega(int N, const double *__restrict__ r, const double *__restrict__ ad,
                        const double *__restrict__ ae, const double *__restrict__ f, DevCtl *ctl) {
    const double dinf = ctl->dinf;
    const double eps = 2.220446049250313e-16;
    double w = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double den = ad[i] + fabs(f[i]);
        const double tau = 1000.0 * N * eps * (ae[i] * dinf + fabs(f[i]));
        if (den <= tau) den = ad[i] + dinf * ae[i];
        const double num = fabs(r[i]);
        double wi = den > 0.0 ? num / den : (num > 0.0 ? INFINITY : 0.0);
        if (isnan(wi)) wi = INFINITY;
        w = fmax(w, wi);
    }
    w = warp_max(w);
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&ctl->omega, (unsigned long long)__double_as_longlong(w));
}

__global__ void k_axpy(double *__restrict__ x, const double *__restrict__ c, int N) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) x[i] += c[i];
}

}  // namespace

void launch_forward(const DevPlan &P, const double *fronts, const double *D, double *x, double *upd,
                    const int32_t *list, int32_t count, int32_t maxf, cudaStream_t st) {
    if (count <= 0) return;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    k_forward<<<count, kSolveThreads, (size_t)maxf * sizeof(double), st>>>(P, fronts, D, x, upd, list);
}

void launch_backward(const DevPlan &P, const double *fronts, double *x, const int32_t *list, int32_t count,
                     int32_t maxf, cudaStream_t st) {
    if (count <= 0) return;
    k_backward<<<count, kSolveThreads, (size_t)maxf * sizeof(double), st>>>(P, fronts, x, list);
}

void launch_permute_in(const DevPlan &P, const double *r7, const double *r1, double *f, cudaStream_t st) {
    k_permute_in<<<(P.N + 255) / 256, 256, 0, st>>>(P.perm, P.N, P.n, r7, r1, f, P.form);
}

void launch_permute_out(const DevPlan &P, const double *x, double *dx, double *dy, cudaStream_t st) {
    k_permute_out<<<(P.N + 255) / 256, 256, 0, st>>>(P.perm, P.N, P.n, x, dx, dy);
}

void launch_residual_omega(const DevPlan &P, const DevVals &V, const double *f, const double *x, double *r,
                           double *ad, double *ae, DevCtl *ctl, cudaStream_t st) {
    const int grid = (P.N + 255) / 256 < 608 ? (P.N + 255) / 256 : 608;
    cudaMemsetAsync(&ctl->dinf, 0, sizeof(double), st);
    cudaMemsetAsync(&ctl->omega, 0, sizeof(double), st);
    k_residual<<<grid, 256, 0, st>>>(P, V, f, x, r, ad, ae, ctl);
    k_omega<<<grid, 256, 0, st>>>(P.N, r, ad, ae, f, ctl);
}

void launch_axpy(double *x, const double *c, int32_t N, cudaStream_t st) {
    k_axpy<<<(N + 255) / 256 < 608 ? (N + 255) / 256 : 608, 256, 0, st>>>(x, c, N);
}

}  // namespace ipm
