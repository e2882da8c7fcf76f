// Normal-equations path (Zanetti & Gondzio, arXiv 2508.04370, Eq. normeq with
// the regularisation of Eq. regul_matrix):
//   Theta~ = (Theta^-1 + rho I)^-1
//   M      = A Theta~ A^T            (formed every iteration; delta enters at the pivot)
//   r8     = r1 + A Theta~ r7,   M_reg dy = r8,   dx = Theta~ (A^T dy - r7).
// Formation is deterministic: every lower entry (r, i) of M sums its own
// contributor pairs a_rj Theta~_j a_ij in ascending column j (no atomics).
#include <cuda_runtime.h>

#include <cstdint>

#include "ipm_dev.h"

namespace ipm {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work) {
    int64_t g = (work + kThreads - 1) / kThreads;
    return (int)(g < 1 ? 1 : (g > 1216 ? 1216 : g));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void k_theta_tilde(const double *__restrict__ theta, double rho, int n, double *__restrict__ tt,
                              DevCtl *ctl) {
    bool bad = false;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double th = theta[j];
        if (!(th > 0.0) || !isfinite(th)) bad = true;
        tt[j] = 1.0 / (1.0 / th + rho);
    }
    if (bad) atomicOr(&ctl->status, kStatNonFinite);
}

__global__ void k_ne_form(int64_t nnz, const int64_t *__restrict__ tptr, const int32_t *__restrict__ ta,
                          const int32_t *__restrict__ tb, const int32_t *__restrict__ tj,
                          const double *__restrict__ Ax, const double *__restrict__ tt, double *__restrict__ nev) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t t = tptr[e]; t < tptr[e + 1]; t++) s += Ax[ta[t]] * (Ax[tb[t]] * tt[tj[t]]);
        nev[e] = s;
    }
}

// r8 in the factorisation order: f[i] = r1[o] + sum_j a_oj (Theta~_j r7_j), o = perm[i]
__global__ void k_ne_rhs(const int32_t *__restrict__ perm, int m, const int64_t *__restrict__ Arp,
                         const int32_t *__restrict__ Aci, const int32_t *__restrict__ Apos,
                         const double *__restrict__ Ax, const double *__restrict__ tt, const double *__restrict__ r7,
                         const double *__restrict__ r1, double *__restrict__ f) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int o = perm[i];
        double s = r1[o];
        for (int64_t p = Arp[o]; p < Arp[o + 1]; p++) {
            const int j = Aci[p];
            s += Ax[Apos[p]] * (tt[j] * r7[j]);
        }
        f[i] = s;
    }
}

// dx_j = Theta~_j (sum_i a_ij dy_i - r7_j)
__global__ void k_ne_dx(int n, const int64_t *__restrict__ Acp, const int32_t *__restrict__ Ari,
                        const double *__restrict__ Ax, const double *__restrict__ tt, const double *__restrict__ dy,
                        const double *__restrict__ r7, double *__restrict__ dx) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = Acp[j]; p < Acp[j + 1]; p++) s += Ax[p] * dy[Ari[p]];
        dx[j] = tt[j] * (s - r7[j]);
    }
}

// Residual of the regularised augmented system in the original order (for
// reporting the backward error on K of a normal-equations solve):
// r = [r7; r1] - K [dx; dy], ad = |K||d|, ae = |K|e, running max |d|.
__global__ void k_residual_K(int n, int m, const int64_t *__restrict__ Acp, const int32_t *__restrict__ Ari,
                             const int64_t *__restrict__ Arp, const int32_t *__restrict__ Aci,
                             const int32_t *__restrict__ Apos, const double *__restrict__ Ax,
                             const double *__restrict__ theta, double rho, double delta,
                             const double *__restrict__ r7, const double *__restrict__ r1,
                             const double *__restrict__ dx, const double *__restrict__ dy, double *__restrict__ f,
                             double *__restrict__ r, double *__restrict__ ad, double *__restrict__ ae, DevCtl *ctl) {
    double xm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        double s, sa, se, fi, di;
        if (i < n) {
            const double dg = -(1.0 / theta[i] + rho);
            di = dx[i];
            fi = r7[i];
            s = dg * di;
            sa = fabs(dg) * fabs(di);
            se = fabs(dg);
            for (int64_t p = Acp[i]; p < Acp[i + 1]; p++) {
                const double a = Ax[p], v = dy[Ari[p]];
                s += a * v;
                sa += fabs(a) * fabs(v);
                se += fabs(a);
            }
        } else {
            const int q = i - n;
            di = dy[q];
            fi = r1[q];
            s = delta * di;
            sa = delta * fabs(di);
            se = delta;
            for (int64_t p = Arp[q]; p < Arp[q + 1]; p++) {
                const double a = Ax[Apos[p]], v = dx[Aci[p]];
                s += a * v;
                sa += fabs(a) * fabs(v);
                se += fabs(a);
            }
        }
        f[i] = fi;
        r[i] = fi - s;
        ad[i] = sa;
        ae[i] = se;
        xm = fmax(xm, fabs(di));
    }
    xm = warp_max(xm);
    if ((threadIdx.x & 31) == 0)
        atomicMax((unsigned long long *)&ctl->dinf, (unsigned long long)__double_as_longlong(xm));
}

}  // namespace

void launch_ne_form(const NeView &E, const double *Ax, const double *theta, double rho, DevCtl *ctl,
                    cudaStream_t st) {
    k_theta_tilde<<<grid_for(E.n), kThreads, 0, st>>>(theta, rho, E.n, E.tt, ctl);
    k_ne_form<<<grid_for(E.nnz), kThreads, 0, st>>>(E.nnz, E.tptr, E.ta, E.tb, E.tj, Ax, E.tt, E.nev);
}

void launch_ne_rhs(const NeView &E, const int32_t *perm, const double *Ax, const double *r7, const double *r1,
                   double *f, cudaStream_t st) {
    k_ne_rhs<<<grid_for(E.m), kThreads, 0, st>>>(perm, E.m, E.Arp, E.Aci, E.Apos, Ax, E.tt, r7, r1, f);
}

void launch_ne_dx(const NeView &E, const double *Ax, const double *dy, const double *r7, double *dx,
                  cudaStream_t st) {
    k_ne_dx<<<grid_for(E.n), kThreads, 0, st>>>(E.n, E.Acp, E.Ari, Ax, E.tt, dy, r7, dx);
}

void launch_residual_K(const NeView &E, const double *Ax, const double *theta, double rho, double delta,
                       const double *r7, const double *r1, const double *dx, const double *dy, double *f, double *r,
                       double *ad, double *ae, DevCtl *ctl, cudaStream_t st) {
    cudaMemsetAsync(&ctl->dinf, 0, sizeof(double), st);
    cudaMemsetAsync(&ctl->omega, 0, sizeof(double), st);
    k_residual_K<<<grid_for((int64_t)E.n + E.m), kThreads, 0, st>>>(E.n, E.m, E.Acp, E.Ari, E.Arp, E.Aci, E.Apos, Ax,
                                                                    theta, rho, delta, r7, r1, dx, dy, f, r, ad, ae,
                                                                    ctl);
}

}  // namespace ipm
