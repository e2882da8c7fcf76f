// Numeric multifrontal factorisation kernels (Zanetti & Gondzio,
// arXiv 2508.04370, Sec. 4.1, 4.4, 4.5), FP64.
//
// Every front s owns a resident f x f slab (column-major, leading dimension
// ld) in one device arena.  After its factorisation the first k columns hold
// L (strictly lower part; D on the diagonal) and the trailing (f-k) x (f-k)
// lower block holds the contribution block (Schur complement) that the
// parent pulls during its own assembly.  Children are always summed in
// ascending order, original entries first, so results do not depend on
// scheduling (Sec. 4.3, determinism).
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

// Pivot decision for pivot p of block [p, b1) held in a column-major array
// Fm with leading dimension ld; executed by one full warp.  Returns the
// accepted pivot on every lane.
__device__ __forceinline__ double decide_pivot(const double *Fm, int ld, int p, int b1, const int8_t *sgn,
                                               double rho, double delta, double b1floor, int lane, double *D_out,
                                               double *dyn_out, DevCtl *ctl) {
    const int sp = sgn[p];
    const double fpp = Fm[(int64_t)p * ld + p];
    const double d = fpp + (sp < 0 ? -rho : delta);
    double b2 = 0.0;
    for (int j = p + 1 + lane; j < b1; j += 32) {
        if (sgn[j] != sp) continue;
        const double fjj = Fm[(int64_t)j * ld + j];
        if (!(sp * fjj > 0.0)) continue;
        const double fjp = Fm[(int64_t)p * ld + j];
        b2 = fmax(b2, fjp * fjp / fabs(fjj));
    }
    b2 = warp_max(b2);
    const double bnd = b1floor > b2 ? b1floor : b2;
    const double sd = sp * d;
    const double dn = sp * (sd > bnd ? sd : bnd);
    if (lane == 0) {
        *D_out = dn;
        *dyn_out = dn - d;
        if (!isfinite(d) || !isfinite(dn) || dn == 0.0) atomicOr(&ctl->status, kStatNonFinite);
    }
    return dn;
}

// ------------------------------------------------------------ small fronts
// One CTA per front, the whole front in shared memory.
template <int NT>
__global__ void __launch_bounds__(NT) k_small_fronts(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                      double *__restrict__ Dg, double *__restrict__ dyng,
                                                      DevCtl *ctl, const int32_t *__restrict__ list, int nb) {
    extern __shared__ double smem[];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    double *F = smem;                 // ld * f
    double *w = smem + (size_t)ld * f;  // f   (unscaled pivot column)
    double *dq = w + f;               // nb  (pivots of the current block)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
    const int8_t *sgn = P.sign + c0;
    const double b1floor = ctl->b1;
    for (int b0 = 0; b0 < k; b0 += nb) {
        const int b1 = min(b0 + nb, k);
        for (int p = b0; p < b1; p++) {
            if (warp == 0) {
                double dn = decide_pivot(F, ld, p, b1, sgn, V.rho, V.delta, b1floor, lane, &Dg[c0 + p],
                                         &dyng[c0 + p], ctl);
                if (lane == 0) dq[p - b0] = dn;
            }
            __syncthreads();
            const double dp = dq[p - b0];
            for (int i = p + 1 + tid; i < f; i += NT) {
                const double v = F[p * ld + i];
                w[i] = v;
                F[p * ld + i] = v / dp;
            }
            if (tid == 0) F[p * ld + p] = dp;
            __syncthreads();
            // rank-1 update of the remaining columns of the block, all rows
            for (int j = p + 1 + warp; j < b1; j += NT / 32) {
                const double wj = w[j];
                for (int i = j + lane; i < f; i += 32) F[j * ld + i] -= F[p * ld + i] * wj;
            }
            __syncthreads();
        }
        // trailing update of columns [b1, f) by the block's pivots
        for (int j = b1 + warp; j < f; j += NT / 32) {
            for (int i = j + lane; i < f; i += 32) {
                double acc = 0.0;
                for (int q = b0; q < b1; q++) acc += F[q * ld + i] * (F[q * ld + j] * dq[q - b0]);
                F[j * ld + i] -= acc;
            }
        }
        __syncthreads();
    }
    double *out = fronts + P.sn_off[s];
    for (int t = tid; t < sz; t += NT) out[t] = F[t];
}

// -------------------------------------------------------------- large fronts
// Assembly of columns [r0, r1) of front s into its slab in global memory.
__global__ void __launch_bounds__(256) k_large_assemble(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                         const PanelItem *__restrict__ items) {
    const PanelItem it = items[blockIdx.x];
    const int s = it.s, c_lo = it.r0, c_hi = it.r1;
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s];
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x;
    const int ncol = c_hi - c_lo;
    for (int t = tid; t < ncol * ld; t += 256) {
        const int jj = c_lo + t / ld, ii = t % ld;
        F[(int64_t)jj * ld + ii] = 0.0;
    }
    __syncthreads();
    if (c_lo < k) {
        const int64_t lo = (int64_t)c_lo * ld, hi = (int64_t)c_hi * ld;
        for (int64_t q = P.orig_ptr[s] + tid; q < P.orig_ptr[s + 1]; q += 256) {
            const int32_t dst = P.orig_dst[q];
            if (dst >= lo && dst < hi) F[dst] = orig_value(P, V, P.orig_src[q]);
        }
    }
    __syncthreads();
    for (int q = P.child_ptr[s]; q < P.child_ptr[s + 1]; q++) {
        const int c = P.child_list[q];
        const int kc = P.sn_k[c], ldc = P.sn_ld[c];
        const int cc = P.sn_f[c] - kc;
        const int32_t *map = P.relmap + P.map_off[c];
        // child columns whose parent column lies in [c_lo, c_hi): map is increasing
        int a = 0, b = cc;
        {
            int lo = 0, hi = cc;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (map[mid] < c_lo) lo = mid + 1;
                else hi = mid;
            }
            a = lo;
            lo = a;
            hi = cc;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (map[mid] < c_hi) lo = mid + 1;
                else hi = mid;
            }
            b = lo;
        }
        if (a < b) {
            const double *CB = fronts + P.sn_off[c] + (int64_t)kc * ldc + kc;
            const int warp = tid >> 5, lane = tid & 31;
            for (int jj = a + warp; jj < b; jj += 8) {
                const int pj = map[jj];
                for (int ii = jj + lane; ii < cc; ii += 32) F[(int64_t)pj * ld + map[ii]] += CB[(int64_t)jj * ldc + ii];
            }
        }
        __syncthreads();
    }
    (void)f;
}

// Panel [p0, p1) of front s: every CTA factorises the nb x nb diagonal block
// redundantly in shared memory (deterministic, identical results), then
// solves its rows [r0, r1) of the panel below it by forward substitution
// with L_DD and D (one reciprocal per pivot, W(q, p) = d_q L_pq staged in
// shared memory); the CTA whose r0 is the first row below the block writes
// the factorised diagonal block, D and the lifts.
__global__ void __launch_bounds__(kPanelRows) k_large_panel(DevPlan P, DevVals V, double *__restrict__ fronts,
                                                             double *__restrict__ Dg, double *__restrict__ dyng,
                                                             DevCtl *ctl, const PanelItem *__restrict__ items,
                                                             int p0, int nb) {
    __shared__ double Fd[32 * 33];
    __shared__ double Wd[32 * 33];
    __shared__ double wv[32];
    __shared__ double dq[32], inv[32];
    __shared__ double Dtmp[32], dyntmp[32];
    const PanelItem it = items[blockIdx.x];
    const int s = it.s;
    const int k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    const int p1 = min(p0 + nb, k);
    const int w = p1 - p0;
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int LDD = 33;
    for (int t = tid; t < w * w; t += kPanelRows) {
        const int jj = t / w, ii = t % w;
        Fd[jj * LDD + ii] = (ii >= jj) ? F[(int64_t)(p0 + jj) * ld + (p0 + ii)] : 0.0;
    }
    __syncthreads();
    const int8_t *sgn = P.sign + c0 + p0;
    const double b1floor = ctl->b1;
    if (warp == 0) {
        for (int p = 0; p < w; p++) {
            double dn = decide_pivot(Fd, LDD, p, w, sgn, V.rho, V.delta, b1floor, lane, &Dtmp[p], &dyntmp[p], ctl);
            if (lane == 0) dq[p] = dn;
            if (lane > p && lane < w) {
                const double v = Fd[p * LDD + lane];
                wv[lane] = v;
                Fd[p * LDD + lane] = v / dn;
            }
            __syncwarp();
            for (int j = p + 1; j < w; j++)
                if (lane >= j && lane < w) Fd[j * LDD + lane] -= Fd[p * LDD + lane] * wv[j];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int t = tid; t < w * w; t += kPanelRows) {
        const int q = t / w, p = t % w;
        Wd[q * LDD + p] = p > q ? dq[q] * Fd[q * LDD + p] : 0.0;
    }
    for (int t = tid; t < 32; t += kPanelRows) inv[t] = t < w ? 1.0 / dq[t] : 0.0;
    __syncthreads();
    for (int i = it.r0 + tid; i < it.r1; i += kPanelRows) {
        double li[32];
#pragma unroll
        for (int p = 0; p < 32; p++) li[p] = p < w ? F[(int64_t)(p0 + p) * ld + i] : 0.0;
#pragma unroll
        for (int q = 0; q < 32; q++) {
            li[q] *= inv[q];
#pragma unroll
            for (int p = q + 1; p < 32; p++) li[p] -= li[q] * Wd[q * LDD + p];
        }
#pragma unroll
        for (int p = 0; p < 32; p++)
            if (p < w) F[(int64_t)(p0 + p) * ld + i] = li[p];
    }
    if (it.r0 == p1) {  // exactly one item per (front, panel) starts at p1
        for (int t = tid; t < w * w; t += kPanelRows) {
            const int jj = t / w, ii = t % w;
            if (ii > jj) F[(int64_t)(p0 + jj) * ld + (p0 + ii)] = Fd[jj * LDD + ii];
            else if (ii == jj) F[(int64_t)(p0 + jj) * ld + (p0 + ii)] = dq[jj];
        }
        for (int t = tid; t < w; t += kPanelRows) {
            Dg[c0 + p0 + t] = Dtmp[t];
            dyng[c0 + p0 + t] = dyntmp[t];
        }
    }
}

// Trailing update of the lower part of columns [p1, f) by the panel
// [p0, p0+w): C(i, j) -= sum_q L(i,q) d_q L(j,q), one 64 x 64 tile per CTA.
__global__ void __launch_bounds__(256) k_large_update(DevPlan P, double *__restrict__ fronts,
                                                      const double *__restrict__ Dg,
                                                      const TileItem *__restrict__ items, int p0, int w) {
    __shared__ double As[32][65];
    __shared__ double Bs[32][65];
    const TileItem it = items[blockIdx.x];
    const int s = it.s;
    const int f = P.sn_f[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    w = min(w, P.sn_k[s] - p0);  // ragged last panel
    double *F = fronts + P.sn_off[s];
    const int tid = threadIdx.x;
    for (int t = tid; t < 32 * 64; t += 256) {
        const int q = t / 64, r = t % 64;
        const int i = it.i0 + r, j = it.j0 + r;
        const bool qa = q < w;
        As[q][r] = (qa && i < f) ? F[(int64_t)(p0 + q) * ld + i] : 0.0;
        Bs[q][r] = (qa && j < f) ? F[(int64_t)(p0 + q) * ld + j] * Dg[c0 + p0 + q] : 0.0;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads, 4 x 4 each
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
    for (int q = 0; q < w; q++) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; a++) av[a] = As[q][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; b++) bv[b] = Bs[q][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] += av[a] * bv[b];
    }
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int j = it.j0 + ty + 16 * b;
        if (j >= f) continue;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int i = it.i0 + tx + 16 * a;
            if (i < f && i >= j) F[(int64_t)j * ld + i] -= acc[a][b];
        }
    }
}

// ||K||_1 of the regularised augmented matrix (maximum absolute row sum of
// the symmetric matrix, fixed summation order per row); also checks that
// Theta is positive and finite.
__global__ void k_norm1(DevPlan P, DevVals V, DevCtl *ctl) {
    double mx = 0.0;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int64_t p = P.kp[i]; p < P.kp[i + 1]; p++) {
            const int64_t src = P.ksrc[p];
            double val;
            if (src >= 0) val = V.Ax[src];
            else if (src == kDualDiag) val = V.delta;
            else {
                const double th = V.theta[-1 - src];
                if (!(th > 0.0) || !isfinite(th)) bad = true;
                val = 1.0 / th + V.rho;
            }
            sum += fabs(val);
        }
        mx = fmax(mx, sum);
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&ctl->norm1, (unsigned long long)__double_as_longlong(mx));
    if (bad) atomicOr(&ctl->status, kStatNonFinite);
}

__global__ void k_set_b1(DevCtl *ctl, double eps_piv) { ctl->b1 = eps_piv * ctl->norm1; }

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

}  // namespace

void launch_small_fronts(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *dyn, DevCtl *ctl,
                         const int32_t *list, int32_t count, int32_t nb, int32_t maxf, cudaStream_t st) {
    if (count <= 0) return;
    const int ldmax = (maxf + 3) & ~3;
    const size_t smem = ((size_t)ldmax * maxf + maxf + 32) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_small_fronts<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    k_small_fronts<256><<<count, 256, smem, st>>>(P, V, fronts, D, dyn, ctl, list, nb);
}

void launch_large_assemble(const DevPlan &P, const DevVals &V, double *fronts, const PanelItem *items,
                           int32_t count, cudaStream_t st) {
    if (count <= 0) return;
    k_large_assemble<<<count, 256, 0, st>>>(P, V, fronts, items);
}

void launch_large_panel(const DevPlan &P, const DevVals &V, double *fronts, double *D, double *dyn, DevCtl *ctl,
                        const PanelItem *items, int32_t count, int32_t p0, int32_t nb, cudaStream_t st) {
    if (count <= 0) return;
    k_large_panel<<<count, kPanelRows, 0, st>>>(P, V, fronts, D, dyn, ctl, items, p0, nb);
}

void launch_large_update(const DevPlan &P, double *fronts, const double *D, const TileItem *items, int32_t count,
                         int32_t p0, int32_t w, cudaStream_t st) {
    if (count <= 0) return;
    k_large_update<<<count, 256, 0, st>>>(P, fronts, D, items, p0, w);
}

void launch_norm1(const DevPlan &P, const DevVals &V, DevCtl *ctl, double eps_piv, cudaStream_t st) {
    const int grid = (P.N + 255) / 256 < 608 ? (P.N + 255) / 256 : 608;
    k_norm1<<<grid > 0 ? grid : 1, 256, 0, st>>>(P, V, ctl);
    k_set_b1<<<1, 1, 0, st>>>(ctl, eps_piv);
}

void launch_factor_stats(const double *D, const double *dyn, int N, double large_reg, DevCtl *ctl, cudaStream_t st) {
    k_factor_stats<<<152, 256, 0, st>>>(D, dyn, N, large_reg, ctl);
}

}  // namespace ipm
