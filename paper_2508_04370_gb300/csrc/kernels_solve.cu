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
// Columns are eliminated in blocks of 32: the 32 x 32 diagonal block of L is
// staged in shared memory for the dependent triangle steps (one warp), then
// all threads apply the block to the rows below it.
__global__ void __launch_bounds__(kSolveThreads) k_forward(DevPlan P, const double *__restrict__ fronts,
                                                            const double *__restrict__ D, double *__restrict__ x,
                                                            double *__restrict__ upd,
                                                            const int32_t *__restrict__ list) {
    extern __shared__ double v[];
    __shared__ double Lb[32 * 33];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    const double *L = fronts + P.sn_off[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
    for (int b0 = 0; b0 < k; b0 += 32) {
        const int b1 = min(b0 + 32, k), w = b1 - b0;
        for (int t = tid; t < w * w; t += kSolveThreads) {
            const int jj = t / w, ii = t - jj * w;
            if (ii > jj) Lb[jj * 33 + ii] = L[(int64_t)(b0 + jj) * ld + (b0 + ii)];
        }
        __syncthreads();
        if (warp == 0) {
            double vi = lane < w ? v[b0 + lane] : 0.0;
            for (int j = 0; j < w; j++) {
                const double yj = __shfl_sync(0xffffffffu, vi, j);
                if (lane > j && lane < w) vi -= Lb[j * 33 + lane] * yj;
            }
            if (lane < w) v[b0 + lane] = vi;
        }
        __syncthreads();
        for (int i = b1 + tid; i < f; i += kSolveThreads) {
            double acc = 0.0;
            for (int j = 0; j < w; j++) acc += L[(int64_t)(b0 + j) * ld + i] * v[b0 + j];
            v[i] -= acc;
        }
        __syncthreads();
    }
    for (int t = tid; t < f; t += kSolveThreads) {
        if (t < k) x[c0 + t] = v[t] / D[c0 + t];
        else upd[P.upd_off[s] + (t - k)] = v[t];
    }
}

// Backward: L^T z = y on the supernodes of one level (ancestors are final).
// Blocks of 32 columns from the last: first the contributions of all rows
// below the block (one warp per column, coalesced), then the triangle with
// the staged diagonal block, column by column (one warp, no reductions).
__global__ void __launch_bounds__(kSolveThreads) k_backward(DevPlan P, const double *__restrict__ fronts,
                                                             double *__restrict__ x,
                                                             const int32_t *__restrict__ list) {
    extern __shared__ double z[];
    __shared__ double Lb[32 * 33];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    const double *L = fronts + P.sn_off[s];
    const int32_t *rows = P.sn_rows + P.sn_rptr[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < f; t += kSolveThreads) z[t] = t < k ? x[c0 + t] : x[rows[t]];
    __syncthreads();
    const int nblk = (k + 31) / 32;
    for (int bb = nblk - 1; bb >= 0; bb--) {
        const int b0 = bb * 32, b1 = min(b0 + 32, k), w = b1 - b0;
        for (int t = tid; t < w * w; t += kSolveThreads) {
            const int jj = t / w, ii = t - jj * w;
            if (ii > jj) Lb[jj * 33 + ii] = L[(int64_t)(b0 + jj) * ld + (b0 + ii)];
        }
        for (int j = b0 + warp; j < b1; j += kSolveThreads / 32) {
            double acc = 0.0;
            for (int i = b1 + lane; i < f; i += 32) acc += L[(int64_t)j * ld + i] * z[i];
            acc = warp_sum(acc);
            if (lane == 0) z[j] -= acc;
        }
        __syncthreads();
        if (warp == 0) {
            double zi = lane < w ? z[b0 + lane] : 0.0;
            for (int j = w - 1; j > 0; j--) {
                const double zj = __shfl_sync(0xffffffffu, zi, j);
                if (lane < j) zi -= Lb[lane * 33 + j] * zj;
            }
            if (lane < w) z[b0 + lane] = zi;
        }
        __syncthreads();
    }
    for (int t = tid; t < k; t += kSolveThreads) x[c0 + t] = z[t];
}

// Sweeps of a factorisation with the pivoting of Sec. 4.5 (1x1 and 2x2
// blocks of D, interchanges among each front's fully-summed columns): as
// k_forward / k_backward, with the front's interchanges applied to its
// fully-summed entries before the forward substitution (position t takes the
// entry of local index lperm[t]) and undone after the backward one; D is
// applied block by block, a 2x2 block [e11 e21; e21 e22] by its inverse.
// Dynamic shared memory: f + k doubles.
__global__ void __launch_bounds__(kSolveThreads) k_forward_bk(DevPlan P, const double *__restrict__ fronts,
                                                               const double *__restrict__ D,
                                                               const double *__restrict__ Doff,
                                                               const int32_t *__restrict__ bsz,
                                                               const int32_t *__restrict__ lperm,
                                                               double *__restrict__ x, double *__restrict__ upd,
                                                               const int32_t *__restrict__ list) {
    extern __shared__ double v[];
    __shared__ double Lb[32 * 33];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    double *tmp = v + f;
    const double *L = fronts + P.sn_off[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
    for (int t = tid; t < k; t += kSolveThreads) tmp[t] = v[lperm[c0 + t]];
    __syncthreads();
    for (int t = tid; t < k; t += kSolveThreads) v[t] = tmp[t];
    __syncthreads();
    for (int b0 = 0; b0 < k; b0 += 32) {
        const int b1 = min(b0 + 32, k), w = b1 - b0;
        for (int t = tid; t < w * w; t += kSolveThreads) {
            const int jj = t / w, ii = t - jj * w;
            if (ii > jj) Lb[jj * 33 + ii] = L[(int64_t)(b0 + jj) * ld + (b0 + ii)];
        }
        __syncthreads();
        if (warp == 0) {
            double vi = lane < w ? v[b0 + lane] : 0.0;
            for (int j = 0; j < w; j++) {
                const double yj = __shfl_sync(0xffffffffu, vi, j);
                if (lane > j && lane < w) vi -= Lb[j * 33 + lane] * yj;
            }
            if (lane < w) v[b0 + lane] = vi;
        }
        __syncthreads();
        for (int i = b1 + tid; i < f; i += kSolveThreads) {
            double acc = 0.0;
            for (int j = 0; j < w; j++) acc += L[(int64_t)(b0 + j) * ld + i] * v[b0 + j];
            v[i] -= acc;
        }
        __syncthreads();
    }
    for (int t = tid; t < f; t += kSolveThreads) {
        if (t < k) {
            const int b = bsz[c0 + t];
            if (b == 1) {
                x[c0 + t] = v[t] / D[c0 + t];
            } else if (b == 2) {
                const double e11 = D[c0 + t], e21 = Doff[c0 + t], e22 = D[c0 + t + 1];
                const double det = e11 * e22 - e21 * e21;
                const double y0 = v[t], y1 = v[t + 1];
                x[c0 + t] = (e22 * y0 - e21 * y1) / det;
                x[c0 + t + 1] = (e11 * y1 - e21 * y0) / det;
            }
        } else {
            upd[P.upd_off[s] + (t - k)] = v[t];
        }
    }
}

__global__ void __launch_bounds__(kSolveThreads) k_backward_bk(DevPlan P, const double *__restrict__ fronts,
                                                                const int32_t *__restrict__ lperm,
                                                                double *__restrict__ x,
                                                                const int32_t *__restrict__ list) {
    extern __shared__ double z[];
    __shared__ double Lb[32 * 33];
    const int s = list[blockIdx.x];
    const int f = P.sn_f[s], k = P.sn_k[s], ld = P.sn_ld[s], c0 = P.sn_c0[s];
    const double *L = fronts + P.sn_off[s];
    const int32_t *rows = P.sn_rows + P.sn_rptr[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < f; t += kSolveThreads) z[t] = t < k ? x[c0 + t] : x[rows[t]];
    __syncthreads();
    const int nblk = (k + 31) / 32;
    for (int bb = nblk - 1; bb >= 0; bb--) {
        const int b0 = bb * 32, b1 = min(b0 + 32, k), w = b1 - b0;
        for (int t = tid; t < w * w; t += kSolveThreads) {
            const int jj = t / w, ii = t - jj * w;
            if (ii > jj) Lb[jj * 33 + ii] = L[(int64_t)(b0 + jj) * ld + (b0 + ii)];
        }
        for (int j = b0 + warp; j < b1; j += kSolveThreads / 32) {
            double acc = 0.0;
            for (int i = b1 + lane; i < f; i += 32) acc += L[(int64_t)j * ld + i] * z[i];
            acc = warp_sum(acc);
            if (lane == 0) z[j] -= acc;
        }
        __syncthreads();
        if (warp == 0) {
            double zi = lane < w ? z[b0 + lane] : 0.0;
            for (int j = w - 1; j > 0; j--) {
                const double zj = __shfl_sync(0xffffffffu, zi, j);
                if (lane < j) zi -= Lb[lane * 33 + j] * zj;
            }
            if (lane < w) z[b0 + lane] = zi;
        }
        __syncthreads();
    }
    for (int t = tid; t < k; t += kSolveThreads) x[c0 + lperm[c0 + t]] = z[t];
}

// --------------------------------------------------------------------------
// Persistent dependency-driven sweeps: one launch per forward or backward
// pass instead of one per tree level.  CTAs take work items from an atomic
// ticket in a topological order, critical path first.  Every dependency of a
// ticket holds a smaller ticket, taken earlier by a running CTA, so waiting
// can always make progress.  Waits are bounded: after S.spin_limit polls
// the CTA records kStatTimeout and carries on, so the launch always
// terminates (with a wrong result and the status set).
// Values produced by other CTAs of the same launch are read with ld.global.cg
// (L2, bypassing the non-coherent L1) and written with st.global.cg.
//
// Forward, supernode s (front rows t, k columns, blocks of 32 columns):
//   v_t  = b_t (t < k) + sum over children, ascending, of their contributions
//   y    = L11^-1 v[0:k),   x[c0:c0+k) = D^-1 y
//   u    = v[k:f) - L21 y   (contribution vector for the parent)
// Backward: z = x[c0:c0+k) - L21^T x[rows k..f),  z <- L11^-T z.
// A supernode with k <= 32 and a small L21 is one item.  Otherwise every
// 32-column block of L11 is an item of its own (fan-in: block b applies the
// finished y of blocks b' < b as they appear, then solves its diagonal
// block; backward in the mirror order, each block also forming its own
// columns of L21^T x), and in the forward L21 is cut into row chunks of
// kRectRows rows that apply the blocks of y as they appear.
__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void wait_count(const int32_t *cnt, int need, DevCtl *ctl, long long limit) {
    if (need <= 0) return;
    long long spins = 0;
    while (ld_acquire(cnt) < need) {
        if (++spins > limit) {
            atomicOr(&ctl->status, kStatTimeout);
            break;
        }
        __nanosleep(64);
    }
}

// The blocks of a split supernode pass their 32 values (y forward, z
// backward) to the next block of the chain through S.yv, filled before the
// sweep with a signalling-NaN pattern that no arithmetic result has: each
// value is stored once per sweep (relaxed, gpu scope), so a relaxed load that
// returns anything else has the final value, and the waiting block reads the
// data itself instead of a counter and then the data.
constexpr unsigned long long kUnset = 0x7FF4DEAD7FF4DEADull;

// Publishes one value for the chain.  The unset pattern itself can only
// come from an input copied through without arithmetic (a signalling NaN in
// a right-hand side); it goes out as the default NaN, so a waiting block
// never takes a written value for one still pending.
__device__ __forceinline__ void publish_value(double *p, double v) {
    long long b = __double_as_longlong(v);
    if ((unsigned long long)b == kUnset) b = 0x7FF8000000000000ll;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}

__device__ __forceinline__ double ld_relaxed(const double *p) {
    long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return __longlong_as_double(v);
}

// One warp: lane q < wp returns p[q] once it is set (0 beyond wp); gives up
// after `limit` rounds like wait_count.
__device__ __forceinline__ double poll_block(const double *p, int wp, DevCtl *ctl, long long limit) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    bool pending = lane < wp;
    long long spins = 0;
    while (true) {
        if (pending) {
            v = ld_relaxed(p + lane);
            pending = (unsigned long long)__double_as_longlong(v) == kUnset;
        }
        if (!__any_sync(0xffffffffu, pending)) break;
        if (++spins > limit) {
            if (lane == 0) atomicOr(&ctl->status, kStatTimeout);
            break;
        }
        __nanosleep(64);
    }
    return lane < wp ? v : 0.0;
}

// Take the next ticket (thread 0) and publish its item and node to the CTA.
__device__ __forceinline__ bool next_item(const SolveSched &S, const SolveItem *items, int nitems, SolveItem &it,
                                          SolveNode &nd, SolveItem *sh_it, SolveNode *sh_nd) {
    if (threadIdx.x == 0) {
        const int t = atomicAdd(S.sync, 1);
        SolveItem a{-1, -1};
        if (t < nitems) {
            a = items[t];
            if (a.r != kLeafGroup) *sh_nd = S.node[a.s];
        }
        *sh_it = a;
    }
    __syncthreads();
    it = *sh_it;
    if (it.s >= 0 && it.r != kLeafGroup) nd = *sh_nd;
    __syncthreads();
    return it.s >= 0;
}

// The last finished item of supernode s reports s to its parent (a
// supernode of one item reports directly).
__device__ __forceinline__ void finish_forward(const SolveNode &nd, int s, int32_t *done, int32_t *cnt) {
    if (nd.nblk + nd.nrect == 1) {
        if (nd.parent >= 0) atomicAdd(&cnt[nd.parent], 1);
        return;
    }
    const int old = atomicAdd(&done[s], 1);
    if (old == nd.nblk + nd.nrect - 1) {
        __threadfence();
        if (nd.parent >= 0) atomicAdd(&cnt[nd.parent], 1);
    }
}

// Row t of the front: its right-hand side (t < k) plus the children's
// contributions, children ascending.
__device__ __forceinline__ double gather_row(const SolveSched &S, const SolveNode &nd, const double *x,
                                             const double *upd, int t) {
    double a = t < nd.k ? x[nd.c0 + t] : 0.0;
    const int64_t e1 = S.gat_rp[nd.rptr + t + 1];
    for (int64_t e = S.gat_rp[nd.rptr + t]; e < e1; e++) a += __ldcg(upd + S.gat_src[e]);
    return a;
}

// Stage the strictly lower part of the w x w diagonal block at column b0.
__device__ __forceinline__ void stage_diag(double *Lb, const double *L, int ld, int b0, int w) {
    for (int q = threadIdx.x; q < w * w; q += kSolveThreads) {
        const int jj = q / w, ii = q - jj * w;
        if (ii > jj) Lb[jj * 33 + ii] = L[(int64_t)(b0 + jj) * ld + (b0 + ii)];
    }
}

// Warp 0: forward substitution with the unit lower diagonal block on v[0:w).
__device__ __forceinline__ void diag_forward(const double *Lb, double *v, int w) {
    const int lane = threadIdx.x & 31;
    double vi = lane < w ? v[lane] : 0.0;
    for (int j = 0; j < w; j++) {
        const double yj = __shfl_sync(0xffffffffu, vi, j);
        if (lane > j && lane < w) vi -= Lb[j * 33 + lane] * yj;
    }
    if (lane < w) v[lane] = vi;
}

// Warp 0: backward substitution with the transposed diagonal block on z[0:w).
__device__ __forceinline__ void diag_backward(const double *Lb, double *z, int w) {
    const int lane = threadIdx.x & 31;
    double zi = lane < w ? z[lane] : 0.0;
    for (int j = w - 1; j > 0; j--) {
        const double zj = __shfl_sync(0xffffffffu, zi, j);
        if (lane < j) zi -= Lb[lane * 33 + j] * zj;
    }
    if (lane < w) z[lane] = zi;
}

// Explicit inverse X = L11^-1 of the unit lower-triangular w x w diagonal
// block b of supernode s (w <= 32), one warp per block, computed once per
// factorisation: lane j builds column j by
//   X_jj = 1,   X_ij = -sum_{j <= t < i} L_it X_tj   (i > j),
// rows in increasing order.  Stored column-major 32 x 32 (X_ij at 32 j + i),
// zero above the diagonal, identity outside [0, w).  The sweeps then apply a
// block as a matrix-vector product spread over four warps instead of a
// substitution of w dependent steps.
constexpr int kInvWarps = 2;
__global__ void __launch_bounds__(32 * kInvWarps) k_diag_inverse(SolveSched S, const double *__restrict__ fronts,
                                                                 double *__restrict__ Linv,
                                                                 const InvItem *__restrict__ items, int count) {
    __shared__ double Ls[kInvWarps][32][33];  // [row i][column t] of the strictly lower block
    __shared__ double Xs[kInvWarps][32][33];  // [row t][column j] of X
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int idx = blockIdx.x * kInvWarps + wl;
    if (idx >= count) return;  // whole warps; no CTA barrier below
    const InvItem it = items[idx];
    const SolveNode nd = S.node[it.s];
    const int b0 = 32 * it.b, w = min(32, nd.k - b0), ld = nd.ld;
    const double *L = fronts + nd.off;
    for (int t = 0; t < 32; t++) {
        Ls[wl][lane][t] = (t < w && lane > t && lane < w) ? L[(int64_t)(b0 + t) * ld + b0 + lane] : 0.0;
        Xs[wl][t][lane] = t == lane ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int i = 1; i < w; i++) {
        double acc = 0.0;
        for (int t = 0; t < i; t++) acc += Ls[wl][i][t] * Xs[wl][t][lane];  // Xs[t][lane] = 0 for t < lane
        __syncwarp();
        if (lane < i) Xs[wl][i][lane] = -acc;
        __syncwarp();
    }
    double *X = Linv + it.dst;
    for (int j = 0; j < 32; j++) X[32 * j + lane] = Xs[wl][lane][j];
}

// Diagonal-block storage in Linv: a supernode with one block keeps its X
// (1024 doubles); one with several keeps, per block b, X_b, then
// W_b = X_b L_{b,b-1} (b >= 1) and V_b = L_{b+1,b} X_b (b + 1 < nblk), each
// 32 x 32 column-major, 3072 doubles per block.
__device__ __forceinline__ int64_t block_slot(const SolveNode &nd, int b) {
    return nd.inv + (int64_t)b * (nd.nblk > 1 ? 3072 : 1024);
}

// W_b and V_b of one block of a multi-block supernode (one CTA of 256
// threads, four outputs of each product per thread, 32 FMAs each), after
// k_diag_inverse has formed X_b.  With them the sweeps take the last
// dependency of a block (the neighbouring block finished just before) with
// one product: forward y_b = X_b v' - W_b y_{b-1}, backward
// z_b = X_b^T z'' - V_b^T z_{b+1}, where v' and z'' hold everything else.
__global__ void __launch_bounds__(256) k_pair_products(SolveSched S, const double *__restrict__ fronts,
                                                       double *__restrict__ Linv, const InvItem *__restrict__ items,
                                                       int count) {
    __shared__ double Xs[32][33];  // [row][column] of X_b
    __shared__ double Ls[32][33];  // [row][column] of the neighbouring L block
    const int tid = threadIdx.x;
    const InvItem it = items[blockIdx.x];
    const SolveNode nd = S.node[it.s];
    const int b = it.b, k = nd.k, ld = nd.ld;
    const double *L = fronts + nd.off;
    double *X = Linv + it.dst;
    for (int q = tid; q < 1024; q += 256) Xs[q & 31][q >> 5] = X[q];
    for (int pass = 0; pass < 2; pass++) {
        // pass 0: W_b = X_b L_{b,b-1} (rows 32b.., columns 32(b-1)..);
        // pass 1: V_b = L_{b+1,b} X_b (rows 32(b+1).., columns 32b..)
        if (pass == 0 && b == 0) continue;
        if (pass == 1 && b + 1 >= nd.nblk) continue;
        const int r0 = pass == 0 ? 32 * b : 32 * (b + 1), cbase = pass == 0 ? 32 * (b - 1) : 32 * b;
        __syncthreads();
        for (int q = tid; q < 1024; q += 256) {
            const int i = q & 31, j = q >> 5;  // L row r0 + i, column cbase + j
            Ls[i][j] = r0 + i < k ? L[(int64_t)(cbase + j) * ld + r0 + i] : 0.0;
        }
        __syncthreads();
        double *out = X + (pass == 0 ? 1024 : 2048);
        const int i = tid & 31;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int j = (tid >> 5) + 8 * c;
            double a = 0.0;
            if (pass == 0)
                for (int t = 0; t < 32; t++) a += Xs[i][t] * Ls[t][j];
            else
                for (int t = 0; t < 32; t++) a += Ls[i][t] * Xs[t][j];
            out[32 * j + i] = a;
        }
    }
}

// Leaves of the elimination tree with one block and f <= 32 (most of the
// supernodes of a nested-dissection or AMD tree) are processed one per
// warp, eight to a ticket (a leaf group), lane i = front row i.  Each
// computes what the single-item path below computes, in the same order of
// operations.
__device__ __forceinline__ void leaf_forward(const SolveSched &S, int s, const double *__restrict__ fronts,
                                             const double *__restrict__ Dinv, double *__restrict__ x, double *upd,
                                             int32_t *cnt) {
    const int lane = threadIdx.x & 31;
    const SolveNode nd = S.node[s];
    const double *L = fronts + nd.off;
    const int f = nd.f, k = nd.k, ld = nd.ld, c0 = nd.c0;
    double v = lane < k ? x[c0 + lane] : 0.0;
    const double dinv = lane < k ? Dinv[c0 + lane] : 0.0;
    double acc = 0.0;  // rows below the block: sum_j L_ij y_j, subtracted at the end
    for (int j = 0; j < k; j++) {
        const double yj = __shfl_sync(0xffffffffu, v, j);
        const double l = (lane > j && lane < f) ? L[(int64_t)j * ld + lane] : 0.0;
        if (lane < k) v -= l * yj;
        else acc += l * yj;
    }
    if (lane < k) x[c0 + lane] = v * dinv;
    else if (lane < f) __stcg(upd + nd.upd + (lane - k), v - acc);
    __syncwarp();
    if (lane == 0 && nd.parent >= 0) {
        __threadfence();
        atomicAdd(&cnt[nd.parent], 1);
    }
}

__device__ __forceinline__ void leaf_backward(const SolveSched &S, int s, const double *__restrict__ fronts,
                                              double *x, const int32_t *flag, DevCtl *ctl) {
    const int lane = threadIdx.x & 31;
    const SolveNode nd = S.node[s];
    const double *L = fronts + nd.off;
    const int f = nd.f, k = nd.k, ld = nd.ld, c0 = nd.c0;
    const int nrr = f - k;
    double z = lane < k ? __ldcg(x + c0 + lane) : 0.0;
    if (lane == 0 && nrr > 0) wait_count(&flag[nd.parent], 1, ctl, S.spin_limit);
    __syncwarp();
    const double xr = lane < nrr ? __ldcg(x + S.sn_rows[nd.rptr + k + lane]) : 0.0;  // x of the rows below
    // z_q -= sum over the rows below of L_iq x_i, in the single-item path's
    // eight row chunks (chunk sums added in chunk order)
    const int chunk = (nrr + 7) / 8;
    double sum = 0.0;
    for (int g = 0; g < 8; g++) {
        double part = 0.0;
        const int t0 = g * chunk, t1 = min(nrr, t0 + chunk);
        for (int t = t0; t < t1; t++) {
            const double xt = __shfl_sync(0xffffffffu, xr, t);
            if (lane < k) part += L[(int64_t)lane * ld + k + t] * xt;
        }
        sum = g == 0 ? part : sum + part;
    }
    if (lane < k) z -= sum;
    for (int j = k - 1; j > 0; j--) {
        const double zj = __shfl_sync(0xffffffffu, z, j);
        if (lane < j) z -= L[(int64_t)lane * ld + j] * zj;
    }
    if (lane < k) __stcg(x + c0 + lane, z);
}


// Stage the w x w inverse of a diagonal block (column-major 32 x 32 in
// Linv) as Lb[j * 33 + i] = X_ij.
__device__ __forceinline__ void stage_inverse(double *Lb, const double *X, int w) {
    for (int q = threadIdx.x; q < 32 * 32; q += kSolveThreads) {
        const int jj = q >> 5, ii = q & 31;
        if (ii < w && jj < w) Lb[jj * 33 + ii] = X[q];
    }
}

// v[0:w) <- X v with X = L11^-1 staged in Lb: warps 0-3 each sum eight
// columns for every row (lane = row), then warp 0 adds the four partial sums
// in warp order.  The caller separates this from the writes of v before it
// and the reads after it with CTA barriers.
__device__ __forceinline__ void apply_inverse_forward(const double *Lb, double *v, double (*part)[33], int w) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        double a = 0.0;
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const int j = 8 * warp + c;
            if (j < w) a += Lb[j * 33 + lane] * v[j];
        }
        part[warp][lane] = a;
    }
    __syncthreads();
    if (warp == 0 && lane < w) v[lane] = ((part[0][lane] + part[1][lane]) + part[2][lane]) + part[3][lane];
}

// z[0:w) <- X^T z: warps 0-3 each sum eight rows for every column (lane =
// column), then warp 0 adds the partial sums in warp order.
__device__ __forceinline__ void apply_inverse_backward(const double *Lb, double *z, double (*part)[33], int w) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        double a = 0.0;
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const int i = 8 * warp + c;
            if (i < w && lane < w) a += Lb[lane * 33 + i] * z[i];
        }
        part[warp][lane] = a;
    }
    __syncthreads();
    if (warp == 0 && lane < w) z[lane] = ((part[0][lane] + part[1][lane]) + part[2][lane]) + part[3][lane];
}

// t[0:w) -= M u (transpose = false) or M^T u (transpose = true) for the
// 32 x 32 product M staged in Mb (Mb[j * 33 + i] = M_ij) and the neighbour
// block's finished values u[0:32): warps 0-3 each sum eight terms, warp 0
// adds the four partial sums in warp order.  CTA barriers inside.
__device__ __forceinline__ void apply_pair(const double *Mb, double *t, const double *u, double (*part)[33], int w,
                                           bool transpose) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        double a = 0.0;
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const int q = 8 * warp + c;
            a += (transpose ? Mb[lane * 33 + q] : Mb[q * 33 + lane]) * u[q];
        }
        part[warp][lane] = a;
    }
    __syncthreads();
    if (warp == 0 && lane < w) t[lane] -= ((part[0][lane] + part[1][lane]) + part[2][lane]) + part[3][lane];
}

__global__ void __launch_bounds__(kSolveThreads, 5) k_forward_persistent(SolveSched S, const double *__restrict__ fronts,
                                                                       const double *__restrict__ Dinv,
                                                                       double *__restrict__ x, double *upd,
                                                                       DevCtl *ctl, const int32_t *skip) {
    extern __shared__ double v[];
    __shared__ double Lb[32 * 33];
    __shared__ double Wb[32 * 33];  // W_b of a multi-block supernode
    __shared__ double part[8][33];
    __shared__ double ys[2][32];
    __shared__ SolveItem sh_it;
    __shared__ SolveNode sh_nd;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (skip && *skip) return;
    int32_t *cnt = S.sync + 1, *done = cnt + S.nsuper;
    SolveItem it;
    SolveNode nd;
    while (next_item(S, S.fwd, S.nfwd, it, nd, &sh_it, &sh_nd)) {
        if (it.r == kLeafGroup) {
            const int ls = S.fwd_leaf[8 * it.s + warp];
            if (ls >= 0) leaf_forward(S, ls, fronts, Dinv, x, upd, cnt);
            __syncthreads();
            continue;
        }
        const int s = it.s;
        const int f = nd.f, k = nd.k, ld = nd.ld, c0 = nd.c0;
        const double *L = fronts + nd.off;
        const bool single = nd.nblk == 1 && nd.nrect == 0;
        if (it.r < 0) {
            const int b = -1 - it.r, b0 = 32 * b, w = min(32, k - b0);
            const bool inv = nd.inv >= 0;
            const bool pair = inv && b > 0 && nd.nblk > 1;  // last dependency through W_b
            // loads that do not depend on other items go out before the wait
            if (inv) stage_inverse(Lb, S.Linv + block_slot(nd, b), w);
            else stage_diag(Lb, L, ld, b0, w);
            if (pair) stage_inverse(Wb, S.Linv + block_slot(nd, b) + 1024, 32);
            const int nr = single ? f : w;  // rows this item gathers
            int64_t e0 = 0, e1 = 0, g[4] = {0, 0, 0, 0};
            double a0 = 0.0, dinv = 0.0;
            if (tid < nr) {
                e0 = S.gat_rp[nd.rptr + b0 + tid];
                e1 = S.gat_rp[nd.rptr + b0 + tid + 1];
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (e0 + q < e1) g[q] = S.gat_src[e0 + q];
                if (tid < w) {
                    a0 = x[c0 + b0 + tid];
                    dinv = Dinv[c0 + b0 + tid];
                }
            }
            if (tid == 0) wait_count(&cnt[s], nd.nchild, ctl, S.spin_limit);
            __syncthreads();
            if (tid < nr) {
                double a = a0;
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (e0 + q < e1) a += __ldcg(upd + g[q]);
                for (int64_t e = e0 + 4; e < e1; e++) a += __ldcg(upd + S.gat_src[e]);
                v[tid] = a;
            }
            for (int t = tid + kSolveThreads; t < nr; t += kSolveThreads) v[t] = gather_row(S, nd, x, upd, t);
            if (b > (pair ? 1 : 0)) {
                // fan-in of the finished blocks b' < b (b' < b - 1 with W_b): warp w
                // applies columns 4w..4w+3 of each
                double acc = 0.0;
                for (int bp = 0; bp < b - (pair ? 1 : 0); bp++) {
                    // (ys alternates: a round writes the buffer the round
                    // before last read, which every warp left at the last barrier)
                    double lv[4];  // independent of the wait: issued before it
#pragma unroll
                    for (int c = 0; c < 4; c++)
                        lv[c] = lane < w ? L[(int64_t)(32 * bp + 4 * warp + c) * ld + b0 + lane] : 0.0;
                    if (warp == 0) ys[bp & 1][lane] = poll_block(S.yv + c0 + 32 * bp, 32, ctl, S.spin_limit);
                    __syncthreads();
                    if (lane < w) {
#pragma unroll
                        for (int c = 0; c < 4; c++) acc += lv[c] * ys[bp & 1][4 * warp + c];
                    }
                }
                part[warp][lane] = acc;
                __syncthreads();
                if (warp == 0 && lane < w) {
                    double sum = part[0][lane];
#pragma unroll
                    for (int q = 1; q < kSolveThreads / 32; q++) sum += part[q][lane];
                    v[lane] -= sum;
                }
            }
            __syncthreads();
            if (inv) apply_inverse_forward(Lb, v, part, w);
            else if (warp == 0) diag_forward(Lb, v, w);
            __syncthreads();
            if (pair) {
                // y_b = X_b v' - W_b y_{b-1}, y_{b-1} being the last block to finish
                if (warp == 0) ys[0][lane] = poll_block(S.yv + c0 + 32 * (b - 1), 32, ctl, S.spin_limit);  // full block
                __syncthreads();
                apply_pair(Wb, v, ys[0], part, w, false);
                __syncthreads();
            }
            if (single) {
                for (int i = w + tid; i < f; i += kSolveThreads) {
                    double acc = 0.0;
                    for (int j = 0; j < w; j++) acc += L[(int64_t)j * ld + i] * v[j];
                    v[i] -= acc;
                }
                __syncthreads();
            }
            for (int q = tid; q < nr; q += kSolveThreads) {
                if (q < w) {
                    const double y = v[q];
                    if (!single) publish_value(S.yv + c0 + b0 + q, y);
                    x[c0 + b0 + q] = y * dinv;  // q == tid here
                } else {
                    __stcg(upd + nd.upd + (q - k), v[q]);
                }
            }
            // publish: the CTA barrier orders every thread's stores before
            // thread 0's fence, which makes them visible device-wide before its
            // counter updates (cumulativity)
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                finish_forward(nd, s, done, cnt);
            }
        } else {
            // rows [i0, i0 + 32) of L21: u_i = contributions_i - sum_j L_ij y_j,
            // applied block by block as the blocks of y finish; warp w takes
            // columns 4w..4w+3 of every block
            const int i = k + it.r * kRectRows + lane;
            const bool ok = i < f;
            if (tid == 0) wait_count(&cnt[s], nd.nchild, ctl, S.spin_limit);
            __syncthreads();
            double u0 = 0.0;
            if (warp == 0 && ok) u0 = gather_row(S, nd, x, upd, i);
            double acc = 0.0;
            for (int bp = 0; bp < nd.nblk; bp++) {
                const int wp = min(32, k - 32 * bp);
                double lv[4];  // independent of the wait: issued before it
#pragma unroll
                for (int c = 0; c < 4; c++)
                    lv[c] = (ok && 4 * warp + c < wp) ? L[(int64_t)(32 * bp + 4 * warp + c) * ld + i] : 0.0;
                if (warp == 0) ys[bp & 1][lane] = poll_block(S.yv + c0 + 32 * bp, wp, ctl, S.spin_limit);
                __syncthreads();
                if (ok) {
#pragma unroll
                    for (int c = 0; c < 4; c++)
                        if (4 * warp + c < wp) acc += lv[c] * ys[bp & 1][4 * warp + c];
                }
            }
            part[warp][lane] = acc;
            __syncthreads();
            if (warp == 0 && ok) {
                double sum = part[0][lane];
#pragma unroll
                for (int q = 1; q < kSolveThreads / 32; q++) sum += part[q][lane];
                __stcg(upd + nd.upd + (i - k), u0 - sum);
            }
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                finish_forward(nd, s, done, cnt);
            }
        }
    }
}

__global__ void __launch_bounds__(kSolveThreads, 5) k_backward_persistent(SolveSched S, const double *__restrict__ fronts,
                                                                        double *x, DevCtl *ctl, const int32_t *skip) {
    extern __shared__ double z[];  // [0, 32): the block; [32, 32 + f - k): x of the rows below
    __shared__ double Lb[32 * 33];
    __shared__ double Wb[32 * 33];  // V_b of a multi-block supernode
    __shared__ double part[8][33];
    __shared__ double zs[2][32];
    __shared__ SolveItem sh_it;
    __shared__ SolveNode sh_nd;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (skip && *skip) return;
    int32_t *flag = S.sync + 1, *tcnt = flag + S.nsuper;
    SolveItem it;
    SolveNode nd;
    while (next_item(S, S.bwd, S.nbwd, it, nd, &sh_it, &sh_nd)) {
        if (it.r == kLeafGroup) {
            const int ls = S.bwd_leaf[8 * it.s + warp];
            if (ls >= 0) leaf_backward(S, ls, fronts, x, flag, ctl);
            __syncthreads();
            continue;
        }
        const int s = it.s;
        const int f = nd.f, k = nd.k, ld = nd.ld, c0 = nd.c0;
        const double *L = fronts + nd.off;
        const int32_t *rows = S.sn_rows + nd.rptr;
        const int b = -1 - it.r, b0 = 32 * b, w = min(32, k - b0);
        const int nrr = f - k;  // rows below the supernode's columns
        // independent of other items: the diagonal block (or its inverse) and
        // this block's values after the forward sweep
        const bool inv = nd.inv >= 0;
        const bool pair = inv && nd.nblk > 1 && b + 1 < nd.nblk;  // last dependency through V_b
        if (inv) stage_inverse(Lb, S.Linv + block_slot(nd, b), w);
        else stage_diag(Lb, L, ld, b0, w);
        if (pair) stage_inverse(Wb, S.Linv + block_slot(nd, b) + 2048, 32);
        const double xb = (tid < w) ? __ldcg(x + c0 + b0 + tid) : 0.0;
        if (tid == 0 && nrr > 0) wait_count(&flag[nd.parent], 1, ctl, S.spin_limit);
        __syncthreads();
        for (int t = tid; t < nrr; t += kSolveThreads) z[32 + t] = __ldcg(x + rows[k + t]);
        __syncthreads();
        // z_q = x_q - sum_{i >= k} L_iq x_rows[i] - sum_{later blocks} L_iq z_i:
        // lane = column q of the block, warp g takes a slice of the rows below
        // and rows 4g..4g+3 of every later block
        double acc = 0.0;
        if (lane < w && nrr > 0) {
            const int chunk = (nrr + 7) / 8, t0 = warp * chunk, t1 = min(nrr, t0 + chunk);
            const double *Lc = L + (int64_t)(b0 + lane) * ld + k;
            for (int t = t0; t < t1; t++) acc += Lc[t] * z[32 + t];
        }
        for (int bp = nd.nblk - 1; bp > b + (pair ? 1 : 0); bp--) {
            const int wp = min(32, k - 32 * bp);
            double lv[4];  // independent of the wait: issued before it
            const double *Lc = L + (int64_t)(b0 + lane) * ld + 32 * bp + 4 * warp;
#pragma unroll
            for (int c = 0; c < 4; c++) lv[c] = (lane < w && 4 * warp + c < wp) ? Lc[c] : 0.0;
            if (warp == 0) zs[bp & 1][lane] = poll_block(S.yv + c0 + 32 * bp, wp, ctl, S.spin_limit);
            __syncthreads();
            if (lane < w) {
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if (4 * warp + c < wp) acc += lv[c] * zs[bp & 1][4 * warp + c];
            }
        }
        part[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && lane < w) {
            double sum = part[0][lane];
#pragma unroll
            for (int q = 1; q < kSolveThreads / 32; q++) sum += part[q][lane];
            z[lane] = xb - sum;
        }
        __syncthreads();
        if (inv) apply_inverse_backward(Lb, z, part, w);
        else if (warp == 0) diag_backward(Lb, z, w);
        __syncthreads();
        if (pair) {
            // z_b = X_b^T z'' - V_b^T z_{b+1}, z_{b+1} being the last block to finish
            const int wn = min(32, k - 32 * (b + 1));  // block b + 1 may be the last, partial one
            if (warp == 0) zs[0][lane] = poll_block(S.yv + c0 + 32 * (b + 1), wn, ctl, S.spin_limit);
            __syncthreads();
            apply_pair(Wb, z, zs[0], part, w, true);
            __syncthreads();
        }
        for (int q = tid; q < w; q += kSolveThreads) {
            __stcg(x + c0 + b0 + q, z[q]);
            if (nd.nblk > 1) publish_value(S.yv + c0 + b0 + q, z[q]);
        }
        // publish: the blocks of a split supernode count themselves done
        // (release); block 0, the last of the chain, acquires all of them
        // before it flags the supernode, so the children that read x rows of
        // any block after the flag see them
        __syncthreads();
        if (tid == 0) {
            if (nd.nblk > 1 && b > 0) {
                __threadfence();
                atomicAdd(&tcnt[s], 1);
            }
            if (b == 0) {
                wait_count(&tcnt[s], nd.nblk - 1, ctl, S.spin_limit);
                __threadfence();
                atomicExch(&flag[s], 1);
            }
        }
    }
}

// Before a persistent sweep: the ticket and the counters to zero, the block
// values of the chains to the unset pattern.
__global__ void k_sweep_reset(int32_t *__restrict__ sync, int32_t ncnt, double *__restrict__ yv, int32_t nyv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncnt || i < nyv; i += gridDim.x * blockDim.x) {
        if (i < ncnt) sync[i] = 0;
        if (i < nyv) yv[i] = __longlong_as_double((long long)kUnset);
    }
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
                              double *__restrict__ dx, double *__restrict__ dy, int form) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int o = perm[i];
        if (form == 2) dy[o] = x[i];
        else if (o < n) dx[o] = x[i];
        else dy[o - n] = x[i];
    }
}

// r = f - K x, ad = |K||x|, ae = |K|e in the factorisation order; also the
// running max of |x| (ctl->dinf, as ordered bits of a non-negative double).
__global__ void k_residual(DevPlan P, DevVals V, const double *__restrict__ f, const double *__restrict__ x,
                           double *__restrict__ r, double *__restrict__ ad, double *__restrict__ ae, DevCtl *ctl,
                           const int32_t *skip) {
    if (skip && *skip) return;
    double xm = 0.0;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
        xm = fmax(xm, fabs(x[i]));
        if (P.kp[i + 1] - P.kp[i] > kLongColumn) continue;  // k_residual_long
        double s = 0.0, sa = 0.0, se = 0.0;
        for (int64_t p = P.kp[i]; p < P.kp[i + 1]; p++) {
            const int64_t src = P.ksrc[p];
            double val;
            if (P.form == 2) val = V.nev[src] + (P.kj[p] == i ? V.delta : 0.0);
            else if (src >= 0) val = V.Ax[src];
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
    }
    xm = warp_max(xm);
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&ctl->dinf, (unsigned long long)__double_as_longlong(xm));
    if (bad) atomicOr(&ctl->status, kStatNonFinite);
}

// The rows of K longer than kLongColumn (dense rows of A), one CTA each:
// thread t sums the t-th of 256 contiguous runs of the row in entry order,
// the runs' sums are added pairwise in a fixed tree.
__global__ void __launch_bounds__(256) k_residual_long(DevPlan P, DevVals V, const double *__restrict__ f,
                                                       const double *__restrict__ x, double *__restrict__ r,
                                                       double *__restrict__ ad, double *__restrict__ ae, DevCtl *ctl,
                                                       const int32_t *skip) {
    if (skip && *skip) return;
    __shared__ double ps[256], pa[256], pe[256];
    const int i = P.long_cols[blockIdx.x];
    const int64_t p0 = P.kp[i], n = P.kp[i + 1] - p0;
    const int64_t run = (n + 255) / 256;
    const int64_t a = p0 + run * threadIdx.x, b = min(a + run, p0 + n);
    double s = 0.0, sa = 0.0, se = 0.0;
    for (int64_t p = a; p < b; p++) {
        const int64_t src = P.ksrc[p];
        double val;
        if (P.form == 2) val = V.nev[src] + (P.kj[p] == i ? V.delta : 0.0);
        else if (src >= 0) val = V.Ax[src];
        else if (src == kDualDiag) val = V.delta;
        else val = -(1.0 / V.theta[-1 - src] + V.rho);
        const double xj = x[P.kj[p]];
        s += val * xj;
        sa += fabs(val) * fabs(xj);
        se += fabs(val);
    }
    ps[threadIdx.x] = s;
    pa[threadIdx.x] = sa;
    pe[threadIdx.x] = se;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            ps[threadIdx.x] += ps[threadIdx.x + h];
            pa[threadIdx.x] += pa[threadIdx.x + h];
            pe[threadIdx.x] += pe[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ri = f[i] - ps[0];
        if (!isfinite(ri)) atomicOr(&ctl->status, kStatNonFinite);
        r[i] = ri;
        ad[i] = pa[0];
        ae[i] = pe[0];
    }
}

// omega = max_i |r_i| / den_i, den_i = (|K||x| + |f|)_i, replaced by
// (|K||x| + ||x||_inf |K|e)_i when den_i <= 1000 N eps (ae_i ||x||_inf + |f_i|);
// a NaN residual or denominator makes omega infinite.
__global__ void k_omega(int N, const double *__restrict__ r, const double *__restrict__ ad,
                        const double *__restrict__ ae, const double *__restrict__ f, DevCtl *ctl,
                        const int32_t *skip) {
    if (skip && *skip) return;
    const double dinf = ctl->dinf;
    const double eps = 2.220446049250313e-16;
    double w = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double den = ad[i] + fabs(f[i]);
        const double tau = 1000.0 * N * eps * (ae[i] * dinf + fabs(f[i]));
        if (den <= tau) den = ad[i] + dinf * ae[i];
        const double num = fabs(r[i]);
        double wi = den > 0.0 ? num / den : (num > 0.0 ? INFINITY : 0.0);
        if (isnan(num) || isnan(den) || isnan(wi)) wi = INFINITY;  // a non-finite residual is no backward error
        w = fmax(w, wi);
    }
    w = warp_max(w);
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&ctl->omega, (unsigned long long)__double_as_longlong(w));
}

__global__ void k_axpy(double *__restrict__ x, const double *__restrict__ c, int N, const int32_t *skip) {
    if (skip && *skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) x[i] += c[i];
}

// Device-side refinement control (used when the solve is captured in a CUDA
// graph and no host decision is possible).  After the first residual:
// best = x, omega_best = omega, done = omega <= target.  After step k:
// keep x as best if omega improved; done once omega <= target, omega failed
// to halve, or k = max_steps.  Kernels of later steps exit at entry when done.
__global__ void k_refine_init(DevCtl *ctl, double target, int max_steps) {
    const double w = ctl->omega;
    ctl->omega_best = w;
    ctl->omega_hist[0] = w;
    ctl->steps = 0;
    ctl->gmres_iters = 0;
    ctl->improved = 1;
    ctl->done = (w <= target || max_steps <= 0) ? 1 : 0;
}

__global__ void k_refine_step(DevCtl *ctl, double target, int step, int max_steps) {
    if (ctl->done) {
        ctl->improved = 0;
        return;
    }
    const double w = ctl->omega;
    ctl->steps = step;
    if (step < 16) ctl->omega_hist[step] = w;
    const bool halved = w <= 0.5 * ctl->omega_best;
    ctl->improved = w < ctl->omega_best ? 1 : 0;
    if (ctl->improved) ctl->omega_best = w;
    ctl->done = (!halved || ctl->omega_best <= target || step >= max_steps) ? 1 : 0;
}

__global__ void k_refine_finish(DevCtl *ctl, double target) {
    if (ctl->omega_best > target) atomicOr(&ctl->status, kStatRefineFail);
}

// dst = src when flag == nullptr or (*flag != 0) != invert
__global__ void k_copy_if(double *__restrict__ dst, const double *__restrict__ src, int N, const int32_t *flag,
                          int invert) {
    if (flag && ((*flag != 0) == (invert != 0))) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

__global__ void k_clear_norms(DevCtl *ctl, const int32_t *skip) {
    if (skip && *skip) return;
    ctl->dinf = 0.0;
    ctl->omega = 0.0;
}

}  // namespace

void launch_forward(const DevPlan &P, const double *fronts, const double *D, double *x, double *upd,
                    const int32_t *list, int32_t count, int32_t maxf, cudaStream_t st) {
    if (count <= 0) return;
    static uint64_t attr = 0;
    if (first_on_device(attr)) {
        cudaFuncSetAttribute(k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmemLimit);
        cudaFuncSetAttribute(k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmemLimit);
    }
    k_forward<<<count, kSolveThreads, (size_t)maxf * sizeof(double), st>>>(P, fronts, D, x, upd, list);
}

void launch_backward(const DevPlan &P, const double *fronts, double *x, const int32_t *list, int32_t count,
                     int32_t maxf, cudaStream_t st) {
    if (count <= 0) return;
    k_backward<<<count, kSolveThreads, (size_t)maxf * sizeof(double), st>>>(P, fronts, x, list);
}

const void *persistent_probe_kernel() { return (const void *)k_forward_persistent; }

void launch_diag_inverse(const SolveSched &S, const double *fronts, double *Linv, const InvItem *items,
                         int32_t count, const InvItem *pairs, int32_t npairs, cudaStream_t st) {
    if (count <= 0) return;
    k_diag_inverse<<<(count + kInvWarps - 1) / kInvWarps, 32 * kInvWarps, 0, st>>>(S, fronts, Linv, items, count);
    if (npairs > 0) k_pair_products<<<npairs, 256, 0, st>>>(S, fronts, Linv, pairs, npairs);
}

void launch_forward_bk(const DevPlan &P, const double *fronts, const double *D, const double *Doff,
                       const int32_t *bsz, const int32_t *lperm, double *x, double *upd, const int32_t *list,
                       int32_t count, int32_t maxf, cudaStream_t st) {
    if (count <= 0) return;
    static uint64_t attr = 0;
    if (first_on_device(attr)) {
        cudaFuncSetAttribute(k_forward_bk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmemLimit);
        cudaFuncSetAttribute(k_backward_bk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmemLimit);
    }
    k_forward_bk<<<count, kSolveThreads, 2 * (size_t)maxf * sizeof(double), st>>>(P, fronts, D, Doff, bsz, lperm, x,
                                                                                  upd, list);
}

void launch_backward_bk(const DevPlan &P, const double *fronts, const int32_t *lperm, double *x,
                        const int32_t *list, int32_t count, int32_t maxf, cudaStream_t st) {
    if (count <= 0) return;
    k_backward_bk<<<count, kSolveThreads, (size_t)maxf * sizeof(double), st>>>(P, fronts, lperm, x, list);
}

void launch_sweep_reset(const SolveSched &S, int32_t ncnt, cudaStream_t st) {
    const int grid = (S.nyv + 255) / 256 < 304 ? (S.nyv + 255) / 256 : 304;
    k_sweep_reset<<<grid > 0 ? grid : 1, 256, 0, st>>>(S.sync, ncnt, S.yv, S.nyv);
}

void launch_forward_persistent(const SolveSched &S, const double *fronts, const double *Dinv, double *x, double *upd,
                               int32_t maxf, int32_t grid, DevCtl *ctl, cudaStream_t st, const int32_t *skip) {
    static uint64_t attr = 0;
    if (first_on_device(attr)) {
        cudaFuncSetAttribute(k_forward_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmemLimit);
        cudaFuncSetAttribute(k_backward_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmemLimit);
    }
    // sync[0] = ticket; then per supernode: finished children, finished items
    launch_sweep_reset(S, 2 * S.nsuper + 1, st);
    const size_t smem = (size_t)(maxf > kRectRows ? maxf : kRectRows) * sizeof(double);
    k_forward_persistent<<<grid, kSolveThreads, smem, st>>>(S, fronts, Dinv, x, upd, ctl, skip);
}

void launch_backward_persistent(const SolveSched &S, const double *fronts, double *x, int32_t maxf, int32_t grid,
                                DevCtl *ctl, cudaStream_t st, const int32_t *skip) {
    // sync[0] = ticket; then per supernode: done flag, finished blocks
    launch_sweep_reset(S, 2 * S.nsuper + 1, st);
    const size_t smem = (size_t)(maxf + 32) * sizeof(double);
    k_backward_persistent<<<grid, kSolveThreads, smem, st>>>(S, fronts, x, ctl, skip);
}

void launch_permute_in(const DevPlan &P, const double *r7, const double *r1, double *f, cudaStream_t st) {
    k_permute_in<<<(P.N + 255) / 256, 256, 0, st>>>(P.perm, P.N, P.n, r7, r1, f, P.form);
}

void launch_permute_out(const DevPlan &P, const double *x, double *dx, double *dy, cudaStream_t st) {
    k_permute_out<<<(P.N + 255) / 256, 256, 0, st>>>(P.perm, P.N, P.n, x, dx, dy, P.form);
}

void launch_residual_omega(const DevPlan &P, const DevVals &V, const double *f, const double *x, double *r,
                           double *ad, double *ae, DevCtl *ctl, cudaStream_t st, const int32_t *skip) {
    const int grid = (P.N + 255) / 256 < 608 ? (P.N + 255) / 256 : 608;
    if (!skip) {
        cudaMemsetAsync(&ctl->dinf, 0, sizeof(double), st);
        cudaMemsetAsync(&ctl->omega, 0, sizeof(double), st);
    } else {
        k_clear_norms<<<1, 1, 0, st>>>(ctl, skip);
    }
    k_residual<<<grid, 256, 0, st>>>(P, V, f, x, r, ad, ae, ctl, skip);
    if (P.nlong > 0) k_residual_long<<<P.nlong, 256, 0, st>>>(P, V, f, x, r, ad, ae, ctl, skip);
    k_omega<<<grid, 256, 0, st>>>(P.N, r, ad, ae, f, ctl, skip);
}

void launch_omega_only(int32_t N, const double *r, const double *ad, const double *ae, const double *f, DevCtl *ctl,
                       cudaStream_t st) {
    const int grid = (N + 255) / 256 < 608 ? (N + 255) / 256 : 608;
    k_omega<<<grid > 0 ? grid : 1, 256, 0, st>>>(N, r, ad, ae, f, ctl, nullptr);
}

void launch_axpy(double *x, const double *c, int32_t N, cudaStream_t st, const int32_t *skip) {
    k_axpy<<<(N + 255) / 256 < 608 ? (N + 255) / 256 : 608, 256, 0, st>>>(x, c, N, skip);
}

void launch_refine_init(DevCtl *ctl, double target, int32_t max_steps, cudaStream_t st) {
    k_refine_init<<<1, 1, 0, st>>>(ctl, target, max_steps);
}

void launch_refine_step(DevCtl *ctl, double target, int32_t step, int32_t max_steps, cudaStream_t st) {
    k_refine_step<<<1, 1, 0, st>>>(ctl, target, step, max_steps);
}

void launch_refine_finish(DevCtl *ctl, double target, cudaStream_t st) { k_refine_finish<<<1, 1, 0, st>>>(ctl, target); }

void launch_copy_if(double *dst, const double *src, int32_t N, const int32_t *flag, int32_t invert, cudaStream_t st) {
    k_copy_if<<<(N + 255) / 256 < 608 ? (N + 255) / 256 : 608, 256, 0, st>>>(dst, src, N, flag, invert);
}

}  // namespace ipm
