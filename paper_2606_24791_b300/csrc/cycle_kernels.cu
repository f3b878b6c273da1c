// sm_103a kernels of the LAMG+ solve phase: the cycle steps of Section 2 (colour-ordered
// Gauss-Seidel, residual, restriction P^T, prolongation P with caliber-2 rows, elimination
// transfers of Eq. 2, dense coarsest solve, mean-zero projection of Eq. 1) and the vector
// kernels of the flexible CG outer iteration.
//
// All of these are memory-bound (no step is a dense contraction): CSR rows are handled by
// groups of TPR lanes so that a group's loads of a row's column ids and values are
// contiguous, group sums are combined with warp shuffles, and every reduction is
// deterministic (fixed per-block partials, summed in a fixed order by the last block to
// finish, which is found with an atomic ticket, not a spin-wait).
#include <cuda_runtime.h>

#include "device.h"

namespace lamg {

constexpr int BS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of NV values over the block; the totals are valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) sh[k][w] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] = warp_sum(lane < nw ? sh[k][lane] : 0.0);
    }
    __syncthreads();
}

// Grid-wide deterministic sum: every block publishes its partials, the last block to arrive
// adds all partials in block order. Returns true in the last block, whose thread 0 holds the
// totals in v. Must be reached by every thread of every block.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], const Reduce red) {
    __shared__ bool last;
    __threadfence();  // publish this thread's global writes before the block signals
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) red.partials[k * RED_MAXG + blockIdx.x] = v[k];
        __threadfence();
        const unsigned t = atomicAdd(red.ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&red.partials[k * RED_MAXG + b]);
        v[k] = s;
    }
    block_sum<NV>(v);
    if (threadIdx.x == 0) *red.ticket = 0u;
    return true;
}

// Sum over a CSR row by a group of TPR lanes (all 32 lanes of the warp must call it).
template <int TPR>
__device__ __forceinline__ double row_sum(int e0, int e1, const int32_t *__restrict__ ci,
                                          const double *__restrict__ val, const double *x) {
    double s = 0.0;
    for (int e = e0; e < e1; e += TPR) s += val[e] * x[ci[e]];
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// ------------------------------------------------------------------------------- cycle steps

// One colour class [r0, r1) of Gauss-Seidel (Section 2): x_u = (b_u - sum_v A_uv x_v) / A_uu.
template <int TPR>
__global__ void __launch_bounds__(BS) k_gs(int r0, int r1, const int32_t *__restrict__ rp,
                                           const int32_t *__restrict__ ci,
                                           const double *__restrict__ val,
                                           const double *__restrict__ diag,
                                           const double *__restrict__ b, double *x) {
    const int g = r0 + (int)((blockIdx.x * (unsigned)BS + threadIdx.x) / TPR);
    const int sub = threadIdx.x % TPR;
    const bool ok = g < r1;
    const int e0 = ok ? rp[g] + sub : 0, e1 = ok ? rp[g + 1] : 0;
    const double s = row_sum<TPR>(e0, e1, ci, val, x);
    if (ok && sub == 0) x[g] = (b[g] - s) / diag[g];
}

// First sweep from x = 0: rows of colour 0 ([0, c1)) have no updated neighbours yet, so
// x_u = b_u / A_uu there; every other row starts at 0.
__global__ void k_gs_first(int n, int c1, const double *__restrict__ diag,
                           const double *__restrict__ b, double *x) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i >= n) return;
    x[i] = i < c1 ? b[i] / diag[i] : 0.0;
}

__global__ void k_zero(int n, double *x) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i < n) x[i] = 0.0;
}

// r = b - A x
template <int TPR>
__global__ void __launch_bounds__(BS) k_resid(int n, const int32_t *__restrict__ rp,
                                              const int32_t *__restrict__ ci,
                                              const double *__restrict__ val,
                                              const double *__restrict__ diag,
                                              const double *__restrict__ x,
                                              const double *__restrict__ b, double *r) {
    const int g = (int)((blockIdx.x * (unsigned)BS + threadIdx.x) / TPR);
    const int sub = threadIdx.x % TPR;
    const bool ok = g < n;
    const int e0 = ok ? rp[g] + sub : 0, e1 = ok ? rp[g + 1] : 0;
    const double s = row_sum<TPR>(e0, e1, ci, val, x);
    if (ok && sub == 0) r[g] = b[g] - (diag[g] * x[g] + s);
}

// Restriction b^c = P^T r (Section 2): segmented sum over the fine rows of each aggregate,
// caliber-2 rows contributing w or 1 - w.
template <int TPR>
__global__ void __launch_bounds__(BS) k_restrict(int nc, const int32_t *__restrict__ ptr,
                                                 const int32_t *__restrict__ row,
                                                 const double *__restrict__ w,
                                                 const double *__restrict__ r, double *bc) {
    const int a = (int)((blockIdx.x * (unsigned)BS + threadIdx.x) / TPR);
    const int sub = threadIdx.x % TPR;
    const bool ok = a < nc;
    const int e0 = ok ? ptr[a] + sub : 0, e1 = ok ? ptr[a + 1] : 0;
    const double s = row_sum<TPR>(e0, e1, row, w, r);
    if (ok && sub == 0) bc[a] = s;
}

// Prolongation x += P x^c: caliber-1 rows gather one coarse value, caliber-2 rows
// w x^c_a + (1 - w) x^c_b (Appendix A.2).
__global__ void k_prolong(int n, const int32_t *__restrict__ agg, const int32_t *__restrict__ agg2,
                          const double *__restrict__ wt, const double *__restrict__ xc, double *x) {
    const int u = blockIdx.x * BS + threadIdx.x;
    if (u >= n) return;
    const int b = agg2[u];
    double s;
    if (b < 0) {
        s = xc[agg[u]];
    } else {
        const double w = wt[u];
        s = (1.0 - w) * xc[b];
        if (w != 0.0) s = w * xc[agg[u]] + s;
    }
    x[u] += s;
}

// Elimination restriction (Eq. 2): b^c_i = b_i + sum_f (P_F)_{f,i} b_f over the F neighbours.
__global__ void k_elim_restrict(int nc, const int32_t *__restrict__ ptr, const int32_t *__restrict__ f,
                                const double *__restrict__ pv, const double *__restrict__ b, double *bc) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i >= nc) return;
    const double *bF = b + nc;
    double s = b[i];
    for (int e = ptr[i]; e < ptr[i + 1]; e++) s += pv[e] * bF[f[e]];
    bc[i] = s;
}

// Elimination interpolation (Eq. 2): x_F = P_F x_C + b_F / A_FF, ELL-4 rows.
__global__ void k_elim_interp(int nc, int nF, const int32_t *__restrict__ col,
                              const double *__restrict__ pv, const double *__restrict__ dF,
                              const double *__restrict__ b, double *x) {
    const int t = blockIdx.x * BS + threadIdx.x;
    if (t >= nF) return;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int c = col[4 * t + j];
        if (c >= 0) s += pv[4 * t + j] * x[c];
    }
    x[nc + t] = s + b[nc + t] / dF[t];
}

// Coarsest level: x = A^+ b (one warp per row of the dense pseudo-inverse), then the mean-zero
// projection done by the last block.
__global__ void __launch_bounds__(BS) k_coarse(int n, const double *__restrict__ pinv,
                                               const double *__restrict__ b, double *x,
                                               const Reduce red) {
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * BS + threadIdx.x) >> 5, nwarps = (gridDim.x * BS) >> 5;
    double part[1] = {0.0};
    for (int i = wg; i < n; i += nwarps) {
        const double *row = pinv + (int64_t)i * n;
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s += row[j] * b[j];
        s = warp_sum(s);
        if (lane == 0) { x[i] = s; part[0] += s; }
    }
    if (grid_sum<1>(part, red)) {
        __shared__ double mean;
        if (threadIdx.x == 0) mean = part[0] / (double)n;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += BS) x[i] = __ldcg(&x[i]) - mean;
    }
}

// ------------------------------------------------------------------------------- outer CG

__global__ void k_gather(int n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                         double *dst) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i < n) dst[i] = src[perm[i]];
}

__global__ void k_scatter(int n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                          double *dst) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i < n) dst[perm[i]] = src[i];
}

// S_MEAN = (sum v) / n
__global__ void __launch_bounds__(BS) k_sum(int n, const double *__restrict__ v, const Reduce red) {
    double s[1] = {0.0};
    for (int i = blockIdx.x * BS + threadIdx.x; i < n; i += gridDim.x * BS) s[0] += v[i];
    if (grid_sum<1>(s, red) && threadIdx.x == 0) red.scal[S_MEAN] = s[0] / (double)n;
}

__global__ void k_sub_mean(int n, double *v, const Reduce red) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i < n) v[i] -= red.scal[S_MEAN];
}

// b <- b - mean(b) (kept in bkeep), S_BN2 = ||b||^2; x = p = zold = 0, S_RZ = 1.
__global__ void __launch_bounds__(BS) k_init_b(int n, double *r, double *bkeep, double *x, double *p,
                                               double *zold, const Reduce red) {
    const double m = red.scal[S_MEAN];
    double s[1] = {0.0};
    for (int i = blockIdx.x * BS + threadIdx.x; i < n; i += gridDim.x * BS) {
        const double v = r[i] - m;
        r[i] = v;
        bkeep[i] = v;
        x[i] = 0.0;
        p[i] = 0.0;
        zold[i] = 0.0;
        s[0] += v * v;
    }
    if (grid_sum<1>(s, red) && threadIdx.x == 0) {
        red.scal[S_BN2] = s[0];
        red.scal[S_RZ] = 1.0;
        red.scal[S_BMEAN] = m;
    }
}

// q = A p, S_ALPHA = S_RZ / (p . q)
template <int TPR>
__global__ void __launch_bounds__(BS) k_spmv_dot(int n, const int32_t *__restrict__ rp,
                                                 const int32_t *__restrict__ ci,
                                                 const double *__restrict__ val,
                                                 const double *__restrict__ diag,
                                                 const double *__restrict__ p, double *q,
                                                 const Reduce red) {
    const int groups = gridDim.x * (BS / TPR);
    const int sub = threadIdx.x % TPR;
    double pq[1] = {0.0};
    const int rounds = (n + groups - 1) / groups;
    int g = (int)((blockIdx.x * (unsigned)BS + threadIdx.x) / TPR);
    for (int it = 0; it < rounds; it++, g += groups) {
        const bool ok = g < n;
        const int e0 = ok ? rp[g] + sub : 0, e1 = ok ? rp[g + 1] : 0;
        const double s = row_sum<TPR>(e0, e1, ci, val, p);
        if (ok && sub == 0) {
            const double qi = diag[g] * p[g] + s;
            q[g] = qi;
            pq[0] += p[g] * qi;
        }
    }
    if (grid_sum<1>(pq, red) && threadIdx.x == 0)
        red.scal[S_ALPHA] = pq[0] != 0.0 ? red.scal[S_RZ] / pq[0] : 0.0;  // b = 0: nothing to do
}

// x += alpha p, r -= alpha q, S_RR = ||r||^2
__global__ void __launch_bounds__(BS) k_update_xr(int n, double *x, double *r, const double *__restrict__ p,
                                                  const double *__restrict__ q, const Reduce red) {
    const double a = red.scal[S_ALPHA];
    double s[1] = {0.0};
    for (int i = blockIdx.x * BS + threadIdx.x; i < n; i += gridDim.x * BS) {
        x[i] += a * p[i];
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        s[0] += ri * ri;
    }
    if (grid_sum<1>(s, red) && threadIdx.x == 0) red.scal[S_RR] = s[0];
}

// z -= mean(z); beta = r.(z - zold) / rz_old; rz = r.z (flexible CG, Polak-Ribiere form)
__global__ void __launch_bounds__(BS) k_proj_dots(int n, double *z, const double *__restrict__ zold,
                                                  const double *__restrict__ r, const Reduce red) {
    const double m = red.scal[S_MEAN];
    double s[2] = {0.0, 0.0};
    for (int i = blockIdx.x * BS + threadIdx.x; i < n; i += gridDim.x * BS) {
        const double zi = z[i] - m;
        z[i] = zi;
        s[0] += r[i] * (zi - zold[i]);
        s[1] += r[i] * zi;
    }
    if (grid_sum<2>(s, red) && threadIdx.x == 0) {
        red.scal[S_BETA] = red.scal[S_RZ] != 0.0 ? s[0] / red.scal[S_RZ] : 0.0;
        red.scal[S_RZ] = s[1];
    }
}

// p = z + beta p, zold = z
__global__ void k_update_p(int n, const double *__restrict__ z, double *p, double *zold, const Reduce red) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i >= n) return;
    const double beta = red.scal[S_BETA];
    const double zi = z[i];
    p[i] = zi + beta * p[i];
    zold[i] = zi;
}

// S_TRUE_RR = ||b - A x||^2
template <int TPR>
__global__ void __launch_bounds__(BS) k_true_resid(int n, const int32_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci,
                                                   const double *__restrict__ val,
                                                   const double *__restrict__ diag,
                                                   const double *__restrict__ x,
                                                   const double *__restrict__ b, const Reduce red) {
    const int groups = gridDim.x * (BS / TPR);
    const int sub = threadIdx.x % TPR;
    double acc[1] = {0.0};
    const int rounds = (n + groups - 1) / groups;
    int g = (int)((blockIdx.x * (unsigned)BS + threadIdx.x) / TPR);
    for (int it = 0; it < rounds; it++, g += groups) {
        const bool ok = g < n;
        const int e0 = ok ? rp[g] + sub : 0, e1 = ok ? rp[g + 1] : 0;
        const double s = row_sum<TPR>(e0, e1, ci, val, x);
        if (ok && sub == 0) {
            const double ri = b[g] - (diag[g] * x[g] + s);
            acc[0] += ri * ri;
        }
    }
    if (grid_sum<1>(acc, red) && threadIdx.x == 0) red.scal[S_TRUE_RR] = acc[0];
}

// ------------------------------------------------------------------------------- launchers

static inline unsigned blocks(int64_t work) { return (unsigned)((work + BS - 1) / BS); }
static inline unsigned red_blocks(int64_t work) {
    int64_t b = (work + BS - 1) / BS;
    if (b < 1) b = 1;
    return (unsigned)(b > RED_MAXG ? RED_MAXG : b);
}

int choose_tpr(double avg_row) {
    int t = 1;
    while (t < 32 && 2.0 * t < avg_row) t *= 2;
    return t;
}

#define TPR_DISPATCH(tpr, KERNEL, GRID, ...)                                  \
    switch (tpr) {                                                            \
        case 1: KERNEL<1><<<GRID(1), BS, 0, s>>>(__VA_ARGS__); break;         \
        case 2: KERNEL<2><<<GRID(2), BS, 0, s>>>(__VA_ARGS__); break;         \
        case 4: KERNEL<4><<<GRID(4), BS, 0, s>>>(__VA_ARGS__); break;         \
        case 8: KERNEL<8><<<GRID(8), BS, 0, s>>>(__VA_ARGS__); break;         \
        case 16: KERNEL<16><<<GRID(16), BS, 0, s>>>(__VA_ARGS__); break;      \
        default: KERNEL<32><<<GRID(32), BS, 0, s>>>(__VA_ARGS__); break;      \
    }

void launch_op(const Op &op, std::vector<DevLevel> &lv, const Reduce &red, cudaStream_t s) {
    DevLevel &L = lv[op.level];
    const int n = (int)L.n;
    switch (op.kind) {
        case OP_GS_FIRST:
            k_gs_first<<<blocks(n), BS, 0, s>>>(n, (int)L.cptr[1], L.diag, L.b, L.x);
            break;
        case OP_ZERO:
            k_zero<<<blocks(n), BS, 0, s>>>(n, L.x);
            break;
        case OP_GS: {
            const int r0 = (int)L.cptr[op.colour], r1 = (int)L.cptr[op.colour + 1];
            const int64_t rows = r1 - r0;
            if (rows <= 0) break;
#define GRID_GS(T) blocks(rows * (T))
            TPR_DISPATCH(L.tpr, k_gs, GRID_GS, r0, r1, L.rp, L.ci, L.val, L.diag, L.b, L.x);
#undef GRID_GS
            break;
        }
        case OP_RESID: {
#define GRID_R(T) blocks((int64_t)n * (T))
            TPR_DISPATCH(L.tpr, k_resid, GRID_R, n, L.rp, L.ci, L.val, L.diag, L.x, L.b, L.r);
#undef GRID_R
            break;
        }
        case OP_RESTRICT: {
            DevLevel &Cl = lv[op.level + 1];
            const int nc = (int)L.nc;
#define GRID_P(T) blocks((int64_t)nc * (T))
            TPR_DISPATCH(L.pt_tpr, k_restrict, GRID_P, nc, L.pt_ptr, L.pt_row, L.pt_w, L.r, Cl.b);
#undef GRID_P
            break;
        }
        case OP_PROLONG:
            k_prolong<<<blocks(n), BS, 0, s>>>(n, L.agg, L.agg2, L.wt, lv[op.level + 1].x, L.x);
            break;
        case OP_ELIM_RESTRICT:
            k_elim_restrict<<<blocks(L.nc), BS, 0, s>>>((int)L.nc, L.pft_ptr, L.pft_f, L.pft_val, L.b,
                                                        lv[op.level + 1].b);
            break;
        case OP_ELIM_INTERP:
            if (L.nF > 0)
                k_elim_interp<<<blocks(L.nF), BS, 0, s>>>((int)L.nc, (int)L.nF, L.pf_col, L.pf_val, L.dF,
                                                          L.b, L.x);
            break;
        case OP_COARSE:
            k_coarse<<<red_blocks((int64_t)n * 32), BS, 0, s>>>(n, L.pinv, L.b, L.x, red);
            break;
    }
}

void launch_gather(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t s) {
    k_gather<<<blocks(n), BS, 0, s>>>((int)n, perm, src, dst);
}

void launch_scatter(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t s) {
    k_scatter<<<blocks(n), BS, 0, s>>>((int)n, perm, src, dst);
}

void launch_sum(int64_t n, const double *v, const Reduce &red, cudaStream_t s) {
    k_sum<<<red_blocks(n), BS, 0, s>>>((int)n, v, red);
}

void launch_sub_mean(int64_t n, double *v, const Reduce &red, cudaStream_t s) {
    k_sub_mean<<<blocks(n), BS, 0, s>>>((int)n, v, red);
}

void launch_init_b(int64_t n, double *r, double *bkeep, double *x, double *p, double *zold,
                   const Reduce &red, cudaStream_t s) {
    k_init_b<<<red_blocks(n), BS, 0, s>>>((int)n, r, bkeep, x, p, zold, red);
}

void launch_spmv_dot(const DevLevel &L, const double *p, double *q, const Reduce &red, cudaStream_t s) {
    const int n = (int)L.n;
#define GRID_S(T) red_blocks((int64_t)n * (T))
    TPR_DISPATCH(L.tpr, k_spmv_dot, GRID_S, n, L.rp, L.ci, L.val, L.diag, p, q, red);
#undef GRID_S
}

void launch_update_xr(int64_t n, double *x, double *r, const double *p, const double *q,
                      const Reduce &red, cudaStream_t s) {
    k_update_xr<<<red_blocks(n), BS, 0, s>>>((int)n, x, r, p, q, red);
}

void launch_proj_dots(int64_t n, double *z, const double *zold, const double *r, const Reduce &red,
                      cudaStream_t s) {
    k_proj_dots<<<red_blocks(n), BS, 0, s>>>((int)n, z, zold, r, red);
}

void launch_update_p(int64_t n, const double *z, double *p, double *zold, const Reduce &red,
                     cudaStream_t s) {
    k_update_p<<<blocks(n), BS, 0, s>>>((int)n, z, p, zold, red);
}

void launch_true_resid(const DevLevel &L, const double *x, const double *b, const Reduce &red,
                       cudaStream_t s) {
    const int n = (int)L.n;
#define GRID_T(T) red_blocks((int64_t)n * (T))
    TPR_DISPATCH(L.tpr, k_true_resid, GRID_T, n, L.rp, L.ci, L.val, L.diag, x, b, red);
#undef GRID_T
}

}  // namespace lamg
