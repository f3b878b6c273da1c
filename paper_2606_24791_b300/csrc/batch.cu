// Multi-RHS solves in SpMM form and the FP32 cycle (lamg_solve_batch; lamg_solve with
// precision LAMG_FP32).
//
// k right-hand sides are stored row-major (entry (u, j) at u*k + j), so one step of the cycle
// reads each matrix row once for all k columns and the gathered neighbour values of a row are
// k contiguous numbers. A row is handled by a group of KL x TPR lanes: KL lanes, one per column
// (KL = k rounded up to a power of two, lanes j >= k idle), times TPR lanes splitting the row's
// entries. Every column runs its own flexible CG (own alpha, beta, r.z, stopping test); a column
// that has converged keeps x and r fixed (its step length is forced to 0) while the others
// continue, so its result equals a solve of that column alone.
//
// The cycle runs in the value type T: double (FP64 cycle) or float (FP32 cycle with FP32 copies
// of the level operators and transfer weights). The outer CG (residual, dot products, step
// lengths, projection) is always FP64; with the FP32 cycle the residual is rounded to FP32 before
// the cycle and the correction widened back to FP64 after it, and the coarsest-level solve
// accumulates in FP64 against the FP64 pseudo-inverse.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "hier.h"
#include "kernels_common.cuh"

namespace lamg {

constexpr int BBS = 256;
constexpr int KMAX = 32;

__device__ __forceinline__ void b_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void b_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

enum BScalar { B_RZ = 0, B_ALPHA, B_BETA, B_RR, B_BN2, B_MEAN, B_TRUE_RR, B_BMEAN, B_ITERS, B_TOL2, B_COUNT = 12 };

struct BRed {
    double *part;      // 2 x KMAX x RED_MAXG
    unsigned *ticket;
    double *sk;        // B_COUNT x KMAX
    int *done;         // KMAX
    int *itc;          // iteration counter
};

// ------------------------------------------------------------------ per-column reductions

// Column totals over the block: the value v of thread t belongs to column t % KL. The lanes of a
// warp that share a column are added by a fixed shuffle tree (none when KL = 32), then the warps
// in order; thread j < KL returns with column j's total. sh is the caller's NV x BBS scratch.
template <int KL, int NV>
__device__ __forceinline__ void block_col_total(double (&v)[NV], double (*sh)[BBS]) {
#pragma unroll
    for (int o = 16; o >= KL; o >>= 1)
#pragma unroll
        for (int q = 0; q < NV; q++) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();   // the scratch may still be read by a previous use
    if (lane < KL) {
#pragma unroll
        for (int q = 0; q < NV; q++) sh[q][w * KL + lane] = v[q];
    }
    __syncthreads();
    if ((int)threadIdx.x < KL) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double s = 0.0;
            for (int ww = 0; ww < BBS / 32; ww++) s += sh[q][ww * KL + threadIdx.x];
            v[q] = s;
        }
    }
}

// Each thread contributes to column threadIdx.x % KL. Deterministic: per-block column sums in a
// fixed order, then the last block to finish adds the blocks in a fixed order. Returns true in
// the last block, where threads j < KL hold column j's totals. The last block reads only the
// partials (fenced before the ticket); the kernel's other writes reach the next kernel through
// the launch boundary.
template <int KL, int NV>
__device__ bool col_sum(double (&v)[NV], const BRed R) {
    __shared__ double sh[NV][BBS];
    __shared__ bool last;
    block_col_total<KL, NV>(v, sh);
    if ((int)threadIdx.x < KL) {
#pragma unroll
        for (int q = 0; q < NV; q++) R.part[(q * KMAX + threadIdx.x) * RED_MAXG + blockIdx.x] = v[q];
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(R.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // threads t = j + KL * m sum blocks m, m + BBS/KL, ... of column j; then the block total
    constexpr int PER = BBS / KL;
    const int j = threadIdx.x % KL, m = threadIdx.x / KL;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double s = 0.0;
        for (int b = m; b < (int)gridDim.x; b += PER) s += __ldcg(&R.part[(q * KMAX + j) * RED_MAXG + b]);
        v[q] = s;
    }
    block_col_total<KL, NV>(v, sh);
    if (threadIdx.x == 0) *R.ticket = 0u;
    return true;
}

// ------------------------------------------------------------------ cycle steps in SpMM form

template <int KL, int TPR>
struct Lanes {
    static constexpr int G = KL * TPR;
    int row_in_grid, sub, j;
    __device__ Lanes() {
        const int t = blockIdx.x * BBS + threadIdx.x;
        row_in_grid = t / G;
        const int lig = t % G;
        j = lig % KL;
        sub = lig / KL;
    }
};

// D entries e, e + TPR, ... of a row for column j added to s in order, their column ids, values
// and gathers all loaded first.
template <int D, typename T, int TPR>
__device__ __forceinline__ void add_entries(T &s, int e, int k, int j, const int32_t *__restrict__ ci,
                                            const T *__restrict__ val, const T *x) {
    int c[D];
    T v[D], xv[D];
#pragma unroll
    for (int q = 0; q < D; q++) c[q] = ci[e + q * TPR];
#pragma unroll
    for (int q = 0; q < D; q++) v[q] = val[e + q * TPR];
#pragma unroll
    for (int q = 0; q < D; q++) xv[q] = x[(size_t)c[q] * k + j];
#pragma unroll
    for (int q = 0; q < D; q++) s += v[q] * xv[q];
}

// A row's entries e0, e0 + TPR, ... for column j, accumulated in entry order. Entries are loaded
// in groups before their products are added, so a lane has several independent gathers in
// flight instead of one; the sum is the same sequence of multiply-adds as a one-entry-at-a-time
// loop. FP32 rows take groups of eight first (their kernels wait on the gathers), FP64 rows
// groups of four (their kernels wait on the FP64 unit, and eight would cost registers).
template <typename T, int KL, int TPR>
__device__ __forceinline__ T rowsum_k(int e0, int e1, int k, int j, const int32_t *__restrict__ ci,
                                      const T *__restrict__ val, const T *x) {
    T s = T(0);
    if (j < k) {
        int e = e0;
        if constexpr (sizeof(T) == 4)
            for (; e + 7 * TPR < e1; e += 8 * TPR) add_entries<8, T, TPR>(s, e, k, j, ci, val, x);
        for (; e + 3 * TPR < e1; e += 4 * TPR) add_entries<4, T, TPR>(s, e, k, j, ci, val, x);
        for (; e < e1; e += TPR) s += val[e] * x[(size_t)ci[e] * k + j];
    }
#pragma unroll
    for (int o = KL; o < KL * TPR; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

template <typename T, int KL>
__device__ __forceinline__ T block_row_k(int e0, int e1, int k, const int32_t *__restrict__ ci,
                                         const T *__restrict__ val, const T *x) {
    __shared__ T sh[BBS / 32][32];
    constexpr int M = BBS / KL;
    const int j = threadIdx.x % KL, m = threadIdx.x / KL;
    T s = T(0);
    if (j < k) {
        // four entries of the lane loaded before their products are added (as rowsum_k): the
        // same sequence of multiply-adds as one entry at a time, four gathers in flight
        int e = e0 + m;
        for (; e + 3 * M < e1; e += 4 * M) {
            const int c0 = ci[e], c1 = ci[e + M], c2 = ci[e + 2 * M], c3 = ci[e + 3 * M];
            const T v0 = val[e], v1 = val[e + M], v2 = val[e + 2 * M], v3 = val[e + 3 * M];
            const T x0 = x[(size_t)c0 * k + j], x1 = x[(size_t)c1 * k + j];
            const T x2 = x[(size_t)c2 * k + j], x3 = x[(size_t)c3 * k + j];
            s += v0 * x0;
            s += v1 * x1;
            s += v2 * x2;
            s += v3 * x3;
        }
        for (; e < e1; e += M) s += val[e] * x[(size_t)ci[e] * k + j];
    }
#pragma unroll
    for (int o = KL; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < KL) sh[w][lane] = s;
    __syncthreads();
    T t = T(0);
    if (threadIdx.x < KL)
        for (int q = 0; q < BBS / 32; q++) t += sh[q][threadIdx.x];
    __syncthreads();
    return t;
}

// Gauss-Seidel on one colour class [r0, r1), all k columns (Section 2). The class's first nl
// rows are long (rows are sorted longest first inside a class): block b < nl takes row r0 + b.
template <typename T, int KL, int TPR>
__global__ void __launch_bounds__(BBS) bk_gs(int r0, int r1, int nl, int k, const int32_t *__restrict__ rp,
                                             const int32_t *__restrict__ ci, const T *__restrict__ val,
                                             const T *__restrict__ idiag, const T *__restrict__ b, T *x) {
    b_trigger();
    if ((int)blockIdx.x < nl) {
        const int row = r0 + (int)blockIdx.x;
        const int e0 = rp[row], e1 = rp[row + 1];
        const T id = idiag[row];
        b_wait();
        const T s = block_row_k<T, KL>(e0, e1, k, ci, val, x);
        if ((int)threadIdx.x < k) x[(size_t)row * k + threadIdx.x] = (b[(size_t)row * k + threadIdx.x] - s) * id;
        return;
    }
    const int t = (blockIdx.x - nl) * BBS + threadIdx.x;
    constexpr int G = KL * TPR;
    const int lig = t % G, j = lig % KL, sub = lig / KL;
    const int row = r0 + nl + t / G;
    const bool ok = row < r1;
    const int e0 = ok ? rp[row] + sub : 0, e1 = ok ? rp[row + 1] : 0;
    const T id = ok ? idiag[row] : T(1);
    b_wait();
    const T s = rowsum_k<T, KL, TPR>(e0, e1, k, j, ci, val, x);
    if (ok && sub == 0 && j < k) x[(size_t)row * k + j] = (b[(size_t)row * k + j] - s) * id;
}

// r = b - A x, all k columns; blocks b < nl take the long rows lr[b], the lane groups skip them.
template <typename T, int KL, int TPR>
__global__ void __launch_bounds__(BBS) bk_resid(int n, int k, const int32_t *__restrict__ rp,
                                                const int32_t *__restrict__ ci, const T *__restrict__ val,
                                                const T *__restrict__ diag, const T *__restrict__ x,
                                                const T *__restrict__ b, T *r, const int32_t *__restrict__ lr,
                                                int nl) {
    b_trigger();
    if ((int)blockIdx.x < nl) {
        const int row = lr[blockIdx.x];
        const int e0 = rp[row], e1 = rp[row + 1];
        const T d = diag[row];
        b_wait();
        const T s = block_row_k<T, KL>(e0, e1, k, ci, val, x);
        if ((int)threadIdx.x < k) {
            const size_t i = (size_t)row * k + threadIdx.x;
            r[i] = b[i] - (d * x[i] + s);
        }
        return;
    }
    const int t = (blockIdx.x - nl) * BBS + threadIdx.x;
    constexpr int G = KL * TPR;
    const int lig = t % G, j = lig % KL, sub = lig / KL;
    const int row = t / G;
    bool ok = row < n;
    int e0 = ok ? rp[row] + sub : 0, e1 = ok ? rp[row + 1] : 0;
    if (ok && e1 - (e0 - sub) > LONG_ROW) { ok = false; e0 = e1; }
    const T d = ok ? diag[row] : T(0);
    b_wait();
    const T s = rowsum_k<T, KL, TPR>(e0, e1, k, j, ci, val, x);
    if (ok && sub == 0 && j < k) {
        const size_t i = (size_t)row * k + j;
        r[i] = b[i] - (d * x[i] + s);
    }
}

// One right-hand side, one thread per row on the sliced-ELLPACK copy in four-entry blocks
// (sell_col_at / sell_val_at: four column ids in one int4, the values two at a time); entries
// summed in order, padding (value 0 at a valid column) included.
template <typename T> struct Pair;
template <> struct Pair<double> { using V = double2; };
template <> struct Pair<float> { using V = float2; };

template <typename T>
__device__ __forceinline__ T sell_row1(int row, const int32_t *__restrict__ sp, const int32_t *__restrict__ sc,
                                       const T *__restrict__ sv, const T *x) {
    using V = typename Pair<T>::V;
    const int s = row >> 5, l = row & 31;
    const int a = sp[s];
    const int nq = (sp[s + 1] - a) >> 7;
    T acc = T(0);
    for (int q = 0; q < nq; q++) {
        const int4 c = __ldg(reinterpret_cast<const int4 *>(sc + a + 128 * q + 4 * l));
        const V va = __ldg(reinterpret_cast<const V *>(sv + a + 128 * q + 2 * l));
        const V vb = __ldg(reinterpret_cast<const V *>(sv + a + 128 * q + 64 + 2 * l));
        const T x0 = x[c.x], x1 = x[c.y], x2 = x[c.z], x3 = x[c.w];
        acc += va.x * x0;
        acc += va.y * x1;
        acc += vb.x * x2;
        acc += vb.y * x3;
    }
    return acc;
}

template <typename T>
__global__ void __launch_bounds__(64) bk_gs_sell(int r0, int r1, int s0, const int32_t *__restrict__ sp,
                                                 const int32_t *__restrict__ sc, const T *__restrict__ sv,
                                                 const T *__restrict__ idiag, const T *__restrict__ b, T *x) {
    b_trigger();
    const int row = 32 * s0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool ok = row >= r0 && row < r1;
    const T id = ok ? idiag[row] : T(1);
    b_wait();
    if (!ok) return;
    const T s = sell_row1<T>(row, sp, sc, sv, x);
    x[row] = (b[row] - s) * id;
}

template <typename T>
__global__ void __launch_bounds__(BBS) bk_resid_sell(int n, const int32_t *__restrict__ sp,
                                                     const int32_t *__restrict__ sc, const T *__restrict__ sv,
                                                     const T *__restrict__ diag, const T *__restrict__ x,
                                                     const T *__restrict__ b, T *r) {
    b_trigger();
    const int row = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool ok = row < n;
    const T d = ok ? diag[row] : T(0);
    b_wait();
    if (!ok) return;
    const T s = sell_row1<T>(row, sp, sc, sv, x);
    r[row] = b[row] - (d * x[row] + s);
}

// One step of the Chebyshev smoothing polynomial for k columns (as k_cheb): every row from the
// previous iterate xin, d <- c1 d + c2 (b - A xin) / A_uu (first step, flags bit 0: c1 term
// absent), xout = xin + d; d not stored on the last step (flags bit 1). Blocks b < nl take the
// long rows lr[b].
template <typename T, int KL, int TPR>
__global__ void __launch_bounds__(BBS) bk_cheb(int n, int k, const int32_t *__restrict__ rp,
                                               const int32_t *__restrict__ ci, const T *__restrict__ val,
                                               const T *__restrict__ diag, const T *__restrict__ idiag,
                                               const T *__restrict__ b, const T *xin, T *xout, T *d, T c1, T c2,
                                               int flags, const int32_t *__restrict__ lr, int nl) {
    const bool first = flags & 1, last = flags & 2;
    b_trigger();
    if ((int)blockIdx.x < nl) {
        const int row = lr[blockIdx.x];
        const int e0 = rp[row], e1 = rp[row + 1];
        const T dg = diag[row], id = idiag[row];
        b_wait();
        const T s = block_row_k<T, KL>(e0, e1, k, ci, val, xin);
        if ((int)threadIdx.x < k) {
            const size_t i = (size_t)row * k + threadIdx.x;
            const T r = b[i] - (dg * xin[i] + s);
            const T dn = (first ? T(0) : c1 * d[i]) + c2 * r * id;
            if (!last) d[i] = dn;
            xout[i] = xin[i] + dn;
        }
        return;
    }
    const int t = (blockIdx.x - nl) * BBS + threadIdx.x;
    constexpr int G = KL * TPR;
    const int lig = t % G, j = lig % KL, sub = lig / KL;
    const int row = t / G;
    bool ok = row < n;
    int e0 = ok ? rp[row] + sub : 0, e1 = ok ? rp[row + 1] : 0;
    if (ok && e1 - (e0 - sub) > LONG_ROW) { ok = false; e0 = e1; }
    const T dg = ok ? diag[row] : T(0), id = ok ? idiag[row] : T(0);
    b_wait();
    const T s = rowsum_k<T, KL, TPR>(e0, e1, k, j, ci, val, xin);
    if (ok && sub == 0 && j < k) {
        const size_t i = (size_t)row * k + j;
        const T r = b[i] - (dg * xin[i] + s);
        const T dn = (first ? T(0) : c1 * d[i]) + c2 * r * id;
        if (!last) d[i] = dn;
        xout[i] = xin[i] + dn;
    }
}

// First Chebyshev step from x = 0 for k columns (as k_cheb_first): out = (c2 b) / A_uu, and the
// direction d = out when the polynomial continues.
template <typename T>
__global__ void bk_cheb_first(int64_t cnt, int k, const T *__restrict__ idiag, const T *__restrict__ b, T c2,
                              T *out, T *d) {
    b_trigger();
    b_wait();
    const int64_t t = (int64_t)blockIdx.x * BBS + threadIdx.x;
    if (t >= cnt) return;
    const T v = c2 * b[t] * idiag[t / k];
    out[t] = v;
    if (d) d[t] = v;
}

template <typename T>
__global__ void bk_copy(int64_t cnt, const T *__restrict__ src, T *dst) {
    b_trigger();
    b_wait();
    const int64_t t = (int64_t)blockIdx.x * BBS + threadIdx.x;
    if (t < cnt) dst[t] = src[t];
}

// b^c = P^T r; with xc set also the row-local start of the coarse level's first visit (x = b / A
// on its rows a < c1, 0 elsewhere, as bk_gs_first / bk_zero)
template <typename T, int KL, int TPR>
__global__ void __launch_bounds__(BBS) bk_restrict(int nc, int k, const int32_t *__restrict__ ptr,
                                                   const int32_t *__restrict__ row, const T *__restrict__ w,
                                                   const T *__restrict__ r, T *bc, T *xc, int c1,
                                                   const T *__restrict__ idc) {
    b_trigger();
    const Lanes<KL, TPR> L;
    const int a = L.row_in_grid;
    const bool ok = a < nc;
    const int e0 = ok ? ptr[a] + L.sub : 0, e1 = ok ? ptr[a + 1] : 0;
    const T id = (xc && ok && a < c1) ? idc[a] : T(0);
    b_wait();
    const T s = rowsum_k<T, KL, TPR>(e0, e1, k, L.j, row, w, r);
    if (ok && L.sub == 0 && L.j < k) {
        bc[(size_t)a * k + L.j] = s;
        if (xc) xc[(size_t)a * k + L.j] = a < c1 ? s * id : T(0);
    }
}

// Element-wise steps: thread -> (row i, column j = threadIdx.x % KL).
template <int KL>
__device__ __forceinline__ void elem_pos(int &i, int &j) {
    const int t = blockIdx.x * BBS + threadIdx.x;
    i = t / KL;
    j = t % KL;
}

template <typename T, int KL>
__global__ void bk_gs_first(int n, int c1, int k, const T *__restrict__ idiag, const T *__restrict__ b, T *x) {
    b_trigger();
    int i, j;
    elem_pos<KL>(i, j);
    const T id = (i < c1) ? idiag[i] : T(1);
    b_wait();
    if (i >= n || j >= k) return;
    const size_t e = (size_t)i * k + j;
    x[e] = i < c1 ? b[e] * id : T(0);
}

template <typename T>
__global__ void bk_zero(int64_t cnt, T *x) {
    b_trigger();
    b_wait();
    const int64_t t = (int64_t)blockIdx.x * BBS + threadIdx.x;
    if (t < cnt) x[t] = T(0);
}

template <typename T, int KL>
__global__ void bk_prolong(int n, int k, const int32_t *__restrict__ agg, const int32_t *__restrict__ agg2,
                           const T *__restrict__ wt, const T *__restrict__ xc, T *x) {
    b_trigger();
    int u, j;
    elem_pos<KL>(u, j);
    const bool ok = u < n;
    const int a = ok ? agg[u] : 0, bb = ok ? agg2[u] : -1;
    const T w = (ok && bb >= 0) ? wt[u] : T(1);
    b_wait();
    if (!ok || j >= k) return;
    T s;
    if (bb < 0) {
        s = xc[(size_t)a * k + j];
    } else {
        s = (T(1) - w) * xc[(size_t)bb * k + j];
        if (w != T(0)) s = w * xc[(size_t)a * k + j] + s;
    }
    x[(size_t)u * k + j] += s;
}

// b^c = b_C + P_F^T b_F (and with xc set the coarse level's row-local first-visit start, as
// bk_restrict). Blocks b < nl take the C rows lr[b] that gather more than LONG_ROW F entries (the
// hubs of power-law graphs), summed by the whole block (as block_row_k) and added to b_C; every
// other C row is summed by its lanes in entry order.
template <typename T, int KL>
__global__ void bk_elim_restrict(int nc, int k, const int32_t *__restrict__ ptr, const int32_t *__restrict__ f,
                                 const T *__restrict__ pv, const T *__restrict__ b, T *bc, T *xc, int c1,
                                 const T *__restrict__ idc, const int32_t *__restrict__ lr, int nl) {
    b_trigger();
    const T *bF = b + (size_t)nc * k;
    if ((int)blockIdx.x < nl) {
        const int i = lr[blockIdx.x];
        const int e0 = ptr[i], e1 = ptr[i + 1];
        const T id = (xc && i < c1) ? idc[i] : T(0);
        b_wait();
        const T sF = block_row_k<T, KL>(e0, e1, k, f, pv, bF);
        if ((int)threadIdx.x < k) {
            const size_t e = (size_t)i * k + threadIdx.x;
            const T s = b[e] + sF;
            bc[e] = s;
            if (xc) xc[e] = i < c1 ? s * id : T(0);
        }
        return;
    }
    const int t = (blockIdx.x - nl) * BBS + threadIdx.x;
    const int i = t / KL, j = t % KL;
    bool ok = i < nc;
    const int e0 = ok ? ptr[i] : 0, e1 = ok ? ptr[i + 1] : 0;
    if (e1 - e0 > LONG_ROW) ok = false;
    const T id = (xc && ok && i < c1) ? idc[i] : T(0);
    b_wait();
    if (!ok || j >= k) return;
    T s = b[(size_t)i * k + j];
    for (int e = e0; e < e1; e++) s += pv[e] * bF[(size_t)f[e] * k + j];
    bc[(size_t)i * k + j] = s;
    if (xc) xc[(size_t)i * k + j] = i < c1 ? s * id : T(0);
}

template <typename T, int KL>
__global__ void bk_elim_interp(int nc, int nF, int k, const int32_t *__restrict__ col, const T *__restrict__ pv,
                               const T *__restrict__ idF, const T *__restrict__ b, T *x) {
    b_trigger();
    int t, j;
    elem_pos<KL>(t, j);
    const bool ok = t < nF;
    int c[4];
    T p[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        c[q] = ok ? col[4 * t + q] : -1;
        p[q] = ok ? pv[4 * t + q] : T(0);
    }
    const T id = ok ? idF[t] : T(1);
    b_wait();
    if (!ok || j >= k) return;
    T s = T(0);
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (c[q] >= 0) s += p[q] * x[(size_t)c[q] * k + j];
    const size_t e = (size_t)(nc + t) * k + j;
    x[e] = s + b[e] * id;
}

// Coarsest level: x = (I - J/n) A^+ b against the FP64 projected pseudo-inverse, accumulated in
// FP64 for either cycle type (b in FP64: an FP32 cycle's right-hand side widened beforehand; the
// FP64 sum rounded to FP32 once at the end). One block per row: KL lanes per column times BBS/KL
// lanes splitting the row, each lane with four independent partial sums (a dependent FP64 add
// takes ~68 clocks on this GPU, so one chain of n/2 adds per lane would set the kernel's time),
// combined in a fixed order: the four partials, the lanes of a warp by a shuffle tree, then the
// warps in order.
template <typename T, int KL>
__global__ void __launch_bounds__(BBS) bk_coarse(int n, int k, const double *__restrict__ pinv,
                                                 const double *__restrict__ b, T *x) {
    b_trigger();
    b_wait();
    __shared__ double sh[BBS / 32][32];
    constexpr int M = BBS / KL;
    const int j = threadIdx.x % KL, m = threadIdx.x / KL;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const double *row = pinv + (size_t)i * n;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        if (j < k) {
            int c = m;
            for (; c + 3 * M < n; c += 4 * M) {
                s0 += row[c] * b[(size_t)c * k + j];
                s1 += row[c + M] * b[(size_t)(c + M) * k + j];
                s2 += row[c + 2 * M] * b[(size_t)(c + 2 * M) * k + j];
                s3 += row[c + 3 * M] * b[(size_t)(c + 3 * M) * k + j];
            }
            for (; c < n; c += M) s0 += row[c] * b[(size_t)c * k + j];
        }
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = KL; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane < KL) sh[w][lane] = s;
        __syncthreads();
        if ((int)threadIdx.x < KL && (int)threadIdx.x < k) {
            double t = 0.0;
            for (int q = 0; q < BBS / 32; q++) t += sh[q][threadIdx.x];
            x[(size_t)i * k + threadIdx.x] = (T)t;
        }
        __syncthreads();
    }
}

// One column: a warp per row, each lane with four partial sums over the columns lane, lane + 32,
// ..., then the warp's shuffle tree (a block per row would spend half as many FP64 adds on its
// 256-lane reduction as on the row's n multiply-adds).
template <typename T>
__global__ void __launch_bounds__(BBS) bk_coarse1(int n, const double *__restrict__ pinv,
                                                  const double *__restrict__ b, T *x) {
    b_trigger();
    b_wait();
    const int lane = threadIdx.x & 31;
    const int wg = (int)((blockIdx.x * BBS + threadIdx.x) >> 5), nw = (int)((gridDim.x * BBS) >> 5);
    for (int i = wg; i < n; i += nw) {
        const double *row = pinv + (size_t)i * n;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int c = lane;
        for (; c + 96 < n; c += 128) {
            s0 += row[c] * b[c];
            s1 += row[c + 32] * b[c + 32];
            s2 += row[c + 64] * b[c + 64];
            s3 += row[c + 96] * b[c + 96];
        }
        for (; c < n; c += 32) s0 += row[c] * b[c];
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = (T)s;
    }
}

// ------------------------------------------------------------------ outer CG, k columns (FP64)

template <typename Tin, typename Tout>
__global__ void bk_cast(int64_t cnt, const Tin *__restrict__ src, Tout *dst) {
    b_trigger();
    b_wait();
    const int64_t t = (int64_t)blockIdx.x * BBS + threadIdx.x;
    if (t < cnt) dst[t] = (Tout)src[t];
}

template <int KL>
__global__ void bk_gather_rows(int n, int k, const int32_t *__restrict__ perm, const double *__restrict__ src,
                               double *dst) {
    b_trigger();
    int i, j;
    elem_pos<KL>(i, j);
    const int pi = i < n ? perm[i] : 0;
    b_wait();
    if (i < n && j < k) dst[(size_t)i * k + j] = src[(size_t)pi * k + j];
}

template <int KL>
__global__ void bk_scatter_rows(int n, int k, const int32_t *__restrict__ perm, const double *__restrict__ src,
                                double *dst) {
    b_trigger();
    int i, j;
    elem_pos<KL>(i, j);
    const int pi = i < n ? perm[i] : 0;
    b_wait();
    if (i < n && j < k) dst[(size_t)pi * k + j] = src[(size_t)i * k + j];
}

// Grid-stride loop over rows for element-wise CG kernels: thread column j = threadIdx.x % KL.
#define FOR_ELEM(n, k)                                                                   \
    const int j = threadIdx.x % KL;                                                      \
    const int rows_per_pass = (gridDim.x * BBS) / KL;                                    \
    for (int i = (blockIdx.x * BBS + threadIdx.x) / KL; i < (n); i += rows_per_pass)     \
        if (j < (k))

// mean_j = sum_i v(i, j) / n
template <int KL>
__global__ void __launch_bounds__(BBS) bk_sum(int n, int k, const double *__restrict__ v, const BRed R) {
    b_trigger();
    b_wait();
    double s[1] = {0.0};
    FOR_ELEM(n, k) s[0] += v[(size_t)i * k + j];
    if (col_sum<KL, 1>(s, R) && threadIdx.x < k) R.sk[B_MEAN * KMAX + threadIdx.x] = s[0] / (double)n;
}

template <int KL>
__global__ void __launch_bounds__(BBS) bk_init_b(int n, int k, double *r, double *bkeep, double *x, double *p,
                                                 double *zold, const BRed R) {
    b_trigger();
    b_wait();
    double s[1] = {0.0};
    {
        const double m = R.sk[B_MEAN * KMAX + (threadIdx.x % KL)];
        FOR_ELEM(n, k) {
            const size_t e = (size_t)i * k + j;
            const double v = r[e] - m;
            r[e] = v;
            bkeep[e] = v;
            x[e] = 0.0;
            p[e] = 0.0;
            zold[e] = 0.0;
            s[0] += v * v;
        }
    }
    if (col_sum<KL, 1>(s, R)) {
        const int c = threadIdx.x;
        if (c < k) {
            R.sk[B_BN2 * KMAX + c] = s[0];
            R.sk[B_RZ * KMAX + c] = 1.0;
            R.sk[B_BMEAN * KMAX + c] = R.sk[B_MEAN * KMAX + c];
            R.sk[B_ITERS * KMAX + c] = 0.0;
            R.done[c] = 0;
        }
        if (c == 0) *R.itc = 0;
    }
}

template <int KL, int TPR>
__global__ void __launch_bounds__(BBS) bk_spmv_dot(int n, int k, const int32_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci, const double *__restrict__ val,
                                                   const double *__restrict__ diag, const double *__restrict__ p,
                                                   double *q, const BRed R, const int32_t *__restrict__ lr, int nl) {
    b_trigger();
    b_wait();
    constexpr int G = KL * TPR;
    const int t = blockIdx.x * BBS + threadIdx.x;
    const int lig = t % G, j = lig % KL, sub = lig / KL;
    const int groups = gridDim.x * (BBS / G);
    const int rounds = (n + groups - 1) / groups;
    double pq[1] = {0.0};
    for (int lt = blockIdx.x; lt < nl; lt += gridDim.x) {
        const int row = lr[lt];
        const double s = block_row_k<double, KL>(rp[row], rp[row + 1], k, ci, val, p);
        if ((int)threadIdx.x < k) {
            const size_t e = (size_t)row * k + threadIdx.x;
            const double qi = diag[row] * p[e] + s;
            q[e] = qi;
            pq[0] += p[e] * qi;
        }
    }
    int row = t / G;
    for (int it = 0; it < rounds; it++, row += groups) {
        bool ok = row < n;
        int e0 = ok ? rp[row] + sub : 0, e1 = ok ? rp[row + 1] : 0;
        if (ok && e1 - (e0 - sub) > LONG_ROW) { ok = false; e0 = e1; }
        const double s = rowsum_k<double, KL, TPR>(e0, e1, k, j, ci, val, p);
        if (ok && sub == 0 && j < k) {
            const size_t e = (size_t)row * k + j;
            const double qi = diag[row] * p[e] + s;
            q[e] = qi;
            pq[0] += p[e] * qi;
        }
    }
    if (col_sum<KL, 1>(pq, R) && threadIdx.x < k) {
        const int c = threadIdx.x;
        const double rz = R.sk[B_RZ * KMAX + c];
        R.sk[B_ALPHA * KMAX + c] = (R.done[c] || pq[0] == 0.0) ? 0.0 : rz / pq[0];
    }
}

// One right-hand side on a level with the sliced copy: q = A p one thread per row (as
// k_spmv_dot_sell), alpha = r.z / (p . q).
__global__ void __launch_bounds__(BBS) bk_spmv_dot_sell(int n, const int32_t *__restrict__ sp,
                                                        const int32_t *__restrict__ sc,
                                                        const double *__restrict__ sv,
                                                        const double *__restrict__ diag,
                                                        const double *__restrict__ p, double *q, const BRed R) {
    b_trigger();
    b_wait();
    double pq[1] = {0.0};
    for (int row = blockIdx.x * BBS + threadIdx.x; row < n; row += gridDim.x * BBS) {
        const double s = sell_row1<double>(row, sp, sc, sv, p);
        const double qi = diag[row] * p[row] + s;
        q[row] = qi;
        pq[0] += p[row] * qi;
    }
    if (col_sum<1, 1>(pq, R) && threadIdx.x == 0) {
        const double rz = R.sk[B_RZ * KMAX];
        R.sk[B_ALPHA * KMAX] = (R.done[0] || pq[0] == 0.0) ? 0.0 : rz / pq[0];
    }
}

template <int KL>
__global__ void __launch_bounds__(BBS) bk_update_xr(int n, int k, double *x, double *r, const double *__restrict__ p,
                                                    const double *__restrict__ q, const BRed R) {
    b_trigger();
    b_wait();
    double s[1] = {0.0};
    {
        const double a = R.sk[B_ALPHA * KMAX + (threadIdx.x % KL)];
        FOR_ELEM(n, k) {
            const size_t e = (size_t)i * k + j;
            x[e] += a * p[e];
            const double ri = r[e] - a * q[e];
            r[e] = ri;
            s[0] += ri * ri;
        }
    }
    if (col_sum<KL, 1>(s, R)) {
        __shared__ int it;
        if (threadIdx.x == 0) it = ++(*R.itc);
        __syncthreads();
        const int c = threadIdx.x;
        if (c < k) {
            R.sk[B_RR * KMAX + c] = s[0];
            const double tol2 = R.sk[B_TOL2 * KMAX];
            if (!R.done[c] && s[0] <= tol2 * R.sk[B_BN2 * KMAX + c]) {
                R.done[c] = 1;
                R.sk[B_ITERS * KMAX + c] = (double)it;
            }
        }
    }
}

template <int KL>
__global__ void __launch_bounds__(BBS) bk_proj_dots(int n, int k, double *z, const double *__restrict__ zold,
                                                    const double *__restrict__ r, const BRed R) {
    b_trigger();
    b_wait();
    double s[2] = {0.0, 0.0};
    {
        const double m = R.sk[B_MEAN * KMAX + (threadIdx.x % KL)];
        FOR_ELEM(n, k) {
            const size_t e = (size_t)i * k + j;
            const double zi = z[e] - m;
            z[e] = zi;
            s[0] += r[e] * (zi - zold[e]);
            s[1] += r[e] * zi;
        }
    }
    if (col_sum<KL, 2>(s, R) && threadIdx.x < k) {
        const int c = threadIdx.x;
        const double rz = R.sk[B_RZ * KMAX + c];
        R.sk[B_BETA * KMAX + c] = rz != 0.0 ? s[0] / rz : 0.0;
        R.sk[B_RZ * KMAX + c] = s[1];
    }
}

template <int KL>
__global__ void bk_update_p(int n, int k, const double *__restrict__ z, double *p, double *zold, const BRed R) {
    b_trigger();
    b_wait();
    int i, j;
    elem_pos<KL>(i, j);
    if (i >= n || j >= k) return;
    const double beta = R.sk[B_BETA * KMAX + j];
    const size_t e = (size_t)i * k + j;
    const double zi = z[e];
    p[e] = zi + beta * p[e];
    zold[e] = zi;
}

template <int KL, int TPR>
__global__ void __launch_bounds__(BBS) bk_true_resid(int n, int k, const int32_t *__restrict__ rp,
                                                     const int32_t *__restrict__ ci, const double *__restrict__ val,
                                                     const double *__restrict__ diag, const double *__restrict__ x,
                                                     const double *__restrict__ b, const BRed R,
                                                     const int32_t *__restrict__ lr, int nl) {
    b_trigger();
    b_wait();
    constexpr int G = KL * TPR;
    const int t = blockIdx.x * BBS + threadIdx.x;
    const int lig = t % G, j = lig % KL, sub = lig / KL;
    const int groups = gridDim.x * (BBS / G);
    const int rounds = (n + groups - 1) / groups;
    double acc[1] = {0.0};
    for (int lt = blockIdx.x; lt < nl; lt += gridDim.x) {
        const int row = lr[lt];
        const double s = block_row_k<double, KL>(rp[row], rp[row + 1], k, ci, val, x);
        if ((int)threadIdx.x < k) {
            const size_t e = (size_t)row * k + threadIdx.x;
            const double ri = b[e] - (diag[row] * x[e] + s);
            acc[0] += ri * ri;
        }
    }
    int row = t / G;
    for (int it = 0; it < rounds; it++, row += groups) {
        bool ok = row < n;
        int e0 = ok ? rp[row] + sub : 0, e1 = ok ? rp[row + 1] : 0;
        if (ok && e1 - (e0 - sub) > LONG_ROW) { ok = false; e0 = e1; }
        const double s = rowsum_k<double, KL, TPR>(e0, e1, k, j, ci, val, x);
        if (ok && sub == 0 && j < k) {
            const size_t e = (size_t)row * k + j;
            const double ri = b[e] - (diag[row] * x[e] + s);
            acc[0] += ri * ri;
        }
    }
    if (col_sum<KL, 1>(acc, R) && threadIdx.x < k) R.sk[B_TRUE_RR * KMAX + threadIdx.x] = acc[0];
}

// ------------------------------------------------------------------ launch helpers

// kernels launched (or captured) by this thread through blaunch / blaunch_bs
static thread_local int64_t t_blaunches = 0;

template <typename... KArgs, typename... Args>
static void blaunch(void (*kernel)(KArgs...), int64_t grid, cudaStream_t s, Args... args) {
    t_blaunches++;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(grid < 1 ? 1 : grid));
    cfg.blockDim = dim3(BBS);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
static void blaunch_bs(void (*kernel)(KArgs...), int64_t grid, unsigned bs, cudaStream_t s, Args... args) {
    t_blaunches++;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(grid < 1 ? 1 : grid));
    cfg.blockDim = dim3(bs);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

static inline int64_t nblocks(int64_t threads) { return (threads + BBS - 1) / BBS; }
static inline int64_t rblocks(int64_t threads) {
    int64_t b = (threads + BBS - 1) / BBS;
    return std::max<int64_t>(1, std::min<int64_t>(b, RED_MAXG));
}

static int pow2_at_least(int k) {
    int p = 1;
    while (p < k) p <<= 1;
    return p;
}

// (KL, TPR) pairs instantiated: KL = 1 with TPR 1..32, KL >= 2 with TPR 1, 2, 4 (KL*TPR <= 32)
#define KT_CODE(KL, TPR) ((KL) * 64 + (TPR))
#define KT_CASES(X, ...)              \
    X(1, 1, __VA_ARGS__)              \
    X(1, 2, __VA_ARGS__)              \
    X(1, 4, __VA_ARGS__)              \
    X(1, 8, __VA_ARGS__)              \
    X(1, 16, __VA_ARGS__)             \
    X(1, 32, __VA_ARGS__)             \
    X(2, 1, __VA_ARGS__)              \
    X(2, 2, __VA_ARGS__)              \
    X(2, 4, __VA_ARGS__)              \
    X(4, 1, __VA_ARGS__)              \
    X(4, 2, __VA_ARGS__)              \
    X(4, 4, __VA_ARGS__)              \
    X(8, 1, __VA_ARGS__)              \
    X(8, 2, __VA_ARGS__)              \
    X(8, 4, __VA_ARGS__)              \
    X(16, 1, __VA_ARGS__)             \
    X(16, 2, __VA_ARGS__)             \
    X(32, 1, __VA_ARGS__)

// Lanes per row for each column of a k-column kernel: from four columns on, one lane per row
// and column, which sums its row's entries in a chain without a shuffle tree (the tree's FP64
// adds and the lanes it idles cost more than the chain's latency; measured on B300, 16-column
// solves: 1024^2 anisotropic grid 75.3 -> 64.2 ms, 192^3 heterogeneous grid 699 -> 508 ms; 8
// columns on a 128^3 grid 159 -> 90 ms, 4 columns 89 -> 65 ms); at two columns the level's lane
// groups stay (56 against 60 ms); one column uses the single-RHS rule of the level.
static int row_tpr(int KL, int level_tpr) {
    if (KL == 1) return level_tpr;
    if (KL >= 4) return 1;
    return std::max(1, std::min(level_tpr, std::min(4, 32 / KL)));
}

#define K_CASES(X, ...) X(1, __VA_ARGS__) X(2, __VA_ARGS__) X(4, __VA_ARGS__) X(8, __VA_ARGS__) X(16, __VA_ARGS__) X(32, __VA_ARGS__)

// ------------------------------------------------------------------ workspace

struct BLev {
    int kind = 0, ncol = 0, tpr = 1, pt_tpr = 1;
    int gs_tpr = 1, rs_tpr = 1;   // one right-hand side: the level's kernel forms (0: sliced)
    int64_t n = 0, nc = 0, nF = 0, nlong = 0;
    std::vector<int64_t> cptr, lptr;
    const int32_t *lrows = nullptr;
    const void *idiag = nullptr;
    const int32_t *sl_ptr = nullptr, *sl_col = nullptr;
    const void *sl_val = nullptr;
    int cheb = 0, cheb_m = 0;
    double cheb_c1[8] = {0}, cheb_c2[8] = {0};
    void *t = nullptr, *d = nullptr;   // Chebyshev second iterate and direction, n x k
    const int32_t *rp = nullptr, *ci = nullptr, *agg = nullptr, *agg2 = nullptr, *pt_ptr = nullptr,
                  *pt_row = nullptr, *pf_col = nullptr, *pft_ptr = nullptr, *pft_f = nullptr;
    const void *val = nullptr, *diag = nullptr, *wt = nullptr, *pt_w = nullptr, *pf_val = nullptr,
               *dF = nullptr, *idF = nullptr, *pft_val = nullptr;
    const int32_t *pft_long = nullptr;   // elimination: C rows with more than LONG_ROW F entries
    int64_t npft_long = 0;
    const double *pinv = nullptr;  // coarsest (I - J/n) A^+, FP64 for either cycle type
    double *b64 = nullptr;         // coarsest, FP32 cycle: the right-hand side widened to FP64
    void *x = nullptr, *b = nullptr, *r = nullptr;
};

struct BatchCtx {
    int k = 0, prec = 0, KL = 1;
    std::vector<BLev> lv;
    double *r = nullptr, *p = nullptr, *q = nullptr, *zold = nullptr, *xs = nullptr, *bkeep = nullptr;
    double *nat_in = nullptr, *nat_out = nullptr, *z64 = nullptr;
    void *b0 = nullptr;  // FP32 copy of the residual fed to the cycle
    BRed red{};
    double *h_sk = nullptr;  // pinned: B_COUNT x KMAX scalars + KMAX done flags
    cudaGraphExec_t g_tail = nullptr, g_head = nullptr;
    int64_t n_tail = 0, n_head = 0;   // kernels in each captured graph
};

void batch_free(BatchCtx *b) {
    if (!b) return;
    if (b->g_tail) cudaGraphExecDestroy(b->g_tail);
    if (b->g_head) cudaGraphExecDestroy(b->g_head);
    if (b->h_sk) cudaFreeHost(b->h_sk);
    delete b;
}

template <typename T>
static int typed_copy(lamg_hier *h, const double *src, int64_t cnt, const void **out) {
    if (!src || cnt <= 0) { *out = nullptr; return LAMG_OK; }
    if (sizeof(T) == sizeof(double)) { *out = src; return LAMG_OK; }
    std::vector<double> tmp(cnt);
    CKR(cudaMemcpyAsync(tmp.data(), src, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    std::vector<T> f(tmp.begin(), tmp.end());
    T *d = nullptr;
    int rc = dupload(h, &d, f);
    *out = d;
    return rc;
}

template <typename T>
static int build_ctx(lamg_hier *h, BatchCtx *c) {
    int rc;
    const int L = (int)h->dev.size();
    const int64_t k = c->k;
    c->lv.resize(L);
    for (int l = 0; l < L; l++) {
        const DevLevel &D = h->dev[l];
        BLev &B = c->lv[l];
        B.kind = D.kind; B.ncol = D.ncol; B.tpr = D.tpr; B.pt_tpr = D.pt_tpr;
        B.n = D.n; B.nc = D.nc; B.nF = D.nF; B.cptr = D.cptr;
        B.nlong = D.nlong; B.lptr = D.lptr; B.lrows = D.lrows;
        B.gs_tpr = D.gs_tpr; B.rs_tpr = D.rs_tpr; B.sl_ptr = D.sl_ptr; B.sl_col = D.sl_col;
        B.cheb = D.cheb;
        B.cheb_m = D.cheb_m;
        for (int q = 0; q < 8; q++) { B.cheb_c1[q] = D.cheb_c1[q]; B.cheb_c2[q] = D.cheb_c2[q]; }
        if (D.sell && (rc = typed_copy<T>(h, D.sl_val, D.sell_nnz, &B.sl_val))) return rc;
        B.rp = D.rp; B.ci = D.ci; B.agg = D.agg; B.agg2 = D.agg2; B.pt_ptr = D.pt_ptr; B.pt_row = D.pt_row;
        B.pf_col = D.pf_col; B.pft_ptr = D.pft_ptr; B.pft_f = D.pft_f;
        B.pft_long = D.pft_long; B.npft_long = D.npft_long;
        B.pinv = D.kind == KIND_COARSEST ? D.pinv : nullptr;
        const int64_t pte = (D.kind == KIND_AGG) ? (int64_t)h->host[l].A.n * 2 : 0;
        int32_t ent = 0;
        if (D.kind == KIND_AGG) {
            CKR(cudaMemcpyAsync(&ent, D.pt_ptr + D.nc, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
            CKR(cudaStreamSynchronize(h->stream));
        }
        (void)pte;
        int32_t fent = 0;
        if (D.kind == KIND_ELIM) {
            CKR(cudaMemcpyAsync(&fent, D.pft_ptr + D.nc, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
            CKR(cudaStreamSynchronize(h->stream));
        }
        if ((rc = typed_copy<T>(h, D.val, D.nnz, &B.val)) || (rc = typed_copy<T>(h, D.diag, D.n, &B.diag)) ||
            (rc = typed_copy<T>(h, D.idiag, D.n, &B.idiag)) ||
            (rc = typed_copy<T>(h, D.wt, D.kind == KIND_AGG ? D.n : 0, &B.wt)) ||
            (rc = typed_copy<T>(h, D.pt_w, ent, &B.pt_w)) ||
            (rc = typed_copy<T>(h, D.pf_val, D.kind == KIND_ELIM ? 4 * D.nF : 0, &B.pf_val)) ||
            (rc = typed_copy<T>(h, D.dF, D.kind == KIND_ELIM ? D.nF : 0, &B.dF)) ||
            (rc = typed_copy<T>(h, D.idF, D.kind == KIND_ELIM ? D.nF : 0, &B.idF)) ||
            (rc = typed_copy<T>(h, D.pft_val, fent, &B.pft_val)))
            return rc;
    }
    const int64_t n0 = h->dev[0].n;
    if ((rc = dalloc(h, &c->r, n0 * k)) || (rc = dalloc(h, &c->p, n0 * k)) || (rc = dalloc(h, &c->q, n0 * k)) ||
        (rc = dalloc(h, &c->zold, n0 * k)) || (rc = dalloc(h, &c->xs, n0 * k)) ||
        (rc = dalloc(h, &c->bkeep, n0 * k)) || (rc = dalloc(h, &c->nat_in, n0 * k)) ||
        (rc = dalloc(h, &c->nat_out, n0 * k)))
        return rc;
    // cycle vectors in T; level 0's right-hand side is the residual (FP64 cycle) or its FP32 copy
    for (int l = 0; l < L; l++) {
        BLev &B = c->lv[l];
        T *x = nullptr, *b = nullptr, *r = nullptr;
        if (l == 0) {
            if (c->prec == LAMG_FP32) {
                if ((rc = dalloc(h, &b, B.n * k))) return rc;
                c->b0 = b;
            } else {
                b = (T *)c->r;
            }
        } else if ((rc = dalloc(h, &b, B.n * k))) {
            return rc;
        }
        if (l == 0 || c->lv[l - 1].kind != KIND_ELIM) {
            if ((rc = dalloc(h, &x, B.n * k))) return rc;
        } else {
            x = (T *)c->lv[l - 1].x;
        }
        if (B.kind == KIND_AGG && (rc = dalloc(h, &r, B.n * k))) return rc;
        if (B.kind == KIND_COARSEST && c->prec == LAMG_FP32 && (rc = dalloc(h, &B.b64, B.n * k))) return rc;
        B.x = x; B.b = b; B.r = r;
        if (B.cheb) {
            T *tt = nullptr, *dd = nullptr;
            if ((rc = dalloc(h, &tt, B.n * k)) || (rc = dalloc(h, &dd, B.n * k))) return rc;
            B.t = tt;
            B.d = dd;
        }
    }
    if (c->prec == LAMG_FP32) {
        if ((rc = dalloc(h, &c->z64, n0 * k))) return rc;
    } else {
        c->z64 = (double *)c->lv[0].x;
    }
    if ((rc = dalloc(h, &c->red.part, 2 * KMAX * RED_MAXG)) || (rc = dalloc(h, &c->red.ticket, 1)) ||
        (rc = dalloc(h, &c->red.sk, B_COUNT * KMAX)) || (rc = dalloc(h, &c->red.done, KMAX)) ||
        (rc = dalloc(h, &c->red.itc, 1)))
        return rc;
    CKR(cudaMemsetAsync(c->red.ticket, 0, sizeof(unsigned), h->stream));
    CKR(cudaMemsetAsync(c->red.sk, 0, B_COUNT * KMAX * sizeof(double), h->stream));
    CKR(cudaMemsetAsync(c->red.done, 0, KMAX * sizeof(int), h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    CKR(cudaHostAlloc(&c->h_sk, (B_COUNT * KMAX + KMAX) * sizeof(double), cudaHostAllocDefault));
    return LAMG_OK;
}

// One step of the cycle schedule for k columns in type T (start: as for launch_op).
template <typename T>
static void bop(const Op &op, BatchCtx *c, cudaStream_t s, const Op *start) {
    BLev &L = c->lv[op.level];
    T *xs = nullptr;
    const T *ids = nullptr;
    int c1 = 0;
    if (start) {
        const BLev &Cs = c->lv[start->level];
        xs = (T *)Cs.x;
        if (start->kind == OP_GS_FIRST) { c1 = (int)Cs.cptr[1]; ids = (const T *)Cs.idiag; }
    }
    const int n = (int)L.n, k = c->k, KL = c->KL;
    const T *val = (const T *)L.val, *diag = (const T *)L.diag, *idiag = (const T *)L.idiag;
    T *x = (T *)L.x, *b = (T *)L.b, *r = (T *)L.r;
    switch (op.kind) {
        case OP_GS_FIRST:
#define C1(KLv, ...) case KLv: blaunch(bk_gs_first<T, KLv>, nblocks((int64_t)n * KLv), s, n, (int)L.cptr[1], k, idiag, (const T *)b, x); break;
            switch (KL) { K_CASES(C1) }
#undef C1
            break;
        case OP_ZERO:
            blaunch(bk_zero<T>, nblocks((int64_t)n * k), s, (int64_t)n * k, x);
            break;
        case OP_GS: {
            const int r0 = (int)L.cptr[op.colour], r1 = (int)L.cptr[op.colour + 1];
            if (r1 <= r0) break;
            if (KL == 1 && L.gs_tpr == 0) {
                const int s0 = r0 / 32, s1 = (r1 + 31) / 32;
                blaunch_bs(bk_gs_sell<T>, (32 * (s1 - s0) + 63) / 64, 64, s, r0, r1, s0, L.sl_ptr, L.sl_col,
                           (const T *)L.sl_val, idiag, (const T *)b, x);
                break;
            }
            const int tpr = KL == 1 ? L.gs_tpr : row_tpr(KL, L.tpr);
            const int nl = L.nlong ? (int)(L.lptr[op.colour + 1] - L.lptr[op.colour]) : 0;
#define C2(KLv, TPRv, ...) case KT_CODE(KLv, TPRv): blaunch(bk_gs<T, KLv, TPRv>, nl + nblocks((int64_t)(r1 - r0 - nl) * KLv * TPRv), s, r0, r1, nl, k, L.rp, L.ci, val, idiag, (const T *)b, x); break;
            switch (KT_CODE(KL, tpr)) { KT_CASES(C2) }
#undef C2
            break;
        }
        case OP_RESID: {
            if (KL == 1 && L.rs_tpr == 0) {
                blaunch(bk_resid_sell<T>, nblocks(n), s, n, L.sl_ptr, L.sl_col, (const T *)L.sl_val, diag,
                        (const T *)x, (const T *)b, r);
                break;
            }
            const int tpr = KL == 1 ? L.rs_tpr : row_tpr(KL, L.tpr);
#define C3(KLv, TPRv, ...) case KT_CODE(KLv, TPRv): blaunch(bk_resid<T, KLv, TPRv>, L.nlong + nblocks((int64_t)n * KLv * TPRv), s, n, k, L.rp, L.ci, val, diag, (const T *)x, (const T *)b, r, L.lrows, (int)L.nlong); break;
            switch (KT_CODE(KL, tpr)) { KT_CASES(C3) }
#undef C3
            break;
        }
        case OP_RESTRICT: {
            const int nc = (int)L.nc;
            const int tpr = row_tpr(KL, L.pt_tpr);
            T *bc = (T *)c->lv[op.level + 1].b;
#define C4(KLv, TPRv, ...) case KT_CODE(KLv, TPRv): blaunch(bk_restrict<T, KLv, TPRv>, nblocks((int64_t)nc * KLv * TPRv), s, nc, k, L.pt_ptr, L.pt_row, (const T *)L.pt_w, (const T *)r, bc, xs, c1, ids); break;
            switch (KT_CODE(KL, tpr)) { KT_CASES(C4) }
#undef C4
            break;
        }
        case OP_PROLONG: {
            const T *xc = (const T *)c->lv[op.level + 1].x;
#define C5(KLv, ...) case KLv: blaunch(bk_prolong<T, KLv>, nblocks((int64_t)n * KLv), s, n, k, L.agg, L.agg2, (const T *)L.wt, xc, x); break;
            switch (KL) { K_CASES(C5) }
#undef C5
            break;
        }
        case OP_ELIM_RESTRICT: {
            T *bc = (T *)c->lv[op.level + 1].b;
            const int nc = (int)L.nc;
#define C6(KLv, ...) case KLv: blaunch(bk_elim_restrict<T, KLv>, L.npft_long + nblocks((int64_t)nc * KLv), s, nc, k, L.pft_ptr, L.pft_f, (const T *)L.pft_val, (const T *)b, bc, xs, c1, ids, L.pft_long, (int)L.npft_long); break;
            switch (KL) { K_CASES(C6) }
#undef C6
            break;
        }
        case OP_ELIM_INTERP: {
            if (L.nF <= 0) break;
            const int nF = (int)L.nF;
#define C7(KLv, ...) case KLv: blaunch(bk_elim_interp<T, KLv>, nblocks((int64_t)nF * KLv), s, (int)L.nc, nF, k, L.pf_col, (const T *)L.pf_val, (const T *)L.idF, (const T *)b, x); break;
            switch (KL) { K_CASES(C7) }
#undef C7
            break;
        }
        case OP_COARSE: {
            // an FP32 cycle's right-hand side is widened once (n k conversions) instead of at
            // every product: FP64 conversions share the FP64 pipe with the n^2 k multiply-adds
            const double *b64 = (const double *)b;
            if (sizeof(T) != sizeof(double)) {
                blaunch(bk_cast<T, double>, nblocks((int64_t)n * k), s, (int64_t)n * k, (const T *)b, L.b64);
                b64 = L.b64;
            }
            if (KL == 1) {
                blaunch(bk_coarse1<T>, std::min<int64_t>((n + BBS / 32 - 1) / (BBS / 32), 148 * 8), s, n, L.pinv, b64, x);
                break;
            }
#define C8(KLv, ...) case KLv: blaunch(bk_coarse<T, KLv>, std::min<int64_t>(n, 148 * 8), s, n, k, L.pinv, b64, x); break;
            switch (KL) { K_CASES(C8) }
#undef C8
            break;
        }
        case OP_CHEB: {
            // colour: step index within the polynomial, + 256 when the step reads t
            const int q = op.colour & 255;
            const bool from_t = op.colour >= 256;
            const T *xin = from_t ? (const T *)L.t : (const T *)x;
            T *xout = from_t ? x : (T *)L.t;
            const int tpr = row_tpr(KL, L.tpr);
            const T c1 = (T)L.cheb_c1[q], c2 = (T)L.cheb_c2[q];
#define C11(KLv, TPRv, ...) case KT_CODE(KLv, TPRv): blaunch(bk_cheb<T, KLv, TPRv>, L.nlong + nblocks((int64_t)n * KLv * TPRv), s, n, k, L.rp, L.ci, val, diag, idiag, (const T *)b, xin, xout, (T *)L.d, c1, c2, (q == 0 ? 1 : 0) | (q == L.cheb_m - 1 ? 2 : 0), L.lrows, (int)L.nlong); break;
            switch (KT_CODE(KL, tpr)) { KT_CASES(C11) }
#undef C11
            break;
        }
        case OP_CHEB_COPY:
            blaunch(bk_copy<T>, nblocks((int64_t)n * k), s, (int64_t)n * k, (const T *)L.t, x);
            break;
        case OP_CHEB_FIRST:
            blaunch(bk_cheb_first<T>, nblocks((int64_t)n * k), s, (int64_t)n * k, k, idiag, (const T *)b,
                    (T)L.cheb_c2[0], op.colour ? (T *)L.t : x, L.cheb_m > 1 ? (T *)L.d : (T *)nullptr);
            break;
    }
}

#define KL_SWITCH(KL, CALL) \
    switch (KL) {           \
        case 1: { constexpr int KLc = 1; CALL; } break;   \
        case 2: { constexpr int KLc = 2; CALL; } break;   \
        case 4: { constexpr int KLc = 4; CALL; } break;   \
        case 8: { constexpr int KLc = 8; CALL; } break;   \
        case 16: { constexpr int KLc = 16; CALL; } break; \
        default: { constexpr int KLc = 32; CALL; } break; \
    }

static void cg_spmv_dot(lamg_hier *h, BatchCtx *c, cudaStream_t s) {
    const DevLevel &F = h->dev[0];
    const int n = (int)F.n, k = c->k;
    if (c->KL == 1 && F.rs_tpr == 0) {
        blaunch(bk_spmv_dot_sell, rblocks(n), s, n, (const int32_t *)F.sl_ptr, (const int32_t *)F.sl_col,
                (const double *)F.sl_val, (const double *)F.diag, (const double *)c->p, c->q, c->red);
        return;
    }
    const int tpr = row_tpr(c->KL, F.tpr);
#define C9(KLv, TPRv, ...) case KT_CODE(KLv, TPRv): blaunch(bk_spmv_dot<KLv, TPRv>, rblocks((int64_t)n * KLv * TPRv), s, n, k, F.rp, F.ci, (const double *)F.val, (const double *)F.diag, (const double *)c->p, c->q, c->red, (const int32_t *)F.lrows, (int)F.nlong); break;
    switch (KT_CODE(c->KL, tpr)) { KT_CASES(C9) }
#undef C9
}

static void cg_true_resid(lamg_hier *h, BatchCtx *c, cudaStream_t s) {
    const DevLevel &F = h->dev[0];
    const int n = (int)F.n, k = c->k;
    const int tpr = row_tpr(c->KL, F.tpr);
#define C10(KLv, TPRv, ...) case KT_CODE(KLv, TPRv): blaunch(bk_true_resid<KLv, TPRv>, rblocks((int64_t)n * KLv * TPRv), s, n, k, F.rp, F.ci, (const double *)F.val, (const double *)F.diag, (const double *)c->xs, (const double *)c->bkeep, c->red, (const int32_t *)F.lrows, (int)F.nlong); break;
    switch (KT_CODE(c->KL, tpr)) { KT_CASES(C10) }
#undef C10
}

// Second half of a CG iteration: cycle on the residual, projection, dots, new direction.
template <typename T>
static void cg_tail(lamg_hier *h, BatchCtx *c, cudaStream_t s) {
    const int n = (int)h->dev[0].n, k = c->k;
    const int64_t cnt = (int64_t)n * k;
    if (c->prec == LAMG_FP32) blaunch(bk_cast<double, float>, nblocks(cnt), s, cnt, (const double *)c->r, (float *)c->b0);
    for (int i = 0; i < (int)h->ops.size(); i++) {
        if (start_fusable(h, i, false)) {
            bop<T>(h->ops[i], c, s, &h->ops[i + 1]);
            i++;
        } else {
            bop<T>(h->ops[i], c, s, nullptr);
        }
    }
    if (c->prec == LAMG_FP32) blaunch(bk_cast<float, double>, nblocks(cnt), s, cnt, (const float *)c->lv[0].x, c->z64);
    KL_SWITCH(c->KL, blaunch(bk_sum<KLc>, rblocks((int64_t)n * KLc), s, n, k, (const double *)c->z64, c->red));
    KL_SWITCH(c->KL, blaunch(bk_proj_dots<KLc>, rblocks((int64_t)n * KLc), s, n, k, c->z64, (const double *)c->zold,
                             (const double *)c->r, c->red));
    KL_SWITCH(c->KL, blaunch(bk_update_p<KLc>, nblocks((int64_t)n * KLc), s, n, k, (const double *)c->z64, c->p,
                             c->zold, c->red));
}

static void cg_head(lamg_hier *h, BatchCtx *c, cudaStream_t s) {
    const int n = (int)h->dev[0].n, k = c->k;
    cg_spmv_dot(h, c, s);
    KL_SWITCH(c->KL, blaunch(bk_update_xr<KLc>, rblocks((int64_t)n * KLc), s, n, k, c->xs, c->r, (const double *)c->p,
                             (const double *)c->q, c->red));
    cudaMemcpyAsync(c->h_sk, c->red.sk, B_COUNT * KMAX * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(c->h_sk + B_COUNT * KMAX, c->red.done, KMAX * sizeof(int), cudaMemcpyDeviceToHost, s);
}

static int capture_ctx(lamg_hier *h, BatchCtx *c) {
    cudaStream_t cs = h->stream;
    for (int which = 0; which < 2; which++) {
        cudaGraph_t g = nullptr;
        CKR(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = t_blaunches;
        if (which == 0) {
            if (c->prec == LAMG_FP32) cg_tail<float>(h, c, cs);
            else cg_tail<double>(h, c, cs);
        } else {
            cg_head(h, c, cs);
        }
        (which == 0 ? c->n_tail : c->n_head) = t_blaunches - l0;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaGraphInstantiate(which == 0 ? &c->g_tail : &c->g_head, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return LAMG_OK;
}

static int get_ctx(lamg_hier *h, int k, int prec, BatchCtx **out) {
    for (BatchCtx *b : h->batch)
        if (b->k == k && b->prec == prec) { *out = b; return LAMG_OK; }
    BatchCtx *c = new BatchCtx();
    c->k = k;
    c->prec = prec;
    c->KL = pow2_at_least(k);
    int rc = prec == LAMG_FP32 ? build_ctx<float>(h, c) : build_ctx<double>(h, c);
    if (!rc) rc = capture_ctx(h, c);
    if (rc) { batch_free(c); return rc; }
    h->batch.push_back(c);
    *out = c;
    return LAMG_OK;
}

// The k-column flexible-CG solve (FP64 outer iteration, cycle in the context's precision).
int solve_batch_impl(lamg_hier *h, int k, const double *B, double *PHI, const lamg_solve_opts *so,
                     lamg_stats *st, int prec) {
    if (k < 1 || k > KMAX || !B || !PHI || !so || !(so->tol > 0) || so->maxit < 1) return LAMG_ERR_INVALID;
    BatchCtx *c = nullptr;
    int rc = get_ctx(h, k, prec, &c);
    if (rc) return rc;
    cudaStream_t s = so->stream ? (cudaStream_t)so->stream : h->stream;
    const bool devp = so->flags & LAMG_DEVICE_PTRS;
    const int n = (int)h->dev[0].n;
    const int64_t cnt = (int64_t)n * k;
    CKR(cudaEventRecord(h->ev_a, s));
    // host vectors of a few hundred MB and more: pipelined pinned chunks with threaded host copies
    const bool staged = !devp && (size_t)cnt * sizeof(double) >= staged_copy_min_bytes();
    if (staged) {
        if ((rc = h2d_staged(c->nat_in, B, cnt * sizeof(double), s, h->wait_timeout_s))) return rc;
    } else {
        CKR(cudaMemcpyAsync(c->nat_in, B, cnt * sizeof(double), devp ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    }
    c->h_sk[B_TOL2 * KMAX] = so->tol * so->tol;
    CKR(cudaMemcpyAsync(c->red.sk + B_TOL2 * KMAX, c->h_sk + B_TOL2 * KMAX, sizeof(double), cudaMemcpyHostToDevice, s));
    KL_SWITCH(c->KL, blaunch(bk_gather_rows<KLc>, nblocks((int64_t)n * KLc), s, n, k, (const int32_t *)h->perm0,
                             (const double *)c->nat_in, c->r));
    KL_SWITCH(c->KL, blaunch(bk_sum<KLc>, rblocks((int64_t)n * KLc), s, n, k, (const double *)c->r, c->red));
    KL_SWITCH(c->KL, blaunch(bk_init_b<KLc>, rblocks((int64_t)n * KLc), s, n, k, c->r, c->bkeep, c->xs, c->p, c->zold,
                             c->red));
    CKR(cudaGetLastError());
    CKR(cudaEventRecord(h->ev_k0, s));
    CKR(cudaGraphLaunch(c->g_tail, s));
    int it = 0, cycles = 1;
    bool all_done = false;
    std::vector<double> rel(k, 1.0);
    if (st)
        for (int j = 0; j < k; j++)
            if (st[j].hist) st[j].hist[0] = 1.0;
    const int *hdone = (const int *)(c->h_sk + B_COUNT * KMAX);
    while (it < so->maxit) {
        CKR(cudaGraphLaunch(c->g_head, s));
        CKR(cudaEventRecord(h->ev_poll, s));
        if ((rc = wait_event(h, h->ev_poll))) return rc;
        it++;
        all_done = true;
        for (int j = 0; j < k; j++) {
            const double bn2 = c->h_sk[B_BN2 * KMAX + j];
            rel[j] = bn2 > 0 ? std::sqrt(c->h_sk[B_RR * KMAX + j] / bn2) : 0.0;
            if (st && st[j].hist && (hdone[j] == 0 || (int)c->h_sk[B_ITERS * KMAX + j] == it)) st[j].hist[it] = rel[j];
            all_done = all_done && hdone[j];
        }
        if (all_done) break;
        CKR(cudaGraphLaunch(c->g_tail, s));
        cycles++;
    }
    CKR(cudaEventRecord(h->ev_k1, s));
    cg_true_resid(h, c, s);
    KL_SWITCH(c->KL, blaunch(bk_scatter_rows<KLc>, nblocks((int64_t)n * KLc), s, n, k, (const int32_t *)h->perm0,
                             (const double *)c->xs, c->nat_out));
    if (!staged)
        CKR(cudaMemcpyAsync(PHI, c->nat_out, cnt * sizeof(double), devp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CKR(cudaMemcpyAsync(c->h_sk, c->red.sk, B_COUNT * KMAX * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKR(cudaMemcpyAsync(c->h_sk + B_COUNT * KMAX, c->red.done, KMAX * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (staged && (rc = d2h_staged(PHI, c->nat_out, cnt * sizeof(double), s, h->wait_timeout_s))) return rc;
    CKR(cudaEventRecord(h->ev_b, s));
    if ((rc = wait_event(h, h->ev_b))) return rc;
    CKR(cudaGetLastError());
    if (st) {
        float ms = 0.f, kms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_a, h->ev_b);
        cudaEventElapsedTime(&kms, h->ev_k0, h->ev_k1);
        const double z0 = (double)h->dev[0].nnz, n0 = (double)n;
        const int pi = prec == LAMG_FP32 ? 1 : 0;
        // per cycle: operator bytes once, vector bytes per column (+ the FP32 casts of r and z);
        // per CG iteration: SpMV operator once, 136 bytes per row and column of CG vectors
        const double cyc = h->cycle_mat[pi] + (double)k * (h->cycle_vec[pi] + (pi ? 24 * n0 : 0.0));
        const double per_it = 12 * z0 + 12 * n0 + 136 * n0 * k;
        const double once = 12 * z0 + 12 * n0 + 24 * n0 * k + 80 * n0 * k;
        for (int j = 0; j < k; j++) {
            const double bn2 = c->h_sk[B_BN2 * KMAX + j];
            st[j].iters = hdone[j] ? (int)c->h_sk[B_ITERS * KMAX + j] : it;
            st[j].nlevels = (int32_t)h->dev.size();
            st[j].relres = bn2 > 0 ? std::sqrt(c->h_sk[B_RR * KMAX + j] / bn2) : 0.0;
            st[j].relres_true = bn2 > 0 ? std::sqrt(c->h_sk[B_TRUE_RR * KMAX + j] / bn2) : 0.0;
            st[j].b_mean = c->h_sk[B_BMEAN * KMAX + j];
            st[j].solve_ms = ms;
            st[j].kernel_ms = kms;
            st[j].alg_bytes = ((double)cycles * cyc + (double)it * per_it + once) / k;  // this column's share
            st[j].launches = 3 + (int64_t)cycles * c->n_tail + (int64_t)it * (c->n_head + 1);
        }
    }
    return all_done ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
}

// Cold-L2 device time of one k-column kernel of the cycle or the outer CG (lamg_time_kernel_batch):
// which 0 residual at an aggregation level, 1 one smoothing sweep at an aggregation level (every
// colour class of Gauss-Seidel, or the cheb_degree steps of the Chebyshev polynomial), 2 the outer
// CG product q = A p with its dots (level 0, FP64), 3 one Chebyshev step (Chebyshev levels). Algorithmic bytes count each operator array
// once, each vector once per column (a gathered vector at most once per launch); flops count one
// multiply-add (2 flops) per stored entry and column plus the per-row arithmetic.
template <typename T>
static int time_batch(lamg_hier *h, BatchCtx *c, int which, int level, int reps, double *out) {
    const DevLevel &D = h->dev[level];
    const double n = (double)D.n, z = (double)D.nnz, k = (double)c->k, sz = (double)sizeof(T);
    std::vector<Op> seq;
    double bytes = 0.0, flops = 0.0;
    if (which == 0) {
        seq.push_back({OP_RESID, level, 0});
        bytes = (4 + sz) * z + 4 * (n + 1) + sz * n + k * sz * 3 * n;
        flops = k * (2 * z + 4 * n);
    } else if ((which == 1 || which == 3) && D.cheb) {
        // which 1: one polynomial from x back into x (steps alternate x -> t -> x ..., a copy
        // t -> x after an odd count); which 3: its first step alone (bk_cheb, x -> t). Per row
        // and column a step reads b and the iterate (its own entry and the gathered ones count
        // once) and writes the new iterate, reads the direction d after the first step and
        // writes it before the last; flops: the product (2 per entry), r = b - (A_uu x + s) (3),
        // d = c1 d + c2 r / A_uu (2 on the first step, 4 after it), x + d (1).
        const int m = h->opt.cheb_degree, steps = which == 3 ? 1 : m;
        for (int q = 0; q < steps; q++) {
            seq.push_back({OP_CHEB, level, q + 256 * (q & 1)});
            const double vecs = 3 + (q > 0 ? 1 : 0) + (q < m - 1 ? 1 : 0);
            bytes += (4 + sz) * z + 4 * (n + 1) + 2 * sz * n + k * sz * vecs * n;
            flops += k * (2 * z + (q ? 8 : 6) * n);
        }
        if (which == 1 && (m & 1)) {
            seq.push_back({OP_CHEB_COPY, level, 0});
            bytes += k * sz * 2 * n;
        }
    } else if (which == 1) {
        std::vector<int32_t> rp(D.n + 1);
        CKR(cudaMemcpy(rp.data(), D.rp, (D.n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        for (int col = 0; col < D.ncol; col++) {
            const int64_t r0 = D.cptr[col], r1 = D.cptr[col + 1];
            const double R = (double)(r1 - r0), zc = (double)(rp[r1] - rp[r0]);
            seq.push_back({OP_GS, level, col});
            bytes += (4 + sz) * zc + 4 * (R + 1) + sz * R + k * sz * (2 * R + std::min(zc, n));
            flops += k * (2 * zc + 2 * R);
        }
    } else if (which == 2) {
        bytes = 12 * z + 4 * (n + 1) + 8 * n + k * 8 * 2 * n;
        flops = k * (2 * z + 4 * n);
    } else {
        return LAMG_ERR_INVALID;
    }
    cudaStream_t s = h->stream;
    const size_t flush_bytes = (size_t)256 << 20;
    void *flush = nullptr;
    CKR(cudaMalloc(&flush, flush_bytes));
    double total = 0.0;
    int rc = LAMG_OK;
    int64_t launches = 0;
    for (int r = 0; r < reps && !rc; r++) {
        cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);
        cudaEventRecord(h->ev_a, s);
        const int64_t l0 = t_blaunches;
        if (which == 2) cg_spmv_dot(h, c, s);
        else for (const Op &op : seq) bop<T>(op, c, s, nullptr);
        launches = t_blaunches - l0;
        cudaEventRecord(h->ev_b, s);
        rc = wait_event(h, h->ev_b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_a, h->ev_b);
        total += ms;
    }
    cudaFree(flush);
    if (rc) return rc;
    CKR(cudaGetLastError());
    out[0] = total / reps;
    out[1] = bytes;
    out[2] = (double)launches;
    out[3] = flops;
    return LAMG_OK;
}

}  // namespace lamg

extern "C" int lamg_time_kernel_batch(lamg_hier *h, int32_t which, int32_t level, int32_t k, int32_t reps,
                                      double *out) {
    using namespace lamg;
    if (!h || !out || reps < 1 || k < 1 || k > KMAX || level < 0 || level >= (int32_t)h->dev.size())
        return LAMG_ERR_INVALID;
    if ((which == 0 || which == 1 || which == 3) && h->dev[level].kind != KIND_AGG) return LAMG_ERR_INVALID;
    if (which == 3 && !h->dev[level].cheb) return LAMG_ERR_INVALID;
    if (which == 2 && level != 0) return LAMG_ERR_INVALID;
    if (which < 0 || which > 3) return LAMG_ERR_INVALID;
    CKR(cudaSetDevice(h->device));
    const int prec = h->opt.precision == LAMG_FP32 ? LAMG_FP32 : LAMG_FP64;
    BatchCtx *c = nullptr;
    int rc = get_ctx(h, k, prec, &c);
    if (rc) return rc;
    return prec == LAMG_FP32 ? time_batch<float>(h, c, which, level, reps, out)
                             : time_batch<double>(h, c, which, level, reps, out);
}

extern "C" int lamg_solve_batch(lamg_hier *h, int32_t k, const double *B, double *PHI, const lamg_solve_opts *so,
                                lamg_stats *st) {
    using namespace lamg;
    if (!h) return LAMG_ERR_INVALID;
    CKR(cudaSetDevice(h->device));
    return lamg::solve_batch_impl(h, k, B, PHI, so, st, h->opt.precision == LAMG_FP32 ? LAMG_FP32 : LAMG_FP64);
}
