// sm_103a kernels of the LAMG+ solve phase: the cycle steps of Section 2 (colour-ordered
// Gauss-Seidel, residual, restriction P^T, prolongation P with caliber-2 rows, elimination
// transfers of Eq. 2, dense coarsest solve with the mean-zero projection of Eq. 1) and the
// vector kernels of the flexible CG outer iteration.
//
// All of these are memory-bound (no step is a dense contraction) and the cycle is a long chain
// of small dependent steps, so the kernels are built for latency:
//  - Programmatic dependent launch: every kernel lets the next one launch as soon as it has
//    started (griddepcontrol.launch_dependents), loads the operands that only setup writes
//    (row pointers, column ids, values, diagonals, transfer weights) and only then waits for
//    the previous kernel to finish (griddepcontrol.wait) before touching the vectors the
//    solve writes. Launch latency and the first two links of each row's load chain overlap
//    the previous step. Every thread reaches the wait, so a kernel never completes before its
//    predecessor and completion order stays transitive along the chain.
//  - CSR rows are handled by groups of TPR lanes (coalesced column/value loads), combined with
//    warp shuffles.
//  - Reductions are deterministic: fixed per-block partials, added in a fixed order by the
//    last block to finish (found with an atomic ticket, not a spin-wait).
#include <cuda_runtime.h>

#include "device.h"
#include "kernels_common.cuh"

namespace lamg {

constexpr int BS = 256;

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


// Grid-wide deterministic sum: every block publishes its partials, the last block to arrive
// adds all partials in block order. Returns true in the last block, whose thread 0 holds the
// totals in v. Must be reached by every thread of every block. The last block reads only the
// partials (published by a fence before the ticket); the kernel's other writes reach the next
// kernel through the launch boundary (its griddepcontrol.wait returns once this grid's memory
// operations are complete and visible), so threads do not fence them here.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], const Reduce red) {
    __shared__ bool last;
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

// A CSR row held by a group of TPR lanes: the first two entries of each lane are loaded before
// the dependency wait, the rest (long rows only) after it.
struct RowPre {
    int e0, e1, c0, c1;
    double v0, v1;
};

template <int TPR>
__device__ __forceinline__ RowPre row_pre(bool ok, int row, int sub, const int32_t *__restrict__ rp,
                                          const int32_t *__restrict__ ci, const double *__restrict__ val) {
    RowPre p;
    p.e0 = ok ? rp[row] + sub : 0;
    p.e1 = ok ? rp[row + 1] : 0;
    p.c0 = -1; p.c1 = -1; p.v0 = 0.0; p.v1 = 0.0;
    if (p.e0 < p.e1) { p.c0 = ci[p.e0]; p.v0 = val[p.e0]; }
    if (p.e0 + TPR < p.e1) { p.c1 = ci[p.e0 + TPR]; p.v1 = val[p.e0 + TPR]; }
    return p;
}

// sum_e val[e] x[ci[e]] over the row (after the wait); group total on every lane of the group.
template <int TPR>
__device__ __forceinline__ double row_finish(const RowPre &p, const int32_t *__restrict__ ci,
                                             const double *__restrict__ val, const double *x) {
    double s = 0.0;
    if (p.c0 >= 0) s += p.v0 * x[p.c0];
    if (p.c1 >= 0) s += p.v1 * x[p.c1];
    for (int e = p.e0 + 2 * TPR; e < p.e1; e += TPR) s += val[e] * x[ci[e]];
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// A row longer than LONG_ROW entries summed by the whole block: thread t takes entries
// e0 + t, e0 + t + BS, ..., then a fixed-order block reduction; the total is valid in thread 0.
__device__ __forceinline__ double block_row(int e0, int e1, const int32_t *__restrict__ ci,
                                            const double *__restrict__ val, const double *x) {
    double v[1] = {0.0};
    for (int e = e0 + (int)threadIdx.x; e < e1; e += BS) v[0] += val[e] * x[ci[e]];
    block_sum<1>(v);
    return v[0];
}

// Lane-group rows of a pass over all rows skip the long rows (a block takes each of those).
__device__ __forceinline__ void drop_long(RowPre &p, bool &ok, int sub) {
    if (ok && p.e1 - (p.e0 - sub) > LONG_ROW) {
        ok = false;
        p.e0 = p.e1;
        p.c0 = -1;
        p.c1 = -1;
    }
}

// ------------------------------------------------------------------------------- cycle steps

// One colour class [r0, r1) of Gauss-Seidel (Section 2): x_u = (b_u - sum_v A_uv x_v) / A_uu.
// (b_u - sum) times the stored reciprocal of A_uu: one FP64 multiply instead of a division,
// whose Newton iteration costs about ten FP64 instructions on a part with few FP64 units.
// The class's first nl rows are long (rows are sorted longest first inside a class): block b
// < nl takes row r0 + b, the other blocks the rows from r0 + nl on.
template <int TPR>
__global__ void __launch_bounds__(BS) k_gs(int r0, int r1, int nl, const int32_t *__restrict__ rp,
                                           const int32_t *__restrict__ ci,
                                           const double *__restrict__ val,
                                           const double *__restrict__ idiag,
                                           const double *__restrict__ b, double *x) {
    pdl_trigger();
    if ((int)blockIdx.x < nl) {
        const int row = r0 + (int)blockIdx.x;
        const int e0 = rp[row], e1 = rp[row + 1];
        const double id = idiag[row];
        pdl_wait();
        const double s = block_row(e0, e1, ci, val, x);
        if (threadIdx.x == 0) x[row] = (b[row] - s) * id;
        return;
    }
    const int g = r0 + nl + (int)(((blockIdx.x - nl) * (unsigned)BS + threadIdx.x) / TPR);
    const int sub = threadIdx.x % TPR;
    const bool ok = g < r1;
    const RowPre p = row_pre<TPR>(ok, g, sub, rp, ci, val);
    const double id = ok ? idiag[g] : 1.0;
    pdl_wait();
    const double s = row_finish<TPR>(p, ci, val, x);
    if (ok && sub == 0) x[g] = (b[g] - s) * id;
}

// --------------------------------------------------- sliced ELLPACK, one thread per row
//
// Rows in 32-row slices stored in four-entry blocks (sell_col_at / sell_val_at): a thread reads
// its row's column ids four at a time (one int4) and its values two at a time (two double2 per
// block), and every such load of a warp is 512 contiguous bytes. Every row is summed by one
// thread in entry order, without a shuffle tree: on a part with few FP64 units the FP64
// instruction count per row is what bounds these kernels. Padding entries hold value 0 at a
// valid column (adding 0 * x to a sum that started at +0 leaves its bits unchanged). The slice
// bounds and the first block of four entries are loaded before the dependency wait.
struct SellPre {
    int a, l, w;        // slice base, lane in the slice, slice width (a multiple of 4)
    int4 c;             // the first four column ids
    double2 v01, v23;   // the first four values
};

__device__ __forceinline__ int4 sell_ids(const int32_t *__restrict__ sc, int a, int l, int q) {
    return __ldg(reinterpret_cast<const int4 *>(sc + a + 128 * q + 4 * l));
}
__device__ __forceinline__ double2 sell_vals(const double *__restrict__ sv, int a, int l, int q, int h) {
    return __ldg(reinterpret_cast<const double2 *>(sv + a + 128 * q + 64 * h + 2 * l));
}

__device__ __forceinline__ SellPre sell_pre(bool ok, int row, const int32_t *__restrict__ sp,
                                            const int32_t *__restrict__ sc, const double *__restrict__ sv) {
    SellPre p;
    const int s = row >> 5;
    p.l = row & 31;
    p.a = ok ? sp[s] : 0;
    p.w = ok ? (sp[s + 1] - p.a) >> 5 : 0;
    if (p.w > 0) {
        p.c = sell_ids(sc, p.a, p.l, 0);
        p.v01 = sell_vals(sv, p.a, p.l, 0, 0);
        p.v23 = sell_vals(sv, p.a, p.l, 0, 1);
    } else {
        p.c = make_int4(0, 0, 0, 0);
        p.v01 = p.v23 = make_double2(0.0, 0.0);
    }
    return p;
}

// The whole row after the dependency wait (kernels with nothing to load before it).
__device__ __forceinline__ double sell_row(int row, const int32_t *__restrict__ sp, const int32_t *__restrict__ sc,
                                           const double *__restrict__ sv, const double *x) {
    const int sl = row >> 5, l = row & 31;
    const int a = sp[sl], nq = (sp[sl + 1] - a) >> 7;
    double s = 0.0;
    for (int q = 0; q < nq; q++) {
        const int4 c = sell_ids(sc, a, l, q);
        const double2 va = sell_vals(sv, a, l, q, 0), vb = sell_vals(sv, a, l, q, 1);
        const double x0 = x[c.x], x1 = x[c.y], x2 = x[c.z], x3 = x[c.w];
        s += va.x * x0;
        s += va.y * x1;
        s += vb.x * x2;
        s += vb.y * x3;
    }
    return s;
}

__device__ __forceinline__ double sell_finish(const SellPre &p, const int32_t *__restrict__ sc,
                                              const double *__restrict__ sv, const double *x) {
    double s = 0.0;
    if (p.w <= 0) return s;
    {
        const double x0 = x[p.c.x], x1 = x[p.c.y], x2 = x[p.c.z], x3 = x[p.c.w];
        s += p.v01.x * x0;
        s += p.v01.y * x1;
        s += p.v23.x * x2;
        s += p.v23.y * x3;
    }
    for (int q = 1; q < (p.w >> 2); q++) {
        const int4 c = sell_ids(sc, p.a, p.l, q);
        const double2 va = sell_vals(sv, p.a, p.l, q, 0), vb = sell_vals(sv, p.a, p.l, q, 1);
        const double x0 = x[c.x], x1 = x[c.y], x2 = x[c.z], x3 = x[c.w];
        s += va.x * x0;
        s += va.y * x1;
        s += vb.x * x2;
        s += vb.y * x3;
    }
    return s;
}

// One colour class [r0, r1) of Gauss-Seidel; thread t of the launch takes row 32 s0 + t
// (s0 = first slice touching the class).
__global__ void __launch_bounds__(64) k_gs_sell(int r0, int r1, int s0, const int32_t *__restrict__ sp,
                                                const int32_t *__restrict__ sc, const double *__restrict__ sv,
                                                const double *__restrict__ idiag,
                                                const double *__restrict__ b, double *x) {
    pdl_trigger();
    const int row = 32 * s0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool ok = row >= r0 && row < r1;
    const SellPre p = sell_pre(ok, row, sp, sc, sv);
    const double id = ok ? idiag[row] : 1.0;
    pdl_wait();
    if (!ok) return;
    const double s = sell_finish(p, sc, sv, x);
    x[row] = (b[row] - s) * id;
}

// r = b - A x
__global__ void __launch_bounds__(BS) k_resid_sell(int n, const int32_t *__restrict__ sp,
                                                   const int32_t *__restrict__ sc, const double *__restrict__ sv,
                                                   const double *__restrict__ diag, const double *__restrict__ x,
                                                   const double *__restrict__ b, double *r) {
    pdl_trigger();
    const int row = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool ok = row < n;
    const SellPre p = sell_pre(ok, row, sp, sc, sv);
    const double d = ok ? diag[row] : 0.0;
    pdl_wait();
    if (!ok) return;
    const double s = sell_finish(p, sc, sv, x);
    r[row] = b[row] - (d * x[row] + s);
}

// First sweep from x = 0: rows of colour 0 ([0, c1)) have no updated neighbours yet, so
// x_u = b_u / A_uu there; every other row starts at 0.
__global__ void k_gs_first(int n, int c1, const double *__restrict__ idiag,
                           const double *__restrict__ b, double *x) {
    pdl_trigger();
    const int i = blockIdx.x * BS + threadIdx.x;
    const double id = (i < c1) ? idiag[i] : 1.0;
    pdl_wait();
    if (i >= n) return;
    x[i] = i < c1 ? b[i] * id : 0.0;
}

__global__ void k_zero(int n, double *x) {
    pdl_trigger();
    pdl_wait();
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i < n) x[i] = 0.0;
}

// r = b - A x; blocks b < nl take the long rows lr[b]
template <int TPR>
__global__ void __launch_bounds__(BS) k_resid(int n, const int32_t *__restrict__ rp,
                                              const int32_t *__restrict__ ci,
                                              const double *__restrict__ val,
                                              const double *__restrict__ diag,
                                              const double *__restrict__ x,
                                              const double *__restrict__ b, double *r,
                                              const int32_t *__restrict__ lr, int nl) {
    pdl_trigger();
    if ((int)blockIdx.x < nl) {
        const int row = lr[blockIdx.x];
        const int e0 = rp[row], e1 = rp[row + 1];
        const double d = diag[row];
        pdl_wait();
        const double s = block_row(e0, e1, ci, val, x);
        if (threadIdx.x == 0) r[row] = b[row] - (d * x[row] + s);
        return;
    }
    const int g = (int)(((blockIdx.x - nl) * (unsigned)BS + threadIdx.x) / TPR);
    const int sub = threadIdx.x % TPR;
    bool ok = g < n;
    RowPre p = row_pre<TPR>(ok, g, sub, rp, ci, val);
    drop_long(p, ok, sub);
    const double d = ok ? diag[g] : 0.0;
    pdl_wait();
    const double s = row_finish<TPR>(p, ci, val, x);
    if (ok && sub == 0) r[g] = b[g] - (d * x[g] + s);
}

// One step of the Chebyshev smoothing polynomial: every row from the previous iterate xin,
// r_u = b_u - (A xin)_u, d_u <- c1 d_u + c2 r_u / A_uu (first step, flags bit 0: d_u = c2 r_u /
// A_uu), xout_u = xin_u + d_u; d is not stored on the last step of the polynomial (flags bit 1),
// where nothing reads it. Blocks b < nl take the long rows lr[b].
template <int TPR>
__global__ void __launch_bounds__(BS) k_cheb(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                             const double *__restrict__ val, const double *__restrict__ diag,
                                             const double *__restrict__ idiag, const double *__restrict__ b,
                                             const double *xin, double *xout, double *d, double c1, double c2,
                                             int flags, const int32_t *__restrict__ lr, int nl) {
    const bool first = flags & 1, last = flags & 2;
    pdl_trigger();
    if ((int)blockIdx.x < nl) {
        const int row = lr[blockIdx.x];
        const int e0 = rp[row], e1 = rp[row + 1];
        const double dg = diag[row], id = idiag[row];
        pdl_wait();
        const double s = block_row(e0, e1, ci, val, xin);
        if (threadIdx.x == 0) {
            const double r = b[row] - (dg * xin[row] + s);
            const double dn = (first ? 0.0 : c1 * d[row]) + c2 * r * id;
            if (!last) d[row] = dn;
            xout[row] = xin[row] + dn;
        }
        return;
    }
    const int g = (int)(((blockIdx.x - nl) * (unsigned)BS + threadIdx.x) / TPR);
    const int sub = threadIdx.x % TPR;
    bool ok = g < n;
    RowPre p = row_pre<TPR>(ok, g, sub, rp, ci, val);
    drop_long(p, ok, sub);
    const double dg = ok ? diag[g] : 0.0, id = ok ? idiag[g] : 0.0;
    pdl_wait();
    const double s = row_finish<TPR>(p, ci, val, xin);
    if (ok && sub == 0) {
        const double r = b[g] - (dg * xin[g] + s);
        const double dn = (first ? 0.0 : c1 * d[g]) + c2 * r * id;
        if (!last) d[g] = dn;
        xout[g] = xin[g] + dn;
    }
}

// First Chebyshev step from x = 0: out = (c2 b) / A_uu as the reciprocal product of k_cheb with
// r = b (the step's direction d = out is stored when the polynomial continues).
__global__ void k_cheb_first(int n, const double *__restrict__ idiag, const double *__restrict__ b, double c2,
                             double *out, double *d) {
    pdl_trigger();
    pdl_wait();
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i >= n) return;
    const double v = c2 * b[i] * idiag[i];
    out[i] = v;
    if (d) d[i] = v;
}

__global__ void k_copy(int n, const double *__restrict__ src, double *dst) {
    pdl_trigger();
    pdl_wait();
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

// Restriction b^c = P^T r (Section 2): segmented sum over the fine rows of each aggregate,
// caliber-2 rows contributing w or 1 - w.
//
// With xc set, the kernel also starts the coarse level's first visit, which begins from x = 0:
// xc_a = b^c_a / A_aa on the coarse rows a < c1 (its first colour class, as k_gs_first), 0 on
// the others (c1 = 0: the whole iterate zeroed, as k_zero). Those steps are row-local, so they
// need no launch of their own.
template <int TPR>
__global__ void __launch_bounds__(BS) k_restrict(int nc, const int32_t *__restrict__ ptr,
                                                 const int32_t *__restrict__ row,
                                                 const double *__restrict__ w,
                                                 const double *__restrict__ r, double *bc, double *xc, int c1,
                                                 const double *__restrict__ idc) {
    pdl_trigger();
    const int a = (int)((blockIdx.x * (unsigned)BS + threadIdx.x) / TPR);
    const int sub = threadIdx.x % TPR;
    const bool ok = a < nc;
    const RowPre p = row_pre<TPR>(ok, a, sub, ptr, row, w);
    const double id = (xc && ok && a < c1) ? idc[a] : 0.0;
    pdl_wait();
    const double s = row_finish<TPR>(p, row, w, r);
    if (ok && sub == 0) {
        bc[a] = s;
        if (xc) xc[a] = a < c1 ? s * id : 0.0;
    }
}

// Prolongation x += P x^c: caliber-1 rows gather one coarse value, caliber-2 rows
// w x^c_a + (1 - w) x^c_b (Appendix A.2).
__global__ void k_prolong(int n, const int32_t *__restrict__ agg, const int32_t *__restrict__ agg2,
                          const double *__restrict__ wt, const double *__restrict__ xc, double *x) {
    pdl_trigger();
    const int u = blockIdx.x * BS + threadIdx.x;
    const bool ok = u < n;
    const int a = ok ? agg[u] : 0, b = ok ? agg2[u] : -1;
    const double w = (ok && b >= 0) ? wt[u] : 1.0;
    pdl_wait();
    if (!ok) return;
    double s;
    if (b < 0) {
        s = xc[a];
    } else {
        s = (1.0 - w) * xc[b];
        if (w != 0.0) s = w * xc[a] + s;
    }
    x[u] += s;
}

// Elimination restriction (Eq. 2): b^c_i = b_i + sum_f (P_F)_{f,i} b_f over the F neighbours.
// xc, c1, idc: the start of the coarse level's first visit, as in k_restrict (the kernel reads
// no iterate, so the coarse iterate may share the fine one's memory).
__global__ void k_elim_restrict(int nc, const int32_t *__restrict__ ptr, const int32_t *__restrict__ f,
                                const double *__restrict__ pv, const double *__restrict__ b, double *bc,
                                double *xc, int c1, const double *__restrict__ idc) {
    pdl_trigger();
    const int i = blockIdx.x * BS + threadIdx.x;
    const bool ok = i < nc;
    const int e0 = ok ? ptr[i] : 0, e1 = ok ? ptr[i + 1] : 0;
    int f0 = -1, f1 = -1;
    double p0 = 0.0, p1 = 0.0;
    if (e0 < e1) { f0 = f[e0]; p0 = pv[e0]; }
    if (e0 + 1 < e1) { f1 = f[e0 + 1]; p1 = pv[e0 + 1]; }
    const double id = (xc && ok && i < c1) ? idc[i] : 0.0;
    pdl_wait();
    if (!ok) return;
    const double *bF = b + nc;
    double s = b[i];
    if (f0 >= 0) s += p0 * bF[f0];
    if (f1 >= 0) s += p1 * bF[f1];
    for (int e = e0 + 2; e < e1; e++) s += pv[e] * bF[f[e]];
    bc[i] = s;
    if (xc) xc[i] = i < c1 ? s * id : 0.0;
}

// Elimination interpolation (Eq. 2): x_F = P_F x_C + b_F / A_FF, ELL-4 rows.
__global__ void k_elim_interp(int nc, int nF, const int32_t *__restrict__ col,
                              const double *__restrict__ pv, const double *__restrict__ dF,
                              const double *__restrict__ b, double *x) {
    pdl_trigger();
    const int t = blockIdx.x * BS + threadIdx.x;
    const bool ok = t < nF;
    int c[4];
    double p[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        c[j] = ok ? col[4 * t + j] : -1;
        p[j] = ok ? pv[4 * t + j] : 0.0;
    }
    const double d = ok ? dF[t] : 1.0;
    pdl_wait();
    if (!ok) return;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; j++)
        if (c[j] >= 0) s += p[j] * x[c[j]];
    x[nc + t] = s + b[nc + t] / d;
}

// Coarsest level: x = Pi A^+ b with the mean-zero projection Pi = I - J/n folded into the stored
// dense matrix (one warp per row).
__global__ void __launch_bounds__(BS) k_coarse(int n, const double *__restrict__ pinv,
                                               const double *__restrict__ b, double *x) {
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * BS + threadIdx.x) >> 5, nwarps = (gridDim.x * BS) >> 5;
    for (int i = wg; i < n; i += nwarps) {
        // four partial sums per lane (columns lane, lane + 32, lane + 64, lane + 96, then every
        // 128th), added as (s0 + s1) + (s2 + s3) before the warp's shuffle tree: four
        // independent FP64 chains per lane instead of one n/32 long
        const double *row = pinv + (int64_t)i * n;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = lane;
        for (; j + 96 < n; j += 128) {
            s0 += row[j] * b[j];
            s1 += row[j + 32] * b[j + 32];
            s2 += row[j + 64] * b[j + 64];
            s3 += row[j + 96] * b[j + 96];
        }
        for (; j < n; j += 32) s0 += row[j] * b[j];
        double s = (s0 + s1) + (s2 + s3);
        s = warp_sum(s);
        if (lane == 0) x[i] = s;
    }
}

// ------------------------------------------------------------------------------- outer CG

__global__ void k_gather(int n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                         double *dst) {
    pdl_trigger();
    const int i = blockIdx.x * BS + threadIdx.x;
    const int j = i < n ? perm[i] : 0;
    pdl_wait();
    if (i < n) dst[i] = src[j];
}

__global__ void k_scatter(int n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                          double *dst) {
    pdl_trigger();
    const int i = blockIdx.x * BS + threadIdx.x;
    const int j = i < n ? perm[i] : 0;
    pdl_wait();
    if (i < n) dst[j] = src[i];
}

// S_MEAN = (sum v) / n
__global__ void __launch_bounds__(BS) k_sum(int n, const double *__restrict__ v, const Reduce red) {
    pdl_trigger();
    pdl_wait();
    double s[1] = {0.0};
    for (int i = blockIdx.x * BS + threadIdx.x; i < n; i += gridDim.x * BS) s[0] += v[i];
    if (grid_sum<1>(s, red) && threadIdx.x == 0) red.scal[S_MEAN] = s[0] / (double)n;
}

__global__ void k_sub_mean(int n, double *v, const Reduce red) {
    pdl_trigger();
    pdl_wait();
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i < n) v[i] -= red.scal[S_MEAN];
}

// b <- b - mean(b) (kept in bkeep), S_BN2 = ||b||^2; x = p = zold = 0, S_RZ = 1.
__global__ void __launch_bounds__(BS) k_init_b(int n, double *r, double *bkeep, double *x, double *p,
                                               double *zold, const Reduce red) {
    pdl_trigger();
    pdl_wait();
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

// q = A p, S_ALPHA = S_RZ / (p . q); block b takes the long rows lr[b], lr[b + grid], ...
template <int TPR>
__global__ void __launch_bounds__(BS) k_spmv_dot(int n, const int32_t *__restrict__ rp,
                                                 const int32_t *__restrict__ ci,
                                                 const double *__restrict__ val,
                                                 const double *__restrict__ diag,
                                                 const double *__restrict__ p, double *q,
                                                 const Reduce red, const int32_t *__restrict__ lr, int nl) {
    pdl_trigger();
    pdl_wait();
    const int groups = gridDim.x * (BS / TPR);
    const int sub = threadIdx.x % TPR;
    double pq[1] = {0.0};
    for (int t = blockIdx.x; t < nl; t += gridDim.x) {
        const int row = lr[t];
        const double s = block_row(rp[row], rp[row + 1], ci, val, p);
        if (threadIdx.x == 0) {
            const double qi = diag[row] * p[row] + s;
            q[row] = qi;
            pq[0] += p[row] * qi;
        }
    }
    const int rounds = (n + groups - 1) / groups;
    int g = (int)((blockIdx.x * (unsigned)BS + threadIdx.x) / TPR);
    for (int it = 0; it < rounds; it++, g += groups) {
        bool ok = g < n;
        int e0 = ok ? rp[g] + sub : 0, e1 = ok ? rp[g + 1] : 0;
        if (ok && e1 - (e0 - sub) > LONG_ROW) { ok = false; e0 = e1; }
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

// q = A p, S_ALPHA = S_RZ / (p . q), one thread per row (sliced ELLPACK)
__global__ void __launch_bounds__(BS, 8) k_spmv_dot_sell(int n, const int32_t *__restrict__ sp,
                                                      const int32_t *__restrict__ sc,
                                                      const double *__restrict__ sv,
                                                      const double *__restrict__ diag,
                                                      const double *__restrict__ p, double *q,
                                                      const Reduce red) {
    pdl_trigger();
    pdl_wait();
    double pq[1] = {0.0};
    for (int row = blockIdx.x * BS + threadIdx.x; row < n; row += gridDim.x * BS) {
        const double s = sell_row(row, sp, sc, sv, p);
        const double qi = diag[row] * p[row] + s;
        q[row] = qi;
        pq[0] += p[row] * qi;
    }
    if (grid_sum<1>(pq, red) && threadIdx.x == 0)
        red.scal[S_ALPHA] = pq[0] != 0.0 ? red.scal[S_RZ] / pq[0] : 0.0;
}

// x += alpha p, r -= alpha q, S_RR = ||r||^2
__global__ void __launch_bounds__(BS) k_update_xr(int n, double *x, double *r, const double *__restrict__ p,
                                                  const double *__restrict__ q, const Reduce red) {
    pdl_trigger();
    pdl_wait();
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
    pdl_trigger();
    pdl_wait();
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
    pdl_trigger();
    pdl_wait();
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i >= n) return;
    const double beta = red.scal[S_BETA];
    const double zi = z[i];
    p[i] = zi + beta * p[i];
    zold[i] = zi;
}

// S_TRUE_RR = ||b - A x||^2; long rows as in k_spmv_dot
template <int TPR>
__global__ void __launch_bounds__(BS) k_true_resid(int n, const int32_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci,
                                                   const double *__restrict__ val,
                                                   const double *__restrict__ diag,
                                                   const double *__restrict__ x,
                                                   const double *__restrict__ b, const Reduce red,
                                                   const int32_t *__restrict__ lr, int nl) {
    pdl_trigger();
    pdl_wait();
    const int groups = gridDim.x * (BS / TPR);
    const int sub = threadIdx.x % TPR;
    double acc[1] = {0.0};
    for (int t = blockIdx.x; t < nl; t += gridDim.x) {
        const int row = lr[t];
        const double s = block_row(rp[row], rp[row + 1], ci, val, x);
        if (threadIdx.x == 0) {
            const double ri = b[row] - (diag[row] * x[row] + s);
            acc[0] += ri * ri;
        }
    }
    const int rounds = (n + groups - 1) / groups;
    int g = (int)((blockIdx.x * (unsigned)BS + threadIdx.x) / TPR);
    for (int it = 0; it < rounds; it++, g += groups) {
        bool ok = g < n;
        int e0 = ok ? rp[g] + sub : 0, e1 = ok ? rp[g + 1] : 0;
        if (ok && e1 - (e0 - sub) > LONG_ROW) { ok = false; e0 = e1; }
        const double s = row_sum<TPR>(e0, e1, ci, val, x);
        if (ok && sub == 0) {
            const double ri = b[g] - (diag[g] * x[g] + s);
            acc[0] += ri * ri;
        }
    }
    if (grid_sum<1>(acc, red) && threadIdx.x == 0) red.scal[S_TRUE_RR] = acc[0];
}

// S_TRUE_RR = ||b - A x||^2, one thread per row (sliced ELLPACK)
__global__ void __launch_bounds__(BS, 8) k_true_resid_sell(int n, const int32_t *__restrict__ sp,
                                                        const int32_t *__restrict__ sc,
                                                        const double *__restrict__ sv,
                                                        const double *__restrict__ diag,
                                                        const double *__restrict__ x,
                                                        const double *__restrict__ b, const Reduce red) {
    pdl_trigger();
    pdl_wait();
    double acc[1] = {0.0};
    for (int row = blockIdx.x * BS + threadIdx.x; row < n; row += gridDim.x * BS) {
        const double s = sell_row(row, sp, sc, sv, x);
        const double ri = b[row] - (diag[row] * x[row] + s);
        acc[0] += ri * ri;
    }
    if (grid_sum<1>(acc, red) && threadIdx.x == 0) red.scal[S_TRUE_RR] = acc[0];
}

// ------------------------------------------------------------------------------- launchers

static bool g_pdl = true;

void set_pdl(bool on) { g_pdl = on; }
bool pdl_enabled() { return g_pdl; }

// Launch with programmatic stream serialisation, so the kernel may start while its
// predecessor in the stream is still running (it waits for it at griddepcontrol.wait).
template <typename... KArgs, typename... Args>
static void launch(void (*kernel)(KArgs...), unsigned grid, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid < 1 ? 1 : grid);
    cfg.blockDim = dim3(BS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
static void launch_bs(void (*kernel)(KArgs...), unsigned grid, unsigned bs, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid < 1 ? 1 : grid);
    cfg.blockDim = dim3(bs);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

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

#define TPR_DISPATCH(tpr, KERNEL, GRID, ...)                          \
    switch (tpr) {                                                    \
        case 1: launch(KERNEL<1>, GRID(1), s, __VA_ARGS__); break;    \
        case 2: launch(KERNEL<2>, GRID(2), s, __VA_ARGS__); break;    \
        case 4: launch(KERNEL<4>, GRID(4), s, __VA_ARGS__); break;    \
        case 8: launch(KERNEL<8>, GRID(8), s, __VA_ARGS__); break;    \
        case 16: launch(KERNEL<16>, GRID(16), s, __VA_ARGS__); break; \
        default: launch(KERNEL<32>, GRID(32), s, __VA_ARGS__); break; \
    }

void launch_op(const Op &op, std::vector<DevLevel> &lv, const Reduce &red, cudaStream_t s, const Op *start) {
    (void)red;
    DevLevel &L = lv[op.level];
    // a restriction followed by the row-local start of the coarse level's first visit
    double *xs = nullptr;
    const double *ids = nullptr;
    int c1 = 0;
    if (start) {
        const DevLevel &Cs = lv[start->level];
        xs = Cs.x;
        if (start->kind == OP_GS_FIRST) { c1 = (int)Cs.cptr[1]; ids = Cs.idiag; }
    }
    const int n = (int)L.n;
    switch (op.kind) {
        case OP_GS_FIRST:
            launch(k_gs_first, blocks(n), s, n, (int)L.cptr[1], (const double *)L.idiag, (const double *)L.b, L.x);
            break;
        case OP_ZERO:
            launch(k_zero, blocks(n), s, n, L.x);
            break;
        case OP_GS: {
            const int r0 = (int)L.cptr[op.colour], r1 = (int)L.cptr[op.colour + 1];
            const int64_t rows = r1 - r0;
            if (rows <= 0) break;
            if (L.gs_tpr == 0) {
                const int s0 = r0 / 32, s1 = (r1 + 31) / 32;
                launch_bs(k_gs_sell, (unsigned)((32 * (s1 - s0) + 63) / 64), 64, s, r0, r1, s0,
                          (const int32_t *)L.sl_ptr, (const int32_t *)L.sl_col, (const double *)L.sl_val,
                          (const double *)L.idiag, (const double *)L.b, L.x);
                break;
            }
            const int nl = L.nlong ? (int)(L.lptr[op.colour + 1] - L.lptr[op.colour]) : 0;
#define GRID_GS(T) (unsigned)nl + blocks((rows - nl) * (T))
            TPR_DISPATCH(L.gs_tpr, k_gs, GRID_GS, r0, r1, nl, (const int32_t *)L.rp, (const int32_t *)L.ci,
                         (const double *)L.val, (const double *)L.idiag, (const double *)L.b, L.x);
#undef GRID_GS
            break;
        }
        case OP_RESID: {
            if (L.rs_tpr == 0) {
                launch(k_resid_sell, blocks(n), s, n, (const int32_t *)L.sl_ptr, (const int32_t *)L.sl_col,
                       (const double *)L.sl_val, (const double *)L.diag, (const double *)L.x,
                       (const double *)L.b, L.r);
                break;
            }
#define GRID_R(T) (unsigned)L.nlong + blocks((int64_t)n * (T))
            TPR_DISPATCH(L.rs_tpr, k_resid, GRID_R, n, (const int32_t *)L.rp, (const int32_t *)L.ci,
                         (const double *)L.val, (const double *)L.diag, (const double *)L.x,
                         (const double *)L.b, L.r, (const int32_t *)L.lrows, (int)L.nlong);
#undef GRID_R
            break;
        }
        case OP_RESTRICT: {
            DevLevel &Cl = lv[op.level + 1];
            const int nc = (int)L.nc;
#define GRID_P(T) blocks((int64_t)nc * (T))
            TPR_DISPATCH(L.pt_tpr, k_restrict, GRID_P, nc, (const int32_t *)L.pt_ptr, (const int32_t *)L.pt_row,
                         (const double *)L.pt_w, (const double *)L.r, Cl.b, xs, c1, ids);
#undef GRID_P
            break;
        }
        case OP_PROLONG:
            launch(k_prolong, blocks(n), s, n, (const int32_t *)L.agg, (const int32_t *)L.agg2,
                   (const double *)L.wt, (const double *)lv[op.level + 1].x, L.x);
            break;
        case OP_ELIM_RESTRICT:
            launch(k_elim_restrict, blocks(L.nc), s, (int)L.nc, (const int32_t *)L.pft_ptr,
                   (const int32_t *)L.pft_f, (const double *)L.pft_val, (const double *)L.b,
                   lv[op.level + 1].b, xs, c1, ids);
            break;
        case OP_ELIM_INTERP:
            if (L.nF > 0)
                launch(k_elim_interp, blocks(L.nF), s, (int)L.nc, (int)L.nF, (const int32_t *)L.pf_col,
                       (const double *)L.pf_val, (const double *)L.dF, (const double *)L.b, L.x);
            break;
        case OP_COARSE:
            launch(k_coarse, red_blocks((int64_t)n * 32), s, n, (const double *)L.pinv, (const double *)L.b, L.x);
            break;
        case OP_CHEB: {
            // colour: step index within the polynomial, + 256 when the step reads t
            const int k = op.colour & 255;
            const bool from_t = op.colour >= 256;
            const double *xin = from_t ? L.t : L.x;
            double *xout = from_t ? L.x : L.t;
            const int tpr = L.gs_tpr > 0 ? L.gs_tpr : L.tpr;
#define GRID_C(T) (unsigned)L.nlong + blocks((int64_t)n * (T))
            TPR_DISPATCH(tpr, k_cheb, GRID_C, n, (const int32_t *)L.rp, (const int32_t *)L.ci, (const double *)L.val,
                         (const double *)L.diag, (const double *)L.idiag, (const double *)L.b, xin, xout, L.d,
                         L.cheb_c1[k], L.cheb_c2[k], (k == 0 ? 1 : 0) | (k == L.cheb_m - 1 ? 2 : 0),
                         (const int32_t *)L.lrows, (int)L.nlong);
#undef GRID_C
            break;
        }
        case OP_CHEB_COPY:
            launch(k_copy, blocks(n), s, n, (const double *)L.t, L.x);
            break;
        case OP_CHEB_FIRST:
            launch(k_cheb_first, blocks(n), s, n, (const double *)L.idiag, (const double *)L.b, L.cheb_c2[0],
                   op.colour ? L.t : L.x, L.cheb_m > 1 ? L.d : (double *)nullptr);
            break;
    }
}

void launch_gather(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t s) {
    launch(k_gather, blocks(n), s, (int)n, perm, src, dst);
}

void launch_scatter(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t s) {
    launch(k_scatter, blocks(n), s, (int)n, perm, src, dst);
}

void launch_sum(int64_t n, const double *v, const Reduce &red, cudaStream_t s) {
    launch(k_sum, red_blocks(n), s, (int)n, v, red);
}

void launch_sub_mean(int64_t n, double *v, const Reduce &red, cudaStream_t s) {
    launch(k_sub_mean, blocks(n), s, (int)n, v, red);
}

void launch_init_b(int64_t n, double *r, double *bkeep, double *x, double *p, double *zold,
                   const Reduce &red, cudaStream_t s) {
    launch(k_init_b, red_blocks(n), s, (int)n, r, bkeep, x, p, zold, red);
}

void launch_spmv_dot(const DevLevel &L, const double *p, double *q, const Reduce &red, cudaStream_t s) {
    const int n = (int)L.n;
    if (L.rs_tpr == 0) {
        launch(k_spmv_dot_sell, red_blocks(n), s, n, (const int32_t *)L.sl_ptr, (const int32_t *)L.sl_col,
               (const double *)L.sl_val, (const double *)L.diag, p, q, red);
        return;
    }
#define GRID_S(T) red_blocks((int64_t)n * (T))
    TPR_DISPATCH(L.rs_tpr, k_spmv_dot, GRID_S, n, (const int32_t *)L.rp, (const int32_t *)L.ci,
                 (const double *)L.val, (const double *)L.diag, p, q, red, (const int32_t *)L.lrows,
                 (int)L.nlong);
#undef GRID_S
}

void launch_update_xr(int64_t n, double *x, double *r, const double *p, const double *q,
                      const Reduce &red, cudaStream_t s) {
    launch(k_update_xr, red_blocks(n), s, (int)n, x, r, p, q, red);
}

void launch_proj_dots(int64_t n, double *z, const double *zold, const double *r, const Reduce &red,
                      cudaStream_t s) {
    launch(k_proj_dots, red_blocks(n), s, (int)n, z, zold, r, red);
}

void launch_update_p(int64_t n, const double *z, double *p, double *zold, const Reduce &red,
                     cudaStream_t s) {
    launch(k_update_p, blocks(n), s, (int)n, z, p, zold, red);
}

void launch_true_resid(const DevLevel &L, const double *x, const double *b, const Reduce &red,
                       cudaStream_t s) {
    const int n = (int)L.n;
    if (L.rs_tpr == 0) {
        launch(k_true_resid_sell, red_blocks(n), s, n, (const int32_t *)L.sl_ptr, (const int32_t *)L.sl_col,
               (const double *)L.sl_val, (const double *)L.diag, x, b, red);
        return;
    }
#define GRID_T(T) red_blocks((int64_t)n * (T))
    TPR_DISPATCH(L.rs_tpr, k_true_resid, GRID_T, n, (const int32_t *)L.rp, (const int32_t *)L.ci,
                 (const double *)L.val, (const double *)L.diag, x, b, red, (const int32_t *)L.lrows,
                 (int)L.nlong);
#undef GRID_T
}

}  // namespace lamg
