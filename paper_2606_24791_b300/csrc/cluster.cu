// Cluster sub-cycle kernel: every step of one visit of a small level, and of all the levels
// below it (the recursion of Section 2 with its gamma visits, elimination transfers of Eq. 2
// and the dense coarsest solve), in one launch of a single thread-block cluster.
//
// On the coarse levels a cycle step moves kilobytes, so run as separate kernels each step
// costs a launch and a chain of dependent loads whatever its size. Here the steps are
// separated by the cluster's hardware barrier (barrier.cluster with release/acquire
// semantics) instead of kernel boundaries: up to 16 CTAs of 512 threads, one row per lane
// group, walk the step list held in shared memory.
//
// Results are bit-identical to the per-step kernels: every row, aggregate and dense row is
// summed by the same number of lanes in the same order, with the same shuffle tree.
// Vectors written during the launch (iterates, right-hand sides, residuals) are read through
// L2 (ld.global.cg), so no CTA reads a stale line from its own L1 after another CTA wrote it.
// The barrier is a hardware barrier reached by every thread the same number of times (the
// step loop is uniform), so there is no software spin-wait to bound.
#include <cuda_runtime.h>

#include "device.h"
#include "kernels_common.cuh"

namespace lamg {

constexpr int CBS = 512;

__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cl_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

struct CPos {
    int tid, nthreads, lane, warp, nwarps;
};

// Read-only operands of a thread's first row of the next step, loaded between the barrier's
// arrive and wait (software pipelining: the loads overlap the barrier; only the gathers of
// vectors written by earlier steps are left after it). CSR lane groups: the lane's first entry
// e0, the row end e1 and the entries e0, e0 + TPR. Sliced ELLPACK: e0 = the lane's entry 0,
// e1 = the slice width, the entries e0, e0 + 32. d = reciprocal diagonal (sweep) or diagonal
// (residual).
struct CPre {
    int e0, e1, c0, c1, sub;
    double v0, v1, d;
};

__device__ __forceinline__ CPre cpre_empty() {
    CPre q;
    q.e0 = q.e1 = q.sub = 0;
    q.c0 = q.c1 = -1;
    q.v0 = q.v1 = 0.0;
    q.d = 1.0;
    return q;
}

template <int TPR>
__device__ __forceinline__ CPre cpre_csr(bool ok, int row, int sub, const int32_t *__restrict__ rp,
                                         const int32_t *__restrict__ ci, const double *__restrict__ val,
                                         const double *__restrict__ dg) {
    CPre q = cpre_empty();
    if (!ok) return q;
    q.e0 = __ldg(&rp[row]) + sub;
    q.e1 = __ldg(&rp[row + 1]);
    if (q.e0 < q.e1) { q.c0 = __ldg(&ci[q.e0]); q.v0 = __ldg(&val[q.e0]); }
    if (q.e0 + TPR < q.e1) { q.c1 = __ldg(&ci[q.e0 + TPR]); q.v1 = __ldg(&val[q.e0 + TPR]); }
    if (dg) q.d = __ldg(&dg[row]);
    return q;
}

// Sliced ELLPACK in four-entry blocks (sell_col_at / sell_val_at): e0 holds the slice base,
// e1 the slice width, sub the lane in the slice; the first two entries come with the prefetch.
__device__ __forceinline__ CPre cpre_sell(bool ok, int row, const PLevel &L, const double *__restrict__ dg) {
    CPre q = cpre_empty();
    if (!ok) return q;
    const int sl = row >> 5;
    const int a = __ldg(&L.sl_ptr[sl]);
    q.e0 = a;
    q.e1 = (__ldg(&L.sl_ptr[sl + 1]) - a) >> 5;
    q.sub = row & 31;
    if (q.e1 > 0) {
        const int2 c = __ldg(reinterpret_cast<const int2 *>(L.sl_col + a + 4 * q.sub));
        const double2 v = __ldg(reinterpret_cast<const double2 *>(L.sl_val + a + 2 * q.sub));
        q.c0 = c.x; q.v0 = v.x;
        q.c1 = c.y; q.v1 = v.y;
    }
    q.d = __ldg(&dg[row]);
    return q;
}

// Sum over a CSR row by TPR lanes (entries e0, e0 + TPR, ...), x read through L2; the first
// two entries of the lane come from the prefetch.
template <int TPR>
__device__ __forceinline__ double cl_row_pre(const CPre &q, const int32_t *__restrict__ ci,
                                             const double *__restrict__ val, const double *x) {
    double s = 0.0;
    if (q.c0 >= 0) s += q.v0 * __ldcg(&x[q.c0]);
    if (q.c1 >= 0) s += q.v1 * __ldcg(&x[q.c1]);
    for (int e = q.e0 + 2 * TPR; e < q.e1; e += TPR) s += __ldg(&val[e]) * __ldcg(&x[__ldg(&ci[e])]);
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Sliced-ELLPACK row sum, entries in order (as the per-step kernels sum them).
__device__ __forceinline__ double cl_sell_pre(const CPre &q, const PLevel &L, const double *x) {
    double acc = 0.0;
    if (q.c0 >= 0) acc += q.v0 * __ldcg(&x[q.c0]);
    if (q.c1 >= 0) acc += q.v1 * __ldcg(&x[q.c1]);
    for (int j = 2; j < q.e1; j++)
        acc += __ldg(&L.sl_val[sell_val_at(q.e0, q.sub, j)]) * __ldcg(&x[__ldg(&L.sl_col[sell_col_at(q.e0, q.sub, j)])]);
    return acc;
}

// One colour class of Gauss-Seidel: x_u = (b_u - sum_v A_uv x_v) / A_uu, u in [r0, r1).
// Round 0 of a thread uses the prefetched operands.
template <int TPR>
__device__ __forceinline__ CPre cl_gs_pre(const PLevel &L, int r0, int r1, const CPos &p) {
    const int row = r0 + p.tid / TPR;
    return cpre_csr<TPR>(row < r1, row, p.tid % TPR, L.rp, L.ci, L.val, L.idiag);
}

template <int TPR>
__device__ __forceinline__ void cl_gs(const PLevel &L, int r0, int r1, const CPos &p, const CPre &q0) {
    const int groups = p.nthreads / TPR, sub = p.tid % TPR;
    const int rounds = (r1 - r0 + groups - 1) / groups;
    int row = r0 + p.tid / TPR;
    for (int it = 0; it < rounds; it++, row += groups) {
        const bool ok = row < r1;
        const CPre q = it == 0 ? q0 : cpre_csr<TPR>(ok, row, sub, L.rp, L.ci, L.val, L.idiag);
        const double s = cl_row_pre<TPR>(q, L.ci, L.val, L.x);
        if (ok && sub == 0) L.x[row] = (__ldcg(&L.b[row]) - s) * q.d;
    }
}

__device__ __forceinline__ CPre cl_gs_sell_pre(const PLevel &L, int r0, int r1, const CPos &p) {
    const int row = 32 * ((r0 >> 5) + p.warp) + p.lane;
    return cpre_sell(row >= r0 && row < r1, row, L, L.idiag);
}

__device__ __forceinline__ void cl_gs_sell(const PLevel &L, int r0, int r1, const CPos &p, const CPre &q0) {
    const int s0 = r0 >> 5, s1 = (r1 + 31) >> 5;
    int it = 0;
    for (int sl = s0 + p.warp; sl < s1; sl += p.nwarps, it++) {
        const int row = 32 * sl + p.lane;
        if (row < r0 || row >= r1) continue;
        const CPre q = it == 0 ? q0 : cpre_sell(true, row, L, L.idiag);
        const double s = cl_sell_pre(q, L, L.x);
        L.x[row] = (__ldcg(&L.b[row]) - s) * q.d;
    }
}

__device__ __forceinline__ CPre cl_resid_sell_pre(const PLevel &L, const CPos &p) {
    const int row = 32 * p.warp + p.lane;
    return cpre_sell(row < L.n, row, L, L.diag);
}

__device__ __forceinline__ void cl_resid_sell(const PLevel &L, const CPos &p, const CPre &q0) {
    const int ns = (L.n + 31) >> 5;
    int it = 0;
    for (int sl = p.warp; sl < ns; sl += p.nwarps, it++) {
        const int row = 32 * sl + p.lane;
        if (row >= L.n) continue;
        const CPre q = it == 0 ? q0 : cpre_sell(true, row, L, L.diag);
        const double s = cl_sell_pre(q, L, L.x);
        L.r[row] = __ldcg(&L.b[row]) - (q.d * __ldcg(&L.x[row]) + s);
    }
}

// r = b - A x
template <int TPR>
__device__ __forceinline__ CPre cl_resid_pre(const PLevel &L, const CPos &p) {
    const int row = p.tid / TPR;
    return cpre_csr<TPR>(row < L.n, row, p.tid % TPR, L.rp, L.ci, L.val, L.diag);
}

template <int TPR>
__device__ __forceinline__ void cl_resid(const PLevel &L, const CPos &p, const CPre &q0) {
    const int groups = p.nthreads / TPR, sub = p.tid % TPR;
    const int rounds = (L.n + groups - 1) / groups;
    int row = p.tid / TPR;
    for (int it = 0; it < rounds; it++, row += groups) {
        const bool ok = row < L.n;
        const CPre q = it == 0 ? q0 : cpre_csr<TPR>(ok, row, sub, L.rp, L.ci, L.val, L.diag);
        const double s = cl_row_pre<TPR>(q, L.ci, L.val, L.x);
        if (ok && sub == 0) L.r[row] = __ldcg(&L.b[row]) - (q.d * __ldcg(&L.x[row]) + s);
    }
}

// b^c = P^T r: one P^T row (aggregate) per TPR lanes.
template <int TPR>
__device__ __forceinline__ CPre cl_restrict_pre(const PLevel &L, const CPos &p) {
    const int a = p.tid / TPR;
    return cpre_csr<TPR>(a < L.nc, a, p.tid % TPR, L.pt_ptr, L.pt_row, L.pt_w, nullptr);
}

template <int TPR>
__device__ __forceinline__ void cl_restrict(const PLevel &L, double *bc, const CPos &p, const CPre &q0) {
    const int groups = p.nthreads / TPR, sub = p.tid % TPR;
    const int rounds = (L.nc + groups - 1) / groups;
    int a = p.tid / TPR;
    for (int it = 0; it < rounds; it++, a += groups) {
        const bool ok = a < L.nc;
        const CPre q = it == 0 ? q0 : cpre_csr<TPR>(ok, a, sub, L.pt_ptr, L.pt_row, L.pt_w, nullptr);
        const double s = cl_row_pre<TPR>(q, L.pt_row, L.pt_w, L.r);
        if (ok && sub == 0) bc[a] = s;
    }
}

#define CL_TPR(tpr, FN, ...)                 \
    switch (tpr) {                           \
        case 1: FN<1>(__VA_ARGS__); break;   \
        case 2: FN<2>(__VA_ARGS__); break;   \
        case 4: FN<4>(__VA_ARGS__); break;   \
        case 8: FN<8>(__VA_ARGS__); break;   \
        case 16: FN<16>(__VA_ARGS__); break; \
        default: FN<32>(__VA_ARGS__); break; \
    }

#define CL_TPR_RET(tpr, OUT, FN, ...)              \
    switch (tpr) {                                 \
        case 1: OUT = FN<1>(__VA_ARGS__); break;   \
        case 2: OUT = FN<2>(__VA_ARGS__); break;   \
        case 4: OUT = FN<4>(__VA_ARGS__); break;   \
        case 8: OUT = FN<8>(__VA_ARGS__); break;   \
        case 16: OUT = FN<16>(__VA_ARGS__); break; \
        default: OUT = FN<32>(__VA_ARGS__); break; \
    }

// Prefetch of a step's read-only row operands (round 0 of this thread); empty for the steps
// without a row structure.
__device__ __forceinline__ CPre cl_prefetch(const Op &op, const PLevel *lv, const int32_t *cptr_all, const CPos &p) {
    const PLevel &L = lv[op.level];
    const int32_t *cptr = cptr_all + L.cptr_off;
    CPre q = cpre_empty();
    switch (op.kind) {
        case OP_GS:
            if (L.gs_tpr == 0) q = cl_gs_sell_pre(L, cptr[op.colour], cptr[op.colour + 1], p);
            else CL_TPR_RET(L.gs_tpr, q, cl_gs_pre, L, cptr[op.colour], cptr[op.colour + 1], p);
            break;
        case OP_RESID:
            if (L.rs_tpr == 0) q = cl_resid_sell_pre(L, p);
            else CL_TPR_RET(L.rs_tpr, q, cl_resid_pre, L, p);
            break;
        case OP_RESTRICT:
            CL_TPR_RET(L.pt_tpr, q, cl_restrict_pre, L, p);
            break;
        default:
            break;
    }
    return q;
}

__device__ __forceinline__ void cl_op(const Op &op, const PLevel *lv, const int32_t *cptr_all, const CPos &p,
                                      const CPre &q) {
    const PLevel &L = lv[op.level];
    const int32_t *cptr = cptr_all + L.cptr_off;
    switch (op.kind) {
        case OP_GS_FIRST: {
            const int c1 = cptr[1];
            for (int i = p.tid; i < L.n; i += p.nthreads)
                L.x[i] = i < c1 ? __ldcg(&L.b[i]) * __ldg(&L.idiag[i]) : 0.0;
            break;
        }
        case OP_ZERO:
            for (int i = p.tid; i < L.n; i += p.nthreads) L.x[i] = 0.0;
            break;
        case OP_GS:
            if (L.gs_tpr == 0) cl_gs_sell(L, cptr[op.colour], cptr[op.colour + 1], p, q);
            else CL_TPR(L.gs_tpr, cl_gs, L, cptr[op.colour], cptr[op.colour + 1], p, q);
            break;
        case OP_RESID:
            if (L.rs_tpr == 0) cl_resid_sell(L, p, q);
            else CL_TPR(L.rs_tpr, cl_resid, L, p, q);
            break;
        case OP_RESTRICT:
            CL_TPR(L.pt_tpr, cl_restrict, L, lv[op.level + 1].b, p, q);
            break;
        case OP_PROLONG: {
            const double *xc = lv[op.level + 1].x;
            for (int u = p.tid; u < L.n; u += p.nthreads) {
                const int a = __ldg(&L.agg[u]), bb = __ldg(&L.agg2[u]);
                double s;
                if (bb < 0) {
                    s = __ldcg(&xc[a]);
                } else {
                    const double w = __ldg(&L.wt[u]);
                    s = (1.0 - w) * __ldcg(&xc[bb]);
                    if (w != 0.0) s = w * __ldcg(&xc[a]) + s;
                }
                L.x[u] = __ldcg(&L.x[u]) + s;
            }
            break;
        }
        case OP_ELIM_RESTRICT: {
            double *bc = lv[op.level + 1].b;
            const double *bF = L.b + L.nc;
            for (int i = p.tid; i < L.nc; i += p.nthreads) {
                const int e0 = __ldg(&L.pft_ptr[i]), e1 = __ldg(&L.pft_ptr[i + 1]);
                double s = __ldcg(&L.b[i]);
                for (int e = e0; e < e1; e++) s += __ldg(&L.pft_val[e]) * __ldcg(&bF[__ldg(&L.pft_f[e])]);
                bc[i] = s;
            }
            break;
        }
        case OP_ELIM_INTERP:
            for (int t = p.tid; t < L.nF; t += p.nthreads) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int c = __ldg(&L.pf_col[4 * t + j]);
                    if (c >= 0) s += __ldg(&L.pf_val[4 * t + j]) * __ldcg(&L.x[c]);
                }
                L.x[L.nc + t] = s + __ldcg(&L.b[L.nc + t]) / __ldg(&L.dF[t]);
            }
            break;
        case OP_COARSE:
            // same summation order as the per-step kernel: four partial sums per lane over the
            // columns lane, lane + 32, lane + 64, lane + 96, then every 128th, added as
            // (s0 + s1) + (s2 + s3), then the warp's shuffle tree
            for (int i = p.warp; i < L.n; i += p.nwarps) {
                const double *row = L.pinv + (size_t)i * L.n;
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                int j = p.lane;
                for (; j + 96 < L.n; j += 128) {
                    const double a0 = __ldg(&row[j]), a1 = __ldg(&row[j + 32]);
                    const double a2 = __ldg(&row[j + 64]), a3 = __ldg(&row[j + 96]);
                    const double v0 = __ldcg(&L.b[j]), v1 = __ldcg(&L.b[j + 32]);
                    const double v2 = __ldcg(&L.b[j + 64]), v3 = __ldcg(&L.b[j + 96]);
                    s0 += a0 * v0;
                    s1 += a1 * v1;
                    s2 += a2 * v2;
                    s3 += a3 * v3;
                }
                for (; j < L.n; j += 32) s0 += __ldg(&row[j]) * __ldcg(&L.b[j]);
                double s = (s0 + s1) + (s2 + s3);
                s = warp_sum(s);
                if (p.lane == 0) L.x[i] = s;
            }
            break;
    }
}


// prof (optional): CTA 0 records %globaltimer before step i (prof[2i]) and after its barrier
// (prof[2i + 1]).
__device__ __forceinline__ unsigned long long cl_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The step loop: step i, barrier; the operands of step i + 1 are prefetched between the
// barrier's arrive and wait (after the arrive, so that its release does not wait for them).
__device__ __forceinline__ void cl_steps(const Op *ops, int nops, const PLevel *lv, const int32_t *cptr,
                                         const CPos &p, CPre q, unsigned long long *prof) {
    for (int i = 0; i < nops; i++) {
        const Op op = ops[i];
        if (prof && p.tid == 0) prof[2 * i] = cl_ns();
        cl_op(op, lv, cptr, p, q);
        cl_arrive();
        if (i + 1 < nops) q = cl_prefetch(ops[i + 1], lv, cptr, p);
        cl_wait();
        if (prof && p.tid == 0) prof[2 * i + 1] = cl_ns();
    }
}

// Level tables of one hierarchy into this CTA's shared memory; returns the step list (shared
// memory when it has at most CL_OPS_SMEM steps, else global).
__device__ __forceinline__ const Op *cl_load_tables(unsigned char *smem, const PLevel *lv_g, int nlev,
                                                    const int32_t *cptr_g, int ncptr, const Op *ops_g,
                                                    int nops, PLevel **s_lv_out, int32_t **s_cptr_out) {
    PLevel *s_lv = reinterpret_cast<PLevel *>(smem);
    int32_t *s_cptr = reinterpret_cast<int32_t *>(s_lv + nlev);
    Op *s_ops = reinterpret_cast<Op *>(s_cptr + ((ncptr + 3) & ~3));
    const bool ops_in_smem = nops <= CL_OPS_SMEM;
    const long long *src = reinterpret_cast<const long long *>(lv_g);
    long long *dst = reinterpret_cast<long long *>(s_lv);
    const int nw = (int)(nlev * sizeof(PLevel) / sizeof(long long));
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < ncptr; i += blockDim.x) s_cptr[i] = cptr_g[i];
    if (ops_in_smem)
        for (int i = threadIdx.x; i < nops; i += blockDim.x) s_ops[i] = ops_g[i];
    __syncthreads();
    *s_lv_out = s_lv;
    *s_cptr_out = s_cptr;
    return ops_in_smem ? s_ops : ops_g;
}

__device__ __forceinline__ CPos cl_pos() {
    // warps are numbered round-robin over the CTAs (warp w of CTA c is cluster warp
    // w * ncta + c), so consecutive rows of a small step spread over all of the cluster's SMs
    // and their FP64 units instead of filling the first CTA
    CPos p;
    p.lane = threadIdx.x & 31;
    p.warp = (int)((threadIdx.x >> 5) * cl_size() + cl_rank());
    p.tid = p.warp * 32 + p.lane;
    p.nthreads = (int)(cl_size() * blockDim.x);
    p.nwarps = p.nthreads >> 5;
    return p;
}

// Steps ops[0 .. nops) on the levels of lv (device tables), run by one cluster.
__global__ void __launch_bounds__(CBS, 1) k_cluster(const PLevel *__restrict__ lv_g, int nlev,
                                                    const int32_t *__restrict__ cptr_g, int ncptr,
                                                    const Op *__restrict__ ops_g, int nops,
                                                    unsigned long long *prof) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    PLevel *s_lv;
    int32_t *s_cptr;
    const Op *ops = cl_load_tables(smem, lv_g, nlev, cptr_g, ncptr, ops_g, nops, &s_lv, &s_cptr);
    const CPos p = cl_pos();
    CPre q = nops > 0 ? cl_prefetch(ops[0], s_lv, s_cptr, p) : cpre_empty();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    cl_steps(ops, nops, s_lv, s_cptr, p, q, prof);
}

// ------------------------------------------------------------ whole solves, one cluster each

// Deterministic all-reduce of NV doubles over the cluster: a fixed-order block sum per CTA,
// the CTA totals through a global partial buffer (alternating halves), then every thread adds
// them in CTA-rank order, so every thread of the cluster holds the same bits.
template <int NV>
__device__ __forceinline__ void cl_allreduce(double (&v)[NV], double *part, unsigned &phase) {
    block_sum<NV>(v);
    double *buf = part + (size_t)(phase & 1u) * (RED_NV * 16);
    phase++;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) __stcg(&buf[k * 16 + cl_rank()], v[k]);
    }
    cl_arrive();
    cl_wait();
    const int nc = (int)cl_size();
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = 0.0;
        for (int c = 0; c < nc; c++) s += __ldcg(&buf[k * 16 + c]);
        v[k] = s;
    }
}

// q = A p and the partial p . q of this thread's rows (level-0 form, lane groups or sliced).
template <int TPR>
__device__ __forceinline__ double cl_spmv_part(const PLevel &F, const double *pv, double *qv, const CPos &p) {
    const int groups = p.nthreads / TPR, sub = p.tid % TPR;
    const int rounds = (F.n + groups - 1) / groups;
    double acc = 0.0;
    int row = p.tid / TPR;
    for (int it = 0; it < rounds; it++, row += groups) {
        const bool ok = row < F.n;
        const CPre q = cpre_csr<TPR>(ok, row, sub, F.rp, F.ci, F.val, F.diag);
        const double s = cl_row_pre<TPR>(q, F.ci, F.val, pv);
        if (ok && sub == 0) {
            const double pi = __ldcg(&pv[row]);
            const double qi = q.d * pi + s;
            __stcg(&qv[row], qi);
            acc += pi * qi;
        }
    }
    return acc;
}

__device__ __forceinline__ double cl_spmv_part_sell(const PLevel &F, const double *pv, double *qv, const CPos &p) {
    const int ns = (F.n + 31) >> 5;
    double acc = 0.0;
    for (int sl = p.warp; sl < ns; sl += p.nwarps) {
        const int row = 32 * sl + p.lane;
        if (row >= F.n) continue;
        const CPre q = cpre_sell(true, row, F, F.diag);
        const double s = cl_sell_pre(q, F, pv);
        const double pi = __ldcg(&pv[row]);
        const double qi = q.d * pi + s;
        __stcg(&qv[row], qi);
        acc += pi * qi;
    }
    return acc;
}

// ||b - A x||^2 partial of this thread's rows.
template <int TPR>
__device__ __forceinline__ double cl_rr_part(const PLevel &F, const double *x, const double *b, const CPos &p) {
    const int groups = p.nthreads / TPR, sub = p.tid % TPR;
    const int rounds = (F.n + groups - 1) / groups;
    double acc = 0.0;
    int row = p.tid / TPR;
    for (int it = 0; it < rounds; it++, row += groups) {
        const bool ok = row < F.n;
        const CPre q = cpre_csr<TPR>(ok, row, sub, F.rp, F.ci, F.val, F.diag);
        const double s = cl_row_pre<TPR>(q, F.ci, F.val, x);
        if (ok && sub == 0) {
            const double ri = __ldcg(&b[row]) - (q.d * __ldcg(&x[row]) + s);
            acc += ri * ri;
        }
    }
    return acc;
}

__device__ __forceinline__ double cl_rr_part_sell(const PLevel &F, const double *x, const double *b, const CPos &p) {
    const int ns = (F.n + 31) >> 5;
    double acc = 0.0;
    for (int sl = p.warp; sl < ns; sl += p.nwarps) {
        const int row = 32 * sl + p.lane;
        if (row >= F.n) continue;
        const CPre q = cpre_sell(true, row, F, F.diag);
        const double s = cl_sell_pre(q, F, x);
        const double ri = __ldcg(&b[row]) - (q.d * __ldcg(&x[row]) + s);
        acc += ri * ri;
    }
    return acc;
}

// One cycle (the static step list), then the flexible-CG update of z = the level-0 iterate:
// z -= mean(z); beta = r.(z - zold) / rz; rz = r.z; p = z + beta p; zold = z.
__device__ __forceinline__ void cl_cycle_and_tail(const MGraph &G, const Op *ops, const PLevel *lv,
                                                  const int32_t *cptr, const CPos &p, unsigned &phase,
                                                  double &rz) {
    const int n = G.n0;
    CPre q = G.nops > 0 ? cl_prefetch(ops[0], lv, cptr, p) : cpre_empty();
    cl_steps(ops, G.nops, lv, cptr, p, q, nullptr);
    double *z = lv[0].x;
    double s1[1] = {0.0};
    for (int i = p.tid; i < n; i += p.nthreads) s1[0] += __ldcg(&z[i]);
    cl_allreduce<1>(s1, G.part, phase);
    const double mean = s1[0] / (double)n;
    double s2[2] = {0.0, 0.0};
    for (int i = p.tid; i < n; i += p.nthreads) {
        const double zi = __ldcg(&z[i]) - mean;
        __stcg(&z[i], zi);
        const double ri = __ldcg(&G.r[i]);
        s2[0] += ri * (zi - __ldcg(&G.zold[i]));
        s2[1] += ri * zi;
    }
    cl_allreduce<2>(s2, G.part, phase);
    const double beta = rz != 0.0 ? s2[0] / rz : 0.0;
    rz = s2[1];
    for (int i = p.tid; i < n; i += p.nthreads) {
        const double zi = __ldcg(&z[i]);
        __stcg(&G.p[i], zi + beta * __ldcg(&G.p[i]));
        __stcg(&G.zold[i], zi);
    }
    cl_arrive();
    cl_wait();
}

// Cluster c solves system c of gs[]: projection of b (Eq. 1), flexible CG preconditioned by
// the cycle of Section 2, stopping test on the recursive residual, true residual, scatter.
// The clusters share nothing and never wait for one another.
__global__ void __launch_bounds__(CBS, 1) k_cluster_solve(const MGraph *__restrict__ gs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const MGraph G = gs[blockIdx.x / cl_size()];
    PLevel *lv;
    int32_t *cptr;
    const Op *ops = cl_load_tables(smem, G.lv, G.nlev, G.cptr, G.ncptr, G.ops, G.nops, &lv, &cptr);
    const CPos p = cl_pos();
    const PLevel &F = lv[0];
    const int n = G.n0;
    unsigned phase = 0;

    double s[1] = {0.0};
    for (int i = p.tid; i < n; i += p.nthreads) {
        const double v = __ldg(&G.b_in[__ldg(&G.perm0[i])]);
        __stcg(&G.r[i], v);
        s[0] += v;
    }
    cl_allreduce<1>(s, G.part, phase);
    const double bmean = s[0] / (double)n;
    s[0] = 0.0;
    for (int i = p.tid; i < n; i += p.nthreads) {
        const double v = __ldcg(&G.r[i]) - bmean;
        __stcg(&G.r[i], v);
        __stcg(&G.bkeep[i], v);
        __stcg(&G.xs[i], 0.0);
        __stcg(&G.p[i], 0.0);
        __stcg(&G.zold[i], 0.0);
        s[0] += v * v;
    }
    cl_allreduce<1>(s, G.part, phase);
    const double bn2 = s[0];
    double rz = 1.0;
    cl_cycle_and_tail(G, ops, lv, cptr, p, phase, rz);
    int it = 0;
    double rr = 0.0;
    const bool lead = cl_rank() == 0 && threadIdx.x == 0;
    if (lead && G.hist) G.hist[0] = 1.0;
    while (it < G.maxit) {
        double pq[1];
        if (F.rs_tpr == 0) pq[0] = cl_spmv_part_sell(F, G.p, G.q, p);
        else CL_TPR_RET(F.rs_tpr, pq[0], cl_spmv_part, F, G.p, G.q, p);
        cl_allreduce<1>(pq, G.part, phase);
        const double alpha = pq[0] != 0.0 ? rz / pq[0] : 0.0;
        double r2[1] = {0.0};
        for (int i = p.tid; i < n; i += p.nthreads) {
            __stcg(&G.xs[i], __ldcg(&G.xs[i]) + alpha * __ldcg(&G.p[i]));
            const double ri = __ldcg(&G.r[i]) - alpha * __ldcg(&G.q[i]);
            __stcg(&G.r[i], ri);
            r2[0] += ri * ri;
        }
        cl_allreduce<1>(r2, G.part, phase);
        rr = r2[0];
        it++;
        const double rel = bn2 > 0.0 ? sqrt(rr / bn2) : 0.0;
        if (lead && G.hist) G.hist[it] = rel;
        if (!(rel > G.tol)) break;
        cl_cycle_and_tail(G, ops, lv, cptr, p, phase, rz);
    }
    double tr[1];
    if (F.rs_tpr == 0) tr[0] = cl_rr_part_sell(F, G.xs, G.bkeep, p);
    else CL_TPR_RET(F.rs_tpr, tr[0], cl_rr_part, F, G.xs, G.bkeep, p);
    cl_allreduce<1>(tr, G.part, phase);
    for (int i = p.tid; i < n; i += p.nthreads) G.phi_out[__ldg(&G.perm0[i])] = __ldcg(&G.xs[i]);
    if (lead) {
        G.out[MG_ITERS] = (double)it;
        G.out[MG_RR] = rr;
        G.out[MG_BN2] = bn2;
        G.out[MG_TRUE_RR] = tr[0];
        G.out[MG_BMEAN] = bmean;
    }
    // no CTA leaves while another may still read its partials
    cl_arrive();
    cl_wait();
}

cudaError_t launch_cluster_solve(const MGraph *g, int G, int cl, size_t smem, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_cluster_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)CL_SMEM_MAX);
        if (e != cudaSuccess) return e;
        cudaFuncSetAttribute(k_cluster_solve, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaGetLastError();
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(G * cl));
    cfg.blockDim = dim3(CBS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cluster_solve, g);
}

size_t cluster_smem(int nlev, int ncptr, int nops) {
    return (size_t)nlev * sizeof(PLevel) + (size_t)((ncptr + 3) & ~3) * sizeof(int32_t) +
           (size_t)(nops <= CL_OPS_SMEM ? nops : 0) * sizeof(Op);
}

// Largest cluster (16, 8 or 4 CTAs of CBS threads) of which one can be resident with smem
// bytes of dynamic shared memory per CTA; 0 if none. The kernel's dynamic shared-memory limit
// is a per-function setting shared by every hierarchy, so it is always set to CL_SMEM_MAX.
int cluster_dim(int device, size_t smem) {
    int ok = 0;
    if (smem > CL_SMEM_MAX) return 0;
    if (cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, device) != cudaSuccess || !ok) return 0;
    if (cudaFuncSetAttribute(k_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM_MAX) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaFuncSetAttribute(k_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int cl : {16, 8, 4}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(CBS);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_cluster, &cfg) == cudaSuccess && n >= 1) return cl;
        cudaGetLastError();
    }
    return 0;
}

void launch_cluster(const PLevel *lv, int nlev, const int32_t *cptr, int ncptr, const Op *ops, int nops,
                    int cl, bool pdl, cudaStream_t s, unsigned long long *prof) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(CBS);
    cfg.dynamicSmemBytes = cluster_smem(nlev, ncptr, nops);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, k_cluster, lv, nlev, cptr, ncptr, ops, nops, prof);
}

}  // namespace lamg
