// Persistent cooperative solve kernel: the whole flexible-CG solve (projection of b, every
// cycle of Section 2, the CG vector updates and the stopping test) in one launch.
//
// The cycle is a fixed list of dependent steps; run as separate kernels each step costs a
// launch plus one latency chain, which dominates on the small coarse levels. Here one CTA
// per SM stays resident for the whole solve and walks the same step list:
//  - steps on large levels are spread over the whole grid, with a grid-wide barrier after
//    each one;
//  - maximal runs of steps on small levels (at most tail_rows rows, and the coarsest level
//    when its dense matrix is small) run inside CTA 0 alone, separated by __syncthreads,
//    while the other CTAs wait at a single grid barrier after the run.
// The level table, the colour-class offsets and the step list are copied into shared memory
// at kernel start, so a step starts without a global-memory round trip.
//
// Each barrier wait is bounded: a CTA that waits longer than the solve's limit (2 s unless the
// caller sets lamg_solve_opts.wait_us; %globaltimer nanoseconds) marks the barrier as failed and
// every CTA returns at its next barrier; the host then reports LAMG_ERR_TIMEOUT.
//
// CG scalars (alpha, beta, r.z, ||r||) are replicated: every CTA adds the same per-block
// partials in the same order, so every CTA holds bit-identical scalars and takes the same
// stopping decision. Partials alternate between two buffers so that a CTA writing the next
// reduction never overwrites values another CTA is still reading.
//
// The residual-then-restriction pair of an aggregation level is fused: each coarse row
// recomputes the residual of the fine rows it restricts from (r is never stored).
#include <cuda_runtime.h>

#include <cstdio>

#include "device.h"
#include "kernels_common.cuh"

namespace lamg {

constexpr int PBS = 512;

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier (all CTAs co-resident by cooperative launch). Returns false on failure: this
// CTA waited longer than wait_ns, or another CTA's wait ran out.
__device__ __forceinline__ bool gsync(GridBar *bar, unsigned &gen, unsigned long long wait_ns) {
    __shared__ int fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        int f = 0;
        bool releaser = false;
        if (atom_add_acq_rel(&bar->count, 1u) == gridDim.x - 1) {
            bar->count = 0u;
            st_release(&bar->gen, gen + 1u);
            releaser = true;
        }
        if (!releaser) {
            const unsigned long long t0 = timer_ns();
            while (ld_relaxed(&bar->gen) == gen) {
                if (timer_ns() - t0 >= wait_ns) {
                    atomicExch(&bar->err, 1u);
                    f = 1;
                    break;
                }
            }
            __threadfence();  // acquire: pairs with the releasing store of the last arrival
        }
        if (ld_relaxed(&bar->err)) f = 1;
        fail = f;
        gen += 1u;
    }
    __syncthreads();
    return !fail;
}

// Replicated deterministic all-reduce of NV doubles over the grid (one barrier).
template <int NV>
__device__ __forceinline__ bool allreduce(double (&v)[NV], const PSolve &P, unsigned &gen, unsigned &ridx) {
    __shared__ double res[NV];
    block_sum<NV>(v);
    double *buf = P.partials + (size_t)(ridx & 1u) * RED_NV * gridDim.x;
    ridx++;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) buf[k * gridDim.x + blockIdx.x] = v[k];
    }
    if (!gsync(P.bar, gen, P.wait_ns)) return false;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&buf[k * gridDim.x + b]);
        v[k] = s;
    }
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) res[k] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = res[k];
    __syncthreads();
    return true;
}

// ------------------------------------------------------------------ work distribution

// Threads taking part in a step: the whole grid, or the calling CTA alone.
struct GridPos {
    int lane, warp, nwarps, tid, nthreads;
    __device__ explicit GridPos(bool whole_grid) {
        lane = threadIdx.x & 31;
        tid = whole_grid ? blockIdx.x * blockDim.x + threadIdx.x : threadIdx.x;
        nthreads = whole_grid ? gridDim.x * blockDim.x : blockDim.x;
        warp = tid >> 5;
        nwarps = nthreads >> 5;
    }
};

// Shared-memory copies of the level table, colour offsets, step list and segment ends.
struct Tables {
    const PLevel *lv;
    const int32_t *cptr;
    const Op *ops;
    const int32_t *tail_end;
};

// Gauss-Seidel on rows [r0, r1) of one colour class. Each lane group works on U rows at once
// (rows w, w + stride, ...) so that U independent load chains are in flight per thread.
template <int TPR>
__device__ __forceinline__ void p_gs(const PLevel &L, int r0, int r1, const GridPos &g) {
    constexpr int GPW = 32 / TPR;
    constexpr int U = 4;
    const int sub = g.lane % TPR;
    const int stride = g.nwarps * GPW;
    for (int w0 = r0 + g.warp * GPW; w0 < r1; w0 += U * stride) {
        int row[U], e0[U], e1[U];
        double s[U];
        int kmax = 0;
#pragma unroll
        for (int u = 0; u < U; u++) {
            row[u] = w0 + u * stride + g.lane / TPR;
            const bool ok = row[u] < r1;
            e0[u] = ok ? L.rp[row[u]] + sub : 0;
            e1[u] = ok ? L.rp[row[u] + 1] : 0;
            s[u] = 0.0;
            kmax = max(kmax, e1[u] - e0[u]);
        }
        for (int k = 0; k < kmax; k += TPR) {
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int e = e0[u] + k;
                if (e < e1[u]) s[u] += L.val[e] * L.x[L.ci[e]];
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
#pragma unroll
            for (int o = TPR / 2; o > 0; o >>= 1) s[u] += __shfl_xor_sync(0xffffffffu, s[u], o);
            if (row[u] < r1 && sub == 0) L.x[row[u]] = (L.b[row[u]] - s[u]) * L.idiag[row[u]];
        }
    }
}

// Fused residual + restriction: b_c[a] = sum_{(u,p) in P^T row a} p (b_u - (A x)_u).
template <int TPR>
__device__ __forceinline__ void p_restrict(const PLevel &L, double *bc, const GridPos &g) {
    constexpr int GPW = 32 / TPR;
    const int sub = g.lane % TPR;
    for (int w0 = g.warp * GPW; w0 < L.nc; w0 += g.nwarps * GPW) {
        const int a = w0 + g.lane / TPR;
        const bool ok = a < L.nc;
        const int t0 = ok ? L.pt_ptr[a] : 0, t1 = ok ? L.pt_ptr[a + 1] : 0;
        // all lanes of the warp loop to the warp's longest P^T row so shuffles stay converged
        int tmax = t1 - t0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        double acc = 0.0;
        for (int t = 0; t < tmax; t++) {
            const bool has = t0 + t < t1;
            const int u = has ? L.pt_row[t0 + t] : 0;
            const int e0 = has ? L.rp[u] + sub : 0, e1 = has ? L.rp[u + 1] : 0;
            const double s = row_sum<TPR>(e0, e1, L.ci, L.val, L.x);
            if (has) acc += L.pt_w[t0 + t] * (L.b[u] - (L.diag[u] * L.x[u] + s));
        }
        if (ok && sub == 0) bc[a] = acc;
    }
}

#define P_TPR(tpr, FN, ...)                  \
    switch (tpr) {                           \
        case 1: FN<1>(__VA_ARGS__); break;   \
        case 2: FN<2>(__VA_ARGS__); break;   \
        case 4: FN<4>(__VA_ARGS__); break;   \
        case 8: FN<8>(__VA_ARGS__); break;   \
        case 16: FN<16>(__VA_ARGS__); break; \
        default: FN<32>(__VA_ARGS__); break; \
    }

__device__ __forceinline__ void p_op(const Op &op, const Tables &T, const GridPos &g) {
    const PLevel &L = T.lv[op.level];
    const int32_t *cptr = T.cptr + L.cptr_off;
    switch (op.kind) {
        case OP_GS_FIRST: {
            const int c1 = cptr[1];
            for (int i = g.tid; i < L.n; i += g.nthreads) L.x[i] = i < c1 ? L.b[i] * L.idiag[i] : 0.0;
            break;
        }
        case OP_ZERO:
            for (int i = g.tid; i < L.n; i += g.nthreads) L.x[i] = 0.0;
            break;
        case OP_GS:
            P_TPR(L.tpr, p_gs, L, cptr[op.colour], cptr[op.colour + 1], g);
            break;
        case OP_RESID:  // fused into the restriction that follows
            break;
        case OP_RESTRICT:
            P_TPR(L.tpr, p_restrict, L, T.lv[op.level + 1].b, g);
            break;
        case OP_PROLONG: {
            const double *xc = T.lv[op.level + 1].x;
            for (int u = g.tid; u < L.n; u += g.nthreads) {
                const int bb = L.agg2[u];
                double s;
                if (bb < 0) {
                    s = xc[L.agg[u]];
                } else {
                    const double w = L.wt[u];
                    s = (1.0 - w) * xc[bb];
                    if (w != 0.0) s = w * xc[L.agg[u]] + s;
                }
                L.x[u] += s;
            }
            break;
        }
        case OP_ELIM_RESTRICT: {
            double *bc = T.lv[op.level + 1].b;
            const double *bF = L.b + L.nc;
            for (int i = g.tid; i < L.nc; i += g.nthreads) {
                double s = L.b[i];
                for (int e = L.pft_ptr[i]; e < L.pft_ptr[i + 1]; e++) s += L.pft_val[e] * bF[L.pft_f[e]];
                bc[i] = s;
            }
            break;
        }
        case OP_ELIM_INTERP:
            for (int t = g.tid; t < L.nF; t += g.nthreads) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int c = L.pf_col[4 * t + j];
                    if (c >= 0) s += L.pf_val[4 * t + j] * L.x[c];
                }
                L.x[L.nc + t] = s + L.b[L.nc + t] / L.dF[t];
            }
            break;
        case OP_COARSE:
            for (int i = g.warp; i < L.n; i += g.nwarps) {
                const double *row = L.pinv + (size_t)i * L.n;
                double s = 0.0;
                for (int j = g.lane; j < L.n; j += 32) s += row[j] * L.b[j];
                s = warp_sum(s);
                if (g.lane == 0) L.x[i] = s;
            }
            break;
    }
}

// One cycle: the static step list, grid steps separated by grid barriers, single-CTA
// segments run by CTA 0 and closed by one grid barrier.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool p_cycle(const PSolve &P, const Tables &T, unsigned &gen,
                                        unsigned long long *prof = nullptr) {
    const GridPos grid(true), local(false);
    int nrec = 0;
    if (prof && blockIdx.x == 0 && threadIdx.x == 0) { prof[0] = 0; prof[1] = global_ns(); }
    for (int i = 0; i < P.nops;) {
        const int te = T.tail_end[i];
        if (te >= 0) {
            if (blockIdx.x == 0) {
                for (int k = i; k < te; k++) {
                    const Op op = T.ops[k];
                    if (op.kind == OP_RESID) continue;
                    p_op(op, T, local);
                    __syncthreads();
                }
            }
            i = te;
        } else {
            const Op op = T.ops[i++];
            if (op.kind == OP_RESID) continue;
            p_op(op, T, grid);
        }
        if (!gsync(P.bar, gen, P.wait_ns)) return false;
        if (prof && blockIdx.x == 0 && threadIdx.x == 0) {
            nrec++;
            prof[2 * nrec] = (unsigned long long)i;   // steps up to (not including) op i are done
            prof[2 * nrec + 1] = global_ns();
            prof[0] = (unsigned long long)nrec;
        }
    }
    return true;
}

template <int TPR>
__device__ __forceinline__ double p_spmv_dot(const PLevel &L, const double *p, double *q, const GridPos &g) {
    constexpr int GPW = 32 / TPR;
    const int sub = g.lane % TPR;
    double pq = 0.0;
    for (int w0 = g.warp * GPW; w0 < L.n; w0 += g.nwarps * GPW) {
        const int row = w0 + g.lane / TPR;
        const bool ok = row < L.n;
        const int e0 = ok ? L.rp[row] + sub : 0, e1 = ok ? L.rp[row + 1] : 0;
        const double s = row_sum<TPR>(e0, e1, L.ci, L.val, p);
        if (ok && sub == 0) {
            const double qi = L.diag[row] * p[row] + s;
            q[row] = qi;
            pq += p[row] * qi;
        }
    }
    return pq;
}

template <int TPR>
__device__ __forceinline__ double p_true_rr(const PLevel &L, const double *x, const double *b, const GridPos &g) {
    constexpr int GPW = 32 / TPR;
    const int sub = g.lane % TPR;
    double acc = 0.0;
    for (int w0 = g.warp * GPW; w0 < L.n; w0 += g.nwarps * GPW) {
        const int row = w0 + g.lane / TPR;
        const bool ok = row < L.n;
        const int e0 = ok ? L.rp[row] + sub : 0, e1 = ok ? L.rp[row + 1] : 0;
        const double s = row_sum<TPR>(e0, e1, L.ci, L.val, x);
        if (ok && sub == 0) {
            const double ri = b[row] - (L.diag[row] * x[row] + s);
            acc += ri * ri;
        }
    }
    return acc;
}

#define P_TPR_RET(tpr, OUT, FN, ...)                \
    switch (tpr) {                                  \
        case 1: OUT = FN<1>(__VA_ARGS__); break;    \
        case 2: OUT = FN<2>(__VA_ARGS__); break;    \
        case 4: OUT = FN<4>(__VA_ARGS__); break;    \
        case 8: OUT = FN<8>(__VA_ARGS__); break;    \
        case 16: OUT = FN<16>(__VA_ARGS__); break;  \
        default: OUT = FN<32>(__VA_ARGS__); break;  \
    }

// z (= level-0 iterate) -= mean(z); beta = r.(z - zold) / rz; rz = r.z; p = z + beta p; zold = z.
__device__ __forceinline__ bool p_cg_tail(const PSolve &P, const Tables &T, unsigned &gen, unsigned &ridx,
                                          double &rz) {
    const GridPos g(true);
    const int n = P.n0;
    double *z = T.lv[0].x;
    double s1[1] = {0.0};
    for (int i = g.tid; i < n; i += g.nthreads) s1[0] += z[i];
    if (!allreduce<1>(s1, P, gen, ridx)) return false;
    const double mean = s1[0] / (double)n;
    double s2[2] = {0.0, 0.0};
    for (int i = g.tid; i < n; i += g.nthreads) {
        const double zi = z[i] - mean;
        z[i] = zi;
        s2[0] += P.r[i] * (zi - P.zold[i]);
        s2[1] += P.r[i] * zi;
    }
    if (!allreduce<2>(s2, P, gen, ridx)) return false;
    const double beta = rz != 0.0 ? s2[0] / rz : 0.0;
    rz = s2[1];
    for (int i = g.tid; i < n; i += g.nthreads) {
        const double zi = z[i];
        P.p[i] = zi + beta * P.p[i];
        P.zold[i] = zi;
    }
    return gsync(P.bar, gen, P.wait_ns);
}

// mode 0: full solve of L phi = b_in (natural order) into phi_out.
// mode 1: one preconditioner application z = M r (r = b_in, natural order), projected.
__global__ void __launch_bounds__(PBS, 2) k_persistent(const PSolve *__restrict__ Pg, int mode, int maxit,
                                                       double tol, const double *__restrict__ b_in,
                                                       double *phi_out, unsigned long long *prof,
                                                       unsigned long long wait_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PSolve sP;
    if (threadIdx.x == 0) {
        sP = *Pg;
        sP.wait_ns = wait_ns;
    }
    __syncthreads();
    const PSolve &P = sP;
    // tables into shared memory
    PLevel *s_lv = reinterpret_cast<PLevel *>(smem);
    Op *s_ops = reinterpret_cast<Op *>(s_lv + P.nlev);
    int32_t *s_tail = reinterpret_cast<int32_t *>(s_ops + P.nops);
    int32_t *s_cptr = s_tail + P.nops;
    {
        const long long *src = reinterpret_cast<const long long *>(P.lv);
        long long *dst = reinterpret_cast<long long *>(s_lv);
        const int nw = (int)(P.nlev * sizeof(PLevel) / sizeof(long long));
        for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
        for (int i = threadIdx.x; i < P.nops; i += blockDim.x) {
            s_ops[i] = P.ops[i];
            s_tail[i] = P.tail_end[i];
        }
        for (int i = threadIdx.x; i < P.ncptr; i += blockDim.x) s_cptr[i] = P.cptr_all[i];
    }
    __syncthreads();
    const Tables T{s_lv, s_cptr, s_ops, s_tail};

    const GridPos g(true);
    unsigned gen = ld_relaxed(&P.bar->gen);
    unsigned ridx = 0;
    const int n = P.n0;

    // b in device order, its mean
    double s[1] = {0.0};
    for (int i = g.tid; i < n; i += g.nthreads) {
        const double v = b_in[P.perm0[i]];
        P.r[i] = v;
        s[0] += v;
    }
    if (!allreduce<1>(s, P, gen, ridx)) return;
    const double bmean = s[0] / (double)n;

    if (mode == 1) {
        if (!p_cycle(P, T, gen, prof)) return;
        const double *z = T.lv[0].x;
        double t[1] = {0.0};
        for (int i = g.tid; i < n; i += g.nthreads) t[0] += z[i];
        if (!allreduce<1>(t, P, gen, ridx)) return;
        const double zm = t[0] / (double)n;
        for (int i = g.tid; i < n; i += g.nthreads) phi_out[P.perm0[i]] = z[i] - zm;
        return;
    }

    // projection of b (Eq. 1), ||b||^2, x = p = zold = 0
    s[0] = 0.0;
    for (int i = g.tid; i < n; i += g.nthreads) {
        const double v = P.r[i] - bmean;
        P.r[i] = v;
        P.bkeep[i] = v;
        P.xs[i] = 0.0;
        P.p[i] = 0.0;
        P.zold[i] = 0.0;
        s[0] += v * v;
    }
    if (!allreduce<1>(s, P, gen, ridx)) return;
    const double bn2 = s[0];
    double rz = 1.0;
    if (!p_cycle(P, T, gen)) return;
    if (!p_cg_tail(P, T, gen, ridx, rz)) return;

    const PLevel &F = T.lv[0];
    int it = 0;
    double rel = 1.0, rr = 0.0;
    if (g.tid == 0) P.hist[0] = 1.0;
    while (it < maxit) {
        double pq[1];
        P_TPR_RET(F.tpr, pq[0], p_spmv_dot, F, P.p, P.q, g);
        if (!allreduce<1>(pq, P, gen, ridx)) return;
        const double alpha = pq[0] != 0.0 ? rz / pq[0] : 0.0;
        double r2[1] = {0.0};
        for (int i = g.tid; i < n; i += g.nthreads) {
            P.xs[i] += alpha * P.p[i];
            const double ri = P.r[i] - alpha * P.q[i];
            P.r[i] = ri;
            r2[0] += ri * ri;
        }
        if (!allreduce<1>(r2, P, gen, ridx)) return;
        rr = r2[0];
        it++;
        rel = bn2 > 0.0 ? sqrt(rr / bn2) : 0.0;
        if (g.tid == 0) P.hist[it] = rel;
        if (!(rel > tol)) break;
        if (!p_cycle(P, T, gen)) return;
        if (!p_cg_tail(P, T, gen, ridx, rz)) return;
    }
    double tr[1];
    P_TPR_RET(F.tpr, tr[0], p_true_rr, F, P.xs, P.bkeep, g);
    if (!allreduce<1>(tr, P, gen, ridx)) return;
    for (int i = g.tid; i < n; i += g.nthreads) phi_out[P.perm0[i]] = P.xs[i];
    if (g.tid == 0) {
        P.scal[S_BN2] = bn2;
        P.scal[S_RR] = rr;
        P.scal[S_TRUE_RR] = tr[0];
        P.scal[S_BMEAN] = bmean;
        P.scal[S_ITERS] = (double)it;
    }
}

size_t persistent_smem(int nlev, int nops, int ncptr) {
    return (size_t)nlev * sizeof(PLevel) + (size_t)nops * (sizeof(Op) + sizeof(int32_t)) +
           (size_t)ncptr * sizeof(int32_t);
}

int persistent_grid(int device, size_t smem) {
    int sms = 0, per = 0;
    if (cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent, PBS, smem) != cudaSuccess) return 0;
    if (per < 1) return 0;
    return sms;  // one CTA per SM: measured faster than two (fewer barrier arrivals)
}

cudaError_t launch_persistent(const PSolve *P, int grid, size_t smem, int mode, int maxit, double tol,
                              const double *b_in, double *phi_out, cudaStream_t s, unsigned long long *prof,
                              unsigned long long wait_ns) {
    void *args[] = {(void *)&P,    (void *)&mode,    (void *)&maxit, (void *)&tol,
                    (void *)&b_in, (void *)&phi_out, (void *)&prof,  (void *)&wait_ns};
    return cudaLaunchCooperativeKernel((const void *)k_persistent, dim3(grid), dim3(PBS), args, smem, s);
}

}  // namespace lamg
