// Stationary outer iteration with iterate recombination (Section 2): the paper's own solver
// loop, as an alternative to flexible CG.
//
//   x <- x + M(b - A x)                                   (one cycle of Section 2)
//   E = [x_1 - x, ..., x_m - x]  (the last m <= kappa saved iterates)
//   alpha = argmin || (b - A x) - A E alpha ||_2           (normal equations, m x m)
//   x <- x + E alpha; save x; x <- x - mean(x)
//
// Every vector step runs on the GPU (residual, A E, the dot products of the normal equations
// with a deterministic two-kernel reduction, the updates); the m x m system (m <= 16) is solved
// on the host by Gaussian elimination with partial pivoting. The per-cycle relative residual
// history is what the paper's convergence factor (ACF) is measured on.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "hier.h"
#include "kernels_common.cuh"

using namespace lamg;

namespace {

constexpr int SBS = 256;
constexpr int KMAXR = 16;           // saved iterates at most
constexpr int SPARTS = 592;         // partial-sum blocks of the dot-product kernel (4 x 148)

// r = b - A x, one thread per row, entries in stored order
__global__ void k_st_resid(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ val, const double *__restrict__ diag,
                           const double *__restrict__ x, const double *__restrict__ b, double *r) {
    const int i = blockIdx.x * SBS + threadIdx.x;
    if (i >= n) return;
    double s = diag[i] * x[i];
    for (int e = rp[i]; e < rp[i + 1]; e++) s += val[e] * x[ci[e]];
    r[i] = b[i] - s;
}

// w = A v
__global__ void k_st_matvec(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ val, const double *__restrict__ diag,
                            const double *__restrict__ v, double *w) {
    const int i = blockIdx.x * SBS + threadIdx.x;
    if (i >= n) return;
    double s = diag[i] * v[i];
    for (int e = rp[i]; e < rp[i + 1]; e++) s += val[e] * v[ci[e]];
    w[i] = s;
}

// out = a - c
__global__ void k_st_sub(int n, const double *__restrict__ a, const double *__restrict__ c, double *out) {
    const int i = blockIdx.x * SBS + threadIdx.x;
    if (i < n) out[i] = a[i] - c[i];
}

// x += z
__global__ void k_st_add(int n, const double *__restrict__ z, double *x) {
    const int i = blockIdx.x * SBS + threadIdx.x;
    if (i < n) x[i] += z[i];
}

// x += sum_j alpha_j E_j (alpha from the host, j in order)
struct Alpha {
    double a[KMAXR];
};
__global__ void k_st_combine(int n, int m, Alpha al, const double *__restrict__ E, double *x) {
    const int i = blockIdx.x * SBS + threadIdx.x;
    if (i >= n) return;
    double v = x[i];
    for (int j = 0; j < m; j++) v += al.a[j] * E[(size_t)j * n + i];
    x[i] = v;
}

// x -= mean (mean from the device scalar)
__global__ void k_st_sub_mean(int n, const double *__restrict__ sum, double *x) {
    const int i = blockIdx.x * SBS + threadIdx.x;
    if (i < n) x[i] -= sum[0] / (double)n;
}

// Block partials of npairs dot products u_q . v_q (q in order), each block a fixed slice of
// the rows and a fixed-order block reduction: part[q * gridDim.x + block].
struct Pairs {
    const double *u[KMAXR * KMAXR + KMAXR + 2];
    const double *v[KMAXR * KMAXR + KMAXR + 2];
};
__global__ void __launch_bounds__(SBS) k_st_dots_part(int n, int np, Pairs pr, double *part) {
    for (int q = 0; q < np; q++) {
        double s[1] = {0.0};
        for (int i = blockIdx.x * SBS + threadIdx.x; i < n; i += gridDim.x * SBS) s[0] += pr.u[q][i] * pr.v[q][i];
        block_sum<1>(s);
        if (threadIdx.x == 0) part[q * gridDim.x + blockIdx.x] = s[0];
    }
}

// out[q] = sum over blocks in order
__global__ void k_st_dots_sum(int np, int nb, const double *__restrict__ part, double *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += part[q * nb + b];
    out[q] = s;
}

struct StWork {
    int kappa = -1, nsaved = 0;
    double *saved = nullptr, *E = nullptr, *AE = nullptr, *part = nullptr, *dout = nullptr, *x = nullptr;
    double *ones = nullptr;
    double *h_out = nullptr;  // pinned
    int order[KMAXR];         // saved slots, oldest first
};

inline unsigned nblk(int64_t n) { return (unsigned)((n + SBS - 1) / SBS); }

// sums of np pairs into h_out (waits)
int dots(lamg_hier *h, StWork &w, int n, int np, const Pairs &pr, cudaStream_t s) {
    k_st_dots_part<<<SPARTS, SBS, 0, s>>>(n, np, pr, w.part);
    k_st_dots_sum<<<(np + 127) / 128, 128, 0, s>>>(np, SPARTS, w.part, w.dout);
    CKR(cudaMemcpyAsync(w.h_out, w.dout, np * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev_poll, s));
    return wait_event(h, h->ev_poll);
}

}  // namespace

extern "C" int lamg_solve_stationary(lamg_hier *h, const double *b, double *phi, int32_t kappa,
                                     const lamg_solve_opts *so, lamg_stats *st) {
    if (!h || !b || !phi || !so || !(so->tol > 0) || so->maxit < 1 || kappa < 0 || kappa > KMAXR)
        return LAMG_ERR_INVALID;
    if (h->opt.precision != LAMG_FP64) return LAMG_ERR_INVALID;
    CKR(cudaSetDevice(h->device));
    cudaStream_t s = so->stream ? (cudaStream_t)so->stream : h->stream;
    const bool devp = so->flags & LAMG_DEVICE_PTRS;
    const DevLevel &F = h->dev[0];
    const int n = (int)F.n;
    int rc = LAMG_OK;
    StWork w;
    const int kc = kappa > 0 ? kappa : 1;
    if ((rc = dalloc(h, &w.saved, (int64_t)kc * n)) || (rc = dalloc(h, &w.E, (int64_t)kc * n)) ||
        (rc = dalloc(h, &w.AE, (int64_t)kc * n)) || (rc = dalloc(h, &w.part, (int64_t)SPARTS * (KMAXR * KMAXR + KMAXR + 2))) ||
        (rc = dalloc(h, &w.dout, KMAXR * KMAXR + KMAXR + 2)) || (rc = dalloc(h, &w.ones, n)))
        return rc;
    std::vector<double> one(n, 1.0);
    CKR(cudaMemcpyAsync(w.ones, one.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    CKR(cudaHostAlloc(&w.h_out, (KMAXR * KMAXR + KMAXR + 2) * sizeof(double), cudaHostAllocDefault));
    double *x = h->xs, *r = h->r, *bb = h->bkeep, *z = F.x;
    // b in device order, projected to mean zero (Eq. 1); ||b||
    CKR(cudaEventRecord(h->ev_a, s));
    CKR(cudaMemcpyAsync(h->nat_in, b, n * sizeof(double), devp ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    launch_gather(n, h->perm0, h->nat_in, bb, s);
    Pairs pr{};
    pr.u[0] = bb; pr.v[0] = w.ones;
    if ((rc = dots(h, w, n, 1, pr, s))) { cudaFreeHost(w.h_out); return rc; }
    const double bmean = w.h_out[0] / (double)n;
    k_st_sub_mean<<<nblk(n), SBS, 0, s>>>(n, w.dout, bb);
    pr.u[0] = bb; pr.v[0] = bb;
    if ((rc = dots(h, w, n, 1, pr, s))) { cudaFreeHost(w.h_out); return rc; }
    const double bn = std::sqrt(w.h_out[0]);
    CKR(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    int it = 0;
    double rel = 1.0;
    if (st && st->hist) st->hist[0] = 1.0;
    while (it < so->maxit && bn > 0.0) {
        // x <- x + M(b - A x)
        k_st_resid<<<nblk(n), SBS, 0, s>>>(n, F.rp, F.ci, F.val, F.diag, x, bb, r);
        CKR(cudaGraphLaunch(h->g_cycle, s));
        k_st_add<<<nblk(n), SBS, 0, s>>>(n, z, x);
        if (kappa > 0) {
            const int m = w.nsaved;
            if (m > 0) {
                for (int j = 0; j < m; j++) {
                    double *Ej = w.E + (size_t)j * n, *AEj = w.AE + (size_t)j * n;
                    k_st_sub<<<nblk(n), SBS, 0, s>>>(n, w.saved + (size_t)w.order[j] * n, x, Ej);
                    k_st_matvec<<<nblk(n), SBS, 0, s>>>(n, F.rp, F.ci, F.val, F.diag, Ej, AEj);
                }
                k_st_resid<<<nblk(n), SBS, 0, s>>>(n, F.rp, F.ci, F.val, F.diag, x, bb, r);
                // g_a = AE_a . r, G_ac = AE_a . AE_c (pairs in that order)
                int np = 0;
                for (int a = 0; a < m; a++) { pr.u[np] = w.AE + (size_t)a * n; pr.v[np] = r; np++; }
                for (int a = 0; a < m; a++)
                    for (int c = 0; c < m; c++) { pr.u[np] = w.AE + (size_t)a * n; pr.v[np] = w.AE + (size_t)c * n; np++; }
                if ((rc = dots(h, w, n, np, pr, s))) break;
                double G[KMAXR * KMAXR], g[KMAXR];
                for (int a = 0; a < m; a++) {
                    g[a] = w.h_out[a];
                    for (int c = 0; c < m; c++) G[a * m + c] = w.h_out[m + a * m + c];
                }
                // Gaussian elimination with partial pivoting
                bool ok = true;
                for (int c = 0; c < m && ok; c++) {
                    int piv = c;
                    for (int a = c + 1; a < m; a++)
                        if (std::fabs(G[a * m + c]) > std::fabs(G[piv * m + c])) piv = a;
                    if (!(std::fabs(G[piv * m + c]) > 0.0)) { ok = false; break; }
                    if (piv != c) {
                        for (int t = 0; t < m; t++) std::swap(G[c * m + t], G[piv * m + t]);
                        std::swap(g[c], g[piv]);
                    }
                    for (int a = c + 1; a < m; a++) {
                        const double f = G[a * m + c] / G[c * m + c];
                        for (int t = c; t < m; t++) G[a * m + t] -= f * G[c * m + t];
                        g[a] -= f * g[c];
                    }
                }
                if (ok) {
                    Alpha al{};
                    for (int a = m - 1; a >= 0; a--) {
                        double v = g[a];
                        for (int t = a + 1; t < m; t++) v -= G[a * m + t] * al.a[t];
                        al.a[a] = v / G[a * m + a];
                    }
                    k_st_combine<<<nblk(n), SBS, 0, s>>>(n, m, al, w.E, x);
                }
            }
            // save x, dropping the oldest
            int slot;
            if (w.nsaved == kappa) {
                slot = w.order[0];
                for (int j = 0; j + 1 < kappa; j++) w.order[j] = w.order[j + 1];
                w.nsaved--;
            } else {
                slot = w.nsaved;
            }
            CKR(cudaMemcpyAsync(w.saved + (size_t)slot * n, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            w.order[w.nsaved++] = slot;
        }
        // x <- x - mean(x); r = b - A x; ||r|| / ||b||
        pr.u[0] = x; pr.v[0] = w.ones;
        if ((rc = dots(h, w, n, 1, pr, s))) break;
        k_st_sub_mean<<<nblk(n), SBS, 0, s>>>(n, w.dout, x);
        k_st_resid<<<nblk(n), SBS, 0, s>>>(n, F.rp, F.ci, F.val, F.diag, x, bb, r);
        pr.u[0] = r; pr.v[0] = r;
        if ((rc = dots(h, w, n, 1, pr, s))) break;
        it++;
        rel = std::sqrt(w.h_out[0]) / bn;
        if (st && st->hist) st->hist[it] = rel;
        if (rel <= so->tol) break;
    }
    if (!rc) {
        launch_scatter(n, h->perm0, x, h->nat_out, s);
        cudaError_t e = cudaMemcpyAsync(phi, h->nat_out, n * sizeof(double),
                                        devp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_b, s);
        rc = e == cudaSuccess ? wait_event(h, h->ev_b) : cuda_status(e);
        if (!rc && cudaGetLastError() != cudaSuccess) rc = LAMG_ERR_CUDA;
    }
    cudaFreeHost(w.h_out);
    // the work vectors go back to the pool (stream-ordered)
    for (void *p : {(void *)w.saved, (void *)w.E, (void *)w.AE, (void *)w.part, (void *)w.dout, (void *)w.ones}) {
        for (size_t k = 0; k < h->allocs.size(); k++)
            if (h->allocs[k] == p) {
                cudaFreeAsync(p, h->stream);
                h->allocs.erase(h->allocs.begin() + (long)k);
                break;
            }
    }
    if (rc) return rc;
    if (st) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_a, h->ev_b);
        st->iters = it;
        st->nlevels = (int32_t)h->dev.size();
        st->relres = rel;
        st->relres_true = rel;
        st->b_mean = bmean;
        st->solve_ms = ms;
        st->kernel_ms = ms;
        st->alg_bytes = 0.0;
        st->launches = 0;
    }
    return rel <= so->tol ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
}
