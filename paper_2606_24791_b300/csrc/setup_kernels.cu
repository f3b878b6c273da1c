// GPU setup kernels (Section 2): the K test vectors (K9) and the per-edge affinity with the
// strength-of-connection flag (K10).
//
// These kernels feed integer decisions on the host (which seed a node joins, whether a row is
// upgraded to caliber-2), so they evaluate their sums in a fixed order with explicitly
// rounded operations (__dmul_rn / __dadd_rn / __ddiv_rn, no fused multiply-add): each row's
// neighbour sum runs over the row's entries in stored order, one thread per row. The result
// is then the exactly rounded value of that left-to-right sum, the same on every run.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdio>
#include <vector>

#include "internal.h"

namespace lamg {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LAMG_OK;
    fprintf(stderr, "lamg: CUDA error %s\n", cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return LAMG_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return LAMG_ERR_NO_DEVICE;
    return LAMG_ERR_CUDA;
}

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) { rc = cuda_status(e_); goto out; } \
    } while (0)

// SplitMix64 (Steele, Lea and Flood 2014): state advanced by 0x9e3779b97f4a7c15, each state
// mixed by two xor-shift-multiply rounds; output i of the stream from `seed` is
// mix(seed + i * increment). The test-vector start of column k at node u of level `lvl` is
// output 1 + ((lvl << 44) | (u << 2) | k) mapped to [-1, 1) through its top 53 bits.
__device__ __forceinline__ double random_start(uint64_t seed, int lvl, int64_t u, int k) {
    uint64_t c = ((uint64_t)lvl << 44) | ((uint64_t)u << 2) | (uint64_t)k;
    uint64_t z = seed + (c + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z = z ^ (z >> 31);
    double r = __dmul_rn((double)(z >> 11), 1.0 / 9007199254740992.0);
    return __dsub_rn(__dmul_rn(2.0, r), 1.0);
}

__global__ void k_tv_start(int64_t n, int K, uint64_t seed, int lvl, double *X) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * K) return;
    X[i] = random_start(seed, lvl, i / K, (int)(i % K));
}

// One Gauss-Seidel colour class on A X = 0 for all K columns: X_u <- -(sum_v A_uv X_v) / A_uu.
// Rows of one colour are pairwise non-adjacent, so they update independently.
template <int K>
__global__ void k_tv_colour(int64_t cnt, const int32_t *__restrict__ rows,
                            const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ val, const double *__restrict__ diag,
                            double *X) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int32_t u = rows[t];
    double s[K];
#pragma unroll
    for (int k = 0; k < K; k++) s[k] = 0.0;
    for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
        const double a = val[e];
        const double *xv = X + (int64_t)ci[e] * K;
#pragma unroll
        for (int k = 0; k < K; k++) s[k] = __dadd_rn(s[k], __dmul_rn(a, xv[k]));
    }
    const double d = diag[u];
#pragma unroll
    for (int k = 0; k < K; k++) X[(int64_t)u * K + k] = __ddiv_rn(__dsub_rn(0.0, s[k]), d);
}

// Generic-K variant.
__global__ void k_tv_colour_any(int K, int64_t cnt, const int32_t *__restrict__ rows,
                                const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const double *__restrict__ val, const double *__restrict__ diag,
                                double *X) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int32_t u = rows[t];
    for (int k = 0; k < K; k++) {
        double s = 0.0;
        for (int64_t e = rp[u]; e < rp[u + 1]; e++)
            s = __dadd_rn(s, __dmul_rn(val[e], X[(int64_t)ci[e] * K + k]));
        X[(int64_t)u * K + k] = __ddiv_rn(__dsub_rn(0.0, s), diag[u]);
    }
}

// Affinity (Eq. 3) per off-diagonal entry and the veto flag of Eq. 9 from the row's side:
// strong = |A_uv| >= tau * max_t |A_ut|.
__global__ void k_affinity(int64_t n, int K, double tau, int veto, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ ci, const double *__restrict__ val,
                           const double *__restrict__ X, double *aff, uint8_t *strong) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    double mx = 0.0;
    for (int64_t e = rp[u]; e < rp[u + 1]; e++) mx = fmax(mx, fabs(val[e]));
    const double thr = __dmul_rn(tau, mx);
    const double *xu = X + u * K;
    double uu = 0.0;
    for (int k = 0; k < K; k++) uu = __dadd_rn(uu, __dmul_rn(xu[k], xu[k]));
    for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
        const double *xv = X + (int64_t)ci[e] * K;
        double uv = 0.0, vv = 0.0;
        for (int k = 0; k < K; k++) uv = __dadd_rn(uv, __dmul_rn(xu[k], xv[k]));
        for (int k = 0; k < K; k++) vv = __dadd_rn(vv, __dmul_rn(xv[k], xv[k]));
        aff[e] = __ddiv_rn(__dmul_rn(uv, uv), __dmul_rn(uu, vv));
        strong[e] = veto ? (fabs(val[e]) >= thr) : 1;
    }
}

// Energy-ratio guard of Eq. 4 from the moments of Appendix B, per entry (u, s) of u's row:
// s0 = sum_v w_uv, s1_k = sum_v w_uv x_vk, s2_k = sum_v w_uv x_vk^2 (w_uv = -A_uv, stored
// order); per column k, relaxed = (s2 - s1^2/s0)/2, forced = (x_sk^2 s0 - 2 x_sk s1 + s2)/2,
// scale = (|s2| + s1^2/|s0|)/2; ratio = forced/relaxed, or 1 / infinity when relaxed <= eps
// scale (1 if forced is as small too); q = the largest ratio over k. adm[e] = strong[e] and
// q <= Q. One thread per row, every operation explicitly rounded (no contraction), so the
// decisions are those of the same formula evaluated on the host.
constexpr int GUARD_KMAX = 16;

__global__ void k_guard(int64_t n, int K, double Q, double eps, const int64_t *__restrict__ rp,
                        const int32_t *__restrict__ ci, const double *__restrict__ val,
                        const double *__restrict__ X, const uint8_t *__restrict__ strong, uint8_t *adm) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    double s0 = 0.0, s1[GUARD_KMAX], s2[GUARD_KMAX];
    for (int k = 0; k < K; k++) { s1[k] = 0.0; s2[k] = 0.0; }
    for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
        const double w = -val[e];
        const double *xv = X + (int64_t)ci[e] * K;
        s0 = __dadd_rn(s0, w);
        for (int k = 0; k < K; k++) {
            const double wx = __dmul_rn(w, xv[k]);
            s1[k] = __dadd_rn(s1[k], wx);
            s2[k] = __dadd_rn(s2[k], __dmul_rn(wx, xv[k]));
        }
    }
    for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
        if (!strong[e]) { adm[e] = 0; continue; }
        const double *xs = X + (int64_t)ci[e] * K;
        double worst = 0.0;
        for (int k = 0; k < K; k++) {
            const double s11 = __dmul_rn(s1[k], s1[k]);
            const double relaxed = __dmul_rn(0.5, __dsub_rn(s2[k], __ddiv_rn(s11, s0)));
            const double forced = __dmul_rn(0.5, __dadd_rn(__dsub_rn(__dmul_rn(__dmul_rn(xs[k], xs[k]), s0),
                                                                     __dmul_rn(__dmul_rn(2.0, xs[k]), s1[k])),
                                                           s2[k]));
            const double scale = __dmul_rn(0.5, __dadd_rn(fabs(s2[k]), __ddiv_rn(s11, fabs(s0))));
            const double lim = __dmul_rn(eps, scale);
            double r;
            if (relaxed <= lim) r = (forced <= lim) ? 1.0 : CUDART_INF;
            else r = __ddiv_rn(forced, relaxed);
            worst = (worst < r) ? r : worst;
        }
        adm[e] = worst <= Q ? 1 : 0;
    }
}

static inline unsigned nblk(int64_t work, int bs) { return (unsigned)((work + bs - 1) / bs); }

// Upload a level operator (natural order) and run K9 (and K10 when aff != nullptr). Everything is
// ordered on a private stream with stream-ordered allocations, so a setup running on a host
// thread never synchronises the whole device (solves of other hierarchies keep running).
static int run_setup_kernels(const HostMat &A, const std::vector<int32_t> *colour, int level,
                             uint64_t seed, int K, int nu, double tau, int veto, double *X,
                             const double *Xin, double *aff, uint8_t *strong, double Q = 0.0,
                             double eps = 0.0, uint8_t *adm = nullptr) {
    int rc = LAMG_OK;
    const int64_t n = A.n, z = A.nnz();
    int64_t *d_rp = nullptr;
    int32_t *d_ci = nullptr, *d_rows = nullptr;
    double *d_val = nullptr, *d_diag = nullptr, *d_X = nullptr, *d_aff = nullptr;
    uint8_t *d_strong = nullptr, *d_adm = nullptr;
    const int bs = 128;
    cudaStream_t st = nullptr;
    std::vector<int32_t> rows;
    std::vector<int64_t> cptr;
    int ncol = 0;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaMallocAsync((void **)&d_rp, (n + 1) * sizeof(int64_t), st));
    CK(cudaMallocAsync((void **)&d_ci, (z ? z : 1) * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_val, (z ? z : 1) * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_diag, n * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_X, n * K * sizeof(double), st));
    CK(cudaMemcpyAsync(d_rp, A.rp.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (z) CK(cudaMemcpyAsync(d_ci, A.ci.data(), z * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (z) CK(cudaMemcpyAsync(d_val, A.val.data(), z * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_diag, A.diag.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (colour) {
        // rows grouped by colour, ascending within a colour
        for (int32_t c : *colour) ncol = std::max(ncol, c + 1);
        cptr.assign(ncol + 1, 0);
        for (int32_t c : *colour) cptr[c + 1]++;
        for (int c = 0; c < ncol; c++) cptr[c + 1] += cptr[c];
        rows.resize(n);
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
        for (int64_t u = 0; u < n; u++) rows[fill[(*colour)[u]]++] = (int32_t)u;
        CK(cudaMallocAsync((void **)&d_rows, n * sizeof(int32_t), st));
        CK(cudaMemcpyAsync(d_rows, rows.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        k_tv_start<<<nblk(n * K, bs), bs, 0, st>>>(n, K, seed, level, d_X);
        for (int s = 0; s < nu; s++) {
            for (int c = 0; c < ncol; c++) {
                const int64_t cnt = cptr[c + 1] - cptr[c];
                if (!cnt) continue;
                if (K == 4)
                    k_tv_colour<4><<<nblk(cnt, bs), bs, 0, st>>>(cnt, d_rows + cptr[c], d_rp, d_ci, d_val, d_diag, d_X);
                else
                    k_tv_colour_any<<<nblk(cnt, bs), bs, 0, st>>>(K, cnt, d_rows + cptr[c], d_rp, d_ci, d_val, d_diag, d_X);
            }
        }
        CK(cudaGetLastError());
        if (X) CK(cudaMemcpyAsync(X, d_X, n * K * sizeof(double), cudaMemcpyDeviceToHost, st));
    } else {
        CK(cudaMemcpyAsync(d_X, Xin, n * K * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    if (aff) {
        CK(cudaMallocAsync((void **)&d_aff, (z ? z : 1) * sizeof(double), st));
        CK(cudaMallocAsync((void **)&d_strong, (z ? z : 1), st));
        k_affinity<<<nblk(n, bs), bs, 0, st>>>(n, K, tau, veto, d_rp, d_ci, d_val, d_X, d_aff, d_strong);
        CK(cudaGetLastError());
        if (z) CK(cudaMemcpyAsync(aff, d_aff, z * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (z) CK(cudaMemcpyAsync(strong, d_strong, z, cudaMemcpyDeviceToHost, st));
        if (adm && K <= GUARD_KMAX) {
            CK(cudaMallocAsync((void **)&d_adm, (z ? z : 1), st));
            k_guard<<<nblk(n, bs), bs, 0, st>>>(n, K, Q, eps, d_rp, d_ci, d_val, d_X, d_strong, d_adm);
            CK(cudaGetLastError());
            if (z) CK(cudaMemcpyAsync(adm, d_adm, z, cudaMemcpyDeviceToHost, st));
        }
    }
    CK(cudaStreamSynchronize(st));
out:
    if (st) {
        void *ptrs[] = {d_rp, d_ci, d_val, d_diag, d_X, d_rows, d_aff, d_strong, d_adm};
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

int gpu_testvectors(const HostMat &A, const std::vector<int32_t> &colour, int level,
                    uint64_t seed, int K, int nu, double *X) {
    return run_setup_kernels(A, &colour, level, seed, K, nu, 0.0, 1, X, nullptr, nullptr, nullptr);
}

int gpu_affinity(const HostMat &A, const double *X, int K, double tau, double *aff,
                 uint8_t *strong) {
    return run_setup_kernels(A, nullptr, 0, 0, K, 0, tau, 1, nullptr, X, aff, strong);
}

int gpu_tv_and_affinity(const HostMat &A, const std::vector<int32_t> &colour, int level,
                        uint64_t seed, int K, int nu, double tau, int veto, double *X,
                        double *aff, uint8_t *strong, double Q, double eps, uint8_t *adm) {
    return run_setup_kernels(A, &colour, level, seed, K, nu, tau, veto, X, nullptr, aff, strong, Q, eps, adm);
}

}  // namespace lamg
