// Inverse of the dense coarsest matrix M = A + J/n (symmetric positive definite for a connected
// Laplacian-like A) on the GPU, by in-place Gauss-Jordan elimination without pivoting: step k
// turns column k into the k-th column of the inverse. With p = M_kk (positive for an SPD matrix,
// the Schur complement diagonal of step k) and r, c the pivot row and column before the step:
//   M_ij -= c_i r_j / p (i, j != k),  M_kj = r_j / p,  M_ik = -c_i / p,  M_kk = 1 / p.
// Each step is two launches: the pivot row and column (scaled) saved to a buffer, then the
// n x n update. For the coarsest sizes used (n <= 4096) the matrix stays in L2 for n up to
// about 3000, so a step costs about a launch.
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>

#include "internal.h"

namespace lamg {

// save: rs[j] = M_kj / p (row), cs[i] = M_ik (column); a non-positive pivot sets *bad
__global__ void k_gj_save(int n, int k, const double *__restrict__ M, double *__restrict__ rs,
                          double *__restrict__ cs, int *bad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double p = M[(size_t)k * n + k];
    if (t == 0 && !(p > 0.0)) *bad = 1;
    rs[t] = M[(size_t)k * n + t] / p;
    cs[t] = M[(size_t)t * n + k];
}

__global__ void k_gj_update(int n, int k, double *__restrict__ M, const double *__restrict__ rs,
                            const double *__restrict__ cs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n) return;
    const double p = cs[k];
    double &m = M[(size_t)i * n + j];
    if (i == k) m = (j == k) ? 1.0 / p : rs[j];
    else if (j == k) m = -cs[i] / p;
    else m = fma(-cs[i], rs[j], m);
}

int gpu_dense_inverse(int64_t n64, std::vector<double> &M) {
    if (n64 < 1 || n64 > 8192 || (int64_t)M.size() != n64 * n64) return LAMG_ERR_INVALID;
    const int n = (int)n64;
    int rc = LAMG_OK, bad = 0;
    double *d_M = nullptr, *d_r = nullptr, *d_c = nullptr;
    int *d_bad = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    const size_t bytes = (size_t)n * n * sizeof(double);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_M, bytes, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_r, n * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_c, n * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_bad, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_M, M.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const unsigned gb = (unsigned)((n + 255) / 256);
        const dim3 grid(gb, (unsigned)n);
        for (int k = 0; k < n; k++) {
            k_gj_save<<<gb, 256, 0, st>>>(n, k, d_M, d_r, d_c, d_bad);
            k_gj_update<<<grid, 256, 0, st>>>(n, k, d_M, d_r, d_c);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.data(), d_M, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_status(e);
    else if (bad) rc = LAMG_ERR_DISCONNECTED;  // not positive definite: the graph is not connected
    if (st) {
        void *ptrs[] = {d_M, d_r, d_c, d_bad};
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

}  // namespace lamg
