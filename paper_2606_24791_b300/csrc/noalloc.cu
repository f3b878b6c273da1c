// Allocation-free variant of the test-vector setup kernel (K9), for callers that cannot
// allocate device memory themselves.
//
// Some callers of this library run where cudaMalloc is not available to them: code inside a
// memory pool owned by another framework, plugins restricted to memory handed to them, or
// code that must not allocate after start-up. lamg_testvectors() copies its host inputs into
// device buffers it allocates; this variant takes device inputs and output from the caller and
// keeps its one piece of scratch (the rows grouped by colour class, and the class offsets) in a
// file-scope __device__ array of fixed size, so it allocates nothing.
//
// Contract:
//  - n <= NOALLOC_MAX_ROWS and ncol <= NOALLOC_MAX_COLOURS, else LAMG_ERR_INVALID.
//  - Rows whose colour is outside [0, ncol) are never relaxed and keep their random start.
//  - The first call on a device looks up the device address of the scratch array
//    (cudaGetSymbolAddress) with that device current; make that first call before any stream
//    capture on the device.
//  - Every call shares the one scratch array per device, which keeps the contents of the last
//    call; the counters that must start at zero are cleared at the start of every call. Calls
//    whose work overlaps on the GPU (other streams, other host threads) race on the scratch:
//    serialise them.
//  - No cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace lamg {

constexpr int64_t NOALLOC_MAX_ROWS = 1 << 21;    // 8 MiB of row ids
constexpr int NOALLOC_MAX_COLOURS = 1024;
constexpr int NA_STRIDE = 32;                    // rows longer than this: one warp (strided order)

struct NoallocScratch {
    int32_t rows[NOALLOC_MAX_ROWS];              // row ids grouped by colour class
    int32_t count[NOALLOC_MAX_COLOURS];          // rows per class summed in stored order
    int32_t count_long[NOALLOC_MAX_COLOURS];     // rows per class summed as strided partials
    int32_t offset[NOALLOC_MAX_COLOURS + 1];     // class start in rows[]
    int32_t loff[NOALLOC_MAX_COLOURS];           // start of the class's strided rows
    int32_t fill[NOALLOC_MAX_COLOURS];           // scatter cursors
    int32_t lfill[NOALLOC_MAX_COLOURS];
};

static __device__ __align__(256) NoallocScratch g_noalloc;

// Same start values and sweep arithmetic as the allocating kernels (setup_kernels.cu):
// SplitMix64 output 1 + ((level << 44) | (u << 4) | k) mapped to [-1, 1), then colour-ordered
// Gauss-Seidel on A x = 0, no FMA contraction: a row in stored order on one thread, or (strided
// order, rows of more than 32 entries) as 32 strided partials on one warp added in lane order.
__device__ __forceinline__ double na_random_start(uint64_t seed, int lvl, int64_t u, int k) {
    uint64_t c = ((uint64_t)lvl << 44) | ((uint64_t)u << 4) | (uint64_t)k;
    uint64_t z = seed + (c + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z = z ^ (z >> 31);
    double r = __dmul_rn((double)(z >> 11), 1.0 / 9007199254740992.0);
    return __dsub_rn(__dmul_rn(2.0, r), 1.0);
}

__device__ __forceinline__ bool na_long(const int64_t *rp, int64_t u, int order) {
    return order == LAMG_TV_STRIDED && rp[u + 1] - rp[u] > NA_STRIDE;
}

__global__ void k_na_clear(NoallocScratch *S, int ncol) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
        S->count[c] = 0;
        S->count_long[c] = 0;
    }
}

__global__ void k_na_count(NoallocScratch *S, int64_t n, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ colour, int ncol, int order, double *X, int K,
                           uint64_t seed, int lvl) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int c = colour[u];
        if (c >= 0 && c < ncol) atomicAdd(na_long(rp, u, order) ? &S->count_long[c] : &S->count[c], 1);
        for (int k = 0; k < K; k++) X[u * K + k] = na_random_start(seed, lvl, u, k);
    }
}

__global__ void k_na_scan(NoallocScratch *S, int ncol) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int32_t acc = 0;
    for (int c = 0; c < ncol; c++) {
        S->offset[c] = acc;
        S->fill[c] = acc;
        acc += S->count[c];
        S->loff[c] = acc;
        S->lfill[c] = acc;
        acc += S->count_long[c];
    }
    S->offset[ncol] = acc;
}

__global__ void k_na_scatter(NoallocScratch *S, int64_t n, const int64_t *__restrict__ rp,
                             const int32_t *__restrict__ colour, int ncol, int order) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int c = colour[u];
        if (c >= 0 && c < ncol)
            S->rows[atomicAdd(na_long(rp, u, order) ? &S->lfill[c] : &S->fill[c], 1)] = (int32_t)u;
    }
}

// The stored-order rows of one colour class, one thread per row; the class range is read from
// the scratch offsets.
__global__ void k_na_colour(const NoallocScratch *S, int c, int K, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const double *__restrict__ val,
                            const double *__restrict__ diag, double *X) {
    const int32_t r0 = S->offset[c], r1 = S->loff[c];
    for (int32_t t = r0 + blockIdx.x * blockDim.x + threadIdx.x; t < r1; t += gridDim.x * blockDim.x) {
        const int32_t u = S->rows[t];
        for (int k = 0; k < K; k++) {
            double s = 0.0;
            for (int64_t e = rp[u]; e < rp[u + 1]; e++)
                s = __dadd_rn(s, __dmul_rn(val[e], X[(int64_t)ci[e] * K + k]));
            X[(int64_t)u * K + k] = __ddiv_rn(__dsub_rn(0.0, s), diag[u]);
        }
    }
}

// The strided rows of one colour class, one warp per row: lane j sums entries j, j + 32, ... in
// order from 0.0, then the 32 partials are added in lane order from 0.0.
__global__ void k_na_long(const NoallocScratch *S, int c, int K, const int64_t *__restrict__ rp,
                          const int32_t *__restrict__ ci, const double *__restrict__ val,
                          const double *__restrict__ diag, double *X) {
    const int32_t r0 = S->loff[c], r1 = S->offset[c + 1];
    const int lane = threadIdx.x & 31;
    const int32_t warps = (int32_t)(gridDim.x * blockDim.x / 32);
    for (int32_t t = r0 + (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < r1; t += warps) {
        const int32_t u = S->rows[t];
        const int64_t e0 = rp[u], e1 = rp[u + 1];
        const double d = diag[u];
        for (int k = 0; k < K; k++) {
            double p = 0.0;
            for (int64_t e = e0 + lane; e < e1; e += NA_STRIDE)
                p = __dadd_rn(p, __dmul_rn(val[e], X[(int64_t)ci[e] * K + k]));
            double s = 0.0;
            for (int j = 0; j < NA_STRIDE; j++) s = __dadd_rn(s, __shfl_sync(0xffffffffu, p, j));
            if (lane == 0) X[(int64_t)u * K + k] = __ddiv_rn(__dsub_rn(0.0, s), d);
        }
    }
}

// Device address of the scratch array, looked up once per device.
static NoallocScratch *scratch_for(int device, int *rc) {
    static std::mutex mu;
    static NoallocScratch *addr[64] = {nullptr};
    *rc = LAMG_OK;
    if (device < 0 || device >= 64) { *rc = LAMG_ERR_INVALID; return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
        if (e != cudaSuccess) { *rc = cuda_status(e); return nullptr; }
        addr[device] = (NoallocScratch *)p;
    }
    return addr[device];
}

}  // namespace lamg

using namespace lamg;

extern "C" int lamg_testvectors_noalloc(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                                        const double *diag, const int32_t *colour, int32_t ncol,
                                        int32_t level, uint64_t seed, int32_t K, int32_t nu, double *X,
                                        void *stream, int32_t order) {
    if (n < 1 || n > NOALLOC_MAX_ROWS || ncol < 1 || ncol > NOALLOC_MAX_COLOURS || K < 1 || K > 16 || nu < 0 ||
        !rp || !diag || !colour || !X || (order != LAMG_TV_STRIDED && order != LAMG_TV_STORED))
        return LAMG_ERR_INVALID;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    int rc;
    NoallocScratch *S = scratch_for(dev, &rc);
    if (!S) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int bs = 128;
    const unsigned g = (unsigned)std::min<int64_t>((n + bs - 1) / bs, 148 * 16);
    k_na_clear<<<(ncol + bs - 1) / bs, bs, 0, s>>>(S, ncol);
    k_na_count<<<g, bs, 0, s>>>(S, n, rp, colour, ncol, order, X, K, seed, level);
    k_na_scan<<<1, 1, 0, s>>>(S, ncol);
    k_na_scatter<<<g, bs, 0, s>>>(S, n, rp, colour, ncol, order);
    for (int sweep = 0; sweep < nu; sweep++)
        for (int c = 0; c < ncol; c++) {
            k_na_colour<<<g, bs, 0, s>>>(S, c, K, rp, ci, val, diag, X);
            if (order == LAMG_TV_STRIDED) k_na_long<<<148, 256, 0, s>>>(S, c, K, rp, ci, val, diag, X);
        }
    e = cudaGetLastError();
    return cuda_status(e);
}
