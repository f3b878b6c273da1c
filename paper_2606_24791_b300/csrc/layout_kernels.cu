// Device layout of a level's operator, built on the GPU at setup from the level's natural-order
// CSR: the colour-ordered (device-order) CSR with its diagonal and reciprocal diagonal, and the
// sliced-ELLPACK copy used by the one-thread-per-row kernels. Both are pure data movement (the
// reciprocal diagonal is an IEEE-rounded division, the same bits as on the host).
#include <cuda_runtime.h>

#include "device.h"

namespace lamg {

// Row i of device order is natural row perm[i]; its entries keep the natural row's order, with
// column ids renamed by iperm (natural id -> device index). One warp per row, lanes striding
// over the entries (coalesced on both sides).
__global__ void k_layout_rows(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ iperm,
                              const int64_t *__restrict__ nrp, const int32_t *__restrict__ nci,
                              const double *__restrict__ nval, const double *__restrict__ ndiag,
                              const int32_t *__restrict__ rp, int32_t *__restrict__ ci, double *__restrict__ val,
                              double *__restrict__ diag, double *__restrict__ idiag) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int32_t u = perm[i];
    const int64_t e0 = nrp[u], len = nrp[u + 1] - e0;
    const int64_t o = rp[i];
    for (int64_t k = lane; k < len; k += 32) {
        ci[o + k] = iperm[nci[e0 + k]];
        val[o + k] = nval[e0 + k];
    }
    if (lane == 0) {
        const double d = ndiag[u];
        diag[i] = d;
        idiag[i] = 1.0 / d;
    }
}

// Sliced ELLPACK in four-entry blocks (sell_col_at / sell_val_at) for j below the slice's width;
// padding (rows shorter than that, and the rows past n in the last slice) holds value 0 at the
// row's own column (the last row for rows past n). One thread per slot row.
__global__ void k_layout_sell(int64_t n, int64_t ns, const int32_t *__restrict__ sp,
                              const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const double *__restrict__ val, int32_t *__restrict__ sc, double *__restrict__ sv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 32 * ns) return;
    const int64_t s = i >> 5, l = i & 31;
    const int64_t base = sp[s], w = (sp[s + 1] - base) >> 5;
    const bool real = i < n;
    const int64_t e0 = real ? rp[i] : 0, len = real ? rp[i + 1] - e0 : 0;
    const int32_t self = (int32_t)(real ? i : n - 1);
    for (int64_t j = 0; j < w; j++) {
        const int64_t ec = sell_col_at(base, (int)l, (int)j), ev = sell_val_at(base, (int)l, (int)j);
        if (j < len) {
            sc[ec] = ci[e0 + j];
            sv[ev] = val[e0 + j];
        } else {
            sc[ec] = self;
            sv[ev] = 0.0;
        }
    }
}

static inline unsigned nblk(int64_t work, int bs) { return (unsigned)((work + bs - 1) / bs); }

void launch_layout_rows(int64_t n, const int32_t *perm, const int32_t *iperm, const int64_t *nrp,
                        const int32_t *nci, const double *nval, const double *ndiag, const int32_t *rp,
                        int32_t *ci, double *val, double *diag, double *idiag, cudaStream_t s) {
    if (n <= 0) return;
    k_layout_rows<<<nblk(32 * n, 256), 256, 0, s>>>(n, perm, iperm, nrp, nci, nval, ndiag, rp, ci, val, diag,
                                                      idiag);
}

void launch_layout_sell(int64_t n, int64_t ns, const int32_t *sp, const int32_t *rp, const int32_t *ci,
                        const double *val, int32_t *sc, double *sv, cudaStream_t s) {
    if (ns <= 0) return;
    k_layout_sell<<<nblk(32 * ns, 256), 256, 0, s>>>(n, ns, sp, rp, ci, val, sc, sv);
}

}  // namespace lamg
