// GPU setup kernels (Section 2): the K test vectors (K9), the per-edge affinity with the
// strength-of-connection flag (K10), the energy-ratio guard of Eq. 4, the Galerkin coarse
// operator P^T A P and the elimination's Schur complement.
//
// These kernels feed integer decisions on the host (which seed a node joins, whether a row is
// upgraded to caliber-2), so they evaluate their sums in a fixed order with explicitly
// rounded operations (__dmul_rn / __dadd_rn / __ddiv_rn, no fused multiply-add): each row's
// neighbour sum runs over the row's entries in stored order, one thread per row. The result
// is then the exactly rounded value of that left-to-right sum, the same on every run.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
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
// mix(seed + i * increment). The test-vector start of column k (< 16) at node u of level `lvl`
// is output 1 + ((lvl << 44) | (u << 4) | k) mapped to [-1, 1) through its top 53 bits.
__device__ __forceinline__ double random_start(uint64_t seed, int lvl, int64_t u, int k) {
    uint64_t c = ((uint64_t)lvl << 44) | ((uint64_t)u << 4) | (uint64_t)k;
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
// Rows of one colour are pairwise non-adjacent, so they update independently. The neighbour sum
// runs in stored order (one thread per row, these kernels) for every row with LAMG_TV_STORED and
// for rows of at most TV_STRIDE entries with LAMG_TV_STRIDED; with LAMG_TV_STRIDED a longer row
// is summed as TV_STRIDE strided partial sums added in order (one warp per row, k_tv_long).
constexpr int TV_STRIDE = 32;
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

// Rows longer than TV_STRIDE entries, one warp per row: lane j sums entries j, j + 32, ... in
// order (from 0.0), lane 0 then adds the 32 partials in lane order (from 0.0).
__global__ void k_tv_long(int K, int64_t cnt, const int32_t *__restrict__ rows, const int64_t *__restrict__ rp,
                          const int32_t *__restrict__ ci, const double *__restrict__ val,
                          const double *__restrict__ diag, double *X) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= cnt) return;  // whole warps leave together
    const int32_t u = rows[t];
    const int64_t e0 = rp[u], e1 = rp[u + 1];
    const double d = diag[u];
    for (int k = 0; k < K; k++) {
        double p = 0.0;
        for (int64_t e = e0 + lane; e < e1; e += TV_STRIDE)
            p = __dadd_rn(p, __dmul_rn(val[e], X[(int64_t)ci[e] * K + k]));
        double s = 0.0;
        for (int j = 0; j < TV_STRIDE; j++) s = __dadd_rn(s, __shfl_sync(0xffffffffu, p, j));
        if (lane == 0) X[(int64_t)u * K + k] = __ddiv_rn(__dsub_rn(0.0, s), d);
    }
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

// Affinity (Eq. 3) per off-diagonal entry, the veto flag of Eq. 9 from the row's side
// (strong = |A_uv| >= tau * max_t |A_ut|), and the energy-ratio guard of Eq. 4 from the moments
// of Appendix B: s0 = sum_v w_uv, s1_k = sum_v w_uv x_vk, s2_k = sum_v w_uv x_vk^2 (w_uv = -A_uv,
// stored order); per column k, relaxed = (s2 - s1^2/s0)/2, forced = (x_sk^2 s0 - 2 x_sk s1 +
// s2)/2, scale = (|s2| + s1^2/|s0|)/2; ratio = forced/relaxed, or 1 / infinity when relaxed <=
// eps scale (1 if forced is as small too); q = the largest ratio over k; adm[e] = strong[e] and
// q <= Q. Every operation is explicitly rounded (no contraction), so the values and decisions
// are those of the same formulas evaluated on the host and in the oracle.
//
// Two passes: one thread per row for the row quantities (the veto threshold, sum_k x_uk^2 and
// the moments, summed in stored order), then one thread per stored entry for everything that
// is per entry, so a hub row's entries are spread over the GPU instead of one thread.
constexpr int GUARD_KMAX = 16;

// row quantities: rs[u * (3 + 2K)] = {tau max|A_ut|, sum_k x_uk^2, s0, s1[K], s2[K]} (the
// moments only with moments set)
__global__ void k_row_stats(int64_t n, int K, double tau, int moments, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const double *__restrict__ val,
                            const double *__restrict__ X, double *__restrict__ rs) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    double *r = rs + u * (3 + 2 * K);
    double mx = 0.0;
    for (int64_t e = rp[u]; e < rp[u + 1]; e++) mx = fmax(mx, fabs(val[e]));
    r[0] = __dmul_rn(tau, mx);
    const double *xu = X + u * K;
    double uu = 0.0;
    for (int k = 0; k < K; k++) uu = __dadd_rn(uu, __dmul_rn(xu[k], xu[k]));
    r[1] = uu;
    if (!moments) return;
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
    r[2] = s0;
    for (int k = 0; k < K; k++) { r[3 + k] = s1[k]; r[3 + K + k] = s2[k]; }
}

// per stored entry e (row u found by binary search in rp): aff[e], strong[e] and, with adm
// set, adm[e]
__global__ void k_entry_affinity(int64_t n, int64_t z, int K, int veto, double Q, double eps,
                                 const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const double *__restrict__ val, const double *__restrict__ X,
                                 const double *__restrict__ rs, double *aff, uint8_t *strong, uint8_t *adm) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= z) return;
    int64_t lo = 0, hi = n - 1;  // the row u with rp[u] <= e < rp[u + 1]
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    const int64_t u = lo;
    const double *r = rs + u * (3 + 2 * K);
    const double *xu = X + u * K, *xv = X + (int64_t)ci[e] * K;
    double uv = 0.0, vv = 0.0;
    for (int k = 0; k < K; k++) uv = __dadd_rn(uv, __dmul_rn(xu[k], xv[k]));
    for (int k = 0; k < K; k++) vv = __dadd_rn(vv, __dmul_rn(xv[k], xv[k]));
    aff[e] = __ddiv_rn(__dmul_rn(uv, uv), __dmul_rn(r[1], vv));
    const uint8_t st = veto ? (fabs(val[e]) >= r[0]) : 1;
    strong[e] = st;
    if (!adm) return;
    if (!st) { adm[e] = 0; return; }
    const double s0 = r[2];
    double worst = 0.0;
    for (int k = 0; k < K; k++) {
        const double s1 = r[3 + k], s2 = r[3 + K + k], xs = xv[k];
        const double s11 = __dmul_rn(s1, s1);
        const double relaxed = __dmul_rn(0.5, __dsub_rn(s2, __ddiv_rn(s11, s0)));
        const double forced = __dmul_rn(0.5, __dadd_rn(__dsub_rn(__dmul_rn(__dmul_rn(xs, xs), s0),
                                                                 __dmul_rn(__dmul_rn(2.0, xs), s1)),
                                                       s2));
        const double scale = __dmul_rn(0.5, __dadd_rn(fabs(s2), __ddiv_rn(s11, fabs(s0))));
        const double lim = __dmul_rn(eps, scale);
        double q;
        if (relaxed <= lim) q = (forced <= lim) ? 1.0 : CUDART_INF;
        else q = __ddiv_rn(forced, relaxed);
        worst = (worst < q) ? q : worst;
    }
    adm[e] = worst <= Q ? 1 : 0;
}

// Caliber-1 aggregation (Section 2) on the GPU, with exactly the result of the sequential pass
// (nodes visited in ascending order; an undecided node joins the admissible strong neighbour of
// largest affinity, ties to the lower index, among seeds and undecided nodes; a chosen undecided
// node becomes a seed). In that pass node u's decision depends only on the decisions of its
// lower-numbered neighbours: u is skipped iff one of them chose u (it is already a seed), and a
// lower-numbered neighbour s is a candidate iff s did not join anyone, while a higher-numbered
// neighbour is not yet visited, so never an associate, and always a candidate if admissible.
// Deciding u as soon as every lower-numbered neighbour is decided (Kahn's order on the DAG of
// lower-to-higher edges) therefore reproduces the pass exactly, in as many parallel rounds as
// the longest index-decreasing path.
//   choice[u]: -2 pending, -1 decided without joining (a seed: chosen by an earlier node or
//   left over), s >= 0 joined s.
__global__ void k_agg_init(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           int32_t *cnt, int32_t *choice, int32_t *front, int32_t *fsize) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int32_t c = 0;
    for (int64_t e = rp[u]; e < rp[u + 1] && ci[e] < u; e++) c++;   // columns ascending
    cnt[u] = c;
    choice[u] = -2;
    if (c == 0) front[atomicAdd(fsize, 1)] = (int32_t)u;
}

__global__ void k_agg_round(const int32_t *__restrict__ front, const int32_t *__restrict__ fsize,
                            const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ aff, const uint8_t *__restrict__ adm, int32_t *cnt,
                            int32_t *choice, int32_t *next, int32_t *nsize) {
    const int32_t t = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (t >= *fsize) return;
    const int32_t u = front[t];
    const int64_t e0 = rp[u], e1 = rp[u + 1];
    bool skipped = false;
    for (int64_t e = e0; e < e1 && ci[e] < u; e++)
        if (choice[ci[e]] == u) skipped = true;
    int32_t best = -1;
    if (!skipped) {
        double bestc = -1.0;
        for (int64_t e = e0; e < e1; e++) {
            const int32_t s = ci[e];
            if (!adm[e] || (s < u && choice[s] >= 0)) continue;
            const double c = aff[e];
            if (c > bestc || (c == bestc && s < best)) { bestc = c; best = s; }
        }
    }
    choice[u] = best;
    for (int64_t e = e1 - 1; e >= e0 && ci[e] > u; e--)
        if (atomicSub(&cnt[ci[e]], 1) == 1) next[atomicAdd(nsize, 1)] = ci[e];
}

// Galerkin coarse operator P^T A P (Section 2), row a by one thread, in the host's order: u
// over the fine rows of aggregate a ascending (P_ua = pa), v over u's diagonal then u's
// entries in stored order, b over v's row of P; each product (pa * A_uv) * P_vb is rounded
// twice and added to entry b (starting from 0.0), all explicitly rounded. The row's entries are
// kept sorted by column in shared memory ([slot][thread], conflict-free), up to GAL_CAP of
// them; a row with more is left to the host (len = -1). Pass 1 (WRITE = false) stores the
// number of nonzero off-diagonal entries of each row, pass 2 writes them at orp[a] in ascending
// column order with the diagonal.
constexpr int GAL_BS = 32;

__device__ __forceinline__ int gal_prow(int32_t v, const int32_t *__restrict__ agg, const int32_t *__restrict__ agg2,
                                        const double *__restrict__ wt, int32_t *c, double *p) {
    if (agg2[v] < 0) { c[0] = agg[v]; p[0] = 1.0; return 1; }
    const double w = wt[v];
    int k = 0;
    if (w != 0.0) { c[k] = agg[v]; p[k] = w; k++; }
    c[k] = agg2[v];
    p[k] = __dsub_rn(1.0, w);
    return k + 1;
}

// add x to entry j of thread t's row; false when the row holds GAL_CAP entries and j is new
__device__ __forceinline__ bool gal_add(int32_t (*key)[GAL_BS], double (*acc)[GAL_BS], int t, int &cnt, int32_t j,
                                        double x) {
    int lo = 0, hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key[mid][t] < j) lo = mid + 1;
        else hi = mid;
    }
    if (lo < cnt && key[lo][t] == j) {
        acc[lo][t] = __dadd_rn(acc[lo][t], x);
        return true;
    }
    if (cnt == GAL_CAP) return false;
    for (int k = cnt; k > lo; k--) {
        key[k][t] = key[k - 1][t];
        acc[k][t] = acc[k - 1][t];
    }
    key[lo][t] = j;
    acc[lo][t] = __dadd_rn(0.0, x);
    cnt++;
    return true;
}

// the products pv * P_vb of one term pv = pa * A_uv over v's row of P
__device__ __forceinline__ bool gal_term(int32_t (*key)[GAL_BS], double (*acc)[GAL_BS], int t, int &cnt, int32_t v,
                                         double pv, const int32_t *__restrict__ agg,
                                         const int32_t *__restrict__ agg2, const double *__restrict__ wt) {
    int32_t c[2];
    double p[2];
    const int k = gal_prow(v, agg, agg2, wt, c, p);
    for (int s = 0; s < k; s++)
        if (!gal_add(key, acc, t, cnt, c[s], __dmul_rn(pv, p[s]))) return false;
    return true;
}

template <bool WRITE>
__global__ void __launch_bounds__(GAL_BS) k_galerkin(
    int64_t nc, const int64_t *__restrict__ ptr, const int32_t *__restrict__ rows, const double *__restrict__ pw,
    const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ val,
    const double *__restrict__ diag, const int32_t *__restrict__ agg, const int32_t *__restrict__ agg2,
    const double *__restrict__ wt, int32_t *__restrict__ len, const int64_t *__restrict__ orp,
    int32_t *__restrict__ oci, double *__restrict__ oval, double *__restrict__ odiag) {
    __shared__ int32_t key[GAL_CAP][GAL_BS];
    __shared__ double acc[GAL_CAP][GAL_BS];
    const int t = threadIdx.x;
    const int64_t a = (int64_t)blockIdx.x * GAL_BS + t;
    if (a >= nc) return;
    if (WRITE && len[a] < 0) return;
    int cnt = 0;
    bool ok = true;
    for (int64_t q = ptr[a]; q < ptr[a + 1] && ok; q++) {
        const int32_t u = rows[q];
        const double pa = pw[q];
        ok = gal_term(key, acc, t, cnt, u, __dmul_rn(pa, diag[u]), agg, agg2, wt);  // the diagonal
        for (int64_t e = rp[u]; e < rp[u + 1] && ok; e++)
            ok = gal_term(key, acc, t, cnt, ci[e], __dmul_rn(pa, val[e]), agg, agg2, wt);
    }
    if (!WRITE) {
        int m = 0;
        for (int k = 0; k < cnt; k++)
            if (key[k][t] != (int32_t)a && acc[k][t] != 0.0) m++;
        len[a] = ok ? m : -1;
        return;
    }
    int64_t o = orp[a];
    double d = 0.0;
    for (int k = 0; k < cnt; k++) {
        if (key[k][t] == (int32_t)a) { d = acc[k][t]; continue; }
        if (acc[k][t] == 0.0) continue;
        oci[o] = key[k][t];
        oval[o] = acc[k][t];
        o++;
    }
    odiag[a] = d;
}

// Exact Schur complement onto C (Eq. 2), row i (node u = cnode[i]) by one thread in the host's
// order: u's entries in stored order; a C neighbour v adds A_uv to entry cidx[v], an F neighbour
// v subtracts (A_uv A_vt) / A_vv (rounded twice) for each of its entries t, from the diagonal
// when t = u, else from entry cidx[t]. Same accumulator and two passes as k_galerkin (a - b is
// a + (-b) exactly, so subtracting through the accumulator's addition keeps the host's bits).
template <bool WRITE>
__global__ void __launch_bounds__(GAL_BS) k_schur(
    int64_t nc, const int32_t *__restrict__ cnode, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
    const double *__restrict__ val, const double *__restrict__ diag, const uint8_t *__restrict__ inF,
    const int32_t *__restrict__ cidx, int32_t *__restrict__ len, const int64_t *__restrict__ orp,
    int32_t *__restrict__ oci, double *__restrict__ oval, double *__restrict__ odiag) {
    __shared__ int32_t key[GAL_CAP][GAL_BS];
    __shared__ double acc[GAL_CAP][GAL_BS];
    const int t = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * GAL_BS + t;
    if (i >= nc) return;
    if (WRITE && len[i] < 0) return;
    const int32_t u = cnode[i];
    double d = diag[u];
    int cnt = 0;
    bool ok = true;
    for (int64_t e = rp[u]; e < rp[u + 1] && ok; e++) {
        const int32_t v = ci[e];
        if (!inF[v]) {
            ok = gal_add(key, acc, t, cnt, cidx[v], val[e]);
            continue;
        }
        const double avv = diag[v], auv = val[e];
        for (int64_t f = rp[v]; f < rp[v + 1] && ok; f++) {
            const int32_t w = ci[f];
            const double term = __ddiv_rn(__dmul_rn(auv, val[f]), avv);
            if (w == u) d = __dsub_rn(d, term);
            else ok = gal_add(key, acc, t, cnt, cidx[w], -term);
        }
    }
    if (!WRITE) {
        int m = 0;
        for (int k = 0; k < cnt; k++)
            if (acc[k][t] != 0.0) m++;
        len[i] = ok ? m : -1;
        return;
    }
    int64_t o = orp[i];
    for (int k = 0; k < cnt; k++) {
        if (acc[k][t] == 0.0) continue;
        oci[o] = key[k][t];
        oval[o] = acc[k][t];
        o++;
    }
    odiag[i] = d;
}

// Input checks of a graph (Eq. 1 needs a symmetric, positive weighting), one thread per stored
// entry e of row u: 0 <= v < n, v != u, columns strictly ascending in the row, w finite and
// positive, and u present in v's row with the same weight. The caller has checked that rp
// starts at 0 and never decreases, so every index formed here is in range; v is used as a row
// only once it is known to be in range. Any failure sets *bad.
__global__ void k_validate(int64_t n, int64_t z, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ w, int *bad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= z) return;
    int64_t lo = 0, hi = n - 1;  // the row u with rp[u] <= e < rp[u + 1]
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    const int64_t u = lo;
    const int32_t v = ci[e];
    const double we = w[e];
    bool ok = v >= 0 && v < n && v != u && we > 0.0 && isfinite(we) && (e == rp[u] || v > ci[e - 1]);
    if (ok) {
        int64_t a = rp[v], b = rp[v + 1];
        const int64_t end = b;
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if (ci[mid] < u) a = mid + 1;
            else b = mid;
        }
        ok = a < end && ci[a] == u && w[a] == we;
    }
    if (!ok) atomicOr(bad, 1);
}

static inline unsigned nblk(int64_t work, int bs) { return (unsigned)((work + bs - 1) / bs); }

// Upload a level operator (natural order) and run K9 (and K10 when aff != nullptr). Everything is
// ordered on a private stream with stream-ordered allocations, so a setup running on a host
// thread never synchronises the whole device (solves of other hierarchies keep running).
static int run_setup_kernels(const HostMat &A, const std::vector<int32_t> *colour, int level,
                             uint64_t seed, int K, int nu, double tau, int veto, double *X,
                             const double *Xin, double *aff, uint8_t *strong, double Q = 0.0,
                             double eps = 0.0, uint8_t *adm = nullptr, int order = LAMG_TV_STRIDED,
                             int32_t *choice = nullptr, int *rounds = nullptr) {
    int rc = LAMG_OK;
    const int64_t n = A.n, z = A.nnz();
    int64_t *d_rp = nullptr;
    int32_t *d_ci = nullptr, *d_rows = nullptr;
    double *d_val = nullptr, *d_diag = nullptr, *d_X = nullptr, *d_aff = nullptr, *d_rs = nullptr;
    uint8_t *d_strong = nullptr, *d_adm = nullptr;
    int32_t *d_agg = nullptr;
    const int bs = 128;
    cudaStream_t st = nullptr;
    std::vector<int32_t> rows;
    std::vector<int64_t> cptr, lptr;
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
        // rows grouped by colour; within a colour the rows summed in stored order, then (with
        // LAMG_TV_STRIDED) the rows of more than TV_STRIDE entries (from lptr[c]), each group
        // ascending
        auto short_row = [&](int64_t u) { return order == LAMG_TV_STORED || A.rp[u + 1] - A.rp[u] <= TV_STRIDE; };
        for (int32_t c : *colour) ncol = std::max(ncol, c + 1);
        cptr.assign(ncol + 1, 0);
        lptr.assign(ncol, 0);
        for (int32_t c : *colour) cptr[c + 1]++;
        for (int c = 0; c < ncol; c++) cptr[c + 1] += cptr[c];
        for (int64_t u = 0; u < n; u++)
            if (short_row(u)) lptr[(*colour)[u]]++;
        for (int c = 0; c < ncol; c++) lptr[c] += cptr[c];
        rows.resize(n);
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1), lfill(lptr);
        for (int64_t u = 0; u < n; u++) {
            const int32_t c = (*colour)[u];
            if (short_row(u)) rows[fill[c]++] = (int32_t)u;
            else rows[lfill[c]++] = (int32_t)u;
        }
        CK(cudaMallocAsync((void **)&d_rows, n * sizeof(int32_t), st));
        CK(cudaMemcpyAsync(d_rows, rows.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        k_tv_start<<<nblk(n * K, bs), bs, 0, st>>>(n, K, seed, level, d_X);
        for (int s = 0; s < nu; s++) {
            for (int c = 0; c < ncol; c++) {
                const int64_t cnt = lptr[c] - cptr[c], lcnt = cptr[c + 1] - lptr[c];
                if (cnt) {
                    if (K == 4)
                        k_tv_colour<4><<<nblk(cnt, bs), bs, 0, st>>>(cnt, d_rows + cptr[c], d_rp, d_ci, d_val, d_diag, d_X);
                    else
                        k_tv_colour_any<<<nblk(cnt, bs), bs, 0, st>>>(K, cnt, d_rows + cptr[c], d_rp, d_ci, d_val, d_diag,
                                                                    d_X);
                }
                if (lcnt)
                    k_tv_long<<<nblk(32 * lcnt, bs), bs, 0, st>>>(K, lcnt, d_rows + lptr[c], d_rp, d_ci, d_val, d_diag,
                                                                 d_X);
            }
        }
        CK(cudaGetLastError());
        if (X) CK(cudaMemcpyAsync(X, d_X, n * K * sizeof(double), cudaMemcpyDeviceToHost, st));
    } else {
        CK(cudaMemcpyAsync(d_X, Xin, n * K * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    if (aff) {
        const bool moments = adm && K <= GUARD_KMAX;
        CK(cudaMallocAsync((void **)&d_aff, (z ? z : 1) * sizeof(double), st));
        CK(cudaMallocAsync((void **)&d_strong, (z ? z : 1), st));
        CK(cudaMallocAsync((void **)&d_rs, n * (3 + 2 * K) * sizeof(double), st));
        if (moments) CK(cudaMallocAsync((void **)&d_adm, (z ? z : 1), st));
        k_row_stats<<<nblk(n, bs), bs, 0, st>>>(n, K, tau, moments ? 1 : 0, d_rp, d_ci, d_val, d_X, d_rs);
        if (z)
            k_entry_affinity<<<nblk(z, 256), 256, 0, st>>>(n, z, K, veto, Q, eps, d_rp, d_ci, d_val, d_X, d_rs, d_aff,
                                                           d_strong, moments ? d_adm : nullptr);
        CK(cudaGetLastError());
        if (z) CK(cudaMemcpyAsync(aff, d_aff, z * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (z) CK(cudaMemcpyAsync(strong, d_strong, z, cudaMemcpyDeviceToHost, st));
        if (moments && z) CK(cudaMemcpyAsync(adm, d_adm, z, cudaMemcpyDeviceToHost, st));
        if (choice && moments) {
            // the aggregation pass in dependency order (k_agg_round), one launch per round; the
            // host reads the next frontier's size between rounds
            CK(cudaMallocAsync((void **)&d_agg, (4 * n + 2) * sizeof(int32_t), st));
            int32_t *cnt = d_agg, *dch = d_agg + n, *fa = d_agg + 2 * n, *fb = d_agg + 3 * n, *sz = d_agg + 4 * n;
            int32_t *h_sz = nullptr;
            CK(cudaHostAlloc((void **)&h_sz, sizeof(int32_t), cudaHostAllocDefault));
            CK(cudaMemsetAsync(sz, 0, 2 * sizeof(int32_t), st));
            k_agg_init<<<nblk(n, bs), bs, 0, st>>>(n, d_rp, d_ci, cnt, dch, fa, sz);
            CK(cudaMemcpyAsync(h_sz, sz, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            int64_t left = n, r = 0;
            int cur = 0;
            while (*h_sz > 0 && left > 0) {
                const int32_t fn = *h_sz;
                left -= fn;
                int32_t *fin = cur ? fb : fa, *fout = cur ? fa : fb;
                CK(cudaMemsetAsync(sz + 1 - cur, 0, sizeof(int32_t), st));
                k_agg_round<<<nblk(fn, bs), bs, 0, st>>>(fin, sz + cur, d_rp, d_ci, d_aff, d_adm, cnt, dch, fout,
                                                         sz + 1 - cur);
                CK(cudaMemcpyAsync(h_sz, sz + 1 - cur, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                cur = 1 - cur;
                r++;
            }
            cudaFreeHost(h_sz);
            if (left != 0) { rc = LAMG_ERR_SETUP; goto out; }   // every node is reached: an invariant
            CK(cudaMemcpyAsync(choice, dch, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            if (rounds) *rounds = (int)r;
        }
    }
    CK(cudaStreamSynchronize(st));
out:
    if (st) {
        void *ptrs[] = {d_rp, d_ci, d_val, d_diag, d_X, d_rows, d_aff, d_strong, d_adm, d_rs, d_agg};
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

int gpu_galerkin(const HostLevel &L, const std::vector<int64_t> &ptr, const std::vector<int32_t> &rows,
                 const std::vector<double> &pw, HostMat &Ac,
                 const GalerkinHostRows &host_rows) {
    int rc = LAMG_OK;
    const HostMat &A = L.A;
    const int64_t n = A.n, z = A.nnz(), nc = L.nc, np = ptr[nc];
    int64_t *d_rp = nullptr, *d_ptr = nullptr, *d_orp = nullptr;
    int32_t *d_ci = nullptr, *d_agg = nullptr, *d_agg2 = nullptr, *d_rows = nullptr, *d_len = nullptr,
            *d_oci = nullptr;
    double *d_val = nullptr, *d_diag = nullptr, *d_wt = nullptr, *d_pw = nullptr, *d_oval = nullptr,
           *d_odiag = nullptr;
    cudaStream_t st = nullptr;
    std::vector<int32_t> len(nc);
    std::vector<int64_t> big;
    std::vector<std::vector<int32_t>> bcol;
    std::vector<std::vector<double>> bval;
    std::vector<double> bdiag;
    int64_t tot = 0;
    if ((int64_t)L.agg.size() != n || (int64_t)L.agg2.size() != n || (int64_t)L.wt.size() != n)
        return LAMG_ERR_INVALID;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaMallocAsync((void **)&d_rp, (n + 1) * sizeof(int64_t), st));
    CK(cudaMallocAsync((void **)&d_ci, (z ? z : 1) * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_val, (z ? z : 1) * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_diag, n * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_agg, n * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_agg2, n * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_wt, n * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_ptr, (nc + 1) * sizeof(int64_t), st));
    CK(cudaMallocAsync((void **)&d_rows, (np ? np : 1) * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_pw, (np ? np : 1) * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_len, nc * sizeof(int32_t), st));
    CK(cudaMemcpyAsync(d_rp, A.rp.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (z) CK(cudaMemcpyAsync(d_ci, A.ci.data(), z * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (z) CK(cudaMemcpyAsync(d_val, A.val.data(), z * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_diag, A.diag.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_agg, L.agg.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_agg2, L.agg2.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_wt, L.wt.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_ptr, ptr.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (np) CK(cudaMemcpyAsync(d_rows, rows.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (np) CK(cudaMemcpyAsync(d_pw, pw.data(), np * sizeof(double), cudaMemcpyHostToDevice, st));
    k_galerkin<false><<<nblk(nc, GAL_BS), GAL_BS, 0, st>>>(nc, d_ptr, d_rows, d_pw, d_rp, d_ci, d_val, d_diag, d_agg,
                                                            d_agg2, d_wt, d_len, nullptr, nullptr, nullptr, nullptr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(len.data(), d_len, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // rows with more distinct columns than the GPU accumulator holds: summed on the host
    for (int64_t a = 0; a < nc; a++)
        if (len[a] < 0) big.push_back(a);
    bcol.resize(big.size());
    bval.resize(big.size());
    bdiag.resize(big.size());
    host_rows(big, bcol, bval, bdiag);
    for (size_t i = 0; i < big.size(); i++) len[big[i]] = (int32_t)bcol[i].size();
    Ac.n = nc;
    Ac.rp.assign(nc + 1, 0);
    for (int64_t a = 0; a < nc; a++) Ac.rp[a + 1] = Ac.rp[a] + len[a];
    tot = Ac.rp[nc];
    Ac.ci.resize(tot);
    Ac.val.resize(tot);
    Ac.diag.assign(nc, 0.0);
    CK(cudaMallocAsync((void **)&d_orp, (nc + 1) * sizeof(int64_t), st));
    CK(cudaMallocAsync((void **)&d_oci, (tot ? tot : 1) * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_oval, (tot ? tot : 1) * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_odiag, nc * sizeof(double), st));
    CK(cudaMemcpyAsync(d_orp, Ac.rp.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    k_galerkin<true><<<nblk(nc, GAL_BS), GAL_BS, 0, st>>>(nc, d_ptr, d_rows, d_pw, d_rp, d_ci, d_val, d_diag, d_agg,
                                                           d_agg2, d_wt, d_len, d_orp, d_oci, d_oval, d_odiag);
    CK(cudaGetLastError());
    if (tot) CK(cudaMemcpyAsync(Ac.ci.data(), d_oci, tot * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (tot) CK(cudaMemcpyAsync(Ac.val.data(), d_oval, tot * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(Ac.diag.data(), d_odiag, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < big.size(); i++) {
        const int64_t a = big[i];
        std::copy(bcol[i].begin(), bcol[i].end(), Ac.ci.begin() + Ac.rp[a]);
        std::copy(bval[i].begin(), bval[i].end(), Ac.val.begin() + Ac.rp[a]);
        Ac.diag[a] = bdiag[i];
    }
out:
    if (st) {
        void *ptrs[] = {d_rp, d_ci, d_val, d_diag, d_agg, d_agg2, d_wt, d_ptr, d_rows, d_pw, d_len,
                        d_orp, d_oci, d_oval, d_odiag};
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

int gpu_schur(const HostMat &A, const std::vector<uint8_t> &inF, const std::vector<int32_t> &cidx,
              const std::vector<int32_t> &cnode, HostMat &Ac, const GalerkinHostRows &host_rows) {
    int rc = LAMG_OK;
    const int64_t n = A.n, z = A.nnz(), nc = (int64_t)cnode.size();
    int64_t *d_rp = nullptr, *d_orp = nullptr;
    int32_t *d_ci = nullptr, *d_cidx = nullptr, *d_cnode = nullptr, *d_len = nullptr, *d_oci = nullptr;
    uint8_t *d_inF = nullptr;
    double *d_val = nullptr, *d_diag = nullptr, *d_oval = nullptr, *d_odiag = nullptr;
    cudaStream_t st = nullptr;
    std::vector<int32_t> len(nc);
    std::vector<int64_t> big;
    std::vector<std::vector<int32_t>> bcol;
    std::vector<std::vector<double>> bval;
    std::vector<double> bdiag;
    int64_t tot = 0;
    if ((int64_t)inF.size() != n || (int64_t)cidx.size() != n) return LAMG_ERR_INVALID;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaMallocAsync((void **)&d_rp, (n + 1) * sizeof(int64_t), st));
    CK(cudaMallocAsync((void **)&d_ci, (z ? z : 1) * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_val, (z ? z : 1) * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_diag, n * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_inF, n, st));
    CK(cudaMallocAsync((void **)&d_cidx, n * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_cnode, (nc ? nc : 1) * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_len, (nc ? nc : 1) * sizeof(int32_t), st));
    CK(cudaMemcpyAsync(d_rp, A.rp.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (z) CK(cudaMemcpyAsync(d_ci, A.ci.data(), z * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (z) CK(cudaMemcpyAsync(d_val, A.val.data(), z * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_diag, A.diag.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_inF, inF.data(), n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_cidx, cidx.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (nc) CK(cudaMemcpyAsync(d_cnode, cnode.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (nc) {
        k_schur<false><<<nblk(nc, GAL_BS), GAL_BS, 0, st>>>(nc, d_cnode, d_rp, d_ci, d_val, d_diag, d_inF, d_cidx,
                                                             d_len, nullptr, nullptr, nullptr, nullptr);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(len.data(), d_len, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    // rows with more distinct columns than the GPU accumulator holds: summed on the host
    for (int64_t a = 0; a < nc; a++)
        if (len[a] < 0) big.push_back(a);
    bcol.resize(big.size());
    bval.resize(big.size());
    bdiag.resize(big.size());
    host_rows(big, bcol, bval, bdiag);
    for (size_t i = 0; i < big.size(); i++) len[big[i]] = (int32_t)bcol[i].size();
    Ac.n = nc;
    Ac.rp.assign(nc + 1, 0);
    for (int64_t a = 0; a < nc; a++) Ac.rp[a + 1] = Ac.rp[a] + len[a];
    tot = Ac.rp[nc];
    Ac.ci.resize(tot);
    Ac.val.resize(tot);
    Ac.diag.assign(nc, 0.0);
    if (nc) {
        CK(cudaMallocAsync((void **)&d_orp, (nc + 1) * sizeof(int64_t), st));
        CK(cudaMallocAsync((void **)&d_oci, (tot ? tot : 1) * sizeof(int32_t), st));
        CK(cudaMallocAsync((void **)&d_oval, (tot ? tot : 1) * sizeof(double), st));
        CK(cudaMallocAsync((void **)&d_odiag, nc * sizeof(double), st));
        CK(cudaMemcpyAsync(d_orp, Ac.rp.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        k_schur<true><<<nblk(nc, GAL_BS), GAL_BS, 0, st>>>(nc, d_cnode, d_rp, d_ci, d_val, d_diag, d_inF, d_cidx,
                                                            d_len, d_orp, d_oci, d_oval, d_odiag);
        CK(cudaGetLastError());
        if (tot) CK(cudaMemcpyAsync(Ac.ci.data(), d_oci, tot * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if (tot) CK(cudaMemcpyAsync(Ac.val.data(), d_oval, tot * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(Ac.diag.data(), d_odiag, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < big.size(); i++) {
        const int64_t a = big[i];
        std::copy(bcol[i].begin(), bcol[i].end(), Ac.ci.begin() + Ac.rp[a]);
        std::copy(bval[i].begin(), bval[i].end(), Ac.val.begin() + Ac.rp[a]);
        Ac.diag[a] = bdiag[i];
    }
out:
    if (st) {
        void *ptrs[] = {d_rp, d_ci, d_val, d_diag, d_inF, d_cidx, d_cnode, d_len, d_orp, d_oci, d_oval, d_odiag};
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

int gpu_validate_entries(const lamg_graph *g, bool *valid) {
    int rc = LAMG_OK;
    const int64_t n = g->n, z = g->rp[n];
    int64_t *d_rp = nullptr;
    int32_t *d_ci = nullptr;
    double *d_w = nullptr;
    int *d_bad = nullptr;
    int bad = 0;
    cudaStream_t st = nullptr;
    *valid = false;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaMallocAsync((void **)&d_rp, (n + 1) * sizeof(int64_t), st));
    CK(cudaMallocAsync((void **)&d_ci, (z ? z : 1) * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_w, (z ? z : 1) * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_bad, sizeof(int), st));
    CK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    CK(cudaMemcpyAsync(d_rp, g->rp, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (z) CK(cudaMemcpyAsync(d_ci, g->ci, z * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (z) CK(cudaMemcpyAsync(d_w, g->w, z * sizeof(double), cudaMemcpyHostToDevice, st));
    if (z) k_validate<<<nblk(z, 256), 256, 0, st>>>(n, z, d_rp, d_ci, d_w, d_bad);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *valid = bad == 0;
out:
    if (st) {
        void *ptrs[] = {d_rp, d_ci, d_w, d_bad};
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

int gpu_testvectors(const HostMat &A, const std::vector<int32_t> &colour, int level,
                    uint64_t seed, int K, int nu, double *X, int order) {
    return run_setup_kernels(A, &colour, level, seed, K, nu, 0.0, 1, X, nullptr, nullptr, nullptr, 0.0, 0.0,
                             nullptr, order);
}

int gpu_affinity(const HostMat &A, const double *X, int K, double tau, double *aff,
                 uint8_t *strong) {
    return run_setup_kernels(A, nullptr, 0, 0, K, 0, tau, 1, nullptr, X, aff, strong);
}

int gpu_tv_and_affinity(const HostMat &A, const std::vector<int32_t> &colour, int level,
                        uint64_t seed, int K, int nu, double tau, int veto, double *X,
                        double *aff, uint8_t *strong, double Q, double eps, uint8_t *adm, int order,
                        int32_t *choice, int *rounds) {
    return run_setup_kernels(A, &colour, level, seed, K, nu, tau, veto, X, nullptr, aff, strong, Q, eps, adm,
                             order, choice, rounds);
}

}  // namespace lamg
