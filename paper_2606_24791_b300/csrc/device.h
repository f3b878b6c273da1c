// Device-side hierarchy layout and the kernel launchers shared by the solver.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace lamg {

// One level in device order. Device order of a level:
//  - aggregation level: rows grouped by Gauss-Seidel colour (colour 0 first), ascending
//    natural id within a colour, so each colour class is a contiguous row range;
//  - elimination level: the kept (C) nodes first, in the next level's device order, then
//    the eliminated (F) nodes in ascending natural id. The first nc entries of the level's
//    iterate are therefore the next level's iterate, and share its memory;
//  - coarsest level: natural order.
struct DevLevel {
    int kind = 0;
    int64_t n = 0, nnz = 0, nc = 0, nF = 0;
    int ncol = 0;
    int tpr = 1;                  // threads per row of the CSR kernels
    std::vector<int64_t> cptr;    // colour class row ranges (aggregation)
    std::vector<int32_t> perm;    // device index -> natural id

    // operator: off-diagonal CSR + diagonal and its reciprocal (FP64), int32 row pointers
    int32_t *rp = nullptr, *ci = nullptr;
    double *val = nullptr, *diag = nullptr, *idiag = nullptr;
    // the same off-diagonal entries as sliced ELLPACK (sell = 1) in four-entry blocks: see
    // sell_col_at / sell_val_at
    int sell = 0;
    int64_t sell_nnz = 0;
    // rows with more than LONG_ROW off-diagonal entries, summed by a whole thread block: their
    // device indices (ascending) and, per colour class, the offsets into that list (an
    // aggregation level's long rows are the first rows of their class)
    int32_t *lrows = nullptr;
    int64_t nlong = 0;
    std::vector<int64_t> lptr;
    // kernel form of the colour-class sweep (gs_tpr) and of the residual-type passes (rs_tpr:
    // residual, A p with its dot product, true residual): 0 one thread per row on the sliced
    // copy, else that many lanes per CSR row; set by rule and refined by timing at setup
    int gs_tpr = 1, rs_tpr = 1;
    // Chebyshev smoothing (levels with many colours): coefficients of each step, the second
    // iterate buffer and the step direction
    int cheb = 0, cheb_m = 0;    // Chebyshev smoothing on this level, polynomial degree
    double cheb_c1[8] = {0}, cheb_c2[8] = {0};
    double *t = nullptr, *d = nullptr;
    int32_t *sl_ptr = nullptr, *sl_col = nullptr;
    double *sl_val = nullptr;
    // aggregation: P rows (coarse device ids) and P^T as CSR over coarse rows
    int32_t *agg = nullptr, *agg2 = nullptr;
    double *wt = nullptr;
    int32_t *pt_ptr = nullptr, *pt_row = nullptr;
    double *pt_w = nullptr;
    int pt_tpr = 1;
    // elimination: F rows as ELL-4 (coarse columns < nc, -1 padding), P_F^T over C rows; for
    // the multi-column kernels also 1 / A_FF and the C rows with more than LONG_ROW F entries
    int32_t *pf_col = nullptr;
    double *pf_val = nullptr, *dF = nullptr, *idF = nullptr;
    int32_t *pft_ptr = nullptr, *pft_f = nullptr, *pft_long = nullptr;
    double *pft_val = nullptr;
    int64_t npft_long = 0;
    // coarsest: dense pseudo-inverse, row-major
    double *pinv = nullptr;
    // iterate, right-hand side, residual
    double *x = nullptr, *b = nullptr, *r = nullptr;
    size_t bytes = 0;
};

enum OpKind {
    OP_GS_FIRST,      // colour-0 rows x = b / d, every other row x = 0 (first visit, x == 0)
    OP_GS,            // one colour class of a Gauss-Seidel sweep
    OP_ZERO,          // x = 0 (first visit without pre-smoothing)
    OP_RESID,         // r = b - A x
    OP_RESTRICT,      // b_{l+1} = P^T r
    OP_PROLONG,       // x += P x_{l+1}
    OP_ELIM_RESTRICT, // b_{l+1} = b_C + P_F^T b_F
    OP_ELIM_INTERP,   // x_F = P_F x_C + b_F / d_F
    OP_COARSE,        // x = A^+ b, then the mean-zero projection
    OP_CHEB,          // step `colour` of the Chebyshev smoothing polynomial (x <-> t alternate)
    OP_CHEB_COPY,     // x = t (after a polynomial of odd degree)
    OP_CHEB_FIRST,    // the first Chebyshev step from x == 0 (first visit): no product with A,
                      // out = c2[0] b / d into x (degree 1) or into t and d (degree > 1)
};

struct Op {
    int kind;
    int level;
    int colour;
};

// Reduction workspace: per-block partial sums, a completion ticket, device scalars.
constexpr int RED_MAXG = 1184;   // 148 SMs x 8 blocks
constexpr int RED_NV = 4;
enum Scalar { S_RZ = 0, S_PQ, S_ALPHA, S_BETA, S_RR, S_BN2, S_MEAN, S_TRUE_RR, S_BMEAN, S_ITERS, S_COUNT = 16 };

struct Reduce {
    double *partials = nullptr;   // RED_NV x RED_MAXG
    unsigned *ticket = nullptr;
    double *scal = nullptr;       // S_COUNT
};

// Sliced ELLPACK in four-entry blocks. Rows come in slices of 32; every row of slice s is
// padded to the slice's width w (its longest row rounded up to a multiple of 4) with value 0 at
// the row's own column (the last row for the slots past n), and the slice occupies 32 w slots
// from sl_ptr[s]. Entry j of row 32 s + l: column id at sell_col_at, value at sell_val_at, so a
// lane reads its row's ids four at a time (one 16-byte int4) and its values two at a time (one
// 16-byte double2), and each such load of a warp covers 512 contiguous bytes.
__host__ __device__ inline int64_t sell_col_at(int64_t base, int l, int j) { return base + 128 * (j >> 2) + 4 * l + (j & 3); }
__host__ __device__ inline int64_t sell_val_at(int64_t base, int l, int j) { return base + 64 * (j >> 1) + 2 * l + (j & 1); }
constexpr int SELL_MAX_ROW = 64;   // longer rows keep the level on the lane-group CSR kernels
constexpr int LONG_ROW = 256;      // longer rows are summed by a whole thread block

// Plain-data view of a level for the persistent and cluster kernels (device pointers only).
struct PLevel {
    int kind, n, nc, nF, ncol, tpr, pt_tpr, cptr_off;  // colour offsets at cptr_all + cptr_off
    int gs_tpr, rs_tpr;                                 // as in DevLevel (0: sliced ELLPACK)
    const int32_t *rp, *ci;
    const double *val, *diag, *idiag;
    const int32_t *sl_ptr, *sl_col;
    const double *sl_val;
    const int32_t *agg, *agg2;
    const double *wt;
    const int32_t *pt_ptr, *pt_row;
    const double *pt_w;
    const int32_t *pf_col;
    const double *pf_val, *dF;
    const int32_t *pft_ptr, *pft_f;
    const double *pft_val;
    const double *pinv;
    double *x, *b, *r;
};

// Grid barrier state: arrival count, generation, failure flag.
struct GridBar {
    unsigned count, gen, err, pad;
};

struct PSolve {
    int nlev, nops, n0, ncptr;
    const PLevel *lv;
    const Op *ops;
    const int32_t *tail_end;      // per op: end of the single-CTA segment starting here, or -1
    const int32_t *cptr_all;      // concatenated colour offsets of all levels
    const int32_t *perm0;
    double *r, *p, *q, *zold, *xs, *bkeep;
    double *partials;             // 2 x RED_NV x grid
    GridBar *bar;
    double *scal;                 // S_COUNT outputs
    double *hist;                 // relres per iteration
    unsigned long long wait_ns;   // limit of one grid-barrier wait (set per launch)
};

size_t persistent_smem(int nlev, int nops, int ncptr);
int persistent_grid(int device, size_t smem);
constexpr unsigned long long WAIT_NS_DEFAULT = 2000000000ULL;   // 2 s
cudaError_t launch_persistent(const PSolve *P, int grid, size_t smem, int mode, int maxit, double tol,
                              const double *b_in, double *phi_out, cudaStream_t s,
                              unsigned long long *prof = nullptr,
                              unsigned long long wait_ns = WAIT_NS_DEFAULT);

// A whole solve run by one thread-block cluster (lamg_solve_many): device pointers of one
// hierarchy and its right-hand side.
enum { MG_ITERS = 0, MG_RR, MG_BN2, MG_TRUE_RR, MG_BMEAN, MG_OUT = 8 };
constexpr int64_t MANY_MAX_ENTRIES = (int64_t)1 << 19;   // n + off-diagonal entries of level 0
struct MGraph {
    const PLevel *lv;
    const int32_t *cptr;
    const Op *ops;
    const int32_t *perm0;
    int nlev, ncptr, nops, n0;
    int maxit, pad_;
    double tol;
    double *r, *p, *q, *zold, *xs, *bkeep;   // level-0 device order
    const double *b_in;                      // caller order
    double *phi_out;                         // caller order
    double *part;                            // 2 x RED_NV x 16 cluster partial sums
    double *out;                             // MG_OUT results
    double *hist;                            // maxit + 1 relative residuals, or null
};
cudaError_t launch_cluster_solve(const MGraph *g, int G, int cl, size_t smem, cudaStream_t s);

// cluster sub-cycle kernel (cluster.cu)
constexpr int CL_OPS_SMEM = 4096;               // longer step lists are read from global memory
constexpr size_t CL_SMEM_MAX = 160 * 1024;      // dynamic shared memory limit of the kernel
int cluster_dim(int device, size_t smem);   // CTAs per cluster that fit (16, 8, 4) or 0
size_t cluster_smem(int nlev, int ncptr, int nops);
void launch_cluster(const PLevel *lv, int nlev, const int32_t *cptr, int ncptr, const Op *ops, int nops,
                    int cl, bool pdl, cudaStream_t s, unsigned long long *prof = nullptr);
bool pdl_enabled();

// launchers (cycle_kernels.cu)
// start: the first step of the coarse level's first visit (OP_GS_FIRST or OP_ZERO on level + 1)
// when op is a restriction that performs it too (start_fusable), else null
// setup: device-order operator of a level from its natural-order CSR (row i = natural row
// perm[i], columns renamed by iperm, entries in the natural row's order), and its sliced-ELLPACK
// copy from that operator (slice pointers sp, 32-row slices)
void launch_layout_rows(int64_t n, const int32_t *perm, const int32_t *iperm, const int64_t *nrp,
                        const int32_t *nci, const double *nval, const double *ndiag, const int32_t *rp,
                        int32_t *ci, double *val, double *diag, double *idiag, cudaStream_t s);
void launch_layout_sell(int64_t n, int64_t ns, const int32_t *sp, const int32_t *rp, const int32_t *ci,
                        const double *val, int32_t *sc, double *sv, cudaStream_t s);
void launch_op(const Op &op, std::vector<DevLevel> &lv, const Reduce &red, cudaStream_t s,
               const Op *start = nullptr);
void launch_gather(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t s);
void launch_scatter(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t s);
void launch_sum(int64_t n, const double *v, const Reduce &red, cudaStream_t s);  // S_MEAN = sum / n
void launch_sub_mean(int64_t n, double *v, const Reduce &red, cudaStream_t s);
void launch_init_b(int64_t n, double *r, double *bkeep, double *x, double *p, double *zold,
                   const Reduce &red, cudaStream_t s);
void launch_spmv_dot(const DevLevel &L, const double *p, double *q, const Reduce &red, cudaStream_t s);
void launch_update_xr(int64_t n, double *x, double *r, const double *p, const double *q,
                      const Reduce &red, cudaStream_t s);
void launch_proj_dots(int64_t n, double *z, const double *zold, const double *r, const Reduce &red,
                      cudaStream_t s);
void launch_update_p(int64_t n, const double *z, double *p, double *zold, const Reduce &red,
                     cudaStream_t s);
void launch_true_resid(const DevLevel &L, const double *x, const double *b, const Reduce &red,
                       cudaStream_t s);
int choose_tpr(double avg_row);

}  // namespace lamg
