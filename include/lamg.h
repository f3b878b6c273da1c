/*
 * lamg.h - C ABI of the B300 LAMG+ solve-phase library.
 *
 * The library solves the compatible graph-Laplacian system of the paper's Eq. 1,
 *     L phi = b,   1^T phi = 0,   1^T b = 0,   L = D - W,
 * for a connected weighted undirected graph, with a multigrid cycle over a LAMG+ hierarchy
 * (Section 2: low-degree elimination, Eq. 2; guarded caliber-1 aggregation, Eqs. 3-4;
 * strength-of-connection veto, Eq. 9; selective caliber-2 interpolation, Section 3.2 and
 * Eq. 13; Galerkin coarse operators; gamma-cycle work rule, Eq. 5) used as the
 * preconditioner of a flexible conjugate-gradient iteration run in FP64 on the GPU.
 *
 * Conventions shared by every entry point
 *  - All sizes are int64_t, node ids int32_t (n < 2^31), values IEEE binary64 unless stated.
 *  - Graphs are given as symmetric adjacency in CSR: rp[n+1] (row pointers), ci[rp[n]]
 *    (neighbour ids, strictly ascending within a row, no self loops), w[rp[n]] (positive
 *    finite weights, w[u->v] == w[v->u]). The library copies what it needs; the caller keeps
 *    ownership of every array it passes and may free it when the call returns.
 *  - Vectors b and phi are indexed by the caller's node ids. By default they are HOST
 *    pointers; with LAMG_DEVICE_PTRS in the flags they are device pointers on the current
 *    CUDA device, and the work is ordered on the stream given in the options (0: the
 *    library's own stream). The library never frees caller memory.
 *  - Every call returns LAMG_OK or an error code; lamg_strerror() names it. A failed call
 *    leaves its outputs unspecified and its inputs untouched. A hierarchy handle must not be
 *    used from two host threads at once.
 *  - Every GPU wait inside the library is bounded; a wait that runs out returns
 *    LAMG_ERR_TIMEOUT instead of hanging.
 */
#ifndef LAMG_H
#define LAMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LAMG_OK 0
#define LAMG_ERR_INVALID 1        /* asymmetric graph, w <= 0 or NaN, self loop, bad sizes */
#define LAMG_ERR_DISCONNECTED 2   /* the paper assumes a connected graph (Section 1) */
#define LAMG_ERR_SETUP 3          /* coarsening stalled above the dense-coarsest limit */
#define LAMG_ERR_OOM 4            /* a device or host allocation failed */
#define LAMG_ERR_NOT_CONVERGED 5  /* maxit reached; the stats are valid */
#define LAMG_ERR_CUDA 6           /* a CUDA runtime call failed */
#define LAMG_ERR_TIMEOUT 7        /* a bounded GPU wait ran out */
#define LAMG_ERR_ADMISSION 8      /* serving: the request can never fit the memory budget */
#define LAMG_ERR_NO_DEVICE 9      /* no CUDA device is visible */

/* flags */
#define LAMG_DEVICE_PTRS 1u       /* vectors are device pointers */
#define LAMG_PERSISTENT 2u        /* run the whole solve as one persistent cooperative kernel
                                     (grid barriers between steps) instead of the default CUDA
                                     graphs of per-step kernels with programmatic dependent
                                     launch; same arithmetic */

/* cycle precision */
#define LAMG_FP64 0
#define LAMG_FP32 1               /* FP32 cycle inside FP64 CG (outer residual, dots, projection
                                     and coarsest solve stay FP64) */

/* Setup options. lamg_options_default() fills the paper's parameter-free values. */
typedef struct lamg_options {
    int32_t K;             /* test vectors per aggregation level: 4 (Section 3.3) */
    int32_t nu_tv;         /* GS sweeps per test vector: 3 (Section 2) */
    int32_t dmax;          /* elimination degree bound: 4 (Eq. 2) */
    int32_t nu_pre;        /* pre-smoothing sweeps: 1 */
    int32_t nu_post;       /* post-smoothing sweeps: 2 ((1,2) cycle, Appendix A, Table 10) */
    int32_t coarsest_max;  /* a level with at most this many nodes is solved densely; 0 (default):
                              min(4096, max(1024, floor(sqrt(1.5 nnz(L))))) for the input's
                              nnz(L) = n + 2m, so the dense coarsest matrix holds about as many
                              bytes as the input operator */
    int32_t max_levels;    /* 100 */
    int32_t veto;          /* strength-of-connection veto on (1) / off (0), Eq. 9 */
    int32_t caliber2;      /* selective caliber-2 on (1) / off (0), Section 3.2 */
    int32_t precision;     /* LAMG_FP64 or LAMG_FP32 cycle */
    uint64_t seed;         /* test-vector random stream (SplitMix64, counter-based) */
    double Q;              /* energy-ratio guard bound: 2.5 (Eq. 4) */
    double tau_soc;        /* veto threshold: 0.05 (Eq. 9) */
    double elim_min_frac;  /* keep an elimination level while |F| >= this * n: 0.01 */
    double snap;           /* caliber-2 weight snap distance to 0/1: 1e-3 */
    double guard_eps;      /* relative size below which a nodal energy counts as zero: 1e-10 */
    double gamma_fixed;    /* > 0: this cycle index on every aggregation level instead of Eq. 5 */
    int32_t device;        /* CUDA device ordinal */
    int32_t tail_rows;     /* levels with at most this many rows run inside one CTA of the
                              persistent solve kernel (no grid barrier per step): 8192 */
    int32_t cluster_rows;  /* graph path: a visit of the first level from which on every level
                              has at most this many rows, with all its sub-visits, runs as one
                              launch of a thread-block cluster (a dense coarsest solve larger
                              than 512 x 512 stays a launch over the whole GPU, between two
                              cluster launches). 0 (default): chosen at setup by
                              timing one cycle of each candidate and of the per-step schedule
                              when autotune is 1, else off; < 0: off. Results are bit-identical
                              whatever the choice. */
    int32_t row_tpr;       /* lanes per CSR row in the operator kernels: 0 (default) picks per
                              level from the mean row length; 1, 2, 4, ..., 32 forces it */
    int32_t sell;          /* operator kernels: 0 (default) one thread per row on a sliced
                              ELLPACK copy (32-row slices, rows padded to a multiple of four
                              entries, read with 16-byte loads) where rows have at most 64
                              entries and padding adds at most 50%, else lane groups on CSR; 1
                              sliced ELLPACK wherever rows have at most 64 entries; -1 CSR only */
    int32_t autotune;      /* 1: setup times the kernel form of each level's sweep and residual
                              (lanes per row, or one thread per row) and, with cluster_rows = 0,
                              the cluster schedule; 0 (default): rules only (measured within
                              timing noise of the timed choice on the benchmark workloads) */
    int32_t dense_rows;    /* a level with at most this many nodes (<= 4096) and at least n^2/8
                              off-diagonal entries is the coarsest, solved densely: 4096; 0 off */
    int32_t cheb_colours;  /* an aggregation level with more colour classes than this is smoothed
                              by a Chebyshev polynomial instead of colour-ordered Gauss-Seidel
                              (polynomial smoothers, the paper's Conclusion): 32; 0 never */
    int32_t cheb_degree;   /* degree of the Jacobi-preconditioned Chebyshev polynomial (interval
                              [lambda/30, lambda], lambda the Gershgorin bound of D^-1 A) that
                              replaces one sweep: 1 (1..8; degree 1 is Jacobi damped by
                              1/theta, theta the interval's centre) */
    int32_t tv_order;      /* summation order of a test-vector row sum (Section 2 relaxation):
                              LAMG_TV_STRIDED (default) or LAMG_TV_STORED, see below */
    int32_t agg_gpu_rows;  /* > 0: aggregation levels with at least this many rows run the
                              aggregation pass of Section 2 on the GPU (each node decided once
                              its lower-numbered neighbours are: the sequential pass's exact
                              result, in as many parallel rounds as the longest index-decreasing
                              path); 0 (default): on the host (one O(m) scan, measured faster) */
    int32_t reserved[1];
} lamg_options;                    /* 144 bytes */

/* Test-vector row sums (lamg_options.tv_order, lamg_testvectors, lamg_testvectors_noalloc).
 * The relaxation x_u <- -(sum_v A_uv x_v) / A_uu is written with the neighbour sum in stored
 * order; the test vectors feed integer aggregation decisions, so the order matters bit for bit.
 *  LAMG_TV_STORED:  every row summed in stored order, one dependent FP64 chain per row: the
 *                   plain definition, bit-identical to the reference evaluation of Section 2.
 *  LAMG_TV_STRIDED: rows of at most 32 entries as above; a longer row (hubs of power-law
 *                   graphs, dense Galerkin rows) as 32 strided partial sums (partial j: entries
 *                   j, j + 32, ... in order, each from 0.0) added in order of j, one warp per
 *                   row. Same values up to rounding; a hub row's dependent chain is 32 times
 *                   shorter, which is what keeps setup of power-law graphs fast on this GPU. */
#define LAMG_TV_STRIDED 0
#define LAMG_TV_STORED 1

typedef struct lamg_graph {
    int64_t n;
    const int64_t *rp;
    const int32_t *ci;
    const double *w;
} lamg_graph;

/* One level of a prebuilt hierarchy, natural node numbering (lamg_import).
 * kind: 0 elimination, 1 aggregation, 2 coarsest.
 * Operator A (all kinds): off-diagonal CSR rp/ci/val (columns ascending) + diag.
 * Aggregation level: colour[n] (Gauss-Seidel colour classes; rows of one colour must be
 *   pairwise non-adjacent), nc aggregates, agg[n], agg2[n] (-1 for caliber-1 rows), wt[n]:
 *   P row u = wt[u] at column agg[u] and 1 - wt[u] at column agg2[u].
 * Elimination level: cidx[n] = coarse index of a kept (C) node, -1 for an eliminated (F)
 *   node; C nodes must be numbered in ascending node order. The next level's operator must
 *   be the Schur complement of Eq. 2.
 * gamma: cycle index of an aggregation level (Eq. 5), ignored otherwise. */
typedef struct lamg_level_desc {
    int32_t kind;
    int32_t pad;
    int64_t n;
    const int64_t *rp;
    const int32_t *ci;
    const double *val;
    const double *diag;
    const int32_t *colour;
    int64_t nc;
    const int32_t *cidx;
    const int32_t *agg;
    const int32_t *agg2;
    const double *wt;
    double gamma;
} lamg_level_desc;

typedef struct lamg_solve_opts {
    double tol;            /* stop when ||b - L phi||_2 / ||b||_2 <= tol (recursive residual) */
    int32_t maxit;         /* outer CG iteration cap */
    uint32_t flags;        /* LAMG_DEVICE_PTRS */
    void *stream;          /* cudaStream_t for device-pointer calls, or 0 */
    int32_t wait_us;       /* limit of each device-side wait (the grid barriers of the
                              LAMG_PERSISTENT kernel): 0 = 2 s; > 0 = this many microseconds;
                              < 0 = give up at once (every wait runs out: LAMG_ERR_TIMEOUT) */
    int32_t pad;
} lamg_solve_opts;

typedef struct lamg_stats {
    int32_t iters;         /* outer iterations done */
    int32_t nlevels;
    double relres;         /* recursive residual norm / ||b|| at exit */
    double relres_true;    /* ||b - L phi|| / ||b|| recomputed at exit (FP64) */
    double b_mean;         /* mean removed from b before solving */
    double solve_ms;       /* device time of the call, copies included (CUDA events) */
    double *hist;          /* optional caller buffer of maxit+1 doubles: relres per iteration */
    double kernel_ms;      /* device time of the solve kernel(s) alone */
    double alg_bytes;      /* algorithmic DRAM bytes of the solve (each array once per step) */
    int64_t launches;      /* kernel launches of the solve */
} lamg_stats;

typedef struct lamg_hier lamg_hier;

/* Fill *opt with the defaults listed above. */
void lamg_options_default(lamg_options *opt);

/* Build a hierarchy for the Laplacian of graph g (Section 2 setup). The host runs
 * elimination, aggregation, caliber-2 and the Galerkin products; the GPU computes the test
 * vectors (K GS sweeps from a SplitMix64 start) and the per-edge affinities with the veto
 * flag. The hierarchy stays resident on the device until lamg_destroy.
 * Errors: INVALID, DISCONNECTED, SETUP, OOM, CUDA, NO_DEVICE. */
int lamg_setup(const lamg_graph *g, const lamg_options *opt, lamg_hier **out);

/* Build the device hierarchy from levels computed elsewhere (same layout as lamg_level_get
 * returns). Used to run the cycle on exactly the hierarchy and colour order of another
 * implementation. Errors: INVALID, OOM, CUDA, NO_DEVICE. */
int lamg_import(const lamg_level_desc *levels, int32_t nlevels, const lamg_options *opt,
                lamg_hier **out);

/* Solve L phi = b (Eq. 1) by flexible CG preconditioned with one cycle per iteration.
 * b (n values) is projected to mean zero first (the removed mean goes to st->b_mean);
 * phi (n values, output) has 1^T phi = 0. st may be NULL. Host vectors of at least 1 MiB pass
 * through pinned staging buffers that the library pools for the life of the process.
 * Errors: INVALID (tol <= 0, maxit < 1), NOT_CONVERGED (phi and st valid), CUDA, TIMEOUT. */
int lamg_solve(lamg_hier *h, const double *b, double *phi, const lamg_solve_opts *so,
               lamg_stats *st);

/* k right-hand sides at once: B and PHI are n x k, row-major (entry (u, j) at u*k + j).
 * Each column is an independent solve with its own CG scalars and stopping test; the cycles
 * run in SpMM form over all still-active columns. st: NULL or an array of k stats. Host
 * matrices of at least 128 MB move through 64 MB pinned chunks, copied on the host by a pool of
 * threads (one per hardware thread, created on first use and kept for the life of the process)
 * while the previous chunk's DMA runs.
 * Errors: as lamg_solve (NOT_CONVERGED if any column did not converge). */
int lamg_solve_batch(lamg_hier *h, int32_t k, const double *B, double *PHI,
                     const lamg_solve_opts *so, lamg_stats *st);

/* Apply the preconditioner once: z = M r (one cycle from zero, then the mean-zero
 * projection), no projection of r. r and z are n values (host, or device with
 * LAMG_DEVICE_PTRS). Errors: CUDA. */
int lamg_cycle(lamg_hier *h, const double *r, double *z, uint32_t flags);

/* Hierarchy shape: info[0] = number of levels; for level l, meta (7 int64 per level) =
 * kind, n, nnz (off-diagonal), colours, nc, caliber-2 rows, device bytes; gamma[l]. */
int lamg_hier_info(const lamg_hier *h, int64_t *nlevels, int64_t *meta, double *gamma);

/* Copy a per-level array of the hierarchy, natural numbering, into dst (sized by the caller
 * from lamg_hier_info; dst may be NULL to query the element count, returned in *count).
 * Names: "rp","ci","val","diag" (int64/int32/double/double), "colour","cidx","agg","agg2"
 * (int32), "wt" (double), "X" (n x K test vectors, double), "aff" (double per off-diagonal
 * entry), "strong" (uint8 per off-diagonal entry), "pinv" (n x n, double).
 * Errors: INVALID for an unknown name or level. */
int lamg_level_get(const lamg_hier *h, int32_t level, const char *name, void *dst,
                   int64_t *count);

/* Release a hierarchy and all its device memory. NULL is allowed. */
void lamg_destroy(lamg_hier *h);

/* Setup kernel K9 on its own (test vectors, Section 2): for a level operator given by host
 * arrays (off-diagonal CSR rp/ci/val + diag, natural order) and a colouring (colour[u] >= 0;
 * rows of one colour pairwise non-adjacent), start each of K <= 16 columns at U[-1, 1) from
 * SplitMix64 output 1 + ((level << 44) | (u << 4) | k) of the stream `seed` and run nu
 * colour-ordered GS sweeps on A x = 0 (colours ascending) on the GPU, row sums in `order`
 * (LAMG_TV_STRIDED or LAMG_TV_STORED). X (host, n x K row-major) receives the result.
 * Errors: INVALID (sizes, K, order, a negative colour), OOM, CUDA, NO_DEVICE. */
int lamg_testvectors(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                     const double *diag, const int32_t *colour, int32_t level, uint64_t seed,
                     int32_t K, int32_t nu, double *X, int32_t order);

/* Setup kernel K10 on its own (Eq. 3 affinity and Eq. 9 veto) on the GPU for host inputs:
 * aff[e] = affinity of off-diagonal entry e, strong[e] = 1 iff |A_e| >= tau * max |A_ut| over
 * u's row. Errors: INVALID, OOM, CUDA, NO_DEVICE. */
int lamg_affinity(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                  const double *X, int32_t K, double tau, double *aff, uint8_t *strong);

/* Time one solve-phase kernel of a hierarchy in isolation (used for roofline figures): `reps`
 * launches on the hierarchy's stream, each after a 256 MB device write that evicts the L2,
 * timed with CUDA events. which: 0 residual r = b - A x at an aggregation level, 1 one full
 * colour-ordered GS sweep at an aggregation level, 2 outer CG SpMV with the p.q dot (level 0),
 * 3 restriction P^T r, 4 prolongation x += P x^c. out[0] = mean device ms per launch (sweep),
 * out[1] = algorithmic DRAM bytes of one launch (sweep), out[2] = kernels per launch.
 * The kernels run on the hierarchy's current vectors. Errors: INVALID, OOM, CUDA, TIMEOUT. */
int lamg_time_kernel(lamg_hier *h, int32_t which, int32_t level, int32_t reps, double *out);

/* Time one k-column kernel of the multi-right-hand-side solve in isolation (roofline figures
 * of lamg_solve_batch, in the hierarchy's cycle precision): `reps` launches on the hierarchy's
 * stream, each after a 256 MB device write that evicts the L2, timed with CUDA events. which: 0
 * residual at an aggregation level, 1 one smoothing sweep at an aggregation level (all colour
 * classes of Gauss-Seidel, or the degree-m Chebyshev polynomial on levels with many colours),
 * 2 the outer CG product A p with its dot products (level 0, FP64), 3 one step of the Chebyshev
 * polynomial alone (Chebyshev levels only). 1 <= k <= 32.
 * out[0] = mean device ms per launch sequence, out[1] = its algorithmic DRAM bytes (operator once,
 * each vector once per column), out[2] = kernels per sequence, out[3] = its algorithmic flops (a
 * multiply-add per stored entry and column, plus per-row arithmetic). No counterpart in the
 * paper. Errors: INVALID, OOM, CUDA, TIMEOUT. */
int lamg_time_kernel_batch(lamg_hier *h, int32_t which, int32_t level, int32_t k, int32_t reps,
                           double *out);

/* Allocation-free variant of lamg_testvectors for callers that cannot allocate device memory:
 * code running inside another framework's memory pool or a plugin that may only use the memory
 * handed to it, and programs that must not allocate after start-up. No counterpart in the
 * paper: it is a deployment form of the same setup kernel. All pointers are DEVICE pointers
 * owned by the caller: rp[n+1] (int64), ci, val, diag, colour[n] and the output X (n x K,
 * row-major). The work is queued on `stream` (a cudaStream_t, 0 for the default stream) and
 * the call returns without waiting. For colours in [0, ncol) (rows of one colour pairwise
 * non-adjacent) X is bit-identical to lamg_testvectors with the same `order`; a row whose colour
 * is outside [0, ncol) is never relaxed and keeps its random start.
 * Scratch (rows grouped by colour class, the class offsets) lives in a fixed 8 MiB __device__
 * array held by every GPU that loads the library until exit: n <= 2^21 and ncol <= 1024, else
 * LAMG_ERR_INVALID. The first call on a device looks up the array's device address and should
 * come before any stream capture on that device. Calls share the array; calls that overlap on
 * the GPU race and must be serialised by the caller. No device memory is allocated.
 * Errors: INVALID, CUDA. */
int lamg_testvectors_noalloc(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                             const double *diag, const int32_t *colour, int32_t ncol, int32_t level,
                             uint64_t seed, int32_t K, int32_t nu, double *X, void *stream,
                             int32_t order);

/* Per-step timing of one cycle of the persistent solve kernel (r = 0): out receives up to cap
 * pairs (next step index, nanoseconds since the previous pair), one per grid barrier, read
 * from %globaltimer in CTA 0; *count = pairs written. Step indices refer to lamg_op_list.
 * Errors: INVALID (no persistent kernel for this hierarchy), CUDA, TIMEOUT. */
int lamg_profile_cycle(lamg_hier *h, int64_t *out, int64_t cap, int64_t *count);

/* The static step list of one cycle: 3 int32 per step (kind, level, colour); kinds 0 first
 * GS colour from zero, 1 GS colour class, 2 zero, 3 residual, 4 restriction, 5 prolongation,
 * 6 elimination restriction, 7 elimination interpolation, 8 coarsest solve, 9 Chebyshev
 * smoothing step (colour = step index within its polynomial, + 256 when it reads the level's
 * second buffer instead of the iterate), 10 copy of the second buffer into the iterate after an
 * odd number of steps, 11 the first Chebyshev step of a first visit (from a zero iterate: no
 * product with A; colour 1 when it writes the second buffer). out may be NULL to query *count.
 * Errors: INVALID. */
int lamg_op_list(const lamg_hier *h, int32_t *out, int64_t cap, int64_t *count);

/* The launch schedule of the graph path (no counterpart in the paper: it records how the
 * cycle of Section 2 is mapped onto kernel launches). out[0] = first level of the cluster
 * sub-cycle (-1: none), out[1] = CTAs per cluster (0: cluster launch unavailable), out[2] =
 * kernel launches of one cycle, out[3] = steps of one cycle, out[4] = levels L, then per
 * level the kernel form of the sweep and of the residual-type passes (0: one thread per row
 * on the sliced copy, t > 0: t lanes per CSR row), then for each schedule timed by the
 * automatic choice a pair (first cluster level or -1, nanoseconds per cycle). cap >= 5 + 2 L
 * int64 entries; *count = entries written. Errors: INVALID. */
int lamg_schedule_info(const lamg_hier *h, int64_t *out, int64_t cap, int64_t *count);

/* The paper's own outer iteration (Section 2): the stationary iteration x <- x + M(b - A x)
 * with M one cycle, each step followed by the min-residual recombination of the last kappa
 * saved iterates, alpha = argmin || (b - A x) - A E alpha || with E = [x_1 - x, ..., x_m - x]
 * (normal equations solved by Gaussian elimination with partial pivoting), x <- x + E alpha,
 * then the mean-zero projection (Eq. 1). kappa = 0: plain stationary cycles. The per-cycle
 * relative residuals (stats.hist) are what the paper's convergence factor is measured on.
 * Same conventions as lamg_solve (b projected, stop when ||b - A x|| / ||b|| <= tol, checked
 * every cycle on the true residual); FP64 hierarchies only; 0 <= kappa <= 16.
 * Errors: INVALID, NOT_CONVERGED (stats valid), CUDA, TIMEOUT. */
int lamg_solve_stationary(lamg_hier *h, const double *b, double *phi, int32_t kappa,
                          const lamg_solve_opts *so, lamg_stats *st);

/* Wall time (ms) of the setup phases of a hierarchy built by lamg_setup, 9 entries: input
 * validation and Laplacian; elimination (Eq. 2); colouring; test vectors and affinities on the
 * GPU (Section 2, Eq. 3, Eq. 9) with their copies; aggregation and caliber-2 (Eqs. 4, 13);
 * Galerkin products; dense pseudo-inverse of the coarsest level; device layout and uploads;
 * step list, timing trials and graph capture. cap >= 9; with cap >= 10, out[9] = the parallel
 * rounds the GPU aggregation pass took, summed over levels (0 when every level aggregated on the
 * host). Errors: INVALID. */
int lamg_setup_times(const lamg_hier *h, double *out, int32_t cap);

/* Solve G independent systems L_g phi_g = b_g (Eq. 1), each on its own hierarchy, with one
 * kernel launch: one thread-block cluster per system runs that system's whole flexible-CG solve
 * (projection of b, every cycle of Section 2, the stopping test, the true residual), with
 * deterministic cluster-scope reductions; the clusters share nothing. Meant for many small
 * graphs, whose solves would otherwise be a few hundred small launches each. A hierarchy the
 * cluster kernel should not take (FP32 cycle, rows longer than 256 entries, more than 2^19
 * stored entries in the finest operator, no cluster launch on the device, level tables over the
 * shared-memory limit) is solved by lamg_solve after the launch.
 * No counterpart in the paper (it batches solves of the same method).
 * hs, b, phi: G entries; b[g], phi[g] of hs[g]'s size, host pointers, or device pointers with
 * LAMG_DEVICE_PTRS; all hierarchies on one device; the work goes to so->stream (0: the first
 * hierarchy's stream). st: NULL or G entries (solve_ms and kernel_ms are the whole launch).
 * Returns LAMG_OK when every system converged, LAMG_ERR_NOT_CONVERGED when one did not (all
 * stats valid). Errors: INVALID, CUDA, TIMEOUT. */
int lamg_solve_many(int32_t G, lamg_hier *const *hs, const double *const *b, double *const *phi,
                    const lamg_solve_opts *so, lamg_stats *st);

/* Per-step device time of one cycle (r = 0) with the steps on levels >= from_level run as
 * cluster launches as cluster_rows forms them (from_level < 0: none), outside any graph: out
 * receives 3 int64 per step
 * (step index, 1 if the step ran inside a cluster launch, nanoseconds). A step inside a
 * cluster is timed by %globaltimer in its first CTA, from before the step to after the
 * barrier that ends it; any other step by CUDA events around its own launch (no overlap with
 * its neighbours). cap >= 3 x steps. No counterpart in the paper. Errors: INVALID (cap, or
 * no cluster launch on this device), CUDA, TIMEOUT. */
int lamg_profile_schedule(lamg_hier *h, int32_t from_level, int64_t *out, int64_t cap, int64_t *count);

/* Name of an error code. */
const char *lamg_strerror(int code);

/* ----------------------------------------------------------------- serving
 * A server owns a device memory budget and a worker thread. lamg_serve() submits one request
 * (graph + right-hand side, both copied), returns at once with a ticket; requests are
 * admitted while their estimated hierarchy + vector bytes fit the budget, set up on host
 * threads, and their CG iterations are interleaved on the device with those of every other
 * admitted request. lamg_serve_poll() reports completion and copies the solution out. */
typedef struct lamg_server lamg_server;

typedef struct lamg_server_opts {
    double budget_bytes;   /* device memory budget for admitted requests */
    int32_t max_inflight;  /* maximum concurrently admitted requests */
    int32_t setup_threads; /* host setup workers */
    double tol;
    int32_t maxit;
    int32_t device;
} lamg_server_opts;

typedef struct lamg_ticket_info {
    int32_t done;          /* 0 pending, 1 finished */
    int32_t status;        /* LAMG_OK or an error code once done */
    int32_t iters;
    int32_t pad;
    double relres;         /* recursive residual at exit */
    double relres_true;    /* ||b - L phi|| / ||b|| recomputed at exit */
    double t_submit_ms, t_admit_ms, t_ready_ms, t_done_ms;  /* server clock: submitted,
                              admitted (setup starts), hierarchy ready, result ready */
} lamg_ticket_info;

/* Create a server on device so->device with the given setup options (NULL: defaults), one
 * executor thread and so->setup_threads setup threads. A served setup runs no timing trials:
 * autotune is taken as 0 and cluster_rows = 0 as -1; coarsest_max = 0 is taken as 1024 (one
 * solve per setup does not recover a larger dense inverse). Errors: INVALID, NO_DEVICE. */
int lamg_server_create(const lamg_server_opts *so, const lamg_options *opt, lamg_server **out);
/* Submit one request (graph + right-hand side, copied; same conventions as lamg_setup and
 * lamg_solve); returns at once with a ticket. A request whose estimated device memory alone
 * exceeds the budget is refused with LAMG_ERR_ADMISSION; an invalid graph is accepted and its
 * ticket finishes with the setup's error code. */
int lamg_serve(lamg_server *s, const lamg_graph *g, const double *b, int64_t *ticket);
/* State of a ticket; when done and phi != NULL, the n-value solution is copied to phi.
 * Errors: INVALID (unknown ticket). */
int lamg_serve_poll(lamg_server *s, int64_t ticket, lamg_ticket_info *info, double *phi);
/* Wait (at most timeout_s seconds) until every submitted request has finished.
 * Errors: TIMEOUT. */
int lamg_server_drain(lamg_server *s, double timeout_s);
/* out[0] device bytes held by in-flight requests, out[1] requests in flight, out[2] requests
 * waiting for admission, out[3] requests not yet finished, out[4] grouped launches so far (the
 * requests that became ready since the executor's previous pass and that the cluster kernel
 * takes are solved together, one thread-block cluster each, as in lamg_solve_many), out[5]
 * requests solved in such launches, out[6] the largest group, out[7] solves whose first launch
 * the executor issued while another request's device work was still in flight (requests sharing
 * the device). 8 entries. */
int lamg_server_stats(lamg_server *s, int64_t *out);
/* Stop the threads and release everything; unfinished requests are dropped. */
void lamg_server_destroy(lamg_server *s);

#ifdef __cplusplus
}
#endif

#endif /* LAMG_H */
