/*
 * LAMG+ oracle: a plain, serial, FP64 CPU statement of the LAMG+ setup and solve phase
 * (Livne, "LAMG+: A Robust Lean Algebraic Multigrid Solver for Graph Laplacians").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the CUDA library links, includes or calls this file;
 * it shares no code, header, table or constant generator with it. Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark load it.
 *
 * Every routine is written for a reader checking it against the paper: loops in the order
 * the paper states the step, no blocking, no fusion. Where the paper is silent the reading
 * chosen is stated at the routine (the same readings are listed with the design notes).
 *
 * Matrix convention: a level operator A is stored as its off-diagonal entries A_uv in CSR
 * (columns ascending in each row) plus the diagonal A_uu. For the finest level A = L = D - W,
 * so A_uv = -w_uv and A_uu = sum_v w_uv (Section 1, Eq. 1). Edge "weights" of a coarse level
 * are w_uv = -A_uv and may be signed after caliber-2 (hence |w| in the veto, Eq. 9).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OK 0
#define ERR_INVALID 1
#define ERR_DISCONNECTED 2
#define ERR_SETUP 3
#define ERR_NOMEM 4

enum { LV_ELIM = 0, LV_AGG = 1, LV_COARSEST = 2 };
enum { ST_UNDECIDED = 0, ST_SEED = 1, ST_ASSOC = 2 };

typedef struct {
    int64_t n, nnz;
    int64_t *rp;
    int32_t *ci;
    double *val;   /* off-diagonal A_uv */
    double *diag;  /* A_uu */
} Mat;

/* Options, filled from flat arrays so that ctypes can pass them. */
typedef struct {
    int K;              /* test vectors, Section 3.3: K = 4 fixed */
    int nu_tv;          /* GS sweeps per test vector, Section 2: nu = 3 */
    int dmax;           /* low-degree elimination bound, Eq. 2: d_max = 4 */
    int nu_pre, nu_post;/* (1,2) cycle, Appendix A, Table 10 */
    int coarsest_max;   /* dense coarsest level when n <= this; 0: the size rule of oracle_setup */
    int dense_rows;     /* dense coarsest level also when n <= this and the level has at least
                           n^2 / 8 off-diagonal entries (0: off) */
    int cheb_colours;   /* an aggregation level with more colours than this is smoothed by a
                           Chebyshev polynomial instead of Gauss-Seidel (0: never) */
    int cheb_degree;    /* degree of the polynomial that replaces one Gauss-Seidel sweep */
    int max_levels;
    int veto;           /* strength-of-connection veto on/off (Eq. 9) */
    int caliber2;       /* selective caliber-2 on/off (Section 3.2) */
    int tv_lex;         /* 1: test-vector GS in lexicographic order, 0: colour order */
    int symmetric;      /* 1: symmetric cycle (nu_pre = nu_post, integer gamma) */
    uint64_t seed;      /* test-vector random stream */
    double Q;           /* energy-ratio guard bound, Eq. 4: Q = 2.5 */
    double tau_soc;     /* Eq. 9: 0.05 */
    double elim_min_frac;   /* elimination level kept while |F| >= this * n */
    double snap;        /* caliber-2 weight snapping distance to 0/1 */
    double guard_eps;   /* relative size under which a nodal energy counts as zero */
    double gamma_fixed; /* > 0: use this gamma on every aggregation level instead of Eq. 5 */
} Opts;

typedef struct {
    int kind;
    Mat A;
    /* colouring (aggregation levels) */
    int ncol;
    int32_t *colour;
    int64_t *cptr;     /* rows grouped by colour: corder[cptr[c] .. cptr[c+1]) */
    int32_t *corder;
    /* elimination level */
    int64_t nc;        /* also used by aggregation levels: number of aggregates */
    int32_t *cidx;     /* coarse index of a C node, -1 for an F node */
    int32_t *cnode;    /* fine node of coarse index i */
    /* aggregation level */
    int32_t *agg, *agg2;   /* P row u: wt[u] on agg[u], 1 - wt[u] on agg2[u] (agg2 = -1: caliber-1) */
    double *wt;
    int32_t *seed_of;      /* seed node of u's aggregate */
    int32_t *status;
    double *X;             /* n x K test vectors, X[u*K + k] */
    double *aff;           /* affinity per off-diagonal entry */
    uint8_t *strong;       /* 1 if the entry survives the veto (u's view) */
    double gamma;
    /* Chebyshev smoothing (levels with many colours): step k of one polynomial is
       d <- c1[k] d + c2[k] D^{-1}(b - A x), x <- x + d */
    int cheb;
    double cheb_lambda, cheb_c1[8], cheb_c2[8];
    /* coarsest */
    double *pinv;          /* dense n x n pseudo-inverse */
    /* cycle state */
    double *x, *b, *r;
    int64_t visits;        /* visit counter j within one finest-level cycle */
    int64_t nvisits;       /* visits of this level in the last cycle (all kinds) */
} Level;

typedef struct {
    int nlev;
    Level *lv;
    Opts o;
    int64_t E0;            /* |E| of the finest level */
} Hier;

/* ------------------------------------------------------------------ utilities */

static void *xcalloc(size_t n, size_t s) {
    void *p = calloc(n ? n : 1, s ? s : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}

static void mat_free(Mat *A) {
    free(A->rp); free(A->ci); free(A->val); free(A->diag);
    memset(A, 0, sizeof(*A));
}

static double dot(const double *a, const double *b, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Mean-zero projection: phi <- phi - (1^T phi / n) 1, the constraint 1^T phi = 0 of Eq. 1. */
static void project_mean(double *v, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += v[i];
    double m = s / (double)n;
    for (int64_t i = 0; i < n; i++) v[i] -= m;
}

/* y = A x with the diagonal. */
static void matvec(const Mat *A, const double *x, double *y) {
    for (int64_t u = 0; u < A->n; u++) {
        double s = A->diag[u] * x[u];
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) s += A->val[e] * x[A->ci[e]];
        y[u] = s;
    }
}

/* r = b - A x */
static void residual(const Mat *A, const double *x, const double *b, double *r) {
    for (int64_t u = 0; u < A->n; u++) {
        double s = A->diag[u] * x[u];
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) s += A->val[e] * x[A->ci[e]];
        r[u] = b[u] - s;
    }
}

/* ------------------------------------------------------------------ random start */

/* SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): the state advances by
 * the golden-ratio increment 0x9e3779b97f4a7c15 and each state is mixed by two
 * xor-shift-multiply rounds. Counter-based use: output number i of the stream started at
 * `seed` is mix(seed + i * increment), i >= 1. */
static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix64(uint64_t seed, uint64_t i) {
    return sm64_mix(seed + i * 0x9e3779b97f4a7c15ULL);
}

/* Random start of test vector k at node u of level l (Section 2: "a random start").
 * Reading: U[-1, 1) from the top 53 bits of SplitMix64 output 1 + ((l << 44) | (u << 4) | k),
 * so every (level, node, column) with k < 16 and u < 2^40 has its own counter. */
double oracle_random_start(uint64_t seed, int level, int64_t u, int k) {
    uint64_t c = ((uint64_t)level << 44) | ((uint64_t)u << 4) | (uint64_t)k;
    uint64_t z = oracle_splitmix64(seed, c + 1);
    double r = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    return 2.0 * r - 1.0;
}

/* ------------------------------------------------------------------ colouring */

/* Greedy colouring in ascending node order, smallest colour unused by coloured neighbours.
 * Rows of one colour are pairwise non-adjacent, so a Gauss-Seidel sweep over one colour is
 * the same whatever order its rows are visited in. */
static void colour_level(Level *L) {
    const Mat *A = &L->A;
    int64_t n = A->n;
    L->colour = xcalloc(n, sizeof(int32_t));
    int maxc = 0;
    int32_t *mark = xcalloc(n + 2, sizeof(int32_t));
    for (int64_t u = 0; u < n; u++) L->colour[u] = -1;
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
            int32_t c = L->colour[A->ci[e]];
            if (c >= 0) mark[c] = (int32_t)(u + 1);
        }
        int c = 0;
        while (mark[c] == (int32_t)(u + 1)) c++;
        L->colour[u] = c;
        if (c + 1 > maxc) maxc = c + 1;
    }
    free(mark);
    L->ncol = maxc;
    L->cptr = xcalloc(maxc + 1, sizeof(int64_t));
    for (int64_t u = 0; u < n; u++) L->cptr[L->colour[u] + 1]++;
    for (int c = 0; c < maxc; c++) L->cptr[c + 1] += L->cptr[c];
    L->corder = xcalloc(n, sizeof(int32_t));
    int64_t *fill = xcalloc(maxc + 1, sizeof(int64_t));
    for (int c = 0; c <= maxc; c++) fill[c] = L->cptr[c];
    for (int64_t u = 0; u < n; u++) L->corder[fill[L->colour[u]]++] = (int32_t)u;
    free(fill);
}

/* ------------------------------------------------------------------ Gauss-Seidel */

/* One Gauss-Seidel update of row u (Section 2, relaxation):
 * phi_u <- (b_u - sum_{v != u} A_uv phi_v) / A_uu. b == NULL means b = 0. */
static void gs_row(const Mat *A, int64_t u, double *x, const double *b) {
    double s = 0.0;
    for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) s += A->val[e] * x[A->ci[e]];
    double bu = b ? b[u] : 0.0;
    x[u] = (bu - s) / A->diag[u];
}

/* Colour-ordered sweep: colours 0..C-1 (forward) or C-1..0 (reverse); rows of a colour in
 * ascending index. */
static void gs_sweep_colour(const Level *L, double *x, const double *b, int reverse) {
    for (int ci = 0; ci < L->ncol; ci++) {
        int c = reverse ? L->ncol - 1 - ci : ci;
        for (int64_t t = L->cptr[c]; t < L->cptr[c + 1]; t++) gs_row(&L->A, L->corder[t], x, b);
    }
}

/* Chebyshev smoothing of A x = b (polynomial smoothing; a reading for levels whose colouring
 * makes a Gauss-Seidel sweep hundreds of parallel steps): the Jacobi-preconditioned Chebyshev
 * iteration of degree m on the interval [lambda/30, lambda] of D^{-1} A, lambda the Gershgorin
 * bound max_u (1 + sum_v |A_uv| / A_uu). With theta = (hi + lo)/2, delta = (hi - lo)/2,
 * sigma = theta/delta and rho_0 = 1/sigma, rho_k = 1/(2 sigma - rho_{k-1}), step k updates every
 * row from the previous iterate: d <- c1[k] d + c2[k] D^{-1}(b - A x), x <- x + d, with
 * c1[0] = 0, c2[0] = 1/theta, c1[k] = rho_k rho_{k-1}, c2[k] = 2 rho_k / delta. */
static void cheb_coefficients(Level *L, int m) {
    const Mat *A = &L->A;
    double lam = 0.0;
    for (int64_t u = 0; u < A->n; u++) {
        double s = 0.0;
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) s += fabs(A->val[e]);
        const double g = 1.0 + s / A->diag[u];
        if (g > lam) lam = g;
    }
    const double hi = lam, lo = lam / 30.0;
    const double theta = (hi + lo) / 2.0, delta = (hi - lo) / 2.0, sigma = theta / delta;
    double rho = 1.0 / sigma;
    L->cheb_lambda = lam;
    L->cheb_c1[0] = 0.0;
    L->cheb_c2[0] = 1.0 / theta;
    for (int k = 1; k < m && k < 8; k++) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        L->cheb_c1[k] = rn * rho;
        L->cheb_c2[k] = 2.0 * rn / delta;
        rho = rn;
    }
}

static void cheb_poly(const Level *L, double *x, const double *b, int m, double *d, double *xn) {
    const Mat *A = &L->A;
    const int64_t n = A->n;
    for (int k = 0; k < m; k++) {
        for (int64_t u = 0; u < n; u++) {
            double s = A->diag[u] * x[u];
            for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) s += A->val[e] * x[A->ci[e]];
            const double du = (k == 0 ? 0.0 : L->cheb_c1[k] * d[u]) + L->cheb_c2[k] * (b[u] - s) / A->diag[u];
            d[u] = du;
            xn[u] = x[u] + du;
        }
        memcpy(x, xn, n * sizeof(double));
    }
}

static void gs_sweep_lex(const Mat *A, double *x, const double *b) {
    for (int64_t u = 0; u < A->n; u++) gs_row(A, u, x, b);
}

/* ------------------------------------------------------------------ elimination */

/* Low-degree elimination (Section 2, Eq. 2). F = greedy maximal independent set of the
 * nodes of degree <= dmax (degree = number of off-diagonal nonzeros), nodes visited in
 * ascending index. Returns |F|; fills inF. */
static int64_t select_F(const Mat *A, int dmax, uint8_t *inF) {
    int64_t n = A->n, nf = 0;
    uint8_t *blocked = xcalloc(n, 1);
    memset(inF, 0, n);
    for (int64_t u = 0; u < n; u++) {
        int64_t deg = A->rp[u + 1] - A->rp[u];
        if (deg > dmax || blocked[u]) continue;
        inF[u] = 1; nf++;
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) blocked[A->ci[e]] = 1;
    }
    free(blocked);
    return nf;
}

/* Gather a sparse accumulator row into sorted CSR form, dropping exact zeros.
 * cols/vals: touched columns in arbitrary order with their sums in acc[]. */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct {
    int64_t n, cap, nnz;
    int64_t *rp; int32_t *ci; double *val; double *diag;
} Builder;

static void bld_init(Builder *B, int64_t n, int64_t cap) {
    B->n = n; B->cap = cap > 16 ? cap : 16; B->nnz = 0;
    B->rp = xcalloc(n + 1, sizeof(int64_t));
    B->ci = xcalloc(B->cap, sizeof(int32_t));
    B->val = xcalloc(B->cap, sizeof(double));
    B->diag = xcalloc(n, sizeof(double));
}

static void bld_push(Builder *B, int32_t c, double v) {
    if (B->nnz == B->cap) {
        B->cap *= 2;
        B->ci = realloc(B->ci, B->cap * sizeof(int32_t));
        B->val = realloc(B->val, B->cap * sizeof(double));
        if (!B->ci || !B->val) abort();
    }
    B->ci[B->nnz] = c; B->val[B->nnz] = v; B->nnz++;
}

static void bld_finish(Builder *B, Mat *out) {
    out->n = B->n; out->nnz = B->nnz; out->rp = B->rp; out->ci = B->ci;
    out->val = B->val; out->diag = B->diag;
}

/* Schur complement onto C = V \ F (Eq. 2): A^c = A_CC - A_CF A_FF^{-1} A_FC. A_FF is diagonal
 * because F is independent. C nodes keep ascending order. */
static void eliminate(const Mat *A, const uint8_t *inF, Level *L, Mat *Ac) {
    int64_t n = A->n;
    L->cidx = xcalloc(n, sizeof(int32_t));
    int64_t nc = 0;
    for (int64_t u = 0; u < n; u++) L->cidx[u] = inF[u] ? -1 : (int32_t)nc++;
    L->nc = nc;
    L->cnode = xcalloc(nc, sizeof(int32_t));
    for (int64_t u = 0; u < n; u++) if (!inF[u]) L->cnode[L->cidx[u]] = (int32_t)u;

    Builder B; bld_init(&B, nc, A->nnz);
    double *acc = xcalloc(nc, sizeof(double));
    int32_t *mark = xcalloc(nc, sizeof(int32_t));
    int32_t *touched = xcalloc(nc, sizeof(int32_t));
    for (int64_t j = 0; j < nc; j++) mark[j] = -1;
    for (int64_t i = 0; i < nc; i++) {
        int64_t u = L->cnode[i];
        int nt = 0;
        double d = A->diag[u];
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
            int32_t v = A->ci[e];
            if (inF[v]) {
                /* - A_uf A_fu / A_ff on the diagonal, - A_uf A_fv / A_ff off it */
                double af = A->diag[v];
                double auf = A->val[e];
                for (int64_t g = A->rp[v]; g < A->rp[v + 1]; g++) {
                    int32_t t = A->ci[g];
                    double term = auf * A->val[g] / af;
                    if (t == u) { d -= term; continue; }
                    int32_t j = L->cidx[t];
                    if (mark[j] != i) { mark[j] = (int32_t)i; acc[j] = 0.0; touched[nt++] = j; }
                    acc[j] -= term;
                }
            } else {
                int32_t j = L->cidx[v];
                if (mark[j] != i) { mark[j] = (int32_t)i; acc[j] = 0.0; touched[nt++] = j; }
                acc[j] += A->val[e];
            }
        }
        qsort(touched, nt, sizeof(int32_t), cmp_i32);
        for (int t = 0; t < nt; t++)
            if (acc[touched[t]] != 0.0) bld_push(&B, touched[t], acc[touched[t]]);
        B.diag[i] = d;
        B.rp[i + 1] = B.nnz;
    }
    bld_finish(&B, Ac);
    free(acc); free(mark); free(touched);
}

/* ------------------------------------------------------------------ test vectors, affinity */

/* One relaxation step of a test vector at row u (Section 2: GS on A x = 0):
 * x_u <- (0 - sum_{v != u} A_uv x_v) / A_uu, the neighbour sum taken in stored (ascending
 * column) order from 0.0, as the relaxation formula is written. */
static void tv_row(const Mat *A, int64_t u, double *x) {
    double s = 0.0;
    for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) s += A->val[e] * x[A->ci[e]];
    x[u] = (0.0 - s) / A->diag[u];
}

/* K test vectors, each nu_tv GS sweeps on A x = 0 from the random start (Section 2), in
 * lexicographic or colour order (colours ascending, rows of a colour in ascending index). */
static void test_vectors(Level *L, const Opts *o, int level) {
    int64_t n = L->A.n;
    int K = o->K;
    L->X = xcalloc(n * K, sizeof(double));
    double *x = xcalloc(n, sizeof(double));
    for (int k = 0; k < K; k++) {
        for (int64_t u = 0; u < n; u++) x[u] = oracle_random_start(o->seed, level, u, k);
        for (int s = 0; s < o->nu_tv; s++) {
            if (o->tv_lex) {
                for (int64_t u = 0; u < n; u++) tv_row(&L->A, u, x);
            } else {
                for (int c = 0; c < L->ncol; c++)
                    for (int64_t t = L->cptr[c]; t < L->cptr[c + 1]; t++) tv_row(&L->A, L->corder[t], x);
            }
        }
        for (int64_t u = 0; u < n; u++) L->X[u * K + k] = x[u];
    }
    free(x);
}

/* Affinity (Eq. 3): c_uv = (sum_k x_u x_v)^2 / ((sum_k x_u^2)(sum_k x_v^2)). */
static double affinity(const double *xu, const double *xv, int K) {
    double uv = 0.0, uu = 0.0, vv = 0.0;
    for (int k = 0; k < K; k++) uv += xu[k] * xv[k];
    for (int k = 0; k < K; k++) uu += xu[k] * xu[k];
    for (int k = 0; k < K; k++) vv += xv[k] * xv[k];
    return (uv * uv) / (uu * vv);
}

/* Per off-diagonal entry: affinity, and the strength-of-connection test of Eq. 9 from u's
 * side: (u,v) is skipped when |w_uv| < tau_soc * max_{t~u} |w_ut|. */
static void affinity_and_veto(Level *L, const Opts *o) {
    const Mat *A = &L->A;
    int K = o->K;
    L->aff = xcalloc(A->nnz, sizeof(double));
    L->strong = xcalloc(A->nnz, 1);
    for (int64_t u = 0; u < A->n; u++) {
        double mx = 0.0;
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) if (fabs(A->val[e]) > mx) mx = fabs(A->val[e]);
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
            L->aff[e] = affinity(&L->X[u * K], &L->X[(int64_t)A->ci[e] * K], K);
            L->strong[e] = o->veto ? (fabs(A->val[e]) >= o->tau_soc * mx) : 1;
        }
    }
}

/* ------------------------------------------------------------------ energy guard */

/* Energy ratio q_{u<-s} of Eq. 4 through the per-node moments of Appendix B:
 * s0 = sum_v w_uv, s1 = sum_v w_uv x_v, s2 = sum_v w_uv x_v^2 (w_uv = -A_uv),
 * relaxed energy min_y E_u = (s2 - s1^2/s0)/2, forced energy E_u(x_s) = (x_s^2 s0 - 2 x_s s1 + s2)/2,
 * q = max over k of forced / relaxed.
 * Reading where the relaxed energy vanishes (e.g. a node with one neighbour): with
 * scale = (|s2| + s1^2/|s0|)/2, a relaxed energy <= guard_eps * scale counts as zero; then the
 * ratio is 1 if the forced energy is also <= guard_eps * scale, else +inf. */
double oracle_guard_q(const double *s0, const double *s1, const double *s2, const double *xs,
                      int K, double guard_eps) {
    double q = 0.0;
    for (int k = 0; k < K; k++) {
        double relaxed = 0.5 * (s2[k] - s1[k] * s1[k] / s0[0]);
        double forced = 0.5 * (xs[k] * xs[k] * s0[0] - 2.0 * xs[k] * s1[k] + s2[k]);
        double scale = 0.5 * (fabs(s2[k]) + s1[k] * s1[k] / fabs(s0[0]));
        double qk;
        if (relaxed <= guard_eps * scale) qk = (forced <= guard_eps * scale) ? 1.0 : INFINITY;
        else qk = forced / relaxed;
        if (qk > q) q = qk;
    }
    return q;
}

/* ------------------------------------------------------------------ aggregation */

/* Caliber-1 aggregation (Section 2) with the veto (Eq. 9).
 * Readings (the paper gives no visit order or seed rule): nodes are visited in ascending
 * index; an undecided node u considers its strong neighbours s that are seeds or still
 * undecided, admissible when q_{u<-s} <= Q (Eq. 4), and joins the one of largest affinity
 * c_us (ties: lower index); the chosen s becomes a seed if it was undecided. No size cap.
 * Nodes left undecided after the pass become singleton seeds. Aggregates are numbered by
 * ascending seed index. */
static void aggregate(Level *L, const Opts *o) {
    const Mat *A = &L->A;
    int64_t n = A->n;
    int K = o->K;
    L->status = xcalloc(n, sizeof(int32_t));
    L->seed_of = xcalloc(n, sizeof(int32_t));
    double *s0 = xcalloc(n, sizeof(double));
    double *s1 = xcalloc(n * K, sizeof(double));
    double *s2 = xcalloc(n * K, sizeof(double));
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
            double w = -A->val[e];
            const double *xv = &L->X[(int64_t)A->ci[e] * K];
            s0[u] += w;
            for (int k = 0; k < K; k++) {
                s1[u * K + k] += w * xv[k];
                s2[u * K + k] += w * xv[k] * xv[k];
            }
        }
    }
    for (int64_t u = 0; u < n; u++) { L->status[u] = ST_UNDECIDED; L->seed_of[u] = -1; }
    for (int64_t u = 0; u < n; u++) {
        if (L->status[u] != ST_UNDECIDED) continue;
        int32_t best = -1;
        double bestc = -1.0;
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
            int32_t s = A->ci[e];
            if (!L->strong[e]) continue;
            if (L->status[s] == ST_ASSOC) continue;
            double q = oracle_guard_q(&s0[u], &s1[u * K], &s2[u * K], &L->X[(int64_t)s * K], K, o->guard_eps);
            if (!(q <= o->Q)) continue;
            double c = L->aff[e];
            if (c > bestc || (c == bestc && s < best)) { bestc = c; best = s; }
        }
        if (best >= 0) {
            if (L->status[best] == ST_UNDECIDED) { L->status[best] = ST_SEED; L->seed_of[best] = best; }
            L->status[u] = ST_ASSOC;
            L->seed_of[u] = best;
        }
    }
    for (int64_t u = 0; u < n; u++)
        if (L->status[u] == ST_UNDECIDED) { L->status[u] = ST_SEED; L->seed_of[u] = (int32_t)u; }
    int32_t *id = xcalloc(n, sizeof(int32_t));
    int64_t nc = 0;
    for (int64_t u = 0; u < n; u++) id[u] = (L->status[u] == ST_SEED) ? (int32_t)nc++ : -1;
    L->nc = nc;
    L->agg = xcalloc(n, sizeof(int32_t));
    L->agg2 = xcalloc(n, sizeof(int32_t));
    L->wt = xcalloc(n, sizeof(double));
    for (int64_t u = 0; u < n; u++) { L->agg[u] = id[L->seed_of[u]]; L->agg2[u] = -1; L->wt[u] = 1.0; }
    free(id); free(s0); free(s1); free(s2);
}

/* Selective caliber-2 (Section 3.2, Appendix A.2, Eq. 13). For a non-seed node u whose strong
 * edges reach exactly two aggregates (its own a and one other b), fit
 * w* = sum_k d_k e_k / sum_k d_k^2 with d_k = x_a - x_b, e_k = x_u - x_b, where x_a, x_b are the
 * test-vector values at the aggregates' seeds (reading). Values within `snap` of 0 or 1 snap
 * to it; the row is upgraded iff 0 <= w <= 1 (w == 1 leaves it caliber-1). */
static int64_t caliber2(Level *L, const Opts *o) {
    const Mat *A = &L->A;
    int K = o->K;
    int64_t nup = 0;
    for (int64_t u = 0; u < A->n; u++) {
        if (L->status[u] != ST_ASSOC) continue;
        int32_t a = L->agg[u], b = -1;
        int many = 0;
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
            if (!L->strong[e]) continue;
            int32_t g = L->agg[A->ci[e]];
            if (g == a) continue;
            if (b < 0) b = g;
            else if (g != b) { many = 1; break; }
        }
        if (many || b < 0) continue;
        /* seeds of a and b */
        int32_t sa = L->seed_of[u], sb = -1;
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
            if (L->strong[e] && L->agg[A->ci[e]] == b) { sb = L->seed_of[A->ci[e]]; break; }
        }
        const double *xu = &L->X[u * K], *xa = &L->X[(int64_t)sa * K], *xb = &L->X[(int64_t)sb * K];
        double num = 0.0, den = 0.0;
        for (int k = 0; k < K; k++) {
            double d = xa[k] - xb[k], ee = xu[k] - xb[k];
            num += d * ee;
            den += d * d;
        }
        if (!(den > 0.0)) continue;
        double w = num / den;
        if (fabs(w) <= o->snap) w = 0.0;
        if (fabs(w - 1.0) <= o->snap) w = 1.0;
        if (!(w >= 0.0 && w <= 1.0) || w == 1.0) continue;
        L->agg2[u] = b;
        L->wt[u] = w;
        nup++;
    }
    return nup;
}

/* ------------------------------------------------------------------ Galerkin */

/* P row u as (column, value) pairs; returns the count (1 or 2). */
static int prow(const Level *L, int64_t u, int32_t *c, double *p) {
    if (L->agg2[u] < 0) { c[0] = L->agg[u]; p[0] = 1.0; return 1; }
    int k = 0;
    if (L->wt[u] != 0.0) { c[k] = L->agg[u]; p[k] = L->wt[u]; k++; }
    c[k] = L->agg2[u]; p[k] = 1.0 - L->wt[u]; k++;
    return k;
}

/* Galerkin coarse operator A^c = P^T A P (Section 2), row by row of A^c:
 * A^c_AB = sum_{u,v} P_uA A_uv P_vB over the fine rows u interpolating from A. */
static void galerkin(const Level *L, Mat *Ac) {
    const Mat *A = &L->A;
    int64_t n = A->n, nc = L->nc;
    /* P^T as lists of fine rows per aggregate */
    int64_t *pp = xcalloc(nc + 1, sizeof(int64_t));
    for (int64_t u = 0; u < n; u++) {
        int32_t c[2]; double p[2];
        int k = prow(L, u, c, p);
        for (int t = 0; t < k; t++) pp[c[t] + 1]++;
    }
    for (int64_t a = 0; a < nc; a++) pp[a + 1] += pp[a];
    int32_t *pu = xcalloc(pp[nc], sizeof(int32_t));
    double *pw = xcalloc(pp[nc], sizeof(double));
    int64_t *fill = xcalloc(nc + 1, sizeof(int64_t));
    for (int64_t a = 0; a <= nc; a++) fill[a] = pp[a];
    for (int64_t u = 0; u < n; u++) {
        int32_t c[2]; double p[2];
        int k = prow(L, u, c, p);
        for (int t = 0; t < k; t++) { pu[fill[c[t]]] = (int32_t)u; pw[fill[c[t]]] = p[t]; fill[c[t]]++; }
    }
    Builder B; bld_init(&B, nc, A->nnz);
    double *acc = xcalloc(nc, sizeof(double));
    int32_t *mark = xcalloc(nc, sizeof(int32_t));
    int32_t *touched = xcalloc(nc, sizeof(int32_t));
    for (int64_t j = 0; j < nc; j++) mark[j] = -1;
    for (int64_t a = 0; a < nc; a++) {
        int nt = 0;
        for (int64_t t = pp[a]; t < pp[a + 1]; t++) {
            int64_t u = pu[t];
            double pa = pw[t];
            /* diagonal entry of row u */
            {
                int32_t c[2]; double p[2];
                int k = prow(L, u, c, p);
                for (int s = 0; s < k; s++) {
                    int32_t j = c[s];
                    if (mark[j] != a) { mark[j] = (int32_t)a; acc[j] = 0.0; touched[nt++] = j; }
                    acc[j] += pa * A->diag[u] * p[s];
                }
            }
            for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
                int32_t c[2]; double p[2];
                int k = prow(L, A->ci[e], c, p);
                for (int s = 0; s < k; s++) {
                    int32_t j = c[s];
                    if (mark[j] != a) { mark[j] = (int32_t)a; acc[j] = 0.0; touched[nt++] = j; }
                    acc[j] += pa * A->val[e] * p[s];
                }
            }
        }
        qsort(touched, nt, sizeof(int32_t), cmp_i32);
        double d = 0.0;
        for (int t = 0; t < nt; t++) {
            int32_t j = touched[t];
            if (j == a) { d = acc[j]; continue; }
            if (acc[j] != 0.0) bld_push(&B, j, acc[j]);
        }
        B.diag[a] = d;
        B.rp[a + 1] = B.nnz;
    }
    bld_finish(&B, Ac);
    free(pp); free(pu); free(pw); free(fill); free(acc); free(mark); free(touched);
}

/* ------------------------------------------------------------------ coarsest level */

/* Dense pseudo-inverse of a connected level's operator: for a symmetric positive semidefinite
 * A with null space span{1}, A + J/n is nonsingular and A^+ = (A + J/n)^{-1} - J/n
 * (J = 1 1^T). The inverse comes from a Cholesky factorisation. */
static int coarsest_pinv(Level *L) {
    const Mat *A = &L->A;
    int64_t n = A->n;
    double *M = xcalloc(n * n, sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        M[i * n + i] = A->diag[i];
        for (int64_t e = A->rp[i]; e < A->rp[i + 1]; e++) M[i * n + A->ci[e]] += A->val[e];
    }
    for (int64_t i = 0; i < n * n; i++) M[i] += 1.0 / (double)n;
    /* Cholesky M = R^T R, R upper triangular stored in M's upper part */
    for (int64_t j = 0; j < n; j++) {
        double s = M[j * n + j];
        for (int64_t k = 0; k < j; k++) s -= M[k * n + j] * M[k * n + j];
        if (!(s > 0.0)) { free(M); return ERR_DISCONNECTED; }
        double rjj = sqrt(s);
        M[j * n + j] = rjj;
        for (int64_t i = j + 1; i < n; i++) {
            double t = M[j * n + i];
            for (int64_t k = 0; k < j; k++) t -= M[k * n + j] * M[k * n + i];
            M[j * n + i] = t / rjj;
        }
    }
    /* columns of M^{-1}: solve R^T y = e_c, R x = y */
    L->pinv = xcalloc(n * n, sizeof(double));
    double *y = xcalloc(n, sizeof(double));
    for (int64_t c = 0; c < n; c++) {
        for (int64_t i = 0; i < n; i++) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int64_t k = 0; k < i; k++) t -= M[k * n + i] * y[k];
            y[i] = t / M[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; i--) {
            double t = y[i];
            for (int64_t k = i + 1; k < n; k++) t -= M[i * n + k] * L->pinv[k * n + c];
            L->pinv[i * n + c] = t / M[i * n + i];
        }
    }
    for (int64_t i = 0; i < n * n; i++) L->pinv[i] -= 1.0 / (double)n;
    free(y); free(M);
    return OK;
}

/* ------------------------------------------------------------------ hierarchy */

static void fill_opts(Opts *o, const int64_t *iopt, const double *dopt) {
    o->K = (int)iopt[0]; o->nu_tv = (int)iopt[1]; o->dmax = (int)iopt[2];
    o->nu_pre = (int)iopt[3]; o->nu_post = (int)iopt[4]; o->coarsest_max = (int)iopt[5];
    o->max_levels = (int)iopt[6]; o->veto = (int)iopt[7]; o->caliber2 = (int)iopt[8];
    o->tv_lex = (int)iopt[9]; o->symmetric = (int)iopt[10]; o->seed = (uint64_t)iopt[11];
    o->dense_rows = (int)iopt[12];
    o->cheb_colours = (int)iopt[13]; o->cheb_degree = (int)iopt[14];
    o->Q = dopt[0]; o->tau_soc = dopt[1]; o->elim_min_frac = dopt[2]; o->snap = dopt[3];
    o->guard_eps = dopt[4]; o->gamma_fixed = dopt[5];
}

static void mat_copy(Mat *dst, int64_t n, const int64_t *rp, const int32_t *ci, const double *val, const double *diag) {
    dst->n = n; dst->nnz = rp[n];
    dst->rp = xcalloc(n + 1, sizeof(int64_t)); memcpy(dst->rp, rp, (n + 1) * sizeof(int64_t));
    dst->ci = xcalloc(dst->nnz, sizeof(int32_t)); memcpy(dst->ci, ci, dst->nnz * sizeof(int32_t));
    dst->val = xcalloc(dst->nnz, sizeof(double)); memcpy(dst->val, val, dst->nnz * sizeof(double));
    dst->diag = xcalloc(n, sizeof(double)); memcpy(dst->diag, diag, n * sizeof(double));
}

/* Graph Laplacian of a weighted graph given as symmetric adjacency (Eq. 1). Validates the
 * input: no self loops, positive finite weights, sorted columns, symmetric. */
static int laplacian_from_graph(int64_t n, const int64_t *rp, const int32_t *ci, const double *w, Mat *A) {
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            if (ci[e] < 0 || ci[e] >= n || ci[e] == u) return ERR_INVALID;
            if (!(w[e] > 0.0) || !isfinite(w[e])) return ERR_INVALID;
            if (e > rp[u] && ci[e] <= ci[e - 1]) return ERR_INVALID;
        }
    }
    /* symmetry: find the mirrored entry by binary search */
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            int32_t v = ci[e];
            int64_t lo = rp[v], hi = rp[v + 1] - 1, f = -1;
            while (lo <= hi) {
                int64_t mid = (lo + hi) / 2;
                if (ci[mid] == u) { f = mid; break; }
                if (ci[mid] < u) lo = mid + 1; else hi = mid - 1;
            }
            if (f < 0 || w[f] != w[e]) return ERR_INVALID;
        }
    }
    A->n = n; A->nnz = rp[n];
    A->rp = xcalloc(n + 1, sizeof(int64_t)); memcpy(A->rp, rp, (n + 1) * sizeof(int64_t));
    A->ci = xcalloc(A->nnz, sizeof(int32_t)); memcpy(A->ci, ci, A->nnz * sizeof(int32_t));
    A->val = xcalloc(A->nnz, sizeof(double));
    A->diag = xcalloc(n, sizeof(double));
    for (int64_t u = 0; u < n; u++) {
        double d = 0.0;
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) { A->val[e] = -w[e]; d += w[e]; }
        A->diag[u] = d;
    }
    return OK;
}

static int connected(const Mat *A) {
    int64_t n = A->n;
    if (n == 0) return 0;
    uint8_t *seen = xcalloc(n, 1);
    int32_t *stack = xcalloc(n, sizeof(int32_t));
    int64_t top = 0, cnt = 1;
    stack[top++] = 0; seen[0] = 1;
    while (top) {
        int32_t u = stack[--top];
        for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
            int32_t v = A->ci[e];
            if (!seen[v]) { seen[v] = 1; stack[top++] = v; cnt++; }
        }
    }
    free(seen); free(stack);
    return cnt == n;
}

static void alloc_vectors(Level *L) {
    int64_t n = L->A.n;
    L->x = xcalloc(n, sizeof(double));
    L->b = xcalloc(n, sizeof(double));
    L->r = xcalloc(n, sizeof(double));
}

/* Cycle index of an aggregation level (Eq. 5): 1.5 while |E_l| > 0.1 |E|, otherwise
 * min(2, 0.7 / tau_l) with tau_l = |E_{l+1}| / |E_l|. Reading: clamped below at 1, so
 * every visit of a level visits the next one at least once. */
static double gamma_rule(int64_t El, int64_t El1, int64_t E0) {
    if ((double)El > 0.1 * (double)E0) return 1.5;
    double g = 2.0;
    if (El > 0 && El1 > 0) {
        double tau = (double)El1 / (double)El;
        g = 0.7 / tau;
        if (g > 2.0) g = 2.0;
    }
    if (g < 1.0) g = 1.0;
    return g;
}

static void level_free(Level *L) {
    mat_free(&L->A);
    free(L->colour); free(L->cptr); free(L->corder); free(L->cidx); free(L->cnode);
    free(L->agg); free(L->agg2); free(L->wt); free(L->seed_of); free(L->status);
    free(L->X); free(L->aff); free(L->strong); free(L->pinv);
    free(L->x); free(L->b); free(L->r);
}

void oracle_free(Hier *H) {
    if (!H) return;
    for (int l = 0; l < H->nlev; l++) level_free(&H->lv[l]);
    free(H->lv);
    free(H);
}

/* Build the hierarchy (Section 2): alternate low-degree elimination (kept while it removes
 * at least elim_min_frac of the nodes) and guarded aggregation, until the level has at most
 * coarsest_max nodes. Readings: a level whose aggregation removes fewer than 10% of its
 * nodes and has at most 4096 nodes becomes the coarsest; so does a level with at most
 * dense_rows nodes and at least n^2/8 off-diagonal entries (the paper leaves the size of the
 * directly solved level open: a dense level costs one dense solve instead of a sweep per
 * colour class); otherwise coarsening continues while it makes progress; at most max_levels
 * levels. */
int oracle_setup(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                 const int64_t *iopt, const double *dopt, Hier **out) {
    *out = NULL;
    Hier *H = xcalloc(1, sizeof(Hier));
    fill_opts(&H->o, iopt, dopt);
    const Opts *o = &H->o;
    if (o->K < 1 || o->K > 16 || o->max_levels < 1) { free(H); return ERR_INVALID; }
    H->lv = xcalloc(o->max_levels + 1, sizeof(Level));
    Mat A;
    int rc = laplacian_from_graph(n, rp, ci, w, &A);
    if (rc) { free(H->lv); free(H); return rc; }
    if (!connected(&A)) { mat_free(&A); free(H->lv); free(H); return ERR_DISCONNECTED; }
    H->E0 = A.nnz / 2;
    /* coarsest size: given, or the largest n whose dense matrix (8 n^2 bytes) is about the size
     * of the input operator: floor(sqrt(1.5 nnz(L))), nnz(L) = n + 2m, within [1024, 4096] */
    int64_t cmax = o->coarsest_max;
    if (cmax <= 0) {
        cmax = (int64_t)floor(sqrt(1.5 * (double)(A.n + A.nnz)));
        if (cmax < 1024) cmax = 1024;
        if (cmax > 4096) cmax = 4096;
    }
    int l = 0;
    for (;;) {
        Level *L = &H->lv[l];
        L->A = A;
        alloc_vectors(L);
        H->nlev = l + 1;
        const int dense = A.n <= o->dense_rows && (double)A.nnz >= (double)A.n * (double)A.n / 8.0;
        if (A.n <= cmax || dense || l + 1 >= o->max_levels) {
            L->kind = LV_COARSEST;
            if (A.n > 4096) { oracle_free(H); return ERR_SETUP; }
            rc = coarsest_pinv(L);
            if (rc) { oracle_free(H); return rc; }
            break;
        }
        uint8_t *inF = xcalloc(A.n, 1);
        int64_t nf = select_F(&A, o->dmax, inF);
        Mat Ac;
        if (nf > 0 && (double)nf >= o->elim_min_frac * (double)A.n) {
            L->kind = LV_ELIM;
            eliminate(&A, inF, L, &Ac);
            free(inF);
        } else {
            free(inF);
            L->kind = LV_AGG;
            colour_level(L);
            if (o->cheb_colours > 0 && L->ncol > o->cheb_colours) {
                L->cheb = 1;
                cheb_coefficients(L, o->cheb_degree);
            }
            test_vectors(L, o, l);
            affinity_and_veto(L, o);
            aggregate(L, o);
            if (o->caliber2) caliber2(L, o);
            if (L->nc >= A.n || ((double)L->nc > 0.9 * (double)A.n && A.n <= 4096)) {
                /* no useful coarsening: this level is the coarsest */
                free(L->agg); free(L->agg2); free(L->wt); L->agg = L->agg2 = NULL; L->wt = NULL;
                L->kind = LV_COARSEST;
                if (A.n > 4096) { oracle_free(H); return ERR_SETUP; }
                rc = coarsest_pinv(L);
                if (rc) { oracle_free(H); return rc; }
                break;
            }
            galerkin(L, &Ac);
        }
        A = Ac;
        l++;
    }
    /* cycle indices */
    for (int k = 0; k < H->nlev; k++) {
        Level *L = &H->lv[k];
        if (L->kind == LV_ELIM) L->gamma = 1.0;
        else if (L->kind == LV_AGG) {
            if (o->gamma_fixed > 0) L->gamma = o->gamma_fixed;
            else L->gamma = gamma_rule(L->A.nnz / 2, H->lv[k + 1].A.nnz / 2, H->E0);
        } else L->gamma = 0.0;
    }
    *out = H;
    return OK;
}

/* ------------------------------------------------------------------ cycle */

/* One visit of level l (Section 2 "Cycle and acceleration"; Eq. 2 for elimination levels).
 * first != 0: the level's iterate starts at zero; otherwise it continues from its value.
 * Aggregation level: nu_pre forward-colour GS sweeps, residual, restriction b^c = P^T r,
 * floor((j+1) gamma) - floor(j gamma) visits of the next level at this level's j-th visit
 * (reading of a fractional gamma), correction x += P x^c, nu_post reverse-colour sweeps.
 * Elimination level: b^c = b_C + P_F^T b_F, one visit of the next level, then
 * x_C = x^c and x_F = P_F x_C + A_FF^{-1} b_F with P_F = -A_FF^{-1} A_FC.
 * Coarsest: x = A^+ b followed by the mean-zero projection. */
static void visit(Hier *H, int l, int first) {
    Level *L = &H->lv[l];
    const Mat *A = &L->A;
    int64_t n = A->n;
    L->nvisits++;
    if (L->kind == LV_COARSEST) {
        for (int64_t i = 0; i < n; i++) {
            double s = 0.0;
            for (int64_t j = 0; j < n; j++) s += L->pinv[i * n + j] * L->b[j];
            L->x[i] = s;
        }
        project_mean(L->x, n);
        return;
    }
    Level *C = &H->lv[l + 1];
    if (L->kind == LV_ELIM) {
        for (int64_t i = 0; i < L->nc; i++) C->b[i] = L->b[L->cnode[i]];
        for (int64_t f = 0; f < n; f++) {
            if (L->cidx[f] >= 0) continue;
            for (int64_t e = A->rp[f]; e < A->rp[f + 1]; e++) {
                double pf = -A->val[e] / A->diag[f];     /* (P_F)_{f,c} */
                C->b[L->cidx[A->ci[e]]] += pf * L->b[f];
            }
        }
        if (first) memset(C->x, 0, C->A.n * sizeof(double));
        visit(H, l + 1, first);
        for (int64_t u = 0; u < n; u++) {
            if (L->cidx[u] >= 0) { L->x[u] = C->x[L->cidx[u]]; continue; }
            double s = 0.0;
            for (int64_t e = A->rp[u]; e < A->rp[u + 1]; e++) {
                double pf = -A->val[e] / A->diag[u];
                s += pf * C->x[L->cidx[A->ci[e]]];
            }
            L->x[u] = s + L->b[u] / A->diag[u];
        }
        return;
    }
    /* aggregation level */
    const Opts *o = &H->o;
    double *cd = NULL, *cx = NULL;
    if (L->cheb) { cd = xcalloc(n, sizeof(double)); cx = xcalloc(n, sizeof(double)); }
    if (first) memset(L->x, 0, n * sizeof(double));
    for (int s = 0; s < o->nu_pre; s++) {
        if (L->cheb) cheb_poly(L, L->x, L->b, o->cheb_degree, cd, cx);
        else gs_sweep_colour(L, L->x, L->b, 0);
    }
    residual(A, L->x, L->b, L->r);
    memset(C->b, 0, C->A.n * sizeof(double));
    for (int64_t u = 0; u < n; u++) {
        int32_t c[2]; double p[2];
        int k = prow(L, u, c, p);
        for (int t = 0; t < k; t++) C->b[c[t]] += p[t] * L->r[u];
    }
    int64_t j = L->visits++;
    int64_t nv = (int64_t)floor((double)(j + 1) * L->gamma) - (int64_t)floor((double)j * L->gamma);
    for (int64_t i = 0; i < nv; i++) visit(H, l + 1, i == 0);
    for (int64_t u = 0; u < n; u++) {
        int32_t c[2]; double p[2];
        int k = prow(L, u, c, p);
        double s = 0.0;
        for (int t = 0; t < k; t++) s += p[t] * C->x[c[t]];
        L->x[u] += s;
    }
    for (int s = 0; s < o->nu_post; s++) {
        if (L->cheb) cheb_poly(L, L->x, L->b, o->cheb_degree, cd, cx);
        else gs_sweep_colour(L, L->x, L->b, 1);
    }
    free(cd);
    free(cx);
}

/* The preconditioner: one cycle on A_0 z = r from z = 0, then the mean-zero projection.
 * All visit counters restart at every cycle. */
static void apply_cycle(Hier *H, const double *r, double *z) {
    Level *F = &H->lv[0];
    for (int l = 0; l < H->nlev; l++) { H->lv[l].visits = 0; H->lv[l].nvisits = 0; }
    memcpy(F->b, r, F->A.n * sizeof(double));
    visit(H, 0, 1);
    memcpy(z, F->x, F->A.n * sizeof(double));
    project_mean(z, F->A.n);
}

void oracle_cycle(Hier *H, const double *r, double *z) { apply_cycle(H, r, z); }

/* Flexible preconditioned conjugate gradients with the cycle as preconditioner, Polak-Ribiere
 * form beta = r_{k+1}^T (z_{k+1} - z_k) / (r_k^T z_k) (the solve loop of the B300 design, in
 * place of the paper's iterate recombination). b is projected to mean zero first; the
 * iteration stops when ||r||/||b|| <= tol for the recursively updated residual.
 * hist[i] = ||r_i||/||b|| (i = 0..iters); xs (optional) receives the iterate after each
 * iteration, row-major (iters x n). Returns the iteration count. */
int64_t oracle_fcg(Hier *H, const double *b_in, double *x, double tol, int64_t maxit,
                   double *hist, double *xs) {
    int64_t n = H->lv[0].A.n;
    const Mat *A = &H->lv[0].A;
    double *b = xcalloc(n, sizeof(double)), *r = xcalloc(n, sizeof(double));
    double *z = xcalloc(n, sizeof(double)), *zn = xcalloc(n, sizeof(double));
    double *p = xcalloc(n, sizeof(double)), *q = xcalloc(n, sizeof(double));
    memcpy(b, b_in, n * sizeof(double));
    project_mean(b, n);
    double bn = sqrt(dot(b, b, n));
    memset(x, 0, n * sizeof(double));
    memcpy(r, b, n * sizeof(double));
    int64_t it = 0;
    if (hist) hist[0] = 1.0;
    if (bn == 0.0) goto done;
    apply_cycle(H, r, z);
    memcpy(p, z, n * sizeof(double));
    double rz = dot(r, z, n);
    while (it < maxit) {
        matvec(A, p, q);
        double alpha = rz / dot(p, q, n);
        for (int64_t i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        it++;
        double rel = sqrt(dot(r, r, n)) / bn;
        if (hist) hist[it] = rel;
        if (xs) memcpy(&xs[(it - 1) * n], x, n * sizeof(double));
        if (rel <= tol) break;
        apply_cycle(H, r, zn);
        double num = 0.0;
        for (int64_t i = 0; i < n; i++) num += r[i] * (zn[i] - z[i]);
        double beta = num / rz;
        rz = dot(r, zn, n);
        for (int64_t i = 0; i < n; i++) p[i] = zn[i] + beta * p[i];
        memcpy(z, zn, n * sizeof(double));
    }
done:
    free(b); free(r); free(z); free(zn); free(p); free(q);
    return it;
}

/* Stationary iteration x <- x + M(b - A x) with the finest-level min-residual recombination
 * of Section 2 over the last kappa iterates: alpha = argmin || r - A E alpha ||,
 * E = [x_1 - x, ..., x_kappa - x], x <- x + E alpha (kappa = 0: no recombination).
 * hist[i] = ||b - A x_i||/||b||. xs (optional, 2 maxit x n) receives, for cycle i, the
 * iterate after the cycle's correction (row 2i) and the recombined iterate that is saved,
 * before the mean-zero projection (row 2i + 1). Returns the number of cycles. */
int64_t oracle_stationary(Hier *H, const double *b_in, double *x, double tol, int64_t maxit,
                          int kappa, double *hist, double *xs) {
    int64_t n = H->lv[0].A.n;
    const Mat *A = &H->lv[0].A;
    double *b = xcalloc(n, sizeof(double)), *r = xcalloc(n, sizeof(double));
    double *z = xcalloc(n, sizeof(double));
    double *saved = xcalloc((size_t)(kappa > 0 ? kappa : 1) * n, sizeof(double));
    double *E = xcalloc((size_t)(kappa > 0 ? kappa : 1) * n, sizeof(double));
    double *AE = xcalloc((size_t)(kappa > 0 ? kappa : 1) * n, sizeof(double));
    int nsaved = 0;
    memcpy(b, b_in, n * sizeof(double));
    project_mean(b, n);
    double bn = sqrt(dot(b, b, n));
    memset(x, 0, n * sizeof(double));
    if (hist) hist[0] = 1.0;
    int64_t it = 0;
    while (it < maxit && bn > 0.0) {
        residual(A, x, b, r);
        apply_cycle(H, r, z);
        for (int64_t i = 0; i < n; i++) x[i] += z[i];
        if (xs) memcpy(&xs[(2 * it) * n], x, n * sizeof(double));
        if (kappa > 0) {
            /* recombine with the saved iterates */
            int m = nsaved;
            if (m > 0) {
                for (int j = 0; j < m; j++) {
                    for (int64_t i = 0; i < n; i++) E[j * n + i] = saved[j * n + i] - x[i];
                    matvec(A, &E[j * n], &AE[j * n]);
                }
                residual(A, x, b, r);
                /* normal equations (AE)^T (AE) alpha = (AE)^T r, solved by Gaussian elimination */
                double G[16 * 16], g[16];
                for (int a = 0; a < m; a++) {
                    g[a] = dot(&AE[a * n], r, n);
                    for (int c = 0; c < m; c++) G[a * m + c] = dot(&AE[a * n], &AE[c * n], n);
                }
                int ok = 1;
                for (int c = 0; c < m && ok; c++) {
                    int piv = c;
                    for (int a = c + 1; a < m; a++) if (fabs(G[a * m + c]) > fabs(G[piv * m + c])) piv = a;
                    if (!(fabs(G[piv * m + c]) > 0.0)) { ok = 0; break; }
                    if (piv != c) {
                        for (int t = 0; t < m; t++) { double s = G[c * m + t]; G[c * m + t] = G[piv * m + t]; G[piv * m + t] = s; }
                        double s = g[c]; g[c] = g[piv]; g[piv] = s;
                    }
                    for (int a = c + 1; a < m; a++) {
                        double f = G[a * m + c] / G[c * m + c];
                        for (int t = c; t < m; t++) G[a * m + t] -= f * G[c * m + t];
                        g[a] -= f * g[c];
                    }
                }
                if (ok) {
                    double al[16];
                    for (int a = m - 1; a >= 0; a--) {
                        double s = g[a];
                        for (int t = a + 1; t < m; t++) s -= G[a * m + t] * al[t];
                        al[a] = s / G[a * m + a];
                    }
                    for (int j = 0; j < m; j++)
                        for (int64_t i = 0; i < n; i++) x[i] += al[j] * E[j * n + i];
                }
            }
            /* save x, dropping the oldest */
            if (nsaved == kappa) {
                memmove(saved, saved + n, (size_t)(kappa - 1) * n * sizeof(double));
                nsaved--;
            }
            memcpy(&saved[nsaved * n], x, n * sizeof(double));
            nsaved++;
        }
        if (xs) memcpy(&xs[(2 * it + 1) * n], x, n * sizeof(double));
        project_mean(x, n);
        residual(A, x, b, r);
        it++;
        double rel = sqrt(dot(r, r, n)) / bn;
        if (hist) hist[it] = rel;
        if (rel <= tol) break;
    }
    free(b); free(r); free(z); free(saved); free(E); free(AE);
    return it;
}

/* ------------------------------------------------------------------ accessors */

int oracle_nlevels(const Hier *H) { return H->nlev; }

/* Override the cycle index of one aggregation level (used by the pins of the visit rule). */
void oracle_set_gamma(Hier *H, int l, double gamma) {
    if (l >= 0 && l < H->nlev && H->lv[l].kind == LV_AGG) H->lv[l].gamma = gamma;
}

/* Visits of each level during the last cycle (apply_cycle restarts the counts). */
void oracle_visit_counts(const Hier *H, int64_t *out) {
    for (int l = 0; l < H->nlev; l++) out[l] = H->lv[l].nvisits;
}

/* meta: kind, n, nnz, ncol, nc, n_caliber2, Chebyshev smoothing; dmeta: gamma, lambda,
 * c1[8], c2[8] */
void oracle_level_meta(const Hier *H, int l, int64_t *meta, double *dmeta) {
    const Level *L = &H->lv[l];
    meta[0] = L->kind; meta[1] = L->A.n; meta[2] = L->A.nnz; meta[3] = L->ncol; meta[4] = L->nc;
    int64_t c2 = 0;
    if (L->kind == LV_AGG) for (int64_t u = 0; u < L->A.n; u++) if (L->agg2[u] >= 0) c2++;
    meta[5] = c2;
    meta[6] = L->cheb;
    dmeta[0] = L->gamma;
    dmeta[1] = L->cheb_lambda;
    for (int k = 0; k < 8; k++) { dmeta[2 + k] = L->cheb_c1[k]; dmeta[10 + k] = L->cheb_c2[k]; }
}

/* Copy a named per-level array into dst; returns the number of elements (0 if absent). */
int64_t oracle_level_array(const Hier *H, int l, const char *name, void *dst) {
    const Level *L = &H->lv[l];
    int64_t n = L->A.n, z = L->A.nnz;
    const void *src = NULL; int64_t cnt = 0; size_t es = 0;
#define SRC(nm, ptr, c, e) if (!strcmp(name, nm)) { src = ptr; cnt = c; es = e; }
    SRC("rp", L->A.rp, n + 1, 8)
    SRC("ci", L->A.ci, z, 4)
    SRC("val", L->A.val, z, 8)
    SRC("diag", L->A.diag, n, 8)
    SRC("colour", L->colour, L->colour ? n : 0, 4)
    SRC("cidx", L->cidx, L->cidx ? n : 0, 4)
    SRC("agg", L->agg, L->agg ? n : 0, 4)
    SRC("agg2", L->agg2, L->agg2 ? n : 0, 4)
    SRC("wt", L->wt, L->wt ? n : 0, 8)
    SRC("seed_of", L->seed_of, L->seed_of ? n : 0, 4)
    SRC("X", L->X, L->X ? n * H->o.K : 0, 8)
    SRC("aff", L->aff, L->aff ? z : 0, 8)
    SRC("strong", L->strong, L->strong ? z : 0, 1)
    SRC("pinv", L->pinv, L->pinv ? n * n : 0, 8)
#undef SRC
    if (src && dst && cnt) memcpy(dst, src, cnt * es);
    return src ? cnt : 0;
}

/* ------------------------------------------------------------------ standalone steps
 * (the same routines, callable on caller-provided matrices for the pin tests) */

int oracle_laplacian(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                     double *val, double *diag) {
    Mat A;
    int rc = laplacian_from_graph(n, rp, ci, w, &A);
    if (rc) return rc;
    memcpy(val, A.val, A.nnz * sizeof(double));
    memcpy(diag, A.diag, n * sizeof(double));
    mat_free(&A);
    return OK;
}

/* Greedy colouring; returns the number of colours. */
int oracle_colour(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *colour) {
    Level L; memset(&L, 0, sizeof(L));
    L.A.n = n; L.A.rp = (int64_t *)rp; L.A.ci = (int32_t *)ci;
    colour_level(&L);
    memcpy(colour, L.colour, n * sizeof(int32_t));
    int nc = L.ncol;
    free(L.colour); free(L.cptr); free(L.corder);
    return nc;
}

/* nsweeps GS sweeps on A x = b (b may be NULL): order 0 forward colours, 1 reverse colours,
 * 2 lexicographic. */
void oracle_gs(int64_t n, const int64_t *rp, const int32_t *ci, const double *val, const double *diag,
               double *x, const double *b, int order, int nsweeps) {
    Level L; memset(&L, 0, sizeof(L));
    L.A.n = n; L.A.nnz = rp[n]; L.A.rp = (int64_t *)rp; L.A.ci = (int32_t *)ci;
    L.A.val = (double *)val; L.A.diag = (double *)diag;
    if (order != 2) colour_level(&L);
    for (int s = 0; s < nsweeps; s++) {
        if (order == 2) gs_sweep_lex(&L.A, x, b);
        else gs_sweep_colour(&L, x, b, order == 1);
    }
    free(L.colour); free(L.cptr); free(L.corder);
}

void oracle_residual(int64_t n, const int64_t *rp, const int32_t *ci, const double *val, const double *diag,
                     const double *x, const double *b, double *r) {
    Mat A = { n, rp[n], (int64_t *)rp, (int32_t *)ci, (double *)val, (double *)diag };
    residual(&A, x, b, r);
}

double oracle_affinity(const double *xu, const double *xv, int K) { return affinity(xu, xv, K); }

/* Elimination step on a caller matrix: fills inF (n), returns |F|; the coarse operator is
 * returned through a temporary level, read back with oracle_mat_get. */
typedef struct { Mat A; } OMat;

int64_t oracle_eliminate(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                         const double *diag, int dmax, uint8_t *inF, OMat **out) {
    Mat A = { n, rp[n], (int64_t *)rp, (int32_t *)ci, (double *)val, (double *)diag };
    int64_t nf = select_F(&A, dmax, inF);
    Level L; memset(&L, 0, sizeof(L));
    OMat *M = xcalloc(1, sizeof(OMat));
    eliminate(&A, inF, &L, &M->A);
    free(L.cidx); free(L.cnode);
    *out = M;
    return nf;
}

/* Galerkin product on caller data (P given by agg, agg2, wt). */
OMat *oracle_galerkin(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                      const double *diag, int64_t nc, const int32_t *agg, const int32_t *agg2,
                      const double *wt) {
    Level L; memset(&L, 0, sizeof(L));
    L.A.n = n; L.A.nnz = rp[n]; L.A.rp = (int64_t *)rp; L.A.ci = (int32_t *)ci;
    L.A.val = (double *)val; L.A.diag = (double *)diag;
    L.nc = nc; L.agg = (int32_t *)agg; L.agg2 = (int32_t *)agg2; L.wt = (double *)wt;
    OMat *M = xcalloc(1, sizeof(OMat));
    galerkin(&L, &M->A);
    return M;
}

/* Dense pseudo-inverse on caller data (connected operator). */
int oracle_pinv(int64_t n, const int64_t *rp, const int32_t *ci, const double *val, const double *diag,
                double *pinv) {
    Level L; memset(&L, 0, sizeof(L));
    L.A.n = n; L.A.nnz = rp[n]; L.A.rp = (int64_t *)rp; L.A.ci = (int32_t *)ci;
    L.A.val = (double *)val; L.A.diag = (double *)diag;
    int rc = coarsest_pinv(&L);
    if (rc == OK) { memcpy(pinv, L.pinv, n * n * sizeof(double)); free(L.pinv); }
    return rc;
}

/* One Chebyshev smoothing polynomial of degree m on A x = b (x updated in place); coef
 * (optional) receives lambda, c1[0..m), c2[0..m). */
void oracle_cheb_apply(int64_t n, const int64_t *rp, const int32_t *ci, const double *val, const double *diag,
                       int m, double *x, const double *b, double *coef) {
    Level L; memset(&L, 0, sizeof(L));
    L.A.n = n; L.A.nnz = rp[n]; L.A.rp = (int64_t *)rp; L.A.ci = (int32_t *)ci;
    L.A.val = (double *)val; L.A.diag = (double *)diag;
    cheb_coefficients(&L, m);
    double *d = xcalloc(n, sizeof(double)), *xn = xcalloc(n, sizeof(double));
    cheb_poly(&L, x, b, m, d, xn);
    free(d); free(xn);
    if (coef) {
        coef[0] = L.cheb_lambda;
        for (int k = 0; k < m && k < 8; k++) { coef[1 + k] = L.cheb_c1[k]; coef[9 + k] = L.cheb_c2[k]; }
    }
}

/* K test vectors (Section 2) of a caller operator in the oracle's greedy colour order: X (n x K)
 * receives nu sweeps on A x = 0 from the random start of (seed, level). */
void oracle_testvectors(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                        const double *diag, int level, uint64_t seed, int K, int nu, double *X) {
    Level L; memset(&L, 0, sizeof(L));
    L.A.n = n; L.A.nnz = rp[n]; L.A.rp = (int64_t *)rp; L.A.ci = (int32_t *)ci;
    L.A.val = (double *)val; L.A.diag = (double *)diag;
    colour_level(&L);
    Opts o; memset(&o, 0, sizeof(o));
    o.K = K; o.nu_tv = nu; o.seed = seed;
    test_vectors(&L, &o, level);
    memcpy(X, L.X, n * K * sizeof(double));
    free(L.X); free(L.colour); free(L.cptr); free(L.corder);
}

/* Caliber-1 aggregation (Section 2) on caller data: operator, K test vectors (n x K), the
 * affinity and strong flag of every off-diagonal entry; seed_of (n) receives the seed node of
 * each node's aggregate. Returns the number of aggregates. */
int64_t oracle_aggregate(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                         const double *diag, const double *X, int K, const double *aff,
                         const uint8_t *strong, double Qb, double guard_eps, int32_t *seed_of) {
    Level L; memset(&L, 0, sizeof(L));
    L.A.n = n; L.A.nnz = rp[n]; L.A.rp = (int64_t *)rp; L.A.ci = (int32_t *)ci;
    L.A.val = (double *)val; L.A.diag = (double *)diag;
    L.X = (double *)X; L.aff = (double *)aff; L.strong = (uint8_t *)strong;
    Opts o; memset(&o, 0, sizeof(o));
    o.K = K; o.Q = Qb; o.guard_eps = guard_eps;
    aggregate(&L, &o);
    memcpy(seed_of, L.seed_of, n * sizeof(int32_t));
    int64_t nc = L.nc;
    free(L.status); free(L.seed_of); free(L.agg); free(L.agg2); free(L.wt);
    return nc;
}

void oracle_mat_meta(const OMat *M, int64_t *nnz_n) { nnz_n[0] = M->A.n; nnz_n[1] = M->A.nnz; }

void oracle_mat_get(const OMat *M, int64_t *rp, int32_t *ci, double *val, double *diag) {
    memcpy(rp, M->A.rp, (M->A.n + 1) * sizeof(int64_t));
    memcpy(ci, M->A.ci, M->A.nnz * sizeof(int32_t));
    memcpy(val, M->A.val, M->A.nnz * sizeof(double));
    memcpy(diag, M->A.diag, M->A.n * sizeof(double));
}

void oracle_mat_free(OMat *M) { if (M) { mat_free(&M->A); free(M); } }
