// Host side of the LAMG+ setup (Section 2): input validation, the Laplacian, low-degree
// elimination (Eq. 2), guarded aggregation (Eqs. 3-4, Appendix B) with the veto (Eq. 9),
// selective caliber-2 (Section 3.2, Eq. 13), Galerkin coarse operators, colouring, the
// cycle index of Eq. 5 and the dense coarsest pseudo-inverse. The test vectors and the
// affinity / veto pass run on the GPU (setup_kernels.cu).
//
// Floating-point expressions are evaluated left to right without contraction (the file is
// compiled with -ffp-contract=off), so that decisions taken from them (guard admissibility,
// affinity maxima, caliber-2 gates) are reproducible.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <condition_variable>
#include <mutex>
#include <thread>

#include "internal.h"

namespace lamg {

// graphs with at least this many stored entries are checked on the GPU
constexpr int64_t GPU_CHECK_MIN = (int64_t)1 << 16;

int validate_graph(const lamg_graph *g) {
    if (!g || g->n < 1 || !g->rp || (g->rp[g->n] > 0 && (!g->ci || !g->w))) return LAMG_ERR_INVALID;
    const int64_t n = g->n;
    if (n >= (int64_t)INT32_MAX) return LAMG_ERR_INVALID;
    if (g->rp[0] != 0) return LAMG_ERR_INVALID;
    for (int64_t u = 0; u < n; u++)
        if (g->rp[u + 1] < g->rp[u]) return LAMG_ERR_INVALID;
    if (g->rp[n] >= GPU_CHECK_MIN) {
        // per-entry checks and symmetry on the GPU, one thread per entry
        bool valid = false;
        const int rc = gpu_validate_entries(g, &valid);
        if (rc) return rc;
        if (!valid) return LAMG_ERR_INVALID;
    } else {
        for (int64_t u = 0; u < n; u++) {
            for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++) {
                int32_t v = g->ci[e];
                if (v < 0 || v >= n || v == u) return LAMG_ERR_INVALID;
                if (e > g->rp[u] && v <= g->ci[e - 1]) return LAMG_ERR_INVALID;
                double w = g->w[e];
                if (!(w > 0.0) || !std::isfinite(w)) return LAMG_ERR_INVALID;
            }
        }
        for (int64_t u = 0; u < n; u++) {
            for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++) {
                int32_t v = g->ci[e];
                const int32_t *b = g->ci + g->rp[v], *end = g->ci + g->rp[v + 1];
                const int32_t *f = std::lower_bound(b, end, (int32_t)u);
                if (f == end || *f != u) return LAMG_ERR_INVALID;
                if (g->w[g->rp[v] + (f - b)] != g->w[e]) return LAMG_ERR_INVALID;
            }
        }
    }
    // connectivity (breadth-first search from node 0)
    std::vector<int32_t> queue(n);
    std::vector<uint8_t> seen(n, 0);
    int64_t head = 0, tail = 0;
    queue[tail++] = 0;
    seen[0] = 1;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++) {
            int32_t v = g->ci[e];
            if (!seen[v]) { seen[v] = 1; queue[tail++] = v; }
        }
    }
    if (tail != n) return LAMG_ERR_DISCONNECTED;
    return LAMG_OK;
}

// L = D - W (Eq. 1).
static void laplacian(const lamg_graph *g, HostMat &A) {
    const int64_t n = g->n, z = g->rp[n];
    A.n = n;
    A.rp.assign(g->rp, g->rp + n + 1);
    A.ci.assign(g->ci, g->ci + z);
    A.val.resize(z);
    A.diag.assign(n, 0.0);
    for (int64_t u = 0; u < n; u++) {
        double d = 0.0;
        for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++) {
            A.val[e] = -g->w[e];
            d += g->w[e];
        }
        A.diag[u] = d;
    }
}

// Greedy colouring: nodes in ascending order take the smallest colour not used by an
// already-coloured neighbour.
int greedy_colour(const HostMat &A, std::vector<int32_t> &colour) {
    const int64_t n = A.n;
    colour.assign(n, -1);
    std::vector<int64_t> used;  // used[c] == u+1 when colour c is taken around u
    int ncol = 0;
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = A.rp[u]; e < A.rp[u + 1]; e++) {
            int32_t c = colour[A.ci[e]];
            if (c < 0) continue;
            if ((int64_t)used.size() <= c) used.resize(c + 1, 0);
            used[c] = u + 1;
        }
        int c = 0;
        while (c < (int)used.size() && used[c] == u + 1) c++;
        colour[u] = c;
        ncol = std::max(ncol, c + 1);
    }
    return ncol;
}

// ----------------------------------------------------------------------------------- elimination

// F: greedy maximal independent set of the nodes of degree <= dmax, ascending order (Eq. 2).
static int64_t pick_F(const HostMat &A, int dmax, std::vector<uint8_t> &inF) {
    const int64_t n = A.n;
    inF.assign(n, 0);
    std::vector<uint8_t> nbrF(n, 0);
    int64_t cnt = 0;
    for (int64_t u = 0; u < n; u++) {
        if (A.rp[u + 1] - A.rp[u] > dmax || nbrF[u]) continue;
        inF[u] = 1;
        cnt++;
        for (int64_t e = A.rp[u]; e < A.rp[u + 1]; e++) nbrF[A.ci[e]] = 1;
    }
    return cnt;
}

// Sparse accumulator for one output row.
int setup_threads() {
    return (int)std::max<unsigned>(1u, std::min<unsigned>(16u, std::thread::hardware_concurrency()));
}

// fn(t, begin, end) on T contiguous chunks of [0, n), one thread each (one thread when n is
// below min_rows per thread). Chunks are in order, so per-chunk outputs concatenated in thread
// order equal a sequential pass.
template <class F>
static void parallel_chunks(int64_t n, int64_t min_rows, F &&fn) {
    const int hw = setup_threads();
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(hw, n / std::max<int64_t>(1, min_rows)));
    if (T == 1) {
        fn(0, (int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < T; t++)
        th.emplace_back([&fn, t, T, n] { fn(t, n * t / T, n * (t + 1) / T); });
    for (auto &x : th) x.join();
}

struct RowAcc {
    std::vector<double> v;
    std::vector<int64_t> stamp;
    std::vector<int32_t> cols;
    int64_t cur = -1;
    explicit RowAcc(int64_t n) : v(n, 0.0), stamp(n, -1) {}
    void start(int64_t row) { cur = row; cols.clear(); }
    double &at(int32_t j) {
        if (stamp[j] != cur) { stamp[j] = cur; v[j] = 0.0; cols.push_back(j); }
        return v[j];
    }
};

// Row i (node u) of the exact Schur complement onto C (Eq. 2): A_uv for the C neighbours v, minus
// A_uv A_vt / A_vv over every F neighbour v and its neighbours t (u's own diagonal for t = u), in
// the order of u's entries and then v's. Appends the row's nonzero off-diagonal entries
// (ascending column) to oc/ov and returns its diagonal.
static double schur_row(const HostMat &A, const std::vector<uint8_t> &inF, const std::vector<int32_t> &cidx,
                        int64_t u, int64_t i, RowAcc &acc, std::vector<int32_t> &oc, std::vector<double> &ov) {
    acc.start(i);
    double d = A.diag[u];
    for (int64_t e = A.rp[u]; e < A.rp[u + 1]; e++) {
        const int32_t v = A.ci[e];
        if (!inF[v]) {
            acc.at(cidx[v]) += A.val[e];
            continue;
        }
        const double avv = A.diag[v], auv = A.val[e];
        for (int64_t f = A.rp[v]; f < A.rp[v + 1]; f++) {
            const int32_t t = A.ci[f];
            const double term = auv * A.val[f] / avv;
            if (t == u) d -= term;
            else acc.at(cidx[t]) -= term;
        }
    }
    std::sort(acc.cols.begin(), acc.cols.end());
    for (int32_t j : acc.cols) {
        if (acc.v[j] == 0.0) continue;
        oc.push_back(j);
        ov.push_back(acc.v[j]);
    }
    return d;
}

// Exact Schur complement onto C (Eq. 2); C keeps ascending node order. Levels of at least
// SCHUR_MIN_ROWS rows form it on the GPU (the same ordered, explicitly rounded sums: the same
// operator), rows the GPU leaves on the setup threads; smaller levels here.
constexpr int64_t SCHUR_MIN_ROWS = 32768;

static int schur(const HostMat &A, const std::vector<uint8_t> &inF, HostLevel &L, HostMat &Ac) {
    const int64_t n = A.n;
    L.cidx.assign(n, -1);
    std::vector<int32_t> cnode;
    for (int64_t u = 0; u < n; u++)
        if (!inF[u]) { L.cidx[u] = (int32_t)cnode.size(); cnode.push_back((int32_t)u); }
    const int64_t nc = (int64_t)cnode.size();
    L.nc = nc;
    if (n >= SCHUR_MIN_ROWS)
        return gpu_schur(A, inF, L.cidx, cnode, Ac,
                         [&](const std::vector<int64_t> &big, std::vector<std::vector<int32_t>> &oc,
                             std::vector<std::vector<double>> &ov, std::vector<double> &od) {
                             parallel_chunks((int64_t)big.size(), 8, [&](int, int64_t i0, int64_t i1) {
                                 RowAcc acc(nc);
                                 for (int64_t i = i0; i < i1; i++)
                                     od[i] = schur_row(A, inF, L.cidx, cnode[big[i]], big[i], acc, oc[i], ov[i]);
                             });
                         });
    Ac.n = nc;
    Ac.rp.assign(nc + 1, 0);
    Ac.diag.assign(nc, 0.0);
    Ac.ci.clear();
    Ac.val.clear();
    Ac.ci.reserve(A.nnz());
    Ac.val.reserve(A.nnz());
    RowAcc acc(nc);
    for (int64_t i = 0; i < nc; i++) {
        Ac.diag[i] = schur_row(A, inF, L.cidx, cnode[i], i, acc, Ac.ci, Ac.val);
        Ac.rp[i + 1] = (int64_t)Ac.ci.size();
    }
    return LAMG_OK;
}

// ----------------------------------------------------------------------------------- aggregation

enum { UNDECIDED = 0, SEED = 1, ASSOCIATE = 2 };

// Energy ratio of Eq. 4 from the moments of Appendix B: per column k,
// relaxed = (s2 - s1^2/s0)/2, forced = (xs^2 s0 - 2 xs s1 + s2)/2, ratio = forced / relaxed,
// maximised over k. The paper divides by the relaxed energy, which vanishes for a node with a
// single neighbour; a relaxed energy <= guard_eps * scale, scale = (|s2| + s1^2/|s0|)/2, counts
// as zero, and the ratio is then 1 if the forced energy is also <= guard_eps * scale, else
// infinite.
static double energy_ratio(double s0, const double *s1, const double *s2, const double *xs,
                           int K, double eps) {
    double worst = 0.0;
    for (int k = 0; k < K; k++) {
        const double relaxed = 0.5 * (s2[k] - s1[k] * s1[k] / s0);
        const double forced = 0.5 * (xs[k] * xs[k] * s0 - 2.0 * xs[k] * s1[k] + s2[k]);
        const double scale = 0.5 * (std::fabs(s2[k]) + s1[k] * s1[k] / std::fabs(s0));
        double r;
        if (relaxed <= eps * scale) r = (forced <= eps * scale) ? 1.0 : INFINITY;
        else r = forced / relaxed;
        worst = std::max(worst, r);
    }
    return worst;
}

// Greedy guarded aggregation in ascending node order; candidates of an undecided node are its
// strong (non-vetoed) neighbours that are seeds or undecided, admissible when the energy
// ratio is <= Q; the node joins the admissible candidate of largest affinity (ties to the
// lower id), which becomes a seed. Leftover undecided nodes are singleton seeds. Aggregates
// are numbered by ascending seed.
static void aggregate(HostLevel &L, const lamg_options &o, std::vector<int32_t> &status,
                      std::vector<int32_t> &seed) {
    const HostMat &A = L.A;
    const int64_t n = A.n;
    const int K = o.K;
    // the guard per entry: from the GPU (L.adm), or the moments and ratios evaluated here
    const bool have_adm = (int64_t)L.adm.size() == A.nnz();
    std::vector<double> s0, s1, s2;
    if (!have_adm) {
        s0.assign(n, 0.0);
        s1.assign(n * K, 0.0);
        s2.assign(n * K, 0.0);
        for (int64_t u = 0; u < n; u++) {
            for (int64_t e = A.rp[u]; e < A.rp[u + 1]; e++) {
                const double w = -A.val[e];
                const double *xv = &L.X[(int64_t)A.ci[e] * K];
                s0[u] += w;
                for (int k = 0; k < K; k++) {
                    s1[u * K + k] += w * xv[k];
                    s2[u * K + k] += w * xv[k] * xv[k];
                }
            }
        }
    }
    status.assign(n, UNDECIDED);
    seed.assign(n, -1);
    for (int64_t u = 0; u < n; u++) {
        if (status[u] != UNDECIDED) continue;
        int32_t pick = -1;
        double pick_aff = -1.0;
        for (int64_t e = A.rp[u]; e < A.rp[u + 1]; e++) {
            const int32_t s = A.ci[e];
            if (!L.strong[e] || status[s] == ASSOCIATE) continue;
            if (have_adm) {
                if (!L.adm[e]) continue;
            } else {
                const double q = energy_ratio(s0[u], &s1[u * K], &s2[u * K], &L.X[(int64_t)s * K], K,
                                              o.guard_eps);
                if (!(q <= o.Q)) continue;
            }
            const double c = L.aff[e];
            if (c > pick_aff || (c == pick_aff && s < pick)) { pick_aff = c; pick = s; }
        }
        if (pick < 0) continue;
        if (status[pick] == UNDECIDED) { status[pick] = SEED; seed[pick] = pick; }
        status[u] = ASSOCIATE;
        seed[u] = pick;
    }
    for (int64_t u = 0; u < n; u++)
        if (status[u] == UNDECIDED) { status[u] = SEED; seed[u] = (int32_t)u; }
    std::vector<int32_t> id(n, -1);
    int64_t nc = 0;
    for (int64_t u = 0; u < n; u++)
        if (status[u] == SEED) id[u] = (int32_t)nc++;
    L.nc = nc;
    L.agg.resize(n);
    L.agg2.assign(n, -1);
    L.wt.assign(n, 1.0);
    for (int64_t u = 0; u < n; u++) L.agg[u] = id[seed[u]];
}

// The aggregates of the GPU pass (choice[u]: the seed u joined, or -1: u is a seed), numbered by
// ascending seed as aggregate() numbers them.
static void aggregate_from_choice(HostLevel &L, const std::vector<int32_t> &choice, std::vector<int32_t> &status,
                                  std::vector<int32_t> &seed) {
    const int64_t n = L.A.n;
    status.assign(n, SEED);
    seed.resize(n);
    std::vector<int32_t> id(n, -1);
    int64_t nc = 0;
    for (int64_t u = 0; u < n; u++) {
        if (choice[u] >= 0) {
            status[u] = ASSOCIATE;
            seed[u] = choice[u];
        } else {
            seed[u] = (int32_t)u;
            id[u] = (int32_t)nc++;
        }
    }
    L.nc = nc;
    L.agg.resize(n);
    L.agg2.assign(n, -1);
    L.wt.assign(n, 1.0);
    for (int64_t u = 0; u < n; u++) L.agg[u] = id[seed[u]];
}

// Selective caliber-2 (Section 3.2, Eq. 13): a non-seed node whose strong edges reach exactly
// one aggregate b besides its own a gets phi_u = w phi_a + (1-w) phi_b with the least-squares
// weight over the test vectors taken at the two seeds, snapped to 0/1 within `snap`, kept
// iff 0 <= w < 1.
static void upgrade_caliber2(HostLevel &L, const lamg_options &o, const std::vector<int32_t> &status,
                             const std::vector<int32_t> &seed) {
    const HostMat &A = L.A;
    const int K = o.K;
    for (int64_t u = 0; u < A.n; u++) {
        if (status[u] != ASSOCIATE) continue;
        const int32_t a = L.agg[u];
        int32_t b = -1, sb = -1;
        bool more = false;
        for (int64_t e = A.rp[u]; e < A.rp[u + 1] && !more; e++) {
            if (!L.strong[e]) continue;
            const int32_t v = A.ci[e];
            const int32_t gv = L.agg[v];
            if (gv == a) continue;
            if (b < 0) { b = gv; sb = seed[v]; }
            else if (gv != b) more = true;
        }
        if (more || b < 0) continue;
        const double *xu = &L.X[u * K];
        const double *xa = &L.X[(int64_t)seed[u] * K];
        const double *xb = &L.X[(int64_t)sb * K];
        double num = 0.0, den = 0.0;
        for (int k = 0; k < K; k++) {
            const double d = xa[k] - xb[k], e = xu[k] - xb[k];
            num += d * e;
            den += d * d;
        }
        if (!(den > 0.0)) continue;
        double w = num / den;
        if (std::fabs(w) <= o.snap) w = 0.0;
        if (std::fabs(w - 1.0) <= o.snap) w = 1.0;
        if (!(w >= 0.0 && w < 1.0)) continue;
        L.agg2[u] = b;
        L.wt[u] = w;
    }
}

// Entries of P's row u.
static inline int p_row(const HostLevel &L, int64_t u, int32_t *col, double *p) {
    if (L.agg2[u] < 0) { col[0] = L.agg[u]; p[0] = 1.0; return 1; }
    int k = 0;
    if (L.wt[u] != 0.0) { col[k] = L.agg[u]; p[k] = L.wt[u]; k++; }
    col[k] = L.agg2[u];
    p[k] = 1.0 - L.wt[u];
    return k + 1;
}

// P^T by coarse row: for aggregate a, the fine rows u with P_ua != 0 in ascending order
// (rows[ptr[a] .. ptr[a + 1])) and their weights P_ua (pw).
void galerkin_pt(const HostLevel &L, std::vector<int64_t> &ptr, std::vector<int32_t> &rows,
                 std::vector<double> &pw) {
    const int64_t n = L.A.n, nc = L.nc;
    ptr.assign(nc + 1, 0);
    for (int64_t u = 0; u < n; u++) {
        int32_t c[2]; double p[2];
        int k = p_row(L, u, c, p);
        for (int t = 0; t < k; t++) ptr[c[t] + 1]++;
    }
    for (int64_t a = 0; a < nc; a++) ptr[a + 1] += ptr[a];
    rows.resize(ptr[nc]);
    pw.resize(ptr[nc]);
    std::vector<int64_t> pos(ptr.begin(), ptr.end() - 1);
    for (int64_t u = 0; u < n; u++) {
        int32_t c[2]; double p[2];
        int k = p_row(L, u, c, p);
        for (int t = 0; t < k; t++) { rows[pos[c[t]]] = (int32_t)u; pw[pos[c[t]]] = p[t]; pos[c[t]]++; }
    }
}

// Row a of the Galerkin coarse operator P^T A P: every product P_ua A_uv P_vb (u over the fine
// rows of a ascending, v over u's diagonal then u's entries in order, b over v's row of P) is
// added to entry b in that order. Appends the row's nonzero off-diagonal entries (ascending
// column) to oc/ov and returns its diagonal.
static double galerkin_row(const HostLevel &L, const std::vector<int64_t> &ptr, const std::vector<int32_t> &rows,
                           const std::vector<double> &pw, int64_t a, RowAcc &acc, std::vector<int32_t> &oc,
                           std::vector<double> &ov) {
    const HostMat &A = L.A;
    acc.start(a);
    for (int64_t q = ptr[a]; q < ptr[a + 1]; q++) {
        const int64_t u = rows[q];
        const double pa = pw[q];
        int32_t c[2]; double p[2];
        int k = p_row(L, u, c, p);
        for (int s = 0; s < k; s++) acc.at(c[s]) += pa * A.diag[u] * p[s];
        for (int64_t e = A.rp[u]; e < A.rp[u + 1]; e++) {
            k = p_row(L, A.ci[e], c, p);
            for (int s = 0; s < k; s++) acc.at(c[s]) += pa * A.val[e] * p[s];
        }
    }
    std::sort(acc.cols.begin(), acc.cols.end());
    double d = 0.0;
    for (int32_t j : acc.cols) {
        if (j == a) { d = acc.v[j]; continue; }
        if (acc.v[j] == 0.0) continue;
        oc.push_back(j);
        ov.push_back(acc.v[j]);
    }
    return d;
}

// Galerkin coarse operator P^T A P on the host, coarse rows in contiguous chunks on up to 16
// threads, each row summed by one thread as in a sequential pass.
static void galerkin(const HostLevel &L, HostMat &Ac) {
    const int64_t nc = L.nc;
    std::vector<int64_t> ptr;
    std::vector<int32_t> rows;
    std::vector<double> pw;
    galerkin_pt(L, ptr, rows, pw);
    Ac.n = nc;
    Ac.rp.assign(nc + 1, 0);
    Ac.diag.assign(nc, 0.0);
    Ac.ci.clear();
    Ac.val.clear();
    std::vector<std::vector<int32_t>> tci(16);
    std::vector<std::vector<double>> tval(16);
    std::vector<int64_t> len(nc, 0);
    parallel_chunks(nc, 65536, [&](int t, int64_t a0, int64_t a1) {
        RowAcc acc(nc);
        std::vector<int32_t> &oc = tci[t];
        std::vector<double> &ov = tval[t];
        for (int64_t a = a0; a < a1; a++) {
            const size_t before = oc.size();
            Ac.diag[a] = galerkin_row(L, ptr, rows, pw, a, acc, oc, ov);
            len[a] = (int64_t)(oc.size() - before);
        }
    });
    for (int64_t a = 0; a < nc; a++) Ac.rp[a + 1] = Ac.rp[a] + len[a];
    Ac.ci.reserve(Ac.rp[nc]);
    Ac.val.reserve(Ac.rp[nc]);
    for (int t = 0; t < 16; t++) {
        Ac.ci.insert(Ac.ci.end(), tci[t].begin(), tci[t].end());
        Ac.val.insert(Ac.val.end(), tval[t].begin(), tval[t].end());
    }
}

// Galerkin on the GPU (same sums, same order, explicitly rounded: the same coarse operator),
// with the rows the GPU leaves (more distinct coarse columns than its per-row accumulator
// holds) summed here; levels below GAL_MIN_ROWS fine rows stay on the host.
constexpr int64_t GAL_MIN_ROWS = 32768;
static int galerkin_device(const HostLevel &L, HostMat &Ac) {
    if (L.A.n < GAL_MIN_ROWS) {  // uploads and launches cost more than the host sums
        galerkin(L, Ac);
        return LAMG_OK;
    }
    std::vector<int64_t> ptr;
    std::vector<int32_t> rows;
    std::vector<double> pw;
    galerkin_pt(L, ptr, rows, pw);
    // the rows the GPU leaves: each heavy (more than GAL_CAP distinct columns), so they are spread
    // over the setup threads, each row summed by one thread as in a sequential pass
    return gpu_galerkin(L, ptr, rows, pw, Ac,
                        [&](const std::vector<int64_t> &big, std::vector<std::vector<int32_t>> &oc,
                            std::vector<std::vector<double>> &ov, std::vector<double> &od) {
                            parallel_chunks((int64_t)big.size(), 8, [&](int, int64_t i0, int64_t i1) {
                                RowAcc acc(L.nc);
                                for (int64_t i = i0; i < i1; i++)
                                    od[i] = galerkin_row(L, ptr, rows, pw, big[i], acc, oc[i], ov[i]);
                            });
                        });
}

// ----------------------------------------------------------------------------------- coarsest

// A^+ = (A + J/n)^{-1} - J/n for a connected Laplacian-like operator (null space span{1}):
// levels of at least DENSE_GPU_MIN rows invert A + J/n on the GPU (gpu_dense_inverse), smaller
// ones through a Cholesky factorisation of A + J/n here.
constexpr int64_t DENSE_GPU_MIN = 256;

// a . b over len entries with four independent partial sums (k mod 4), added as
// (s0 + s1) + (s2 + s3): four dependency chains instead of one
static inline double dot4(const double *a, const double *b, int64_t len) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t k = 0;
    for (; k + 4 <= len; k += 4) {
        s0 += a[k] * b[k];
        s1 += a[k + 1] * b[k + 1];
        s2 += a[k + 2] * b[k + 2];
        s3 += a[k + 3] * b[k + 3];
    }
    for (; k < len; k++) s0 += a[k] * b[k];
    return (s0 + s1) + (s2 + s3);
}

int dense_pinv(const HostMat &A, std::vector<double> &pinv) {
    const int64_t n = A.n;
    std::vector<double> M(n * n, 1.0 / (double)n);
    for (int64_t i = 0; i < n; i++) {
        M[i * n + i] += A.diag[i];
        for (int64_t e = A.rp[i]; e < A.rp[i + 1]; e++) M[i * n + A.ci[e]] += A.val[e];
    }
    if (n >= DENSE_GPU_MIN) {
        // Gauss-Jordan inverse on the GPU, then the symmetric part minus J/n
        const int rc = gpu_dense_inverse(n, M);
        if (rc) return rc;
        pinv.assign(n * n, 0.0);
        const double jn = 1.0 / (double)n;
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j <= i; j++) {
                const double v = 0.5 * (M[i * n + j] + M[j * n + i]) - jn;
                pinv[i * n + j] = v;
                pinv[j * n + i] = v;
            }
        return LAMG_OK;
    }
    const int nthr = setup_threads();
    // lower Cholesky factor G (row-major, in place): M = G G^T, right-looking in panels of NB
    // columns. Per panel: the diagonal block by one thread, then the rows below it (a forward
    // substitution each) and the trailing lower triangle (one dot product of NB per entry)
    // split over threads by rows, with a barrier after each of the three parts.
    constexpr int64_t NB = 64;
    bool spd = true;
    std::mutex mu;
    std::condition_variable cv;
    int arrived = 0;
    int64_t phase = 0;
    const int T = n < 256 ? 1 : nthr;
    auto barrier = [&]() {
        if (T == 1) return;
        std::unique_lock<std::mutex> lk(mu);
        const int64_t my = phase;
        if (++arrived == T) {
            arrived = 0;
            phase++;
            cv.notify_all();
        } else {
            cv.wait(lk, [&] { return phase != my; });
        }
    };
    auto worker = [&](int t) {
        for (int64_t k0 = 0; k0 < n; k0 += NB) {
            const int64_t k1 = std::min(n, k0 + NB);
            if (t == 0) {
                for (int64_t j = k0; j < k1 && spd; j++) {
                    double *gj = &M[j * n];
                    double d = gj[j];
                    for (int64_t k = k0; k < j; k++) d -= gj[k] * gj[k];
                    if (!(d > 0.0)) { spd = false; break; }
                    gj[j] = std::sqrt(d);
                    for (int64_t i = j + 1; i < k1; i++) {
                        double *gi = &M[i * n];
                        double v = gi[j];
                        for (int64_t k = k0; k < j; k++) v -= gi[k] * gj[k];
                        gi[j] = v / gj[j];
                    }
                }
            }
            barrier();
            if (!spd) return;
            // rows below the panel: G[i, k0:k1] = M[i, k0:k1] D^{-T}
            for (int64_t i = k1 + t; i < n; i += T) {
                double *gi = &M[i * n];
                for (int64_t j = k0; j < k1; j++) {
                    const double *gj = &M[j * n];
                    double v = gi[j];
                    for (int64_t k = k0; k < j; k++) v -= gi[k] * gj[k];
                    gi[j] = v / gj[j];
                }
            }
            barrier();
            // trailing lower triangle: M[i, j] -= G[i, k0:k1] . G[j, k0:k1], k1 <= j <= i
            for (int64_t i = k1 + t; i < n; i += T) {
                double *gi = &M[i * n];
                for (int64_t j = k1; j <= i; j++) gi[j] -= dot4(gi + k0, &M[j * n + k0], k1 - k0);
            }
            barrier();
        }
    };
    if (T == 1) {
        worker(0);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < T; t++) th.emplace_back(worker, t);
        for (auto &x : th) x.join();
    }
    if (!spd) return LAMG_ERR_DISCONNECTED;
    // M^{-1} = G^{-T} G^{-1}. Row c of H = G^{-T} (stored row-major) is column c of G^{-1}, the
    // forward substitution G y = e_c (y_i = 0 for i < c); then (M^{-1})_{ij} = H_i . H_j over
    // k >= max(i, j). All inner loops run over contiguous memory; rows are split over threads.
    std::vector<double> H(n * n, 0.0);
    auto parallel_rows = [&](auto &&fn) {
        if (n < 128 || nthr == 1) {
            for (int64_t r = 0; r < n; r++) fn(r);
            return;
        }
        std::vector<std::thread> th;
        for (int t = 0; t < nthr; t++)
            th.emplace_back([&, t] {
                for (int64_t r = t; r < n; r += nthr) fn(r);
            });
        for (auto &x : th) x.join();
    };
    parallel_rows([&](int64_t c) {
        double *y = &H[c * n];
        y[c] = 1.0 / M[c * n + c];
        for (int64_t i = c + 1; i < n; i++) {
            const double *gi = &M[i * n];
            y[i] = -dot4(gi + c, y + c, i - c) / gi[i];
        }
    });
    pinv.assign(n * n, 0.0);
    parallel_rows([&](int64_t i) {
        const double *hi = &H[i * n];
        for (int64_t j = 0; j <= i; j++) pinv[i * n + j] = dot4(hi + i, &H[j * n + i], n - i) - 1.0 / (double)n;
    });
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < i; j++) pinv[j * n + i] = pinv[i * n + j];
    return LAMG_OK;
}

// Eq. 5 with the reading that gamma is clamped to [1, 2].
double cycle_index(int64_t El, int64_t El1, int64_t E0) {
    if ((double)El > 0.1 * (double)E0) return 1.5;
    double g = 2.0;
    if (El > 0 && El1 > 0) g = std::min(2.0, 0.7 / ((double)El1 / (double)El));
    return std::max(1.0, g);
}

// Chebyshev smoothing of an aggregation level whose colouring has more than cheb_colours
// classes (a sweep would be that many dependent parallel steps): the Jacobi-preconditioned
// Chebyshev iteration of degree cheb_degree on [lambda/30, lambda], lambda the Gershgorin
// bound max_u (1 + sum_v |A_uv| / A_uu) of D^{-1} A. With theta = (hi + lo)/2,
// delta = (hi - lo)/2, sigma = theta/delta, rho_0 = 1/sigma and rho_k = 1/(2 sigma - rho_{k-1}):
// c1[0] = 0, c2[0] = 1/theta, c1[k] = rho_k rho_{k-1}, c2[k] = 2 rho_k / delta.
void cheb_setup(HostLevel &L, const lamg_options &o) {
    L.cheb = (o.cheb_colours > 0 && L.ncol > o.cheb_colours) ? 1 : 0;
    if (!L.cheb) return;
    const HostMat &A = L.A;
    double lam = 0.0;
    for (int64_t u = 0; u < A.n; u++) {
        double s = 0.0;
        for (int64_t e = A.rp[u]; e < A.rp[u + 1]; e++) s += std::fabs(A.val[e]);
        const double g = 1.0 + s / A.diag[u];
        if (g > lam) lam = g;
    }
    const double hi = lam, lo = lam / 30.0;
    const double theta = (hi + lo) / 2.0, delta = (hi - lo) / 2.0, sigma = theta / delta;
    double rho = 1.0 / sigma;
    L.cheb_lambda = lam;
    L.cheb_c1[0] = 0.0;
    L.cheb_c2[0] = 1.0 / theta;
    for (int k = 1; k < o.cheb_degree && k < 8; k++) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        L.cheb_c1[k] = rn * rho;
        L.cheb_c2[k] = 2.0 * rn / delta;
        rho = rn;
    }
}

// ----------------------------------------------------------------------------------- driver

int build_hierarchy(const lamg_graph *g, const lamg_options &o, std::vector<HostLevel> &levels, double *times) {
    using clk = std::chrono::steady_clock;
    auto t = clk::now();
    // wall time of each setup phase (SETUP_* order) added to times[]
    auto lap = [&](int phase) {
        const auto now = clk::now();
        if (times) times[phase] += std::chrono::duration<double, std::milli>(now - t).count();
        t = now;
    };
    int rc = validate_graph(g);
    if (rc) return rc;
    if (o.K < 1 || o.K > 16 || o.nu_tv < 0 || (o.tv_order != LAMG_TV_STRIDED && o.tv_order != LAMG_TV_STORED) || o.coarsest_max < 0 || o.max_levels < 1 || o.dense_rows < 0 ||
        o.dense_rows > 4096 || o.cheb_colours < 0 || (o.cheb_colours > 0 && (o.cheb_degree < 1 || o.cheb_degree > 8)))
        return LAMG_ERR_INVALID;
    levels.clear();
    HostMat A;
    laplacian(g, A);
    const int64_t E0 = A.nnz() / 2;
    // coarsest size (the paper's "small"): given, or by default the largest n whose dense matrix
    // (8 n^2 bytes) is about the size of the input operator, floor(sqrt(1.5 nnz(L))) with
    // nnz(L) = n + 2m, within [1024, 4096]
    const int64_t cmax = o.coarsest_max > 0
                             ? o.coarsest_max
                             : std::min<int64_t>(4096, std::max<int64_t>(1024, (int64_t)std::floor(std::sqrt(
                                                                                1.5 * (double)(A.n + A.nnz())))));
    lap(SETUP_INPUT);
    for (int l = 0;; l++) {
        levels.emplace_back();
        HostLevel &L = levels.back();
        L.A = std::move(A);
        const int64_t n = L.A.n;
        // a small level with at least n^2/8 off-diagonal entries is solved directly
        const bool dense = n <= o.dense_rows && (double)L.A.nnz() >= (double)n * (double)n / 8.0;
        if (n <= cmax || dense || l + 1 >= o.max_levels) {
            L.kind = KIND_COARSEST;
            break;
        }
        std::vector<uint8_t> inF;
        const int64_t nF = pick_F(L.A, o.dmax, inF);
        HostMat Ac;
        if (nF > 0 && (double)nF >= o.elim_min_frac * (double)n) {
            L.kind = KIND_ELIM;
            if ((rc = schur(L.A, inF, L, Ac))) return rc;
            lap(SETUP_ELIM);
        } else {
            lap(SETUP_ELIM);
            L.kind = KIND_AGG;
            L.ncol = greedy_colour(L.A, L.colour);
            cheb_setup(L, o);
            lap(SETUP_COLOUR);
            L.X.resize(n * o.K);
            L.aff.resize(L.A.nnz());
            L.strong.resize(L.A.nnz());
            L.adm.resize(L.A.nnz());
            // the GPU pass takes as many rounds as the longest index-decreasing path (thousands
            // per level on natural-order meshes and dense power-law levels), so the host's one
            // O(m) scan stays the default
            const bool gpu_agg = o.agg_gpu_rows > 0 && n >= o.agg_gpu_rows;
            std::vector<int32_t> choice(gpu_agg ? n : 0);
            int rounds = 0;
            rc = gpu_tv_and_affinity(L.A, L.colour, l, o.seed, o.K, o.nu_tv, o.tau_soc, o.veto,
                                     L.X.data(), L.aff.data(), L.strong.data(), o.Q, o.guard_eps,
                                     L.adm.data(), o.tv_order, gpu_agg ? choice.data() : nullptr, &rounds);
            if (rc) return rc;
            if (times) times[SETUP_NPHASE] += rounds;
            lap(SETUP_TV_AFFINITY);
            std::vector<int32_t> status, seed;
            if (gpu_agg) aggregate_from_choice(L, choice, status, seed);
            else aggregate(L, o, status, seed);
            if (o.caliber2) upgrade_caliber2(L, o, status, seed);
            lap(SETUP_AGGREGATE);
            if (L.nc >= n || ((double)L.nc > 0.9 * (double)n && n <= 4096)) {
                // no useful coarsening: this level becomes the coarsest
                L.kind = KIND_COARSEST;
                L.agg.clear(); L.agg2.clear(); L.wt.clear();
                break;
            }
            if ((rc = galerkin_device(L, Ac))) return rc;
            lap(SETUP_GALERKIN);
        }
        A = std::move(Ac);
    }
    HostLevel &last = levels.back();
    if (last.A.n > 4096) return LAMG_ERR_SETUP;
    if (dense_pinv(last.A, last.pinv)) return LAMG_ERR_SETUP;
    lap(SETUP_DENSE);
    for (size_t l = 0; l < levels.size(); l++) {
        HostLevel &L = levels[l];
        if (L.kind == KIND_ELIM) L.gamma = 1.0;
        else if (L.kind == KIND_AGG)
            L.gamma = o.gamma_fixed > 0 ? o.gamma_fixed
                                        : cycle_index(L.A.nnz() / 2, levels[l + 1].A.nnz() / 2, E0);
        else L.gamma = 0.0;
    }
    return LAMG_OK;
}

}  // namespace lamg
