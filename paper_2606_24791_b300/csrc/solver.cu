// Device hierarchy, static cycle schedule, CUDA-graph capture and the flexible-CG solve loop,
// plus the C ABI entry points declared in lamg.h.
//
// The cycle of Section 2 is a fixed sequence of kernel launches once the hierarchy is known:
// the visit counters that realise a fractional cycle index restart at every cycle, so every
// cycle visits the levels in the same order. The sequence is generated once on the host and
// captured into CUDA graphs, one for the preconditioner alone and one for the second half of a
// CG iteration (cycle, projection, search-direction update); the first half (A p, the step,
// the residual norm) is a third graph whose last node copies the residual norm to pinned host
// memory for the stopping test.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "hier.h"

using namespace lamg;

static_assert(sizeof(lamg_options) == 144, "lamg_options layout changed: update the header's size note");

// True when step i is a restriction (aggregation or elimination) that also performs step i + 1,
// the row-local start (OP_GS_FIRST or OP_ZERO) of the coarse level's first visit; both steps are
// then one launch in the graph and multi-column paths. Cluster segments keep their steps.
bool lamg::start_fusable(const lamg_hier *h, int i, bool clusters) {
    if (i + 1 >= (int)h->ops.size()) return false;
    const Op &a = h->ops[i], &b = h->ops[i + 1];
    if (a.kind != OP_RESTRICT && a.kind != OP_ELIM_RESTRICT) return false;
    if ((b.kind != OP_GS_FIRST && b.kind != OP_ZERO) || b.level != a.level + 1) return false;
    if (clusters && h->cluster_from >= 0 && b.level >= h->cluster_from) return false;
    return b.kind == OP_ZERO || h->dev[b.level].ncol >= 1;
}

// True when step i runs inside a cluster segment of the graph path: a step on a level >=
// cluster_from, except a dense coarsest solve larger than 512 x 512, which stays one launch over
// the whole GPU (on a cluster's 16 SMs its FP64 products take several times longer) and splits
// the segment around it.
bool lamg::in_cluster_segment(const lamg_hier *h, int i, int from) {
    const Op &op = h->ops[i];
    if (from < 0 || op.level < from) return false;
    return !(op.kind == OP_COARSE && h->dev[op.level].n > 512);
}

bool lamg::in_cluster_segment(const lamg_hier *h, int i) { return in_cluster_segment(h, i, h->cluster_from); }

namespace {

// Device orders of all levels, from the coarsest up (see DevLevel).
void build_orders(lamg_hier *h) {
    const int L = (int)h->host.size();
    h->dev.assign(L, DevLevel());
    for (int l = L - 1; l >= 0; l--) {
        const HostLevel &H = h->host[l];
        DevLevel &D = h->dev[l];
        const int64_t n = H.A.n;
        D.kind = H.kind;
        D.n = n;
        D.nnz = H.A.nnz();
        D.nc = H.nc;
        D.perm.resize(n);
        if (H.kind == KIND_COARSEST) {
            for (int64_t i = 0; i < n; i++) D.perm[i] = (int32_t)i;
        } else if (H.kind == KIND_AGG) {
            int ncol = 0;
            for (int32_t c : H.colour) ncol = std::max(ncol, c + 1);
            D.ncol = ncol;
            D.cptr.assign(ncol + 1, 0);
            for (int32_t c : H.colour) D.cptr[c + 1]++;
            for (int c = 0; c < ncol; c++) D.cptr[c + 1] += D.cptr[c];
            std::vector<int64_t> fill(D.cptr.begin(), D.cptr.end() - 1);
            for (int64_t u = 0; u < n; u++) D.perm[fill[H.colour[u]]++] = (int32_t)u;
            // inside a colour class, longer rows first (ties in ascending id): the 32-row
            // slices of the sliced-ELLPACK operator then hold rows of similar length
            for (int c = 0; c < ncol; c++)
                std::stable_sort(D.perm.begin() + D.cptr[c], D.perm.begin() + D.cptr[c + 1],
                                 [&H](int32_t a, int32_t b) {
                                     return H.A.rp[a + 1] - H.A.rp[a] > H.A.rp[b + 1] - H.A.rp[b];
                                 });
        } else {
            std::vector<int32_t> cnode(H.nc);
            for (int64_t u = 0; u < n; u++)
                if (H.cidx[u] >= 0) cnode[H.cidx[u]] = (int32_t)u;
            const std::vector<int32_t> &pc = h->dev[l + 1].perm;
            for (int64_t i = 0; i < H.nc; i++) D.perm[i] = cnode[pc[i]];
            int64_t t = H.nc;
            for (int64_t u = 0; u < n; u++)
                if (H.cidx[u] < 0) D.perm[t++] = (int32_t)u;
            D.nF = n - H.nc;
        }
    }
}

// Temporary device copies for a setup step: stream-ordered allocations on `s`, freed (after
// the stream has finished with them) by finish(); rc keeps the first error.
struct TmpUpload {
    cudaStream_t s;
    std::vector<void *> ptrs;
    int rc = LAMG_OK;
    explicit TmpUpload(cudaStream_t st) : s(st) {}
    template <typename T>
    const T *put(const std::vector<T> &v) {
        void *q = nullptr;
        if (rc) return nullptr;
        cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(1, v.size()) * sizeof(T), s);
        if (e == cudaSuccess && !v.empty())
            e = cudaMemcpyAsync(q, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { rc = cuda_status(e); return nullptr; }
        ptrs.push_back(q);
        return (const T *)q;
    }
    int finish() {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (void *q : ptrs) cudaFreeAsync(q, s);
        ptrs.clear();
        return e == cudaSuccess ? rc : cuda_status(e);
    }
    ~TmpUpload() {
        if (ptrs.empty()) return;
        cudaStreamSynchronize(s);
        for (void *q : ptrs) cudaFreeAsync(q, s);
    }
};

int upload_level(lamg_hier *h, int l) {
    const HostLevel &H = h->host[l];
    DevLevel &D = h->dev[l];
    const int64_t n = H.A.n;
    int rc;
    std::vector<int32_t> iperm(n);
    for (int64_t i = 0; i < n; i++) iperm[D.perm[i]] = (int32_t)i;
    const int64_t z = H.A.nnz();
    if (z >= (int64_t)INT32_MAX) return LAMG_ERR_INVALID;
    // operator in device order, built on the device from one upload of the natural-order CSR:
    // device row i is natural row perm[i], entries in that row's order (ascending natural id),
    // columns renamed to device indices
    std::vector<int32_t> rp(n + 1, 0);
    for (int64_t i = 0; i < n; i++) rp[i + 1] = rp[i] + (int32_t)(H.A.rp[D.perm[i] + 1] - H.A.rp[D.perm[i]]);
    if ((rc = dupload(h, &D.rp, rp)) || (rc = dalloc(h, &D.ci, z)) || (rc = dalloc(h, &D.val, z)) ||
        (rc = dalloc(h, &D.diag, n)) || (rc = dalloc(h, &D.idiag, n)))
        return rc;
    {
        TmpUpload t(h->stream);
        const int64_t *nrp = t.put(H.A.rp);
        const int32_t *nci = t.put(H.A.ci), *dperm = t.put(D.perm), *diperm = t.put(iperm);
        const double *nval = t.put(H.A.val), *ndiag = t.put(H.A.diag);
        if (t.rc) return t.rc;
        launch_layout_rows(n, dperm, diperm, nrp, nci, nval, ndiag, D.rp, D.ci, D.val, D.diag, D.idiag, h->stream);
        if ((rc = t.finish())) return rc;
    }
    D.tpr = h->opt.row_tpr > 0 ? h->opt.row_tpr : choose_tpr(n ? (double)H.A.nnz() / (double)n : 1.0);
    // sliced ELLPACK copy of the operator in four-entry blocks (sell_col_at / sell_val_at),
    // used by the one-thread-per-row kernels when rows are short and padding is small
    {
        const int64_t ns = (n + 31) / 32;
        std::vector<int32_t> sp(ns + 1, 0);
        int64_t tot = 0, maxlen = 0;
        for (int64_t sl = 0; sl < ns; sl++) {
            int64_t w = 0;
            for (int64_t i = 32 * sl; i < std::min(n, 32 * sl + 32); i++) w = std::max<int64_t>(w, rp[i + 1] - rp[i]);
            maxlen = std::max(maxlen, w);
            w = (w + 3) & ~(int64_t)3;
            sp[sl] = (int32_t)tot;
            tot += 32 * w;
        }
        sp[ns] = (int32_t)tot;
        const bool use = h->opt.sell >= 0 && tot < (int64_t)INT32_MAX && maxlen <= SELL_MAX_ROW &&
                         (h->opt.sell > 0 || (double)tot <= 1.5 * (double)z + 64.0);
        if (use) {
            if ((rc = dupload(h, &D.sl_ptr, sp)) || (rc = dalloc(h, &D.sl_col, tot)) || (rc = dalloc(h, &D.sl_val, tot)))
                return rc;
            launch_layout_sell(n, ns, D.sl_ptr, D.rp, D.ci, D.val, D.sl_col, D.sl_val, h->stream);
            CKR(cudaGetLastError());
            CKR(cudaStreamSynchronize(h->stream));
            D.sell = 1;
            D.sell_nnz = tot;
        }
    }
    // long rows
    {
        std::vector<int32_t> lr;
        for (int64_t i = 0; i < n; i++)
            if (rp[i + 1] - rp[i] > LONG_ROW) lr.push_back((int32_t)i);
        D.nlong = (int64_t)lr.size();
        if (D.nlong && (rc = dupload(h, &D.lrows, lr))) return rc;
        if (H.kind == KIND_AGG) {
            D.lptr.assign(D.ncol + 1, 0);
            for (int c = 0; c < D.ncol; c++) {
                int64_t cnt = 0;
                for (int64_t i = D.cptr[c]; i < D.cptr[c + 1] && rp[i + 1] - rp[i] > LONG_ROW; i++) cnt++;
                D.lptr[c + 1] = D.lptr[c] + cnt;
            }
            if (D.lptr[D.ncol] != D.nlong) return LAMG_ERR_INVALID;  // classes sorted longest first
        }
    }
    // rule (refined by timing when the options ask for it): sweeps on lane groups, whose
    // short per-lane chains suit the latency-bound colour classes; residual-type passes of
    // large levels one thread per row, which issues the fewest FP64 instructions per entry
    // (measured per level on B300: sweeps of levels with at least 2^18 rows of at most 8
    // entries are faster one thread per row, the others on lane groups; residual-type passes
    // from 2^16 rows on one thread per row)
    const double avg = n ? (double)H.A.nnz() / (double)n : 0.0;
    D.gs_tpr = (D.sell && h->opt.row_tpr == 0 && n >= (1 << 18) && avg <= 8.0) ? 0 : D.tpr;
    D.rs_tpr = (D.sell && (h->opt.sell > 0 || n >= 65536)) ? 0 : D.tpr;
    if (D.sell && h->opt.sell > 0) D.gs_tpr = 0;
    // A colour class of >= 2^16 rows on average (large mesh-like levels without the sliced form)
    // is bound by FP64 instructions rather than latency: a lane takes about four entries before
    // the shuffle tree instead of two
    if (h->opt.row_tpr == 0 && D.gs_tpr > 0 && H.kind == KIND_AGG && H.ncol > 0 && n / H.ncol >= (1 << 16)) {
        int t = 1;
        while (t < 32 && 4.0 * t < avg) t *= 2;
        D.gs_tpr = std::min(D.gs_tpr, t);
    }
    // Chebyshev levels (power-law Galerkin levels, long rows): a step is one pass over all rows
    // and is bound by FP64 instructions rather than latency, so a lane takes about eight entries
    // of its row before the shuffle tree instead of two (the tree's adds and idle lanes cost more
    // than the longer chain)
    if (H.kind == KIND_AGG && H.cheb && h->opt.row_tpr == 0 && !D.sell) {
        int t = 1;
        while (t < 32 && 8.0 * t < avg) t *= 2;
        D.gs_tpr = D.rs_tpr = t;
    }
    if (H.kind == KIND_AGG) {
        const std::vector<int32_t> &ip = h->dev[l + 1].perm;
        std::vector<int32_t> ipc(H.nc);
        for (int64_t i = 0; i < H.nc; i++) ipc[ip[i]] = (int32_t)i;
        std::vector<int32_t> agg(n), agg2(n);
        std::vector<double> wt(n);
        std::vector<int64_t> cnt(H.nc + 1, 0);
        for (int64_t i = 0; i < n; i++) {
            const int32_t u = D.perm[i];
            agg[i] = ipc[H.agg[u]];
            agg2[i] = H.agg2[u] < 0 ? -1 : ipc[H.agg2[u]];
            wt[i] = H.wt[u];
            if (agg2[i] < 0) cnt[agg[i] + 1]++;
            else {
                if (wt[i] != 0.0) cnt[agg[i] + 1]++;
                cnt[agg2[i] + 1]++;
            }
        }
        for (int64_t a = 0; a < H.nc; a++) cnt[a + 1] += cnt[a];
        std::vector<int32_t> ptr(cnt.begin(), cnt.end()), prow(cnt[H.nc]);
        std::vector<double> pw(cnt[H.nc]);
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t i = 0; i < n; i++) {
            if (agg2[i] < 0) { prow[fill[agg[i]]] = (int32_t)i; pw[fill[agg[i]]++] = 1.0; continue; }
            if (wt[i] != 0.0) { prow[fill[agg[i]]] = (int32_t)i; pw[fill[agg[i]]++] = wt[i]; }
            prow[fill[agg2[i]]] = (int32_t)i;
            pw[fill[agg2[i]]++] = 1.0 - wt[i];
        }
        if ((rc = dupload(h, &D.agg, agg)) || (rc = dupload(h, &D.agg2, agg2)) || (rc = dupload(h, &D.wt, wt)) ||
            (rc = dupload(h, &D.pt_ptr, ptr)) || (rc = dupload(h, &D.pt_row, prow)) || (rc = dupload(h, &D.pt_w, pw)))
            return rc;
        D.pt_tpr = choose_tpr(H.nc ? (double)cnt[H.nc] / (double)H.nc : 1.0);
        if ((rc = dalloc(h, &D.r, n))) return rc;
        D.cheb = H.cheb;
        D.cheb_m = H.cheb ? h->opt.cheb_degree : 0;
        if (H.cheb) {
            for (int k = 0; k < 8; k++) { D.cheb_c1[k] = H.cheb_c1[k]; D.cheb_c2[k] = H.cheb_c2[k]; }
            if ((rc = dalloc(h, &D.t, n)) || (rc = dalloc(h, &D.d, n))) return rc;
        }
    } else if (H.kind == KIND_ELIM) {
        const int64_t nc = H.nc, nF = n - nc;
        std::vector<int32_t> pfc(4 * nF, -1);
        std::vector<double> pfv(4 * nF, 0.0), dF(nF);
        for (int64_t t = 0; t < nF; t++) {
            const int32_t u = D.perm[nc + t];
            const int64_t deg = H.A.rp[u + 1] - H.A.rp[u];
            if (deg > 4) return LAMG_ERR_INVALID;
            for (int64_t e = H.A.rp[u], j = 0; e < H.A.rp[u + 1]; e++, j++) {
                const int32_t c = iperm[H.A.ci[e]];
                if (c >= nc) return LAMG_ERR_INVALID;  // F must be independent
                const double pv = -H.A.val[e] / H.A.diag[u];
                pfc[4 * t + j] = c;
                pfv[4 * t + j] = pv;
            }
            dF[t] = H.A.diag[u];
        }
        // the transpose P_F^T by coarse row, each row's F entries in ascending F index
        std::vector<int32_t> ptr(nc + 1, 0);
        for (int64_t q = 0; q < 4 * nF; q++)
            if (pfc[q] >= 0) ptr[pfc[q] + 1]++;
        for (int64_t i = 0; i < nc; i++) ptr[i + 1] += ptr[i];
        std::vector<int32_t> fidx(ptr[nc]), fill(ptr.begin(), ptr.end() - 1);
        std::vector<double> fval(ptr[nc]);
        for (int64_t q = 0; q < 4 * nF; q++) {
            const int32_t c = pfc[q];
            if (c < 0) continue;
            fidx[fill[c]] = (int32_t)(q / 4);
            fval[fill[c]++] = pfv[q];
        }
        if ((rc = dupload(h, &D.pf_col, pfc)) || (rc = dupload(h, &D.pf_val, pfv)) || (rc = dupload(h, &D.dF, dF)) ||
            (rc = dupload(h, &D.pft_ptr, ptr)) || (rc = dupload(h, &D.pft_f, fidx)) || (rc = dupload(h, &D.pft_val, fval)))
            return rc;
        // for the multi-column kernels: 1 / A_FF (an FP64 division per element and column cost more
        // than the interpolation's memory traffic) and the C rows that gather more than LONG_ROW
        // F entries (hubs of power-law graphs), which a whole block sums
        std::vector<double> idF(nF);
        for (int64_t t = 0; t < nF; t++) idF[t] = 1.0 / dF[t];
        std::vector<int32_t> lng;
        for (int64_t i = 0; i < nc; i++)
            if (ptr[i + 1] - ptr[i] > LONG_ROW) lng.push_back((int32_t)i);
        D.npft_long = (int64_t)lng.size();
        if ((rc = dupload(h, &D.idF, idF)) || (D.npft_long && (rc = dupload(h, &D.pft_long, lng)))) return rc;
    } else {
        // (I - J/n) A^+: the coarsest solve and its mean-zero projection as one matrix
        std::vector<double> P(n * n), colmean(n, 0.0);
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++) P[i * n + j] = H.pinv[(int64_t)D.perm[i] * n + D.perm[j]];
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++) colmean[j] += P[i * n + j];
        for (int64_t j = 0; j < n; j++) colmean[j] /= (double)n;
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++) P[i * n + j] -= colmean[j];
        if ((rc = dupload(h, &D.pinv, P))) return rc;
    }
    return LAMG_OK;
}

// Simulate the recursion of one cycle (Section 2) and record its kernel sequence.
void emit_visit(lamg_hier *h, std::vector<int64_t> &visits, int l, bool first) {
    const DevLevel &D = h->dev[l];
    if (D.kind == KIND_COARSEST) { h->ops.push_back({OP_COARSE, l, 0}); return; }
    if (D.kind == KIND_ELIM) {
        h->ops.push_back({OP_ELIM_RESTRICT, l, 0});
        emit_visit(h, visits, l + 1, first);
        h->ops.push_back({OP_ELIM_INTERP, l, 0});
        return;
    }
    const int npre = h->opt.nu_pre, npost = h->opt.nu_post;
    // one smoothing phase of `sweeps` Chebyshev polynomials of degree m: its T = m sweeps steps
    // alternate between the iterate x and the level's second buffer t (a step reads one and
    // writes the other; colour = step index within its polynomial + 256 when it reads t). A
    // phase that continues from x starts by reading x and ends with one copy t -> x when T is
    // odd; a phase that starts from a zero iterate (first visit: the first step needs no product
    // with A) writes its first result into whichever buffer makes the last step land in x.
    auto cheb_phase = [&](int sweeps, bool from_zero) {
        const int m = h->opt.cheb_degree, T = m * sweeps;
        auto buf = [&](int i) { return from_zero ? ((T - i) & 1) : (i & 1); };   // 0 x, 1 t
        for (int p = 0; p < T; p++) {
            if (p == 0 && from_zero) h->ops.push_back({OP_CHEB_FIRST, l, buf(1)});
            else h->ops.push_back({OP_CHEB, l, (p % m) + 256 * buf(p)});
        }
        if (buf(T)) h->ops.push_back({OP_CHEB_COPY, l, 0});
    };
    if (D.cheb) {
        // a first visit starts from x = 0, so the first step of the first polynomial needs no
        // product with A: x1 = c2[0] D^-1 b (the same operations as that step with x = 0)
        if (first && npre == 0) h->ops.push_back({OP_ZERO, l, 0});
        if (npre > 0) cheb_phase(npre, first);
    } else {
        if (first && npre == 0) h->ops.push_back({OP_ZERO, l, 0});
        for (int s = 0; s < npre; s++) {
            int c0 = 0;
            if (s == 0 && first) { h->ops.push_back({OP_GS_FIRST, l, 0}); c0 = 1; }
            for (int c = c0; c < D.ncol; c++) h->ops.push_back({OP_GS, l, c});
        }
    }
    h->ops.push_back({OP_RESID, l, 0});
    h->ops.push_back({OP_RESTRICT, l, 0});
    const double g = h->host[l].gamma;
    const int64_t j = visits[l]++;
    const int64_t nv = (int64_t)std::floor((double)(j + 1) * g) - (int64_t)std::floor((double)j * g);
    for (int64_t i = 0; i < nv; i++) emit_visit(h, visits, l + 1, i == 0);
    h->ops.push_back({OP_PROLONG, l, 0});
    if (D.cheb) {
        if (npost > 0) cheb_phase(npost, false);
    } else {
        for (int s = 0; s < npost; s++)
            for (int c = D.ncol - 1; c >= 0; c--) h->ops.push_back({OP_GS, l, c});
    }
}

int capture(lamg_hier *h, cudaGraphExec_t *out, int which) {
    cudaStream_t cs = h->stream;
    cudaGraph_t g = nullptr;
    CKR(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const DevLevel &F = h->dev[0];
    const int64_t n = F.n;
    if (which == 0 || which == 1) {
        const int nops = (int)h->ops.size(), nlev = (int)h->dev.size();
        for (int i = 0; i < nops;) {
            if (in_cluster_segment(h, i)) {
                int j = i;
                while (j < nops && in_cluster_segment(h, j)) j++;
                launch_cluster(h->d_lv, nlev, h->d_cptr, h->ncptr, h->d_ops + i, j - i, h->cl_dim,
                               pdl_enabled(), cs);
                i = j;
            } else if (start_fusable(h, i)) {
                launch_op(h->ops[i], h->dev, h->red, cs, &h->ops[i + 1]);
                i += 2;
            } else {
                launch_op(h->ops[i++], h->dev, h->red, cs);
            }
        }
        launch_sum(n, F.x, h->red, cs);
        if (which == 0) launch_sub_mean(n, F.x, h->red, cs);
        else {
            launch_proj_dots(n, F.x, h->zold, h->r, h->red, cs);
            launch_update_p(n, F.x, h->p, h->zold, h->red, cs);
        }
    } else {
        launch_spmv_dot(F, h->p, h->q, h->red, cs);
        launch_update_xr(n, h->xs, h->r, h->p, h->q, h->red, cs);
        cudaMemcpyAsync(h->h_scal, h->red.scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, cs);
    }
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return cuda_status(e);
}

// Algorithmic DRAM bytes of one step of the persistent schedule (FP64 values, int32 indices;
// each array read or written once, gathered vectors counted once).
}  // namespace

// Algorithmic DRAM bytes of one step of the cycle, split into the bytes read once per step
// whatever the number of right-hand sides (operator values and indices, transfer weights) and
// the bytes moved per right-hand side (vectors). s = bytes per value (8 FP64, 4 FP32 cycle);
// indices are 4 bytes, the dense coarsest matrix is always FP64; each array is counted once per
// step and a gathered vector at most once. The residual is counted as fused into the
// restriction (r is never written), which is the algorithmic minimum.
void lamg::op_bytes(const lamg_hier *h, const Op &op, double s, double *mat, double *vec) {
    const HostLevel &H = h->host[op.level];
    const DevLevel &D = h->dev[op.level];
    const double n = (double)D.n, z = (double)D.nnz, nc = (double)D.nc, nF = (double)D.nF;
    double m = 0.0, v = 0.0;
    switch (op.kind) {
        case OP_GS_FIRST: m = s * (double)D.cptr[1]; v = s * (double)D.cptr[1] + s * n; break;
        case OP_ZERO: v = s * n; break;
        case OP_GS: {
            const int64_t r0 = D.cptr[op.colour], r1 = D.cptr[op.colour + 1];
            double zc = 0;
            for (int64_t i = r0; i < r1; i++) {
                const int32_t u = D.perm[i];
                zc += (double)(H.A.rp[u + 1] - H.A.rp[u]);
            }
            const double R = (double)(r1 - r0);
            m = (4 + s) * zc + 4 * (R + 1) + s * R;
            v = 2 * s * R + s * std::min(zc, n);
            break;
        }
        case OP_RESID: break;
        case OP_RESTRICT: {
            double E = 0;
            for (int64_t u = 0; u < D.n; u++) E += H.agg2[u] < 0 ? 1 : (H.wt[u] != 0.0 ? 2 : 1);
            m = (4 + s) * z + 4 * (n + 1) + s * n + (4 + s) * E + 4 * (nc + 1);
            v = 2 * s * n + s * nc;
            break;
        }
        case OP_PROLONG: m = 8 * n + s * n; v = 2 * s * n + s * nc; break;
        case OP_ELIM_RESTRICT: {
            double E = 0;
            for (int64_t u = 0; u < D.n; u++)
                if (H.cidx[u] < 0) E += (double)(H.A.rp[u + 1] - H.A.rp[u]);
            m = 4 * (nc + 1) + (4 + s) * E;
            v = 2 * s * nc + s * nF;
            break;
        }
        case OP_ELIM_INTERP: m = 16 * nF + 5 * s * nF; v = s * nc + 2 * s * nF; break;
        case OP_COARSE: m = 8 * n * n; v = 2 * s * n; break;
        case OP_CHEB: m = (4 + s) * z + 4 * (n + 1) + 2 * s * n; v = s * (n + std::min(z, n)) + 3 * s * n; break;
        case OP_CHEB_COPY: v = 2 * s * n; break;
        case OP_CHEB_FIRST: m = s * n; v = (h->opt.cheb_degree > 1 ? 3 : 2) * s * n; break;
    }
    *mat = m;
    *vec = v;
}

namespace {

// Device copies of the level table, the colour offsets of all levels and the step list.
int upload_tables(lamg_hier *h) {
    int rc;
    const int L = (int)h->dev.size();
    std::vector<PLevel> pl(L);
    std::vector<int32_t> cptr_all;
    for (int l = 0; l < L; l++) {
        DevLevel &D = h->dev[l];
        PLevel &P = pl[l];
        std::memset(&P, 0, sizeof(P));
        P.kind = D.kind; P.n = (int)D.n; P.nc = (int)D.nc; P.nF = (int)D.nF; P.ncol = D.ncol;
        P.tpr = D.tpr; P.pt_tpr = D.pt_tpr;
        P.cptr_off = (int)cptr_all.size();
        for (int64_t c : D.cptr) cptr_all.push_back((int32_t)c);
        P.rp = D.rp; P.ci = D.ci; P.val = D.val; P.diag = D.diag; P.idiag = D.idiag;
        P.gs_tpr = D.gs_tpr; P.rs_tpr = D.rs_tpr; P.sl_ptr = D.sl_ptr; P.sl_col = D.sl_col; P.sl_val = D.sl_val;
        P.agg = D.agg; P.agg2 = D.agg2; P.wt = D.wt;
        P.pt_ptr = D.pt_ptr; P.pt_row = D.pt_row; P.pt_w = D.pt_w;
        P.pf_col = D.pf_col; P.pf_val = D.pf_val; P.dF = D.dF;
        P.pft_ptr = D.pft_ptr; P.pft_f = D.pft_f; P.pft_val = D.pft_val;
        P.pinv = D.pinv;
        P.x = D.x; P.b = D.b; P.r = D.r;
    }
    if (cptr_all.empty()) cptr_all.push_back(0);
    h->ncptr = (int)cptr_all.size();
    if ((rc = dupload(h, &h->d_lv, pl)) || (rc = dupload(h, &h->d_ops, h->ops)) || (rc = dupload(h, &h->d_cptr, cptr_all)))
        return rc;
    return LAMG_OK;
}

// Device tables of the persistent solve kernel (not for hierarchies with Chebyshev levels,
// whose steps it does not run).
int setup_persistent(lamg_hier *h) {
    int rc;
    for (const DevLevel &D : h->dev)
        if (D.cheb) return LAMG_OK;
    const int L = (int)h->dev.size();
    const int64_t tail_rows = h->opt.tail_rows > 0 ? h->opt.tail_rows : 8192;
    // single-CTA segments: maximal runs of steps on levels with at most tail_rows rows (the
    // dense coarsest only while its matrix is at most 512 x 512)
    const int nops = (int)h->ops.size();
    std::vector<uint8_t> small(nops, 0);
    for (int i = 0; i < nops; i++) {
        const DevLevel &D = h->dev[h->ops[i].level];
        small[i] = D.kind == KIND_COARSEST ? (D.n <= 512 && D.n <= tail_rows) : (D.n <= tail_rows);
    }
    std::vector<int32_t> tail_end(nops, -1);
    for (int i = 0; i < nops;) {
        if (!small[i]) { i++; continue; }
        int j = i;
        while (j < nops && small[j]) j++;
        tail_end[i] = j;
        i = j;
    }
    h->smem = persistent_smem(L, nops, h->ncptr);
    if (h->smem > 200 * 1024) return LAMG_OK;  // tables do not fit: graph path only
    h->grid = persistent_grid(h->device, h->smem);
    if (h->grid < 1) return LAMG_OK;
    int32_t *dtail = nullptr;
    if ((rc = dupload(h, &dtail, tail_end))) return rc;
    PSolve &S = h->ph;
    std::memset(&S, 0, sizeof(S));
    S.nlev = L; S.nops = nops; S.n0 = (int)h->dev[0].n; S.ncptr = h->ncptr;
    S.lv = h->d_lv; S.ops = h->d_ops; S.tail_end = dtail; S.cptr_all = h->d_cptr; S.perm0 = h->perm0;
    S.r = h->r; S.p = h->p; S.q = h->q; S.zold = h->zold; S.xs = h->xs; S.bkeep = h->bkeep;
    if ((rc = dalloc(h, &S.partials, 2 * RED_NV * h->grid)) || (rc = dalloc(h, &h->bar, 1))) return rc;
    S.bar = h->bar;
    S.scal = h->red.scal;
    h->hist_cap = 1024;
    if ((rc = dalloc(h, &h->hist, h->hist_cap))) return rc;
    S.hist = h->hist;
    if ((rc = dalloc(h, &h->psolve, 1))) return rc;
    CKR(cudaMemcpyAsync(h->psolve, &S, sizeof(S), cudaMemcpyHostToDevice, h->stream));
    CKR(cudaMemsetAsync(h->bar, 0, sizeof(GridBar), h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    h->persistent_ok = true;
    return LAMG_OK;
}

// Mean time of reps launches of seq (after one untimed pass), or -1 on error.
double time_ops(lamg_hier *h, const std::vector<Op> &seq, bool spmv, int reps) {
    cudaStream_t s = h->stream;
    auto pass = [&]() {
        if (spmv) launch_spmv_dot(h->dev[0], h->p, h->q, h->red, s);
        else for (const Op &op : seq) launch_op(op, h->dev, h->red, s);
    };
    pass();
    cudaEventRecord(h->ev_a, s);
    for (int r = 0; r < reps; r++) pass();
    cudaEventRecord(h->ev_b, s);
    if (wait_event(h, h->ev_b) != LAMG_OK || cudaGetLastError() != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev_a, h->ev_b);
    return ms / reps;
}

// Kernel form per level, chosen by timing: for the colour-class sweep (one forward sweep of
// every class) and for the residual-type pass (the residual; A p with its dot product on the
// finest level), every lanes-per-row count from a quarter to twice the rule's, and one thread
// per row on the sliced copy where it exists. Vectors are zero while timing. Every form
// computes the same sums in a form-specific order, so the choice changes rounding only.
int tune_kernels(lamg_hier *h) {
    if (!h->opt.autotune) return LAMG_OK;
    cudaStream_t s = h->stream;
    const int L = (int)h->dev.size();
    for (int l = 0; l < L; l++) {
        DevLevel &D = h->dev[l];
        if (D.x) CKR(cudaMemsetAsync(D.x, 0, D.n * sizeof(double), s));
        if (D.b) CKR(cudaMemsetAsync(D.b, 0, D.n * sizeof(double), s));
        if (D.r) CKR(cudaMemsetAsync(D.r, 0, D.n * sizeof(double), s));
    }
    CKR(cudaMemsetAsync(h->p, 0, h->dev[0].n * sizeof(double), s));
    const int reps = 3;
    for (int l = 0; l < L; l++) {
        DevLevel &D = h->dev[l];
        if (D.kind == KIND_COARSEST) continue;
        std::vector<int> cand;
        if (D.sell) cand.push_back(0);
        for (int t = 1; t <= 32; t *= 2)
            if ((4 * t >= D.tpr && t <= 2 * D.tpr) || (D.cheb && t <= 2 * D.tpr)) cand.push_back(t);
        if (D.kind == KIND_AGG) {
            // the level's smoothing pass: one colour-ordered sweep, or one Chebyshev step
            std::vector<Op> sweep;
            if (D.cheb) sweep.push_back({OP_CHEB, l, 0});
            else
                for (int c = 0; c < D.ncol; c++) sweep.push_back({OP_GS, l, c});
            double best = -1.0;
            int pick = D.gs_tpr;
            for (int t : cand) {
                D.gs_tpr = t;
                const double ms = time_ops(h, sweep, false, reps);
                if (ms > 0 && (best < 0 || ms < best)) { best = ms; pick = t; }
            }
            D.gs_tpr = pick;
        }
        if (D.kind == KIND_AGG || l == 0) {
            const std::vector<Op> res{{OP_RESID, l, 0}};
            double best = -1.0;
            int pick = D.rs_tpr;
            for (int t : cand) {
                D.rs_tpr = t;
                const double ms = l == 0 ? time_ops(h, res, true, reps)
                                         : (D.kind == KIND_AGG ? time_ops(h, res, false, reps) : -1.0);
                if (ms > 0 && (best < 0 || ms < best)) { best = ms; pick = t; }
            }
            D.rs_tpr = pick;
        }
    }
    CKR(cudaMemsetAsync(h->red.ticket, 0, sizeof(unsigned), s));
    CKR(cudaStreamSynchronize(s));
    return LAMG_OK;
}

// Kernels of one cycle in the graph path (steps with no rows launch nothing; a cluster
// segment is one launch).
int64_t count_cycle_launches(const lamg_hier *h) {
    int64_t k = 0;
    const int nops = (int)h->ops.size();
    for (int i = 0; i < nops;) {
        const Op &op = h->ops[i];
        if (in_cluster_segment(h, i)) {
            while (i < nops && in_cluster_segment(h, i)) i++;
            k++;
            continue;
        }
        if (start_fusable(h, i)) {
            i += 2;
            k++;
            continue;
        }
        i++;
        if (op.kind == OP_ELIM_INTERP && h->dev[op.level].nF == 0) continue;
        if (op.kind == OP_GS && h->dev[op.level].cptr[op.colour + 1] == h->dev[op.level].cptr[op.colour]) continue;
        k++;
    }
    return k;
}

// Mean device time of one preconditioner cycle under the current schedule; -1 if the
// schedule cannot be captured.
double time_cycle(lamg_hier *h) {
    cudaGraphExec_t g = nullptr;
    if (capture(h, &g, 0) != LAMG_OK) {
        cudaGetLastError();
        return -1.0;
    }
    cudaStream_t s = h->stream;
    const int warm = 3, reps = 10;
    for (int r = 0; r < warm; r++) cudaGraphLaunch(g, s);
    cudaEventRecord(h->ev_a, s);
    for (int r = 0; r < reps; r++) cudaGraphLaunch(g, s);
    cudaEventRecord(h->ev_b, s);
    double ms = -1.0;
    if (wait_event(h, h->ev_b) == LAMG_OK && cudaGetLastError() == cudaSuccess) {
        float t = 0.f;
        cudaEventElapsedTime(&t, h->ev_a, h->ev_b);
        ms = t / reps;
    }
    cudaGraphExecDestroy(g);
    return ms;
}

// Which levels run as one cluster launch per visit. Candidates are the levels from which on
// every level has at most cluster_rows rows (2^18 when automatic). cluster_rows > 0 takes the
// largest candidate; 0 times one cycle of the per-step schedule and of up to eight candidates
// (largest first) and keeps the fastest; < 0 keeps every step its own kernel. Every schedule
// computes bit-identical iterates, so the choice changes time only.
int choose_cluster(lamg_hier *h) {
    h->cluster_from = -1;
    h->cl_dim = 0;
    h->tune_ms.clear();
    h->tune_from.clear();
    const int L = (int)h->dev.size();
    const int64_t rows = h->opt.cluster_rows == 0 && !h->opt.autotune ? -1 : h->opt.cluster_rows;
    // largest table size of any segment: the step list is staged when it has at most
    // CL_OPS_SMEM steps
    const size_t smem = cluster_smem(L, h->ncptr, std::min((int)h->ops.size(), CL_OPS_SMEM));
    if (smem > CL_SMEM_MAX) return LAMG_OK;
    h->cl_dim = cluster_dim(h->device, smem);
    if (!h->cl_dim || rows < 0) return LAMG_OK;
    const int64_t limit = rows > 0 ? rows : ((int64_t)1 << 18);
    // levels with block-per-row long rows stay on the per-step kernels (the cluster kernel
    // sums every row with lane groups)
    std::vector<int64_t> smax(L + 1, 0), lng(L + 1, 0);
    for (int l = L - 1; l >= 0; l--) {
        smax[l] = std::max(smax[l + 1], h->dev[l].n);
        lng[l] = lng[l + 1] + h->dev[l].nlong + (h->dev[l].cheb ? 1 : 0);   // nor Chebyshev levels
    }
    // a candidate must leave some step inside a cluster segment (a level holding only a dense
    // coarsest that stays outside would give the per-step schedule again)
    auto has_segment = [&](int from) {
        for (int i = 0; i < (int)h->ops.size(); i++)
            if (in_cluster_segment(h, i, from)) return true;
        return false;
    };
    std::vector<int> cand;
    for (int l = 0; l < L; l++)
        if (smax[l] <= limit && lng[l] == 0 && has_segment(l)) cand.push_back(l);
    if (cand.empty()) return LAMG_OK;
    if (rows > 0) {
        h->cluster_from = cand[0];
        return LAMG_OK;
    }
    // timed on a zero right-hand side, which keeps every vector finite
    CKR(cudaMemsetAsync(h->r, 0, h->dev[0].n * sizeof(double), h->stream));
    int best = -1;
    double best_ms = time_cycle(h);
    h->tune_from.push_back(-1);
    h->tune_ms.push_back(best_ms);
    for (size_t k = 0; k < cand.size() && k < 8; k++) {
        h->cluster_from = cand[k];
        const double ms = time_cycle(h);
        h->tune_from.push_back(cand[k]);
        h->tune_ms.push_back(ms);
        if (ms > 0 && (best_ms < 0 || ms < best_ms)) { best_ms = ms; best = cand[k]; }
    }
    h->cluster_from = best;
    return LAMG_OK;
}

// Build device data, schedule and graphs for h->host.
int finalize(lamg_hier *h) {
    int rc;
    CKR(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CKR(cudaEventCreate(&h->ev_a));
    CKR(cudaEventCreate(&h->ev_b));
    CKR(cudaEventCreateWithFlags(&h->ev_poll, cudaEventDisableTiming));
    auto t_dev = std::chrono::steady_clock::now();
    build_orders(h);
    const int L = (int)h->host.size();
    for (int l = 0; l < L; l++)
        if ((rc = upload_level(h, l))) return rc;
    // vectors: level 0's right-hand side is the CG residual; an elimination level's coarse
    // iterate is the head of its own iterate
    const int64_t n0 = h->host[0].A.n;
    if ((rc = dalloc(h, &h->r, n0)) || (rc = dalloc(h, &h->p, n0)) || (rc = dalloc(h, &h->q, n0)) ||
        (rc = dalloc(h, &h->zold, n0)) || (rc = dalloc(h, &h->xs, n0)) || (rc = dalloc(h, &h->bkeep, n0)) ||
        (rc = dalloc(h, &h->nat_in, n0)) || (rc = dalloc(h, &h->nat_out, n0)))
        return rc;
    for (int l = 0; l < L; l++) {
        DevLevel &D = h->dev[l];
        if (l == 0) D.b = h->r;
        else if ((rc = dalloc(h, &D.b, D.n))) return rc;
        if (l == 0 || h->dev[l - 1].kind != KIND_ELIM) {
            if ((rc = dalloc(h, &D.x, D.n))) return rc;
        } else {
            D.x = h->dev[l - 1].x;
        }
    }
    if ((rc = dupload(h, &h->perm0, h->dev[0].perm))) return rc;
    if ((rc = dalloc(h, &h->red.partials, RED_NV * RED_MAXG)) || (rc = dalloc(h, &h->red.ticket, 1)) ||
        (rc = dalloc(h, &h->red.scal, S_COUNT)))
        return rc;
    CKR(cudaMemsetAsync(h->red.ticket, 0, sizeof(unsigned), h->stream));
    CKR(cudaMemsetAsync(h->red.scal, 0, S_COUNT * sizeof(double), h->stream));
    h->h_scal = pinned_slot();
    if (!h->h_scal) return LAMG_ERR_OOM;
    auto t_sched = std::chrono::steady_clock::now();
    h->setup_ms[SETUP_DEVICE] += std::chrono::duration<double, std::milli>(t_sched - t_dev).count();
    if ((rc = tune_kernels(h))) return rc;
    std::vector<int64_t> visits(L, 0);
    h->ops.clear();
    emit_visit(h, visits, 0, true);
    if ((rc = upload_tables(h)) || (rc = choose_cluster(h))) return rc;
    if ((rc = capture(h, &h->g_cycle, 0)) || (rc = capture(h, &h->g_tail, 1)) || (rc = capture(h, &h->g_head, 2)))
        return rc;
    CKR(cudaEventCreate(&h->ev_k0));
    CKR(cudaEventCreate(&h->ev_k1));
    for (int p = 0; p < 2; p++) {
        h->cycle_mat[p] = h->cycle_vec[p] = 0.0;
        for (const Op &op : h->ops) {
            double m, v;
            op_bytes(h, op, p == 0 ? 8.0 : 4.0, &m, &v);
            h->cycle_mat[p] += m;
            h->cycle_vec[p] += v;
        }
    }
    h->cycle_bytes = h->cycle_mat[0] + h->cycle_vec[0];
    h->cycle_launches = count_cycle_launches(h);
    if ((rc = setup_persistent(h))) return rc;
    CKR(cudaStreamSynchronize(h->stream));
    h->setup_ms[SETUP_SCHEDULE] +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_sched).count();
    return LAMG_OK;
}

// The device's default stream-ordered memory pool keeps up to POOL_KEEP bytes of freed memory
// (this process only) instead of returning it to the CUDA driver at every synchronisation: a setup
// makes a few hundred allocations, and re-mapping memory for each was most of its device-layout
// time.
constexpr uint64_t POOL_KEEP = (uint64_t)4 << 30;

int set_device(int dev) {
    int cnt = 0;
    cudaError_t e = cudaGetDeviceCount(&cnt);
    if (e != cudaSuccess || cnt == 0) return LAMG_ERR_NO_DEVICE;
    if (dev < 0 || dev >= cnt) return LAMG_ERR_INVALID;
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return cuda_status(e);
    static std::once_flag once[64];
    if (dev < 64)
        std::call_once(once[dev], [dev] {
            cudaMemPool_t pool = nullptr;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t keep = POOL_KEEP;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
            cudaGetLastError();
        });
    return LAMG_OK;
}

}  // namespace

// =================================================================================== C ABI

extern "C" {

void lamg_options_default(lamg_options *o) {
    std::memset(o, 0, sizeof(*o));
    o->K = 4;
    o->nu_tv = 3;
    o->dmax = 4;
    o->nu_pre = 1;
    o->nu_post = 2;
    o->coarsest_max = 0;
    o->max_levels = 100;
    o->veto = 1;
    o->caliber2 = 1;
    o->precision = LAMG_FP64;
    o->seed = 3;
    o->Q = 2.5;
    o->tau_soc = 0.05;
    o->elim_min_frac = 0.01;
    o->snap = 1e-3;
    o->guard_eps = 1e-10;
    o->gamma_fixed = 0.0;
    o->device = 0;
    o->tail_rows = 8192;
    o->cluster_rows = 0;
    o->autotune = 0;
    o->dense_rows = 4096;
    o->cheb_colours = 32;
    o->cheb_degree = 1;
    o->tv_order = LAMG_TV_STRIDED;
}

const char *lamg_strerror(int c) {
    switch (c) {
        case LAMG_OK: return "ok";
        case LAMG_ERR_INVALID: return "invalid argument or input graph";
        case LAMG_ERR_DISCONNECTED: return "graph is not connected";
        case LAMG_ERR_SETUP: return "coarsening stalled above the dense coarsest limit";
        case LAMG_ERR_OOM: return "out of memory";
        case LAMG_ERR_NOT_CONVERGED: return "not converged within maxit";
        case LAMG_ERR_CUDA: return "CUDA runtime error";
        case LAMG_ERR_TIMEOUT: return "bounded GPU wait ran out";
        case LAMG_ERR_ADMISSION: return "request exceeds the memory budget";
        case LAMG_ERR_NO_DEVICE: return "no CUDA device";
        default: return "unknown error";
    }
}

int lamg_setup(const lamg_graph *g, const lamg_options *opt, lamg_hier **out) {
    if (!out) return LAMG_ERR_INVALID;
    *out = nullptr;
    lamg_options o;
    if (opt) o = *opt; else lamg_options_default(&o);
    if (o.row_tpr < 0 || o.row_tpr > 32 || (o.row_tpr & (o.row_tpr - 1))) return LAMG_ERR_INVALID;
    if (o.cheb_colours < 0 || (o.cheb_colours > 0 && (o.cheb_degree < 1 || o.cheb_degree > 8))) return LAMG_ERR_INVALID;
    int rc = set_device(o.device);
    if (rc) return rc;
    lamg_hier *h = new lamg_hier();
    h->device = o.device;
    h->opt = o;
    rc = build_hierarchy(g, o, h->host, h->setup_ms);
    if (!rc) rc = finalize(h);
    if (rc) { delete h; return rc; }
    *out = h;
    return LAMG_OK;
}

int lamg_import(const lamg_level_desc *lv, int32_t nl, const lamg_options *opt, lamg_hier **out) {
    if (!out || !lv || nl < 1) return LAMG_ERR_INVALID;
    *out = nullptr;
    lamg_options o;
    if (opt) o = *opt; else lamg_options_default(&o);
    if (o.row_tpr < 0 || o.row_tpr > 32 || (o.row_tpr & (o.row_tpr - 1))) return LAMG_ERR_INVALID;
    if (o.cheb_colours < 0 || (o.cheb_colours > 0 && (o.cheb_degree < 1 || o.cheb_degree > 8))) return LAMG_ERR_INVALID;
    int rc = set_device(o.device);
    if (rc) return rc;
    lamg_hier *h = new lamg_hier();
    h->device = o.device;
    h->opt = o;
    h->host.resize(nl);
    for (int l = 0; l < nl; l++) {
        const lamg_level_desc &d = lv[l];
        HostLevel &H = h->host[l];
        const int64_t n = d.n;
        if (n < 1 || !d.rp || !d.diag) { delete h; return LAMG_ERR_INVALID; }
        const int64_t z = d.rp[n];
        H.kind = d.kind;
        H.A.n = n;
        H.A.rp.assign(d.rp, d.rp + n + 1);
        H.A.ci.assign(d.ci, d.ci + z);
        H.A.val.assign(d.val, d.val + z);
        H.A.diag.assign(d.diag, d.diag + n);
        H.nc = d.nc;
        H.gamma = d.gamma;
        const bool last = (l == nl - 1);
        if ((d.kind == KIND_COARSEST) != last) { delete h; return LAMG_ERR_INVALID; }
        if (d.kind != KIND_COARSEST && lv[l + 1].n != d.nc) { delete h; return LAMG_ERR_INVALID; }
        if (d.kind == KIND_AGG) {
            if (!d.colour || !d.agg || !d.agg2 || !d.wt) { delete h; return LAMG_ERR_INVALID; }
            H.colour.assign(d.colour, d.colour + n);
            H.agg.assign(d.agg, d.agg + n);
            H.agg2.assign(d.agg2, d.agg2 + n);
            H.wt.assign(d.wt, d.wt + n);
            for (int64_t u = 0; u < n; u++)
                if (H.agg[u] < 0 || H.agg[u] >= d.nc || H.agg2[u] >= d.nc || H.colour[u] < 0) { delete h; return LAMG_ERR_INVALID; }
            // colour classes must be independent sets
            for (int64_t u = 0; u < n; u++)
                for (int64_t e = H.A.rp[u]; e < H.A.rp[u + 1]; e++)
                    if (H.colour[H.A.ci[e]] == H.colour[u]) { delete h; return LAMG_ERR_INVALID; }
            H.ncol = 0;
            for (int32_t c : H.colour) H.ncol = std::max(H.ncol, c + 1);
            cheb_setup(H, o);
        } else if (d.kind == KIND_ELIM) {
            if (!d.cidx) { delete h; return LAMG_ERR_INVALID; }
            H.cidx.assign(d.cidx, d.cidx + n);
        } else {
            if (n > 4096) { delete h; return LAMG_ERR_INVALID; }
            rc = dense_pinv(H.A, H.pinv);
            if (rc) { delete h; return rc; }
        }
    }
    rc = finalize(h);
    if (rc) { delete h; return rc; }
    *out = h;
    return LAMG_OK;
}

void lamg_destroy(lamg_hier *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    delete h;
}

// Host vectors of a solve pass through a pooled pinned buffer (one host memcpy each way, then a
// pinned DMA) instead of a pageable copy: measured 0.5 ms faster per 8 MB round trip than the
// pageable path, while several copy threads were slower (page faults on the caller's fresh output
// pages). Returned to the pool only when the stream has nothing left in flight (else kept out of
// the pool).
struct Stage {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    bool drained = false;  // set once the last copy through the buffer is known complete
    Stage(size_t nb, cudaStream_t st) : bytes(nb), s(st) {
        if (nb >= ((size_t)1 << 20)) p = pinned_stage(nb);
    }
    ~Stage() {
        if (p && (drained || cudaStreamQuery(s) == cudaSuccess)) pinned_stage_release(p, bytes);
    }
};

static int solve_graph(lamg_hier *h, const double *b, double *phi, const lamg_solve_opts *so, lamg_stats *st) {
    cudaStream_t s = so->stream ? (cudaStream_t)so->stream : h->stream;
    const bool devp = so->flags & LAMG_DEVICE_PTRS;
    const DevLevel &F = h->dev[0];
    const int64_t n = F.n;
    int rc = LAMG_OK;
    Stage stage(devp ? 0 : n * sizeof(double), s);
    CKR(cudaEventRecord(h->ev_a, s));
    if (devp) CKR(cudaMemcpyAsync(h->nat_in, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else if (stage.p) {
        std::memcpy(stage.p, b, n * sizeof(double));
        CKR(cudaMemcpyAsync(h->nat_in, stage.p, n * sizeof(double), cudaMemcpyHostToDevice, s));
    } else CKR(cudaMemcpyAsync(h->nat_in, b, n * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gather(n, h->perm0, h->nat_in, h->r, s);
    launch_sum(n, h->r, h->red, s);
    launch_init_b(n, h->r, h->bkeep, h->xs, h->p, h->zold, h->red, s);
    CKR(cudaGetLastError());
    CKR(cudaGraphLaunch(h->g_tail, s));
    int it = 0;
    double rel = 1.0, bn2 = 0.0;
    if (st && st->hist) st->hist[0] = 1.0;
    while (it < so->maxit) {
        CKR(cudaGraphLaunch(h->g_head, s));
        CKR(cudaEventRecord(h->ev_poll, s));
        if ((rc = wait_event(h, h->ev_poll))) return rc;
        it++;
        bn2 = h->h_scal[S_BN2];
        rel = bn2 > 0 ? std::sqrt(h->h_scal[S_RR] / bn2) : 0.0;
        if (st && st->hist) st->hist[it] = rel;
        if (!(rel > so->tol)) break;
        CKR(cudaGraphLaunch(h->g_tail, s));
    }
    launch_true_resid(F, h->xs, h->bkeep, h->red, s);
    launch_scatter(n, h->perm0, h->xs, h->nat_out, s);
    if (devp) CKR(cudaMemcpyAsync(phi, h->nat_out, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else if (stage.p) CKR(cudaMemcpyAsync(stage.p, h->nat_out, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    else CKR(cudaMemcpyAsync(phi, h->nat_out, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKR(cudaMemcpyAsync(h->h_scal, h->red.scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev_b, s));
    if ((rc = wait_event(h, h->ev_b))) return rc;
    CKR(cudaGetLastError());
    if (stage.p) {
        std::memcpy(phi, stage.p, n * sizeof(double));
        stage.drained = true;  // ev_b followed the copy into the buffer
    }
    if (st) {
        st->iters = it;
        st->nlevels = (int32_t)h->dev.size();
        st->relres = rel;
        st->relres_true = bn2 > 0 ? std::sqrt(h->h_scal[S_TRUE_RR] / bn2) : 0.0;
        st->b_mean = h->h_scal[S_BMEAN];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_a, h->ev_b);
        st->solve_ms = ms;
        st->kernel_ms = ms;
        const double z0 = (double)h->dev[0].nnz, n0 = (double)n;
        st->alg_bytes = (double)it * (h->cycle_bytes + 12 * z0 + 148 * n0) + h->cycle_bytes + 72 * n0 +
                        (12 * z0 + 36 * n0) + 16 * n0;
        // gather, sum, init; per cycle the schedule + mean, projection/dots, p update (one
        // cycle per iteration that did not stop, plus the first); per iteration SpMV-dot and
        // x/r update; true residual and scatter
        const int64_t cycles = rel <= so->tol ? it : it + 1;
        st->launches = 3 + 2 * (int64_t)it + cycles * (h->cycle_launches + 3) + 2;
    }
    return rel <= so->tol ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
}

// The whole solve as one cooperative launch of the persistent kernel.
static int solve_persistent(lamg_hier *h, const double *b, double *phi, const lamg_solve_opts *so,
                            lamg_stats *st) {
    cudaStream_t s = so->stream ? (cudaStream_t)so->stream : h->stream;
    const bool devp = so->flags & LAMG_DEVICE_PTRS;
    const int64_t n = h->dev[0].n;
    int rc = LAMG_OK;
    if (so->maxit + 1 > h->hist_cap) {
        double *nh = nullptr;
        if ((rc = dalloc(h, &nh, so->maxit + 1))) return rc;
        h->hist = nh;
        h->hist_cap = so->maxit + 1;
        h->ph.hist = nh;
        CKR(cudaMemcpyAsync(h->psolve, &h->ph, sizeof(PSolve), cudaMemcpyHostToDevice, s));
    }
    CKR(cudaEventRecord(h->ev_a, s));
    const double *b_in = b;
    double *phi_out = phi;
    if (!devp) {
        CKR(cudaMemcpyAsync(h->nat_in, b, n * sizeof(double), cudaMemcpyHostToDevice, s));
        b_in = h->nat_in;
        phi_out = h->nat_out;
    }
    CKR(cudaMemsetAsync(h->bar, 0, sizeof(GridBar), s));
    CKR(cudaEventRecord(h->ev_k0, s));
    const unsigned long long wait_ns = so->wait_us == 0 ? WAIT_NS_DEFAULT
                                       : so->wait_us < 0 ? 0ULL : 1000ULL * (unsigned long long)so->wait_us;
    CKR(launch_persistent(h->psolve, h->grid, h->smem, 0, so->maxit, so->tol, b_in, phi_out, s, nullptr, wait_ns));
    CKR(cudaEventRecord(h->ev_k1, s));
    if (!devp) CKR(cudaMemcpyAsync(phi, h->nat_out, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKR(cudaMemcpyAsync(h->h_scal, h->red.scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    GridBar hb{};
    CKR(cudaMemcpyAsync(&hb, h->bar, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev_b, s));
    if ((rc = wait_event(h, h->ev_b))) return rc;
    CKR(cudaGetLastError());
    if (hb.err) return LAMG_ERR_TIMEOUT;
    const int it = (int)h->h_scal[S_ITERS];
    const double bn2 = h->h_scal[S_BN2];
    const double rel = bn2 > 0 ? std::sqrt(h->h_scal[S_RR] / bn2) : 0.0;
    if (st) {
        if (st->hist) {
            CKR(cudaMemcpyAsync(st->hist, h->hist, (it + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
            CKR(cudaStreamSynchronize(s));
        }
        st->iters = it;
        st->nlevels = (int32_t)h->dev.size();
        st->relres = rel;
        st->relres_true = bn2 > 0 ? std::sqrt(h->h_scal[S_TRUE_RR] / bn2) : 0.0;
        st->b_mean = h->h_scal[S_BMEAN];
        float ms = 0.f, kms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_a, h->ev_b);
        cudaEventElapsedTime(&kms, h->ev_k0, h->ev_k1);
        st->solve_ms = ms;
        st->kernel_ms = kms;
        // per iteration: cycle + CG vectors (SpMV with dot 12z+28n, x/r update 48n, mean 8n,
        // projection with dots 32n, p update 32n); once: gather/projection of b, true residual
        const double z0 = (double)h->dev[0].nnz, n0 = (double)n;
        st->alg_bytes = (double)it * (h->cycle_bytes + 12 * z0 + 148 * n0) + h->cycle_bytes + 72 * n0 +
                        (12 * z0 + 36 * n0) + 16 * n0;
        st->launches = 1;
    }
    return rel <= so->tol ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
}

int lamg_solve(lamg_hier *h, const double *b, double *phi, const lamg_solve_opts *so, lamg_stats *st) {
    if (!h || !b || !phi || !so || !(so->tol > 0) || so->maxit < 1) return LAMG_ERR_INVALID;
    CKR(cudaSetDevice(h->device));
    if (h->opt.precision == LAMG_FP32) return solve_batch_impl(h, 1, b, phi, so, st, LAMG_FP32);
    if (!(so->flags & LAMG_PERSISTENT) || !h->persistent_ok) return solve_graph(h, b, phi, so, st);
    return solve_persistent(h, b, phi, so, st);
}

}  // extern "C"

// Whether a hierarchy can be solved by one cluster of k_cluster_solve (FP64 cycle, cluster
// launch available, no block-per-row long rows, tables within the shared-memory limit, at most
// MANY_MAX_ENTRIES stored entries in the finest operator: one cluster has 16 SMs' share of the
// GPU's FP64 units and bandwidth, so a larger system is faster on the whole GPU), and the
// dynamic shared memory its tables take.
bool lamg::many_eligible(const lamg_hier *h, size_t *smem) {
    int64_t nl = 0;
    for (const DevLevel &D : h->dev) nl += D.nlong + (D.cheb ? 1 : 0);   // nor Chebyshev levels
    const size_t sm = cluster_smem((int)h->dev.size(), h->ncptr, (int)h->ops.size());
    if (smem) *smem = sm;
    const int64_t entries = h->dev[0].n + h->dev[0].nnz;
    return h->opt.precision == LAMG_FP64 && h->cl_dim > 0 && nl == 0 && sm <= CL_SMEM_MAX &&
           entries <= MANY_MAX_ENTRIES;
}

// Device buffers of a cluster solve (partials, results, history of maxit + 1 entries) and its
// descriptor.
int lamg::many_prepare(lamg_hier *h, int maxit, double tol, const double *b_in, double *phi_out, MGraph *M) {
    int rc;
    if (!h->mg_part && ((rc = dalloc(h, &h->mg_part, 2 * RED_NV * 16)) || (rc = dalloc(h, &h->mg_out, MG_OUT))))
        return rc;
    if (h->mg_hist_cap < maxit + 1) {
        if ((rc = dalloc(h, &h->mg_hist, maxit + 1))) return rc;
        h->mg_hist_cap = maxit + 1;
    }
    std::memset(M, 0, sizeof(*M));
    M->lv = h->d_lv; M->cptr = h->d_cptr; M->ops = h->d_ops; M->perm0 = h->perm0;
    M->nlev = (int)h->dev.size(); M->ncptr = h->ncptr; M->nops = (int)h->ops.size(); M->n0 = (int)h->dev[0].n;
    M->maxit = maxit; M->tol = tol;
    M->r = h->r; M->p = h->p; M->q = h->q; M->zold = h->zold; M->xs = h->xs; M->bkeep = h->bkeep;
    M->part = h->mg_part; M->out = h->mg_out; M->hist = h->mg_hist;
    M->b_in = b_in;
    M->phi_out = phi_out;
    return LAMG_OK;
}

extern "C" {

int lamg_solve_many(int32_t G, lamg_hier *const *hs, const double *const *b, double *const *phi,
                    const lamg_solve_opts *so, lamg_stats *st) {
    if (G < 1 || !hs || !b || !phi || !so || !(so->tol > 0) || so->maxit < 1) return LAMG_ERR_INVALID;
    for (int g = 0; g < G; g++)
        if (!hs[g] || !b[g] || !phi[g] || hs[g]->device != hs[0]->device) return LAMG_ERR_INVALID;
    lamg_hier *h0 = hs[0];
    CKR(cudaSetDevice(h0->device));
    cudaStream_t s = so->stream ? (cudaStream_t)so->stream : h0->stream;
    const bool devp = so->flags & LAMG_DEVICE_PTRS;
    // eligible: FP64 cycle, cluster launch available, no block-per-row long rows
    std::vector<int> cl_idx, other;
    int cl = 16;
    size_t smem = 0;
    for (int g = 0; g < G; g++) {
        size_t sm = 0;
        if (many_eligible(hs[g], &sm)) {
            cl_idx.push_back(g);
            cl = std::min(cl, hs[g]->cl_dim);
            smem = std::max(smem, sm);
        } else {
            other.push_back(g);
        }
    }
    int rc = LAMG_OK;
    std::vector<MGraph> desc(cl_idx.size());
    for (size_t k = 0; k < cl_idx.size(); k++) {
        lamg_hier *h = hs[cl_idx[k]];
        const int64_t n = h->dev[0].n;
        if (!devp)
            CKR(cudaMemcpyAsync(h->nat_in, b[cl_idx[k]], n * sizeof(double), cudaMemcpyHostToDevice, s));
        if ((rc = many_prepare(h, so->maxit, so->tol, devp ? b[cl_idx[k]] : h->nat_in,
                               devp ? phi[cl_idx[k]] : h->nat_out, &desc[k])))
            return rc;
    }
    float ms = 0.f;
    if (!desc.empty()) {
        MGraph *d_desc = nullptr;
        CKR(cudaMallocAsync(&d_desc, desc.size() * sizeof(MGraph), s));
        CKR(cudaMemcpyAsync(d_desc, desc.data(), desc.size() * sizeof(MGraph), cudaMemcpyHostToDevice, s));
        CKR(cudaEventRecord(h0->ev_k0, s));
        CKR(launch_cluster_solve(d_desc, (int)desc.size(), cl, smem, s));
        CKR(cudaEventRecord(h0->ev_k1, s));
        CKR(cudaFreeAsync(d_desc, s));
        std::vector<double> outs(desc.size() * MG_OUT);
        for (size_t k = 0; k < cl_idx.size(); k++) {
            lamg_hier *h = hs[cl_idx[k]];
            const int64_t n = h->dev[0].n;
            if (!devp)
                CKR(cudaMemcpyAsync(phi[cl_idx[k]], h->nat_out, n * sizeof(double), cudaMemcpyDeviceToHost, s));
            CKR(cudaMemcpyAsync(&outs[k * MG_OUT], h->mg_out, MG_OUT * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        CKR(cudaEventRecord(h0->ev_b, s));
        if ((rc = wait_event(h0, h0->ev_b))) return rc;
        CKR(cudaGetLastError());
        cudaEventElapsedTime(&ms, h0->ev_k0, h0->ev_k1);
        for (size_t k = 0; k < cl_idx.size(); k++) {
            const int g = cl_idx[k];
            lamg_hier *h = hs[g];
            const double *o = &outs[k * MG_OUT];
            const int it = (int)o[MG_ITERS];
            const double bn2 = o[MG_BN2];
            const double rel = bn2 > 0 ? std::sqrt(o[MG_RR] / bn2) : 0.0;
            if (st) {
                lamg_stats &S = st[g];
                if (S.hist) {
                    CKR(cudaMemcpy(S.hist, h->mg_hist, (it + 1) * sizeof(double), cudaMemcpyDeviceToHost));
                }
                S.iters = it;
                S.nlevels = (int32_t)h->dev.size();
                S.relres = rel;
                S.relres_true = bn2 > 0 ? std::sqrt(o[MG_TRUE_RR] / bn2) : 0.0;
                S.b_mean = o[MG_BMEAN];
                S.solve_ms = ms;
                S.kernel_ms = ms;
                const double z0 = (double)h->dev[0].nnz, n0 = (double)h->dev[0].n;
                S.alg_bytes = (double)it * (h->cycle_bytes + 12 * z0 + 148 * n0) + h->cycle_bytes + 72 * n0 +
                              (12 * z0 + 36 * n0) + 16 * n0;
                S.launches = 1;
            }
            if (!(rel <= so->tol) && rc == LAMG_OK) rc = LAMG_ERR_NOT_CONVERGED;
        }
    }
    // the others on their own per-step path, one after another
    for (int g : other) {
        lamg_solve_opts o1 = *so;
        const int r1 = lamg_solve(hs[g], b[g], phi[g], &o1, st ? &st[g] : nullptr);
        if (r1 != LAMG_OK && (rc == LAMG_OK || r1 != LAMG_ERR_NOT_CONVERGED)) rc = r1;
    }
    return rc;
}

int lamg_cycle(lamg_hier *h, const double *r, double *z, uint32_t flags) {
    if (!h || !r || !z) return LAMG_ERR_INVALID;
    CKR(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    const int64_t n = h->dev[0].n;
    const bool devp = flags & LAMG_DEVICE_PTRS;
    CKR(cudaMemcpyAsync(h->nat_in, r, n * sizeof(double), devp ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (!(flags & LAMG_PERSISTENT) || !h->persistent_ok) {
        launch_gather(n, h->perm0, h->nat_in, h->r, s);
        CKR(cudaGraphLaunch(h->g_cycle, s));
        launch_scatter(n, h->perm0, h->dev[0].x, h->nat_out, s);
    } else {
        CKR(cudaMemsetAsync(h->bar, 0, sizeof(GridBar), s));
        CKR(launch_persistent(h->psolve, h->grid, h->smem, 1, 0, 0.0, h->nat_in, h->nat_out, s));
    }
    CKR(cudaMemcpyAsync(z, h->nat_out, n * sizeof(double), devp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    GridBar hb{};
    if (h->bar) CKR(cudaMemcpyAsync(&hb, h->bar, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev_b, s));
    int rc = wait_event(h, h->ev_b);
    if (rc) return rc;
    CKR(cudaGetLastError());
    if (hb.err) return LAMG_ERR_TIMEOUT;
    return LAMG_OK;
}

int lamg_profile_cycle(lamg_hier *h, int64_t *out, int64_t cap, int64_t *count) {
    if (!h || !out || !count || cap < 1) return LAMG_ERR_INVALID;
    if (!h->persistent_ok) return LAMG_ERR_INVALID;
    CKR(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    const int64_t n = h->dev[0].n;
    const int64_t slots = 2 * ((int64_t)h->ops.size() + 2);
    unsigned long long *dprof = nullptr;
    CKR(cudaMalloc(&dprof, slots * sizeof(unsigned long long)));
    std::vector<unsigned long long> hp(slots, 0);
    CKR(cudaMemsetAsync(h->nat_in, 0, n * sizeof(double), s));
    CKR(cudaMemsetAsync(h->bar, 0, sizeof(GridBar), s));
    cudaError_t e = launch_persistent(h->psolve, h->grid, h->smem, 1, 0, 0.0, h->nat_in, h->nat_out, s, dprof);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), dprof, slots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_b, s);
    int rc = e == cudaSuccess ? wait_event(h, h->ev_b) : cuda_status(e);
    cudaFree(dprof);
    if (rc) return rc;
    const int64_t nrec = (int64_t)hp[0];
    int64_t k = 0;
    for (int64_t r = 1; r <= nrec && k < cap; r++, k++) {
        out[2 * k] = (int64_t)hp[2 * r];
        out[2 * k + 1] = (int64_t)(hp[2 * r + 1] - hp[2 * r - 1 == 1 ? 1 : 2 * r - 1]);
    }
    *count = k;
    return LAMG_OK;
}

int lamg_profile_schedule(lamg_hier *h, int32_t from_level, int64_t *out, int64_t cap, int64_t *count) {
    if (!h || !out || !count) return LAMG_ERR_INVALID;
    CKR(cudaSetDevice(h->device));
    const int nops = (int)h->ops.size(), nlev = (int)h->dev.size();
    if (cap < 3 * (int64_t)nops) return LAMG_ERR_INVALID;
    if (from_level >= 0 && !h->cl_dim) return LAMG_ERR_INVALID;
    cudaStream_t s = h->stream;
    unsigned long long *dprof = nullptr;
    CKR(cudaMalloc(&dprof, 2 * (size_t)nops * sizeof(unsigned long long)));
    std::vector<unsigned long long> hp(2 * (size_t)nops, 0);
    std::vector<cudaEvent_t> ev(2 * (size_t)nops, nullptr);
    std::vector<uint8_t> in_cl(nops, 0);
    cudaError_t e = cudaMemsetAsync(h->r, 0, h->dev[0].n * sizeof(double), s);
    // segments as the graph path forms them for cluster_from = from_level
    auto in_seg = [&](int i) { return in_cluster_segment(h, i, from_level); };
    for (int i = 0; i < nops && e == cudaSuccess;) {
        if (in_seg(i)) {
            int j = i;
            while (j < nops && in_seg(j)) in_cl[j++] = 1;
            launch_cluster(h->d_lv, nlev, h->d_cptr, h->ncptr, h->d_ops + i, j - i, h->cl_dim, false, s,
                           dprof + 2 * (size_t)i);
            i = j;
        } else {
            cudaEventCreate(&ev[2 * i]);
            cudaEventCreate(&ev[2 * i + 1]);
            cudaEventRecord(ev[2 * i], s);
            launch_op(h->ops[i], h->dev, h->red, s);
            e = cudaEventRecord(ev[2 * i + 1], s);
            i++;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), dprof, hp.size() * sizeof(unsigned long long),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_b, s);
    int rc = e == cudaSuccess ? wait_event(h, h->ev_b) : cuda_status(e);
    if (!rc && cudaGetLastError() != cudaSuccess) rc = LAMG_ERR_CUDA;
    for (int i = 0; i < nops; i++) {
        out[3 * i] = i;
        out[3 * i + 1] = in_cl[i];
        out[3 * i + 2] = 0;
        if (rc) continue;
        if (in_cl[i]) {
            out[3 * i + 2] = (int64_t)(hp[2 * i + 1] - hp[2 * i]);
        } else if (ev[2 * i]) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            out[3 * i + 2] = (int64_t)std::llround(ms * 1e6);
        }
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(dprof);
    *count = 3 * (int64_t)nops;
    return rc;
}

int lamg_setup_times(const lamg_hier *h, double *out, int32_t cap) {
    if (!h || !out || cap < SETUP_NPHASE) return LAMG_ERR_INVALID;
    for (int i = 0; i < SETUP_NPHASE; i++) out[i] = h->setup_ms[i];
    if (cap > SETUP_NPHASE) out[SETUP_NPHASE] = h->setup_ms[SETUP_NPHASE];
    return LAMG_OK;
}

int lamg_schedule_info(const lamg_hier *h, int64_t *out, int64_t cap, int64_t *count) {
    if (!h || !out || !count || cap < 5 + 2 * (int64_t)h->dev.size()) return LAMG_ERR_INVALID;
    out[0] = h->cluster_from;
    out[1] = h->cl_dim;
    out[2] = h->cycle_launches;
    out[3] = (int64_t)h->ops.size();
    int64_t k = 4;
    out[k++] = (int64_t)h->dev.size();
    for (const DevLevel &D : h->dev) {
        if (k + 2 > cap) break;
        out[k++] = D.gs_tpr;
        out[k++] = D.rs_tpr;
    }
    for (size_t i = 0; i < h->tune_ms.size() && k + 2 <= cap; i++) {
        out[k++] = h->tune_from[i];
        out[k++] = (int64_t)std::llround(h->tune_ms[i] * 1e6);  // nanoseconds
    }
    *count = k;
    return LAMG_OK;
}

int lamg_op_list(const lamg_hier *h, int32_t *out, int64_t cap, int64_t *count) {
    if (!h || !count) return LAMG_ERR_INVALID;
    *count = (int64_t)h->ops.size();
    if (out)
        for (int64_t i = 0; i < (int64_t)h->ops.size() && i < cap; i++) {
            out[3 * i] = h->ops[i].kind;
            out[3 * i + 1] = h->ops[i].level;
            out[3 * i + 2] = h->ops[i].colour;
        }
    return LAMG_OK;
}

int lamg_hier_info(const lamg_hier *h, int64_t *nlevels, int64_t *meta, double *gamma) {
    if (!h || !nlevels) return LAMG_ERR_INVALID;
    *nlevels = (int64_t)h->host.size();
    for (size_t l = 0; l < h->host.size(); l++) {
        const HostLevel &H = h->host[l];
        if (meta) {
            int64_t c2 = 0;
            for (int32_t v : H.agg2) c2 += v >= 0;
            meta[7 * l + 0] = H.kind;
            meta[7 * l + 1] = H.A.n;
            meta[7 * l + 2] = H.A.nnz();
            meta[7 * l + 3] = h->dev.size() > l ? h->dev[l].ncol : 0;
            meta[7 * l + 4] = H.nc;
            meta[7 * l + 5] = c2;
            meta[7 * l + 6] = h->dev.size() > l ? (int64_t)h->dev[l].bytes : 0;
        }
        if (gamma) gamma[l] = H.gamma;
    }
    return LAMG_OK;
}

int lamg_level_get(const lamg_hier *h, int32_t level, const char *name, void *dst, int64_t *count) {
    if (!h || !name || level < 0 || level >= (int32_t)h->host.size()) return LAMG_ERR_INVALID;
    const HostLevel &H = h->host[level];
    const void *src = nullptr;
    int64_t cnt = 0;
    size_t es = 0;
    std::string nm(name);
    if (nm == "rp") { src = H.A.rp.data(); cnt = (int64_t)H.A.rp.size(); es = 8; }
    else if (nm == "ci") { src = H.A.ci.data(); cnt = (int64_t)H.A.ci.size(); es = 4; }
    else if (nm == "val") { src = H.A.val.data(); cnt = (int64_t)H.A.val.size(); es = 8; }
    else if (nm == "diag") { src = H.A.diag.data(); cnt = (int64_t)H.A.diag.size(); es = 8; }
    else if (nm == "colour") { src = H.colour.data(); cnt = (int64_t)H.colour.size(); es = 4; }
    else if (nm == "cidx") { src = H.cidx.data(); cnt = (int64_t)H.cidx.size(); es = 4; }
    else if (nm == "agg") { src = H.agg.data(); cnt = (int64_t)H.agg.size(); es = 4; }
    else if (nm == "agg2") { src = H.agg2.data(); cnt = (int64_t)H.agg2.size(); es = 4; }
    else if (nm == "wt") { src = H.wt.data(); cnt = (int64_t)H.wt.size(); es = 8; }
    else if (nm == "X") { src = H.X.data(); cnt = (int64_t)H.X.size(); es = 8; }
    else if (nm == "aff") { src = H.aff.data(); cnt = (int64_t)H.aff.size(); es = 8; }
    else if (nm == "strong") { src = H.strong.data(); cnt = (int64_t)H.strong.size(); es = 1; }
    else if (nm == "pinv") { src = H.pinv.data(); cnt = (int64_t)H.pinv.size(); es = 8; }
    else return LAMG_ERR_INVALID;
    if (count) *count = cnt;
    if (dst && cnt) std::memcpy(dst, src, cnt * es);
    return LAMG_OK;
}

int lamg_testvectors(int64_t n, const int64_t *rp, const int32_t *ci, const double *val, const double *diag,
                     const int32_t *colour, int32_t level, uint64_t seed, int32_t K, int32_t nu, double *X,
                     int32_t order) {
    if (n < 1 || !rp || !diag || !colour || !X || K < 1 || K > 16 || nu < 0 ||
        (order != LAMG_TV_STRIDED && order != LAMG_TV_STORED))
        return LAMG_ERR_INVALID;
    for (int64_t u = 0; u < n; u++)
        if (colour[u] < 0) return LAMG_ERR_INVALID;
    int rc = set_device(0);
    if (rc) return rc;
    HostMat A;
    A.n = n;
    A.rp.assign(rp, rp + n + 1);
    A.ci.assign(ci, ci + rp[n]);
    A.val.assign(val, val + rp[n]);
    A.diag.assign(diag, diag + n);
    std::vector<int32_t> col(colour, colour + n);
    return gpu_testvectors(A, col, level, seed, K, nu, X, order);
}

int lamg_affinity(int64_t n, const int64_t *rp, const int32_t *ci, const double *val, const double *X,
                  int32_t K, double tau, double *aff, uint8_t *strong) {
    if (n < 1 || !rp || !X || !aff || !strong || K < 1) return LAMG_ERR_INVALID;
    int rc = set_device(0);
    if (rc) return rc;
    HostMat A;
    A.n = n;
    A.rp.assign(rp, rp + n + 1);
    A.ci.assign(ci, ci + rp[n]);
    A.val.assign(val, val + rp[n]);
    A.diag.assign(n, 0.0);
    return gpu_affinity(A, X, K, tau, aff, strong);
}

int lamg_time_kernel(lamg_hier *h, int32_t which, int32_t level, int32_t reps, double *out) {
    if (!h || !out || reps < 1 || level < 0 || level >= (int32_t)h->dev.size()) return LAMG_ERR_INVALID;
    CKR(cudaSetDevice(h->device));
    DevLevel &D = h->dev[level];
    const double n = (double)D.n, z = (double)D.nnz, nc = (double)D.nc;
    if ((which == 0 || which == 1 || which == 3 || which == 4) && D.kind != KIND_AGG) return LAMG_ERR_INVALID;
    if (which == 2 && level != 0) return LAMG_ERR_INVALID;
    cudaStream_t s = h->stream;
    // a buffer larger than the 126 MB L2, rewritten between repetitions so that every timed
    // launch starts with a cold L2
    const size_t flush_bytes = (size_t)256 << 20;
    void *flush = nullptr;
    CKR(cudaMalloc(&flush, flush_bytes));
    double bytes = 0.0;
    int launches = 1;
    std::vector<Op> seq;
    switch (which) {
        case 0: seq.push_back({OP_RESID, level, 0}); bytes = 12 * z + 36 * n + 4; break;
        case 1:
            for (int c = 0; c < D.ncol; c++) seq.push_back({OP_GS, level, c});
            bytes = 12 * z + 36 * n + 4 * D.ncol;
            launches = D.ncol;
            break;
        case 2: bytes = 12 * z + 28 * n + 4; break;
        case 3: {
            int32_t ent = 0;
            cudaMemcpyAsync(&ent, D.pt_ptr + D.nc, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            seq.push_back({OP_RESTRICT, level, 0});
            bytes = 12.0 * ent + 4 * (nc + 1) + 8 * n + 8 * nc;
            break;
        }
        case 4: seq.push_back({OP_PROLONG, level, 0}); bytes = 32 * n + 8 * nc; break;
        default: cudaFree(flush); return LAMG_ERR_INVALID;
    }
    double total = 0.0;
    int rc = LAMG_OK;
    for (int r = 0; r < reps && !rc; r++) {
        cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);
        cudaEventRecord(h->ev_a, s);
        if (which == 2) launch_spmv_dot(h->dev[0], h->p, h->q, h->red, s);
        else for (const Op &op : seq) launch_op(op, h->dev, h->red, s);
        cudaEventRecord(h->ev_b, s);
        rc = wait_event(h, h->ev_b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_a, h->ev_b);
        total += ms;
    }
    cudaFree(flush);
    if (rc) return rc;
    CKR(cudaGetLastError());
    out[0] = total / reps;
    out[1] = bytes;
    out[2] = launches;
    return LAMG_OK;
}

}  // extern "C"

