// The hierarchy handle (lamg_hier) and the device-memory helpers shared by the solver files.
#pragma once

#include <chrono>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "device.h"
#include "internal.h"

namespace lamg {
struct BatchCtx;                  // multi-RHS / FP32-cycle workspace (batch.cu)
void batch_free(BatchCtx *b);
// 16-double slots of pinned host memory carved from process-lifetime slabs, so that creating
// and destroying hierarchies never calls cudaFreeHost (which can synchronise the device).
double *pinned_slot();
void pinned_release(double *p);
// Pinned host staging buffers of at least `bytes` from a process-lifetime pool (never freed, for
// the same reason); nullptr when no pinned memory can be had.
void *pinned_stage(size_t bytes);
void pinned_stage_release(void *p, size_t bytes);
}  // namespace lamg

struct lamg_hier {
    int device = 0;
    lamg_options opt{};
    std::vector<lamg::HostLevel> host;
    std::vector<lamg::DevLevel> dev;
    std::vector<lamg::Op> ops;
    cudaStream_t stream = nullptr;
    // outer CG vectors, device order of level 0
    double *r = nullptr, *p = nullptr, *q = nullptr, *zold = nullptr, *xs = nullptr, *bkeep = nullptr;
    double *nat_in = nullptr, *nat_out = nullptr;  // natural-order staging
    int32_t *perm0 = nullptr;
    lamg::Reduce red;
    double *h_scal = nullptr;  // pinned
    cudaGraphExec_t g_cycle = nullptr, g_tail = nullptr, g_head = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_poll = nullptr, ev_k0 = nullptr, ev_k1 = nullptr;
    // persistent solve kernel
    lamg::PSolve *psolve = nullptr;   // device copy
    lamg::PSolve ph{};                // host copy of the same pointers
    lamg::GridBar *bar = nullptr;
    double *hist = nullptr;
    int hist_cap = 0;
    int grid = 0;
    size_t smem = 0;
    bool persistent_ok = false;
    double cycle_bytes = 0.0;     // algorithmic DRAM bytes of one cycle (FP64, one RHS)
    double cycle_mat[2] = {0, 0}; // per cycle, read once whatever k: [FP64 cycle, FP32 cycle]
    double cycle_vec[2] = {0, 0}; // per cycle and right-hand side
    int64_t cycle_launches = 0;   // kernels of one cycle in the graph path
    // device copies of the level table, colour offsets and step list (persistent and cluster
    // kernels)
    lamg::PLevel *d_lv = nullptr;
    int32_t *d_cptr = nullptr;
    lamg::Op *d_ops = nullptr;
    int ncptr = 0;
    // cluster sub-cycle: steps on levels >= cluster_from run as one cluster launch per visit
    int cl_dim = 0;               // CTAs per cluster (0: cluster launch unavailable)
    int cluster_from = -1;        // -1: every step is its own kernel
    std::vector<double> tune_ms;  // cycle time of each candidate tried by the automatic choice
    std::vector<int> tune_from;
    // lamg_solve_many: cluster partial sums, results, residual history
    double *mg_part = nullptr, *mg_out = nullptr, *mg_hist = nullptr;
    int mg_hist_cap = 0;
    double setup_ms[lamg::SETUP_NPHASE + 1] = {0};   // + rounds of the GPU aggregation pass
    // multi-RHS / FP32 workspaces, one per (k, precision) used so far
    std::vector<lamg::BatchCtx *> batch;
    std::vector<void *> allocs;
    size_t dev_bytes = 0;
    double wait_timeout_s = 120.0;

    ~lamg_hier() {
        for (lamg::BatchCtx *b : batch) lamg::batch_free(b);
        if (ev_k0) cudaEventDestroy(ev_k0);
        if (ev_k1) cudaEventDestroy(ev_k1);
        if (g_cycle) cudaGraphExecDestroy(g_cycle);
        if (g_tail) cudaGraphExecDestroy(g_tail);
        if (g_head) cudaGraphExecDestroy(g_head);
        if (ev_a) cudaEventDestroy(ev_a);
        if (ev_b) cudaEventDestroy(ev_b);
        if (ev_poll) cudaEventDestroy(ev_poll);
        // stream-ordered frees: releasing one hierarchy never waits for other streams' work
        for (void *a : allocs) cudaFreeAsync(a, stream);
        if (h_scal) lamg::pinned_release(h_scal);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace lamg {

#define CKR(x)                                         \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

// Device allocation owned by the hierarchy (freed by lamg_destroy), 256-byte granularity,
// stream-ordered on the hierarchy's stream (which exists before the first allocation) and
// ready for any stream when this returns.
template <typename T>
inline int dalloc(lamg_hier *h, T **p, int64_t count) {
    size_t bytes = (size_t)(count > 1 ? count : 1) * sizeof(T);
    bytes = (bytes + 255) & ~(size_t)255;
    void *q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, bytes, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    h->allocs.push_back(q);
    h->dev_bytes += bytes;
    *p = (T *)q;
    return LAMG_OK;
}

template <typename T>
inline int dupload(lamg_hier *h, T **p, const std::vector<T> &v) {
    int rc = dalloc(h, p, (int64_t)v.size());
    if (rc) return rc;
    if (!v.empty()) {
        CKR(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
        CKR(cudaStreamSynchronize(h->stream));
    }
    return LAMG_OK;
}

// Bounded wait for an event recorded on one of the hierarchy's streams.
inline int wait_event(lamg_hier *h, cudaEvent_t ev) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return LAMG_OK;
        if (e != cudaErrorNotReady) return cuda_status(e);
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > h->wait_timeout_s) return LAMG_ERR_TIMEOUT;
    }
}

// Host <-> device copies of large caller vectors through pipelined pinned chunks (host_copy.cpp);
// d2h_staged returns once dst holds the data, h2d_staged once every chunk's DMA is queued and
// its staging buffer released. Waits are bounded by timeout_s. Worth it from
// staged_copy_min_bytes() on.
size_t staged_copy_min_bytes();
int h2d_staged(void *dst, const void *src, size_t bytes, cudaStream_t s, double timeout_s);
int d2h_staged(void *dst, const void *src, size_t bytes, cudaStream_t s, double timeout_s);

void op_bytes(const lamg_hier *h, const Op &op, double s, double *mat, double *vec);
bool many_eligible(const lamg_hier *h, size_t *smem);
// step i is a restriction that also performs step i + 1, the row-local start of the coarse
// level's first visit (with clusters: not when that step belongs to a cluster segment)
bool start_fusable(const lamg_hier *h, int i, bool clusters = true);
// Step i runs inside a cluster segment when the sub-cycle starts at level `from` (the
// hierarchy's own cluster_from in the two-argument form).
bool in_cluster_segment(const lamg_hier *h, int i, int from);
bool in_cluster_segment(const lamg_hier *h, int i);
int many_prepare(lamg_hier *h, int maxit, double tol, const double *b_in, double *phi_out, MGraph *M);
int solve_batch_impl(lamg_hier *h, int k, const double *B, double *PHI, const lamg_solve_opts *so,
                     lamg_stats *st, int prec);

}  // namespace lamg
