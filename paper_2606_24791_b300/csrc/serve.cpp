// Serving runtime (lamg_serve): continuous batching of many solves on one GPU.
//
// A request (a graph and one right-hand side, both copied) is admitted while the device memory
// it is estimated to need fits the server's budget next to the requests already in flight;
// otherwise it waits, in arrival order, until finished requests release memory. Admitted
// requests are set up by host worker threads (the setup's GPU kernels run on private streams).
// One executor thread keeps every ready request moving: each pass launches, for every request
// whose previous CG half-iteration has finished, the next one (CUDA graphs on that request's own
// stream), so the iterations of all in-flight requests overlap on the device, and requests that
// become ready join at the next pass. A finished request's hierarchy is released at once and its
// memory admits the next waiting request. Latency is measured from submission to the result.
//
// The arithmetic of a served solve is exactly that of lamg_solve on the same hierarchy (the
// same graphs and kernels), so a result is the same whether the request ran alone or in a mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "hier.h"

using namespace lamg;

namespace lamg {

// ------------------------------------------------------------------ pinned slots

namespace {
std::mutex g_pin_mu;
std::vector<double *> g_pin_free;
constexpr int SLOT_DOUBLES = 16;
constexpr int SLAB_SLOTS = 4096;
}  // namespace

double *pinned_slot() {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (g_pin_free.empty()) {
        double *slab = nullptr;
        if (cudaHostAlloc(&slab, SLAB_SLOTS * SLOT_DOUBLES * sizeof(double), cudaHostAllocDefault) != cudaSuccess)
            return nullptr;
        for (int i = SLAB_SLOTS - 1; i >= 0; i--) g_pin_free.push_back(slab + i * SLOT_DOUBLES);
    }
    double *p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void pinned_release(double *p) {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back(p);
}

namespace {
std::map<size_t, std::vector<void *>> g_stage_free;  // by power-of-two size
}

static size_t stage_class(size_t bytes) {
    size_t c = (size_t)1 << 20;
    while (c < bytes) c <<= 1;
    return c;
}

void *pinned_stage(size_t bytes) {
    const size_t c = stage_class(bytes);
    std::lock_guard<std::mutex> lock(g_pin_mu);
    std::vector<void *> &f = g_stage_free[c];
    if (!f.empty()) {
        void *p = f.back();
        f.pop_back();
        return p;
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pinned_stage_release(void *p, size_t bytes) {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_stage_free[stage_class(bytes)].push_back(p);
}

}  // namespace lamg

namespace {

enum { R_WAITING = 0, R_SETUP, R_RUNNING, R_DONE };

struct Request {
    int64_t id = 0, n = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> w, b, phi;
    int state = R_WAITING, status = LAMG_OK;
    size_t est = 0, held = 0;
    lamg_hier *h = nullptr;
    int phase = 0, it = 0;
    double rel = 1.0, relres_true = 0.0;
    double *pin_b = nullptr, *pin_x = nullptr;
    double t_submit = 0, t_admit = 0, t_ready = 0, t_done = 0;
};

// Pinned staging buffers for right-hand sides and solutions, reused across requests.
struct PinPool {
    std::mutex mu;
    std::multimap<size_t, double *> free;
    std::vector<double *> all;
    double *get(size_t n) {
        std::lock_guard<std::mutex> lock(mu);
        auto it = free.lower_bound(n);
        if (it != free.end()) {
            double *p = it->second;
            free.erase(it);
            return p;
        }
        double *p = nullptr;
        if (cudaHostAlloc(&p, std::max<size_t>(n, 1) * sizeof(double), cudaHostAllocDefault) != cudaSuccess) return nullptr;
        all.push_back(p);
        sizes[p] = n;
        return p;
    }
    void put(double *p) {
        if (!p) return;
        std::lock_guard<std::mutex> lock(mu);
        free.emplace(sizes[p], p);
    }
    void release_all() {
        for (double *p : all) cudaFreeHost(p);
        all.clear();
        free.clear();
    }
    std::map<double *, size_t> sizes;
};

// Device bytes a request's hierarchy is expected to take before it is built: operator levels
// shrink geometrically, so about twice the finest level's CSR plus the per-row vectors of all
// levels and of the outer iteration; corrected to the measured size once setup is done.
size_t estimate_bytes(int64_t n, int64_t nnz) {
    return (size_t)(32 * nnz + 320 * n) + ((size_t)8 << 20);
}

}  // namespace

// Requests solved together by one launch of the cluster solve kernel (one cluster each).
struct Group {
    std::vector<Request *> reqs;
    cudaEvent_t ev = nullptr;
    MGraph *d_desc = nullptr;
    double *pin_out = nullptr;   // MG_OUT results per request
};

struct lamg_server {
    lamg_server_opts so{};
    lamg_options opt{};
    std::mutex mu;
    std::condition_variable cv_setup, cv_done;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::deque<Request *> waiting, setup_q;
    std::vector<Request *> running;
    size_t used = 0;
    int inflight = 0;
    int64_t next_id = 1, outstanding = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::thread exec;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    PinPool pins;
    // grouped launches (executor thread only, counters read under mu)
    cudaStream_t gstream = nullptr;
    std::vector<Group> groups;
    int64_t n_groups = 0, n_grouped = 0, max_group = 0;
    // solves whose first launch was issued while another request's device work was in flight
    // (the executor's own record of requests sharing the device)
    int64_t n_overlap_starts = 0;

    // the executor's current pass over the ready requests (executor thread only)
    std::vector<Request *> pass;

    // another admitted request has launched work not yet seen complete (executor thread)
    bool device_busy_except(const Request *r) const {
        for (const Request *q : pass)
            if (q != r && (q->phase == 1 || q->phase == 2 || q->phase == 6)) return true;
        return !groups.empty();
    }

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }

    // Admit waiting requests in arrival order while memory and slots allow (mu held).
    void admit_locked() {
        while (!waiting.empty() && inflight < so.max_inflight) {
            Request *r = waiting.front();
            if (inflight > 0 && used + r->est > (size_t)so.budget_bytes) break;
            waiting.pop_front();
            used += r->est;
            r->held = r->est;
            inflight++;
            r->state = R_SETUP;
            r->t_admit = now_ms();
            setup_q.push_back(r);
            cv_setup.notify_one();
        }
    }

    void finish_locked(Request *r, int status) {
        r->status = status;
        r->state = R_DONE;
        r->t_done = now_ms();
        used -= std::min(used, r->held);
        r->held = 0;
        inflight--;
        outstanding--;
        admit_locked();
        cv_done.notify_all();
    }

    void setup_worker() {
        cudaSetDevice(so.device);
        for (;;) {
            Request *r = nullptr;
            {
                std::unique_lock<std::mutex> lock(mu);
                cv_setup.wait(lock, [&] { return stop || !setup_q.empty(); });
                if (stop) return;
                r = setup_q.front();
                setup_q.pop_front();
            }
            lamg_graph g{r->n, r->rp.data(), r->ci.data(), r->w.data()};
            lamg_hier *h = nullptr;
            const int rc = lamg_setup(&g, &opt, &h);
            std::lock_guard<std::mutex> lock(mu);
            if (rc) {
                finish_locked(r, rc);
                continue;
            }
            r->h = h;
            used = used - r->held + h->dev_bytes;
            r->held = h->dev_bytes;
            r->state = R_RUNNING;
            r->t_ready = now_ms();
            running.push_back(r);
        }
    }

    // Advance one request without blocking; returns true if anything was launched or finished.
    bool step(Request *r) {
        lamg_hier *h = r->h;
        cudaStream_t s = h->stream;
        const int64_t n = h->dev[0].n;
        cudaError_t e = cudaSuccess;
        switch (r->phase) {
            case 0: {
                if (device_busy_except(r)) {
                    std::lock_guard<std::mutex> lock(mu);
                    n_overlap_starts++;
                }
                r->pin_b = pins.get(n);
                r->pin_x = pins.get(n);
                if (!r->pin_b || !r->pin_x) { r->phase = 4; r->status = LAMG_ERR_OOM; return true; }
                std::copy(r->b.begin(), r->b.end(), r->pin_b);
                cudaMemcpyAsync(h->nat_in, r->pin_b, n * sizeof(double), cudaMemcpyHostToDevice, s);
                launch_gather(n, h->perm0, h->nat_in, h->r, s);
                launch_sum(n, h->r, h->red, s);
                launch_init_b(n, h->r, h->bkeep, h->xs, h->p, h->zold, h->red, s);
                cudaGraphLaunch(h->g_tail, s);
                cudaGraphLaunch(h->g_head, s);
                e = cudaEventRecord(h->ev_poll, s);
                r->phase = 1;
                break;
            }
            case 1: {
                e = cudaEventQuery(h->ev_poll);
                if (e == cudaErrorNotReady) return false;
                if (e != cudaSuccess) break;
                r->it++;
                const double bn2 = h->h_scal[S_BN2];
                r->rel = bn2 > 0 ? std::sqrt(h->h_scal[S_RR] / bn2) : 0.0;
                if (!(r->rel > so.tol) || r->it >= so.maxit) {
                    launch_true_resid(h->dev[0], h->xs, h->bkeep, h->red, s);
                    launch_scatter(n, h->perm0, h->xs, h->nat_out, s);
                    cudaMemcpyAsync(r->pin_x, h->nat_out, n * sizeof(double), cudaMemcpyDeviceToHost, s);
                    cudaMemcpyAsync(h->h_scal, h->red.scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
                    e = cudaEventRecord(h->ev_b, s);
                    r->phase = 2;
                } else {
                    cudaGraphLaunch(h->g_tail, s);
                    cudaGraphLaunch(h->g_head, s);
                    e = cudaEventRecord(h->ev_poll, s);
                }
                break;
            }
            case 2: {
                e = cudaEventQuery(h->ev_b);
                if (e == cudaErrorNotReady) return false;
                if (e != cudaSuccess) break;
                r->phi.assign(r->pin_x, r->pin_x + n);
                const double bn2 = h->h_scal[S_BN2];
                r->relres_true = bn2 > 0 ? std::sqrt(h->h_scal[S_TRUE_RR] / bn2) : 0.0;
                r->status = r->rel <= so.tol ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
                r->phase = 4;
                return true;
            }
            default:
                return false;
        }
        if (e != cudaSuccess && e != cudaErrorNotReady) {
            r->status = cuda_status(e);
            r->phase = 4;
        }
        return true;
    }

    // Launch every request in `fresh` (ready, not started, taken by the cluster kernel) as one
    // group: copies in, one k_cluster_solve launch, copies out, an event; phase 6 until done.
    void launch_group(std::vector<Request *> &fresh) {
        Group g;
        std::vector<MGraph> desc(fresh.size());
        int64_t overlapped = 0;
        {
            bool busy = !groups.empty();
            for (const Request *q : pass)
                if (std::find(fresh.begin(), fresh.end(), q) == fresh.end() && (q->phase == 1 || q->phase == 2 || q->phase == 6))
                    busy = true;
            overlapped = busy ? (int64_t)fresh.size() : 0;
        }
        int cl = 16;
        size_t smem = 0;
        cudaError_t e = cudaSuccess;
        g.pin_out = pins.get(MG_OUT * fresh.size());
        for (size_t k = 0; k < fresh.size() && e == cudaSuccess; k++) {
            Request *r = fresh[k];
            lamg_hier *h = r->h;
            const int64_t n = h->dev[0].n;
            size_t sm = 0;
            many_eligible(h, &sm);
            cl = std::min(cl, h->cl_dim);
            smem = std::max(smem, sm);
            r->pin_b = pins.get(n);
            r->pin_x = pins.get(n);
            if (!r->pin_b || !r->pin_x || !g.pin_out) { e = cudaErrorMemoryAllocation; break; }
            std::copy(r->b.begin(), r->b.end(), r->pin_b);
            e = cudaMemcpyAsync(h->nat_in, r->pin_b, n * sizeof(double), cudaMemcpyHostToDevice, gstream);
            if (e == cudaSuccess && many_prepare(h, so.maxit, so.tol, h->nat_in, h->nat_out, &desc[k]) != LAMG_OK)
                e = cudaErrorMemoryAllocation;
        }
        if (e == cudaSuccess) e = cudaMallocAsync(&g.d_desc, desc.size() * sizeof(MGraph), gstream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g.d_desc, desc.data(), desc.size() * sizeof(MGraph), cudaMemcpyHostToDevice, gstream);
        if (e == cudaSuccess) e = launch_cluster_solve(g.d_desc, (int)fresh.size(), cl, smem, gstream);
        for (size_t k = 0; k < fresh.size() && e == cudaSuccess; k++) {
            lamg_hier *h = fresh[k]->h;
            e = cudaMemcpyAsync(fresh[k]->pin_x, h->nat_out, h->dev[0].n * sizeof(double), cudaMemcpyDeviceToHost,
                                gstream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(g.pin_out + k * MG_OUT, h->mg_out, MG_OUT * sizeof(double),
                                    cudaMemcpyDeviceToHost, gstream);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(g.ev, gstream);
        g.reqs = fresh;
        for (Request *r : fresh) r->phase = 6;
        if (e != cudaSuccess) {
            cudaGetLastError();
            // copies already queued on gstream may still read the requests' device inputs and
            // pinned buffers: let them finish before those are released (phase 4 frees them)
            cudaStreamSynchronize(gstream);
            cudaGetLastError();
            if (g.d_desc) cudaFreeAsync(g.d_desc, gstream);
            for (Request *r : fresh) { r->status = cuda_status(e); r->phase = 4; }
            if (g.ev) cudaEventDestroy(g.ev);
            pins.put(g.pin_out);
            return;
        }
        {
            std::lock_guard<std::mutex> lock(mu);
            n_groups++;
            n_grouped += (int64_t)fresh.size();
            n_overlap_starts += overlapped;
            max_group = std::max<int64_t>(max_group, (int64_t)fresh.size());
        }
        groups.push_back(std::move(g));
    }

    // Finish the groups whose launch has completed; true if any did.
    bool poll_groups() {
        bool any = false;
        for (size_t i = 0; i < groups.size();) {
            Group &g = groups[i];
            const cudaError_t e = cudaEventQuery(g.ev);
            if (e == cudaErrorNotReady) { i++; continue; }
            for (size_t k = 0; k < g.reqs.size(); k++) {
                Request *r = g.reqs[k];
                if (e != cudaSuccess) {
                    r->status = cuda_status(e);
                } else {
                    const double *o = g.pin_out + k * MG_OUT;
                    const double bn2 = o[MG_BN2];
                    r->it = (int)o[MG_ITERS];
                    r->rel = bn2 > 0 ? std::sqrt(o[MG_RR] / bn2) : 0.0;
                    r->relres_true = bn2 > 0 ? std::sqrt(o[MG_TRUE_RR] / bn2) : 0.0;
                    r->phi.assign(r->pin_x, r->pin_x + r->h->dev[0].n);
                    r->status = r->rel <= so.tol ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
                }
                r->phase = 4;
            }
            cudaEventDestroy(g.ev);
            cudaFreeAsync(g.d_desc, gstream);
            pins.put(g.pin_out);
            groups.erase(groups.begin() + i);
            any = true;
        }
        return any;
    }

    void executor() {
        cudaSetDevice(so.device);
        cudaStreamCreateWithFlags(&gstream, cudaStreamNonBlocking);
        std::vector<Request *> act, fresh;
        for (;;) {
            {
                std::lock_guard<std::mutex> lock(mu);
                if (stop) break;
                act = running;
            }
            pass = act;
            // continuous batching: every request whose setup finished since the last pass and
            // that the cluster kernel takes joins one launch
            fresh.clear();
            for (Request *r : act)
                if (r->phase == 0 && many_eligible(r->h, nullptr)) fresh.push_back(r);
            bool progressed = false;
            if (!fresh.empty()) {
                launch_group(fresh);
                progressed = true;
            }
            progressed |= poll_groups();
            for (Request *r : act) {
                progressed |= step(r);
                if (r->phase == 4) {
                    lamg_hier *h = r->h;
                    r->h = nullptr;
                    cudaStreamSynchronize(h->stream);
                    lamg_destroy(h);
                    pins.put(r->pin_b);
                    pins.put(r->pin_x);
                    r->pin_b = r->pin_x = nullptr;
                    std::lock_guard<std::mutex> lock(mu);
                    running.erase(std::find(running.begin(), running.end(), r));
                    finish_locked(r, r->status);
                }
            }
            if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        // stopping: let launched groups finish before their hierarchies are released
        if (gstream) cudaStreamSynchronize(gstream);
        for (Group &g : groups) {
            cudaEventDestroy(g.ev);
            pins.put(g.pin_out);
        }
        groups.clear();
        if (gstream) cudaStreamDestroy(gstream);
    }
};

extern "C" {

int lamg_server_create(const lamg_server_opts *so, const lamg_options *opt, lamg_server **out) {
    if (!out || !so || !(so->budget_bytes > 0) || so->max_inflight < 1 || !(so->tol > 0) || so->maxit < 1)
        return LAMG_ERR_INVALID;
    *out = nullptr;
    int cnt = 0;
    if (cudaGetDeviceCount(&cnt) != cudaSuccess || cnt == 0) return LAMG_ERR_NO_DEVICE;
    if (so->device < 0 || so->device >= cnt) return LAMG_ERR_INVALID;
    lamg_server *s = new lamg_server();
    s->so = *so;
    if (opt) s->opt = *opt;
    else lamg_options_default(&s->opt);
    s->opt.device = so->device;
    // a served setup runs no timing trials (kernel forms, launch schedule): they would queue
    // behind other requests' solves and lengthen every setup
    s->opt.autotune = 0;
    if (s->opt.cluster_rows == 0) s->opt.cluster_rows = -1;
    // one solve per setup: the default coarsest size rule trades a larger dense inverse at setup
    // for fewer levels in every later solve, which a one-shot request never recovers
    if (s->opt.coarsest_max == 0) s->opt.coarsest_max = 1024;
    const int nw = std::max(1, so->setup_threads);
    for (int i = 0; i < nw; i++) s->workers.emplace_back([s] { s->setup_worker(); });
    s->exec = std::thread([s] { s->executor(); });
    *out = s;
    return LAMG_OK;
}

int lamg_serve(lamg_server *s, const lamg_graph *g, const double *b, int64_t *ticket) {
    if (!s || !g || !b || !ticket || g->n < 1 || !g->rp) return LAMG_ERR_INVALID;
    const int64_t n = g->n, z = g->rp[n];
    if (z < 0 || (z > 0 && (!g->ci || !g->w))) return LAMG_ERR_INVALID;
    const size_t est = estimate_bytes(n, z);
    if (est > (size_t)s->so.budget_bytes) return LAMG_ERR_ADMISSION;
    auto r = std::make_unique<Request>();
    r->n = n;
    r->rp.assign(g->rp, g->rp + n + 1);
    r->ci.assign(g->ci, g->ci + z);
    r->w.assign(g->w, g->w + z);
    r->b.assign(b, b + n);
    r->est = est;
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    r->t_submit = s->now_ms();
    *ticket = r->id;
    s->waiting.push_back(r.get());
    s->reqs[r->id] = std::move(r);
    s->outstanding++;
    s->admit_locked();
    return LAMG_OK;
}

int lamg_serve_poll(lamg_server *s, int64_t ticket, lamg_ticket_info *info, double *phi) {
    if (!s || !info) return LAMG_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LAMG_ERR_INVALID;
    const Request *r = it->second.get();
    std::memset(info, 0, sizeof(*info));
    info->done = r->state == R_DONE;
    info->status = r->status;
    info->iters = r->it;
    info->relres = r->rel;
    info->relres_true = r->relres_true;
    info->t_submit_ms = r->t_submit;
    info->t_admit_ms = r->t_admit;
    info->t_ready_ms = r->t_ready;
    info->t_done_ms = r->t_done;
    if (info->done && phi && !r->phi.empty()) std::copy(r->phi.begin(), r->phi.end(), phi);
    return LAMG_OK;
}

int lamg_server_drain(lamg_server *s, double timeout_s) {
    if (!s) return LAMG_ERR_INVALID;
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                        [&] { return s->outstanding == 0; });
    return ok ? LAMG_OK : LAMG_ERR_TIMEOUT;
}

int lamg_server_stats(lamg_server *s, int64_t *out) {
    if (!s || !out) return LAMG_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    out[0] = (int64_t)s->used;
    out[1] = s->inflight;
    out[2] = (int64_t)s->waiting.size();
    out[3] = s->outstanding;
    out[4] = s->n_groups;
    out[5] = s->n_grouped;
    out[6] = s->max_group;
    out[7] = s->n_overlap_starts;
    return LAMG_OK;
}

void lamg_server_destroy(lamg_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_setup.notify_all();
    for (auto &t : s->workers) t.join();
    s->exec.join();
    for (auto &kv : s->reqs) {
        Request *r = kv.second.get();
        if (r->h) lamg_destroy(r->h);
    }
    s->pins.release_all();
    delete s;
}

}  // extern "C"
