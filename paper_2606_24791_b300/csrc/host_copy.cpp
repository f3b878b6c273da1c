// Large host <-> device copies of caller vectors (lamg_solve_batch with host pointers): the
// caller's pageable memory is copied through pinned staging chunks, the host side of each chunk
// split over a few worker threads, the DMA of one chunk overlapping the host copy of the next.
// A pageable cudaMemcpy of 1 GB runs at a fraction of the link's rate (the driver stages it
// through a small pinned buffer with one thread); this path keeps both the copy threads and the
// DMA engine busy.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "hier.h"

namespace lamg {

namespace {

// A fixed set of worker threads running one parallel memcpy at a time.
class CopyPool {
  public:
    // Created on first use and never destroyed: its detached workers wait on the condition
    // variable for the life of the process, and destroying a condition variable that has waiters
    // would block (glibc waits for them) when the process exits.
    static CopyPool &get() {
        static CopyPool *pool = new CopyPool();
        return *pool;
    }
    // dst[0, bytes) = src[0, bytes), split into nthreads() slices copied concurrently.
    void copy(void *dst, const void *src, size_t bytes) {
        std::lock_guard<std::mutex> one(call_mu_);
        const int nt = (int)workers_.size() + 1;
        const size_t slice = ((bytes / nt) + 4095) & ~(size_t)4095;
        {
            std::lock_guard<std::mutex> lk(mu_);
            dst_ = (char *)dst;
            src_ = (const char *)src;
            bytes_ = bytes;
            slice_ = slice;
            pending_ = (int)workers_.size();
            gen_++;
        }
        cv_.notify_all();
        part(0);  // the calling thread takes slice 0
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return pending_ == 0; });
    }

  private:
    CopyPool() {
        // one copying thread per hardware thread (the caller included), at most 32: a host
        // memcpy from pageable memory runs at ~10 GB/s on one thread and the host's memory
        // system saturates near 43 GB/s with 16 (measured on a 16-thread B300 host, where the
        // pinned DMA runs at 55 GB/s each way); the caller waits for the copy anyway
        const unsigned hw = std::max(2u, std::thread::hardware_concurrency());
        const int n = (int)std::min(31u, hw - 1);
        for (int i = 0; i < n; i++) workers_.emplace_back([this, i] { loop(i + 1); });
        for (auto &t : workers_) t.detach();   // process-lifetime pool
    }
    void part(int i) {
        const size_t a = std::min(bytes_, (size_t)i * slice_), b = std::min(bytes_, a + slice_);
        if (b > a) std::memcpy(dst_ + a, src_ + a, b - a);
    }
    void loop(int i) {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
            }
            part(i);
            std::lock_guard<std::mutex> lk(mu_);
            if (--pending_ == 0) done_cv_.notify_one();
        }
    }
    std::vector<std::thread> workers_;
    std::mutex call_mu_, mu_;
    std::condition_variable cv_, done_cv_;
    char *dst_ = nullptr;
    const char *src_ = nullptr;
    size_t bytes_ = 0, slice_ = 0;
    int pending_ = 0;
    uint64_t gen_ = 0;
};

constexpr size_t CHUNK = (size_t)64 << 20;
constexpr int NBUF = 3;

// Bounded wait for an event (LAMG_OK, LAMG_ERR_TIMEOUT or the CUDA error's code).
int wait_ev(cudaEvent_t ev, double timeout_s) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return LAMG_OK;
        if (e != cudaErrorNotReady) return cuda_status(e);
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s)
            return LAMG_ERR_TIMEOUT;
        std::this_thread::yield();
    }
}

// NBUF pinned chunks from the process pool, each with the event of its last DMA. A chunk whose
// DMA cannot be confirmed complete is not returned to the pool.
struct Buffers {
    void *p[NBUF] = {nullptr};
    cudaEvent_t ev[NBUF] = {nullptr};
    bool used[NBUF] = {false};
    double timeout_s;
    bool ok = true;
    explicit Buffers(double t) : timeout_s(t) {
        for (int i = 0; i < NBUF; i++) {
            p[i] = pinned_stage(CHUNK);
            if (!p[i] || cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) ok = false;
        }
    }
    ~Buffers() {
        for (int i = 0; i < NBUF; i++) {
            const bool idle = !used[i] || (ev[i] && wait_ev(ev[i], timeout_s) == LAMG_OK);
            if (ev[i]) cudaEventDestroy(ev[i]);
            if (p[i] && idle) pinned_stage_release(p[i], CHUNK);
        }
    }
};

}  // namespace

size_t staged_copy_min_bytes() { return 2 * CHUNK; }

int h2d_staged(void *dst, const void *src, size_t bytes, cudaStream_t s, double timeout_s) {
    Buffers B(timeout_s);
    if (!B.ok) return cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    int rc = LAMG_OK;
    for (size_t off = 0, c = 0; off < bytes && rc == LAMG_OK; off += CHUNK, c++) {
        const int i = (int)(c % NBUF);
        const size_t nb = std::min(CHUNK, bytes - off);
        if (B.used[i] && (rc = wait_ev(B.ev[i], timeout_s))) break;   // the chunk's previous DMA is done
        CopyPool::get().copy(B.p[i], (const char *)src + off, nb);
        rc = cuda_status(cudaMemcpyAsync((char *)dst + off, B.p[i], nb, cudaMemcpyHostToDevice, s));
        if (rc == LAMG_OK) rc = cuda_status(cudaEventRecord(B.ev[i], s));
        B.used[i] = true;
    }
    return rc;   // ~Buffers waits for the last DMAs before the chunks go back to the pool
}

int d2h_staged(void *dst, const void *src, size_t bytes, cudaStream_t s, double timeout_s) {
    Buffers B(timeout_s);
    if (!B.ok) {
        cudaEvent_t ev = nullptr;
        int rc = cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
        if (rc == LAMG_OK) rc = cuda_status(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (rc == LAMG_OK) rc = cuda_status(cudaEventRecord(ev, s));
        if (rc == LAMG_OK) rc = wait_ev(ev, timeout_s);
        if (ev) cudaEventDestroy(ev);
        return rc;
    }
    const size_t nchunk = (bytes + CHUNK - 1) / CHUNK;
    int rc = LAMG_OK;
    // NBUF DMAs queued ahead of the host copy
    auto issue = [&](size_t c) {
        const int i = (int)(c % NBUF);
        const size_t off = c * CHUNK, nb = std::min(CHUNK, bytes - off);
        B.used[i] = true;
        int r = cuda_status(cudaMemcpyAsync(B.p[i], (const char *)src + off, nb, cudaMemcpyDeviceToHost, s));
        return r == LAMG_OK ? cuda_status(cudaEventRecord(B.ev[i], s)) : r;
    };
    for (size_t c = 0; c < std::min<size_t>(NBUF, nchunk) && rc == LAMG_OK; c++) rc = issue(c);
    for (size_t c = 0; c < nchunk && rc == LAMG_OK; c++) {
        const int i = (int)(c % NBUF);
        const size_t off = c * CHUNK, nb = std::min(CHUNK, bytes - off);
        if ((rc = wait_ev(B.ev[i], timeout_s))) break;
        CopyPool::get().copy((char *)dst + off, B.p[i], nb);
        if (c + NBUF < nchunk) rc = issue(c + NBUF);
    }
    return rc;
}

}  // namespace lamg
