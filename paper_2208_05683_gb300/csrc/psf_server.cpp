// psf_server.cpp -- serving loop with continuous batching (psf_server_*).
//
// Requests wait in one FIFO.  Each worker thread owns a CUDA stream; when it
// is free it admits the oldest waiting requests that fit its batch size and
// the device-memory budget and evaluates them together (psf_eval_batch, one
// block-diagonal batch) on its stream.  Several workers run batches at the
// same time, so requests arriving while others are on the GPU start as soon
// as a worker and memory are free and their kernels overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "psf_internal.h"

using namespace psf::host;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    psf_series_t series;
    psf_csr_t Z;
    uint64_t tag;
    Clock::time_point t_submit;
    long long bytes;  // predicted device footprint
};

// Predicted device memory of one request: the entry pool of its PS phase
// (pool + two candidate lists, 36 bytes per entry, sized for up to 400
// entries per entry of Z, as for a 2D Laplacian of 1-norm 4 at tol 1e-12)
// and the per-row arrays (column-sum words, row slots: about 1 KB per row).
long long predict_bytes(const psf_csr_t& Z) {
    return (long long)Z.nnz * 400LL * 36LL + (long long)Z.n * 1024LL + (1LL << 20);
}

}  // namespace

struct psf_server_s {
    psf_server_config_t cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::deque<psf_completion_t> done;
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;  // one per worker; destroyed with the server
    bool stopping = false;
    long long inflight_bytes = 0;
    int busy = 0;
    psf_server_stats_t st{};

    void worker(cudaStream_t stream);
};

void psf_server_s::worker(cudaStream_t stream) {
    cudaSetDevice(device);
    std::vector<Request> batch;
    for (;;) {
        batch.clear();
        long long bytes = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (!pending.empty()) {
                    // admit the oldest requests that fit (the first one always
                    // fits when nothing else is in flight)
                    while (!pending.empty() && (int)batch.size() < cfg.max_batch) {
                        const Request& r = pending.front();
                        const bool fits = inflight_bytes + bytes + r.bytes <= cfg.hbm_budget;
                        if (!fits && !(batch.empty() && inflight_bytes == 0)) break;
                        bytes += r.bytes;
                        batch.push_back(r);
                        pending.pop_front();
                    }
                    if (!batch.empty()) break;
                }
                if (stopping && pending.empty()) break;
                cv_work.wait(lk);
            }
            if (batch.empty()) break;  // stopping
            inflight_bytes += bytes;
            ++busy;
            ++st.batches;
            st.max_concurrent = std::max(st.max_concurrent, busy);
            st.budget_peak = std::max(st.budget_peak, (int64_t)inflight_bytes);
        }
        const Clock::time_point t_admit = Clock::now();
        // fault injection (PSF_TUNE_FAIL_ADMISSION): the request whose
        // admission brings the count down to zero fails as if its device
        // memory could not be allocated; the rest of the batch runs
        std::vector<psf_completion_t> failed_adm;
        for (size_t i = 0; i < batch.size();) {
            long long k = g_fail_admission.load();
            bool inject = false;
            while (k > 0 && !g_fail_admission.compare_exchange_weak(k, k - 1)) {
            }
            inject = k == 1;
            if (!inject) {
                ++i;
                continue;
            }
            psf_completion_t c{};
            c.tag = batch[i].tag;
            c.status = PSF_ENOMEM;
            c.batch_size = (int)batch.size();
            c.queue_ms = ms_between(batch[i].t_submit, t_admit);
            c.latency_ms = ms_between(batch[i].t_submit, Clock::now());
            failed_adm.push_back(c);
            batch.erase(batch.begin() + (long)i);
        }
        if (!failed_adm.empty()) {
            std::lock_guard<std::mutex> lk(mu);
            for (const psf_completion_t& c : failed_adm) {
                done.push_back(c);
                ++st.completed;
                ++st.failed;
            }
        }
        if (batch.empty()) {
            {
                std::lock_guard<std::mutex> lk(mu);
                inflight_bytes -= bytes;
                --busy;
            }
            cv_done.notify_all();
            cv_work.notify_all();
            continue;
        }
        const int count = (int)batch.size();
        std::vector<psf_series_t> ser((size_t)count);
        std::vector<psf_csr_t> zs((size_t)count);
        std::vector<psf_result_t> outs((size_t)count, nullptr);
        std::vector<int> status((size_t)count, PSF_OK);
        for (int i = 0; i < count; ++i) {
            ser[(size_t)i] = batch[(size_t)i].series;
            zs[(size_t)i] = batch[(size_t)i].Z;
        }
        int rc = psf_eval_batch(ser.data(), zs.data(), count, stream, outs.data());
        if (rc != PSF_OK) {
            // find the failing request(s): evaluate one by one
            for (int i = 0; i < count; ++i) {
                outs[(size_t)i] = nullptr;
                status[(size_t)i] = psf_eval_batch(&ser[(size_t)i], &zs[(size_t)i], 1, stream, &outs[(size_t)i]);
            }
        }
        cudaStreamSynchronize(stream);
        const Clock::time_point t_end = Clock::now();
        {
            std::lock_guard<std::mutex> lk(mu);
            for (int i = 0; i < count; ++i) {
                psf_completion_t c{};
                c.tag = batch[(size_t)i].tag;
                c.status = status[(size_t)i];
                c.batch_size = count;
                c.result = status[(size_t)i] == PSF_OK ? outs[(size_t)i] : nullptr;
                c.queue_ms = ms_between(batch[(size_t)i].t_submit, t_admit);
                c.latency_ms = ms_between(batch[(size_t)i].t_submit, t_end);
                done.push_back(c);
                ++st.completed;
                if (c.status != PSF_OK) ++st.failed;
            }
            inflight_bytes -= bytes;
            --busy;
        }
        cv_done.notify_all();
        cv_work.notify_all();  // memory was freed
    }
}

extern "C" {

int psf_server_create(const psf_server_config_t* config, psf_server_t* out) {
    if (!out) return fail(PSF_EINVAL, "out is null");
    *out = nullptr;
    psf_server_config_t cfg{};
    if (config) cfg = *config;
    if (cfg.workers <= 0) cfg.workers = 4;
    if (cfg.max_batch <= 0) cfg.max_batch = 64;
    if (cfg.workers > 64) return fail(PSF_EINVAL, "at most 64 workers");
    if (cfg.max_batch > 1024) return fail(PSF_EINVAL, "max_batch must be <= 1024");
    int rc = prepare(nullptr);
    if (rc) return rc;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (cfg.hbm_budget <= 0) {
        size_t fr = 0, tot = 0;
        CU(cudaMemGetInfo(&fr, &tot));
        cfg.hbm_budget = (int64_t)(fr / 2);
    }
    psf_server_s* s = new (std::nothrow) psf_server_s();
    if (!s) return fail(PSF_ENOMEM, "host allocation");
    s->cfg = cfg;
    s->device = dev;
    for (int i = 0; i < cfg.workers; ++i) {
        cudaStream_t q = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return fail(PSF_ECUDA, "worker stream: %s", cudaGetErrorString(e));
        }
        s->streams.push_back(q);
    }
    try {
        for (int i = 0; i < cfg.workers; ++i) {
            cudaStream_t q = s->streams[(size_t)i];
            s->threads.emplace_back([s, q] { s->worker(q); });
        }
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
        }
        s->cv_work.notify_all();
        for (auto& t : s->threads) t.join();
        for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
        delete s;
        return fail(PSF_ENOMEM, "cannot start worker threads");
    }
    *out = s;
    return PSF_OK;
}

int psf_server_submit(psf_server_t s, psf_series_t series, const psf_csr_t* Z, uint64_t tag) {
    if (!s || !series || !Z) return fail(PSF_EINVAL, "null argument");
    if (series->flags & PSF_Z_ESTIMATE) return fail(PSF_EINVAL, "PSF_Z_ESTIMATE is for psf_eval only");
    int rc = check_csr(Z, Z->n, "Z");
    if (rc) return rc;
    Request r{series, *Z, tag, Clock::now(), predict_bytes(*Z)};
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return fail(PSF_EINVAL, "server is shutting down");
        s->pending.push_back(r);
        ++s->st.submitted;
    }
    s->cv_work.notify_one();
    return PSF_OK;
}

int psf_server_cancel(psf_server_t s, uint64_t tag, int32_t* cancelled) {
    if (!s || !cancelled) return fail(PSF_EINVAL, "null argument");
    *cancelled = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
            if (it->tag != tag) continue;
            psf_completion_t c{};
            c.tag = tag;
            c.status = PSF_ECANCELED;
            c.queue_ms = c.latency_ms = ms_between(it->t_submit, Clock::now());
            s->pending.erase(it);
            s->done.push_back(c);
            ++s->st.completed;
            ++s->st.cancelled;
            *cancelled = 1;
            break;
        }
    }
    if (*cancelled) {
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    return PSF_OK;
}

int psf_server_poll(psf_server_t s, psf_completion_t* out, int32_t max, int32_t wait_ms, int32_t* got) {
    if (!s || !got || (max > 0 && !out)) return fail(PSF_EINVAL, "null argument");
    *got = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return !s->done.empty() || (s->pending.empty() && s->busy == 0); };
    if (wait_ms < 0) {
        s->cv_done.wait(lk, ready);
    } else if (wait_ms > 0) {
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    }
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *got = n;
    return PSF_OK;
}

int psf_server_stats(psf_server_t s, psf_server_stats_t* stats) {
    if (!s || !stats) return fail(PSF_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *stats = s->st;
    stats->pending = (int32_t)s->pending.size();
    return PSF_OK;
}

int psf_server_destroy(psf_server_t s) {
    if (!s) return PSF_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->threads) t.join();
    for (psf_completion_t& c : s->done)
        if (c.result) psf_result_destroy(c.result);
    for (cudaStream_t x : s->streams) {
        cudaStreamSynchronize(x);
        cudaStreamDestroy(x);
    }
    delete s;
    return PSF_OK;
}

}  // extern "C"
