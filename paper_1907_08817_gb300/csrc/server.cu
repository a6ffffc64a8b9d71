// server.cu -- continuous-batching sort server: admission against an HBM budget, a queue of
// admitted requests, and worker threads that each own a CUDA stream and turn whatever is queued
// into their next batch (copy in, per-request device training, one batched sort, copy out).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "nnsort.h"

namespace {

struct Req {
    uint64_t id = 0;
    void *h_keys = nullptr;
    int32_t *h_pay = nullptr;
    uint64_t n = 0;
    int32_t dtype = 0;
    uint64_t seed = 0;
    size_t bytes = 0;
    double t_submit = 0.0, t_done = 0.0;
    int status = NNSORT_PENDING;
    nnsort_stats st{};
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int key_bytes(int dt) { return (dt == NNSORT_F32 || dt == NNSORT_U32) ? 4 : 8; }

}  // namespace

struct nnsort_server {
    nnsort_server_opts o;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> waiting;  // submitted, waiting for budget (arrival order)
    std::deque<uint64_t> ready;    // admitted, not yet in a batch
    std::map<uint64_t, Req> reqs;
    size_t used = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

// device bytes a request holds while it is processed (its arrays, its share of the stream's
// sort workspace and the training buffers)
size_t request_bytes(const nnsort_server *s, uint64_t n, int dtype, bool pay) {
    const size_t kb = key_bytes(dtype);
    const uint64_t S = s->o.train.sample_n ? s->o.train.sample_n : 1;
    return n * kb + (pay ? n * 4 : 0) + nnsort_workspace_bytes(n, dtype, pay ? 1 : 0, &s->o.sort) +
           S * (2 * kb + 16) + (1u << 20);
}

void admit_locked(nnsort_server *s) {
    while (!s->waiting.empty()) {
        Req &r = s->reqs[s->waiting.front()];
        if (s->used + r.bytes > s->o.hbm_budget) break;
        s->used += r.bytes;
        s->ready.push_back(r.id);
        s->waiting.pop_front();
    }
    s->cv_work.notify_all();
}

void worker_main(nnsort_server *s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    for (;;) {
        std::vector<Req> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return !s->ready.empty() || (s->stop && s->waiting.empty()); });
            if (s->ready.empty()) break;  // stopping and nothing left to do
            // this worker's next batch: queued requests of the first one's key type
            const int32_t dt = s->reqs[s->ready.front()].dtype;
            uint64_t keys = 0;
            for (auto it = s->ready.begin(); it != s->ready.end() && (int)batch.size() < s->o.max_batch;) {
                Req &r = s->reqs[*it];
                if (r.dtype != dt || (!batch.empty() && s->o.max_batch_keys &&
                                      keys + r.n > s->o.max_batch_keys)) {
                    ++it;
                    continue;
                }
                keys += r.n;
                batch.push_back(r);
                it = s->ready.erase(it);
            }
        }
        const int cnt = (int)batch.size();
        const int32_t dt = batch[0].dtype;
        const size_t kb = key_bytes(dt);
        std::vector<void *> dk(cnt, nullptr);
        std::vector<int32_t *> dp(cnt, nullptr);
        std::vector<nnsort_model *> models(cnt, nullptr);
        std::vector<int> rc(cnt, NNSORT_OK);
        for (int i = 0; i < cnt; ++i) {
            const Req &r = batch[i];
            if (cudaMallocAsync(&dk[i], r.n * kb, st) != cudaSuccess ||
                (r.h_pay && cudaMallocAsync((void **)&dp[i], r.n * 4, st) != cudaSuccess)) {
                cudaGetLastError();
                rc[i] = NNSORT_E_OOM;
                continue;
            }
            cudaMemcpyAsync(dk[i], r.h_keys, r.n * kb, cudaMemcpyHostToDevice, st);
            if (r.h_pay) cudaMemcpyAsync(dp[i], r.h_pay, r.n * 4, cudaMemcpyHostToDevice, st);
        }
        for (int i = 0; i < cnt; ++i) {
            if (rc[i]) continue;
            nnsort_train_opts to = s->o.train;
            to.seed = batch[i].seed;
            to.sample_n = std::max<uint64_t>(1, std::min<uint64_t>(to.sample_n, batch[i].n));
            rc[i] = nnsort_train(dk[i], batch[i].n, dt, &to, &models[i], nullptr, st);
        }
        // one pass of the pipeline over every request that trained
        std::vector<void *> sk;
        std::vector<int32_t *> sp;
        std::vector<uint64_t> sn;
        std::vector<const nnsort_model *> sf;
        std::vector<int> idx;
        bool anypay = false;
        for (int i = 0; i < cnt; ++i) {
            if (rc[i]) continue;
            sk.push_back(dk[i]);
            sp.push_back(dp[i]);
            sn.push_back(batch[i].n);
            sf.push_back(models[i]);
            idx.push_back(i);
            anypay |= dp[i] != nullptr;
        }
        std::vector<nnsort_stats> sst(idx.size());
        if (!idx.empty()) {
            nnsort_sort_opts so = s->o.sort;
            so.d_slots = nullptr;
            so.d_fate = nullptr;
            const int b = nnsort_sort_batch(sk.data(), anypay ? sp.data() : nullptr, sn.data(),
                                            (int32_t)idx.size(), dt, sf.data(), &so, sst.data(), st);
            for (size_t q = 0; q < idx.size(); ++q) rc[idx[q]] = b;
        }
        for (int i = 0; i < cnt; ++i) {
            if (rc[i] == NNSORT_OK) {
                cudaMemcpyAsync(batch[i].h_keys, dk[i], batch[i].n * kb, cudaMemcpyDeviceToHost, st);
                if (dp[i]) cudaMemcpyAsync(batch[i].h_pay, dp[i], batch[i].n * 4, cudaMemcpyDeviceToHost, st);
            }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            for (int i = 0; i < cnt; ++i) if (!rc[i]) rc[i] = NNSORT_E_CUDA;
        }
        for (int i = 0; i < cnt; ++i) {
            if (models[i]) nnsort_model_free(models[i]);
            if (dk[i]) cudaFreeAsync(dk[i], st);
            if (dp[i]) cudaFreeAsync(dp[i], st);
        }
        cudaStreamSynchronize(st);
        const double t = now_s();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int i = 0; i < cnt; ++i) {
                auto it = s->reqs.find(batch[i].id);
                if (it == s->reqs.end()) continue;
                Req &r = it->second;
                r.status = rc[i];
                r.t_done = t;
                s->used -= r.bytes;
            }
            for (size_t q = 0; q < idx.size(); ++q) s->reqs[batch[idx[q]].id].st = sst[q];
            admit_locked(s);
        }
        s->cv_done.notify_all();
    }
    cudaStreamDestroy(st);
}

int take_result_locked(nnsort_server *s, uint64_t ticket, nnsort_stats *st, double *lat) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return NNSORT_E_STATE;
    Req &r = it->second;
    if (r.status == NNSORT_PENDING) return NNSORT_PENDING;
    const int rc = r.status;
    if (st) *st = r.st;
    if (lat) *lat = r.t_done - r.t_submit;
    s->reqs.erase(it);
    return rc;
}

}  // namespace

extern "C" {

void nnsort_default_server_opts(nnsort_server_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->hbm_budget = (size_t)120 << 30;
    o->workers = 2;
    o->max_batch = 32;
    o->max_batch_keys = 0;
    nnsort_default_train_opts(&o->train);
    nnsort_default_sort_opts(&o->sort);
}

int nnsort_server_create(const nnsort_server_opts *o, nnsort_server **out) {
    if (!out) return NNSORT_E_INVALID_ARG;
    nnsort_server_opts opts;
    if (o) opts = *o; else nnsort_default_server_opts(&opts);
    if (opts.workers < 1 || opts.workers > 8 || opts.max_batch < 1 || opts.hbm_budget == 0)
        return NNSORT_E_INVALID_ARG;
    if (opts.sort.d_slots || opts.sort.d_fate) return NNSORT_E_INVALID_ARG;
    nnsort_server *s = new (std::nothrow) nnsort_server();
    if (!s) return NNSORT_E_OOM;
    s->o = opts;
    cudaGetDevice(&s->device);
    for (int i = 0; i < opts.workers; ++i) s->workers.emplace_back(worker_main, s);
    *out = s;
    return NNSORT_OK;
}

int nnsort_server_submit(nnsort_server *s, void *h_keys, int32_t *h_payload, uint64_t n, int32_t dtype,
                         uint64_t seed, uint64_t *ticket) {
    if (!s || !h_keys || n == 0 || !ticket || dtype < NNSORT_F32 || dtype > NNSORT_U64)
        return NNSORT_E_INVALID_ARG;
    Req r;
    r.h_keys = h_keys;
    r.h_pay = h_payload;
    r.n = n;
    r.dtype = dtype;
    r.seed = seed;
    r.bytes = request_bytes(s, n, dtype, h_payload != nullptr);
    if (r.bytes > s->o.hbm_budget) return NNSORT_E_BUDGET;
    r.t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return NNSORT_E_STATE;
    r.id = s->next_id++;
    *ticket = r.id;
    s->reqs[r.id] = r;
    s->waiting.push_back(r.id);
    admit_locked(s);
    return NNSORT_OK;
}

int nnsort_server_poll(nnsort_server *s, uint64_t ticket, nnsort_stats *st, double *latency_s) {
    if (!s) return NNSORT_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    return take_result_locked(s, ticket, st, latency_s);
}

int nnsort_server_wait(nnsort_server *s, uint64_t ticket, nnsort_stats *st, double *latency_s) {
    if (!s) return NNSORT_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        const int rc = take_result_locked(s, ticket, st, latency_s);
        if (rc != NNSORT_PENDING) return rc;
        s->cv_done.wait(lk);
    }
}

int nnsort_server_destroy(nnsort_server *s) {
    if (!s) return NNSORT_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
    return NNSORT_OK;
}

}  // extern "C"
