// Continuous-batching request server (sampling, Sec. 4.1; scoring, Sec. 4.3;
// single-mutant scans, Sec. 4.4) over resident models.
//
// One worker thread owns every CUDA call of the server.  Its loop:
//   1. retire: requests whose completion event has fired release their
//      stream slot and their share of the scratch budget;
//   2. admit: queued requests are scanned in arrival order and every one
//      whose scratch fits beside the running ones gets a free stream slot;
//      its whole job (stream-ordered scratch allocation, upload, kernels,
//      download, scratch free, completion event) is enqueued on that stream
//      at once, so jobs of different requests overlap on the device;
//   3. sleep until a submission or a short poll interval.
// Submitters and waiters only touch the queue and the completion state
// under the mutex.
#include "bm_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t id = 0;
    bm_request r{};
    size_t need = 0;  // device scratch bytes
    double t_submit = 0.0, t_done = 0.0;
    int status = BM_OK;
    int slot = -1;
    bool done = false;
};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

struct bm_server_s {
    int device = 0;
    size_t budget = 0, used = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<int> free_slots;
    std::vector<bm_model_s *> models;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::vector<Req *> running;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    long long submitted = 0, completed = 0, failed = 0;
    std::vector<double> lat_ms;
    double seqs = 0.0, t_first = -1.0, t_last = 0.0;
    int max_running = 0;
};

namespace {

size_t scratch_bytes(const bm_model_s *m, const bm_request &r)
{
    const size_t L = (size_t)m->L, q = (size_t)m->q;
    switch (r.type) {
    case BM_REQ_SAMPLE: return round256((size_t)r.n * L);
    case BM_REQ_SCORE: return round256((size_t)r.n * L) + round256((size_t)r.n * 4);
    case BM_REQ_SCAN: return round256(L) + round256(L * q * 4);
    default: return 0;
    }
}

// Enqueue the whole job of request r on stream st (worker thread only).
int launch(bm_server_s *s, Req *rq, cudaStream_t st, cudaEvent_t ev)
{
    bm_model_s *m = s->models[rq->r.model];
    const bm_request &r = rq->r;
    const int L = m->L, q = m->q;
    unsigned char *d = nullptr;
    BM_CK(cudaMallocAsync((void **)&d, rq->need, st));
    int rc = BM_OK;
    cudaError_t e = cudaSuccess;
    switch (r.type) {
    case BM_REQ_SAMPLE: {
        bm_chains_s c;  // view of the request's scratch; only the fields the sweeps read
        c.M = r.n;
        c.L = L;
        c.q = q;
        c.device = s->device;
        c.s = d;
        c.seed = r.seed;
        c.sweep = 0;
        rc = bm_launch_chains_init(c.s, r.n, L, q, r.seed, 0, st);
        if (rc == BM_OK) rc = bm_sweep_run(m, &c, r.nsweeps, r.beta, st);
        if (rc == BM_OK) e = cudaMemcpyAsync(r.out, c.s, (size_t)r.n * L, cudaMemcpyDefault, st);
        break;
    }
    case BM_REQ_SCORE: {
        uint8_t *seq = d;
        float *E = reinterpret_cast<float *>(d + round256((size_t)r.n * L));
        e = cudaMemcpyAsync(seq, r.in, (size_t)r.n * L, cudaMemcpyDefault, st);
        if (e == cudaSuccess) rc = bm_gather_prepare(m, st);
        if (e == cudaSuccess && rc == BM_OK) rc = bm_launch_energy(m, seq, r.n, E, m->dflags + 4, st);
        if (rc == BM_OK && e == cudaSuccess) e = cudaMemcpyAsync(r.out, E, (size_t)r.n * 4, cudaMemcpyDefault, st);
        break;
    }
    case BM_REQ_SCAN: {
        uint8_t *wt = d;
        float *dE = reinterpret_cast<float *>(d + round256((size_t)L));
        e = cudaMemcpyAsync(wt, r.in, (size_t)L, cudaMemcpyDefault, st);
        if (e == cudaSuccess) rc = bm_launch_mutant_scan(m->h, m->J, L, q, wt, dE, st);
        if (rc == BM_OK && e == cudaSuccess) e = cudaMemcpyAsync(r.out, dE, (size_t)L * q * 4, cudaMemcpyDefault, st);
        break;
    }
    default: rc = bm_fail(BM_EINVAL, "server: unknown request type %d", r.type);
    }
    if (e != cudaSuccess && rc == BM_OK) rc = bm_cuda_fail(e, "server: copy");
    cudaFreeAsync(d, st);  // stream-ordered: after the job's kernels and copies
    const cudaError_t e2 = cudaEventRecord(ev, st);
    if (e2 != cudaSuccess && rc == BM_OK) rc = bm_cuda_fail(e2, "server: cudaEventRecord");
    return rc;
}

void finish(bm_server_s *s, Req *rq, int status)
{
    rq->status = status;
    rq->t_done = now_s();
    rq->done = true;
    ++s->completed;
    if (status != BM_OK) {
        ++s->failed;
    } else {
        s->lat_ms.push_back((rq->t_done - rq->t_submit) * 1e3);
        const bm_model_s *m = s->models[rq->r.model];
        s->seqs += rq->r.type == BM_REQ_SCAN ? (double)m->L * m->q : (double)rq->r.n;
    }
    s->t_last = std::max(s->t_last, rq->t_done);
}

void worker_main(bm_server_s *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // 1. retire
        for (size_t k = 0; k < s->running.size();) {
            Req *rq = s->running[k];
            const cudaError_t qe = cudaEventQuery(s->events[rq->slot]);
            if (qe == cudaErrorNotReady) {
                ++k;
                continue;
            }
            s->used -= rq->need;
            s->free_slots.push_back(rq->slot);
            finish(s, rq, qe == cudaSuccess ? rq->status : bm_cuda_fail(qe, "server: request failed on the device"));
            s->running.erase(s->running.begin() + (long)k);
            s->cv_done.notify_all();
        }
        // 2. admit in arrival order, skipping requests that do not fit yet
        for (auto it = s->queue.begin(); it != s->queue.end() && !s->free_slots.empty();) {
            Req *rq = *it;
            if (s->used + rq->need > s->budget) {
                ++it;
                continue;
            }
            const int slot = s->free_slots.back();
            s->free_slots.pop_back();
            rq->slot = slot;
            s->used += rq->need;
            it = s->queue.erase(it);
            const int rc = launch(s, rq, s->streams[slot], s->events[slot]);
            rq->status = rc;
            s->running.push_back(rq);  // retired when its event fires (also after a launch error)
            s->max_running = std::max(s->max_running, (int)s->running.size());
        }
        if (s->stop && s->queue.empty() && s->running.empty()) break;
        if (s->running.empty())
            s->cv_work.wait(lk, [s] { return s->stop || !s->queue.empty(); });
        else
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" {

int bm_server_create(size_t budget_bytes, int slots, bm_server *out)
{
    if (!out) return bm_fail(BM_EINVAL, "bm_server_create: out is NULL");
    *out = nullptr;
    if (slots < 1 || slots > 256) return bm_fail(BM_EINVAL, "bm_server_create: slots=%d not in 1..256", slots);
    if (budget_bytes == 0) return bm_fail(BM_EINVAL, "bm_server_create: zero budget");
    bm_server_s *s = new (std::nothrow) bm_server_s();
    if (!s) return bm_fail(BM_ENOMEM, "bm_server_create: host allocation failed");
    s->budget = budget_bytes;
    cudaError_t e = cudaGetDevice(&s->device);
    for (int k = 0; k < slots && e == cudaSuccess; ++k) {
        cudaStream_t st;
        cudaEvent_t ev;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) break;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaStreamDestroy(st);
            break;
        }
        s->streams.push_back(st);
        s->events.push_back(ev);
        s->free_slots.push_back(k);
    }
    if (e != cudaSuccess) {
        for (auto st : s->streams) cudaStreamDestroy(st);
        for (auto ev : s->events) cudaEventDestroy(ev);
        delete s;
        return bm_cuda_fail(e, "bm_server_create: streams");
    }
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        for (auto st : s->streams) cudaStreamDestroy(st);
        for (auto ev : s->events) cudaEventDestroy(ev);
        delete s;
        return bm_fail(BM_ENOMEM, "bm_server_create: cannot start the worker thread");
    }
    *out = s;
    return BM_OK;
}

int bm_server_destroy(bm_server s)
{
    if (!s) return BM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
    for (auto st : s->streams) cudaStreamDestroy(st);
    for (auto ev : s->events) cudaEventDestroy(ev);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return BM_OK;
}

int bm_server_add_model(bm_server s, bm_model m, int *id)
{
    if (!s || !m || !id) return bm_fail(BM_EINVAL, "bm_server_add_model: NULL argument");
    // The lazily built layouts (gather layout, split J, in-block corrections)
    // are brought up to date here, once and synchronously: requests run on
    // different streams, so a layout built lazily by one request could be
    // read by a concurrent one before its build kernel ran.  The tensor-core
    // ones are built for every model a tensor-core form could serve (AUTO's
    // choice depends on each request's chain count).
    cudaStream_t st = nullptr;
    BM_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = bm_gather_prepare(m, st);
    const bool tc = m->engine != BM_ENGINE_SIMT && m->q >= 2;
    if (rc == BM_OK && tc && (bm_gibbs_mma_chains_per_cta(m, 1) > 0 || bm_gibbs_pair_chains_per_cluster(m, 1) > 0)) {
        rc = bm_split_prepare(m, 0, st);
        if (rc == BM_OK) rc = bm_corr_prepare(m, st);
    }
    const cudaError_t e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc != BM_OK) return rc;
    if (e != cudaSuccess) return bm_cuda_fail(e, "bm_server_add_model");
    std::lock_guard<std::mutex> lk(s->mu);
    s->models.push_back(m);
    *id = (int)s->models.size() - 1;
    return BM_OK;
}

int bm_server_submit(bm_server s, const bm_request *r, uint64_t *id)
{
    if (!s || !r || !id) return bm_fail(BM_EINVAL, "bm_server_submit: NULL argument");
    Req *rq = new (std::nothrow) Req();
    if (!rq) return bm_fail(BM_ENOMEM, "bm_server_submit: host allocation failed");
    rq->r = *r;
    std::unique_lock<std::mutex> lk(s->mu);
    int rc = BM_OK;
    if (r->model < 0 || r->model >= (int)s->models.size()) {
        rc = bm_fail(BM_EINVAL, "bm_server_submit: unknown model %d", r->model);
    } else if (r->type != BM_REQ_SAMPLE && r->type != BM_REQ_SCORE && r->type != BM_REQ_SCAN) {
        rc = bm_fail(BM_EINVAL, "bm_server_submit: unknown request type %d", r->type);
    } else if (!r->out || (r->type != BM_REQ_SAMPLE && !r->in)) {
        rc = bm_fail(BM_EINVAL, "bm_server_submit: NULL buffer");
    } else if (r->type != BM_REQ_SCAN && r->n < 1) {
        rc = bm_fail(BM_EINVAL, "bm_server_submit: n=%d < 1", r->n);
    } else if (r->type == BM_REQ_SAMPLE && (r->nsweeps < 0 || !std::isfinite(r->beta))) {
        rc = bm_fail(BM_EINVAL, "bm_server_submit: bad nsweeps or beta");
    } else {
        rq->need = scratch_bytes(s->models[r->model], *r);
        if (rq->need > s->budget)
            rc = bm_fail(BM_ENOMEM, "bm_server_submit: request needs %zu bytes, budget %zu", rq->need, s->budget);
    }
    if (rc != BM_OK) {
        delete rq;
        return rc;
    }
    rq->id = s->next_id++;
    rq->t_submit = now_s();
    if (s->t_first < 0) s->t_first = rq->t_submit;
    ++s->submitted;
    s->reqs[rq->id] = rq;
    s->queue.push_back(rq);
    *id = rq->id;
    lk.unlock();
    s->cv_work.notify_one();
    return BM_OK;
}

int bm_server_wait(bm_server s, uint64_t id, double timeout_ms, int *status, double *latency_ms)
{
    if (!s) return bm_fail(BM_EINVAL, "bm_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return bm_fail(BM_EINVAL, "bm_server_wait: unknown request %llu", (unsigned long long)id);
    Req *rq = it->second;
    auto done = [rq] { return rq->done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), done)) {
        return bm_fail(BM_ETIMEOUT, "bm_server_wait: request %llu not complete", (unsigned long long)id);
    }
    if (status) *status = rq->status;
    if (latency_ms) *latency_ms = (rq->t_done - rq->t_submit) * 1e3;
    s->reqs.erase(it);
    delete rq;
    return BM_OK;
}

int bm_server_stats_get(bm_server s, bm_server_stats *out, int reset)
{
    if (!s || !out) return bm_fail(BM_EINVAL, "bm_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    bm_server_stats r{};
    r.submitted = s->submitted;
    r.completed = s->completed;
    r.failed = s->failed;
    r.sequences = s->seqs;
    r.max_running = s->max_running;
    r.span_s = s->t_first >= 0 ? s->t_last - s->t_first : 0.0;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&v](double p) {  // nearest rank
            const size_t k = (size_t)std::ceil(p * (double)v.size());
            return v[std::min(v.size(), std::max<size_t>(k, 1)) - 1];
        };
        r.p50_ms = pct(0.50);
        r.p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        r.mean_ms = sum / (double)v.size();
    }
    *out = r;
    if (reset) {
        s->submitted = s->completed = s->failed = 0;
        s->lat_ms.clear();
        s->seqs = 0.0;
        s->t_first = -1.0;
        s->t_last = 0.0;
        s->max_running = (int)s->running.size();
    }
    return BM_OK;
}

}  // extern "C"
