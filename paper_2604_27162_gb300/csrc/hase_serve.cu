// hase_serve.cu -- the rollout server declared in include/hase_serve.h.
//
// Clients submit and poll from any thread under one mutex; a worker thread
// owns the GPU work.  Each round it takes queued requests in arrival order
// (within the in-flight limit), sorts them by horizon, cuts them into batches
// of similar horizons, and admits each batch whose bytes fit the budget as
// one handle whose envs keep their request's seed and env ids (so all of a
// batch's requests share every step launch), on the stream with the fewest
// unfinished requests.  A batch's steps are enqueued
// up to each request's horizon in turn, each followed by that request's range
// digest and a copy of it to pinned memory with an event; requests retire as
// their events fire, and a batch's handle is freed (stream-ordered pool) with
// its last request.  Batches run on a pool of streams and overlap.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hase_serve.h"

namespace hase {
hase_status validate_desc(const hase_env_desc& d, char* msg, size_t n);  // hase_api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

constexpr uint32_t kBatchEnvs = 16384;  // envs of one shared batch at most (default)
constexpr size_t kAdmitRound = 256;     // requests placed per admission round (retirement runs between)

uint32_t emitting_agents(const hase_env_desc& d) {
    return ((d.obs_teams & HASE_OBS_SEEKERS) ? d.n_seekers : 0u) +
           ((d.obs_teams & HASE_OBS_HIDERS) ? d.n_agents - d.n_seekers : 0u);
}

uint32_t words_per_plane(const hase_env_desc& d) {
    uint32_t r = 0;
    if ((d.obs_teams & HASE_OBS_SEEKERS) && d.n_seekers) r = std::max(r, d.r_seek);
    if ((d.obs_teams & HASE_OBS_HIDERS) && d.n_agents > d.n_seekers) r = std::max(r, d.r_hide);
    const uint32_t D = 2 * r + 1;
    return (D * D + 63) / 64;
}

struct Entry {
    hase_request r;
    hase_request_result res;
    bool done = false;
};

struct Pending {  // one request of a batch, waiting for its digest copy
    uint64_t id;
    cudaEvent_t ev;
    uint32_t slot;
};

struct Batch {
    hase_handle* h = nullptr;
    std::vector<Pending> wait;
    uint64_t bytes = 0;
    uint32_t stream = 0;  // index into the server's streams
};

}  // namespace

struct hase_server {
    hase_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Entry> reqs;
    uint64_t next_id = 1;
    size_t admitting = 0;  // requests the worker took off the queue and has not placed yet
    bool stopping = false;
    hase_status dev_status = HASE_OK;
    hase_serve_stats stats{};
    Clock::time_point t0;
    std::thread worker;
    // worker-owned (created by hase_server_create)
    std::vector<cudaStream_t> streams;
    std::vector<uint32_t> stream_load;  // unfinished requests enqueued on each stream
    std::vector<cudaEvent_t> free_events;
    std::vector<uint32_t> free_slots;
    hase_digest_out* d_out = nullptr;
    hase_digest_out* h_out = nullptr;
    std::vector<Batch> active;
    uint64_t used = 0;
    uint32_t inflight = 0, rr = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    // a request finishes: its result becomes pollable (caller holds no lock)
    void finish(uint64_t id, const hase_request_result& r) {
        {
            std::lock_guard<std::mutex> lock(mu);
            Entry& e = reqs[id];
            e.res = r;
            e.done = true;
            stats.requests += 1;
            stats.makespan = std::max(stats.makespan, r.finished);
        }
        cv_done.notify_all();
    }

    bool cuda_ok(cudaError_t e) {
        if (e != cudaSuccess && dev_status == HASE_OK) dev_status = HASE_ECUDA;
        return e == cudaSuccess;
    }

    void admit(std::vector<uint64_t>& cand);
    void retire();
    void run();
};

namespace {

uint64_t request_bytes_steps(const hase_request& r, uint32_t steps) {
    const hase_env_desc& d = r.desc;
    const uint64_t E = r.n_envs, A = d.n_agents;
    const uint64_t per_step = E * (emitting_agents(d) * 3ull * words_per_plane(d) * 8ull + A * 4ull + 1ull);
    const uint64_t rw = (d.side + 8u + 63u) / 64u;
    const uint64_t state = E * (32 + 8 + 4 + 4 + 8 + 4 + 4 * A + (d.side + 8ull) * rw * 8ull + 16);
    const uint64_t fixed = 8 * 3 * 256 + 64 + 16 * 1024;  // scratch, counters, allocation granules
    return (uint64_t)steps * per_step + state + fixed;
}

}  // namespace

// Take the candidates (ids, arrival order) into batches; what does not fit
// the budget goes back to the front of the queue.
void hase_server::admit(std::vector<uint64_t>& cand) {
    std::vector<std::pair<uint64_t, hase_request>> rs;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (uint64_t id : cand) rs.emplace_back(id, reqs[id].r);
    }
    std::stable_sort(rs.begin(), rs.end(),
                     [](const auto& a, const auto& b) { return a.second.steps < b.second.steps; });
    const uint32_t max_envs = cfg.max_batch_envs ? cfg.max_batch_envs : kBatchEnvs;
    const uint32_t max_req = cfg.max_batch ? cfg.max_batch : 256u;
    std::vector<uint64_t> back;
    size_t i = 0;
    bool full = false;
    while (i < rs.size()) {
        if (full || dev_status != HASE_OK) {
            back.push_back(rs[i++].first);
            continue;
        }
        // a batch: horizons within 2x of its first, bounded envs and requests,
        // bytes within the free budget
        size_t j = i;
        uint64_t envs = 0, bytes = 0;
        const uint32_t H0 = rs[i].second.steps;
        // requests of more than max_envs / 32 envs fill the GPU alone: they
        // get a handle of their own
        const bool share = rs[i].second.n_envs <= max_envs / 32u;
        while (j < rs.size() && j - i < (share ? max_req : 1u) && rs[j].second.steps <= 2ull * H0 &&
               rs[j].second.n_envs <= (j == i || share ? std::max(max_envs / 32u, rs[i].second.n_envs) : 0u) &&
               envs + rs[j].second.n_envs <= std::max<uint64_t>(max_envs, rs[i].second.n_envs)) {
            uint64_t b2 = 0;  // bytes of the batch with request j added (ring = its horizon, the longest)
            for (size_t k = i; k <= j; ++k) b2 += request_bytes_steps(rs[k].second, rs[j].second.steps);
            if (used + b2 > cfg.budget_bytes) break;
            bytes = b2;
            envs += rs[j].second.n_envs;
            ++j;
        }
        if (j == i) {  // not even one request fits now: wait for memory
            full = true;
            continue;
        }
        const uint32_t H = rs[j - 1].second.steps;
        std::vector<hase_env_desc> descs;
        std::vector<uint64_t> seeds;
        std::vector<uint32_t> ids;
        std::vector<uint32_t> first(j - i);
        descs.reserve(envs);
        seeds.reserve(envs);
        ids.reserve(envs);
        for (size_t k = i; k < j; ++k) {
            const hase_request& r = rs[k].second;
            first[k - i] = (uint32_t)descs.size();
            for (uint32_t e = 0; e < r.n_envs; ++e) {
                descs.push_back(r.desc);
                seeds.push_back(r.seed);
                ids.push_back(e);
            }
        }
        // the stream with the fewest unfinished requests (a small request
        // does not queue behind a large one)
        uint32_t si = rr++ % (uint32_t)streams.size();
        for (uint32_t q = 0; q < streams.size(); ++q)
            if (stream_load[q] < stream_load[si]) si = q;
        cudaStream_t st = streams[si];
        hase_config c{};
        c.n_envs = (uint32_t)envs;
        c.seed = 0;
        c.envs = descs.data();
        c.n_desc = (uint32_t)envs;
        c.ring_steps = H;
        c.flags = HASE_ASYNC_CREATE | HASE_POOL_ALLOC;
        c.env_seeds = seeds.data();
        c.env_ids = ids.data();
        const double t_adm = now();
        Batch B;
        B.bytes = bytes;
        B.stream = si;
        hase_status cs = hase_create(&c, st, &B.h);
        if (cs != HASE_OK) {  // the requests were validated at submission: device memory or a device failure
            if (cs == HASE_ECUDA) dev_status = HASE_ECUDA;
            for (size_t k = i; k < j; ++k) {
                hase_request_result r{};
                r.submitted = 0;
                r.admitted = r.finished = t_adm;
                r.status = cs;
                r.batch_size = (uint32_t)(j - i);
                finish(rs[k].first, r);
            }
            i = j;
            continue;
        }
        uint32_t t = 0;
        for (size_t k = i; k < j; ++k) {
            const hase_request& r = rs[k].second;
            const uint32_t slot = free_slots.back();
            free_slots.pop_back();
            cudaEvent_t ev = nullptr;
            if (!free_events.empty()) {
                ev = free_events.back();
                free_events.pop_back();
            } else {
                cuda_ok(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            }
            hase_status ss = HASE_OK;
            if (r.steps > t) ss = hase_step(B.h, r.steps - t, st);
            t = std::max(t, r.steps);
            if (ss == HASE_OK)
                ss = hase_digest_range(B.h, 0, r.steps, first[k - i], r.n_envs, d_out + slot, nullptr, st);
            if (ss == HASE_OK && !cuda_ok(cudaMemcpyAsync(h_out + slot, d_out + slot, sizeof(hase_digest_out),
                                                         cudaMemcpyDeviceToHost, st)))
                ss = HASE_ECUDA;
            if (ss == HASE_OK && !cuda_ok(cudaEventRecord(ev, st))) ss = HASE_ECUDA;
            if (ss != HASE_OK && dev_status == HASE_OK) dev_status = HASE_ECUDA;
            {
                std::lock_guard<std::mutex> lock(mu);
                Entry& e = reqs[rs[k].first];
                e.res.admitted = t_adm;
                e.res.bytes = request_bytes_steps(r, H);
                e.res.batch_size = (uint32_t)(j - i);
            }
            B.wait.push_back(Pending{rs[k].first, ev, slot});
        }
        used += bytes;
        inflight += (uint32_t)(j - i);
        stream_load[si] += (uint32_t)(j - i);
        {
            std::lock_guard<std::mutex> lock(mu);
            stats.peak_bytes = std::max(stats.peak_bytes, used);
            stats.peak_inflight = std::max(stats.peak_inflight, inflight);
            stats.batches += 1;
        }
        active.push_back(std::move(B));
        i = j;
    }
    if (!back.empty()) {
        std::lock_guard<std::mutex> lock(mu);
        for (auto it = back.rbegin(); it != back.rend(); ++it) queue.push_front(*it);
    }
}

void hase_server::retire() {
    for (size_t b = 0; b < active.size();) {
        Batch& B = active[b];
        for (size_t k = 0; k < B.wait.size();) {
            Pending& w = B.wait[k];
            const cudaError_t q = cudaEventQuery(w.ev);
            if (q == cudaErrorNotReady) {
                ++k;
                continue;
            }
            hase_request_result r;
            {
                std::lock_guard<std::mutex> lock(mu);
                r = reqs[w.id].res;
            }
            r.finished = now();
            if (!cuda_ok(q)) {
                r.status = HASE_ECUDA;
            } else {
                const hase_digest_out& d = h_out[w.slot];
                r.digest = d.digest;
                r.episodes = d.episodes;
                r.reward_sum = d.reward_sum;
                r.status = d.gen_error ? (d.gen_error & 2u ? HASE_ETIMEOUT : HASE_EINVAL) : HASE_OK;
            }
            finish(w.id, r);
            free_slots.push_back(w.slot);
            free_events.push_back(w.ev);
            --inflight;
            --stream_load[B.stream];
            B.wait[k] = B.wait.back();
            B.wait.pop_back();
        }
        if (B.wait.empty()) {
            hase_destroy(B.h);
            used -= B.bytes;
            active[b] = std::move(active.back());
            active.pop_back();
        } else {
            ++b;
        }
    }
}

void hase_server::run() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<uint64_t> cand;
        bool stop = false;
        {
            std::unique_lock<std::mutex> lock(mu);
            if (queue.empty() && active.empty()) {
                if (stopping) break;
                cv_work.wait_for(lock, std::chrono::milliseconds(5));
            }
            stop = stopping;
            while (!queue.empty() && inflight + cand.size() < cfg.max_inflight && cand.size() < free_slots.size() &&
                   cand.size() < kAdmitRound) {
                cand.push_back(queue.front());
                queue.pop_front();
            }
            admitting = cand.size();
        }
        (void)stop;
        if (!cand.empty()) admit(cand);
        {
            std::lock_guard<std::mutex> lock(mu);
            admitting = 0;
        }
        retire();
        if (dev_status != HASE_OK) break;
        if (cand.empty() && !active.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (dev_status != HASE_OK) {  // a device failure: fail what is left
        cudaDeviceSynchronize();
        for (Batch& B : active) {
            for (Pending& w : B.wait) {
                hase_request_result r{};
                r.finished = now();
                r.status = HASE_ECUDA;
                finish(w.id, r);
                free_events.push_back(w.ev);
            }
            hase_destroy(B.h);
        }
        active.clear();
        std::deque<uint64_t> left;
        {
            std::lock_guard<std::mutex> lock(mu);
            left.swap(queue);
            stopping = true;
        }
        for (uint64_t id : left) {
            hase_request_result r{};
            r.finished = now();
            r.status = HASE_ECUDA;
            finish(id, r);
        }
    }
    cudaDeviceSynchronize();
}

extern "C" {

uint64_t hase_request_bytes(const hase_request* r) { return r ? request_bytes_steps(*r, r->steps) : 0; }

hase_status hase_server_create(const hase_server_config* cfg, hase_server** out) {
    if (!out) return HASE_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->n_streams < 1 || cfg->n_streams > 64 || cfg->max_inflight < 1 || cfg->queue_capacity < 1)
        return HASE_EINVAL;
    hase_server* s = new hase_server();
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    s->streams.assign(cfg->n_streams, nullptr);
    s->stream_load.assign(cfg->n_streams, 0u);
    bool ok = true;
    for (auto& st : s->streams) ok &= cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    ok &= cudaMalloc(&s->d_out, sizeof(hase_digest_out) * cfg->max_inflight) == cudaSuccess;
    ok &= cudaMallocHost(&s->h_out, sizeof(hase_digest_out) * cfg->max_inflight) == cudaSuccess;
    if (!ok) {
        for (auto& st : s->streams)
            if (st) cudaStreamDestroy(st);
        if (s->d_out) cudaFree(s->d_out);
        if (s->h_out) cudaFreeHost(s->h_out);
        delete s;
        return HASE_ECUDA;
    }
    for (uint32_t k = 0; k < cfg->max_inflight; ++k) s->free_slots.push_back(cfg->max_inflight - 1 - k);
    s->t0 = Clock::now();
    s->worker = std::thread([s]() { s->run(); });
    *out = s;
    return HASE_OK;
}

hase_status hase_server_submit(hase_server* s, const hase_request* r, uint64_t* id) {
    if (!s || !r) return HASE_EINVAL;
    char msg[256];
    if (r->n_envs < 1 || r->steps < 1 || hase::validate_desc(r->desc, msg, sizeof msg) != HASE_OK) return HASE_EINVAL;
    const bool too_big = request_bytes_steps(*r, r->steps) > s->cfg.budget_bytes;
    uint64_t k;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) return HASE_ESTATE;
        if (!too_big && s->queue.size() + s->admitting >= s->cfg.queue_capacity) return HASE_EBUSY;
        k = s->next_id++;
        Entry& e = s->reqs[k];
        e.r = *r;
        e.res = hase_request_result{};
        e.res.submitted = s->now();
        if (too_big) {  // can never fit: finished at once
            e.res.admitted = e.res.finished = e.res.submitted;
            e.res.status = HASE_ENOMEM;
            e.res.bytes = request_bytes_steps(*r, r->steps);
            e.done = true;
            s->stats.rejected += 1;
        } else {
            s->queue.push_back(k);
        }
    }
    if (id) *id = k;
    if (too_big)
        s->cv_done.notify_all();
    else
        s->cv_work.notify_one();
    return HASE_OK;
}

hase_status hase_server_poll(hase_server* s, uint64_t id, double timeout_s, hase_request_result* res) {
    if (!s) return HASE_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return HASE_EINVAL;
    if (!it->second.done && timeout_s > 0) {
        const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                              std::chrono::duration<double>(std::min(timeout_s, 1e6)));
        s->cv_done.wait_until(lock, until, [&]() {
            auto j = s->reqs.find(id);
            return j == s->reqs.end() || j->second.done;
        });
        it = s->reqs.find(id);
        if (it == s->reqs.end()) return HASE_EINVAL;  // collected by another thread meanwhile
    }
    if (!it->second.done) return HASE_ETIMEOUT;
    if (res) *res = it->second.res;
    s->reqs.erase(it);
    return HASE_OK;
}

hase_status hase_server_stats(hase_server* s, hase_serve_stats* out) {
    if (!s || !out) return HASE_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    return HASE_OK;
}

hase_status hase_server_shutdown(hase_server* s) {
    if (!s) return HASE_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    return s->dev_status;
}

void hase_server_destroy(hase_server* s) {
    if (!s) return;
    hase_server_shutdown(s);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    for (auto& st : s->streams)
        if (st) cudaStreamDestroy(st);
    if (s->d_out) cudaFree(s->d_out);
    if (s->h_out) cudaFreeHost(s->h_out);
    delete s;
}

hase_status hase_serve(const hase_request* reqs, uint32_t n, const hase_serve_config* cfg, hase_request_result* res,
                       hase_serve_stats* stats) {
    if (!cfg || (!reqs && n) || (!res && n)) return HASE_EINVAL;
    if (cfg->n_streams < 1 || cfg->n_streams > 64 || cfg->max_inflight < 1 || cfg->time_scale < 0)
        return HASE_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        if (reqs[i].n_envs < 1 || reqs[i].steps < 1) return HASE_EINVAL;
        if (i && reqs[i].arrival < reqs[i - 1].arrival) return HASE_EINVAL;
    }
    hase_server_config sc{};
    sc.budget_bytes = cfg->budget_bytes;
    sc.n_streams = cfg->n_streams;
    sc.max_inflight = cfg->max_inflight;
    sc.queue_capacity = n ? n : 1;
    sc.max_batch = cfg->max_batch;
    hase_server* s = nullptr;
    hase_status st = hase_server_create(&sc, &s);
    if (st != HASE_OK) return st;
    std::vector<uint64_t> ids(n, 0);
    for (uint32_t i = 0; i < n; ++i) {
        const double due = reqs[i].arrival * cfg->time_scale;
        const double wait = due - s->now();
        if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
        const hase_status ss = hase_server_submit(s, &reqs[i], &ids[i]);
        if (ss != HASE_OK) {  // validated above except the descriptor
            std::memset(&res[i], 0, sizeof(res[i]));
            res[i].status = ss;
            ids[i] = 0;
        }
    }
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] && hase_server_poll(s, ids[i], 1e6, &res[i]) != HASE_OK) res[i].status = HASE_ECUDA;
    st = hase_server_shutdown(s);
    if (stats) hase_server_stats(s, stats);
    hase_server_destroy(s);
    return st;
}

}  // extern "C"
