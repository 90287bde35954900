// hase_serve.cu -- the rollout server declared in include/hase_serve.h.
//
// One host thread runs an event loop: admit arrived requests in order while
// the budget and the in-flight limit allow (create the request's handle from
// the stream-ordered pool without waiting, enqueue its whole horizon, its
// digest and the copy of the digest to pinned memory, and an event), then
// retire every request whose event has completed (read the digest, destroy
// the handle, give its bytes back).  Requests run on a pool of streams, so
// the kernels of requests in flight overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/hase_serve.h"

namespace {

struct Inflight {
    uint32_t req;
    hase_handle* h;
    cudaEvent_t ev;
    uint32_t slot;
    uint64_t bytes;
};

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

}  // namespace

extern "C" {

uint64_t hase_request_bytes(const hase_request* r) {
    const hase_env_desc& d = r->desc;
    const uint64_t E = r->n_envs, A = d.n_agents;
    const uint64_t per_step = E * (emitting_agents(d) * 3ull * words_per_plane(d) * 8ull + A * 4ull + 1ull);
    const uint64_t rw = (d.side + 8u + 63u) / 64u;
    const uint64_t state = E * (32 + 8 + 4 + 4 + 4 * A + (d.side + 8ull) * rw * 8ull + 16);
    const uint64_t fixed = 8 * 3 * 256 + 64 + 16 * 1024;  // scratch, counters, allocation granules
    return (uint64_t)r->steps * per_step + state + fixed;
}

hase_status hase_serve(const hase_request* reqs, uint32_t n, const hase_serve_config* cfg,
                       hase_request_result* res, hase_serve_stats* stats) {
    if (!cfg || (!reqs && n) || (!res && n)) return HASE_EINVAL;
    if (cfg->n_streams < 1 || cfg->n_streams > 64 || cfg->max_inflight < 1 || cfg->time_scale < 0)
        return HASE_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        if (reqs[i].n_envs < 1 || reqs[i].steps < 1) return HASE_EINVAL;
        if (i && reqs[i].arrival < reqs[i - 1].arrival) return HASE_EINVAL;
    }
    hase_serve_stats st{};
    std::vector<cudaStream_t> streams(cfg->n_streams, nullptr);
    std::vector<cudaEvent_t> free_events;
    hase_digest_out* d_out = nullptr;
    hase_digest_out* h_out = nullptr;
    const uint32_t slots = cfg->max_inflight;
    hase_status status = HASE_OK;
    auto cuda_ok = [&](cudaError_t e) {
        if (e != cudaSuccess && status == HASE_OK) status = HASE_ECUDA;
        return e == cudaSuccess;
    };
    for (auto& s : streams) cuda_ok(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cuda_ok(cudaMalloc(&d_out, sizeof(hase_digest_out) * slots));
    cuda_ok(cudaMallocHost(&h_out, sizeof(hase_digest_out) * slots));
    std::vector<uint32_t> free_slots;
    for (uint32_t s = 0; s < slots; ++s) free_slots.push_back(slots - 1 - s);
    std::vector<Inflight> active;
    const auto t0 = std::chrono::steady_clock::now();
    auto now = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    uint32_t next = 0, finished = 0, rr = 0;
    uint64_t used = 0;
    for (uint32_t i = 0; i < n; ++i) std::memset(&res[i], 0, sizeof(res[i]));

    while (status == HASE_OK && finished < n) {
        bool progress = false;
        // admit in arrival order while the budget and the slots allow
        while (next < n && reqs[next].arrival * cfg->time_scale <= now() && !free_slots.empty()) {
            const hase_request& r = reqs[next];
            hase_request_result& out = res[next];
            const uint64_t bytes = hase_request_bytes(&r);
            if (bytes > cfg->budget_bytes) {  // can never fit
                out.status = HASE_ENOMEM;
                out.admitted = out.finished = now();
                ++st.rejected;
                ++finished;
                ++next;
                progress = true;
                continue;
            }
            if (used + bytes > cfg->budget_bytes) break;  // wait for memory
            cudaStream_t s = streams[rr++ % streams.size()];
            hase_config c{};
            c.n_envs = r.n_envs;
            c.seed = r.seed;
            c.envs = &r.desc;
            c.n_desc = 1;
            c.ring_steps = r.steps;
            c.flags = HASE_ASYNC_CREATE | HASE_POOL_ALLOC;
            out.admitted = now();
            out.bytes = bytes;
            hase_handle* h = nullptr;
            hase_status cs = hase_create(&c, s, &h);
            if (cs != HASE_OK) {
                out.status = cs;
                out.finished = now();
                ++finished;
                ++next;
                progress = true;
                if (cs == HASE_ECUDA) status = HASE_ECUDA;
                continue;
            }
            const uint32_t slot = free_slots.back();
            free_slots.pop_back();
            cudaEvent_t ev = nullptr;
            if (!free_events.empty()) {
                ev = free_events.back();
                free_events.pop_back();
            } else {
                cuda_ok(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            }
            hase_status ss = hase_step(h, r.steps, s);
            if (ss == HASE_OK) ss = hase_digest(h, r.steps, d_out + slot, nullptr, s);
            if (ss == HASE_OK && !cuda_ok(cudaMemcpyAsync(h_out + slot, d_out + slot, sizeof(hase_digest_out),
                                                         cudaMemcpyDeviceToHost, s)))
                ss = HASE_ECUDA;
            if (ss == HASE_OK && !cuda_ok(cudaEventRecord(ev, s))) ss = HASE_ECUDA;
            if (ss != HASE_OK) {
                out.status = ss;
                if (ss == HASE_ECUDA) status = HASE_ECUDA;
                hase_destroy(h);
                free_slots.push_back(slot);
                free_events.push_back(ev);
                out.finished = now();
                ++finished;
                ++next;
                progress = true;
                continue;
            }
            active.push_back(Inflight{next, h, ev, slot, bytes});
            used += bytes;
            st.peak_bytes = std::max(st.peak_bytes, used);
            st.peak_inflight = std::max<uint32_t>(st.peak_inflight, (uint32_t)active.size());
            ++next;
            progress = true;
        }
        // retire completed requests
        for (size_t i = 0; i < active.size();) {
            Inflight& a = active[i];
            const cudaError_t q = cudaEventQuery(a.ev);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            hase_request_result& out = res[a.req];
            out.finished = now();
            if (q != cudaSuccess) {
                cuda_ok(q);
                out.status = HASE_ECUDA;
            } else {
                const hase_digest_out& d = h_out[a.slot];
                out.digest = d.digest;
                out.episodes = d.episodes;
                out.reward_sum = d.reward_sum;
                out.status = d.gen_error ? HASE_EINVAL : HASE_OK;
            }
            hase_destroy(a.h);
            used -= a.bytes;
            free_slots.push_back(a.slot);
            free_events.push_back(a.ev);
            ++finished;
            active[i] = active.back();
            active.pop_back();
            progress = true;
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // a device failure: wait for what is in flight, then release everything
    cudaDeviceSynchronize();
    for (Inflight& a : active) {
        res[a.req].status = HASE_ECUDA;
        hase_destroy(a.h);
        free_events.push_back(a.ev);
    }
    for (uint32_t i = next; i < n; ++i) res[i].status = HASE_ECUDA;
    st.makespan = now();
    for (cudaEvent_t e : free_events) cudaEventDestroy(e);
    for (auto& s : streams)
        if (s) cudaStreamDestroy(s);
    if (d_out) cudaFree(d_out);
    if (h_out) cudaFreeHost(h_out);
    if (stats) *stats = st;
    return status;
}

}  // extern "C"
