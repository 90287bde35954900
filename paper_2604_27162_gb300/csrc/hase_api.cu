// hase_api.cu -- host side of the C ABI declared in include/hase.h: config
// validation, HBM layout, CTA grouping, launches, checkpoint blobs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hase.h"
#include "hase_internal.cuh"
#include "hase_stream_plan.h"

namespace hase {
cudaError_t launch_generate(const EnvRT* env, const uint32_t* thr, uint32_t n_envs, const uint2* keys,
                            uint16_t* pos, uint16_t* start, uint64_t* rows, uint32_t* err, cudaStream_t st);
cudaError_t launch_prestep(const EnvRT* env, uint32_t n_envs, const uint2* keys, const EnvState* est,
                           const uint64_t* rows, uint16_t* pos, cudaStream_t st);
cudaError_t launch_observe(const EnvRT* env, uint32_t n_envs, const uint16_t* pos,
                           const uint64_t* rows, uint64_t* obs, uint8_t* unp, cudaStream_t st);
cudaError_t launch_step(int family, bool stream, const StepParams& p, uint32_t n_groups, uint32_t threads,
                        uint32_t smem, cudaStream_t st);
cudaError_t launch_advance(uint64_t* clock, uint32_t n, cudaStream_t st);
cudaError_t launch_central_init(const EnvRT* env, uint32_t n_envs, const uint16_t* pos, const uint64_t* rows,
                                const uint32_t* coff, uint64_t* central, cudaStream_t st);
cudaError_t launch_state_init(const uint16_t* pos, const EnvState* est, uint32_t agents, uint32_t n_envs,
                              uint16_t* cells, uint32_t* ept, cudaStream_t st);
cudaError_t launch_fog_init(const EnvRT* env, uint32_t n_envs, const uint16_t* pos, const uint64_t* rows,
                            const uint32_t* foff, uint32_t per_agent, uint64_t* fog, uint64_t* state,
                            cudaStream_t st);
cudaError_t launch_digest(const uint64_t* obs, const uint8_t* done, const int32_t* rew, DigestSpan ow, DigestSpan ev,
                          DigestSpan ag, uint32_t ring, uint64_t first, uint32_t n_steps, uint64_t* scratch,
                          uint32_t n_part, const uint32_t* err, uint64_t* out, int64_t* agent_rew, cudaStream_t st);
cudaError_t digest_scratch_address(uint64_t** p, size_t* words);
cudaError_t prepare_step(uint32_t smem);
}  // namespace hase

using namespace hase;

struct hase_handle {
    int device = 0;
    uint32_t n_envs = 0, ring = 1, flags = 0;
    uint64_t seed = 0;
    std::vector<EnvRT> env;
    std::vector<uint32_t> thr;
    std::vector<uint2> keys;  // per env: Philox key words
    uint2* d_keys = nullptr;
    std::vector<Group> groups;
    std::vector<uint32_t> env_list;
    std::vector<uint64_t> agent_off, obs_off, unp_off, central_off;
    uint64_t central_words = 0;
    uint64_t* d_central = nullptr;
    uint32_t* d_coff = nullptr;
    uint16_t* d_cells = nullptr;  // true state rings (HASE_EXPORT_STATE)
    uint32_t* d_ept = nullptr;
    // fog of war (HASE_EXPORT_FOG): ring, per-env offsets, discovery rows
    std::vector<uint64_t> fog_off;
    std::vector<uint32_t> fog_off32;
    uint64_t fog_words = 0;
    uint16_t base_flags = 0;  // group flags from the config: kFog, kFogAgent, kCentral
    uint64_t* d_fog = nullptr;
    uint32_t* d_fog_off = nullptr;
    uint64_t* d_fog_state = nullptr;
    uint64_t agents = 0, obs_words = 0, unp_bytes = 0, rows_words = 0;
    uint32_t smem = 0, threads = 0, kc = 16, emit_warps = 0, steps_per_launch = 0, n_dyn = 1;
    uint32_t smem_budget = kSmemBudget;
    bool waves = false;  // more CTAs than SMs (the batch is grouped one dynamics warp a CTA)
    // launches of one step: the groups of each kernel family (contiguous)
    struct Family {
        int fam;
        uint32_t first, count, smem, n_dyn, emit_warps, threads;
        bool stream;  // the streaming form (stream_kernel) runs this family
    };
    std::vector<Family> fams;
    std::vector<EnvState> est0;  // episode clocks at create / reset
    uint64_t t = 0;
    uint64_t* d_clock = nullptr;  // steps enqueued before the running launch
    uint64_t* d_scratch = nullptr;  // digest partial sums [kDigestBlocks][3]
    cudaStream_t last_stream = nullptr;  // stream of the latest call (pool frees)
    cudaStream_t cap_stream = nullptr;
    std::map<uint32_t, cudaGraphExec_t> graphs;
    // device memory
    EnvRT* d_env = nullptr;
    EnvState* d_est = nullptr;
    uint16_t* d_pos = nullptr;
    uint16_t* d_start = nullptr;
    uint64_t* d_rows = nullptr;
    Group* d_groups = nullptr;
    uint32_t* d_env_list = nullptr;
    uint64_t* d_obs = nullptr;
    int32_t* d_rew = nullptr;
    uint8_t* d_done = nullptr;
    uint8_t* d_act = nullptr;
    uint8_t* d_unp = nullptr;
    uint32_t* d_err = nullptr;
    uint32_t* d_thr = nullptr;
    std::string err;
};

static std::string g_create_err;

static hase_status fail(hase_handle* h, hase_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_err = buf;
    return st;
}

static hase_status cuda_fail(hase_handle* h, cudaError_t e, const char* what) {
    return fail(h, e == cudaErrorMemoryAllocation ? HASE_ENOMEM : HASE_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define HASE_CUDA(h, call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);   \
    } while (0)

static void free_all(hase_handle* h) {
    void* ptrs[] = {h->d_env, h->d_est,  h->d_pos, h->d_start, h->d_rows, h->d_groups,
                    h->d_obs, h->d_rew, h->d_done, h->d_act,  h->d_unp,  h->d_err, h->d_thr, h->d_env_list,
                    h->d_clock, h->d_scratch, h->d_central, h->d_coff, h->d_cells, h->d_ept,
                    h->d_fog, h->d_fog_off, h->d_fog_state, h->d_keys};
    const bool pool = h->flags & HASE_POOL_ALLOC;
    for (void* p : ptrs)
        if (p) {
            if (pool)
                cudaFreeAsync(p, h->last_stream);
            else
                cudaFree(p);
        }
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.second);
    h->graphs.clear();
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
}

static bool emits(const hase_env_desc& d, uint32_t a) {
    const uint32_t team = a < d.n_seekers ? 0u : 1u;
    return (d.obs_teams >> team) & 1u;
}

static uint32_t radius(const hase_env_desc& d, uint32_t a) { return a < d.n_seekers ? d.r_seek : d.r_hide; }

static hase_status validate(const hase_env_desc& d, uint32_t i) {
    if (d.side < 2 || d.side > HASE_MAX_SIDE)
        return fail(nullptr, HASE_EINVAL, "env desc %u: side %u outside 2..%d", i, d.side, HASE_MAX_SIDE);
    if (d.n_agents < 1 || d.n_agents > HASE_MAX_AGENTS || d.n_agents > d.side * d.side)
        return fail(nullptr, HASE_EINVAL, "env desc %u: n_agents %u outside 1..min(%d, side^2)", i,
                    d.n_agents, HASE_MAX_AGENTS);
    if (d.n_seekers > d.n_agents)
        return fail(nullptr, HASE_EINVAL, "env desc %u: n_seekers %u > n_agents %u", i, d.n_seekers,
                    d.n_agents);
    if (d.r_seek > HASE_MAX_RADIUS || d.r_hide > HASE_MAX_RADIUS)
        return fail(nullptr, HASE_EINVAL, "env desc %u: view radius above %d", i, HASE_MAX_RADIUS);
    if (d.cap < 1 || d.cap > 0x7fffffffu)
        return fail(nullptr, HASE_EINVAL, "env desc %u: episode cap outside 1..2^31-1", i);
    if (d.obs_teams > 7u) return fail(nullptr, HASE_EINVAL, "env desc %u: obs_teams must be 0..7", i);
    return HASE_OK;
}

namespace hase {
// The checks hase_create makes of one descriptor (for callers that queue
// descriptors before any handle exists, such as the rollout server).
hase_status validate_desc(const hase_env_desc& d, char* msg, size_t n) {
    const hase_status s = validate(d, 0);
    if (msg && n) snprintf(msg, n, "%s", g_create_err.c_str());
    return s;
}
}  // namespace hase

// CTA grouping.  Envs are ordered by their kernel-relevant shape (row width,
// cell packing, radii, emitting teams, agent and seeker counts) so that every group is
// uniform, then packed in that order.  With few envs (at most 16 per SM) the
// envs are spread evenly over one CTA per SM (persistent, balanced); with
// many envs a group is one dynamics warp (<= 32 agents) and the CTAs run in
// waves.  Per group the obstacle plane comes from per-cell window tables when
// they fit the shared-memory budget.
static uint64_t shape_key(const EnvRT& E) {
    return ((uint64_t)E.rw << 56) | ((uint64_t)E.r_seek << 48) | ((uint64_t)E.r_hide << 40) |
           ((uint64_t)E.obs_teams << 32) | ((uint64_t)cell_shift(E) << 24) | ((uint64_t)E.n_agents << 8) |
           (uint64_t)E.n_seekers;
}

// The streaming form runs families 1-8 unless the handle exports the
// centralized observation or the fog of war (or asks for the chunked form).
static bool streams(const hase_handle* h, int fam) {
    // the emission warps write the steps of up to kStreamRing + one block of
    // items in any order: their output slots must all differ
    const bool can = fam >= 1 && fam <= 8 && !(h->base_flags & (kFog | kCentral)) && h->ring >= kStreamMinOutRing;
    if (!can || (h->flags & HASE_CHUNKED_STEP)) return false;
    // measured: the streaming form wins when CTAs run in waves (65,536 uneven
    // envs: +13 %); with one CTA per SM the chunked form wins (1024 envs x 10
    // agents: +8 %; 1024 envs x 2 agents with the unpacked export, both forms
    // staging it: 8.1e9 against 6.3e9 env-steps/s)
    return (h->flags & HASE_STREAM_STEP) || h->waves;
}

static bool plan_for(const hase_handle* h, const EnvRT* envs, int n, uint16_t flags, GroupPlan& plan) {
    if (n > 0 && streams(h, family_of(envs[0]))) return plan_stream(envs, n, flags, plan);
    return plan_group(envs, n, (int)h->kc, flags, plan);
}

static bool make_groups(hase_handle* h, uint32_t max_envs_cfg, uint32_t n_sm) {
    const uint32_t E = h->n_envs;
    h->env_list.resize(E);
    for (uint32_t e = 0; e < E; ++e) h->env_list[e] = e;
    std::stable_sort(h->env_list.begin(), h->env_list.end(), [&](uint32_t a, uint32_t b) {
        const int fa = family_of(h->env[a]), fb = family_of(h->env[b]);
        if (fa != fb) return fa < fb;
        return shape_key(h->env[a]) < shape_key(h->env[b]);
    });
    uint32_t epc;
    if (max_envs_cfg)
        epc = max_envs_cfg;
    else if (E <= 16u * n_sm)
        epc = (E + n_sm - 1) / n_sm;
    else
        epc = kMaxGroupEnvs;  // bounded by one dynamics warp below
    const bool many = !max_envs_cfg && E > 16u * n_sm;
    h->waves = many;
    h->groups.clear();
    h->fams.clear();
    uint32_t smem_max = 0, dyn_max = 1;
    GroupPlan plan;
    std::vector<EnvRT> genv;
    uint32_t i = 0;
    while (i < E) {
        const uint64_t key = shape_key(h->env[h->env_list[i]]);
        Group g;
        g.list_first = i;
        g.n_envs = 0;
        g.n_slots = 0;
        g.flags = 0;
        g.n_dyn = 1;
        g.pad = 0;
        genv.clear();
        while (i < E && g.n_envs < epc && g.n_envs < (uint32_t)kMaxGroupEnvs) {
            const EnvRT& En = h->env[h->env_list[i]];
            if (shape_key(En) != key) break;
            if (g.n_slots + En.n_agents > (uint32_t)kMaxGroupSlots) break;
            if (many && g.n_slots + En.n_agents > 32u) break;
            genv.push_back(En);
            const uint16_t flags = h->base_flags;
            if (!plan_for(h, genv.data(), (int)genv.size(), flags, plan) || plan.total > h->smem_budget) {
                genv.pop_back();
                break;
            }
            g.n_slots += En.n_agents;
            g.n_envs += 1;
            ++i;
        }
        if (g.n_envs == 0) return false;  // one env alone exceeds the budget
        uint16_t flags = h->base_flags;
        plan_for(h, genv.data(), g.n_envs, flags | kUseTable, plan);
        const int fam0 = family_of(genv[0]);
        if (plan.total <= h->smem_budget) {
            flags |= kUseTable;
        } else if (fam0 >= 9 && fam0 <= 12) {  // one-word line-of-sight families: one table for both radii
            plan_group(genv.data(), g.n_envs, (int)h->kc, flags | kUseTable | kSharedTable, plan);
            if (plan.total <= h->smem_budget) flags |= kUseTable | kSharedTable;
        }
        if (fam0 >= 1 && h->unp_bytes) {  // the one-thread emission stages the unpacked export of consecutive envs
            bool consecutive = true;
            for (uint32_t j = 1; j < g.n_envs; ++j)
                consecutive &= h->env_list[g.list_first + j] == h->env_list[g.list_first] + j;
            if (consecutive && plan_for(h, genv.data(), g.n_envs, flags | kUnpStage, plan) &&
                plan.total <= h->smem_budget)
                flags |= kUnpStage;
        }
        plan_for(h, genv.data(), g.n_envs, flags, plan);
        g.flags = flags;
        g.n_dyn = (uint8_t)plan.n_dyn;
        smem_max = std::max(smem_max, plan.total);
        dyn_max = std::max(dyn_max, plan.n_dyn);
        const int fam = family_of(genv[0]);
        if (h->fams.empty() || h->fams.back().fam != fam)
            h->fams.push_back({fam, (uint32_t)h->groups.size(), 0u, 0u, 1u, 0u, 0u, streams(h, fam)});
        auto& F = h->fams.back();
        F.count += 1;
        F.smem = std::max(F.smem, plan.total);
        F.n_dyn = std::max(F.n_dyn, plan.n_dyn);
        h->groups.push_back(g);
    }
    h->smem = smem_max;
    h->n_dyn = dyn_max;
    return true;
}

extern "C" {

const char* hase_last_error(const hase_handle* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

hase_status hase_create(const hase_config* cfg, void* stream, hase_handle** out) {
    if (!out) return fail(nullptr, HASE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, HASE_EINVAL, "cfg is NULL");
    if (cfg->n_envs < 1) return fail(nullptr, HASE_EINVAL, "n_envs must be >= 1");
    if (!cfg->envs) return fail(nullptr, HASE_EINVAL, "envs is NULL");
    if (cfg->n_desc != 1 && cfg->n_desc != cfg->n_envs)
        return fail(nullptr, HASE_EINVAL, "n_desc must be 1 or n_envs");
    if (cfg->ring_steps < 1) return fail(nullptr, HASE_EINVAL, "ring_steps must be >= 1");
    if (!cfg->env_ids && (uint64_t)cfg->env_id_base + cfg->n_envs > 0x100000000ull)
        return fail(nullptr, HASE_EINVAL, "env ids exceed 32 bits");
    if (cfg->flags & ~(HASE_EXPORT_ACTIONS | HASE_EXPORT_UNPACKED | HASE_ASYNC_CREATE | HASE_POOL_ALLOC |
                       HASE_DESYNC_START | HASE_EXPORT_CENTRAL | HASE_EXPORT_STATE | HASE_SKIP_OBS |
                       HASE_EXPORT_FOG | HASE_FOG_PER_AGENT | HASE_CHUNKED_STEP | HASE_STREAM_STEP))
        return fail(nullptr, HASE_EINVAL, "unknown flags 0x%x", cfg->flags);
    if ((cfg->flags & HASE_SKIP_OBS) && (cfg->flags & HASE_EXPORT_UNPACKED))
        return fail(nullptr, HASE_EINVAL, "HASE_EXPORT_UNPACKED needs the decentralized observation");
    if ((cfg->flags & HASE_CHUNKED_STEP) && (cfg->flags & HASE_STREAM_STEP))
        return fail(nullptr, HASE_EINVAL, "HASE_CHUNKED_STEP and HASE_STREAM_STEP exclude each other");
    if ((cfg->flags & HASE_FOG_PER_AGENT) && !(cfg->flags & HASE_EXPORT_FOG))
        return fail(nullptr, HASE_EINVAL, "HASE_FOG_PER_AGENT needs HASE_EXPORT_FOG");
    if (cfg->chunk_steps != 0 && (cfg->chunk_steps < 1 || cfg->chunk_steps > (uint32_t)kMaxChunk))
        return fail(nullptr, HASE_EINVAL, "chunk_steps outside 1..%d", kMaxChunk);
    if (cfg->emit_warps > 12) return fail(nullptr, HASE_EINVAL, "emit_warps outside 1..12");
    if (cfg->max_group_envs > (uint32_t)kMaxGroupEnvs)
        return fail(nullptr, HASE_EINVAL, "max_group_envs outside 1..%d", kMaxGroupEnvs);
    if (cfg->smem_cap != 0 && (cfg->smem_cap < 16384u || cfg->smem_cap > kSmemBudget))
        return fail(nullptr, HASE_EINVAL, "smem_cap outside 16384..%u", kSmemBudget);
    for (uint32_t i = 0; i < cfg->n_desc; ++i) {
        hase_status s = validate(cfg->envs[i], i);
        if (s != HASE_OK) return s;
    }

    hase_handle* h = new hase_handle();
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    h->n_envs = cfg->n_envs;
    h->ring = cfg->ring_steps;
    h->flags = cfg->flags;
    h->seed = cfg->seed;
    h->kc = cfg->chunk_steps ? cfg->chunk_steps : 64;
    // steps of one chunk are written concurrently: they must own distinct
    // ring slots, so a chunk never spans more steps than the ring holds
    h->kc = std::min(h->kc, h->ring);
    h->steps_per_launch = cfg->steps_per_launch;

    h->env.resize(h->n_envs);
    h->thr.resize(h->n_envs);
    h->keys.resize(h->n_envs);
    h->agent_off.assign(h->n_envs + 1, 0);
    h->obs_off.assign(h->n_envs + 1, 0);
    h->unp_off.assign(h->n_envs + 1, 0);
    uint64_t rows = 0;
    for (uint32_t e = 0; e < h->n_envs; ++e) {
        const hase_env_desc& d = cfg->envs[cfg->n_desc == 1 ? 0 : e];
        uint32_t wmax = 0, n_obs = 0;
        uint64_t unp = 0;
        const bool skip_obs = (cfg->flags & HASE_SKIP_OBS) != 0u;
        for (uint32_t a = 0; a < d.n_agents; ++a) {
            if (skip_obs || !emits(d, a)) continue;
            const uint32_t D = 2 * radius(d, a) + 1;
            wmax = std::max(wmax, (D * D + 63) / 64);
            n_obs += 1;
            unp += 3ull * D * D;
        }
        EnvRT E;
        E.side = (uint8_t)d.side;
        E.n_agents = (uint8_t)d.n_agents;
        E.n_seekers = (uint8_t)d.n_seekers;
        E.r_seek = (uint8_t)d.r_seek;
        E.r_hide = (uint8_t)d.r_hide;
        E.obs_teams = (uint8_t)(d.obs_teams | (skip_obs ? kObsNoDec : 0u));
        E.wpp = (uint8_t)wmax;
        E.rw = (uint8_t)((d.side + 2 * kPad <= 64) ? 1 : 2);
        E.cap = d.cap;
        E.agent_off = (uint32_t)h->agent_off[e];
        E.obs_off = (uint32_t)h->obs_off[e];
        E.unp_off = (uint32_t)h->unp_off[e];
        E.rows_off = (uint32_t)rows;
        E.env_id = cfg->env_ids ? cfg->env_ids[e] : cfg->env_id_base + e;
        h->env[e] = E;
        h->thr[e] = d.density_thr;
        const uint64_t sd = cfg->env_seeds ? cfg->env_seeds[e] : cfg->seed;
        h->keys[e] = make_uint2((uint32_t)(sd & 0xffffffffu), (uint32_t)(sd >> 32));
        h->agent_off[e + 1] = h->agent_off[e] + d.n_agents;
        h->obs_off[e + 1] = h->obs_off[e] + (uint64_t)n_obs * 3 * wmax;
        h->unp_off[e + 1] = h->unp_off[e] + unp;
        rows += (uint64_t)(d.side + 2 * kPad) * E.rw;
    }
    h->agents = h->agent_off[h->n_envs];
    h->obs_words = h->obs_off[h->n_envs];
    h->unp_bytes = (h->flags & HASE_EXPORT_UNPACKED) ? h->unp_off[h->n_envs] : 0;
    h->rows_words = rows;
    // centralized observation: four planes of `side` one-word rows per env
    h->central_off.assign(h->n_envs + 1, 0);
    for (uint32_t e = 0; e < h->n_envs; ++e) h->central_off[e + 1] = h->central_off[e] + 4ull * h->env[e].side;
    h->central_words = (h->flags & HASE_EXPORT_CENTRAL) ? h->central_off[h->n_envs] : 0;
    // fog of war: per env [units][2][side] words (offsets all 0 without it)
    h->fog_off.assign(h->n_envs + 1, 0);
    if (h->flags & HASE_EXPORT_FOG) {
        const bool per_agent = (h->flags & HASE_FOG_PER_AGENT) != 0u;
        h->base_flags = (uint16_t)(kFog | (per_agent ? kFogAgent : 0u));
        for (uint32_t e = 0; e < h->n_envs; ++e)
            h->fog_off[e + 1] = h->fog_off[e] + 2ull * fog_units(h->env[e], per_agent) * h->env[e].side;
        h->fog_words = h->fog_off[h->n_envs];
        h->fog_off32.assign(h->fog_off.begin(), h->fog_off.end() - 1);
    }
    if (h->flags & HASE_EXPORT_CENTRAL) h->base_flags |= kCentral;  // base group flags
    if (h->obs_words > 0xffffffffull || h->agents > 0xffffffffull || h->unp_bytes > 0xffffffffull ||
        h->central_words > 0xffffffffull || h->fog_words > 0xffffffffull) {
        delete h;
        return fail(nullptr, HASE_EINVAL, "per-step output slice exceeds 2^32 entries");
    }
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device);
    if (n_sm <= 0) n_sm = 1;
    if (cfg->smem_cap) h->smem_budget = cfg->smem_cap;
    if (!make_groups(h, cfg->max_group_envs, (uint32_t)n_sm)) {
        delete h;
        return fail(nullptr, HASE_EINVAL, "smem_cap %u is too small for one env of this batch", cfg->smem_cap);
    }
    // emission warps per family.  Persistent regime (one CTA per SM): nine
    // for the one-thread families (3 + 9 warps keep the 384-thread, 168
    // register kernel), twelve for the general one; CTAs in waves: six.  The
    // one-thread families run at most 12 warps a CTA in all.
    const bool persistent = h->groups.size() <= (size_t)n_sm;
    h->emit_warps = cfg->emit_warps;
    h->threads = 0;
    for (auto& F : h->fams) {
        uint32_t M = cfg->emit_warps ? cfg->emit_warps : (!persistent ? 6u : (F.fam ? 9u : 12u));
        if (F.fam) M = std::min(M, 12u - F.n_dyn);
        if (F.stream) M = std::max(1u, std::min(M, 11u - F.n_dyn));  // one more warp draws the actions
        F.emit_warps = M;
        F.threads = 32 * (F.n_dyn + M + (F.stream ? 1u : 0u));
        h->threads = std::max(h->threads, F.threads);
    }
    if (!h->emit_warps && !h->fams.empty()) h->emit_warps = h->fams[0].emit_warps;

    h->last_stream = st;
    if (h->flags & HASE_POOL_ALLOC) {
        // keep freed pool memory cached for the next handles (once per device;
        // handles may be created from several threads)
        static std::mutex pool_mu;
        static bool pool_ready[64] = {false};
        std::lock_guard<std::mutex> lock(pool_mu);
        if (h->device >= 0 && h->device < 64 && !pool_ready[h->device]) {
            cudaMemPool_t mp;
            if (cudaDeviceGetDefaultMemPool(&mp, h->device) == cudaSuccess) {
                uint64_t thr = ~0ull;
                cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
            }
            pool_ready[h->device] = true;
        }
    }
    auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
        if (h->flags & HASE_POOL_ALLOC) return cudaMallocAsync(p, bytes ? bytes : 16, st);
        return cudaMalloc(p, bytes ? bytes : 16);
    };
    const uint64_t R = h->ring;
    cudaError_t ce = cudaSuccess;
#define HASE_ALLOC(ptr, bytes)                                      \
    if (ce == cudaSuccess) ce = alloc((void**)&(ptr), (bytes));
    HASE_ALLOC(h->d_env, sizeof(EnvRT) * h->n_envs);
    HASE_ALLOC(h->d_est, sizeof(EnvState) * h->n_envs);
    HASE_ALLOC(h->d_pos, 2 * h->agents);
    HASE_ALLOC(h->d_start, 2 * h->agents);
    HASE_ALLOC(h->d_rows, 8 * h->rows_words);
    HASE_ALLOC(h->d_groups, sizeof(Group) * h->groups.size());
    HASE_ALLOC(h->d_env_list, 4 * h->n_envs);
    HASE_ALLOC(h->d_obs, 8 * R * h->obs_words);
    HASE_ALLOC(h->d_rew, 4 * R * h->agents);
    HASE_ALLOC(h->d_done, R * h->n_envs);
    if (h->flags & HASE_EXPORT_ACTIONS) HASE_ALLOC(h->d_act, R * h->agents);
    if (h->flags & HASE_EXPORT_UNPACKED) HASE_ALLOC(h->d_unp, R * h->unp_bytes);
    if (h->flags & HASE_EXPORT_CENTRAL) {
        HASE_ALLOC(h->d_central, 8 * R * h->central_words);
        HASE_ALLOC(h->d_coff, 4 * h->n_envs);
    }
    if (h->flags & HASE_EXPORT_STATE) {
        HASE_ALLOC(h->d_cells, 2 * R * h->agents);
        HASE_ALLOC(h->d_ept, 4 * R * h->n_envs);
    }
    if (h->flags & HASE_EXPORT_FOG) {
        HASE_ALLOC(h->d_fog, 8 * R * h->fog_words);
        HASE_ALLOC(h->d_fog_off, 4 * h->n_envs);
        HASE_ALLOC(h->d_fog_state, 4 * h->fog_words);  // half the words of a slot
    }
    HASE_ALLOC(h->d_err, 4);
    HASE_ALLOC(h->d_thr, 4 * h->n_envs);
    HASE_ALLOC(h->d_keys, sizeof(uint2) * h->n_envs);
    HASE_ALLOC(h->d_clock, 8);
    HASE_ALLOC(h->d_scratch, 8 * 3 * kDigestBlocks);
#undef HASE_ALLOC
    if (ce != cudaSuccess) {
        hase_status s = cuda_fail(nullptr, ce, "cudaMalloc");
        free_all(h);
        delete h;
        return s;
    }
    auto finish = [&](cudaError_t e, const char* what) -> hase_status {
        if (e == cudaSuccess) return HASE_OK;
        hase_status s = cuda_fail(nullptr, e, what);
        free_all(h);
        delete h;
        return s;
    };
    hase_status s;
    if ((s = finish(cudaMemcpyAsync(h->d_env, h->env.data(), sizeof(EnvRT) * h->n_envs,
                                    cudaMemcpyHostToDevice, st), "copy env")) != HASE_OK) return s;
    if ((s = finish(cudaMemcpyAsync(h->d_thr, h->thr.data(), 4 * h->n_envs, cudaMemcpyHostToDevice, st),
                    "copy thresholds")) != HASE_OK) return s;
    if ((s = finish(cudaMemcpyAsync(h->d_keys, h->keys.data(), sizeof(uint2) * h->n_envs, cudaMemcpyHostToDevice,
                                    st),
                    "copy keys")) != HASE_OK)
        return s;
    if ((s = finish(cudaMemcpyAsync(h->d_env_list, h->env_list.data(), 4 * h->n_envs, cudaMemcpyHostToDevice, st),
                    "copy env list")) != HASE_OK) return s;
    if ((s = finish(cudaMemcpyAsync(h->d_groups, h->groups.data(), sizeof(Group) * h->groups.size(),
                                    cudaMemcpyHostToDevice, st), "copy groups")) != HASE_OK) return s;
    // episode clocks: 0, or the desynchronised start offsets
    h->est0.assign(h->n_envs, EnvState{0u, 0u});
    if (h->flags & HASE_DESYNC_START) {
        for (uint32_t e = 0; e < h->n_envs; ++e) {
            uint32_t c0 = 0u, c1 = 0u, c2 = h->env[e].env_id, c3 = 3u;
            philox4x32_10(c0, c1, c2, c3, h->keys[e].x, h->keys[e].y);
            h->est0[e].ep_t = (uint32_t)(((uint64_t)c0 * h->env[e].cap) >> 32);
        }
    }
    if ((s = finish(cudaMemcpyAsync(h->d_est, h->est0.data(), sizeof(EnvState) * h->n_envs,
                                    cudaMemcpyHostToDevice, st), "copy clocks")) != HASE_OK)
        return s;
    if ((s = finish(cudaMemsetAsync(h->d_err, 0, 4, st), "memset")) != HASE_OK) return s;
    if ((s = finish(cudaMemsetAsync(h->d_clock, 0, 8, st), "memset")) != HASE_OK) return s;
    if ((s = finish(prepare_step(h->smem), "shared memory opt-in")) != HASE_OK) return s;
    if ((s = finish(cudaMemsetAsync(h->d_obs, 0, 8 * R * h->obs_words, st), "memset")) != HASE_OK) return s;
    if ((s = finish(cudaMemsetAsync(h->d_rew, 0, 4 * R * h->agents, st), "memset")) != HASE_OK) return s;
    if ((s = finish(cudaMemsetAsync(h->d_done, 0, R * h->n_envs, st), "memset")) != HASE_OK) return s;
    if (h->d_act && (s = finish(cudaMemsetAsync(h->d_act, 0, R * h->agents, st), "memset")) != HASE_OK)
        return s;
    if (h->d_unp && (s = finish(cudaMemsetAsync(h->d_unp, 0, R * h->unp_bytes, st), "memset")) != HASE_OK)
        return s;
    if (h->d_cells && (s = finish(cudaMemsetAsync(h->d_cells, 0, 2 * R * h->agents, st), "memset")) != HASE_OK)
        return s;
    if (h->d_ept && (s = finish(cudaMemsetAsync(h->d_ept, 0, 4 * R * h->n_envs, st), "memset")) != HASE_OK)
        return s;
    if (h->d_fog) {
        if ((s = finish(cudaMemsetAsync(h->d_fog, 0, 8 * R * h->fog_words, st), "memset")) != HASE_OK) return s;
        if ((s = finish(cudaMemcpyAsync(h->d_fog_off, h->fog_off32.data(), 4 * h->n_envs, cudaMemcpyHostToDevice,
                                        st),
                        "copy fog offsets")) != HASE_OK)
            return s;
    }
    if ((s = finish(launch_generate(h->d_env, h->d_thr, h->n_envs, h->d_keys, h->d_pos, h->d_start, h->d_rows,
                                    h->d_err, st), "generate")) != HASE_OK)
        return s;
    if ((h->flags & HASE_DESYNC_START) &&
        (s = finish(launch_prestep(h->d_env, h->n_envs, h->d_keys, h->d_est, h->d_rows, h->d_pos, st),
                    "desynchronised start")) != HASE_OK)
        return s;
    const uint64_t last = R - 1;
    if ((s = finish(launch_observe(h->d_env, h->n_envs, h->d_pos, h->d_rows, h->d_obs + last * h->obs_words,
                                   h->d_unp ? h->d_unp + last * h->unp_bytes : nullptr, st),
                    "observe")) != HASE_OK)
        return s;
    if (h->d_cells && (s = finish(launch_state_init(h->d_pos, h->d_est, (uint32_t)h->agents, h->n_envs,
                                                    h->d_cells + last * h->agents, h->d_ept + last * h->n_envs,
                                                    st),
                                  "true state")) != HASE_OK)
        return s;
    if (h->d_fog && (s = finish(launch_fog_init(h->d_env, h->n_envs, h->d_pos, h->d_rows, h->d_fog_off,
                                                (h->flags & HASE_FOG_PER_AGENT) ? 1u : 0u,
                                                h->d_fog + last * h->fog_words, h->d_fog_state, st),
                                "fog of war")) != HASE_OK)
        return s;
    if (h->d_central) {
        std::vector<uint32_t> coff(h->n_envs);
        for (uint32_t e = 0; e < h->n_envs; ++e) coff[e] = (uint32_t)h->central_off[e];
        if ((s = finish(cudaMemsetAsync(h->d_central, 0, 8 * R * h->central_words, st), "memset")) != HASE_OK)
            return s;
        if ((s = finish(cudaMemcpyAsync(h->d_coff, coff.data(), 4 * h->n_envs, cudaMemcpyHostToDevice, st),
                        "copy central offsets")) != HASE_OK)
            return s;
        if ((s = finish(cudaStreamSynchronize(st), "central offsets")) != HASE_OK) return s;  // coff is local
        if ((s = finish(launch_central_init(h->d_env, h->n_envs, h->d_pos, h->d_rows, h->d_coff,
                                            h->d_central + last * h->central_words, st),
                        "central")) != HASE_OK)
            return s;
    }
    if (h->flags & HASE_ASYNC_CREATE) {  // the generation flag is read by hase_sync / hase_digest
        *out = h;
        return HASE_OK;
    }
    uint32_t herr = 0;
    if ((s = finish(cudaMemcpyAsync(&herr, h->d_err, 4, cudaMemcpyDeviceToHost, st), "copy err")) != HASE_OK)
        return s;
    if ((s = finish(cudaStreamSynchronize(st), "generate sync")) != HASE_OK) return s;
    if (herr) {
        free_all(h);
        delete h;
        return fail(nullptr, HASE_EINVAL, "start-cell draw did not terminate");
    }
    *out = h;
    return HASE_OK;
}

hase_status hase_reset(hase_handle* h, void* stream) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    const uint64_t last = h->ring - 1;
    HASE_CUDA(h, cudaMemcpyAsync(h->d_pos, h->d_start, 2 * h->agents, cudaMemcpyDeviceToDevice, st));
    HASE_CUDA(h, cudaMemcpyAsync(h->d_est, h->est0.data(), sizeof(EnvState) * h->n_envs, cudaMemcpyHostToDevice,
                                 st));
    if (h->flags & HASE_DESYNC_START)
        HASE_CUDA(h, launch_prestep(h->d_env, h->n_envs, h->d_keys, h->d_est, h->d_rows, h->d_pos, st));
    HASE_CUDA(h, cudaMemsetAsync(h->d_rew + last * h->agents, 0, 4 * h->agents, st));
    HASE_CUDA(h, cudaMemsetAsync(h->d_done + last * h->n_envs, 0, h->n_envs, st));
    if (h->d_act) HASE_CUDA(h, cudaMemsetAsync(h->d_act + last * h->agents, 0, h->agents, st));
    HASE_CUDA(h, launch_observe(h->d_env, h->n_envs, h->d_pos, h->d_rows, h->d_obs + last * h->obs_words,
                                h->d_unp ? h->d_unp + last * h->unp_bytes : nullptr, st));
    if (h->d_central)
        HASE_CUDA(h, launch_central_init(h->d_env, h->n_envs, h->d_pos, h->d_rows, h->d_coff,
                                         h->d_central + last * h->central_words, st));
    if (h->d_cells)
        HASE_CUDA(h, launch_state_init(h->d_pos, h->d_est, (uint32_t)h->agents, h->n_envs,
                                       h->d_cells + last * h->agents, h->d_ept + last * h->n_envs, st));
    if (h->d_fog)
        HASE_CUDA(h, launch_fog_init(h->d_env, h->n_envs, h->d_pos, h->d_rows, h->d_fog_off,
                                     (h->flags & HASE_FOG_PER_AGENT) ? 1u : 0u, h->d_fog + last * h->fog_words,
                                     h->d_fog_state, st));
    HASE_CUDA(h, cudaMemsetAsync(h->d_clock, 0, 8, st));
    h->t = 0;
    return HASE_OK;
}

// Enqueue the launches of n_steps steps and the counter advance; the kernels
// read the step count from d_clock, so the same launches replay correctly.
static hase_status enqueue_steps(hase_handle* h, uint32_t n_steps, cudaStream_t st) {
    const uint32_t K = h->steps_per_launch ? h->steps_per_launch : 65536u;
    uint32_t done = 0;
    while (done < n_steps) {
        const uint32_t n = std::min(n_steps - done, K);
        StepParams p;
        p.env = h->d_env;
        p.est = h->d_est;
        p.pos = h->d_pos;
        p.start = h->d_start;
        p.rows = h->d_rows;
        p.groups = h->d_groups;
        p.env_list = h->d_env_list;
        p.obs = h->d_obs;
        p.rew = h->d_rew;
        p.done = h->d_done;
        p.act_out = h->d_act;
        p.unp = h->d_unp;
        p.central = h->d_central;
        p.central_off = h->d_coff;
        p.central_words = h->central_words;
        p.st_cells = h->d_cells;
        p.st_ept = h->d_ept;
        p.fog = h->d_fog;
        p.fog_off = h->d_fog_off;
        p.fog_state = h->d_fog_state;
        p.fog_words = h->fog_words;
        p.obs_words = h->obs_words;
        p.agents = h->agents;
        p.unp_bytes = h->unp_bytes;
        p.clock = h->d_clock;
        p.t0 = done;
        p.n_envs = h->n_envs;
        p.ring = h->ring;
        p.n_steps = n;
        p.kc = h->kc;
        p.key0 = (uint32_t)(h->seed & 0xffffffffu);
        p.key1 = (uint32_t)(h->seed >> 32);
        p.keys = h->d_keys;
        p.err = h->d_err;
        for (const auto& F : h->fams) {
            p.groups = h->d_groups + F.first;
            p.emit_warps = F.emit_warps;
            p.n_dyn = F.n_dyn;
            p.dyn_ids = stream_dyn_ids((int)F.n_dyn, (int)(F.threads / 32), 0);
            HASE_CUDA(h, launch_step(F.fam, F.stream, p, F.count, F.threads, F.smem, st));
        }
        done += n;
    }
    HASE_CUDA(h, launch_advance(h->d_clock, n_steps, st));
    return HASE_OK;
}

static hase_status check_steps(hase_handle* h, uint32_t n_steps) {
    if (((h->t + n_steps) >> 2) > 0xffffffffull)
        return fail(h, HASE_EINVAL, "step counter would exceed 2^34 (Philox counter word)");
    return HASE_OK;
}

hase_status hase_step(hase_handle* h, uint32_t n_steps, void* stream) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    if (n_steps == 0) return HASE_OK;
    hase_status s = check_steps(h, n_steps);
    if (s != HASE_OK) return s;
    h->last_stream = (cudaStream_t)stream;
    s = enqueue_steps(h, n_steps, (cudaStream_t)stream);
    if (s != HASE_OK) return s;
    h->t += n_steps;
    return HASE_OK;
}

hase_status hase_step_graph(hase_handle* h, uint32_t n_steps, void* stream) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    if (n_steps == 0) return HASE_OK;
    hase_status s = check_steps(h, n_steps);
    if (s != HASE_OK) return s;
    auto it = h->graphs.find(n_steps);
    if (it == h->graphs.end()) {
        if (!h->cap_stream) HASE_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        HASE_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        s = enqueue_steps(h, n_steps, h->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
        if (s != HASE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        HASE_CUDA(h, ce);
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        HASE_CUDA(h, ie);
        it = h->graphs.emplace(n_steps, exec).first;
    }
    h->last_stream = (cudaStream_t)stream;
    HASE_CUDA(h, cudaGraphLaunch(it->second, (cudaStream_t)stream));
    h->t += n_steps;
    return HASE_OK;
}

hase_status hase_obs_ptr(hase_handle* h, uint64_t** packed, uint8_t** unpacked) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    if (packed) *packed = h->d_obs;
    if (unpacked) *unpacked = h->d_unp;
    return HASE_OK;
}

hase_status hase_reward_ptr(hase_handle* h, int32_t** reward) {
    if (!h || !reward) return fail(h, HASE_EINVAL, "NULL argument");
    *reward = h->d_rew;
    return HASE_OK;
}

hase_status hase_done_ptr(hase_handle* h, uint8_t** done) {
    if (!h || !done) return fail(h, HASE_EINVAL, "NULL argument");
    *done = h->d_done;
    return HASE_OK;
}

hase_status hase_central_ptr(hase_handle* h, uint64_t** central) {
    if (!h || !central) return fail(h, HASE_EINVAL, "NULL argument");
    *central = h->d_central;
    return HASE_OK;
}

hase_status hase_fog_ptr(hase_handle* h, uint64_t** fog) {
    if (!h || !fog) return fail(h, HASE_EINVAL, "NULL argument");
    *fog = h->d_fog;
    return HASE_OK;
}

hase_status hase_state_ptr(hase_handle* h, uint16_t** cells, uint32_t** ep_t) {
    if (!h || !cells || !ep_t) return fail(h, HASE_EINVAL, "NULL argument");
    *cells = h->d_cells;
    *ep_t = h->d_ept;
    return HASE_OK;
}

hase_status hase_actions_ptr(hase_handle* h, uint8_t** actions) {
    if (!h || !actions) return fail(h, HASE_EINVAL, "NULL argument");
    *actions = h->d_act;
    return HASE_OK;
}

hase_status hase_layout_get(hase_handle* h, hase_layout* out) {
    if (!h || !out) return fail(h, HASE_EINVAL, "NULL argument");
    out->n_envs = h->n_envs;
    out->ring_steps = h->ring;
    out->agents = h->agents;
    out->obs_words = h->obs_words;
    out->unp_bytes = h->unp_bytes;
    out->agent_off = h->agent_off.data();
    out->obs_off = h->obs_off.data();
    out->unp_off = h->unp_off.data();
    out->central_words = h->central_words;
    out->central_off = h->central_off.data();
    out->fog_words = h->fog_words;
    out->fog_off = h->fog_off.data();
    return HASE_OK;
}

hase_status hase_step_count(hase_handle* h, uint64_t* t) {
    if (!h || !t) return fail(h, HASE_EINVAL, "NULL argument");
    *t = h->t;
    return HASE_OK;
}

static const uint64_t kBlobMagic = 0x3130455341484742ull;  // "BGHASE01"

hase_status hase_get_state(hase_handle* h, void* buf, size_t* size, void* stream) {
    if (!h || !size) return fail(h, HASE_EINVAL, "NULL argument");
    const size_t need = 4 * 8 + 2 * h->agents + sizeof(EnvState) * h->n_envs + 4 * h->fog_words;
    if (!buf) {
        *size = need;
        return HASE_OK;
    }
    if (*size < need) return fail(h, HASE_EINVAL, "state buffer too small (%zu < %zu)", *size, need);
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* hdr = (uint64_t*)buf;
    hdr[0] = kBlobMagic;
    hdr[1] = h->n_envs;
    hdr[2] = h->agents;
    hdr[3] = h->t;
    uint8_t* p = (uint8_t*)buf + 32;
    HASE_CUDA(h, cudaMemcpyAsync(p, h->d_pos, 2 * h->agents, cudaMemcpyDeviceToHost, st));
    HASE_CUDA(h, cudaMemcpyAsync(p + 2 * h->agents, h->d_est, sizeof(EnvState) * h->n_envs,
                                 cudaMemcpyDeviceToHost, st));
    if (h->d_fog_state)
        HASE_CUDA(h, cudaMemcpyAsync(p + 2 * h->agents + sizeof(EnvState) * h->n_envs, h->d_fog_state,
                                     4 * h->fog_words, cudaMemcpyDeviceToHost, st));
    HASE_CUDA(h, cudaStreamSynchronize(st));
    *size = need;
    return HASE_OK;
}

hase_status hase_set_state(hase_handle* h, const void* buf, size_t size, void* stream) {
    if (!h || !buf) return fail(h, HASE_EINVAL, "NULL argument");
    const size_t need = 4 * 8 + 2 * h->agents + sizeof(EnvState) * h->n_envs + 4 * h->fog_words;
    if (size != need) return fail(h, HASE_EINVAL, "state blob has %zu bytes, expected %zu", size, need);
    const uint64_t* hdr = (const uint64_t*)buf;
    if (hdr[0] != kBlobMagic || hdr[1] != h->n_envs || hdr[2] != h->agents)
        return fail(h, HASE_EINVAL, "state blob does not match this handle");
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t* p = (const uint8_t*)buf + 32;
    // every position must lie on its env's grid (the kernels index by it)
    for (uint32_t e = 0; e < h->n_envs; ++e) {
        const EnvRT& E = h->env[e];
        for (uint32_t a = 0; a < E.n_agents; ++a) {
            uint16_t q;
            memcpy(&q, p + 2 * ((size_t)E.agent_off + a), 2);
            if (q >= 4096u || px(q) >= E.side || py(q) >= E.side)
                return fail(h, HASE_EINVAL, "state blob: agent %u of env %u off the grid", a, e);
        }
    }
    // discovery rows: no bits outside the env's columns
    const uint8_t* pf = p + 2 * h->agents + sizeof(EnvState) * h->n_envs;
    for (uint32_t e = 0; h->d_fog_state && e < h->n_envs; ++e) {
        const uint32_t S = h->env[e].side;
        const uint64_t smask = S == 64 ? ~0ull : ((1ull << S) - 1ull);
        for (uint64_t i = h->fog_off[e] / 2; i < h->fog_off[e + 1] / 2; ++i) {
            uint64_t v;
            memcpy(&v, pf + 8 * i, 8);
            if (v & ~smask) return fail(h, HASE_EINVAL, "state blob: fog row of env %u outside the grid", e);
        }
    }
    HASE_CUDA(h, cudaMemcpyAsync(h->d_pos, p, 2 * h->agents, cudaMemcpyHostToDevice, st));
    HASE_CUDA(h, cudaMemcpyAsync(h->d_est, p + 2 * h->agents, sizeof(EnvState) * h->n_envs,
                                 cudaMemcpyHostToDevice, st));
    if (h->d_fog_state)
        HASE_CUDA(h, cudaMemcpyAsync(h->d_fog_state, pf, 4 * h->fog_words, cudaMemcpyHostToDevice, st));
    const uint64_t tt = hdr[3];
    HASE_CUDA(h, cudaMemcpyAsync(h->d_clock, &tt, 8, cudaMemcpyHostToDevice, st));
    HASE_CUDA(h, cudaStreamSynchronize(st));
    h->t = tt;
    return HASE_OK;
}

hase_status hase_get_world(hase_handle* h, uint32_t e, uint8_t* grid, int32_t* start_xy) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    if (e >= h->n_envs) return fail(h, HASE_EINVAL, "env %u out of range", e);
    const EnvRT& E = h->env[e];
    const int S = E.side, rw = E.rw;
    if (grid) {
        std::vector<uint64_t> rows((size_t)(S + 2 * kPad) * rw);
        HASE_CUDA(h, cudaMemcpy(rows.data(), h->d_rows + E.rows_off, 8 * rows.size(), cudaMemcpyDeviceToHost));
        for (int y = 0; y < S; ++y)
            for (int x = 0; x < S; ++x) {
                const int b = x + kPad;
                grid[y * S + x] = (uint8_t)((rows[(size_t)(y + kPad) * rw + (b >> 6)] >> (b & 63)) & 1u);
            }
    }
    if (start_xy) {
        std::vector<uint16_t> st(E.n_agents);
        HASE_CUDA(h, cudaMemcpy(st.data(), h->d_start + E.agent_off, 2 * st.size(), cudaMemcpyDeviceToHost));
        for (int a = 0; a < E.n_agents; ++a) {
            start_xy[2 * a] = (int32_t)px(st[a]);
            start_xy[2 * a + 1] = (int32_t)py(st[a]);
        }
    }
    return HASE_OK;
}

hase_status hase_sync(hase_handle* h) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    HASE_CUDA(h, cudaDeviceSynchronize());
    uint32_t herr = 0;
    HASE_CUDA(h, cudaMemcpy(&herr, h->d_err, 4, cudaMemcpyDeviceToHost));
    if (herr & kErrWaitTimeout)
        return fail(h, HASE_ETIMEOUT, "a bounded wait of the step kernel ran out; the outputs are incomplete");
    if (herr & kErrSmemPlan)
        return fail(h, HASE_ECUDA, "a CTA's shared-memory plan exceeded its launch; the outputs are incomplete");
    if (herr) return fail(h, HASE_EINVAL, "start-cell draw did not terminate");
    return HASE_OK;
}

// The digest of steps [first, first + n) of envs [e0, e0 + ne): spans of
// the obs words, done bytes and rewards of one slot, and the partial-sum
// count of its first pass.
struct DigestJob {
    DigestSpan ow, ev, ag;
    uint64_t first;
    uint32_t n_steps, n_part;
};

static hase_status digest_job(hase_handle* h, uint64_t first, uint32_t n_steps, uint32_t e0, uint32_t ne,
                              DigestJob& J) {
    if (n_steps < 1 || first + n_steps > h->t || h->t - first > h->ring)
        return fail(h, HASE_EINVAL, "steps [%llu, %llu) are not all in the ring (steps taken %llu, ring %u)",
                    (unsigned long long)first, (unsigned long long)(first + n_steps), (unsigned long long)h->t,
                    h->ring);
    if (ne < 1 || (uint64_t)e0 + ne > h->n_envs)
        return fail(h, HASE_EINVAL, "env range [%u, %llu) outside 0..%u", e0, (unsigned long long)e0 + ne, h->n_envs);
    J.ow = DigestSpan{h->obs_words, h->obs_off[e0], h->obs_off[e0 + ne] - h->obs_off[e0]};
    J.ev = DigestSpan{h->n_envs, e0, ne};
    J.ag = DigestSpan{h->agents, h->agent_off[e0], h->agent_off[e0 + ne] - h->agent_off[e0]};
    J.first = first;
    J.n_steps = n_steps;
    const uint64_t total = (uint64_t)n_steps * std::max<uint64_t>(J.ow.count, J.ag.count);
    J.n_part = (uint32_t)std::min<uint64_t>(kDigestBlocks, std::max<uint64_t>(1, (total + 255) / 256));
    return HASE_OK;
}

static hase_status run_digest(hase_handle* h, const DigestJob& J, uint64_t* scratch, hase_digest_out* out,
                              int64_t* agent_rew, cudaStream_t st) {
    h->last_stream = st;
    HASE_CUDA(h, launch_digest(h->d_obs, h->d_done, h->d_rew, J.ow, J.ev, J.ag, h->ring, J.first, J.n_steps, scratch,
                               J.n_part, h->d_err, reinterpret_cast<uint64_t*>(out), agent_rew, st));
    return HASE_OK;
}

hase_status hase_digest_noalloc(hase_handle* h, uint32_t n_steps, hase_digest_out* out, int64_t* agent_rew,
                                void* stream) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    if (!out) return fail(h, HASE_EINVAL, "out is NULL");
    if (n_steps < 1 || n_steps > h->ring || n_steps > h->t)
        return fail(h, HASE_EINVAL, "n_steps must be in 1..min(ring_steps, steps taken)");
    int dev = -1;
    HASE_CUDA(h, cudaGetDevice(&dev));
    if (dev != h->device) return fail(h, HASE_EINVAL, "the handle's device (%d) is not current (%d)", h->device, dev);
    if (dev < 0 || dev >= 64) return fail(h, HASE_EINVAL, "device index %d beyond the scratch table", dev);
    // the static scratch's address, looked up once per device with it current
    static std::mutex mu;
    static uint64_t* addr[64] = {nullptr};
    static size_t words[64] = {0};
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!addr[dev]) HASE_CUDA(h, digest_scratch_address(&addr[dev], &words[dev]));
    }
    DigestJob J;
    hase_status s = digest_job(h, h->t - n_steps, n_steps, 0, h->n_envs, J);
    if (s != HASE_OK) return s;
    // the first pass runs at most kDigestBlocks blocks, which stride over the
    // outputs: every digest fits the array (a consistency check)
    if ((uint64_t)3 * J.n_part > words[dev])
        return fail(h, HASE_ECUDA, "internal: %u partial sums exceed the static scratch (%zu)", J.n_part,
                    words[dev] / 3);
    return run_digest(h, J, addr[dev], out, agent_rew, (cudaStream_t)stream);
}

hase_status hase_digest(hase_handle* h, uint32_t n_steps, hase_digest_out* out, int64_t* agent_rew,
                        void* stream) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    if (!out) return fail(h, HASE_EINVAL, "out is NULL");
    if (n_steps < 1 || n_steps > h->ring || n_steps > h->t)
        return fail(h, HASE_EINVAL, "n_steps must be in 1..min(ring_steps, steps taken)");
    DigestJob J;
    hase_status s = digest_job(h, h->t - n_steps, n_steps, 0, h->n_envs, J);
    if (s != HASE_OK) return s;
    return run_digest(h, J, h->d_scratch, out, agent_rew, (cudaStream_t)stream);
}

hase_status hase_digest_range(hase_handle* h, uint64_t first_step, uint32_t n_steps, uint32_t env_first,
                              uint32_t env_count, hase_digest_out* out, int64_t* agent_rew, void* stream) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    if (!out) return fail(h, HASE_EINVAL, "out is NULL");
    DigestJob J;
    hase_status s = digest_job(h, first_step, n_steps, env_first, env_count, J);
    if (s != HASE_OK) return s;
    return run_digest(h, J, h->d_scratch, out, agent_rew, (cudaStream_t)stream);
}

hase_status hase_launch_info(hase_handle* h, uint32_t* ctas, uint32_t* threads, uint32_t* smem,
                             uint32_t* steps_per_launch) {
    if (!h) return fail(nullptr, HASE_EINVAL, "handle is NULL");
    if (ctas) *ctas = (uint32_t)h->groups.size();
    if (threads) *threads = h->threads;
    if (smem) *smem = h->smem;
    if (steps_per_launch) *steps_per_launch = h->steps_per_launch;
    return HASE_OK;
}

void hase_destroy(hase_handle* h) {
    if (!h) return;
    free_all(h);
    delete h;
}

}  // extern "C"
