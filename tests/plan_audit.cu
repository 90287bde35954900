// plan_audit.cu -- host-only audit of the step kernels' shared-memory plans
// (plan_group: chunked form, plan_stream: streaming form).  Built with nvcc
// and run on the CPU by tests/test_plan_audit.py; no GPU call is made.
//
// Input (stdin): one env per line, "side agents seekers r_seek r_hide
// obs_teams".  For every env alone, and for runs of consecutive envs of one
// kernel shape (as a CTA group holds them), every flag combination is
// planned and checked against sizes recomputed here from the env parameters:
// every buffer lies inside the plan's total, no two overlap, the 16-byte
// aligned ones are, and the dynamics warps hold whole envs of at most 32
// agent slots.  Prints "OK <plans>" or the first failure.
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

#include "hase_internal.cuh"

using namespace hase;

namespace {

struct Region {
    const char* name;
    uint64_t off, size;
    bool align16;
};

int failures = 0;

void fail(const char* what, int i0, int n, uint32_t flags, bool stream) {
    if (failures++ < 5)
        std::printf("FAIL %s: group of %d envs from %d, flags 0x%x, %s form\n", what, n, i0, flags,
                    stream ? "streaming" : "chunked");
}

uint32_t radius_words(int r) { return (uint32_t)(((2 * r + 1) * (2 * r + 1) + 63) / 64); }

// team t (0 seekers, 1 hiders) observes (its sightlines count), and also
// writes the decentralized planes unless they are switched off
bool sees(const EnvRT& E, int t) { return (E.obs_teams >> t) & 1u; }
bool emits(const EnvRT& E, int t) { return sees(E, t) && !(E.obs_teams & kObsNoDec); }

// bytes of one env's unpacked export: 3 (2r + 1)^2 per emitting agent
uint32_t unpacked_of(const EnvRT& E) {
    uint32_t u = 0;
    for (int a = 0; a < E.n_agents; ++a) {
        const bool seeker = a < E.n_seekers;
        if (!emits(E, seeker ? 0 : 1)) continue;
        const int r = seeker ? E.r_seek : E.r_hide;
        u += 3u * (2u * r + 1u) * (2u * r + 1u);
    }
    return u;
}

bool check(const std::vector<EnvRT>& envs, int i0, int n, uint32_t flags, bool stream) {
    GroupPlan G;
    std::memset(&G, 0xcd, sizeof(G));
    const EnvRT* e = envs.data() + i0;
    const bool ok = stream ? plan_stream(e, n, (uint16_t)flags, G) : plan_group(e, n, 64, (uint16_t)flags, G);
    // the dynamics warps: whole envs, at most 32 slots each, at most kMaxDyn warps
    uint32_t slots = 0;
    for (int i = 0; i < n; ++i) slots += e[i].n_agents;
    int need = 1;
    uint32_t in_warp = 0;
    for (int i = 0; i < n; ++i) {
        if (in_warp + e[i].n_agents > 32u) {
            ++need;
            in_warp = 0;
        }
        in_warp += e[i].n_agents;
    }
    if (need > kMaxDyn) {
        if (ok) fail("more dynamics warps than kMaxDyn accepted", i0, n, flags, stream);
        return ok;
    }
    if (!ok) {
        fail("a plan that fits the dynamics warps refused", i0, n, flags, stream);
        return false;
    }
    if (G.n_envs != (uint32_t)n || G.n_slots != slots || G.n_dyn != (uint32_t)need)
        fail("env, slot or dynamics-warp count", i0, n, flags, stream);
    uint32_t s = 0;
    for (int i = 0; i < n; ++i) {
        if (G.first_slot[i] != s) fail("first slot", i0, n, flags, stream);
        s += e[i].n_agents;
    }
    for (uint32_t d = 0; d < G.n_dyn; ++d) {
        const uint32_t a = G.dyn_first[d], b = G.dyn_first[d + 1];
        if (b <= a || b - a > 32u) fail("dynamics warp slot range", i0, n, flags, stream);
        bool starts_env = false;
        for (int i = 0; i < n; ++i) starts_env |= G.first_slot[i] == a;
        if (!starts_env) fail("dynamics warp splits an env", i0, n, flags, stream);
    }
    // sizes recomputed from the env parameters
    uint64_t rows = 0, cells = 0, tables = 0, fog_rows = 0;
    const bool use_table = flags & kUseTable, shared_table = flags & kSharedTable;
    for (int i = 0; i < n; ++i) {
        const EnvRT& E = e[i];
        if (G.rows_off[i] != rows) fail("rows offset", i0, n, flags, stream);
        if (G.cell_off[i] != cells) fail("cell offset", i0, n, flags, stream);
        rows += (uint64_t)(E.side + 2 * kPad) * E.rw;
        cells += (uint64_t)(E.side <= 32 ? 32u : 64u) * E.side;
        const bool los = (E.obs_teams & kObsLos) != 0;
        int rmax = 0;
        for (int t = 0; t < 2; ++t)
            if (emits(E, t)) rmax = std::max(rmax, t ? (int)E.r_hide : (int)E.r_seek);
        for (int t = 0; t < 2; ++t) {
            if (!use_table || !emits(E, t)) continue;
            const bool seeker_emits = emits(E, 0);
            if (t == 1 && seeker_emits && (E.r_hide == E.r_seek || (!stream && shared_table))) continue;
            const int r = (!stream && shared_table) ? rmax : (t ? E.r_hide : E.r_seek);
            tables += (uint64_t)E.side * E.side * radius_words(r) * (!stream && los ? 2u : 1u);
        }
        if (!stream && (flags & kFog)) {
            uint32_t units = 1;
            if (flags & kFogAgent) {
                units = 0;
                for (int a = 0; a < E.n_agents; ++a) units += sees(E, a < E.n_seekers ? 0 : 1);
            }
            fog_rows += (uint64_t)units * E.side;
        }
    }
    uint32_t max_side = 0;
    for (int i = 0; i < n; ++i) max_side = std::max<uint32_t>(max_side, e[i].side);
    const uint64_t stage = (flags & kUnpStage) ? ((32ull * unpacked_of(e[0]) + 15ull * 34ull + 15ull) / 16ull * 16ull) : 0;
    std::vector<Region> R;
    if (!stream) {
        const uint64_t act_words = ((64u + 3u) / 4u) * (uint64_t)slots;
        R.push_back({"action buffers", G.act, 3 * act_words * 4, false});
        R.push_back({"trajectory", G.traj, 2ull * 64 * slots * 2, true});
        R.push_back({"rows", G.rows, rows * 8, true});
        R.push_back({"claims", G.claim, cells * 4, false});
        R.push_back({"tables", G.tbl, tables * 8, true});
        R.push_back({"state", G.state, cells, false});
        R.push_back({"fog", G.fog, fog_rows * 8, true});
        R.push_back({"central", G.cen, (flags & kCentral) ? (uint64_t)kMaxEmitWarps * 8 * max_side * 8 : 0, true});
        R.push_back({"staging", G.stage, (uint64_t)kMaxEmitWarps * stage, true});
    } else {
        const uint64_t rec = slots ? stream_rec_words(e[0].n_agents) : 1;
        R.push_back({"trajectory ring", G.traj, (uint64_t)kStreamRing * n * rec * 4, true});
        R.push_back({"pristine records", G.prist, (uint64_t)n * rec * 4, true});
        R.push_back({"rows", G.rows, rows * 8, true});
        R.push_back({"tables", G.tbl, tables * 8, true});
        R.push_back({"state", G.state, cells, false});
        R.push_back({"claims", G.claim, cells * 4, true});
        R.push_back({"action ring", G.act, (uint64_t)kActRing * slots * 4, true});
        R.push_back({"staging", G.stage, (uint64_t)kMaxEmitWarps * stage, true});
    }
    if ((flags & kUnpStage) && G.stage_bytes != stage) fail("staging bytes", i0, n, flags, stream);
    std::sort(R.begin(), R.end(), [](const Region& a, const Region& b) { return a.off < b.off; });
    uint64_t end = 0;
    for (const Region& r : R) {
        if (r.size == 0) continue;
        if (r.off < end) fail(r.name, i0, n, flags, stream);
        if (r.align16 && (r.off & 15u)) fail("alignment", i0, n, flags, stream);
        end = r.off + r.size;
    }
    if (end > G.total || (G.total & 15u)) fail("total", i0, n, flags, stream);
    return true;
}

bool same_shape(const EnvRT& a, const EnvRT& b) {
    return a.n_agents == b.n_agents && a.n_seekers == b.n_seekers && a.r_seek == b.r_seek && a.r_hide == b.r_hide &&
           a.obs_teams == b.obs_teams && a.rw == b.rw && (a.side <= 32) == (b.side <= 32);
}

}  // namespace

int main() {
    std::vector<EnvRT> envs;
    unsigned side, A, ns, rs, rh, teams;
    while (std::scanf("%u %u %u %u %u %u", &side, &A, &ns, &rs, &rh, &teams) == 6) {
        EnvRT E;
        std::memset(&E, 0, sizeof(E));
        E.side = (uint8_t)side;
        E.n_agents = (uint8_t)A;
        E.n_seekers = (uint8_t)ns;
        E.r_seek = (uint8_t)rs;
        E.r_hide = (uint8_t)rh;
        E.obs_teams = (uint8_t)teams;
        int rmax = 0;
        for (int t = 0; t < 2; ++t)
            if (emits(E, t)) rmax = std::max(rmax, (int)(t ? rh : rs));
        E.wpp = (uint8_t)radius_words(rmax);
        E.rw = (uint8_t)(side + 2 * kPad <= 64 ? 1 : 2);
        E.cap = 100;
        envs.push_back(E);
    }
    const uint32_t flag_sets[] = {0u,
                                  kUseTable,
                                  kUseTable | kSharedTable,
                                  kFog,
                                  kFog | kFogAgent,
                                  kUseTable | kFog | kFogAgent,
                                  kCentral,
                                  kUseTable | kCentral,
                                  kUnpStage,
                                  kUseTable | kUnpStage};
    long plans = 0;
    const int N = (int)envs.size();
    for (int i0 = 0; i0 < N; ++i0) {
        int n_max = 1;
        while (i0 + n_max < N && n_max < kMaxGroupEnvs && same_shape(envs[i0], envs[i0 + n_max])) ++n_max;
        const int sizes[] = {1, 2, 3, 4, 8, 16, n_max};
        int last = 0;
        for (int n : sizes) {
            if (n > n_max || n <= last) continue;
            last = n;
            for (uint32_t f : flag_sets) {
                check(envs, i0, n, f, false);
                ++plans;
                const bool streamable = !(f & (kFog | kFogAgent | kCentral | kSharedTable)) &&
                                        !(envs[i0].obs_teams & kObsLos);
                if (streamable) {
                    check(envs, i0, n, f, true);
                    ++plans;
                }
            }
        }
    }
    if (failures) {
        std::printf("FAILED %d of %ld plans\n", failures, plans);
        return 1;
    }
    std::printf("OK %ld\n", plans);
    return 0;
}
