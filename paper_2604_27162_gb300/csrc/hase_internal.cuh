// hase_internal.cuh -- data layout shared by the host API and the kernels of
// the batched hide-and-seek environment step (Hide-And-Seek-Engine, arxiv
// 2604.27162).
//
// HBM layout of one handle (device arrays, structure of arrays):
//   EnvRT    env[E]        per-env constants (32 B each)
//   EnvState est[E]        episode counters
//   uint16   pos[sumA]     current cell of every agent, packed x | y << 6
//   uint16   start[sumA]   pristine start cells (Sec. 4.2 template)
//   uint64   rows[...]     per env (S + 8) padded obstacle rows of rw words:
//                          bit x + 4 of row y + 4 is cell (x, y); every bit
//                          outside the grid is 1, so windows that leave the
//                          grid read obstacles without bounds checks
//   Group    groups[G]     the envs one CTA steps together (through a
//   uint32   env_list[E]   permutation of the env indices)
//   outputs                ring of ring_steps slots (see hase.h)
#pragma once

#include <stdint.h>

namespace hase {

constexpr int kPad = 4;               // padding cells around the grid (max radius)
constexpr int kMaxAgents = 32;        // agents per env (one dynamics lane each, whole envs per warp)
constexpr int kFastAgents = 16;       // agents per env of the one-thread emission families 1-16
constexpr int kMaxGroupEnvs = 64;     // envs per CTA
constexpr int kMaxGroupSlots = 128;   // agents per CTA (four dynamics warps)
constexpr int kMaxDyn = 4;            // dynamics warps per CTA
constexpr int kMaxChunk = 64;         // steps per on-chip chunk
constexpr int kMaxEmitWarps = 12;     // emission warps per CTA
constexpr int kObsHiders = 2;         // obs_teams value: only hiders emit
constexpr uint32_t kObsLos = 4;       // obs_teams bit: line of sight masks the windows
constexpr uint32_t kObsNoDec = 8;     // obs_teams bit: no decentralized planes are written
constexpr uint32_t kDoneBit = 0x8000u;
constexpr uint32_t kOccBit = 0x80u;   // occupancy bit of the neighbour map
constexpr uint32_t kSmemBudget = 216 * 1024;  // dynamic shared memory per CTA
constexpr uint32_t kDigestBlocks = 256;        // partial sums of the digest's first pass

__host__ __device__ inline uint32_t pack_xy(uint32_t x, uint32_t y) { return x | (y << 6); }
__host__ __device__ inline uint32_t px(uint32_t p) { return p & 63u; }
__host__ __device__ inline uint32_t py(uint32_t p) { return (p >> 6) & 63u; }

struct EnvRT {
    uint8_t side, n_agents, n_seekers, r_seek;
    uint8_t r_hide, obs_teams, wpp, rw;  // wpp: uint64 words per plane; rw: words per row
    uint32_t cap;
    uint32_t agent_off;  // first agent (reward / action / position index)
    uint32_t obs_off;    // first obs word inside one slot
    uint32_t unp_off;    // first unpacked byte inside one slot
    uint32_t rows_off;   // first padded row word in rows[]
    uint32_t env_id;     // global env index used in Philox counters
};
static_assert(sizeof(EnvRT) == 32, "EnvRT layout");

struct EnvState {
    uint32_t ep_t;    // steps taken in the current episode
    uint32_t ep_idx;  // finished episodes
};

// Group flags.
constexpr uint16_t kUseTable = 1;   // obstacle plane from per-cell window tables
constexpr uint16_t kFog = 2;        // fog-of-war maps (one unit per env)
constexpr uint16_t kFogAgent = 4;   // with kFog: one unit per observing agent
constexpr uint16_t kSharedTable = 8;  // with kUseTable: one table of the larger emitting radius
                                      // serves both teams (line-of-sight families)
constexpr uint16_t kCentral = 16;     // centralized observation: two row buffers per emission warp
constexpr uint16_t kUnpStage = 32;    // the unpacked export is staged in shared memory by each emission warp
                                      // and written per step as one contiguous run (envs consecutive in the
                                      // layout; the one-thread emission of either form)

// All envs of a group share the radii, the emitting teams, the row width and
// the agent and seeker counts, so one code path serves the whole CTA.
struct Group {
    uint32_t list_first;  // first entry in env_list
    uint16_t n_envs;
    uint16_t n_slots;
    uint16_t flags;
    uint8_t n_dyn;        // dynamics warps (whole envs of <= 32 agents each)
    uint8_t pad;
};

__host__ __device__ inline uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }
// team_sees: the team's sightlines feed the centralized observation;
// team_emits: the team also writes decentralized planes.
__host__ __device__ inline bool team_sees(const EnvRT& E, int team) { return (E.obs_teams >> team) & 1u; }
__host__ __device__ inline bool team_emits(const EnvRT& E, int team) {
    return team_sees(E, team) && !(E.obs_teams & kObsNoDec);
}
__host__ __device__ inline bool only_hiders_emit(const EnvRT& E) { return (E.obs_teams & 3u) == (uint32_t)kObsHiders; }
__host__ __device__ inline bool line_of_sight(const EnvRT& E) { return (E.obs_teams & kObsLos) != 0u; }
__host__ __device__ inline int team_radius(const EnvRT& E, int team) { return team ? E.r_hide : E.r_seek; }
__host__ __device__ inline uint32_t words_of_radius(int r) {
    return (uint32_t)(((2 * r + 1) * (2 * r + 1) + 63) / 64);
}
// uint64 words of one window-table entry: the obstacle plane, then (with
// line of sight) the visibility mask
__host__ __device__ inline uint32_t table_words(const EnvRT& E, int r) {
    return words_of_radius(r) * (line_of_sight(E) ? 2u : 1u);
}

// Inside a CTA a cell is packed as x | y << sh with sh = 5 for grids up to
// 32 wide and 6 above; the per-env cell arrays are indexed by that value.
__host__ __device__ inline uint32_t cell_shift(const EnvRT& E) { return E.side <= 32 ? 5u : 6u; }

// Shared-memory plan of one CTA, computed identically on the host (to size
// the launch) and on the device (to place the buffers).
struct GroupPlan {
    uint32_t rows_off[kMaxGroupEnvs];    // uint64 units (padded obstacle rows)
    uint32_t cell_off[kMaxGroupEnvs];    // cells (2^sh * side per env): claim word + state byte
    uint32_t tbl_off[kMaxGroupEnvs][2];  // uint64 units per team, ~0u = none
    uint32_t fog_off[kMaxGroupEnvs + 1]; // fog-of-war rows (uint64 units; [units][side] per env)
    uint8_t first_slot[kMaxGroupEnvs];
    uint8_t dyn_first[kMaxDyn + 1];      // slot range of every dynamics warp
    uint32_t n_dyn;
    uint32_t n_envs;
    uint32_t n_slots;
    uint32_t max_side;                   // largest grid side of the group (sides may differ)
    uint32_t act_words;                  // uint32 words per action buffer
    uint32_t act, traj, rows, claim, tbl, state, fog, cen, total;  // byte offsets
    uint32_t prist;                      // streaming form: pristine records (byte offset)
    uint32_t rec_words;                  // streaming form: uint32 words of one (step, env) record
    uint32_t ring;                       // streaming form: trajectory steps held on chip
    uint32_t stage, stage_bytes;         // streaming form: unpacked staging (byte offset, bytes per emission warp)
    uint32_t unp_env;                    // streaming form: unpacked bytes of one env (uniform in the group)
    uint16_t flags;
};

// One thread emits a whole (step, env) when the seekers are the first
// ceil(A / 2) of at most 16 agents (windows of up to two words a plane);
// other shapes take the lane-per-agent emission.
__host__ __device__ inline bool fast_emission(const EnvRT& E) {
    return E.wpp <= 2 && E.n_agents <= (uint32_t)kFastAgents && E.n_seekers == (E.n_agents + 1u) / 2u;
}

// Kernel families: family 0 runs the general (lane per agent) emission;
// families 1..4 the one-thread emission for A in 1-4, 5-8, 9-12, 13-16 with
// one word a plane, families 5..8 the same with two words a plane (radius 4),
// families 9..12 and 13..16 the one- and two-word forms with line of sight.
// Each group is launched with the kernel of its family.
constexpr int kFamilies = 17;
__host__ __device__ inline int family_of(const EnvRT& E) {
    if (!fast_emission(E)) return 0;
    const int base = (E.obs_teams & kObsLos) ? (E.wpp == 2 ? 13 : 9) : (E.wpp == 2 ? 5 : 1);
    return base + ((int)E.n_agents - 1) / 4;
}

// Radius of the shared window table: the larger emitting radius.
__host__ __device__ inline int table_radius(const EnvRT& E) {
    const int rs = team_emits(E, 0) ? (int)E.r_seek : 0, rh = team_emits(E, 1) ? (int)E.r_hide : 0;
    return rs > rh ? rs : rh;
}

// Fog-of-war units of an env: all observing agents together, or each
// observing agent (seekers first).
__host__ __device__ inline uint32_t fog_units(const EnvRT& E, bool per_agent) {
    if (!per_agent) return 1u;
    return (team_sees(E, 0) ? E.n_seekers : 0u) + (team_sees(E, 1) ? E.n_agents - E.n_seekers : 0u);
}

// Unpacked bytes of one env: 3 (2r + 1)^2 per emitting agent.
__host__ __device__ inline uint32_t unpacked_bytes(const EnvRT& E) {
    uint32_t unp = 0;
    for (int a = 0; a < E.n_agents; ++a) {
        const int t = a < E.n_seekers ? 0 : 1;
        if (team_emits(E, t)) unp += 3u * (2u * team_radius(E, t) + 1u) * (2u * team_radius(E, t) + 1u);
    }
    return unp;
}

// Staging bytes of one emission warp for the unpacked export (kUnpStage): 32
// (step, env) items, and up to 15 bytes before each step run of a block (at
// most 32 runs), so that every run sits at its destination's offset mod 16.
__host__ __device__ inline uint32_t stage_bytes_of(uint32_t unp_env) {
    return align_up(32u * unp_env + 15u * 34u, 16);
}

// envs: the group's env constants in slot order.  Returns false when the
// group does not fit the dynamics warps.
__host__ __device__ inline bool plan_group(const EnvRT* envs, int n, int kc, uint16_t flags,
                                           GroupPlan& G) {
    uint32_t ro = 0, co = 0, to = 0, fo = 0, slot = 0, max_side = 0;
    int dyn = 0;
    uint32_t dyn_slots = 0;
    G.dyn_first[0] = 0;
    for (int i = 0; i < n; ++i) {
        const EnvRT& E = envs[i];
        if (dyn_slots + E.n_agents > 32u) {
            if (dyn + 1 >= kMaxDyn) return false;
            ++dyn;
            G.dyn_first[dyn] = (uint8_t)slot;
            dyn_slots = 0;
        }
        dyn_slots += E.n_agents;
        G.first_slot[i] = (uint8_t)slot;
        slot += E.n_agents;
        max_side = E.side > max_side ? E.side : max_side;
        G.rows_off[i] = ro;
        ro += (uint32_t)(E.side + 2 * kPad) * E.rw;
        G.cell_off[i] = co;
        co += (1u << cell_shift(E)) * E.side;
        G.fog_off[i] = fo;
        if (flags & kFog) fo += fog_units(E, (flags & kFogAgent) != 0) * E.side;
        for (int t = 0; t < 2; ++t) {
            G.tbl_off[i][t] = ~0u;
            if (!(flags & kUseTable) || !team_emits(E, t)) continue;
            if (t == 1 && team_emits(E, 0) && (E.r_hide == E.r_seek || (flags & kSharedTable))) {
                G.tbl_off[i][1] = G.tbl_off[i][0];
                continue;
            }
            G.tbl_off[i][t] = to;
            const int r = (flags & kSharedTable) ? table_radius(E) : team_radius(E, t);
            to += (uint32_t)E.side * E.side * table_words(E, r);
        }
    }
    G.fog_off[n] = fo;
    G.n_dyn = (uint32_t)dyn + 1;
    G.n_envs = (uint32_t)n;
    G.max_side = max_side;
    G.n_slots = slot;
    G.dyn_first[dyn + 1] = (uint8_t)slot;
    const uint32_t ns = slot, kcu = (uint32_t)kc;
    G.act_words = ((kcu + 3) / 4) * ns;                  // [kc/4][slots] words of 4 steps
    G.act = 0;                                           // uint32 [3][act_words]
    G.traj = align_up(G.act + 3 * G.act_words * 4, 16);  // uint16 [2][kc][slots]
    G.rows = align_up(G.traj + 2 * kcu * ns * 2, 16);
    G.claim = G.rows + ro * 8;                           // uint32 per cell
    G.tbl = align_up(G.claim + co * 4, 16);
    G.state = G.tbl + to * 8;                            // uint8 per cell
    G.fog = align_up(G.state + co, 16);                  // uint64 per fog row
    G.cen = align_up(G.fog + fo * 8, 16);                // uint64 [emit warps][2][4][side]
    const uint32_t cen_words = (flags & kCentral) ? kMaxEmitWarps * 8u * max_side : 0u;
    G.stage = align_up(G.cen + cen_words * 8, 16);  // uint8 [kMaxEmitWarps][stage_bytes]
    G.unp_env = n > 0 ? unpacked_bytes(envs[0]) : 0u;
    G.stage_bytes = (flags & kUnpStage) ? stage_bytes_of(G.unp_env) : 0u;
    G.total = align_up(G.stage + kMaxEmitWarps * G.stage_bytes, 16);
    G.prist = 0;
    G.rec_words = 0;
    G.ring = 0;
    G.flags = flags;
    return true;
}

// The streaming form of the step (stream_kernel): the dynamics warps write
// one record per (step, env) into an on-chip trajectory ring -- the cell
// x | y << sh of every agent as uint16, bit 15 of agent 0's entry set on the
// step that ends the episode -- and the emission warps consume them behind
// progress counters, with no block-wide barrier.  Record size by agent count.
__host__ __device__ constexpr uint32_t stream_rec_words(uint32_t A) {
    return A <= 2u ? 1u : (A <= 4u ? 2u : (A <= 8u ? 4u : 8u));
}
constexpr uint32_t kStreamRing = 64;   // trajectory steps on chip (power of two)
constexpr uint32_t kActRing = 16;      // Philox blocks (quads of steps) per agent slot on chip (power of two)
constexpr uint32_t kStreamGroup = 16;  // steps between the dynamics' progress updates
constexpr uint32_t kStreamMinOutRing = 2 * kStreamRing + 32;  // output ring steps the streaming form needs
constexpr uint32_t kErrWaitTimeout = 2u;  // error-word bit: a bounded wait of the step ran out
constexpr uint32_t kErrSmemPlan = 4u;     // error-word bit: a CTA's shared-memory plan exceeds its launch's
                                          // dynamic shared memory (the CTA returns before touching it)

#ifdef __CUDACC__
// Dynamic shared memory of the running launch, in bytes.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}
#endif

// Shared-memory plan of one CTA of the streaming form (the dynamics state
// bytes, obstacle rows and window tables as in plan_group; no claim words,
// action buffers or chunk trajectories).
__host__ __device__ inline bool plan_stream(const EnvRT* envs, int n, uint16_t flags, GroupPlan& G) {
    uint32_t ro = 0, co = 0, to = 0, slot = 0, max_side = 0;
    int dyn = 0;
    uint32_t dyn_slots = 0;
    G.dyn_first[0] = 0;
    for (int i = 0; i < n; ++i) {
        const EnvRT& E = envs[i];
        if (dyn_slots + E.n_agents > 32u) {
            if (dyn + 1 >= kMaxDyn) return false;
            ++dyn;
            G.dyn_first[dyn] = (uint8_t)slot;
            dyn_slots = 0;
        }
        dyn_slots += E.n_agents;
        G.first_slot[i] = (uint8_t)slot;
        slot += E.n_agents;
        max_side = E.side > max_side ? E.side : max_side;
        G.rows_off[i] = ro;
        ro += (uint32_t)(E.side + 2 * kPad) * E.rw;
        G.cell_off[i] = co;
        co += (1u << cell_shift(E)) * E.side;
        G.fog_off[i] = 0;
        for (int t = 0; t < 2; ++t) {
            G.tbl_off[i][t] = ~0u;
            if (!(flags & kUseTable) || !team_emits(E, t)) continue;
            if (t == 1 && team_emits(E, 0) && E.r_hide == E.r_seek) {
                G.tbl_off[i][1] = G.tbl_off[i][0];
                continue;
            }
            G.tbl_off[i][t] = to;
            to += (uint32_t)E.side * E.side * words_of_radius(team_radius(E, t));
        }
    }
    G.fog_off[n] = 0;
    G.n_dyn = (uint32_t)dyn + 1;
    G.n_envs = (uint32_t)n;
    G.max_side = max_side;
    G.n_slots = slot;
    G.dyn_first[dyn + 1] = (uint8_t)slot;
    G.act_words = 0;
    G.rec_words = n ? stream_rec_words(envs[0].n_agents) : 1u;
    G.ring = kStreamRing;
    G.traj = 0;                                                   // uint32 [ring][n][rec_words]
    G.prist = align_up(G.traj + G.ring * (uint32_t)n * G.rec_words * 4u, 16);  // uint32 [n][rec_words]
    G.rows = align_up(G.prist + (uint32_t)n * G.rec_words * 4u, 16);
    G.tbl = align_up(G.rows + ro * 8, 16);
    G.state = G.tbl + to * 8;                                     // uint8 per cell
    G.claim = align_up(G.state + co, 16);                         // uint32 per cell
    G.act_words = slot;                                           // uint32 action words of one quad
    G.act = align_up(G.claim + co * 4, 16);                       // uint32 [kActRing][slots]
    G.fog = G.cen = 0;
    G.unp_env = n > 0 ? unpacked_bytes(envs[0]) : 0u;
    G.stage = align_up(G.act + kActRing * slot * 4, 16);          // uint8 [kMaxEmitWarps][stage_bytes]
    G.stage_bytes = (flags & kUnpStage) ? stage_bytes_of(G.unp_env) : 0u;
    G.total = align_up(G.stage + kMaxEmitWarps * G.stage_bytes, 16);
    G.flags = flags;
    return true;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// two-multiplier bijection with the Weyl key schedule.
__host__ __device__ inline void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
#else
        const uint32_t hi0 = (uint32_t)(((uint64_t)0xD2511F53u * c0) >> 32);
        const uint32_t hi1 = (uint32_t)(((uint64_t)0xCD9E8D57u * c2) >> 32);
#endif
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Entries [first, first + count) of every ring slot of `stride` entries
// (run digests over the whole batch or over one env range).
struct DigestSpan {
    uint64_t stride, first, count;
};

struct StepParams {
    const EnvRT* env;
    EnvState* est;
    uint16_t* pos;
    const uint16_t* start;
    const uint64_t* rows;
    const Group* groups;
    const uint32_t* env_list;
    uint64_t* obs;       // ring [ring][obs_words]
    int32_t* rew;        // ring [ring][agents]
    uint8_t* done;       // ring [ring][n_envs]
    uint8_t* act_out;    // ring [ring][agents] or null
    uint8_t* unp;        // ring [ring][unp_bytes] or null
    uint64_t* central;   // ring [ring][central_words] or null (centralized observation)
    const uint32_t* central_off;  // per env: first word of its centralized observation
    uint64_t* fog;       // ring [ring][fog_words] or null (fog of war)
    const uint32_t* fog_off;  // per env: first word of its fog units in a slot
    uint64_t* fog_state; // per env at fog_off / 2: the discovery rows after the last step
    uint64_t fog_words;
    uint16_t* st_cells;  // ring [ring][agents] or null (true state: cells x | y << 6)
    uint32_t* st_ept;    // ring [ring][n_envs] or null (true state: episode clocks)
    uint64_t central_words;
    uint64_t obs_words;
    uint64_t agents;
    uint64_t unp_bytes;
    const uint64_t* clock;  // device step counter (steps taken before this enqueue)
    uint64_t t0;         // offset of the launch's first step from *clock
    uint32_t n_envs;
    uint32_t ring;
    uint32_t n_steps;
    uint32_t kc;         // steps per chunk (<= kMaxChunk, <= ring)
    uint32_t n_dyn;      // dynamics warps per CTA (the largest group's)
    uint32_t emit_warps;
    uint32_t key0, key1;        // (unused by the kernels: every env has its own key in `keys`)
    const uint2* keys;          // per env: Philox key (seed & 0xffffffff, seed >> 32)
    uint32_t dyn_ids;           // streaming form: warp id of dynamics warp d in bits [4d, 4d + 4),
                                // of the action warp in bits [16, 20)
    uint32_t* err;              // error word (kErrWaitTimeout)
};

}  // namespace hase
