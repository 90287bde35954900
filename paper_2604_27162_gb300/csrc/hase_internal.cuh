// hase_internal.cuh -- data layout shared by the host API and the kernels of
// the batched hide-and-seek environment step (Hide-And-Seek-Engine, arxiv
// 2604.27162).
//
// HBM layout of one handle (all device arrays, structure of arrays):
//   EnvRT    env[E]        per-env constants (32 B each)
//   EnvState est[E]        episode counters
//   uint16   pos[sumA]     current cell of every agent, x | y << 8
//   uint16   start[sumA]   pristine start cells (Sec. 4.2 template)
//   uint64   rows[...]     per env (S + 8) padded obstacle rows of RW words:
//                          bit x + 4 of row y + 4 is cell (x, y); every bit
//                          outside the grid is 1, so windows that leave the
//                          grid read obstacles without bounds checks
//   Group    groups[G]     the envs one CTA steps together
//   outputs                ring of ring_steps slots (see hase.h)
#pragma once

#include <stdint.h>

namespace hase {

constexpr int kPad = 4;          // padding cells around the grid (max radius)
constexpr int kMaxSlots = 16;    // agents per CTA group (half a warp)
constexpr int kMaxGroupEnvs = 16;
constexpr int kMaxChunk = 32;    // steps per on-chip chunk
constexpr int kObsHiders = 2;    // obs_teams value: only hiders emit

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

struct Group {
    uint32_t env_first;  // first env (envs of a group are consecutive)
    uint16_t n_envs;
    uint16_t n_slots;    // total agents of the group (<= kMaxSlots)
};

// Dynamic shared memory layout of one CTA (offsets in bytes from the base).
struct SmemLayout {
    uint32_t rows, nbr, act, traj, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// rows_words: padded row words of the group; nbr_bytes: sum of S*S.
__host__ __device__ inline SmemLayout smem_layout(uint32_t rows_words, uint32_t nbr_bytes) {
    SmemLayout L;
    L.act = 0;                                         // uint8 [3][16][kMaxChunk]
    L.traj = L.act + 3 * kMaxSlots * kMaxChunk;        // uint16 [2][kMaxChunk][16]
    L.rows = align_up(L.traj + 2 * kMaxChunk * kMaxSlots * 2, 16);  // uint64
    L.nbr = L.rows + rows_words * 8;                   // uint8
    L.total = align_up(L.nbr + nbr_bytes, 16);
    return L;
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

struct StepParams {
    const EnvRT* env;
    EnvState* est;
    uint16_t* pos;
    const uint16_t* start;
    const uint64_t* rows;
    const Group* groups;
    uint64_t* obs;       // ring [ring][obs_words]
    int32_t* rew;        // ring [ring][agents]
    uint8_t* done;       // ring [ring][n_envs]
    uint8_t* act_out;    // ring [ring][agents] or null
    uint8_t* unp;        // ring [ring][unp_bytes] or null
    uint64_t obs_words;
    uint64_t agents;
    uint64_t unp_bytes;
    uint64_t t0;         // global step index of the first step of the launch
    uint32_t n_envs;
    uint32_t ring;
    uint32_t slot0;      // t0 mod ring
    uint32_t n_steps;
    uint32_t kc;         // steps per chunk (<= kMaxChunk)
    uint32_t emit_warps;
    uint32_t key0, key1;
};

}  // namespace hase
