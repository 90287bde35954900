// hase_kernels.cu -- sm_103a kernels of the batched hide-and-seek environment
// step (Hide-And-Seek-Engine, arxiv 2604.27162).
//
//   gen_kernel      a0: start cells and Bernoulli obstacle rows (Sec. 3.2,
//                   Sec. 4.2 pristine template), one warp per env
//   observe_kernel  the step -1 observation after create / reset
//   step_kernel     a1-a9 fused over K steps.  One CTA steps a group of
//                   envs with at most 16 agents in total, all state in
//                   shared memory / registers for the whole launch:
//                     warp 0 ("dynamics") advances positions step by step;
//                       lanes 0-15 present each agent's current cell, lanes
//                       16-31 its move target, and one __match_any_sync
//                       resolves "target occupied" and "lowest index wins"
//                       for all agents at once (a2, a3, a7, a8);
//                     warps 1..M ("emission") run one chunk behind: for
//                       every (step, agent) of the previous chunk they
//                       encode the three observation planes, evaluate the
//                       reward with a warp ballot, write all outputs, and
//                       draw the Philox actions of the next chunk (a1, a5,
//                       a6, a9).
//                   The sequential part (positions) is thus decoupled from
//                   the bulk of the arithmetic and memory traffic, which is
//                   parallel over steps.
#include <cuda_runtime.h>

#include "hase_internal.cuh"

namespace hase {

// --------------------------------------------------------------------------
// Small helpers.
// --------------------------------------------------------------------------

// floor(u * n / 2^32)
__device__ __forceinline__ uint32_t mulhi_n(uint32_t u, uint32_t n) { return __umulhi(u, n); }

// D consecutive bits of a padded row starting at bit `start`.
__device__ __forceinline__ uint32_t row_bits(const uint64_t* row, int rw, int start, uint32_t mask) {
    if (rw == 1) return (uint32_t)(row[0] >> start) & mask;
    const uint64_t lo = row[0], hi = row[1];
    uint64_t v;
    if (start >= 64)
        v = hi >> (start - 64);
    else if (start == 0)
        v = lo;
    else
        v = (lo >> start) | (hi << (64 - start));
    return (uint32_t)v & mask;
}

// OR a short bit string v into the two-word plane (lo, hi) at bit sh.
__device__ __forceinline__ void or_bits(uint64_t& lo, uint64_t& hi, uint64_t v, int sh) {
    if (sh < 64) {
        lo |= v << sh;
        if (sh > 0) hi |= v >> (64 - sh);
    } else {
        hi |= v << (sh - 64);
    }
}

__device__ __forceinline__ int delta_of(uint32_t a) {
    // 1 N: y - 1, 2 S: y + 1, 3 E: x + 1, 4 W: x - 1 (cells packed x | y << 8)
    return a == 1u ? -256 : a == 2u ? 256 : a == 3u ? 1 : a == 4u ? -1 : 0;
}

// Three observation planes (a5) of agent a of one env at (x, y) with radius
// r, from the env's padded obstacle rows and the packed positions P[0..A).
__device__ __forceinline__ void encode_planes(const uint64_t* rows, int rw, int x, int y, int r,
                                              int a, int A, int ns, const uint16_t* P,
                                              uint64_t pl[3][2]) {
    const int D = 2 * r + 1;
    const uint32_t mask = (1u << D) - 1u;
#pragma unroll
    for (int q = 0; q < 3; ++q) pl[q][0] = pl[q][1] = 0;
    const int xs = x - r + kPad;
    const uint64_t* row = rows + (y - r + kPad) * rw;
    for (int dy = 0; dy < D; ++dy) {
        const uint32_t b = row_bits(row + dy * rw, rw, xs, mask);
        or_bits(pl[0][0], pl[0][1], b, dy * D);
    }
    const bool a_seek = a < ns;
    for (int b = 0; b < A; ++b) {
        if (b == a) continue;
        const uint32_t q = P[b];
        const int dx = (int)(q & 0xffu) - x + r;
        const int dy = (int)((q >> 8) & 0x7fu) - y + r;
        if ((unsigned)dx < (unsigned)D && (unsigned)dy < (unsigned)D) {
            const int bit = dy * D + dx;
            const int plane = ((b < ns) == a_seek) ? 1 : 2;
            if (bit < 64)
                pl[plane][0] |= 1ull << bit;
            else
                pl[plane][1] |= 1ull << (bit - 64);
        }
    }
}

// --------------------------------------------------------------------------
// a0: generation.  One warp per env.
// --------------------------------------------------------------------------
__global__ void gen_kernel(const EnvRT* __restrict__ env, const uint32_t* __restrict__ thr,
                           uint32_t n_envs, uint32_t key0,
                           uint32_t key1, uint16_t* __restrict__ pos, uint16_t* __restrict__ start,
                           uint64_t* __restrict__ rows, uint32_t* __restrict__ err) {
    const uint32_t e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (e >= n_envs) return;
    const EnvRT E = env[e];
    const uint32_t density_thr = thr[e];
    const int S = E.side, A = E.n_agents, rw = E.rw;
    // start cells: agent a draws word 0 of counter (attempt, a, env, 2),
    // redrawing while the cell is taken by an earlier agent.  Lane 0 alone.
    if (lane == 0) {
        uint32_t mine[kMaxSlots];
        for (int a = 0; a < A; ++a) {
            uint32_t attempt = 0, cell = 0;
            for (;;) {
                uint32_t c0 = attempt, c1 = (uint32_t)a, c2 = E.env_id, c3 = 2u;
                philox4x32_10(c0, c1, c2, c3, key0, key1);
                cell = mulhi_n(c0, (uint32_t)(S * S));
                bool dup = false;
                for (int b = 0; b < a; ++b) dup |= (mine[b] == cell);
                if (!dup) break;
                if (++attempt > (1u << 24)) {  // cannot happen for A <= S*S; bounded anyway
                    atomicOr(err, 1u);
                    break;
                }
            }
            mine[a] = cell;
            const uint16_t p = (uint16_t)((cell % S) | ((cell / S) << 8));
            start[E.agent_off + a] = p;
            pos[E.agent_off + a] = p;
        }
    }
    __syncwarp();  // start cells (global) visible to the whole warp
    // obstacle rows: cell c = y*S + x is blocked iff word c%4 of counter
    // (c/4, 0, env, 1) is below the threshold; start cells forced free.
    const int R = S + 2 * kPad;
    uint64_t* out = rows + E.rows_off;
    for (int pr = lane; pr < R; pr += 32) {
        const int y = pr - kPad;
        uint64_t w0 = ~0ull, w1 = ~0ull;
        if (y >= 0 && y < S) {
            uint32_t blk = 0xffffffffu, u[4] = {0, 0, 0, 0};
            for (int x = 0; x < S; ++x) {
                const uint32_t c = (uint32_t)(y * S + x);
                if ((c >> 2) != blk) {
                    blk = c >> 2;
                    uint32_t c0 = blk, c1 = 0u, c2 = E.env_id, c3 = 1u;
                    philox4x32_10(c0, c1, c2, c3, key0, key1);
                    u[0] = c0; u[1] = c1; u[2] = c2; u[3] = c3;
                }
                bool blocked = u[c & 3u] < density_thr;
                for (int a = 0; a < A; ++a) {
                    const uint16_t p = start[E.agent_off + a];
                    if ((p & 0xff) == x && (p >> 8) == y) blocked = false;
                }
                if (!blocked) {
                    const int bit = x + kPad;
                    if (bit < 64)
                        w0 &= ~(1ull << bit);
                    else
                        w1 &= ~(1ull << (bit - 64));
                }
            }
        }
        out[pr * rw] = w0;
        if (rw == 2) out[pr * rw + 1] = w1;
    }
}

// --------------------------------------------------------------------------
// The current-state observation (step -1 after create / reset): one thread
// per agent, reads positions and rows from global memory.
// --------------------------------------------------------------------------
__global__ void observe_kernel(const EnvRT* __restrict__ env, uint32_t n_envs,
                               const uint16_t* __restrict__ pos, const uint64_t* __restrict__ rows,
                               uint64_t* __restrict__ obs, uint8_t* __restrict__ unp) {
    const uint32_t e = blockIdx.x;
    if (e >= n_envs) return;
    const EnvRT E = env[e];
    const int a = threadIdx.x;
    if (a >= E.n_agents) return;
    const int ns = E.n_seekers;
    const bool seek = a < ns;
    if (!((E.obs_teams >> (seek ? 0 : 1)) & 1u)) return;
    const int r = seek ? E.r_seek : E.r_hide;
    const uint32_t p = pos[E.agent_off + a];
    uint64_t pl[3][2];
    encode_planes(rows + E.rows_off, E.rw, p & 0xff, p >> 8, r, a, E.n_agents, ns,
                  pos + E.agent_off, pl);
    const int ai = (E.obs_teams == kObsHiders) ? a - ns : a;
    const int W = E.wpp;
    uint64_t* o = obs + E.obs_off + (uint64_t)ai * 3 * W;
    for (int q = 0; q < 3; ++q)
        for (int j = 0; j < W; ++j) o[q * W + j] = pl[q][j];
    if (unp) {
        const int D = 2 * r + 1;
        // unpacked bytes of earlier emitting agents: same radius for a team
        uint8_t* u = unp + E.unp_off;
        for (int b = 0; b < a; ++b) {
            const bool bs = b < ns;
            if ((E.obs_teams >> (bs ? 0 : 1)) & 1u) {
                const int rb = bs ? E.r_seek : E.r_hide;
                u += 3 * (2 * rb + 1) * (2 * rb + 1);
            }
        }
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < D * D; ++k) u[q * D * D + k] = (uint8_t)((pl[q][k >> 6] >> (k & 63)) & 1u);
    }
}

// --------------------------------------------------------------------------
// a1-a9 fused over n_steps steps.
// --------------------------------------------------------------------------
struct CtaShared {
    EnvRT env[kMaxGroupEnvs];
    uint32_t rows_off[kMaxGroupEnvs];
    uint32_t nbr_off[kMaxGroupEnvs];
    uint32_t unp_rel[kMaxSlots];   // unpacked byte offset of the slot inside its env
    uint16_t start[kMaxSlots];
    uint16_t env_mask[kMaxSlots];  // slots (bits) sharing the env of slot s
    uint8_t slot_env[kMaxSlots];
    uint8_t slot_agent[kMaxSlots];
    uint8_t first_slot[kMaxGroupEnvs];
    uint32_t rows_total, nbr_total;
};

__global__ void __launch_bounds__(512) step_kernel(const StepParams P) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ CtaShared H;
    const Group G = P.groups[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    const int ne = G.n_envs, nsl = G.n_slots;

    if (tid == 0) {
        uint32_t ro = 0, no = 0;
        int slot = 0;
        for (int i = 0; i < ne; ++i) {
            const EnvRT E = P.env[G.env_first + i];
            H.env[i] = E;
            H.rows_off[i] = ro;
            ro += (uint32_t)(E.side + 2 * kPad) * E.rw;
            H.nbr_off[i] = no;
            no += (uint32_t)E.side * E.side;
            H.first_slot[i] = (uint8_t)slot;
            uint32_t urel = 0;
            for (int a = 0; a < E.n_agents; ++a) {
                H.slot_env[slot] = (uint8_t)i;
                H.slot_agent[slot] = (uint8_t)a;
                H.unp_rel[slot] = urel;
                const bool sk = a < E.n_seekers;
                if ((E.obs_teams >> (sk ? 0 : 1)) & 1u) {
                    const int r = sk ? E.r_seek : E.r_hide;
                    urel += 3u * (2 * r + 1) * (2 * r + 1);
                }
                ++slot;
            }
            const uint16_t m = (uint16_t)(((1u << E.n_agents) - 1u) << H.first_slot[i]);
            for (int a = 0; a < E.n_agents; ++a) H.env_mask[H.first_slot[i] + a] = m;
        }
        H.rows_total = ro;
        H.nbr_total = no;
    }
    __syncthreads();
    const SmemLayout L = smem_layout(H.rows_total, H.nbr_total);
    uint8_t* s_act = sm + L.act;                         // [3][16][kMaxChunk]
    uint16_t* s_traj = (uint16_t*)(sm + L.traj);         // [2][kMaxChunk][16]
    uint64_t* s_rows = (uint64_t*)(sm + L.rows);
    uint8_t* s_nbr = sm + L.nbr;

    // stage the pristine template: padded rows and start cells
    for (int i = 0; i < ne; ++i) {
        const EnvRT& E = H.env[i];
        const uint32_t n = (uint32_t)(E.side + 2 * kPad) * E.rw;
        for (uint32_t j = tid; j < n; j += nthreads) s_rows[H.rows_off[i] + j] = P.rows[E.rows_off + j];
    }
    if (tid < nsl) {
        const EnvRT& E = H.env[H.slot_env[tid]];
        H.start[tid] = P.start[E.agent_off + H.slot_agent[tid]];
    }
    __syncthreads();
    // passable-neighbour masks: bit a set iff action a (1 N, 2 S, 3 E, 4 W)
    // leads onto a free cell inside the grid
    for (int i = 0; i < ne; ++i) {
        const EnvRT& E = H.env[i];
        const int S = E.side, rw = E.rw;
        const uint64_t* R = s_rows + H.rows_off[i];
        for (int c = tid; c < S * S; c += nthreads) {
            const int x = c % S, y = c / S;
            auto blocked = [&](int xx, int yy) -> uint32_t {
                const int b = xx + kPad;
                return (uint32_t)((R[(yy + kPad) * rw + (b >> 6)] >> (b & 63)) & 1ull);
            };
            const uint32_t m = ((blocked(x, y - 1) ^ 1u) << 1) | ((blocked(x, y + 1) ^ 1u) << 2) |
                               ((blocked(x + 1, y) ^ 1u) << 3) | ((blocked(x - 1, y) ^ 1u) << 4);
            s_nbr[H.nbr_off[i] + c] = (uint8_t)m;
        }
    }

    const uint32_t kc = P.kc;
    const uint32_t n_chunks = (P.n_steps + kc - 1) / kc;
    const int M = P.emit_warps;

    // a1: Philox actions of chunk c into buffer c % 3.  Items (block, slot);
    // one Philox block serves four consecutive steps.
    auto draw_actions = [&](uint32_t c, int worker, int n_workers) {
        const uint64_t ts = P.t0 + (uint64_t)c * kc;
        const uint32_t len = min(kc, P.n_steps - c * kc);
        const uint64_t te = ts + len;
        const uint64_t b0 = ts >> 2, b1 = (te - 1) >> 2;
        const uint32_t nblk = (uint32_t)(b1 - b0 + 1);
        uint8_t* A = s_act + (c % 3u) * (kMaxSlots * kMaxChunk);
        for (uint32_t it = worker; it < nblk * (uint32_t)nsl; it += n_workers) {
            const uint32_t bi = it / nsl, s = it % nsl;
            const EnvRT& E = H.env[H.slot_env[s]];
            uint32_t c0 = (uint32_t)(b0 + bi), c1 = H.slot_agent[s], c2 = E.env_id, c3 = 0u;
            philox4x32_10(c0, c1, c2, c3, P.key0, P.key1);
            const uint32_t u[4] = {c0, c1, c2, c3};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t t = (b0 + bi) * 4 + j;
                if (t >= ts && t < te) A[s * kMaxChunk + (uint32_t)(t - ts)] = (uint8_t)mulhi_n(u[j], 5u);
            }
        }
    };

    if (n_chunks > 0) draw_actions(0, tid, nthreads);
    __syncthreads();

    // ---------------- dynamics warp state ----------------
    const int s_dyn = lane & 15;
    const bool up = lane >= 16;
    const bool live = (warp == 0) && s_dyn < nsl;
    uint32_t p = 0, p0 = 0, nbr_cur = 0, nbr0 = 0, ep_t = 0, ep_idx = 0, cap = 1;
    uint32_t eb = 0, S_dyn = 1, lowmask = 0xffffffffu;
    const uint8_t* nb = s_nbr;
    int env_dyn = 0;
    if (warp == 0) {
        if (live) {
            env_dyn = H.slot_env[s_dyn];
            const EnvRT& E = H.env[env_dyn];
            S_dyn = E.side;
            nb = s_nbr + H.nbr_off[env_dyn];
            p = P.pos[E.agent_off + H.slot_agent[s_dyn]];
            p0 = H.start[s_dyn];
            nbr_cur = nb[(p >> 8) * S_dyn + (p & 0xff)];
            nbr0 = nb[(p0 >> 8) * S_dyn + (p0 & 0xff)];
            const EnvState st = P.est[G.env_first + env_dyn];
            ep_t = st.ep_t;
            ep_idx = st.ep_idx;
            cap = E.cap;
            eb = (uint32_t)env_dyn << 16;
        }
        if (up) lowmask = 0xffffu | (((1u << s_dyn) - 1u) << 16);
    }
    const uint32_t sent = 0x80000000u | (uint32_t)lane;

    // ---------------- emission lane mapping ----------------
    const int ew = warp - 1;                   // emission warp index
    const int segs = 32 / nsl;                 // (step, group) segments per warp
    const int seg = lane / nsl;
    const int s_em = lane - seg * nsl;
    const bool em_lane = seg < segs;

    for (uint32_t c = 0; c <= n_chunks; ++c) {
        if (warp == 0) {
            if (c < n_chunks) {
                // ---------------- a2 a3 a7 a8: positions of chunk c ----------------
                const uint32_t len = min(kc, P.n_steps - c * kc);
                const uint8_t* A = s_act + (c % 3u) * (kMaxSlots * kMaxChunk) + s_dyn * kMaxChunk;
                uint16_t* T = s_traj + (c & 1u) * (kMaxChunk * kMaxSlots);
                for (uint32_t k = 0; k < len; ++k) {
                    const uint32_t a = live ? A[k] : 0u;
                    const uint32_t tgt = p + (uint32_t)delta_of(a);
                    const bool valid = live && ((nbr_cur >> a) & 1u);
                    uint32_t ntgt = 0;
                    if (valid) ntgt = nb[(tgt >> 8) * S_dyn + (tgt & 0xff)];
                    const uint32_t key = !live ? sent : (up ? (valid ? (eb | tgt) : sent) : (eb | p));
                    const uint32_t m = __match_any_sync(0xffffffffu, key);
                    const bool won = up && valid && ((m & lowmask) == 0u);
                    const uint32_t bal = __ballot_sync(0xffffffffu, won);
                    if ((bal >> (16 + s_dyn)) & 1u) {
                        p = tgt;
                        nbr_cur = ntgt;
                    }
                    ++ep_t;
                    const bool done = ep_t == cap;
                    if (live && !up) T[k * kMaxSlots + s_dyn] = (uint16_t)(p | (done ? 0x8000u : 0u));
                    if (done) {
                        p = p0;
                        nbr_cur = nbr0;
                        ep_t = 0;
                        ++ep_idx;
                    }
                }
            }
        } else {
          if (c >= 1) {
            // ---------------- a5 a6 a9: outputs of chunk c - 1 ----------------
            const uint32_t cp = c - 1;
            const uint32_t len = min(kc, P.n_steps - cp * kc);
            const uint16_t* T = s_traj + (cp & 1u) * (kMaxChunk * kMaxSlots);
            const uint8_t* Aact = s_act + (cp % 3u) * (kMaxSlots * kMaxChunk);
            // ring slot of the chunk's first step
            const uint32_t base_slot = (uint32_t)(((uint64_t)P.slot0 + (uint64_t)cp * kc) % P.ring);
            const int ei = em_lane ? H.slot_env[s_em] : 0;
            const EnvRT& E = H.env[ei];
            const int a = em_lane ? H.slot_agent[s_em] : 0;
            const int ns = E.n_seekers, An = E.n_agents;
            const bool seek = a < ns;
            const bool emits = em_lane && ((E.obs_teams >> (seek ? 0 : 1)) & 1u);
            const int r = seek ? E.r_seek : E.r_hide;
            const int W = E.wpp;
            const int ai = (E.obs_teams == kObsHiders) ? a - ns : a;
            const int first = H.first_slot[ei];
            const uint32_t envmask = em_lane ? ((uint32_t)H.env_mask[s_em] << (seg * nsl)) : 0u;
            const uint32_t rs = E.r_seek;
            for (uint32_t kb = (uint32_t)(ew * segs); kb < len; kb += (uint32_t)(M * segs)) {
                const uint32_t k = kb + (uint32_t)seg;
                const bool act_item = em_lane && k < len;
                const uint16_t* Tk = T + (act_item ? k : 0) * kMaxSlots;
                const uint32_t v = Tk[s_em];
                const bool done = (v >> 15) & 1u;
                // a6: hider seen by a seeker (post-move, pre-reset positions)
                bool seen = false;
                if (act_item && !seek) {
                    const int hx = v & 0xff, hy = (v >> 8) & 0x7f;
                    for (int j = 0; j < ns; ++j) {
                        const uint32_t q = Tk[first + j];
                        const int dx = abs((int)(q & 0xff) - hx), dy = abs((int)((q >> 8) & 0x7f) - hy);
                        seen |= max(dx, dy) <= (int)rs;
                    }
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, seen);
                if (!act_item) continue;
                const int32_t reward = seek ? (int32_t)__popc(bal & envmask) : (seen ? -1 : 0);
                uint32_t slot = base_slot + k;
                while (slot >= P.ring) slot -= P.ring;
                P.rew[(uint64_t)slot * P.agents + E.agent_off + a] = reward;
                if (a == 0) P.done[(uint64_t)slot * P.n_envs + G.env_first + ei] = done ? 3u : 0u;
                if (P.act_out) P.act_out[(uint64_t)slot * P.agents + E.agent_off + a] = Aact[s_em * kMaxChunk + k];
                if (emits) {
                    // a5 on the post-reset positions
                    const uint16_t* Pos = done ? (H.start + first) : (Tk + first);
                    const uint32_t pp = Pos[a];
                    uint64_t pl[3][2];
                    encode_planes(s_rows + H.rows_off[ei], E.rw, pp & 0xff, (pp >> 8) & 0x7f, r, a, An,
                                  ns, Pos, pl);
                    uint64_t* o = P.obs + (uint64_t)slot * P.obs_words + E.obs_off + (uint64_t)ai * 3 * W;
                    for (int q = 0; q < 3; ++q)
                        for (int j = 0; j < W; ++j) o[q * W + j] = pl[q][j];
                    if (P.unp) {
                        const int D = 2 * r + 1;
                        uint8_t* u = P.unp + (uint64_t)slot * P.unp_bytes + E.unp_off + H.unp_rel[s_em];
                        for (int q = 0; q < 3; ++q)
                            for (int kk = 0; kk < D * D; ++kk)
                                u[q * D * D + kk] = (uint8_t)((pl[q][kk >> 6] >> (kk & 63)) & 1u);
                    }
                }
            }
          }
          // a1 for chunk c + 1
          if (c + 1 < n_chunks) draw_actions(c + 1, tid - 32, M * 32);
        }
        __syncthreads();
    }

    // write back the dynamic state
    if (warp == 0 && live && !up) {
        const EnvRT& E = H.env[env_dyn];
        P.pos[E.agent_off + H.slot_agent[s_dyn]] = (uint16_t)p;
        if (H.slot_agent[s_dyn] == 0) {
            EnvState st;
            st.ep_t = ep_t;
            st.ep_idx = ep_idx;
            P.est[G.env_first + env_dyn] = st;
        }
    }
}

// --------------------------------------------------------------------------
// Launchers (host).
// --------------------------------------------------------------------------
cudaError_t launch_generate(const EnvRT* env, const uint32_t* thr, uint32_t n_envs, uint32_t key0,
                            uint32_t key1, uint16_t* pos, uint16_t* start, uint64_t* rows, uint32_t* err,
                            cudaStream_t st) {
    if (n_envs == 0) return cudaSuccess;
    const uint32_t wpb = 4;
    gen_kernel<<<(n_envs + wpb - 1) / wpb, wpb * 32, 0, st>>>(env, thr, n_envs, key0, key1, pos, start,
                                                              rows, err);
    return cudaGetLastError();
}

cudaError_t launch_observe(const EnvRT* env, uint32_t n_envs, const uint16_t* pos,
                           const uint64_t* rows, uint64_t* obs, uint8_t* unp, cudaStream_t st) {
    if (n_envs == 0) return cudaSuccess;
    observe_kernel<<<n_envs, 32, 0, st>>>(env, n_envs, pos, rows, obs, unp);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem,
                        cudaStream_t st) {
    if (n_groups == 0 || p.n_steps == 0) return cudaSuccess;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    step_kernel<<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hase
