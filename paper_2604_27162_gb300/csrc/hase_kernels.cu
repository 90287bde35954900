// hase_kernels.cu -- sm_103a kernels of the batched hide-and-seek environment
// step (Hide-And-Seek-Engine, arxiv 2604.27162) other than the fused step:
//
//   gen_kernel      a0: start cells and Bernoulli obstacle rows (Sec. 3.2,
//                   Sec. 4.2 pristine template), one warp per env
//   prestep_kernel  the desynchronised start: each env's moves before its
//                   first observation (Sec. 3.3, last paragraph)
//   observe_kernel  the step -1 observation after create / reset (and
//                   central_init_kernel, state_init_kernel, fog_init_kernel:
//                   its centralized observation, true state and fog of war)
//   digest kernels  the run summary of hase_digest / hase_digest_noalloc
//   advance_kernel  the device step counter
// and the host launchers; the step kernel itself is in hase_step.cuh.
#include <mutex>

#include "hase_step.cuh"

namespace hase {

// --------------------------------------------------------------------------
// a0: generation.  One warp per env.
// --------------------------------------------------------------------------
__global__ void gen_kernel(const EnvRT* __restrict__ env, const uint32_t* __restrict__ thr,
                           uint32_t n_envs, const uint2* __restrict__ keys, uint16_t* __restrict__ pos,
                           uint16_t* __restrict__ start, uint64_t* __restrict__ rows,
                           uint32_t* __restrict__ err) {
    const uint32_t e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (e >= n_envs) return;
    const EnvRT E = env[e];
    const uint32_t density_thr = thr[e];
    const uint32_t key0 = keys[e].x, key1 = keys[e].y;  // the env's Philox key
    const int S = E.side, A = E.n_agents, rw = E.rw;
    // start cells: agent a draws word 0 of counter (attempt, a, env, 2),
    // redrawing while the cell is taken by an earlier agent.  Lane 0 alone.
    if (lane == 0) {
        uint32_t mine[kMaxAgents];
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
            const uint16_t p = (uint16_t)pack_xy(cell % S, cell / S);
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
                    u[0] = c0;
                    u[1] = c1;
                    u[2] = c2;
                    u[3] = c3;
                }
                bool blocked = u[c & 3u] < density_thr;
                for (int a = 0; a < A; ++a)
                    if (start[E.agent_off + a] == pack_xy(x, y)) blocked = false;
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
// Desynchronised start (Sec. 3.3, last paragraph: the envs of a batch are
// stepped stochastically at initialisation).  Env e takes ep_t(e) steps of
// its dynamics from the start cells before its first observation, with
// actions of their own Philox stream: pre-step tau uses word tau % 4 of
// counter (tau / 4, agent, env id, 4).  A move is valid when the action is
// not "stay" and the target is inside the grid, free of obstacles and not
// any agent's current cell; among valid movers with the same target the
// lowest agent index moves.  One warp per env, lane a = agent a; ep_t < cap,
// so no episode ends, and nothing is written but the positions.
// --------------------------------------------------------------------------
__global__ void prestep_kernel(const EnvRT* __restrict__ env, uint32_t n_envs, const uint2* __restrict__ keys,
                               const EnvState* __restrict__ est, const uint64_t* __restrict__ rows,
                               uint16_t* __restrict__ pos) {
    const uint32_t e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31;
    if (e >= n_envs) return;  // whole warps
    const EnvRT E = env[e];
    const uint32_t A = E.n_agents, rw = E.rw;
    const uint64_t* R = rows + E.rows_off;
    const bool live = lane < A;
    int x = 0, y = 0;
    if (live) {
        const uint32_t p = pos[E.agent_off + lane];
        x = (int)px(p);
        y = (int)py(p);
    }
    const uint32_t n = est[e].ep_t, key0 = keys[e].x, key1 = keys[e].y;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    for (uint32_t tau = 0; tau < n; ++tau) {
        if ((tau & 3u) == 0u) {
            uint32_t c0 = tau >> 2, c1 = lane, c2 = E.env_id, c3 = 4u;
            philox4x32_10(c0, c1, c2, c3, key0, key1);
            w[0] = c0;
            w[1] = c1;
            w[2] = c2;
            w[3] = c3;
        }
        const uint32_t u = (tau & 3u) == 0u ? w[0] : (tau & 3u) == 1u ? w[1] : (tau & 3u) == 2u ? w[2] : w[3];
        const uint32_t act = mulhi_n(u, 5u);  // 0 stay, 1 N, 2 S, 3 E, 4 W
        const int tx = x + (act == 3u) - (act == 4u);
        const int ty = y + (act == 2u) - (act == 1u);
        bool ok = live && act != 0u;
        if (ok) {  // padded rows: row ty + kPad, bit tx + kPad; outside the grid reads blocked
            const uint32_t bit = (uint32_t)(tx + kPad);
            ok = ((R[(uint32_t)(ty + kPad) * rw + (bit >> 6)] >> (bit & 63u)) & 1ull) == 0ull;
        }
        const uint32_t cur = live ? pack_xy((uint32_t)x, (uint32_t)y) : 0xffffffffu;
        const uint32_t tgt = ok ? pack_xy((uint32_t)tx, (uint32_t)ty) : 0xfffffffeu;
        // every lane takes part in every shuffle (no short-circuit around them)
        for (uint32_t b = 0; b < A; ++b) {  // target held by some agent now
            const uint32_t cb = __shfl_sync(0xffffffffu, cur, b);
            ok = ok && cb != tgt;
        }
        const uint32_t claim = ok ? tgt : 0xfffffffeu;
        bool moves = ok;
        for (uint32_t b = 0; b < A; ++b) {  // a lower valid mover wants the same cell
            const uint32_t cl = __shfl_sync(0xffffffffu, claim, b);
            moves = moves && !(b < lane && cl == claim);
        }
        if (moves) {
            x = tx;
            y = ty;
        }
    }
    if (live) pos[E.agent_off + lane] = (uint16_t)pack_xy((uint32_t)x, (uint32_t)y);
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
    const int team = a < ns ? 0 : 1;
    if (!team_emits(E, team)) return;
    const int r = team_radius(E, team);
    const uint32_t p = pos[E.agent_off + a];
    uint64_t pl[3][2];
    obstacle_plane(rows + E.rows_off, E.rw, px(p), py(p), r, pl[0][0], pl[0][1]);
    team_planes_pairwise(px(p), py(p), r, a, E.n_agents, ns, pos + E.agent_off, pl[1][0], pl[1][1],
                         pl[2][0], pl[2][1]);
    if (line_of_sight(E)) {  // hidden cells read 0 in every plane
        uint64_t vl, vh;
        window_visibility(pl[0][0], pl[0][1], r, vl, vh);
        for (int q = 0; q < 3; ++q) {
            pl[q][0] &= vl;
            pl[q][1] &= vh;
        }
    }
    const int ai = only_hiders_emit(E) ? a - ns : a;
    const int W = E.wpp;
    uint64_t* o = obs + E.obs_off + (uint64_t)ai * 3 * W;
    for (int q = 0; q < 3; ++q)
        for (int j = 0; j < W; ++j) o[q * W + j] = pl[q][j];
    if (unp) {
        const int D = 2 * r + 1;
        uint8_t* u = unp + E.unp_off;
        for (int b = 0; b < a; ++b) {
            const int tb = b < ns ? 0 : 1;
            if (team_emits(E, tb)) {
                const int rb = team_radius(E, tb);
                u += 3 * (2 * rb + 1) * (2 * rb + 1);
            }
        }
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < D * D; ++k) u[q * D * D + k] = (uint8_t)((pl[q][k >> 6] >> (k & 63)) & 1u);
    }
}

// The centralized observation after create / reset, one thread per env.
__global__ void central_init_kernel(const EnvRT* __restrict__ env, uint32_t n_envs, const uint16_t* __restrict__ pos,
                                    const uint64_t* __restrict__ rows, const uint32_t* __restrict__ coff,
                                    uint64_t* __restrict__ central) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_envs) return;
    const EnvRT E = env[e];
    central_env(E, rows + E.rows_off, pos + E.agent_off, 6u, central + coff[e]);
}

cudaError_t launch_central_init(const EnvRT* env, uint32_t n_envs, const uint16_t* pos, const uint64_t* rows,
                                const uint32_t* coff, uint64_t* central, cudaStream_t st) {
    if (n_envs == 0) return cudaSuccess;
    central_init_kernel<<<(n_envs + 63) / 64, 64, 0, st>>>(env, n_envs, pos, rows, coff, central);
    return cudaGetLastError();
}

// The true state after create / reset: the cells (the handle's positions are
// already x | y << 6) and the episode clocks, one thread per agent or env.
__global__ void state_init_kernel(const uint16_t* __restrict__ pos, const EnvState* __restrict__ est,
                                  uint32_t agents, uint32_t n_envs, uint16_t* __restrict__ cells,
                                  uint32_t* __restrict__ ept) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < agents) cells[i] = pos[i];
    if (i < n_envs) ept[i] = est[i].ep_t;
}

cudaError_t launch_state_init(const uint16_t* pos, const EnvState* est, uint32_t agents, uint32_t n_envs,
                              uint16_t* cells, uint32_t* ept, cudaStream_t st) {
    const uint32_t n = agents > n_envs ? agents : n_envs;
    if (n == 0) return cudaSuccess;
    state_init_kernel<<<(n + 255) / 256, 256, 0, st>>>(pos, est, agents, n_envs, cells, ept);
    return cudaGetLastError();
}

// The fog of war after create / reset: the first observation of an episode
// starts every map (discovered = newly discovered = seen), one thread per env.
__global__ void fog_init_kernel(const EnvRT* __restrict__ env, uint32_t n_envs, const uint16_t* __restrict__ pos,
                                const uint64_t* __restrict__ rows, const uint32_t* __restrict__ foff,
                                uint32_t per_agent, uint64_t* __restrict__ fog, uint64_t* __restrict__ state) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_envs) return;
    const EnvRT E = env[e];
    const uint32_t S = E.side, units = fog_units(E, per_agent != 0u);
    const int ns = E.n_seekers;
    const uint16_t* p = pos + E.agent_off;
    for (uint32_t j = 0; j < units; ++j) {
        const int a0 = per_agent ? (team_sees(E, 0) ? (int)j : ns + (int)j) : 0;
        const int a1 = per_agent ? a0 + 1 : (int)E.n_agents;
        for (uint32_t y = 0; y < S; ++y) {
            uint64_t seen = 0;
            for (int a = a0; a < a1; ++a) {
                const int team = a < ns ? 0 : 1;
                if (team_sees(E, team)) seen |= agent_seen_row(E, rows + E.rows_off, p[a], 6u, team, (int)y);
            }
            fog[foff[e] + j * 2u * S + y] = seen;
            fog[foff[e] + j * 2u * S + S + y] = seen;
            state[foff[e] / 2u + j * S + y] = seen;
        }
    }
}

cudaError_t launch_fog_init(const EnvRT* env, uint32_t n_envs, const uint16_t* pos, const uint64_t* rows,
                            const uint32_t* foff, uint32_t per_agent, uint64_t* fog, uint64_t* state,
                            cudaStream_t st) {
    if (n_envs == 0) return cudaSuccess;
    fog_init_kernel<<<(n_envs + 63) / 64, 64, 0, st>>>(env, n_envs, pos, rows, foff, per_agent, fog, state);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Launchers (host).
// --------------------------------------------------------------------------
cudaError_t launch_generate(const EnvRT* env, const uint32_t* thr, uint32_t n_envs, const uint2* keys,
                            uint16_t* pos, uint16_t* start, uint64_t* rows, uint32_t* err, cudaStream_t st) {
    if (n_envs == 0) return cudaSuccess;
    const uint32_t wpb = 4;
    gen_kernel<<<(n_envs + wpb - 1) / wpb, wpb * 32, 0, st>>>(env, thr, n_envs, keys, pos, start,
                                                              rows, err);
    return cudaGetLastError();
}

cudaError_t launch_prestep(const EnvRT* env, uint32_t n_envs, const uint2* keys, const EnvState* est,
                           const uint64_t* rows, uint16_t* pos, cudaStream_t st) {
    if (n_envs == 0) return cudaSuccess;
    const uint32_t wpb = 4;
    prestep_kernel<<<(n_envs + wpb - 1) / wpb, wpb * 32, 0, st>>>(env, n_envs, keys, est, rows, pos);
    return cudaGetLastError();
}

cudaError_t launch_observe(const EnvRT* env, uint32_t n_envs, const uint16_t* pos,
                           const uint64_t* rows, uint64_t* obs, uint8_t* unp, cudaStream_t st) {
    if (n_envs == 0) return cudaSuccess;
    observe_kernel<<<n_envs, 32, 0, st>>>(env, n_envs, pos, rows, obs, unp);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Run digest: order-independent sums (mod 2^64) over the ring slots of n
// consecutive steps, of one span (stride, first, count) per slot of the obs
// words, the done bytes and the rewards (the whole slot, or one env range).
// Pass 1: every block reduces a grid-stride share of the obs words, done
// bytes and rewards into scratch[block] (three words); pass 2: one block adds
// the partials.  A third kernel gives per-agent reward sums.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    __syncthreads();
    return s;  // valid in thread 0
}

// Flattened (step, item) walk: start at `i`, advance by the grid size.
struct Walk {
    uint64_t s, j, q, r;
    __device__ Walk(uint64_t i, uint64_t items) {
        s = i / items;
        j = i - s * items;
        const uint64_t g = (uint64_t)gridDim.x * blockDim.x;
        q = g / items;
        r = g - q * items;
    }
    __device__ void next(uint64_t items) {
        j += r;
        s += q;
        if (j >= items) {
            j -= items;
            ++s;
        }
    }
};

__global__ void digest_partial_kernel(const uint64_t* obs, const uint8_t* done, const int32_t* rew, DigestSpan ow,
                                      DigestSpan ev, DigestSpan ag, uint32_t ring, uint64_t first, uint32_t n_steps,
                                      uint64_t* scratch) {
    __shared__ uint64_t red[32];
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t dig = 0, eps = 0, rs = 0;
    if (ow.count) {  // digest index of word j of step s: s * count + j
        const uint64_t total = (uint64_t)n_steps * ow.count;
        Walk w(i0, ow.count);
        for (uint64_t i = i0; i < total; i += (uint64_t)gridDim.x * blockDim.x, w.next(ow.count)) {
            const uint64_t slot = (first + w.s) % ring;
            dig += splitmix64(obs[slot * ow.stride + ow.first + w.j] ^ i);
        }
    }
    if (ev.count) {
        const uint64_t total = (uint64_t)n_steps * ev.count;
        Walk w(i0, ev.count);
        for (uint64_t i = i0; i < total; i += (uint64_t)gridDim.x * blockDim.x, w.next(ev.count))
            eps += done[((first + w.s) % ring) * ev.stride + ev.first + w.j] & 1u;
    }
    if (ag.count) {
        const uint64_t total = (uint64_t)n_steps * ag.count;
        Walk w(i0, ag.count);
        for (uint64_t i = i0; i < total; i += (uint64_t)gridDim.x * blockDim.x, w.next(ag.count))
            rs += (uint64_t)(int64_t)rew[((first + w.s) % ring) * ag.stride + ag.first + w.j];
    }
    dig = block_sum(dig, red);
    eps = block_sum(eps, red);
    rs = block_sum(rs, red);
    if (threadIdx.x == 0) {
        scratch[3 * blockIdx.x + 0] = dig;
        scratch[3 * blockIdx.x + 1] = eps;
        scratch[3 * blockIdx.x + 2] = rs;
    }
}

__global__ void digest_final_kernel(const uint64_t* scratch, uint32_t n_part, const uint32_t* err, uint64_t* out) {
    __shared__ uint64_t red[32];
    uint64_t v[3] = {0, 0, 0};
    for (uint32_t b = threadIdx.x; b < n_part; b += blockDim.x)
        for (int k = 0; k < 3; ++k) v[k] += scratch[3 * b + k];
    for (int k = 0; k < 3; ++k) v[k] = block_sum(v[k], red);
    if (threadIdx.x == 0) {
        out[0] = v[0];
        out[1] = v[1];
        out[2] = v[2];
        out[3] = err ? (uint64_t)*err : 0ull;
    }
}

__global__ void agent_reward_kernel(const int32_t* rew, DigestSpan ag, uint32_t ring, uint64_t first,
                                    uint32_t n_steps, int64_t* agent_rew) {
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < ag.count;
         a += (uint64_t)gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (uint32_t k = 0; k < n_steps; ++k) s += rew[((first + k) % ring) * ag.stride + ag.first + a];
        agent_rew[a] = s;
    }
}

// Scratch of hase_digest_noalloc: the first pass's partial sums, 3 words per
// block for at most kDigestBlocks blocks (6 KiB).  Pass 1 writes every slot
// pass 2 reads, so nothing in it has to start at zero.
static __device__ __align__(256) uint64_t g_digest_scratch[3 * kDigestBlocks];

cudaError_t digest_scratch_address(uint64_t** p, size_t* words) {
    *words = 3 * kDigestBlocks;
    return cudaGetSymbolAddress(reinterpret_cast<void**>(p), g_digest_scratch);
}

cudaError_t launch_digest(const uint64_t* obs, const uint8_t* done, const int32_t* rew, DigestSpan ow, DigestSpan ev,
                          DigestSpan ag, uint32_t ring, uint64_t first, uint32_t n_steps, uint64_t* scratch,
                          uint32_t n_part, const uint32_t* err, uint64_t* out, int64_t* agent_rew, cudaStream_t st) {
    digest_partial_kernel<<<n_part, 256, 0, st>>>(obs, done, rew, ow, ev, ag, ring, first, n_steps, scratch);
    digest_final_kernel<<<1, 256, 0, st>>>(scratch, n_part, err, out);
    if (agent_rew && ag.count)
        agent_reward_kernel<<<(uint32_t)std::min<uint64_t>((ag.count + 255) / 256, 1024), 256, 0, st>>>(
            rew, ag, ring, first, n_steps, agent_rew);
    return cudaGetLastError();
}

// The device step counter moves on once the launches of an enqueue are in.
__global__ void advance_kernel(uint64_t* clock, uint32_t n) { *clock += n; }

cudaError_t launch_advance(uint64_t* clock, uint32_t n, cudaStream_t st) {
    advance_kernel<<<1, 1, 0, st>>>(clock, n);
    return cudaGetLastError();
}

// The step kernel families live in their own translation units.
#define HASE_FAMILY_DECL(f)                                                                                   \
    cudaError_t opt_in_f##f(int optin);                                                                       \
    cudaError_t launch_f##f(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem,        \
                            cudaStream_t st);                                                                 \
    cudaError_t launch_stream_f##f(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem, \
                                   cudaStream_t st);
HASE_FAMILY_DECL(0)
HASE_FAMILY_DECL(1)
HASE_FAMILY_DECL(2)
HASE_FAMILY_DECL(3)
HASE_FAMILY_DECL(4)
HASE_FAMILY_DECL(5)
HASE_FAMILY_DECL(6)
HASE_FAMILY_DECL(7)
HASE_FAMILY_DECL(8)
HASE_FAMILY_DECL(9)
HASE_FAMILY_DECL(10)
HASE_FAMILY_DECL(11)
HASE_FAMILY_DECL(12)
HASE_FAMILY_DECL(13)
HASE_FAMILY_DECL(14)
HASE_FAMILY_DECL(15)
HASE_FAMILY_DECL(16)
#undef HASE_FAMILY_DECL

// Opt in, once per device and outside any capture, to all the dynamic shared
// memory a block may have beside each kernel's static share.  One attribute
// per kernel serves every handle (a per-handle value would cap the others'
// launches).
cudaError_t prepare_step(uint32_t smem) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;  // handles may be created from several threads
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if ((int)smem + 8 * 1024 > optin) return cudaErrorInvalidValue;
    cudaError_t (*opt[])(int) = {opt_in_f0, opt_in_f1, opt_in_f2,  opt_in_f3,  opt_in_f4,  opt_in_f5, opt_in_f6,
                                 opt_in_f7, opt_in_f8, opt_in_f9, opt_in_f10, opt_in_f11, opt_in_f12,
                                 opt_in_f13, opt_in_f14, opt_in_f15, opt_in_f16};
    for (auto f : opt)
        if ((e = f(optin)) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
    return cudaSuccess;
}

// One launch of the groups of one kernel family (stream: its streaming form).
cudaError_t launch_step(int family, bool stream, const StepParams& p, uint32_t n_groups, uint32_t threads,
                        uint32_t smem, cudaStream_t st) {
    if (n_groups == 0 || p.n_steps == 0) return cudaSuccess;
    if (stream) {
        switch (family) {
            case 1: return launch_stream_f1(p, n_groups, threads, smem, st);
            case 2: return launch_stream_f2(p, n_groups, threads, smem, st);
            case 3: return launch_stream_f3(p, n_groups, threads, smem, st);
            case 4: return launch_stream_f4(p, n_groups, threads, smem, st);
            case 5: return launch_stream_f5(p, n_groups, threads, smem, st);
            case 6: return launch_stream_f6(p, n_groups, threads, smem, st);
            case 7: return launch_stream_f7(p, n_groups, threads, smem, st);
            case 8: return launch_stream_f8(p, n_groups, threads, smem, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (family) {
        case 0: return launch_f0(p, n_groups, threads, smem, st);
        case 1: return launch_f1(p, n_groups, threads, smem, st);
        case 2: return launch_f2(p, n_groups, threads, smem, st);
        case 3: return launch_f3(p, n_groups, threads, smem, st);
        case 4: return launch_f4(p, n_groups, threads, smem, st);
        case 5: return launch_f5(p, n_groups, threads, smem, st);
        case 6: return launch_f6(p, n_groups, threads, smem, st);
        case 7: return launch_f7(p, n_groups, threads, smem, st);
        case 8: return launch_f8(p, n_groups, threads, smem, st);
        case 9: return launch_f9(p, n_groups, threads, smem, st);
        case 10: return launch_f10(p, n_groups, threads, smem, st);
        case 11: return launch_f11(p, n_groups, threads, smem, st);
        case 12: return launch_f12(p, n_groups, threads, smem, st);
        case 13: return launch_f13(p, n_groups, threads, smem, st);
        case 14: return launch_f14(p, n_groups, threads, smem, st);
        case 15: return launch_f15(p, n_groups, threads, smem, st);
        case 16: return launch_f16(p, n_groups, threads, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hase
