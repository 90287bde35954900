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
//                   The sequential part (positions) is decoupled from the
//                   bulk of the arithmetic and memory traffic, which is
//                   parallel over steps.
#include <cuda_runtime.h>

#include <algorithm>

#include "hase_internal.cuh"

namespace hase {

// --------------------------------------------------------------------------
// Small helpers.
// --------------------------------------------------------------------------

// floor(u * n / 2^32)
__device__ __forceinline__ uint32_t mulhi_n(uint32_t u, uint32_t n) { return __umulhi(u, n); }

// D consecutive bits (mask) of a padded row of rw words starting at bit s.
__device__ __forceinline__ uint32_t row_bits(const uint64_t* row, int rw, int s, uint32_t mask) {
    if (rw == 1) return (uint32_t)(row[0] >> s) & mask;
    const uint64_t lo = row[0], hi = row[1];
    uint64_t v;
    if (s >= 64)
        v = hi >> (s - 64);
    else if (s == 0)
        v = lo;
    else
        v = (lo >> s) | (hi << (64 - s));
    return (uint32_t)v & mask;
}

// OR a short bit string v (at most 9 bits) into the two-word plane (lo, hi)
// at bit sh.
__device__ __forceinline__ void or_bits(uint64_t& lo, uint64_t& hi, uint64_t v, int sh) {
    if (sh < 64) {
        lo |= v << sh;
        if (sh > 55) hi |= v >> (64 - sh);
    } else {
        hi |= v << (sh - 64);
    }
}

__device__ __forceinline__ void set_bit(uint64_t& lo, uint64_t& hi, int bit) {
    if (bit < 64)
        lo |= 1ull << bit;
    else
        hi |= 1ull << (bit - 64);
}

// packed-cell displacement of action a (x | y << 6): 1 N y-1, 2 S y+1,
// 3 E x+1, 4 W x-1, 0 stay
__device__ __forceinline__ int delta_of(uint32_t a) {
    return a == 1u ? -64 : a == 2u ? 64 : a == 3u ? 1 : a == 4u ? -1 : 0;
}

// Obstacle plane (plane 0) of a window of radius r centred on (x, y) from
// padded rows (rows point at padded row 0 of the env).
__device__ __forceinline__ void obstacle_plane(const uint64_t* rows, int rw, int x, int y, int r,
                                               uint64_t& lo, uint64_t& hi) {
    const int D = 2 * r + 1;
    const uint32_t mask = (1u << D) - 1u;
    const int s = x - r + kPad;
    const uint64_t* row = rows + (y - r + kPad) * rw;
    lo = hi = 0;
    for (int dy = 0; dy < D; ++dy) or_bits(lo, hi, row_bits(row + dy * rw, rw, s, mask), dy * D);
}

// Ally / opponent planes of agent a from the packed positions P[0..A)
// (pairwise; used for small groups and by the step -1 observation).
__device__ __forceinline__ void team_planes_pairwise(int x, int y, int r, int a, int A, int ns,
                                                     const uint16_t* P, uint64_t& al, uint64_t& ah,
                                                     uint64_t& ol, uint64_t& oh) {
    const int D = 2 * r + 1;
    const bool a_seek = a < ns;
    al = ah = ol = oh = 0;
    for (int b = 0; b < A; ++b) {
        if (b == a) continue;
        const uint32_t q = P[b];
        const int dx = (int)px(q) - x + r;
        const int dy = (int)py(q) - y + r;
        if ((unsigned)dx < (unsigned)D && (unsigned)dy < (unsigned)D) {
            const int bit = dy * D + dx;
            if ((b < ns) == a_seek)
                set_bit(al, ah, bit);
            else
                set_bit(ol, oh, bit);
        }
    }
}

// --------------------------------------------------------------------------
// a0: generation.  One warp per env.
// --------------------------------------------------------------------------
__global__ void gen_kernel(const EnvRT* __restrict__ env, const uint32_t* __restrict__ thr,
                           uint32_t n_envs, uint32_t key0, uint32_t key1, uint16_t* __restrict__ pos,
                           uint16_t* __restrict__ start, uint64_t* __restrict__ rows,
                           uint32_t* __restrict__ err) {
    const uint32_t e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (e >= n_envs) return;
    const EnvRT E = env[e];
    const uint32_t density_thr = thr[e];
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
    const int ai = (E.obs_teams == kObsHiders) ? a - ns : a;
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

// --------------------------------------------------------------------------
// a1-a9 fused over n_steps steps.
// --------------------------------------------------------------------------
struct SlotRec {
    uint32_t obs_rel;  // first obs word of this agent inside a slot, ~0u if it emits none
    uint32_t rew_rel;  // reward / action index inside a slot
    uint32_t unp_rel;  // first unpacked byte inside a slot
    uint16_t p0;       // pristine start cell (CTA packing x | y << sh)
    uint8_t env;       // env index inside the group
    uint8_t agent;     // agent index inside its env
};

struct CtaShared {
    EnvRT env[kMaxGroupEnvs];
    uint32_t gidx[kMaxGroupEnvs];  // handle env index (done byte, counters)
    GroupPlan plan;
    SlotRec slot[kMaxGroupSlots];
    uint16_t p0[kMaxGroupSlots];  // pristine start cells (CTA packing)
    uint2 key[kMaxGroupSlots];     // Philox action counter words (agent, env id)
    uint8_t team_list[2][kMaxGroupSlots];
    uint32_t team_n[2];
};

__device__ __forceinline__ uint32_t to_cta(uint32_t p6, uint32_t sh) { return (p6 & 63u) | ((p6 >> 6) << sh); }
__device__ __forceinline__ uint32_t to_hbm(uint32_t p, uint32_t sh) {
    return (p & ((1u << sh) - 1u)) | ((p >> sh) << 6);
}

// action byte of (step k, slot s) in an action buffer of [kc/4][slots] words
__device__ __forceinline__ uint32_t act_index(uint32_t k, uint32_t s, uint32_t nsl) {
    return ((k >> 2) * nsl + s) * 4 + (k & 3);
}

// Context of one chunk's emission.
struct EmitCtx {
    const uint16_t* T;      // trajectory [kc][slots]
    const uint8_t* act;     // action buffer of the chunk
    const uint64_t* rows;   // padded obstacle rows
    const uint64_t* tbl;    // obstacle-window tables
    uint32_t len;           // steps in the chunk
    uint32_t base_slot;     // ring slot of the chunk's first step
    int worker, n_workers;  // this thread among the emission threads
};

// ---------------------------------------------------------------------------
// Segment emission (a5, a6, a9): one thread handles all agents of one
// (step, env) with the positions in registers.  For every ordered pair
// (a, b) it tests b against a's window (radius of a's team); the bit goes to
// a's plane of b's team.  When a is a seeker and b a hider the same test is
// the reward's "seen" test (seeker radius).  The agent count A (<= 16) and
// the seeker count are runtime values shared by the group; the loops are
// unrolled to 16 and skip past A (warp-uniform).  NW = 32-bit words per
// plane: 2 when every window fits 64 bits, 3 with radius 4.
// ---------------------------------------------------------------------------
template <int NW>
struct Plane {
    uint64_t lo;
    uint32_t hi;  // bits 64.. (NW == 3)
};

template <int NW>
__device__ __forceinline__ void plane_or(Plane<NW>& pl, bool in, uint32_t bit) {
    if constexpr (NW == 2) {
        pl.lo |= ((uint64_t)in) << (bit & 63u);  // bit < 64 whenever in
    } else {
        pl.lo |= ((uint64_t)(in && bit < 64u)) << (bit & 63u);
        pl.hi |= (in && bit >= 64u) ? (1u << ((bit - 64u) & 31u)) : 0u;
    }
}

// Lane-per-agent emission.  The lanes of one warp are cut into segments of
// A lanes (A = agents per env, uniform in the group); a segment is one
// (step, env) and lane a of it is agent a.  Every lane loads the env's A
// positions (the same shared-memory words within a segment: broadcast),
// tests the other agents against its own window, and the reward's "seen"
// test is combined across the segment with warp ballots.
template <int NW>
__device__ __forceinline__ void emit_chunk(const StepParams& P, const CtaShared& H, const EmitCtx& C,
                                           int ew, int M, int lane) {
    constexpr int AM = kMaxAgents;
    const GroupPlan& L = H.plan;
    const uint32_t nsl = L.n_slots, ne = L.n_envs;
    const EnvRT& E0 = H.env[0];
    const int A = E0.n_agents, ns = E0.n_seekers;  // uniform in the group
    const int segs = 32 / A;
    const int seg = lane / A, a = lane - seg * A;
    const bool seg_lane = seg < segs;
    const uint32_t segmask = ((A == 32) ? 0xffffffffu : ((1u << A) - 1u)) << (seg_lane ? seg * A : 0);
    const bool ta = a >= ns;
    const int R = ta ? E0.r_hide : E0.r_seek;
    const int D = 2 * R + 1;
    const uint32_t twoR = (uint32_t)(2 * R);
    const int rs = E0.r_seek;
    const bool emits = team_emits(E0, ta ? 1 : 0);
    const int ai = (E0.obs_teams == kObsHiders) ? a - ns : a;
    const int W64 = E0.wpp;
    const bool use_table = L.flags & kUseTable;
    const uint32_t n_items = C.len * ne;
    const uint32_t step_items = (uint32_t)(M * segs);
    // this lane's first item and the stride of its (step, env) counters
    uint32_t item = (uint32_t)(ew * segs + seg);
    uint32_t k = item / ne, e = item % ne;
    const uint32_t dk = step_items / ne, de = step_items % ne;
    for (uint32_t base = (uint32_t)(ew * segs); base < n_items; base += step_items) {
        const bool valid = seg_lane && item < n_items;
        const uint32_t kk = valid ? k : 0u, ee = valid ? e : 0u;
        const int first = L.first_slot[ee];
        const uint32_t sh = cell_shift(H.env[ee]), xmask = (1u << sh) - 1u;
        const uint16_t* Tk = C.T + kk * nsl + first;
        const bool done = (Tk[0] & kDoneBit) != 0u;
        int x[AM], y[AM];
        uint32_t myseen = 0;  // seeker lanes: hiders b seen by this seeker
        if (done) {
            // the reward's "seen" test on the pre-reset positions
            const uint32_t pa = Tk[a] & 0x0fffu;
            const int xa = (int)(pa & xmask), ya = (int)(pa >> sh);
#pragma unroll
            for (int b = 0; b < AM; ++b) {
                if (b >= A) break;
                const uint32_t v = Tk[b] & 0x0fffu;
                const int dx = abs((int)(v & xmask) - xa), dy = abs((int)(v >> sh) - ya);
                if (!ta && b >= ns) myseen |= (uint32_t)(max(dx, dy) <= rs) << b;
            }
#pragma unroll
            for (int b = 0; b < AM; ++b) {
                if (b >= A) break;
                const uint32_t p = H.slot[first + b].p0;
                x[b] = (int)(p & xmask);
                y[b] = (int)(p >> sh);
            }
        } else {
#pragma unroll
            for (int b = 0; b < AM; ++b) {
                if (b >= A) break;
                const uint32_t v = Tk[b];
                x[b] = (int)(v & xmask);
                y[b] = (int)((v & 0x0fffu) >> sh);
            }
        }
        const uint32_t po = done ? (uint32_t)H.slot[first + a].p0 : (Tk[a] & 0x0fffu);
        const int xo = (int)(po & xmask), yo = (int)(po >> sh);
        const int xra = xo - R, yra = yo - R;
        Plane<NW> ps, ph;  // bits of seekers / hiders in this agent's window
        ps.lo = ph.lo = 0;
        ps.hi = ph.hi = 0;
#pragma unroll
        for (int b = 0; b < AM; ++b) {
            if (b >= A) break;
            const uint32_t dx = (uint32_t)(x[b] - xra), dy = (uint32_t)(y[b] - yra);
            const bool in = (max(dx, dy) <= twoR) && b != a;
            const uint32_t bit = dy * (uint32_t)D + dx;
            if (b < ns) {
                plane_or<NW>(ps, in, bit);
            } else {
                plane_or<NW>(ph, in, bit);
                if (!ta && !done) myseen |= (uint32_t)in << b;  // seeker window: radius rs
            }
        }
        // a6: a hider is seen when some seeker of its segment sees it
        uint32_t n_seen = 0;
        bool me_seen = false;
#pragma unroll
        for (int h = 0; h < AM; ++h) {
            if (h >= A) break;
            if (h < ns) continue;
            const uint32_t bal = __ballot_sync(0xffffffffu, valid && ((myseen >> h) & 1u));
            const bool any = (bal & segmask) != 0u;
            n_seen += any ? 1u : 0u;
            me_seen |= any && h == a;
        }
        if (valid) {
            uint32_t sl = C.base_slot + kk;
            if (sl >= P.ring) sl -= P.ring;
            const EnvRT& E = H.env[ee];
            P.rew[(uint64_t)sl * P.agents + E.agent_off + a] = ta ? -(int32_t)me_seen : (int32_t)n_seen;
            if (a == 0) P.done[(uint64_t)sl * P.n_envs + H.gidx[ee]] = done ? 3u : 0u;
            if (P.act_out)
                P.act_out[(uint64_t)sl * P.agents + E.agent_off + a] = C.act[act_index(kk, (uint32_t)(first + a), nsl)];
            if (emits) {
                // a5 obstacle plane
                Plane<NW> o0;
                if (use_table) {
                    const uint32_t W = words_of_radius(R);
                    const uint64_t* tw = C.tbl + L.tbl_off[ee][ta ? 1 : 0] + (uint32_t)(yo * E.side + xo) * W;
                    o0.lo = tw[0];
                    o0.hi = (NW == 3 && W == 2) ? (uint32_t)tw[1] : 0u;
                } else {
                    uint64_t lo, hi;
                    obstacle_plane(C.rows + L.rows_off[ee], E.rw, xo, yo, R, lo, hi);
                    o0.lo = lo;
                    o0.hi = (uint32_t)hi;
                }
                const Plane<NW>& al = ta ? ph : ps;
                const Plane<NW>& opp = ta ? ps : ph;
                uint64_t* o = P.obs + (uint64_t)sl * P.obs_words + E.obs_off + (uint32_t)ai * 3u * (uint32_t)W64;
                if (W64 == 1) {
                    o[0] = o0.lo;
                    o[1] = al.lo;
                    o[2] = opp.lo;
                } else {
                    o[0] = o0.lo;
                    o[1] = (uint64_t)o0.hi;
                    o[2] = al.lo;
                    o[3] = (uint64_t)al.hi;
                    o[4] = opp.lo;
                    o[5] = (uint64_t)opp.hi;
                }
                if (P.unp) {
                    uint8_t* u = P.unp + (uint64_t)sl * P.unp_bytes + H.slot[first + a].unp_rel;
                    const int DD = D * D;
                    for (int q = 0; q < DD; ++q) {
                        const uint32_t b0 = q < 64 ? (uint32_t)(o0.lo >> q) : (o0.hi >> (q - 64));
                        const uint32_t b1 = q < 64 ? (uint32_t)(al.lo >> q) : (al.hi >> (q - 64));
                        const uint32_t b2 = q < 64 ? (uint32_t)(opp.lo >> q) : (opp.hi >> (q - 64));
                        u[q] = (uint8_t)(b0 & 1u);
                        u[DD + q] = (uint8_t)(b1 & 1u);
                        u[2 * DD + q] = (uint8_t)(b2 & 1u);
                    }
                }
            }
        }
        item += step_items;
        e += de;
        k += dk;
        if (e >= ne) {
            e -= ne;
            ++k;
        }
    }
}

// Reward "seen" mask of a segment whose episode ended in this step: the test
// runs on the pre-reset positions (one step in cap takes this path).
__device__ __forceinline__ uint32_t seen_pre_reset(const uint16_t* Tk, int A, int ns, int rs, uint32_t sh) {
    const uint32_t xmask = (1u << sh) - 1u;
    uint32_t seen = 0;
    for (int h = ns; h < A; ++h) {
        const uint32_t vh = Tk[h] & 0x0fffu;
        const int hx = (int)(vh & xmask), hy = (int)(vh >> sh);
        for (int s = 0; s < ns; ++s) {
            const uint32_t vs = Tk[s] & 0x0fffu;
            const int dx = abs((int)(vs & xmask) - hx), dy = abs((int)(vs >> sh) - hy);
            if (max(dx, dy) <= rs) seen |= 1u << h;
        }
    }
    return seen;
}

// PTX shifts clamp the amount at the register width: 1 << n is 0 for n >= 32.
__device__ __forceinline__ uint32_t shl_clamp(uint32_t v, uint32_t n) {
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(n));
    return r;
}

// Byte q of w (q a compile-time constant after unrolling).
__device__ __forceinline__ uint32_t byte_of(uint32_t w, int q) { return q == 3 ? w >> 24 : (w >> (8 * q)) & 0xffu; }

// Segment emission with compile-time A (seekers NS = ceil(A/2)) and windows
// of at most 64 bits (radius <= 3): one thread handles one (step, env), and
// the window tests run four agents at a time on bytes packed in a word.
//   X4 / Y4: byte b & 3 of word b >> 2 holds agent b's x / y;
//   P4:      the same byte holds (y D + x) mod 256 for the team's D.
// For observer a with radius R, adding (0x80 + R - x_a) to every byte of X4
// gives dx + R + 0x80 in [0x41, 0xc3] (no carry leaves a byte); b lies in the
// window iff both that byte and its y twin are in [0x80, 0x80 + 2R].  The
// window bit (dy + R) D + (dx + R) equals P4_b - P4_a + R D + R mod 256 for
// agents inside the window; a byte-wise add (carries kept inside each byte)
// forms it, and bit 7 is set in the bytes of agents outside, which makes the
// shifts below yield 0 for them (PTX clamps shift amounts at 32).  Observer a
// meets itself at the window centre of its ally plane, cleared afterwards
// (no other agent shares its cell).
// Loop-invariant inputs of one team's observers in one (step, env).
struct TeamCtx {
    const uint16_t* src;  // observed positions (CTA packing), shared memory
    const uint64_t* tbl;  // obstacle-window table of the team radius, shared memory
    const uint64_t* rows; // obstacle rows of the env (used without a table)
    uint64_t* ob;         // obs words of the env's first emitting agent, global
    uint8_t* unp;         // unpacked bytes of the slot (null unless exported)
    const SlotRec* slot;  // slot records of the env's agents
    uint32_t sh, xmask, side, rw;
    int ai0;              // emitting index of agent 0 of the team base
    bool emits, use_table;
};

template <int A, bool TA>
__device__ __forceinline__ void emit_team_fast(const TeamCtx& T, uint32_t R, const uint32_t (&X4)[(A + 3) / 4],
                                               const uint32_t (&Y4)[(A + 3) / 4], const uint32_t (&P4)[(A + 3) / 4],
                                               uint32_t (&seenf)[(A + 3) / 4]) {
    constexpr int NS = (A + 1) / 2, NW = (A + 3) / 4;
    const uint32_t D = 2u * R + 1u;
    const uint32_t KR = (0x80u + R) * 0x01010101u;
    const uint32_t C2 = (0x7fu - 2u * R) * 0x01010101u;
    const uint32_t KP = R * D + R;
    const uint32_t centre = ~shl_clamp(1u, KP), centre_hi = ~shl_clamp(1u, KP - 32u);
#pragma unroll 1
    for (int a = TA ? NS : 0; a < (TA ? A : NS); ++a) {
        const uint32_t v = T.src[a] & 0x0fffu;
        const uint32_t xa = v & T.xmask, ya = v >> T.sh;
        const uint32_t Kx = KR - xa * 0x01010101u, Ky = KR - ya * 0x01010101u;
        const uint32_t Kp = ((KP - (ya * D + xa)) & 0xffu) * 0x01010101u;
        const uint32_t Kp7 = Kp & 0x7f7f7f7fu;
        uint32_t al0 = 0, al1 = 0, op0 = 0, op1 = 0;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const uint32_t vx = X4[j] + Kx, vy = Y4[j] + Ky;
            const uint32_t wx = (vx & 0x7f7f7f7fu) + C2, wy = (vy & 0x7f7f7f7fu) + C2;
            const uint32_t fail = (~vx | wx | ~vy | wy) & 0x80808080u;
            if (!TA) {
                uint32_t hid = 0;  // bytes of hiders in this word
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (4 * j + q >= NS && 4 * j + q < A) hid |= 0x80u << (8 * q);
                seenf[j] |= ~fail & hid;
            }
            const uint32_t n4 = (((P4[j] & 0x7f7f7f7fu) + Kp7) ^ ((P4[j] ^ Kp) & 0x80808080u)) | fail;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int b = 4 * j + q;
                if (b >= A) continue;
                const uint32_t n = __byte_perm(n4, 0u, 0x4440u | (uint32_t)q);
                const uint32_t m0 = shl_clamp(1u, n), m1 = shl_clamp(1u, n - 32u);
                if ((b >= NS) == TA) {
                    al0 |= m0;
                    al1 |= m1;
                } else {
                    op0 |= m0;
                    op1 |= m1;
                }
            }
        }
        if (!T.emits) continue;
        al0 &= centre;
        al1 &= centre_hi;
        // a5 obstacle plane and the agent's three words
        uint64_t o0;
        if (T.use_table) {
            o0 = T.tbl[ya * T.side + xa];
        } else {
            uint64_t unused;
            obstacle_plane(T.rows, (int)T.rw, (int)xa, (int)ya, (int)R, o0, unused);
        }
        const uint64_t al = (uint64_t)al0 | ((uint64_t)al1 << 32);
        const uint64_t op = (uint64_t)op0 | ((uint64_t)op1 << 32);
        uint64_t* o = T.ob + 3 * (a - T.ai0);
        o[0] = o0;
        o[1] = al;
        o[2] = op;
        if (T.unp) {
            uint8_t* u = T.unp + T.slot[a].unp_rel;
            const uint32_t DD = D * D;
            for (uint32_t q = 0; q < DD; ++q) {
                u[q] = (uint8_t)((o0 >> q) & 1u);
                u[DD + q] = (uint8_t)((al >> q) & 1u);
                u[2 * DD + q] = (uint8_t)((op >> q) & 1u);
            }
        }
    }
}

template <int A>
__device__ __forceinline__ void emit_segment_fast(const StepParams& P, const CtaShared& H, const EmitCtx& C,
                                                  uint32_t k, uint32_t e) {
    constexpr int NS = (A + 1) / 2, NW = (A + 3) / 4;
    const GroupPlan& L = H.plan;
    const EnvRT E = H.env[e];  // a register copy: the stores below cannot alias it
    const uint32_t nsl = L.n_slots;
    const uint32_t sh = cell_shift(E), xmask = (1u << sh) - 1u;
    const int first = L.first_slot[e];
    const uint16_t* Tk = C.T + k * nsl + first;
    const bool done = (Tk[0] & kDoneBit) != 0u;
    const uint16_t* src = done ? (H.p0 + first) : Tk;  // observed positions
    const uint32_t rs = E.r_seek, rh = E.r_hide, Ds = 2u * rs + 1u, Dh = 2u * rh + 1u;
    uint32_t X4[NW], Y4[NW], Ps[NW], Ph[NW], seenf[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) X4[j] = Y4[j] = Ps[j] = Ph[j] = seenf[j] = 0u;
#pragma unroll
    for (int b = 0; b < A; ++b) {
        const uint32_t v = src[b] & 0x0fffu;
        const uint32_t x = v & xmask, y = v >> sh;
        const int j = b >> 2, s8 = 8 * (b & 3);
        X4[j] |= x << s8;
        Y4[j] |= y << s8;
        Ps[j] |= ((y * Ds + x) & 0xffu) << s8;
        Ph[j] |= ((y * Dh + x) & 0xffu) << s8;
    }
    uint32_t sl = C.base_slot + k;
    if (sl >= P.ring) sl -= P.ring;
    const bool emit_s = team_emits(E, 0), emit_h = team_emits(E, 1);
    TeamCtx T;
    T.src = src;
    T.rows = C.rows + L.rows_off[e];
    T.ob = P.obs + (uint64_t)sl * P.obs_words + E.obs_off;
    T.unp = P.unp ? P.unp + (uint64_t)sl * P.unp_bytes : nullptr;
    T.slot = H.slot + first;
    T.sh = sh;
    T.xmask = xmask;
    T.side = E.side;
    T.rw = E.rw;
    T.use_table = L.flags & kUseTable;
    T.tbl = C.tbl + L.tbl_off[e][0];
    T.ai0 = 0;
    T.emits = emit_s;
    emit_team_fast<A, false>(T, rs, X4, Y4, Ps, seenf);
    if (A > 1 && emit_h) {
        T.tbl = C.tbl + L.tbl_off[e][1];
        T.ai0 = emit_s ? 0 : NS;
        T.emits = true;
        emit_team_fast<A, true>(T, rh, X4, Y4, Ph, seenf);
    }
    uint32_t seen = 0;
    if (done) {
        seen = seen_pre_reset(Tk, A, NS, (int)rs, sh);
    } else {
#pragma unroll
        for (int b = NS; b < A; ++b) seen |= ((seenf[b >> 2] >> (8 * (b & 3) + 7)) & 1u) << b;
    }
    // a6 rewards, a7 done byte, actions
    const int32_t n_seen = (int32_t)__popc(seen);
    int32_t* rw = P.rew + (uint64_t)sl * P.agents + E.agent_off;
    uint8_t* dn = P.done + (uint64_t)sl * P.n_envs + H.gidx[e];
#pragma unroll
    for (int a = 0; a < A; ++a) rw[a] = a < NS ? n_seen : -(int32_t)((seen >> a) & 1u);
    *dn = done ? 3u : 0u;
    if (P.act_out) {
        uint8_t* ao = P.act_out + (uint64_t)sl * P.agents + E.agent_off;
#pragma unroll
        for (int a = 0; a < A; ++a) ao[a] = C.act[act_index(k, (uint32_t)(first + a), nsl)];
    }
}

template <int A>
__device__ __forceinline__ void emit_segments_fast(const StepParams& P, const CtaShared& H, const EmitCtx& C) {
    const uint32_t ne = H.plan.n_envs;
    const uint32_t total = C.len * ne;
    const uint32_t dk = (uint32_t)C.n_workers / ne, de = (uint32_t)C.n_workers % ne;
    uint32_t k = (uint32_t)C.worker / ne, e = (uint32_t)C.worker % ne;
    for (uint32_t it = (uint32_t)C.worker; it < total; it += (uint32_t)C.n_workers) {
        emit_segment_fast<A>(P, H, C, k, e);
        e += de;
        k += dk;
        if (e >= ne) {
            e -= ne;
            ++k;
        }
    }
}

__device__ __forceinline__ void emit_fast_dispatch(int A, const StepParams& P, const CtaShared& H,
                                                   const EmitCtx& C) {
    switch (A) {
        case 1: emit_segments_fast<1>(P, H, C); break;
        case 2: emit_segments_fast<2>(P, H, C); break;
        case 3: emit_segments_fast<3>(P, H, C); break;
        case 4: emit_segments_fast<4>(P, H, C); break;
        case 5: emit_segments_fast<5>(P, H, C); break;
        case 6: emit_segments_fast<6>(P, H, C); break;
        case 7: emit_segments_fast<7>(P, H, C); break;
        case 8: emit_segments_fast<8>(P, H, C); break;
        case 9: emit_segments_fast<9>(P, H, C); break;
        case 10: emit_segments_fast<10>(P, H, C); break;
        case 11: emit_segments_fast<11>(P, H, C); break;
        case 12: emit_segments_fast<12>(P, H, C); break;
        case 13: emit_segments_fast<13>(P, H, C); break;
        case 14: emit_segments_fast<14>(P, H, C); break;
        case 15: emit_segments_fast<15>(P, H, C); break;
        default: emit_segments_fast<16>(P, H, C); break;
    }
}

// Per-cell shared state of the dynamics: a claim word (byte a-1 holds the
// lane claiming the cell through action a, 1 N 2 S 3 E 4 W; 0xff = none)
// and a state byte (bits 1..4: action a leads onto a free cell of the grid;
// bit 7: occupied).
constexpr uint32_t kNoClaims = 0xffffffffu;

template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) step_kernel(const StepParams P) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ CtaShared H;
    const Group G = P.groups[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    const int ne = G.n_envs, nsl = G.n_slots;
    const int n_dyn = (int)P.n_dyn;  // dynamics warps of the launch (>= the group's)
    const int M = (int)P.emit_warps;
    const uint32_t kc = P.kc;

    if (tid == 0) {
        int slot = 0;
        H.team_n[0] = H.team_n[1] = 0;
        for (int i = 0; i < ne; ++i) {
            const uint32_t g = P.env_list[G.list_first + i];
            const EnvRT E = P.env[g];
            H.env[i] = E;
            H.gidx[i] = g;
            uint32_t urel = E.unp_off;
            for (int a = 0; a < E.n_agents; ++a) {
                const int t = a < E.n_seekers ? 0 : 1;
                SlotRec r;
                r.env = (uint8_t)i;
                r.agent = (uint8_t)a;
                r.rew_rel = E.agent_off + a;
                r.p0 = 0;
                r.unp_rel = urel;
                if (team_emits(E, t)) {
                    const int ai = (E.obs_teams == kObsHiders) ? a - E.n_seekers : a;
                    r.obs_rel = E.obs_off + (uint32_t)ai * 3u * E.wpp;
                    const int rr = team_radius(E, t);
                    urel += 3u * (2 * rr + 1) * (2 * rr + 1);
                } else {
                    r.obs_rel = ~0u;
                }
                H.slot[slot] = r;
                H.team_list[t][H.team_n[t]++] = (uint8_t)slot;
                ++slot;
            }
        }
        plan_group(H.env, ne, (int)kc, G.flags, H.plan);
    }
    __syncthreads();
    const GroupPlan& L = H.plan;
    const bool use_table = L.flags & kUseTable;
    uint8_t* s_act = sm + L.act;                     // [3][act_words] (bytes of 4 steps)
    uint16_t* s_traj = (uint16_t*)(sm + L.traj);     // [2][kc][slots]
    uint64_t* s_rows = (uint64_t*)(sm + L.rows);
    uint32_t* s_claim = (uint32_t*)(sm + L.claim);   // per cell
    uint8_t* s_state = sm + L.state;                 // per cell
    uint64_t* s_tbl = (uint64_t*)(sm + L.tbl);
    const uint32_t act_bytes = L.act_words * 4;

    // stage the pristine template: padded rows and start cells
    for (int i = 0; i < ne; ++i) {
        const EnvRT& E = H.env[i];
        const uint32_t n = (uint32_t)(E.side + 2 * kPad) * E.rw;
        for (uint32_t j = tid; j < n; j += nthreads) s_rows[L.rows_off[i] + j] = P.rows[E.rows_off + j];
    }
    for (int sidx = tid; sidx < nsl; sidx += nthreads) {
        const SlotRec& r = H.slot[sidx];
        const EnvRT& E = H.env[r.env];
        H.slot[sidx].p0 = (uint16_t)to_cta(P.start[E.agent_off + r.agent], cell_shift(E));
        H.p0[sidx] = H.slot[sidx].p0;
        H.key[sidx] = make_uint2(r.agent, E.env_id);
    }
    __syncthreads();
    // cell state and claims, obstacle-window tables (plane 0 of every cell
    // for each emitting radius)
    for (int i = 0; i < ne; ++i) {
        const EnvRT& E = H.env[i];
        const int S = E.side, rw = E.rw;
        const uint32_t sh = cell_shift(E);
        const uint64_t* Rw = s_rows + L.rows_off[i];
        for (int c = tid; c < (S << sh); c += nthreads) {
            const int x = c & ((1 << sh) - 1), y = c >> sh;
            uint32_t m = 0;
            if (x < S) {
                auto freecell = [&](int xx, int yy) -> uint32_t {
                    const int b = xx + kPad;
                    return (uint32_t)(((Rw[(yy + kPad) * rw + (b >> 6)] >> (b & 63)) & 1ull) ^ 1ull);
                };
                m = (freecell(x, y - 1) << 1) | (freecell(x, y + 1) << 2) | (freecell(x + 1, y) << 3) |
                    (freecell(x - 1, y) << 4);
            }
            s_state[L.cell_off[i] + c] = (uint8_t)m;
            s_claim[L.cell_off[i] + c] = kNoClaims;
        }
        if (use_table) {
            for (int t = 0; t < 2; ++t) {
                if (L.tbl_off[i][t] == ~0u) continue;
                if (t == 1 && L.tbl_off[i][1] == L.tbl_off[i][0]) continue;
                const int r = team_radius(E, t);
                const uint32_t W = words_of_radius(r);
                uint64_t* Tb = s_tbl + L.tbl_off[i][t];
                for (int c = tid; c < S * S; c += nthreads) {
                    uint64_t lo, hi;
                    obstacle_plane(Rw, rw, c % S, c / S, r, lo, hi);
                    Tb[c * W] = lo;
                    if (W == 2) Tb[c * W + 1] = hi;
                }
            }
        }
    }
    __syncthreads();
    // occupancy bits of the current cells
    for (int sidx = tid; sidx < nsl; sidx += nthreads) {
        const SlotRec& r = H.slot[sidx];
        const EnvRT& E = H.env[r.env];
        const uint32_t p = to_cta(P.pos[E.agent_off + r.agent], cell_shift(E));
        s_state[L.cell_off[r.env] + p] |= (uint8_t)kOccBit;
    }

    const uint32_t n_chunks = (P.n_steps + kc - 1) / kc;
    const uint64_t T0 = *P.clock + P.t0;  // global step index of the launch's first step

    // a1: Philox actions of chunk c into buffer c % 3.  One Philox block
    // (counter word 0 = step >> 2) serves four consecutive steps of one
    // agent slot; work items are (block, slot) pairs, slot fastest, and a
    // thread draws two items at a time (independent rounds interleave).
    // When the chunk starts on a block boundary a block fills one u32 word
    // of the buffer (byte k & 3 of word (k >> 2) nsl + s is step k of slot s).
    auto draw_actions = [&](uint32_t c, int worker, int n_workers) {
        const uint64_t ts = T0 + (uint64_t)c * kc;
        const uint32_t len = min(kc, P.n_steps - c * kc);
        const uint64_t b0 = ts >> 2;
        const uint32_t off = (uint32_t)(ts & 3u);
        const uint32_t nblk = (off + len + 3u) >> 2;
        uint8_t* A8 = s_act + (c % 3u) * act_bytes;
        uint32_t* A32 = reinterpret_cast<uint32_t*>(A8);
        const uint32_t ns = (uint32_t)nsl;
        const uint32_t n_items = nblk * ns;
        const uint32_t stride = 2u * (uint32_t)n_workers;
        auto put = [&](uint32_t it, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
            const uint32_t s = it % ns, bi = it / ns;
            const uint32_t w = mulhi_n(c0, 5u) | (mulhi_n(c1, 5u) << 8) | (mulhi_n(c2, 5u) << 16) |
                               (mulhi_n(c3, 5u) << 24);
            if (off == 0u) {
                A32[bi * ns + s] = w;
            } else {
#pragma unroll
                for (uint32_t j = 0; j < 4; ++j) {
                    const uint32_t k = 4u * bi + j - off;  // wraps past len below 0
                    if (k < len) A8[act_index(k, s, ns)] = (uint8_t)(w >> (8u * j));
                }
            }
        };
        for (uint32_t it = (uint32_t)worker; it < n_items; it += stride) {
            const uint32_t it2 = it + (uint32_t)n_workers;
            const bool two = it2 < n_items;
            const uint2 ka = H.key[it % ns], kb = H.key[(two ? it2 : it) % ns];
            uint32_t a0 = (uint32_t)(b0 + it / ns), a1 = ka.x, a2 = ka.y, a3 = 0u;
            uint32_t d0 = (uint32_t)(b0 + (two ? it2 : it) / ns), d1 = kb.x, d2 = kb.y, d3 = 0u;
            philox4x32_10(a0, a1, a2, a3, P.key0, P.key1);
            philox4x32_10(d0, d1, d2, d3, P.key0, P.key1);
            put(it, a0, a1, a2, a3);
            if (two) put(it2, d0, d1, d2, d3);
        }
    };

    if (n_chunks > 0) draw_actions(0, tid, nthreads);
    __syncthreads();

    if (warp < n_dyn) {
        // ================= dynamics warps: a2 a3 a7 a8 =================
        // lane = agent slot; whole envs per warp, lanes in agent order.  A
        // mover claims its target in the byte of its incoming direction;
        // after a __syncwarp it reads the target's claim word and state: it
        // moves iff the target was unoccupied and no lower lane claimed it.
        // Episode ends are known in advance (truncation only), so the reset
        // path is a warp-uniform branch taken once per episode.
        const int d_first = warp < (int)L.n_dyn ? L.dyn_first[warp] : 0;
        const int d_end = warp < (int)L.n_dyn ? L.dyn_first[warp + 1] : 0;
        const int s = d_first + lane;
        const bool live = s < d_end;
        uint32_t p = 0, p0 = 0, nbr_cur = 0, nbr0 = 0, ep_idx = 0, cap = 1, sh = 5;
        uint32_t next_done = 0xffffffffu;  // launch step index of this lane's next episode end
        int env = 0;
        uint8_t* st8 = s_state;
        uint8_t* cl8 = reinterpret_cast<uint8_t*>(s_claim);
        if (live) {
            const SlotRec& r = H.slot[s];
            env = r.env;
            const EnvRT& E = H.env[env];
            sh = cell_shift(E);
            st8 = s_state + L.cell_off[env];
            cl8 = reinterpret_cast<uint8_t*>(s_claim + L.cell_off[env]);
            p = to_cta(P.pos[E.agent_off + r.agent], sh);
            p0 = r.p0;
            nbr_cur = st8[p] & 0x1eu;
            nbr0 = st8[p0] & 0x1eu;
            const EnvState est = P.est[H.gidx[env]];
            ep_idx = est.ep_idx;
            cap = E.cap;
            next_done = cap - 1u - est.ep_t;
        }
        uint32_t warp_next = __reduce_min_sync(0xffffffffu, next_done);
        const uint32_t lane_rep = 0x01010101u * (uint32_t)lane;
        // byte a-1: displacement of action a (1 N, 2 S, 3 E, 4 W) plus 64
        const uint32_t dn = 1u << sh;
        const uint32_t dlut = (64u - dn) | ((64u + dn) << 8) | (65u << 16) | (63u << 24);
        __syncwarp();
        // One step: claim, read, resolve, update.  g: step inside the launch.
        auto step = [&](uint32_t a, uint16_t* Tk, uint32_t g) {
            const uint32_t dd = __byte_perm(dlut, 0, 0x4440u | ((a + 3u) & 3u)) - 64u;
            const uint32_t tgt = p + dd;
            const uint32_t open = (nbr_cur >> a) & 1u;  // inside the grid, no obstacle (a = 0: never)
            if (open) cl8[tgt * 4 + a - 1] = (uint8_t)lane;  // claim the byte of direction a
            __syncwarp();
            uint32_t claims = 0u, tst = kOccBit;         // not open: reads as occupied
            if (open) {
                claims = *reinterpret_cast<const uint32_t*>(cl8 + tgt * 4);
                tst = st8[tgt];
            }
            const uint32_t lower = ~((claims | 0x80808080u) - lane_rep) & 0x80808080u;
            const bool won = ((tst & kOccBit) | lower) == 0u;
            __syncwarp();  // every read of this step is done
            if (open) cl8[tgt * 4 + a - 1] = 0xffu;          // release the claim
            if (won) {
                st8[p] = (uint8_t)nbr_cur;
                st8[tgt] = (uint8_t)(tst | kOccBit);
            }
            p = won ? tgt : p;
            nbr_cur = won ? (tst & 0x1eu) : nbr_cur;
            if (live) *Tk = (uint16_t)(p | (g == next_done ? kDoneBit : 0u));
            if (g == warp_next) {  // some env of this warp ends its episode (a8)
                const bool done = g == next_done;
                __syncwarp();
                if (done) st8[p] = (uint8_t)nbr_cur;
                __syncwarp();
                if (done) {
                    st8[p0] = (uint8_t)(nbr0 | kOccBit);
                    p = p0;
                    nbr_cur = nbr0;
                    next_done += cap;
                    ++ep_idx;
                }
                warp_next = __reduce_min_sync(0xffffffffu, next_done);
            }
            __syncwarp();  // state writes visible to the next step
        };
        for (uint32_t c = 0; c <= n_chunks; ++c) {
            if (c < n_chunks) {
                const uint32_t len = min(kc, P.n_steps - c * kc);
                const uint32_t* A = reinterpret_cast<const uint32_t*>(s_act + (c % 3u) * act_bytes) + s;
                uint16_t* T = s_traj + (c & 1u) * (kc * nsl) + s;
                const uint32_t g0 = c * kc;
                uint32_t k = 0;
                uint32_t aw = live ? A[0] : 0u;
                for (; k + 4 <= len; k += 4) {
                    const uint32_t aw_next = (live && k + 4 < len) ? A[((k + 4) >> 2) * nsl] : 0u;
#pragma unroll
                    for (uint32_t j = 0; j < 4; ++j)
                        step(__byte_perm(aw, 0, 0x4440u + j), T + (k + j) * nsl, g0 + k + j);
                    aw = aw_next;
                }
                for (; k < len; ++k) step(__byte_perm(aw, 0, 0x4440u + (k & 3u)), T + k * nsl, g0 + k);
            }
            __syncthreads();
        }
        // write back the dynamic state
        if (live) {
            const SlotRec& r = H.slot[s];
            const EnvRT& E = H.env[env];
            P.pos[E.agent_off + r.agent] = (uint16_t)to_hbm(p, sh);
            if (r.agent == 0) {
                EnvState est;
                est.ep_t = cap - 1u - (next_done - P.n_steps);
                est.ep_idx = ep_idx;
                P.est[H.gidx[env]] = est;
            }
        }
        return;
    }

    // ================= emission warps: a5 a6 a9 (+ a1 ahead) =================
    const int worker = tid - n_dyn * 32;
    const int n_workers = M * 32;
    const bool wide = H.env[0].wpp == 2;  // the group shares its radii
    // one thread per (step, env) when the seekers are ceil(A/2) and every
    // window fits one word; else one lane per agent
    const bool fast = fast_emission(H.env[0]);
    for (uint32_t c = 0; c <= n_chunks; ++c) {
        if (c >= 1) {
            const uint32_t cp = c - 1;
            EmitCtx C;
            C.len = min(kc, P.n_steps - cp * kc);
            C.T = s_traj + (cp & 1u) * (kc * nsl);
            C.act = s_act + (cp % 3u) * act_bytes;
            C.rows = s_rows;
            C.tbl = s_tbl;
            C.base_slot = (uint32_t)((T0 + (uint64_t)cp * kc) % P.ring);
            C.worker = worker;
            C.n_workers = n_workers;
            if (fast)
                emit_fast_dispatch(H.env[0].n_agents, P, H, C);
            else if (wide)
                emit_chunk<3>(P, H, C, warp - n_dyn, M, lane);
            else
                emit_chunk<2>(P, H, C, warp - n_dyn, M, lane);
        }
        // a1 for chunk c + 1
        if (c + 1 < n_chunks) draw_actions(c + 1, worker, n_workers);
        __syncthreads();
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

// --------------------------------------------------------------------------
// Run digest: order-independent sums (mod 2^64) over the ring slots of the
// last n steps.  Pass 1: every block reduces a grid-stride share of the obs
// words, done bytes and rewards into scratch[block] (three words); pass 2: one
// block adds the partials.  A third kernel gives per-agent reward sums.
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

__global__ void digest_partial_kernel(const uint64_t* obs, const uint8_t* done, const int32_t* rew,
                                      uint64_t obs_words, uint64_t n_envs, uint64_t agents, uint32_t ring,
                                      uint64_t first, uint32_t n_steps, uint64_t* scratch) {
    __shared__ uint64_t red[32];
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t dig = 0, eps = 0, rs = 0;
    if (obs_words) {
        const uint64_t total = (uint64_t)n_steps * obs_words;
        Walk w(i0, obs_words);
        for (uint64_t i = i0; i < total; i += (uint64_t)gridDim.x * blockDim.x, w.next(obs_words)) {
            const uint64_t slot = (first + w.s) % ring;
            dig += splitmix64(obs[slot * obs_words + w.j] ^ i);
        }
    }
    {
        const uint64_t total = (uint64_t)n_steps * n_envs;
        Walk w(i0, n_envs);
        for (uint64_t i = i0; i < total; i += (uint64_t)gridDim.x * blockDim.x, w.next(n_envs))
            eps += done[((first + w.s) % ring) * n_envs + w.j] & 1u;
    }
    {
        const uint64_t total = (uint64_t)n_steps * agents;
        Walk w(i0, agents);
        for (uint64_t i = i0; i < total; i += (uint64_t)gridDim.x * blockDim.x, w.next(agents))
            rs += (uint64_t)(int64_t)rew[((first + w.s) % ring) * agents + w.j];
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

__global__ void agent_reward_kernel(const int32_t* rew, uint64_t agents, uint32_t ring, uint64_t first,
                                    uint32_t n_steps, int64_t* agent_rew) {
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < agents;
         a += (uint64_t)gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (uint32_t k = 0; k < n_steps; ++k) s += rew[((first + k) % ring) * agents + a];
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

cudaError_t launch_digest(const uint64_t* obs, const uint8_t* done, const int32_t* rew, uint64_t obs_words,
                          uint64_t n_envs, uint64_t agents, uint32_t ring, uint64_t first, uint32_t n_steps,
                          uint64_t* scratch, uint32_t n_part, const uint32_t* err, uint64_t* out,
                          int64_t* agent_rew, cudaStream_t st) {
    digest_partial_kernel<<<n_part, 256, 0, st>>>(obs, done, rew, obs_words, n_envs, agents, ring, first, n_steps,
                                                  scratch);
    digest_final_kernel<<<1, 256, 0, st>>>(scratch, n_part, err, out);
    if (agent_rew && agents)
        agent_reward_kernel<<<(uint32_t)std::min<uint64_t>((agents + 255) / 256, 1024), 256, 0, st>>>(
            rew, agents, ring, first, n_steps, agent_rew);
    return cudaGetLastError();
}

// The device step counter moves on once the launches of an enqueue are in.
__global__ void advance_kernel(uint64_t* clock, uint32_t n) { *clock += n; }

cudaError_t launch_advance(uint64_t* clock, uint32_t n, cudaStream_t st) {
    advance_kernel<<<1, 1, 0, st>>>(clock, n);
    return cudaGetLastError();
}

// Opt in, once per device and outside any capture, to all the dynamic shared
// memory a block may have beside the kernel's static share.  One attribute
// serves every handle (a per-handle value would cap the others' launches).
cudaError_t prepare_step(uint32_t smem) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static int done[64] = {0};
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, step_kernel<512, 1>);
    if (e != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if ((int)smem > dyn) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(step_kernel<512, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
    return e;
}

template <int MAXT, int MINB>
static cudaError_t launch_step_t(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem,
                                 cudaStream_t st) {
    step_kernel<MAXT, MINB><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

// One instantiation: every CTA shape (64..512 threads) runs with a cap of
// 128 registers a thread, which is what 512 threads x 1 CTA leaves and also
// what 64 threads x 8 CTAs would; residency is then set by shared memory.
cudaError_t launch_step(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem,
                        cudaStream_t st) {
    if (n_groups == 0 || p.n_steps == 0) return cudaSuccess;
    if (threads <= 512) return launch_step_t<512, 1>(p, n_groups, threads, smem, st);
    return cudaErrorInvalidConfiguration;
}

}  // namespace hase
