// hase_step.cuh -- device code of the fused step kernel (a1-a9), included
// by one translation unit per kernel family (hase_step_f0.cu ..
// hase_step_f16.cu, compiled in parallel) and by hase_kernels.cu for the
// shared helpers.
//
//   step_kernel     a1-a9 fused over K steps.  One CTA owns a group of envs
//                   of one kernel shape (agents, teams, radii, cell packing)
//                   for the whole launch, all dynamic state in shared memory
//                   and registers:
//                     dynamics warps (a2, a3, a7, a8): one lane per agent
//                       slot, whole envs per warp; a mover writes its lane
//                       into the claim byte of its incoming direction in the
//                       target cell and, after __syncwarp, moves iff the
//                       target is free and no lower lane claimed it; the
//                       warp writes each step's cells into the chunk
//                       trajectory;
//                     emission warps (a1, a4-a6, a9), one chunk behind:
//                       one thread per (step, env) builds every agent's
//                       three planes with packed-byte window tests (one lane
//                       per agent for the shapes outside the families
//                       1-16), the rewards and the done byte, stores them,
//                       writes the optional exports (centralized
//                       observation, true state, fog of war), and draws the
//                       Philox actions of the next chunk.
#pragma once

#include <type_traits>

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

// Line of sight: window cell (dx, dy) is visible iff every cell strictly
// between it and the centre on the discrete line -- (rnd(i dx / n),
// rnd(i dy / n)) for i = 1 .. n-1, n = max(|dx|, |dy|), rnd rounding halves
// away from zero -- is free in the window's obstacle plane (lo, hi), whose
// out-of-grid cells are already set.

// The cells strictly between the centre and every window cell, per radius
// 0..4 (window cell k of radius r at entry block_off(r) + k, where
// block_off(r) = sum of (2r' + 1)^2 over r' < r; bits 0-63 in lo, 64-80 in
// hi), evaluated by the compiler.
__host__ __device__ constexpr int block_off(int r) { return (4 * r * r * r - r) / 3; }
struct BlockerTable {
    unsigned long long lo[165];
    unsigned int hi[165];
};
constexpr int rnd_half_away_ce(int p, int n) { return p >= 0 ? (2 * p + n) / (2 * n) : -((-2 * p + n) / (2 * n)); }
constexpr BlockerTable make_blockers() {
    BlockerTable t{};
    for (int r = 0; r <= 4; ++r) {
        const int D = 2 * r + 1;
        for (int dy = -r; dy <= r; ++dy) {
            for (int dx = -r; dx <= r; ++dx) {
                const int n = (dx < 0 ? -dx : dx) > (dy < 0 ? -dy : dy) ? (dx < 0 ? -dx : dx) : (dy < 0 ? -dy : dy);
                const int e = block_off(r) + (dy + r) * D + (dx + r);
                for (int i = 1; i < n; ++i) {
                    const int k = (rnd_half_away_ce(i * dy, n) + r) * D + (rnd_half_away_ce(i * dx, n) + r);
                    if (k < 64)
                        t.lo[e] |= 1ull << k;
                    else
                        t.hi[e] |= 1u << (k - 64);
                }
            }
        }
    }
    return t;
}
static __constant__ BlockerTable c_blockers = make_blockers();

__device__ inline void window_visibility(uint64_t lo, uint64_t hi, int r, uint64_t& vlo, uint64_t& vhi) {
    const int DD = (2 * r + 1) * (2 * r + 1), o = block_off(r);
    vlo = vhi = 0;
    for (int k = 0; k < DD; ++k) {
        const uint64_t blocked = (lo & c_blockers.lo[o + k]) | (hi & (uint64_t)c_blockers.hi[o + k]);
        const uint64_t vis = blocked == 0ull ? 1ull : 0ull;
        if (k < 64)
            vlo |= vis << k;
        else
            vhi |= vis << (k - 64);
    }
}

// Centralized observation of one env (Section 3.3, observability mode 3):
// four planes over the grid, S rows of one word each (S <= 64) -- 0 cells
// inside some observing agent's window (with line of sight: visible to it),
// 1 seen obstacles, 2 seen seekers, 3 seen hiders; bit x of row y is cell
// (x, y).  src holds the agents' cells packed x | y << sh; rows are the env's
// padded obstacle rows.
// Row dy (-R..R) of a window's visibility mask (vl, vh: window bits k =
// (dy + R)(2R + 1) + (dx + R)), as 2R + 1 bits.
__device__ __forceinline__ uint64_t window_row(uint64_t vl, uint64_t vh, int R, int dy) {
    const int D = 2 * R + 1, off = (dy + R) * D;
    return off >= 64 ? vh >> (off - 64) : (vl >> off) | (off + D > 64 ? vh << (64 - off) : 0ull);
}

// Row y of the cells agent (cell v = x | y << sh) of `team` sees: its window
// and, with line of sight, only the visible part; bit x = column x.
__device__ inline uint64_t agent_seen_row(const EnvRT& E, const uint64_t* rows, uint32_t v, uint32_t sh, int team,
                                          int y) {
    const int R = team_radius(E, team), D = 2 * R + 1;
    const int xa = (int)(v & ((1u << sh) - 1u)), ya = (int)(v >> sh);
    const int dy = y - ya;
    if (dy < -R || dy > R) return 0ull;
    uint64_t wrow = (1ull << D) - 1ull;
    if (line_of_sight(E)) {
        uint64_t lo, hi, vl, vh;
        obstacle_plane(rows, E.rw, xa, ya, R, lo, hi);
        window_visibility(lo, hi, R, vl, vh);
        wrow &= window_row(vl, vh, R, dy);
    }
    const int x0 = xa - R;
    const uint64_t smask = E.side == 64 ? ~0ull : ((1ull << E.side) - 1ull);
    return (x0 >= 0 ? (wrow << x0) : (wrow >> (-x0))) & smask;
}

__device__ inline void central_env(const EnvRT& E, const uint64_t* rows, const uint16_t* src, uint32_t sh,
                                   uint64_t* out) {
    const int S = E.side, A = E.n_agents, ns = E.n_seekers, rw = E.rw;
    const uint32_t xmask = (1u << sh) - 1u;
    const uint64_t smask = S == 64 ? ~0ull : ((1ull << S) - 1ull);
    const bool los = line_of_sight(E);
    uint64_t vl[kMaxAgents], vh[kMaxAgents];  // visible cells of each window (line of sight)
    if (los) {
        for (int a = 0; a < A; ++a) {
            const int team = a < ns ? 0 : 1;
            vl[a] = vh[a] = 0;
            if (!team_sees(E, team)) continue;
            const uint32_t v = src[a] & 0x0fffu;
            const int r = team_radius(E, team);
            uint64_t lo, hi;
            obstacle_plane(rows, rw, (int)(v & xmask), (int)(v >> sh), r, lo, hi);
            window_visibility(lo, hi, r, vl[a], vh[a]);
        }
    }
    for (int y = 0; y < S; ++y) {
        uint64_t seen = 0, sk = 0, hd = 0;
        for (int a = 0; a < A; ++a) {
            const uint32_t v = src[a] & 0x0fffu;
            const int xa = (int)(v & xmask), ya = (int)(v >> sh);
            if (ya == y) {
                if (a < ns)
                    sk |= 1ull << xa;
                else
                    hd |= 1ull << xa;
            }
            const int team = a < ns ? 0 : 1;
            if (!team_sees(E, team)) continue;
            const int R = team_radius(E, team), D = 2 * R + 1;
            const int dy = y - ya;
            if (dy < -R || dy > R) continue;
            uint64_t wrow = (1ull << D) - 1ull;
            if (los) wrow &= window_row(vl[a], vh[a], R, dy);  // row dy of the window's visible cells
            const int x0 = xa - R;
            seen |= x0 >= 0 ? (wrow << x0) : (wrow >> (-x0));
        }
        seen &= smask;
        const uint64_t* pr = rows + (y + kPad) * rw;
        const uint64_t obst = (rw == 1 ? (pr[0] >> kPad) : ((pr[0] >> kPad) | (pr[1] << (64 - kPad)))) & smask;
        out[y] = seen;
        out[S + y] = seen & obst;
        out[2 * S + y] = seen & sk;
        out[3 * S + y] = seen & hd;
    }
}

// OR of a row into a shared-memory row word, as native 32-bit atomics on
// its halves (the upper half only for grids over 32 columns).
__device__ __forceinline__ void or_row(uint64_t* w, uint64_t bits, bool wide) {
    unsigned* h = reinterpret_cast<unsigned*>(w);
    if ((uint32_t)bits) atomicOr(h, (unsigned)bits);
    if (wide && (bits >> 32)) atomicOr(h + 1, (unsigned)(bits >> 32));
}

// Bulk asynchronous copies from shared to global memory (the untiled
// cp.async.bulk: both addresses 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(ssrc);
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(s), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until every copy group has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Order this thread's shared-memory writes before later bulk copies read them.
__device__ __forceinline__ void fence_smem_to_bulk() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Wait until no copy group still reads its shared source.
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Centralized observation of one (step, env) by one half-warp (16 lanes;
// the two halves of a warp build two blocks at once), in a buffer of 4 S
// words of shared memory laid out as the output block ([4][S]: seen, seen
// obstacles, seen seekers, seen hiders).  Lane hl of the half takes agents
// hl, hl + 16 (A <= 32): it ORs each one's cell into the seeker or hider rows
// (words 2S.., 3S..) and, if its team observes, its window rows (with line of
// sight: only the visible cells, from one visibility mask) into the seen
// rows; then the half's lanes turn
// rows into output values in place, 16 rows at a time, and its lane 0
// copies the block to global memory with one bulk copy.  `live`: this half
// has an item (the warp's barriers are taken by all 32 lanes either way).
// The caller makes sure the buffer is no longer read by an earlier copy.
__device__ inline void central_half(const EnvRT& E, const uint64_t* rows, const uint16_t* src, uint32_t sh,
                                    int hl, bool live, uint64_t* buf, uint64_t* out) {
    const int S = E.side, A = E.n_agents, ns = E.n_seekers, rw = E.rw;
    const uint64_t smask = S == 64 ? ~0ull : ((1ull << S) - 1ull);
    if (live)
        for (int y = hl; y < 4 * S; y += 16) buf[y] = 0ull;
    __syncwarp();
    for (int a = hl; live && a < A; a += 16) {
        const uint32_t v = src[a] & 0x0fffu;
        const int xa = (int)(v & ((1u << sh) - 1u)), ya = (int)(v >> sh);
        const int team = a < ns ? 0 : 1;
        const bool wide = S > 32;
        or_row(buf + (team ? 3 * S : 2 * S) + ya, 1ull << xa, wide);
        if (team_sees(E, team)) {
            const int R = team_radius(E, team);
            const uint64_t wfull = (1ull << (2 * R + 1)) - 1ull;
            uint64_t vl = 0, vh = 0;
            const bool los = line_of_sight(E);
            if (los) {
                uint64_t lo, hi;
                obstacle_plane(rows, rw, xa, ya, R, lo, hi);
                window_visibility(lo, hi, R, vl, vh);
            }
            const int x0 = xa - R;
            for (int dy = -R; dy <= R; ++dy) {
                const int y = ya + dy;
                if (y < 0 || y >= S) continue;
                const uint64_t w = los ? (wfull & window_row(vl, vh, R, dy)) : wfull;
                const uint64_t bits = (x0 >= 0 ? (w << x0) : (w >> (-x0))) & smask;
                or_row(buf + y, bits, wide);
            }
        }
    }
    __syncwarp();
    if (live) {
        for (int y = hl; y < S; y += 16) {  // each lane reads, then rewrites, only its rows
            const uint64_t seen = buf[y];
            const uint64_t* pr = rows + (y + kPad) * rw;
            const uint64_t obst = (rw == 1 ? (pr[0] >> kPad) : ((pr[0] >> kPad) | (pr[1] << (64 - kPad)))) & smask;
            const uint64_t sk = buf[2 * S + y], hd = buf[3 * S + y];
            buf[S + y] = seen & obst;
            buf[2 * S + y] = seen & sk;
            buf[3 * S + y] = seen & hd;
        }
        fence_smem_to_bulk();
    }
    __syncwarp();
    if (live && hl == 0) bulk_store(out, buf, 32u * (uint32_t)S);
}

// Row y of the cells seen by agents a0..a1-1 of an env without line of
// sight: the union of their window rows.  The constants of the env are
// taken once (row_seen_ctx) and reused over the steps of a chunk.
struct RowSeen {
    uint64_t ws, wh, smask;  // window rows of the seekers / hiders, grid columns
    uint32_t sh, xmask;
    int ns, rs, rh;
    bool s_sees, h_sees;
};
__device__ __forceinline__ RowSeen row_seen_ctx(const EnvRT& E) {
    RowSeen c;
    c.sh = cell_shift(E);
    c.xmask = (1u << c.sh) - 1u;
    c.ns = E.n_seekers;
    c.rs = E.r_seek;
    c.rh = E.r_hide;
    c.ws = (1ull << (2 * c.rs + 1)) - 1ull;
    c.wh = (1ull << (2 * c.rh + 1)) - 1ull;
    c.smask = E.side == 64 ? ~0ull : ((1ull << E.side) - 1ull);
    c.s_sees = team_sees(E, 0);
    c.h_sees = team_sees(E, 1);
    return c;
}
// The same for N steps at once (N independent chains for the scheduler):
// src[j] holds step j's cells.
template <int N>
__device__ __forceinline__ void row_seen_n(const RowSeen& c, const uint16_t* const (&src)[N], int a0, int a1, int y,
                                           uint64_t (&seen)[N]) {
#pragma unroll
    for (int j = 0; j < N; ++j) seen[j] = 0ull;
    for (int a = a0; a < a1; ++a) {
        const bool hider = a >= c.ns;
        if (!(hider ? c.h_sees : c.s_sees)) continue;
        const int R = hider ? c.rh : c.rs;
        const uint64_t w = hider ? c.wh : c.ws;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const uint32_t v = src[j][a] & 0x0fffu;
            const int x0 = (int)(v & c.xmask) - R;
            const bool in = (uint32_t)(y - (int)(v >> c.sh) + R) <= (uint32_t)(2 * R);
            const uint64_t bits = x0 >= 0 ? (w << x0) : (w >> (-x0));
            seen[j] |= in ? bits : 0ull;
        }
    }
#pragma unroll
    for (int j = 0; j < N; ++j) seen[j] &= c.smask;
}

__device__ __forceinline__ uint64_t row_seen(const RowSeen& c, const uint16_t* src, int a0, int a1, int y) {
    uint64_t seen = 0;
    for (int a = a0; a < a1; ++a) {
        const bool hider = a >= c.ns;
        if (!(hider ? c.h_sees : c.s_sees)) continue;
        const uint32_t v = src[a] & 0x0fffu;
        const int R = hider ? c.rh : c.rs;
        if ((uint32_t)(y - (int)(v >> c.sh) + R) > (uint32_t)(2 * R)) continue;
        const int x0 = (int)(v & c.xmask) - R;
        const uint64_t w = hider ? c.wh : c.ws;
        seen |= x0 >= 0 ? (w << x0) : (w >> (-x0));
    }
    return seen & c.smask;
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
// a1-a9 fused over n_steps steps.
// --------------------------------------------------------------------------
struct SlotRec {
    uint32_t unp_rel;  // first unpacked byte inside a slot
    uint16_t p0;       // pristine start cell (CTA packing x | y << sh)
    uint8_t env;       // env index inside the group
    uint8_t agent;     // agent index inside its env
};

struct CtaShared {
    EnvRT env[kMaxGroupEnvs];
    uint32_t gidx[kMaxGroupEnvs];  // handle env index (done byte, counters)
    uint32_t coff[kMaxGroupEnvs];  // first word of the env's centralized observation
    uint32_t ept0[kMaxGroupEnvs];  // episode clock before the launch's first step
    uint32_t foff[kMaxGroupEnvs];  // first word of the env's fog units in a slot
    GroupPlan plan;
    SlotRec slot[kMaxGroupSlots];
    uint16_t p0[kMaxGroupSlots];  // pristine start cells (CTA packing)
    uint4 key[kMaxGroupSlots];     // Philox action counter words (agent, env id) and the env's key
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
    uint32_t k0;            // steps of the launch before the chunk
    int worker, n_workers;  // this thread among the emission threads
    uint8_t* stage;         // this warp's staging area of the unpacked export (kUnpStage)
};

// ---------------------------------------------------------------------------
// General emission (a5, a6, a9), for groups outside the one-thread form
// below (line of sight, or seekers other than ceil(A/2)): one lane per
// agent of a (step, env).  Each lane tests every other agent against its own
// window (radius of its team) and sets the bit in the plane of that agent's
// team; the reward's "seen" test (seeker radius) is combined over the
// segment's lanes with warp ballots.  NW = 32-bit words per plane: 2 when
// every window fits 64 bits, 3 with radius 4.
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
    const int ai = only_hiders_emit(E0) ? a - ns : a;
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
        }
        // the observed positions: the pristine start cells after a reset
        const uint16_t* src = done ? H.p0 + first : Tk;
        const uint32_t po = src[a] & 0x0fffu;
        const int xo = (int)(po & xmask), yo = (int)(po >> sh);
        const int xra = xo - R, yra = yo - R;
        Plane<NW> ps, ph;  // bits of seekers / hiders in this agent's window
        ps.lo = ph.lo = 0;
        ps.hi = ph.hi = 0;
#pragma unroll
        for (int b = 0; b < AM; ++b) {
            if (b >= A) break;
            const uint32_t v = src[b] & 0x0fffu;
            const uint32_t dx = (uint32_t)((int)(v & xmask) - xra), dy = (uint32_t)((int)(v >> sh) - yra);
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
                // a5 obstacle plane (and, with line of sight, the visible cells)
                Plane<NW> o0, vis;
                vis.lo = ~0ull;
                vis.hi = ~0u;
                const bool los = line_of_sight(E);
                if (use_table) {
                    const uint32_t W = words_of_radius(R);
                    const uint64_t* tw =
                        C.tbl + L.tbl_off[ee][ta ? 1 : 0] + (uint32_t)(yo * E.side + xo) * table_words(E, R);
                    o0.lo = tw[0];
                    o0.hi = (NW == 3 && W == 2) ? (uint32_t)tw[1] : 0u;
                    if (los) {
                        vis.lo = tw[W];
                        vis.hi = (NW == 3 && W == 2) ? (uint32_t)tw[W + 1] : 0u;
                    }
                } else {
                    uint64_t lo, hi;
                    obstacle_plane(C.rows + L.rows_off[ee], E.rw, xo, yo, R, lo, hi);
                    o0.lo = lo;
                    o0.hi = (uint32_t)hi;
                    if (los) {
                        uint64_t vl, vh;
                        window_visibility(lo, hi, R, vl, vh);
                        vis.lo = vl;
                        vis.hi = (uint32_t)vh;
                    }
                }
                Plane<NW> al = ta ? ph : ps;
                Plane<NW> opp = ta ? ps : ph;
                if (los) {  // hidden cells read 0 in every plane
                    o0.lo &= vis.lo;
                    o0.hi &= vis.hi;
                    al.lo &= vis.lo;
                    al.hi &= vis.hi;
                    opp.lo &= vis.lo;
                    opp.hi &= vis.hi;
                }
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
    uint32_t tr;          // radius of the table's windows (> R: the team cuts its window out)
    bool use_table;
    bool v16;             // the env's obs words start 16-byte aligned
};

// Streaming (evict-first) global stores of the outputs.
__device__ __forceinline__ void st_cs_u8(uint8_t* p, uint32_t a) { asm volatile("st.global.cs.u8 [%0], %1;" ::"l"(p), "r"(a)); }
__device__ __forceinline__ void st_cs_v4(uint8_t* p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w));
}

// The unpacked export of one agent: byte i of its 3 DD bytes (DD <= 64) is
// bit i of the string p0 | p1 << DD | p2 << 2 DD (plane after plane; bits of
// a plane above DD are 0).  The string is shifted by the h bytes before the
// first 4-byte boundary of u, and every aligned 32-bit word then takes four
// bits: (b * 0x00204081) & 0x01010101 moves bit j of a 4-bit value b to bit
// 0 of byte j.  The h bytes and the bytes after the last boundary are stored
// singly.
__device__ __forceinline__ void unpack_planes(uint8_t* u, uint64_t p0, uint64_t p1, uint64_t p2, uint32_t DD) {
    const uint32_t n = 3u * DD;
    uint64_t s0 = p0, s1 = 0ull, s2 = 0ull;  // the string, bits 0-63, 64-127, 128-191
    auto put = [&](uint64_t v, uint32_t b) {  // OR v in at bit b (b + 64 <= 192 or v short enough)
        const uint32_t q = b >> 6, r = b & 63u;
        const uint64_t lo = v << r, hi = r ? v >> (64u - r) : 0ull;
        s0 |= q == 0u ? lo : 0ull;
        s1 |= q == 1u ? lo : (q == 0u ? hi : 0ull);
        s2 |= q == 2u ? lo : (q == 1u ? hi : 0ull);
    };
    put(p1, DD);
    put(p2, 2u * DD);
    auto bit = [&](uint32_t b) -> uint32_t {
        const uint64_t w = b < 64u ? s0 : (b < 128u ? s1 : s2);
        return (uint32_t)(w >> (b & 63u)) & 1u;
    };
    const uint32_t h = min(n, (4u - ((uint32_t)reinterpret_cast<uintptr_t>(u) & 3u)) & 3u);
    for (uint32_t i = 0; i < h; ++i) u[i] = (uint8_t)bit(i);
    uint64_t t0 = s0, t1 = s1, t2 = s2;  // the string from bit h on
    if (h) {
        t0 = (s0 >> h) | (s1 << (64u - h));
        t1 = (s1 >> h) | (s2 << (64u - h));
        t2 = s2 >> h;
    }
    const uint32_t nq = (n - h) >> 2;  // whole words
    uint32_t* w = reinterpret_cast<uint32_t*>(u + h);
#pragma unroll 1
    for (uint32_t g = 0; 16u * g < nq; ++g) {
        const uint64_t t = g == 0u ? t0 : (g == 1u ? t1 : t2);
#pragma unroll
        for (uint32_t j = 0; j < 16u; ++j) {
            const uint32_t q = 16u * g + j;
            if (q < nq) w[q] = (((uint32_t)(t >> (4u * j)) & 15u) * 0x00204081u) & 0x01010101u;
        }
    }
    for (uint32_t i = h + 4u * nq; i < n; ++i) u[i] = (uint8_t)bit(i);
}

// Observer a's three planes (obstacle, ally, opponent): bits 0-63 and, with
// radius-4 windows (W2), bits 64-80; a seeker also marks the hiders inside its
// window in seenf.
struct Words3 {
    uint64_t o0, al, op;
    uint32_t o0h, alh, oph;
};

// The unpacked export of windows over 64 bits (radius 4): byte by byte.
__device__ __forceinline__ void unpack_planes_wide(uint8_t* u, const Words3& w, uint32_t DD) {
    for (uint32_t q = 0; q < DD; ++q) {
        const bool lo = q < 64u;
        u[q] = (uint8_t)(lo ? (w.o0 >> q) & 1u : (w.o0h >> (q - 64u)) & 1u);
        u[DD + q] = (uint8_t)(lo ? (w.al >> q) & 1u : (w.alh >> (q - 64u)) & 1u);
        u[2 * DD + q] = (uint8_t)(lo ? (w.op >> q) & 1u : (w.oph >> (q - 64u)) & 1u);
    }
}

// The inner (2 rs + 1)^2 window of a (2 rb + 1)^2 window plane (rb <= 3)
// centred on the same cell.  A smaller window's obstacle and visibility bits
// equal the inner part of the larger one's: its cells, and the cells between
// them and the centre, all lie inside it.
__device__ __forceinline__ uint64_t sub_window(uint64_t w, uint32_t rb, uint32_t rs) {
    const uint32_t db = 2u * rb + 1u, ds = 2u * rs + 1u, off = rb - rs;
    const uint64_t m = (1ull << ds) - 1ull;
    uint64_t out = 0;
    for (uint32_t i = 0; i < ds; ++i) out |= ((w >> ((i + off) * db + off)) & m) << (i * ds);
    return out;
}

template <int A, bool TA, bool HI, bool W2, bool LOS>
__device__ __forceinline__ Words3 observer_words(const TeamCtx& T, int a, uint32_t R, uint32_t D, uint32_t KR,
                                                 uint32_t C2, uint32_t KP, uint32_t centre, uint32_t centre_hi,
                                                 const uint32_t (&X4)[(A + 3) / 4], const uint32_t (&Y4)[(A + 3) / 4],
                                                 const uint32_t (&P4)[(A + 3) / 4], const uint32_t (&P8)[(A + 3) / 4],
                                                 uint32_t (&seenf)[(A + 3) / 4]) {
    constexpr int NS = (A + 1) / 2, NW = (A + 3) / 4;
    const uint32_t v = T.src[a] & 0x0fffu;
    const uint32_t xa = v & T.xmask, ya = v >> T.sh;
    const uint32_t Kx = KR - xa * 0x01010101u, Ky = KR - ya * 0x01010101u;
    const uint32_t Kp = ((KP - (ya * D + xa)) & 0xffu) * 0x01010101u;
    const uint32_t Kp7 = Kp & 0x7f7f7f7fu, Kp8 = Kp & 0x80808080u;
    uint32_t al0 = 0, al1 = 0, op0 = 0, op1 = 0, al2 = 0, op2 = 0;
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
        // P4[j] holds the bytes' low 7 bits, P8[j] their bit 7 (split once per segment)
        const uint32_t n4 = ((P4[j] + Kp7) ^ (P8[j] ^ Kp8)) | fail;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = 4 * j + q;
            if (b >= A) continue;
            const uint32_t n = __byte_perm(n4, 0u, 0x4440u | (uint32_t)q);
            const uint32_t m0 = shl_clamp(1u, n);
            const uint32_t m1 = HI ? shl_clamp(1u, n - 32u) : 0u;  // windows of over 32 bits only
            const uint32_t m2 = W2 ? shl_clamp(1u, n - 64u) : 0u;  // windows of over 64 bits only
            if ((b >= NS) == TA) {
                al0 |= m0;
                if (HI) al1 |= m1;
                if (W2) al2 |= m2;
            } else {
                op0 |= m0;
                if (HI) op1 |= m1;
                if (W2) op2 |= m2;
            }
        }
    }
    Words3 w;
    w.al = (uint64_t)(al0 & centre) | ((uint64_t)(al1 & centre_hi) << 32);
    w.op = (uint64_t)op0 | ((uint64_t)op1 << 32);
    w.alh = al2;  // the centre bit (R D + R <= 40) is never in the high word
    w.oph = op2;
    w.o0 = 0;
    w.o0h = 0;
    {  // a5 obstacle plane (and, with line of sight, the visible cells)
        uint64_t vis = ~0ull;
        uint32_t vis_hi = ~0u;  // bits 64-80 of two-word windows
        if (T.use_table) {
            if (W2 && R == 4u) {  // two table words a cell (four with line of sight)
                const uint64_t* c = T.tbl + (LOS ? 4u : 2u) * (ya * T.side + xa);
                w.o0 = c[0];
                w.o0h = (uint32_t)c[1];
                if (LOS) {
                    vis = c[2];
                    vis_hi = (uint32_t)c[3];
                }
            } else if (LOS) {  // one-word windows: obstacle plane, then visibility
                const uint64_t* c = T.tbl + 2u * (ya * T.side + xa);
                w.o0 = c[0];
                vis = c[1];
                if (T.tr != R) {  // a shared table of a larger radius: the inner window
                    w.o0 = sub_window(w.o0, T.tr, R);
                    vis = sub_window(vis, T.tr, R);
                }
            } else {
                w.o0 = T.tbl[ya * T.side + xa];
            }
        } else {
            uint64_t hi;
            obstacle_plane(T.rows, (int)T.rw, (int)xa, (int)ya, (int)R, w.o0, hi);
            w.o0h = (uint32_t)hi;
            if (LOS) {
                uint64_t vh;
                window_visibility(w.o0, hi, (int)R, vis, vh);
                vis_hi = (uint32_t)vh;
            }
        }
        if (LOS) {  // hidden cells read 0 in all three planes
            w.o0 &= vis;
            w.al &= vis;
            w.op &= vis;
            if (W2) {
                w.o0h &= vis_hi;
                w.alh &= vis_hi;
                w.oph &= vis_hi;
            }
        }
        if (T.unp) {
            if (W2)
                unpack_planes_wide(T.unp + T.slot[a].unp_rel, w, D * D);
            else
                unpack_planes(T.unp + T.slot[a].unp_rel, w.o0, w.al, w.op, D * D);
        }
    }
    return w;
}

__device__ __forceinline__ void st16(uint64_t* p, uint64_t a, uint64_t b) {
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(a, b);
}

// Global stores of 8, 16 and 32 bytes (CS: evict-first).
template <bool CS>
__device__ __forceinline__ void out8(uint64_t* p, uint64_t a) {
    if (CS)
        asm volatile("st.global.cs.u64 [%0], %1;" ::"l"(p), "l"(a));
    else
        *p = a;
}
template <bool CS>
__device__ __forceinline__ void out16(uint64_t* p, uint64_t a, uint64_t b) {
    if (CS)
        asm volatile("st.global.cs.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b));
    else
        *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(a, b);
}
template <bool CS>
__device__ __forceinline__ void out32(uint64_t* p, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    if (CS)
        asm volatile("st.global.cs.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d));
    else
        asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d));
}

// Six consecutive output words at o (8-byte aligned) with as few stores as
// the alignment allows: at a 32-byte boundary or 16 bytes past one, one
// 32-byte and one 16-byte store (a store per 32-byte sector where it can:
// the store path handles each lane's sectors one by one, and scattered
// half-sector stores of the emission hold up the dynamics warps' shared
// memory accesses; measured on 1024 envs x 10 agents, same GPU: +1.5 %, and
// without any observation stores +7 %); otherwise 8 + 16 + 16 + 8 bytes, or
// 8 + 32 + 8 at 24 bytes past a boundary.  (The streaming form keeps its
// 16-byte stores: 32-byte ones measured 1.3 % slower there.)
template <bool CS>
__device__ __forceinline__ void out6(uint64_t* o, uint64_t w0, uint64_t w1, uint64_t w2, uint64_t w3, uint64_t w4,
                                     uint64_t w5) {
    const uint32_t q = (uint32_t)reinterpret_cast<uintptr_t>(o) & 31u;
    if (!(q & 8u)) {
        const bool q0 = q == 0u;
        out32<CS>(q0 ? o : o + 2, q0 ? w0 : w2, q0 ? w1 : w3, q0 ? w2 : w4, q0 ? w3 : w5);
        out16<CS>(q0 ? o + 4 : o, q0 ? w4 : w0, q0 ? w5 : w1);
    } else {
        out8<CS>(o, w0);
        if (q == 24u) {
            out32<CS>(o + 1, w1, w2, w3, w4);
        } else {
            out16<CS>(o + 1, w1, w2);
            out16<CS>(o + 3, w3, w4);
        }
        out8<CS>(o + 5, w5);
    }
}

// One team's observers.  With 16-byte aligned records (T.v16) the three
// words of two consecutive observers leave as three 16-byte stores, and a
// lone observer as one 16-byte and one 8-byte store; otherwise three 8-byte
// stores per observer.
template <int A, bool TA, bool HI, bool W2, bool LOS>
__device__ __forceinline__ void emit_team_fast(const TeamCtx& T, uint32_t R, const uint32_t (&X4)[(A + 3) / 4],
                                               const uint32_t (&Y4)[(A + 3) / 4], const uint32_t (&P4)[(A + 3) / 4],
                                               const uint32_t (&P8)[(A + 3) / 4], uint32_t (&seenf)[(A + 3) / 4]) {
    constexpr int NS = (A + 1) / 2;
    const uint32_t D = 2u * R + 1u;
    const uint32_t KR = (0x80u + R) * 0x01010101u;
    const uint32_t C2 = (0x7fu - 2u * R) * 0x01010101u;
    const uint32_t KP = R * D + R;
    const uint32_t centre = ~shl_clamp(1u, KP), centre_hi = ~shl_clamp(1u, KP - 32u);
    constexpr int first = TA ? NS : 0, end = TA ? A : NS;
    if constexpr (W2) {  // two words a plane: six words an observer, three 16-byte stores
#pragma unroll 1
        for (int a = first; a < end; ++a) {
            const Words3 p =
                observer_words<A, TA, HI, W2, LOS>(T, a, R, D, KR, C2, KP, centre, centre_hi, X4, Y4, P4, P8, seenf);
            uint64_t* o = T.ob + 6 * (a - T.ai0);
            if (T.v16) {
                out6<false>(o, p.o0, p.o0h, p.al, p.alh, p.op, p.oph);
            } else {
                o[0] = p.o0;
                o[1] = p.o0h;
                o[2] = p.al;
                o[3] = p.alh;
                o[4] = p.op;
                o[5] = p.oph;
            }
        }
    } else {
#pragma unroll 1
        for (int a = first; a < end;) {
            const Words3 p =
                observer_words<A, TA, HI, W2, LOS>(T, a, R, D, KR, C2, KP, centre, centre_hi, X4, Y4, P4, P8, seenf);
            const int w = 3 * (a - T.ai0);
            uint64_t* o = T.ob + w;
            if (T.v16 && !(w & 1) && a + 1 < end) {
                const Words3 q = observer_words<A, TA, HI, W2, LOS>(T, a + 1, R, D, KR, C2, KP, centre, centre_hi, X4, Y4,
                                                               P4, P8, seenf);
                out6<false>(o, p.o0, p.al, p.op, q.o0, q.al, q.op);
                a += 2;
            } else if (T.v16 && (w & 1)) {
                o[0] = p.o0;
                st16(o + 1, p.al, p.op);
                ++a;
            } else if (T.v16) {
                st16(o, p.o0, p.al);
                o[2] = p.op;
                ++a;
            } else {
                o[0] = p.o0;
                o[1] = p.al;
                o[2] = p.op;
                ++a;
            }
        }
    }
}

template <int A, bool W2, bool LOS>
__device__ __forceinline__ void emit_segment_fast(const StepParams& P, const CtaShared& H, const EmitCtx& C,
                                                  uint32_t k, uint32_t e, uint8_t* stage_item) {
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
    uint32_t sl = C.base_slot + k;
    if (sl >= P.ring) sl -= P.ring;
    const bool emit_s = team_emits(E, 0), emit_h = A > 1 && team_emits(E, 1);
    uint32_t X4[NW], Y4[NW], Ps[NW], Ph[NW], seenf[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) X4[j] = Y4[j] = Ps[j] = Ph[j] = seenf[j] = 0u;
    if (emit_s || emit_h) {
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
        uint32_t Ps8[NW], Ph8[NW];
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            Ps8[j] = Ps[j] & 0x80808080u;
            Ps[j] &= 0x7f7f7f7fu;
            Ph8[j] = Ph[j] & 0x80808080u;
            Ph[j] &= 0x7f7f7f7fu;
        }
        TeamCtx T;
        T.src = src;
        T.rows = C.rows + L.rows_off[e];
        T.ob = P.obs + (uint64_t)sl * P.obs_words + E.obs_off;
        // the unpacked planes of agent a go to unp + unp_rel(a): the slot in
        // global memory, or this item's place in the warp's staging area
        T.unp = !P.unp ? nullptr : (stage_item ? stage_item - E.unp_off : P.unp + (uint64_t)sl * P.unp_bytes);
        T.slot = H.slot + first;
        T.sh = sh;
        T.xmask = xmask;
        T.side = E.side;
        T.rw = E.rw;
        T.use_table = L.flags & kUseTable;
        T.v16 = (reinterpret_cast<uintptr_t>(T.ob) & 15u) == 0u;
        T.tbl = C.tbl + L.tbl_off[e][0];
        T.tr = (L.flags & kSharedTable) ? (uint32_t)table_radius(E) : rs;
        T.ai0 = 0;
        if (emit_s) {
            if (W2)
                emit_team_fast<A, false, true, true, LOS>(T, rs, X4, Y4, Ps, Ps8, seenf);
            else if (Ds * Ds > 32u)
                emit_team_fast<A, false, true, false, LOS>(T, rs, X4, Y4, Ps, Ps8, seenf);
            else
                emit_team_fast<A, false, false, false, LOS>(T, rs, X4, Y4, Ps, Ps8, seenf);
        }
        if (emit_h) {
            T.tbl = C.tbl + L.tbl_off[e][1];
            T.tr = (L.flags & kSharedTable) ? (uint32_t)table_radius(E) : rh;
            T.ai0 = emit_s ? 0 : NS;
            if (W2)
                emit_team_fast<A, true, true, true, LOS>(T, rh, X4, Y4, Ph, Ph8, seenf);
            else if (Dh * Dh > 32u)
                emit_team_fast<A, true, true, false, LOS>(T, rh, X4, Y4, Ph, Ph8, seenf);
            else
                emit_team_fast<A, true, false, false, LOS>(T, rh, X4, Y4, Ph, Ph8, seenf);
        }
    }
    uint32_t seen = 0;
    if (done || !emit_s) {  // the reward's test straight from the positions
        seen = seen_pre_reset(Tk, A, NS, (int)rs, sh);
    } else {
#pragma unroll
        for (int b = NS; b < A; ++b) seen |= ((seenf[b >> 2] >> (8 * (b & 3) + 7)) & 1u) << b;
    }
    // a6 rewards, a7 done byte, actions
    const int32_t n_seen = (int32_t)__popc(seen);
    int32_t* rw = P.rew + (uint64_t)sl * P.agents + E.agent_off;
    uint8_t* dn = P.done + (uint64_t)sl * P.n_envs + H.gidx[e];
    if ((reinterpret_cast<uintptr_t>(rw) & 7u) == 0u) {  // 8-byte pairs
#pragma unroll
        for (int a = 0; a + 1 < A; a += 2) {
            const int32_t r0 = a < NS ? n_seen : -(int32_t)((seen >> a) & 1u);
            const int32_t r1 = a + 1 < NS ? n_seen : -(int32_t)((seen >> (a + 1)) & 1u);
            *reinterpret_cast<int2*>(rw + a) = make_int2(r0, r1);
        }
        if (A & 1) rw[A - 1] = A - 1 < NS ? n_seen : -(int32_t)((seen >> (A - 1)) & 1u);
    } else {
#pragma unroll
        for (int a = 0; a < A; ++a) rw[a] = a < NS ? n_seen : -(int32_t)((seen >> a) & 1u);
    }
    *dn = done ? 3u : 0u;
    if (P.act_out) {
        uint8_t* ao = P.act_out + (uint64_t)sl * P.agents + E.agent_off;
#pragma unroll
        for (int a = 0; a < A; ++a) ao[a] = C.act[act_index(k, (uint32_t)(first + a), nsl)];
    }
}

template <int A, bool W2, bool LOS>
__device__ __forceinline__ void emit_segments_fast(const StepParams& P, const CtaShared& H, const EmitCtx& C) {
    const GroupPlan& L = H.plan;
    const uint32_t ne = L.n_envs;
    const uint32_t total = C.len * ne;
    const uint32_t dk = (uint32_t)C.n_workers / ne, de = (uint32_t)C.n_workers % ne;
    uint32_t k = (uint32_t)C.worker / ne, e = (uint32_t)C.worker % ne;
    if (!((L.flags & kUnpStage) && P.unp)) {
        for (uint32_t it = (uint32_t)C.worker; it < total; it += (uint32_t)C.n_workers) {
            emit_segment_fast<A, W2, LOS>(P, H, C, k, e, nullptr);
            e += de;
            k += dk;
            if (e >= ne) {
                e -= ne;
                ++k;
            }
        }
        return;
    }
    // The unpacked export staged per warp: a round's 32 consecutive items
    // form one contiguous run per step (envs e_a..e_b of step kk sit at
    // unp_off[e_a] of its slot); each run is staged at an offset congruent
    // to its destination mod 16 and leaves with 16-byte stores.
    const int lane = C.worker & 31;
    uint8_t* const stage = C.stage;
    auto run_dst = [&](uint32_t kk, uint32_t e_a) {
        uint32_t sl = C.base_slot + kk;
        if (sl >= P.ring) sl -= P.ring;
        return P.unp + (uint64_t)sl * P.unp_bytes + H.env[e_a].unp_off;
    };
    for (uint32_t i0 = (uint32_t)C.worker - (uint32_t)lane; i0 < total; i0 += (uint32_t)C.n_workers) {
        const uint32_t i = i0 + (uint32_t)lane, last = min(i0 + 31u, total - 1u);
        const uint32_t k_a = i0 / ne, k_b = last / ne;
        if (i < total) {
            uint32_t off = 0;
            uint8_t* stage_item = nullptr;
            for (uint32_t kk = k_a; kk <= k; ++kk) {
                const uint32_t first = max(i0, kk * ne), end = min(last + 1u, (kk + 1u) * ne);
                off += ((uint32_t)reinterpret_cast<uintptr_t>(run_dst(kk, first - kk * ne)) - off) & 15u;
                if (kk == k) stage_item = stage + off + (i - first) * L.unp_env;
                off += (end - first) * L.unp_env;
            }
            emit_segment_fast<A, W2, LOS>(P, H, C, k, e, stage_item);
        }
        __syncwarp();  // every lane has staged its bytes
        uint32_t off = 0;
        for (uint32_t kk = k_a; kk <= k_b; ++kk) {
            const uint32_t first = max(i0, kk * ne), end = min(last + 1u, (kk + 1u) * ne);
            uint8_t* g = run_dst(kk, first - kk * ne);
            const uint32_t mis = (uint32_t)reinterpret_cast<uintptr_t>(g) & 15u;
            off += (mis - off) & 15u;
            const uint8_t* src = stage + off;  // src = g mod 16
            const uint32_t len = (end - first) * L.unp_env;
            const uint32_t head = min(len, (16u - mis) & 15u);
            const uint32_t body = (len - head) >> 4, tail0 = head + 16u * body;
            if ((uint32_t)lane < head) st_cs_u8(g + lane, src[lane]);
            for (uint32_t c = (uint32_t)lane; c < body; c += 32u)
                st_cs_v4(g + head + 16u * c, *reinterpret_cast<const uint4*>(src + head + 16u * c));
            if ((uint32_t)lane < len - tail0) st_cs_u8(g + tail0 + lane, src[tail0 + lane]);
            off += len;
        }
        __syncwarp();  // the staging area is read before the next round writes it
        e += de;
        k += dk;
        if (e >= ne) {
            e -= ne;
            ++k;
        }
    }
}


template <int FAM>
__device__ __forceinline__ void emit_fast_dispatch(int A, const StepParams& P, const CtaShared& H,
                                                   const EmitCtx& C) {
    constexpr int a0 = 4 * ((FAM - 1) % 4) + 1;
    constexpr bool W2 = (FAM >= 5 && FAM <= 8) || FAM >= 13;  // two words a plane
    constexpr bool LOS = FAM >= 9;                             // line of sight
    if (A == a0) emit_segments_fast<a0, W2, LOS>(P, H, C);
    else if (A == a0 + 1) emit_segments_fast<a0 + 1, W2, LOS>(P, H, C);
    else if (A == a0 + 2) emit_segments_fast<a0 + 2, W2, LOS>(P, H, C);
    else emit_segments_fast<a0 + 3, W2, LOS>(P, H, C);
}

// Per-cell shared state of the dynamics: a claim word (byte a-1 holds the
// lane claiming the cell through action a, 1 N 2 S 3 E 4 W; 0xff = none)
// and a state byte (bits 1..4: action a leads onto a free cell of the grid;
// bit 7: occupied).
constexpr uint32_t kNoClaims = 0xffffffffu;

template <int MAXT, int MINB, int FAM>
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
        for (int i = 0; i < ne; ++i) {
            const uint32_t g = P.env_list[G.list_first + i];
            const EnvRT E = P.env[g];
            H.env[i] = E;
            H.gidx[i] = g;
            H.coff[i] = P.central ? P.central_off[g] : 0u;
            H.ept0[i] = P.st_ept ? P.est[g].ep_t : 0u;
            H.foff[i] = P.fog ? P.fog_off[g] : 0u;
            uint32_t urel = E.unp_off;
            for (int a = 0; a < E.n_agents; ++a) {
                const int t = a < E.n_seekers ? 0 : 1;
                SlotRec r;
                r.env = (uint8_t)i;
                r.agent = (uint8_t)a;
                r.p0 = 0;
                r.unp_rel = urel;
                if (team_emits(E, t)) {
                    const int rr = team_radius(E, t);
                    urel += 3u * (2 * rr + 1) * (2 * rr + 1);
                }
                H.slot[slot] = r;
                ++slot;
            }
        }
        plan_group(H.env, ne, (int)kc, G.flags, H.plan);
    }
    __syncthreads();
    if (H.plan.total > dynamic_smem_bytes()) {  // the host sized the launch by the same plan: cannot happen
        if (tid == 0) atomicOr(P.err, kErrSmemPlan);
        return;  // the whole CTA (H.plan is shared)
    }
    const GroupPlan& L = H.plan;
    const bool use_table = L.flags & kUseTable;
    uint8_t* s_act = sm + L.act;                     // [3][act_words] (bytes of 4 steps)
    uint16_t* s_traj = (uint16_t*)(sm + L.traj);     // [2][kc][slots]
    uint64_t* s_rows = (uint64_t*)(sm + L.rows);
    uint32_t* s_claim = (uint32_t*)(sm + L.claim);   // per cell
    uint8_t* s_state = sm + L.state;                 // per cell
    uint64_t* s_tbl = (uint64_t*)(sm + L.tbl);
    uint64_t* s_fog = (uint64_t*)(sm + L.fog);     // per fog row: discovered cells
    const uint32_t act_bytes = L.act_words * 4;
    const uint32_t fog_rows = L.fog_off[ne];
    // env of fog row u (rows are grouped by env)
    auto fog_env_of = [&](uint32_t u) {
        int e = 0;
        while (L.fog_off[e + 1] <= u) ++e;
        return e;
    };

    // the discovery rows after the previous launch
    for (uint32_t u = tid; u < fog_rows; u += nthreads) {
        const int e = fog_env_of(u);
        s_fog[u] = P.fog_state[H.foff[e] / 2u + (u - L.fog_off[e])];
    }
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
        const uint2 k = P.keys[H.gidx[r.env]];
        H.key[sidx] = make_uint4(r.agent, E.env_id, k.x, k.y);
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
                const int r = (L.flags & kSharedTable) ? table_radius(E) : team_radius(E, t);
                const uint32_t W = words_of_radius(r), Wt = table_words(E, r);
                const bool los = line_of_sight(E);
                uint64_t* Tb = s_tbl + L.tbl_off[i][t];
                for (int c = tid; c < S * S; c += nthreads) {
                    uint64_t lo, hi;
                    obstacle_plane(Rw, rw, c % S, c / S, r, lo, hi);
                    Tb[c * Wt] = lo;
                    if (W == 2) Tb[c * Wt + 1] = hi;
                    if (los) {  // then the visible cells of the window
                        uint64_t vl, vh;
                        window_visibility(lo, hi, r, vl, vh);
                        Tb[c * Wt + W] = vl;
                        if (W == 2) Tb[c * Wt + W + 1] = vh;
                    }
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
            const uint4 ka = H.key[it % ns], kb = H.key[(two ? it2 : it) % ns];
            uint32_t a0 = (uint32_t)(b0 + it / ns), a1 = ka.x, a2 = ka.y, a3 = 0u;
            uint32_t d0 = (uint32_t)(b0 + (two ? it2 : it) / ns), d1 = kb.x, d2 = kb.y, d3 = 0u;
            philox4x32_10(a0, a1, a2, a3, ka.z, ka.w);
            philox4x32_10(d0, d1, d2, d3, kb.z, kb.w);
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
        // ENDS: the step may end an episode (the launch step index g is checked
        // against warp_next); a group of four steps that ends none runs the
        // step without the check (measured: the check, with its warp barriers,
        // cost ~30 cycles a step even when not taken).
        auto step = [&](uint32_t a, uint16_t* Tk, uint32_t g, auto ends) {
            constexpr bool ENDS = decltype(ends)::value;
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
            if (live) *Tk = (uint16_t)(p | (ENDS && g == next_done ? kDoneBit : 0u));
            if (ENDS && g == warp_next) {  // some env of this warp ends its episode (a8)
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
                    if (warp_next - (g0 + k) >= 4u) {  // no episode ends in these four steps (warp-uniform)
#pragma unroll
                        for (uint32_t j = 0; j < 4; ++j)
                            step(__byte_perm(aw, 0, 0x4440u + j), T + (k + j) * nsl, g0 + k + j, std::false_type{});
                    } else {
#pragma unroll
                        for (uint32_t j = 0; j < 4; ++j)
                            step(__byte_perm(aw, 0, 0x4440u + j), T + (k + j) * nsl, g0 + k + j, std::true_type{});
                    }
                    aw = aw_next;
                }
                for (; k < len; ++k)
                    step(__byte_perm(aw, 0, 0x4440u + (k & 3u)), T + k * nsl, g0 + k, std::true_type{});
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
    (void)wide;
    uint32_t cen_items = 0;  // centralized-observation items this warp has copied out
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
            C.k0 = cp * kc;
            C.worker = worker;
            C.n_workers = n_workers;
            C.stage = sm + L.stage + (uint32_t)(warp - n_dyn) * L.stage_bytes;
            if constexpr (FAM > 0) {
                emit_fast_dispatch<FAM>(H.env[0].n_agents, P, H, C);
            } else {
                if (wide)
                    emit_chunk<3>(P, H, C, warp - n_dyn, M, lane);
                else
                    emit_chunk<2>(P, H, C, warp - n_dyn, M, lane);
            }
            if (P.central) {  // centralized observation, two (step, env) items per warp
                // block buffers of the group's largest side (envs of a group
                // share their packing, not necessarily their side)
                const uint32_t S = L.max_side;
                const int half = lane >> 4, hl = lane & 15;
                uint64_t* buf = reinterpret_cast<uint64_t*>(sm + L.cen) + ((warp - n_dyn) * 2 + half) * 4 * S;
                const uint32_t n_items = C.len * (uint32_t)ne;
                for (uint32_t it0 = 2u * (uint32_t)(warp - n_dyn); it0 < n_items; it0 += 2u * (uint32_t)M) {
                    const uint32_t it = it0 + (uint32_t)half;
                    const bool live = it < n_items;
                    const uint32_t k = live ? it / (uint32_t)ne : 0u, e = live ? it - k * (uint32_t)ne : 0u;
                    const int first = L.first_slot[e];
                    const uint16_t* Tk = C.T + k * nsl + first;
                    const uint16_t* src = (Tk[0] & kDoneBit) ? H.p0 + first : Tk;
                    uint32_t sl = C.base_slot + k;
                    if (sl >= P.ring) sl -= P.ring;
                    // the half's previous copy must have read the buffer
                    if (cen_items && hl == 0) bulk_wait_read0();
                    __syncwarp();
                    central_half(H.env[e], C.rows + L.rows_off[e], src, cell_shift(H.env[e]), hl, live, buf,
                                 P.central + (uint64_t)sl * P.central_words + H.coff[e]);
                    ++cen_items;
                }
            }
            if (P.st_cells) {  // per (step, env)
                const uint32_t ne_ = (uint32_t)ne;
                for (uint32_t it = (uint32_t)worker; it < C.len * ne_; it += (uint32_t)n_workers) {
                    const uint32_t k = it / ne_, e = it - k * ne_;
                    const int first = L.first_slot[e];
                    const uint16_t* Tk = C.T + k * nsl + first;
                    const uint16_t* src = (Tk[0] & kDoneBit) ? H.p0 + first : Tk;
                    const EnvRT& E = H.env[e];
                    const uint32_t sh = cell_shift(E);
                    uint32_t sl = C.base_slot + k;
                    if (sl >= P.ring) sl -= P.ring;
                    // the observed state: cells and the episode clock after the step
                    uint16_t* cl = P.st_cells + (uint64_t)sl * P.agents + E.agent_off;
                    for (int b = 0; b < E.n_agents; ++b) cl[b] = (uint16_t)to_hbm(src[b] & 0x0fffu, sh);
                    P.st_ept[(uint64_t)sl * P.n_envs + H.gidx[e]] =
                        (uint32_t)(((uint64_t)H.ept0[e] + C.k0 + k + 1u) % E.cap);
                }
            }
            // Fog of war: one thread per fog row (env, unit, row y) scans the
            // chunk's steps in order; an episode's first observation (a done
            // step: the reset state) starts the row afresh.
            if (fog_rows) {
                const bool per_agent = (L.flags & kFogAgent) != 0;
                const bool los = line_of_sight(H.env[0]);  // uniform in the group
                for (uint32_t u = (uint32_t)worker; u < fog_rows; u += (uint32_t)n_workers) {
                    const int e = fog_env_of(u);
                    const EnvRT& E = H.env[e];
                    const uint32_t S = E.side, rel = u - L.fog_off[e], j = rel / S, y = rel - j * S;
                    const int ns = E.n_seekers;
                    const int a0 = per_agent ? (team_sees(E, 0) ? (int)j : ns + (int)j) : 0;
                    const int a1 = per_agent ? a0 + 1 : (int)E.n_agents;
                    const int first = L.first_slot[e];
                    const uint64_t* rows_e = C.rows + L.rows_off[e];
                    const RowSeen rs = row_seen_ctx(E);
                    uint64_t* out = P.fog + H.foff[e] + j * 2u * S + y;
                    uint64_t disc = s_fog[u];
                    uint32_t sl = C.base_slot;
                    uint32_t k = 0;
                    if (!los) {  // several steps' rows at a time, then the scan in step order
                        constexpr int NB = FAM == 0 ? 4 : 8;  // family 0 runs at 128 registers
                        for (; k + NB <= C.len; k += NB) {
                            const uint16_t* src[NB];
                            bool done[NB];
#pragma unroll
                            for (int j = 0; j < NB; ++j) {
                                const uint16_t* Tk = C.T + (k + j) * nsl + first;
                                done[j] = (Tk[0] & kDoneBit) != 0u;
                                src[j] = done[j] ? H.p0 + first : Tk;
                            }
                            uint64_t seen[NB];
                            row_seen_n<NB>(rs, src, a0, a1, (int)y, seen);
#pragma unroll
                            for (int j = 0; j < NB; ++j) {
                                const uint64_t prev = done[j] ? 0ull : disc;
                                disc = prev | seen[j];
                                uint64_t* o = out + (uint64_t)sl * P.fog_words;
                                o[0] = disc;
                                o[S] = seen[j] & ~prev;
                                if (++sl == P.ring) sl = 0;
                            }
                        }
                    }
                    for (; k < C.len; ++k) {
                        const uint16_t* Tk = C.T + k * nsl + first;
                        const bool done = (Tk[0] & kDoneBit) != 0u;
                        const uint16_t* src = done ? H.p0 + first : Tk;
                        uint64_t seen = 0;
                        if (los) {
                            for (int a = a0; a < a1; ++a) {
                                const int team = a < ns ? 0 : 1;
                                if (team_sees(E, team))
                                    seen |= agent_seen_row(E, rows_e, src[a] & 0x0fffu, rs.sh, team, (int)y);
                            }
                        } else {
                            seen = row_seen(rs, src, a0, a1, (int)y);
                        }
                        const uint64_t prev = done ? 0ull : disc;
                        disc = prev | seen;
                        uint64_t* o = out + (uint64_t)sl * P.fog_words;
                        o[0] = disc;
                        o[S] = seen & ~prev;
                        if (++sl == P.ring) sl = 0;
                    }
                    s_fog[u] = disc;
                }
            }
        }
        // a1 for chunk c + 1
        if (c + 1 < n_chunks) draw_actions(c + 1, worker, n_workers);
        __syncthreads();
    }
    // every bulk copy of this warp has completed (its shared source stays
    // valid until then); lanes 0 and 16 issued them
    if (cen_items && (lane & 15) == 0) bulk_wait_all();
    // the discovery rows for the next launch
    for (uint32_t u = (uint32_t)worker; u < fog_rows; u += (uint32_t)n_workers) {
        const int e = fog_env_of(u);
        P.fog_state[H.foff[e] / 2u + (u - L.fog_off[e])] = s_fog[u];
    }
}

}  // namespace hase
