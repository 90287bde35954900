// hase_stream.cuh -- the streaming form of the fused step kernel (a1-a9)
// for the one-thread emission families 1-8 (A <= 16, seekers = ceil(A/2),
// no line of sight, no centralized observation, no fog of war).
//
// One CTA owns a group of envs of one shape for the whole launch, as in
// step_kernel, but its warps never meet at a block-wide barrier after the
// prologue; three roles hand work on through rings in shared memory, each
// behind progress counters (release stores, acquire loads):
//
//   action warp (a1): draws the Philox blocks of every agent slot (one block
//     = four steps), up to kActRing quads ahead of the dynamics.
//   dynamics warps (a2, a3, a7, a8) sit on the warp ids the launch names (by
//     default 0, 4, 8, 12: one SM sub-partition; measured faster than
//     spreading them).  One lane per agent slot, whole envs per warp.  A
//     step: a mover writes its lane into the claim byte of its incoming
//     direction in the target cell's claim word; after __syncwarp it reads
//     the claim word and the target's state byte (free neighbours +
//     occupancy) and moves iff the target is unoccupied and no lower lane
//     claimed it (Section 3.2: blocking tiles; lowest index wins; one round
//     decides every conflict because moves into occupied cells are
//     blocked).  The warp writes each step's record (every agent's cell, the
//     episode-end flag) into a ring of kStreamRing steps and publishes its
//     progress every kStreamGroup steps.
//   emission warps (a4-a6, a9) take blocks of 32 consecutive (step, env)
//     items, round robin, each after the dynamics have passed the block's
//     last step, and publish how far they have read so the dynamics may
//     reuse ring slots.  One thread per item builds every observer's three
//     planes with packed-byte window tests, the rewards and the done byte.
//
// With the unpacked export and envs consecutive in its layout, each emission
// warp stages its block's unpacked bytes in shared memory and writes them per
// step as one contiguous run of 16-byte stores (the chunked form does the
// same per round of its emission warps).
//
// Measured on a GB300 against the chunked form (step_kernel): +13 % on
// 65,536 uneven envs (CTAs in waves); -8 % on 1024 envs x 10 agents and -22 %
// on 1024 envs x 2 agents with the unpacked export (one CTA per SM, where the
// chunked dynamics step faster).  A warp-wide __match_any_sync over the targets was tried for the
// collision round and measured at ~800 cycles with ~30 distinct keys (~45
// with a handful): its cost grows with the number of distinct keys.
//
// Every wait is bounded: after kMaxSpins polls the warp sets kErrWaitTimeout
// in the error word and leaves the kernel (the host reports HASE_ETIMEOUT).
#pragma once

#include <type_traits>

#include "hase_step.cuh"
#include "hase_stream_plan.h"

namespace hase {

constexpr uint32_t kMaxSpins = 1u << 22;  // polls of a progress counter before giving up

// What the emission needs of env e besides its EnvRT, one 16-byte load:
// x, y = uint64 offsets of the seeker and hider window tables in shared
// memory (~0u: none), z = uint64 offset of its padded obstacle rows, w =
// handle env index.
struct StreamShared {
    EnvRT env[kMaxGroupEnvs];
    uint4 emit_env[kMaxGroupEnvs];
    uint32_t gidx[kMaxGroupEnvs];  // handle env index
    uint32_t ept0[kMaxGroupEnvs];  // episode clock before the launch (true-state export)
    GroupPlan plan;
    SlotRec slot[kMaxGroupSlots];
    uint16_t scratch[128 + 2 * 4 * 32 * kMaxDyn];  // dynamics lanes without work: record and byte scratch
    uint4 key[kMaxGroupSlots];          // Philox action counter words (agent, env id) and the env's key
    uint32_t act_prog;                  // quads of actions the action warp has drawn (from the launch's first)
    uint32_t dyn_prog[kMaxDyn];         // steps every dynamics warp has recorded
    uint32_t emit_prog[kMaxEmitWarps];  // steps every emission warp has finished reading
};

// Shared-memory accesses by 32-bit shared-window address (the dynamics' state
// lives in shared memory; these keep every access a plain LDS / STS).
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void sts8(uint32_t a, uint32_t v) { asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v)); }
__device__ __forceinline__ void sts16(uint32_t a, uint32_t v) { asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "r"(v)); }
__device__ __forceinline__ uint32_t lds8(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// Progress counters in shared memory: a release store after the producer's
// writes, an acquire load before the consumer's reads (CTA scope).
__device__ __forceinline__ void store_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v)
                 : "memory");
}
__device__ __forceinline__ void store_release_lane0(uint32_t* p, uint32_t v, int lane) {
    __syncwarp();  // the whole warp's writes come before lane 0's release
    if (lane == 0) store_release(p, v);
}
__device__ __forceinline__ uint32_t load_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];"
                 : "=r"(v)
                 : "r"((uint32_t)__cvta_generic_to_shared(p))
                 : "memory");
    return v;
}

// Poll until the minimum of the n counters cnt[0..n) reaches `need` (one
// counter per lane, combined with a warp reduction).  Returns false when the
// bound ran out.
__device__ __forceinline__ bool wait_min(const uint32_t* cnt, int n, uint32_t need, int lane) {
    for (uint32_t spins = 0;; ++spins) {
        const uint32_t v = lane < n ? load_acquire(cnt + lane) : 0xffffffffu;
        if (__reduce_min_sync(0xffffffffu, v) >= need) break;
        if (spins >= kMaxSpins) return false;
        __nanosleep(32);
    }
    return true;
}

// Agents' cells of one record as bytes: X[j] byte q = x of agent 4j + q, Y
// likewise.  Records hold two uint16 cells x | y << sh a word.
template <int A>
struct Cells {
    uint32_t X[(A + 3) / 4], Y[(A + 3) / 4];
};

template <int A>
__device__ __forceinline__ bool load_record(const uint32_t* rec, uint32_t sh, uint32_t xm2, Cells<A>& Q) {
    constexpr int NW = (A + 3) / 4;
    constexpr uint32_t RW = stream_rec_words(A);
    uint32_t w[8];
    if constexpr (RW == 1) {
        w[0] = rec[0];
        w[1] = 0u;
    } else if constexpr (RW == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(rec);
        w[0] = v.x;
        w[1] = v.y;
    } else if constexpr (RW == 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(rec);
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    } else {
        const uint4 v = *reinterpret_cast<const uint4*>(rec);
        const uint4 u = *reinterpret_cast<const uint4*>(rec + 4);
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
        w[4] = u.x;
        w[5] = u.y;
        w[6] = u.z;
        w[7] = u.w;
    }
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint32_t a = w[2 * j], b = w[2 * j + 1];
        Q.X[j] = __byte_perm(a & xm2, b & xm2, 0x6420u);
        Q.Y[j] = __byte_perm((a >> sh) & 0x003f003fu, (b >> sh) & 0x003f003fu, 0x6420u);
    }
    return (w[0] >> 15) & 1u;
}

// Bit 7 of the bytes of hiders (agents NS..A-1) in packed word j.
template <int A>
__host__ __device__ constexpr uint32_t hider_bytes(int j) {
    uint32_t m = 0;
    for (int q = 0; q < 4; ++q)
        if (4 * j + q >= (A + 1) / 2 && 4 * j + q < A) m |= 0x80u << (8 * q);
    return m;
}

// The window test of observer b (radius R) against every packed agent:
// fail bytes have bit 7 set; n4 bytes hold the window bit (dy+R)(2R+1) +
// (dx+R) of the agents inside.  With K = (0x80 + R) per byte, X + K - x_b
// holds dx + R + 0x80 without carries between bytes; inside the window the
// low nibble is dx + R, and the nibble products with D <= 9 stay in a byte.
struct WinConst {
    uint32_t KR, C2, D;
};
__device__ __forceinline__ WinConst win_const(uint32_t R) {
    WinConst c;
    c.KR = (0x80u + R) * 0x01010101u;
    c.C2 = (0x7fu - 2u * R) * 0x01010101u;
    c.D = 2u * R + 1u;
    return c;
}

template <int A>
__device__ __forceinline__ void seen_test(const Cells<A>& Q, uint32_t rs, uint32_t (&seen)[(A + 3) / 4]) {
    constexpr int NS = (A + 1) / 2, NW = (A + 3) / 4;
    const WinConst c = win_const(rs);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const uint32_t sel = (uint32_t)(s & 3) * 0x1111u;
        const uint32_t Kx = c.KR - __byte_perm(Q.X[s >> 2], 0u, sel), Ky = c.KR - __byte_perm(Q.Y[s >> 2], 0u, sel);
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            if (!hider_bytes<A>(j)) continue;
            const uint32_t vx = Q.X[j] + Kx, vy = Q.Y[j] + Ky;
            const uint32_t wx = (vx & 0x7f7f7f7fu) + c.C2, wy = (vy & 0x7f7f7f7fu) + c.C2;
            seen[j] |= (vx & vy & ~wx & ~wy) & hider_bytes<A>(j);
        }
    }
}

// Inputs of one team's observers in one item.
struct TeamIn {
    const uint64_t* tbl;   // obstacle-window table of the team radius (shared), or null
    const uint64_t* rows;  // padded obstacle rows of the env (shared)
    uint64_t* ob;          // obs words of the env's first emitting agent (global)
    uint8_t* unp;          // unpacked slot (global) or null
    const SlotRec* slot;   // slot records of the env's agents
    uint32_t side, rw;
    int ai0;               // emitting index of agent 0
};

// Observer b's three planes (bits 0-63; with W2 bits 64-80 in the high
// words).  v: its cell x | y << sh.  The observer meets itself at the window
// centre of its own team's plane; that bit is cleared (no other agent shares
// its cell).
struct TeamWin {
    WinConst c;
    uint32_t centre, centre_hi;  // masks clearing the centre bit (bits 0-31, 32-63)
};
__device__ __forceinline__ TeamWin team_win(uint32_t R) {
    TeamWin w;
    w.c = win_const(R);
    const uint32_t kc = R * w.c.D + R;
    w.centre = ~shl_clamp(1u, kc);
    w.centre_hi = ~shl_clamp(1u, kc - 32u);
    return w;
}

template <int A, bool TB, bool HI, bool W2>
__device__ __forceinline__ Words3 stream_observer(const TeamIn& T, const Cells<A>& Q, uint32_t v, uint32_t sh,
                                                  uint32_t R, const TeamWin& tw, uint32_t (&seenf)[(A + 3) / 4]) {
    constexpr int NS = (A + 1) / 2, NW = (A + 3) / 4;
    const uint32_t xa = v & ((1u << sh) - 1u), ya = (v >> sh) & 63u;
    const uint32_t Kx = tw.c.KR - xa * 0x01010101u, Ky = tw.c.KR - ya * 0x01010101u;
    uint32_t al0 = 0, al1 = 0, al2 = 0, op0 = 0, op1 = 0, op2 = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint32_t vx = Q.X[j] + Kx, vy = Q.Y[j] + Ky;
        const uint32_t wx = (vx & 0x7f7f7f7fu) + tw.c.C2, wy = (vy & 0x7f7f7f7fu) + tw.c.C2;
        const uint32_t fail = (~vx | wx | ~vy | wy) & 0x80808080u;
        if (!TB) seenf[j] |= ~fail & hider_bytes<A>(j);
        const uint32_t n4 = ((vy & 0x0f0f0f0fu) * tw.c.D + (vx & 0x0f0f0f0fu)) | fail;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int a = 4 * j + q;
            if (a >= A) continue;
            const uint32_t n = __byte_perm(n4, 0u, 0x4440u | (uint32_t)q);
            const uint32_t m0 = shl_clamp(1u, n);
            const uint32_t m1 = HI ? shl_clamp(1u, n - 32u) : 0u;
            const uint32_t m2 = W2 ? shl_clamp(1u, n - 64u) : 0u;
            if ((a >= NS) == TB) {
                al0 |= m0;
                al1 |= m1;
                al2 |= m2;
            } else {
                op0 |= m0;
                op1 |= m1;
                op2 |= m2;
            }
        }
    }
    Words3 w;
    w.al = (uint64_t)(al0 & tw.centre) | ((uint64_t)(al1 & tw.centre_hi) << 32);
    w.op = (uint64_t)op0 | ((uint64_t)op1 << 32);
    w.alh = al2;  // the centre bit (R D + R <= 40) is never in the high word
    w.oph = op2;
    if (T.tbl) {
        if (W2 && R == 4u) {
            const uint64_t* e = T.tbl + 2u * (ya * T.side + xa);
            w.o0 = e[0];
            w.o0h = (uint32_t)e[1];
        } else {
            w.o0 = T.tbl[ya * T.side + xa];
            w.o0h = 0u;
        }
    } else {
        uint64_t hi;
        obstacle_plane(T.rows, (int)T.rw, (int)xa, (int)ya, (int)R, w.o0, hi);
        w.o0h = (uint32_t)hi;
    }
    return w;
}

// Output stores: st.global (the compiler then knows they cannot overwrite the
// shared-memory data it keeps in registers) with the streaming cache hint
// (every output is written once).
__device__ __forceinline__ void gst16(uint64_t* p, uint64_t a, uint64_t b) {
    asm volatile("st.global.cs.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b));
}
__device__ __forceinline__ void gst8(uint64_t* p, uint64_t a) { asm volatile("st.global.cs.u64 [%0], %1;" ::"l"(p), "l"(a)); }
__device__ __forceinline__ void gst_i2(int32_t* p, int32_t a, int32_t b) {
    asm volatile("st.global.cs.v2.s32 [%0], {%1, %2};" ::"l"(p), "r"(a), "r"(b));
}
__device__ __forceinline__ void gst_i1(int32_t* p, int32_t a) { asm volatile("st.global.cs.s32 [%0], %1;" ::"l"(p), "r"(a)); }
__device__ __forceinline__ void gst_u8(uint8_t* p, uint32_t a) { asm volatile("st.global.cs.u8 [%0], %1;" ::"l"(p), "r"(a)); }
__device__ __forceinline__ void gst_u16(uint16_t* p, uint32_t a) { asm volatile("st.global.cs.u16 [%0], %1;" ::"l"(p), "r"(a)); }
__device__ __forceinline__ void gst_u32(uint32_t* p, uint32_t a) { asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(a)); }


// Stores of one observer's words (three, or six with W2) at o, whose
// 16-byte alignment is known from the address.
template <bool W2>
__device__ __forceinline__ void store_one(uint64_t* o, const Words3& p) {
    const bool odd = (reinterpret_cast<uintptr_t>(o) & 8u) != 0u;
    if constexpr (W2) {
        if (!odd) {
            gst16(o, p.o0, p.o0h);
            gst16(o + 2, p.al, p.alh);
            gst16(o + 4, p.op, p.oph);
        } else {
            gst8(o, p.o0);
            gst16(o + 1, p.o0h, p.al);
            gst16(o + 3, p.alh, p.op);
            gst8(o + 5, p.oph);
        }
    } else {
        if (!odd) {
            gst16(o, p.o0, p.al);
            gst8(o + 2, p.op);
        } else {
            gst8(o, p.o0);
            gst16(o + 1, p.al, p.op);
        }
    }
}

// Two consecutive one-word observers: six words at o.
__device__ __forceinline__ void store_two(uint64_t* o, const Words3& p, const Words3& q) {
    if (!(reinterpret_cast<uintptr_t>(o) & 8u)) {
        gst16(o, p.o0, p.al);
        gst16(o + 2, p.op, q.o0);
        gst16(o + 4, q.al, q.op);
    } else {
        gst8(o, p.o0);
        gst16(o + 1, p.al, p.op);
        gst16(o + 3, q.o0, q.al);
        gst8(o + 5, q.op);
    }
}

// One team's observers in pairs (a loop, not unrolled: the code of every
// observer is the same, and an unrolled team does not fit the instruction
// cache beside the rest of the kernel).  src: the observed record (uint16
// cells of the env's agents).
template <int A, bool TB, bool HI, bool W2>
__device__ __forceinline__ void stream_team(const TeamIn& T, const Cells<A>& Q, const uint16_t* src, uint32_t sh,
                                            uint32_t R, uint32_t (&seenf)[(A + 3) / 4]) {
    constexpr int NS = (A + 1) / 2;
    constexpr int first = TB ? NS : 0, end = TB ? A : NS;
    const TeamWin tw = team_win(R);
    constexpr int W = W2 ? 6 : 3;
    const uint32_t DD = tw.c.D * tw.c.D;
#pragma unroll 1
    for (int b = first; b < end; b += 2) {
        const bool two = b + 1 < end;
        const uint32_t vv = *reinterpret_cast<const uint32_t*>(src + (b & ~1));  // cells of agents b & ~1, b | 1
        const uint32_t v0 = (b & 1) ? (vv >> 16) : (vv & 0xffffu);
        const uint32_t v1 = !two ? 0u : ((b & 1) ? (uint32_t)src[b + 1] : (vv >> 16));
        const Words3 p = stream_observer<A, TB, HI, W2>(T, Q, v0 & 0x7fffu, sh, R, tw, seenf);
        uint64_t* o = T.ob + W * (b - T.ai0);
        if (two) {
            const Words3 q = stream_observer<A, TB, HI, W2>(T, Q, v1 & 0x7fffu, sh, R, tw, seenf);
            if (!W2) {
                store_two(o, p, q);
            } else {
                store_one<W2>(o, p);
                store_one<W2>(o + W, q);
            }
            if (T.unp) {
                if (W2) {
                    unpack_planes_wide(T.unp + T.slot[b].unp_rel, p, DD);
                    unpack_planes_wide(T.unp + T.slot[b + 1].unp_rel, q, DD);
                } else {
                    unpack_planes(T.unp + T.slot[b].unp_rel, p.o0, p.al, p.op, DD);
                    unpack_planes(T.unp + T.slot[b + 1].unp_rel, q.o0, q.al, q.op, DD);
                }
            }
        } else {
            store_one<W2>(o, p);
            if (T.unp) {
                if (W2)
                    unpack_planes_wide(T.unp + T.slot[b].unp_rel, p, DD);
                else
                    unpack_planes(T.unp + T.slot[b].unp_rel, p.o0, p.al, p.op, DD);
            }
        }
    }
}

// The group's shared-memory layout as the emission uses it, in registers.
struct EmitPlan {
    const uint32_t* ring;  // trajectory records [ring][n_envs][rec_words]
    const uint32_t* prist; // pristine records [n_envs][rec_words]
    const uint64_t* base;  // shared memory as uint64 (tables and rows by offset)
    uint32_t ring_mask, n_envs;
};

// One (step k, env e) item: observations, rewards, done byte (and the
// optional unpacked observation and true state).  sl: its ring slot.
template <int A, bool W2>
__device__ __forceinline__ void stream_item(const StepParams& P, const StreamShared& H, const EmitPlan& U,
                                            uint32_t k, uint32_t e, uint32_t sl, uint8_t* stage_item) {
    constexpr int NS = (A + 1) / 2, NW = (A + 3) / 4;
    constexpr uint32_t RW = stream_rec_words(A);
    const EnvRT E = H.env[e];      // register copies: no later store can alias them
    const uint4 ee = H.emit_env[e];
    const uint32_t sh = cell_shift(E), xm2 = ((1u << sh) - 1u) * 0x00010001u;
    Cells<A> Q;
    const uint32_t* rec = U.ring + ((k & U.ring_mask) * U.n_envs + e) * RW;
    const bool done = load_record<A>(rec, sh, xm2, Q);
    const uint32_t rs = E.r_seek, rh = E.r_hide;
    const bool emit_s = team_emits(E, 0), emit_h = A > 1 && team_emits(E, 1);
    uint32_t seen[NW], seen_obs[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) seen[j] = seen_obs[j] = 0u;
    if (done || !emit_s) {
        seen_test<A>(Q, rs, seen);  // the reward's test on the positions before any reset
        if (done) {  // a8: the pristine state is observed
            rec = U.prist + e * RW;
            load_record<A>(rec, sh, xm2, Q);
        }
    }
    const uint16_t* src = reinterpret_cast<const uint16_t*>(rec);
    if (emit_s || emit_h) {
        TeamIn T;
        T.rows = U.base + ee.z;
        T.ob = P.obs + (uint64_t)sl * P.obs_words + E.obs_off;
        // the unpacked planes of agent a go to unp + unp_rel(a): the slot in
        // global memory, or this item's place in the warp's staging area
        T.unp = !P.unp ? nullptr : (stage_item ? stage_item - E.unp_off : P.unp + (uint64_t)sl * P.unp_bytes);
        T.slot = T.unp ? H.slot + H.plan.first_slot[e] : nullptr;
        T.side = E.side;
        T.rw = E.rw;
        if (emit_s) {
            T.tbl = ee.x != ~0u ? U.base + ee.x : nullptr;
            T.ai0 = 0;
            const uint32_t Ds = 2u * rs + 1u;
            if (W2)
                stream_team<A, false, true, true>(T, Q, src, sh, rs, seen_obs);
            else if (Ds * Ds > 32u)
                stream_team<A, false, true, false>(T, Q, src, sh, rs, seen_obs);
            else
                stream_team<A, false, false, false>(T, Q, src, sh, rs, seen_obs);
        }
        if (emit_h) {
            T.tbl = ee.y != ~0u ? U.base + ee.y : nullptr;
            T.ai0 = emit_s ? 0 : NS;
            const uint32_t Dh = 2u * rh + 1u;
            if (W2)
                stream_team<A, true, true, true>(T, Q, src, sh, rh, seen_obs);
            else if (Dh * Dh > 32u)
                stream_team<A, true, true, false>(T, Q, src, sh, rh, seen_obs);
            else
                stream_team<A, true, false, false>(T, Q, src, sh, rh, seen_obs);
        }
    }
    // a6: every seeker gets the number of hiders some seeker sees, each seen
    // hider -1 (bit 7 of the hider bytes)
    int32_t n_seen = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        if (!done && emit_s) seen[j] = seen_obs[j];
        n_seen += __popc(seen[j]);
    }
    auto rew_of = [&](int a) -> int32_t {
        return a < NS ? n_seen : -(int32_t)((seen[a >> 2] >> (8 * (a & 3) + 7)) & 1u);
    };
    int32_t* rw = P.rew + (uint64_t)sl * P.agents + E.agent_off;
    if (!(reinterpret_cast<uintptr_t>(rw) & 7u)) {
#pragma unroll
        for (int a = 0; a + 1 < A; a += 2) gst_i2(rw + a, rew_of(a), rew_of(a + 1));
        if (A & 1) gst_i1(rw + A - 1, rew_of(A - 1));
    } else {
        gst_i1(rw, rew_of(0));
#pragma unroll
        for (int a = 1; a + 1 < A; a += 2) gst_i2(rw + a, rew_of(a), rew_of(a + 1));
        if (!(A & 1)) gst_i1(rw + A - 1, rew_of(A - 1));
    }
    gst_u8(P.done + (uint64_t)sl * P.n_envs + ee.w, done ? 3u : 0u);
    if (P.st_cells) {  // the observed state: cells x | y << 6 and the episode clock after the step
        uint16_t* cl = P.st_cells + (uint64_t)sl * P.agents + E.agent_off;
#pragma unroll
        for (int a = 0; a < A; ++a) {
            const uint32_t sel = 0x4440u | (uint32_t)(a & 3);
            gst_u16(cl + a, __byte_perm(Q.X[a >> 2], 0u, sel) | (__byte_perm(Q.Y[a >> 2], 0u, sel) << 6));
        }
        gst_u32(P.st_ept + (uint64_t)sl * P.n_envs + ee.w, (uint32_t)(((uint64_t)H.ept0[e] + k + 1u) % E.cap));
    }
}

// The emission warp `ei` of M: blocks m = ei, ei + M, ... of 32 items each.
template <int A, bool W2>
__device__ __forceinline__ void stream_emit(const StepParams& P, StreamShared& H, const uint8_t* sm, int ei, int M, int lane,
                            uint64_t T0) {
    const GroupPlan& L = H.plan;
    const uint32_t ne = L.n_envs, n = P.n_steps;
    const uint32_t n_items = n * ne;
    EmitPlan U;
    U.ring = reinterpret_cast<const uint32_t*>(sm + L.traj);
    U.prist = reinterpret_cast<const uint32_t*>(sm + L.prist);
    U.base = reinterpret_cast<const uint64_t*>(sm);
    U.ring_mask = L.ring - 1u;
    U.n_envs = ne;
    const uint32_t n_dyn_g = L.n_dyn;
    uint8_t* const stage =
        (L.flags & kUnpStage) && P.unp ? const_cast<uint8_t*>(sm) + L.stage + (uint32_t)ei * L.stage_bytes : nullptr;
    const uint32_t stride = 32u * (uint32_t)M;
    const uint32_t dk = stride / ne, de = stride % ne;
    uint32_t i = 32u * (uint32_t)ei + (uint32_t)lane;
    uint32_t k = i / ne, e = i % ne;
    const uint32_t ring = P.ring;
    uint32_t sl = (uint32_t)((T0 + k) % ring);
    for (uint32_t m = (uint32_t)ei; 32u * m < n_items; m += (uint32_t)M) {
        const uint32_t k_last = min((32u * m + 31u) / ne, n - 1u);
        if (!wait_min(H.dyn_prog, (int)n_dyn_g, k_last + 1u, lane)) {
            if (lane == 0) atomicOr(P.err, kErrWaitTimeout);
            return;
        }
        // The block's unpacked bytes form one contiguous run per step (envs
        // e_a..e_b of step kk sit at unp_off[e_a] of its slot).  Each run is
        // staged at an offset congruent to its destination mod 16, so that it
        // leaves with 16-byte stores; its items follow one another.
        const uint32_t i0 = 32u * m, last = min(i0 + 31u, n_items - 1u);
        const uint32_t k_a = i0 / ne, k_b = last / ne;
        const uint32_t sl_a = __shfl_sync(0xffffffffu, sl, 0);  // slot of step k_a (lane 0 holds item i0)
        auto run_dst = [&](uint32_t kk, uint32_t e_a) {
            uint32_t sl_k = sl_a + (kk - k_a);  // kk - k_a <= 32 < ring: one wrap at most
            if (sl_k >= ring) sl_k -= ring;
            return P.unp + (uint64_t)sl_k * P.unp_bytes + H.env[e_a].unp_off;
        };
        uint8_t* stage_item = nullptr;
        if (stage && i < n_items) {
            uint32_t off = 0;
            for (uint32_t kk = k_a; kk <= k; ++kk) {
                const uint32_t first = max(i0, kk * ne), end = min(last + 1u, (kk + 1u) * ne);
                off += ((uint32_t)reinterpret_cast<uintptr_t>(run_dst(kk, first - kk * ne)) - off) & 15u;
                if (kk == k) stage_item = stage + off + (i - first) * L.unp_env;
                off += (end - first) * L.unp_env;
            }
        }
        if (i < n_items) stream_item<A, W2>(P, H, U, k, e, sl, stage_item);
        __syncwarp();  // every lane has read its record (and staged its bytes)
        if (stage) {
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
                if ((uint32_t)lane < head) gst_u8(g + lane, src[lane]);
                for (uint32_t c = (uint32_t)lane; c < body; c += 32u)
                    st_cs_v4(g + head + 16u * c, *reinterpret_cast<const uint4*>(src + head + 16u * c));
                if ((uint32_t)lane < len - tail0) gst_u8(g + tail0 + lane, src[tail0 + lane]);
                off += len;
            }
            __syncwarp();  // the staging area is read before the next block writes it
        }
        if (lane == 0) store_release(H.emit_prog + ei, min(n, (32u * (m + (uint32_t)M)) / ne));
        i += stride;
        e += de;
        k += dk;
        sl += dk;
        if (e >= ne) {
            e -= ne;
            ++k;
            ++sl;
        }
        if (sl >= ring) sl = (uint32_t)((T0 + k) % ring);
    }
    if (lane == 0) store_release(H.emit_prog + ei, n);
}

template <int FAM>
__device__ __forceinline__ void stream_emit_dispatch(int A, const StepParams& P, StreamShared& H, const uint8_t* sm,
                                                     int ei, int M, int lane, uint64_t T0) {
    constexpr int a0 = 4 * ((FAM - 1) % 4) + 1;
    constexpr bool W2 = FAM >= 5;
    if (A == a0)
        stream_emit<a0, W2>(P, H, sm, ei, M, lane, T0);
    else if (A == a0 + 1)
        stream_emit<a0 + 1, W2>(P, H, sm, ei, M, lane, T0);
    else if (A == a0 + 2)
        stream_emit<a0 + 2, W2>(P, H, sm, ei, M, lane, T0);
    else
        stream_emit<a0 + 3, W2>(P, H, sm, ei, M, lane, T0);
}

template <int MAXT, int FAM>
__global__ void __launch_bounds__(MAXT, 1) stream_kernel(const StepParams P) {
    static_assert(FAM >= 1 && FAM <= 8, "streaming form: families 1-8");
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ StreamShared H;
    const Group G = P.groups[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    const int ne = G.n_envs, nsl = G.n_slots;
    const int n_dyn = (int)P.n_dyn;  // dynamics warps of the launch (>= the group's)
    const int M = (int)P.emit_warps;

    if (tid == 0) {
        int slot = 0;
        for (int i = 0; i < ne; ++i) {
            const uint32_t g = P.env_list[G.list_first + i];
            const EnvRT E = P.env[g];
            H.env[i] = E;
            H.gidx[i] = g;
            H.ept0[i] = P.st_ept ? P.est[g].ep_t : 0u;
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
        plan_stream(H.env, ne, G.flags, H.plan);
        const GroupPlan& L0 = H.plan;
        const uint32_t tb = L0.tbl / 8u, ro = L0.rows / 8u;
        for (int i = 0; i < ne; ++i) {
            const bool tab = (G.flags & kUseTable) != 0;
            H.emit_env[i] = make_uint4(tab && L0.tbl_off[i][0] != ~0u ? tb + L0.tbl_off[i][0] : ~0u,
                                       tab && L0.tbl_off[i][1] != ~0u ? tb + L0.tbl_off[i][1] : ~0u,
                                       ro + L0.rows_off[i], H.gidx[i]);
        }
    }
    if (tid < kMaxDyn) H.dyn_prog[tid] = 0u;
    if (tid == 0) H.act_prog = 0u;
    // an emission warp has read every step before its first block
    if (tid < kMaxEmitWarps) H.emit_prog[tid] = min(P.n_steps, (32u * (uint32_t)tid) / (uint32_t)ne);
    __syncthreads();
    if (H.plan.total > dynamic_smem_bytes()) {  // the host sized the launch by the same plan: cannot happen
        if (tid == 0) atomicOr(P.err, kErrSmemPlan);
        return;  // the whole CTA (H.plan is shared)
    }
    const GroupPlan& L = H.plan;
    const bool use_table = L.flags & kUseTable;
    uint64_t* s_rows = reinterpret_cast<uint64_t*>(sm + L.rows);
    uint8_t* s_state = sm + L.state;
    uint64_t* s_tbl = reinterpret_cast<uint64_t*>(sm + L.tbl);
    uint16_t* s_prist = reinterpret_cast<uint16_t*>(sm + L.prist);
    uint16_t* s_traj = reinterpret_cast<uint16_t*>(sm + L.traj);
    uint32_t* s_claim = reinterpret_cast<uint32_t*>(sm + L.claim);  // per cell: claim bytes, 0xff = none
    uint16_t* s_scr = H.scratch;
    const uint32_t rec16 = 2u * L.rec_words;  // uint16 entries of one record

    // the pristine template: padded rows and start cells
    for (int i = 0; i < ne; ++i) {
        const EnvRT& E = H.env[i];
        const uint32_t nr = (uint32_t)(E.side + 2 * kPad) * E.rw;
        for (uint32_t j = tid; j < nr; j += nthreads) s_rows[L.rows_off[i] + j] = P.rows[E.rows_off + j];
    }
    for (uint32_t j = tid; j < (uint32_t)ne * rec16; j += nthreads) s_prist[j] = 0;
    __syncthreads();
    for (int sidx = tid; sidx < nsl; sidx += nthreads) {
        const SlotRec& r = H.slot[sidx];
        const EnvRT& E = H.env[r.env];
        const uint16_t p0 = (uint16_t)to_cta(P.start[E.agent_off + r.agent], cell_shift(E));
        H.slot[sidx].p0 = p0;
        const uint2 kk = P.keys[H.gidx[r.env]];
        H.key[sidx] = make_uint4(r.agent, E.env_id, kk.x, kk.y);
        s_prist[r.env * rec16 + r.agent] = p0;
    }
    // state bytes (free neighbours) and window tables
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
    __syncthreads();

    const uint64_t T0 = *P.clock + P.t0;  // global step index of the launch's first step
    const uint32_t n = P.n_steps;
    int d = -1, nbelow = 0;  // this warp's dynamics index; dynamics and action warps with a smaller id
    for (int q = 0; q < n_dyn; ++q) {
        const int id = (int)((P.dyn_ids >> (4 * q)) & 15u);
        if (id == warp) d = q;
        if (id < warp) ++nbelow;
    }
    const int act_warp = (int)((P.dyn_ids >> 16) & 15u);
    if (act_warp < warp) ++nbelow;
    const uint32_t* s_act_ring = reinterpret_cast<const uint32_t*>(sm + L.act);
    const uint32_t q0 = (uint32_t)(T0 >> 2), n_quads = (uint32_t)((T0 + n + 3u) >> 2) - q0;

    if (warp == act_warp) {
        // ================= actions: a1 =================
        // Quads [4c, 4c + 4) of slot s: word (quad mod kActRing) * slots + s;
        // byte j of a word is step 4 (q0 + quad) + j.  A chunk overwrites the
        // quads kActRing earlier once every dynamics warp has passed them.
        uint32_t* ring = reinterpret_cast<uint32_t*>(sm + L.act);
        const uint32_t ns = L.n_slots;
        const uint32_t ring_ag = P.ring;
        for (uint32_t c = 0; 4u * c < n_quads; ++c) {
            const uint32_t r0 = 4u * c, r1 = min(r0 + 4u, n_quads);
            if (r1 > kActRing) {  // quads r1 - 1 - kActRing and before are free once their steps are done
                const uint64_t t_free = 4ull * (q0 + (r1 - kActRing)) - T0;
                if (!wait_min(H.dyn_prog, (int)L.n_dyn, t_free < n ? (uint32_t)t_free : n, lane)) {
                    if (lane == 0) atomicOr(P.err, kErrWaitTimeout);
                    return;
                }
            }
            const uint32_t items = (r1 - r0) * ns;
            for (uint32_t it = (uint32_t)lane; it < items; it += 64u) {
                const uint32_t it2 = it + 32u;
                const bool two = it2 < items;
                const uint32_t ja = it / ns, sa = it - ja * ns;
                const uint32_t jb = two ? it2 / ns : ja, sb = two ? it2 - jb * ns : sa;
                const uint4 ka = H.key[sa], kb = H.key[sb];
                uint32_t a0 = q0 + r0 + ja, a1 = ka.x, a2 = ka.y, a3 = 0u;
                uint32_t b0 = q0 + r0 + jb, b1 = kb.x, b2 = kb.y, b3 = 0u;
                philox4x32_10(a0, a1, a2, a3, ka.z, ka.w);
                philox4x32_10(b0, b1, b2, b3, kb.z, kb.w);
                const uint32_t wa = mulhi_n(a0, 5u) | (mulhi_n(a1, 5u) << 8) | (mulhi_n(a2, 5u) << 16) |
                                    (mulhi_n(a3, 5u) << 24);
                const uint32_t wb = mulhi_n(b0, 5u) | (mulhi_n(b1, 5u) << 8) | (mulhi_n(b2, 5u) << 16) |
                                    (mulhi_n(b3, 5u) << 24);
                ring[((r0 + ja) & (kActRing - 1u)) * ns + sa] = wa;
                if (two) ring[((r0 + jb) & (kActRing - 1u)) * ns + sb] = wb;
                if (P.act_out) {  // the action export: the steps of the quad inside the launch
                    for (int h = 0; h < 2; ++h) {
                        if (h && !two) break;
                        const uint32_t jj = h ? jb : ja, ss = h ? sb : sa, w = h ? wb : wa;
                        const SlotRec& rr = H.slot[ss];
                        const uint64_t tq = 4ull * (q0 + r0 + jj);
                        for (uint32_t b = 0; b < 4; ++b) {
                            const uint64_t tt = tq + b;
                            if (tt < T0 || tt >= T0 + n) continue;
                            gst_u8(P.act_out + (tt % ring_ag) * P.agents + H.env[rr.env].agent_off + rr.agent,
                                   (w >> (8 * b)) & 0xffu);
                        }
                    }
                }
            }
            store_release_lane0(&H.act_prog, r1, lane);
        }
        return;
    }

    if (d >= 0) {
        // ================= dynamics: a1 a2 a3 a7 a8 =================
        if (d >= (int)L.n_dyn) return;  // no envs of this group (the emission waits on the group's warps only)
        const int d_first = L.dyn_first[d], d_end = L.dyn_first[d + 1];
        const int s = d_first + lane;
        const bool live = s < d_end;
        uint32_t p = 0, p0 = 0, nbr = 0, nbr0 = 0, ep_idx = 0, cap = 1, sh = 5, agent = 0;
        uint32_t next_done = 0xffffffffu;
        int env = 0;
        uint8_t* st8 = s_state;
        uint8_t* cl8 = reinterpret_cast<uint8_t*>(s_claim);
        uint16_t* rec = s_scr + 32 * d + lane;  // dead lanes: scratch
        if (live) {
            const SlotRec& r = H.slot[s];
            env = r.env;
            agent = r.agent;
            const EnvRT& E = H.env[env];
            sh = cell_shift(E);
            st8 = s_state + L.cell_off[env];
            cl8 = reinterpret_cast<uint8_t*>(s_claim + L.cell_off[env]);
            p = to_cta(P.pos[E.agent_off + r.agent], sh);
            p0 = r.p0;
            nbr = st8[p] & 0x1eu;
            nbr0 = st8[p0] & 0x1eu;
            const EnvState est = P.est[H.gidx[env]];
            ep_idx = est.ep_idx;
            cap = E.cap;
            next_done = cap - 1u - est.ep_t;
            rec = s_traj + env * rec16 + agent;
        }
        const uint32_t lane_rep = 0x01010101u * (uint32_t)lane;
        uint32_t warp_next = __reduce_min_sync(0xffffffffu, next_done);
        const uint32_t dn = 1u << sh;
        const uint32_t dlut = (64u - dn) | ((64u + dn) << 8) | (65u << 16) | (63u << 24);
        const uint32_t slot_stride = (uint32_t)ne * rec16;  // uint16 entries of one ring slot
        const bool agent0 = agent == 0u;
        const uint32_t ring_mask = live ? L.ring - 1u : 0u, ring_steps = L.ring;
        // shared-window addresses: claim words, state bytes, this lane's record
        // column, and its scratch claim and state bytes
        const uint32_t cl_a = smem_addr(cl8), st_a = smem_addr(st8), rec_a = smem_addr(rec);
        const uint32_t cl_scr = smem_addr(reinterpret_cast<uint8_t*>(s_scr + 128) + 4 * (32 * d + lane));
        const uint32_t st_scr = cl_scr + 2u;
        bool ok = true;

        // One step of this lane: claim, read, resolve, update, record (and, in
        // the rare step where some env of the warp ends its episode, the
        // reset).  Branch-free except for that warp-uniform case: a lane with
        // nothing to claim, read or write addresses its own scratch bytes.
        // ENDS: the step may end an episode; a quad that ends none runs the
        // step without the check (with its warp barriers it cost ~30 cycles
        // a step even when not taken).
        auto step = [&](uint32_t a, uint32_t g, auto ends) {
            constexpr bool ENDS = decltype(ends)::value;
            const uint32_t dd = __byte_perm(dlut, 0, 0x4440u | ((a + 3u) & 3u)) - 64u;
            const uint32_t tgt = p + dd;
            const bool open = (nbr >> a) & 1u;  // inside the grid, no obstacle (a = 0: never)
            const uint32_t cb = open ? cl_a + tgt * 4u + a - 1u : cl_scr;  // claim byte of direction a
            sts8(cb, lane);
            __syncwarp();
            const uint32_t rd = open ? tgt : p;  // the own cell when not moving (never won)
            const uint32_t claims = lds32(cl_a + rd * 4u);
            const uint32_t tst = lds8(st_a + rd);
            const uint32_t lower = ~((claims | 0x80808080u) - lane_rep) & 0x80808080u;
            const bool won = open && ((tst & kOccBit) | lower) == 0u;
            __syncwarp();  // every read of this step is done
            sts8(cb, 0xffu);  // release the claim
            sts8(won ? st_a + p : st_scr, nbr);
            sts8(won ? st_a + tgt : st_scr, tst | kOccBit);
            p = won ? tgt : p;
            nbr = won ? (tst & 0x1eu) : nbr;
            sts16(rec_a + 2u * ((g & ring_mask) * slot_stride), p | ((ENDS && g == next_done && agent0) ? 0x8000u : 0u));
            if (ENDS && g == warp_next) {  // some env of this warp ends its episode (a8)
                const bool done = g == next_done;
                __syncwarp();
                if (done) sts8(st_a + p, nbr);
                __syncwarp();
                if (done) {
                    sts8(st_a + p0, nbr0 | kOccBit);
                    p = p0;
                    nbr = nbr0;
                    next_done += cap;
                    ++ep_idx;
                }
                warp_next = __reduce_min_sync(0xffffffffu, next_done);
            }
            __syncwarp();  // state writes visible to the next step
        };

        // The action word of each quad (four steps) comes from the action
        // warp's ring; the progress is published, and the rings checked,
        // every kStreamGroup steps.
        const uint32_t act_a = smem_addr(s_act_ring) + 4u * (uint32_t)min(s, nsl - 1);
        const uint32_t act_row = 4u * L.n_slots;
        uint32_t g = 0, sync_at = 0;
        uint64_t t = T0;
        uint32_t qr = 0;  // quad of step t, counted from the launch's first
        while (g < n) {
            if (g >= sync_at) {
                if (g) store_release_lane0(H.dyn_prog + d, g, lane);  // the records of steps < g are written
                // the ring slots of the steps up to the next check must have been read, and
                // their actions drawn
                const uint32_t span = min(kStreamGroup + 3u, n - g);
                const uint32_t need_q = min(n_quads, (uint32_t)(((t + span + 3u) >> 2) - q0));
                if ((g + span > ring_steps && !wait_min(H.emit_prog, M, g + span - ring_steps, lane)) ||
                    !wait_min(&H.act_prog, 1, need_q, lane)) {
                    if (lane == 0) atomicOr(P.err, kErrWaitTimeout);
                    ok = false;
                    break;
                }
                sync_at = g + kStreamGroup;
            }
            const uint32_t cur = lds32(act_a + (qr & (kActRing - 1u)) * act_row);
            const uint32_t j0 = (uint32_t)(t & 3u), len = min(4u - j0, n - g);
            if (len == 4u && warp_next - g >= 4u) {  // no episode ends in this quad (warp-uniform)
#pragma unroll
                for (uint32_t j = 0; j < 4; ++j) step((cur >> (8 * j)) & 0xffu, g + j, std::false_type{});
            } else if (len == 4u) {
#pragma unroll
                for (uint32_t j = 0; j < 4; ++j) step((cur >> (8 * j)) & 0xffu, g + j, std::true_type{});
            } else {
#pragma unroll 1
                for (uint32_t j = 0; j < len; ++j) step((cur >> (8 * (j0 + j))) & 0xffu, g + j, std::true_type{});
            }
            g += len;
            t += len;
            ++qr;
        }
        if (ok) store_release_lane0(H.dyn_prog + d, g, lane);
        // write back the dynamic state
        if (ok && live) {
            const SlotRec& r = H.slot[s];
            const EnvRT& E = H.env[env];
            P.pos[E.agent_off + r.agent] = (uint16_t)to_hbm(p, sh);
            if (r.agent == 0) {
                EnvState est;
                est.ep_t = cap - 1u - (next_done - n);
                est.ep_idx = ep_idx;
                P.est[H.gidx[env]] = est;
            }
        }
        return;
    }
    // ================= emission: a4 a5 a6 a9 =================
    const int ei = warp - nbelow;
    stream_emit_dispatch<FAM>(H.env[0].n_agents, P, H, sm, ei, M, lane, T0);
}

}  // namespace hase
