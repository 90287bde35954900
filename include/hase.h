/*
 * hase.h -- C ABI of the GB300-native batched hide-and-seek environment step
 * (Hide-And-Seek-Engine, arxiv 2604.27162).
 *
 * One handle owns a batch of independent grid environments resident in GPU
 * memory.  hase_step advances every environment by n steps on the caller's
 * CUDA stream; each step performs, per environment and agent (paper Sec. 3.1
 * Dec-POMDP with per-agent actions, observations and rewards):
 *   a1  random actions: Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *       seed, counter (t >> 2, agent, env, 0), word t & 3, mapped to
 *       {0 stay, 1 N, 2 S, 3 E, 4 W} as floor(u * 5 / 2^32)  [Sec. 4.1]
 *   a2  move proposal on the grid; blocking tiles are impassable [Sec. 3.2]
 *   a3  collisions: a move into any currently occupied cell is blocked; of
 *       the valid movers with one target the lowest agent index moves
 *   a5  decentralized observation [Sec. 3.3, mode 1]: a (2r+1)^2 window
 *       centred on the agent, three planes (0 obstacle or outside the grid,
 *       1 ally other than the agent itself, 2 opponent), window cell
 *       (dx, dy) at bit k = (dy + r)(2r + 1) + (dx + r), LSB first, plane p
 *       in words [p*W, (p+1)*W) with W = ceil((2 r_max + 1)^2 / 64)
 *   a6  reward: every seeker gets +(number of hiders within Chebyshev
 *       distance r_seek of some seeker), every such hider -1
 *   a7  episode counter, truncation at the cap (done byte = 3: bit 0 done,
 *       bit 1 truncated)
 *   a8  same-step auto-reset to the pristine start cells [Sec. 4.2]; the
 *       step's reward and done describe the finished step, its observation
 *       the reset state.
 * Creation (a0) draws each env's start cells (counter (attempt, agent, env,
 * 2), word 0, cell floor(u * S^2 / 2^32), redrawn while taken) and obstacles
 * (cell c blocked iff word c%4 of counter (c/4, 0, env, 1) < density_thr),
 * start cells forced free.
 *
 * Memory: every buffer lives in device memory and is owned by the handle.
 * Outputs of global step t (0-based, counted since create or reset) sit in
 * ring slot t mod ring_steps; the observation of the state after create or
 * reset ("step -1") sits in slot ring_steps - 1 with zero reward and done.
 * Layout of one slot (hase_layout gives the sizes and per-env offsets):
 *   obs      uint64 [obs_words]  env e at obs_off[e]: [A_obs(e)][3][W(e)]
 *   reward   int32  [agents]     env e at agent_off[e]: [A(e)]
 *   done     uint8  [n_envs]
 *   actions  uint8  [agents]     (only with HASE_EXPORT_ACTIONS)
 *   unpacked uint8  [unp_bytes]  env e at unp_off[e]: [A_obs][3][2r+1][2r+1]
 *                                (only with HASE_EXPORT_UNPACKED)
 *   central  uint64 [central_words] env e at central_off[e]: [4][S]
 *                                (only with HASE_EXPORT_CENTRAL)
 *   cells    uint16 [agents]     env e at agent_off[e]: the cell x | y << 6
 *                                of every agent (only with HASE_EXPORT_STATE)
 *   ep_t     uint32 [n_envs]     steps into the current episode
 *                                (only with HASE_EXPORT_STATE)
 *   fog      uint64 [fog_words]  env e at fog_off[e]: [U(e)][2][S]
 *                                (only with HASE_EXPORT_FOG)
 * A_obs(e) counts the agents whose team emits observations (seekers first).
 * Pointers returned by the *_ptr calls stay valid until hase_destroy; their
 * contents are valid once the stream work that wrote them has completed.
 *
 * Errors: every call returns a hase_status; the message of the last failure
 * on a handle is returned by hase_last_error (creation failures by
 * hase_last_error(NULL)).  No call throws across the ABI.  Launches are
 * asynchronous: device-side faults surface on a later call or hase_sync as
 * HASE_ECUDA.
 */
#ifndef HASE_H
#define HASE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hase_status {
    HASE_OK = 0,
    HASE_EINVAL = 1,   /* invalid argument or configuration             */
    HASE_ENOMEM = 2,   /* device or host allocation failed              */
    HASE_ECUDA = 3,    /* a CUDA runtime call failed                    */
    HASE_ETIMEOUT = 4, /* a bounded wait ran out (hase_sync after the   */
                       /* streaming step kernel; hase_server_poll)      */
    HASE_EBUSY = 5,    /* hase_server_submit: the queue is full         */
    HASE_ESTATE = 6    /* the server was shut down (hase_server_*)      */
} hase_status;

/* Limits of this implementation (checked at create). */
#define HASE_MAX_SIDE 64
#define HASE_MAX_AGENTS 32
#define HASE_MAX_RADIUS 4

/* Configuration flags. */
#define HASE_EXPORT_ACTIONS 1u  /* keep the actions of every step          */
#define HASE_EXPORT_UNPACKED 2u /* also write the uint8 unpacked obs       */
#define HASE_ASYNC_CREATE 4u    /* hase_create does not wait for the world   */
                                /* generation; a failed start-cell draw is   */
                                /* reported by hase_sync and hase_digest     */
#define HASE_EXPORT_CENTRAL 32u /* also write the centralized observation   */
                                /* [Sec. 3.3, mode 3]: per env four planes   */
                                /* over its grid -- 0 cells inside some      */
                                /* observing agent's window (visible to it   */
                                /* with HASE_OBS_LOS), 1 seen obstacles,     */
                                /* 2 seen seekers, 3 seen hiders -- each S   */
                                /* rows of one uint64 (bit x = column x)     */
#define HASE_DESYNC_START 16u  /* desynchronised start [Sec. 3.3, last    */
                                /* paragraph: stepped stochastically at      */
                                /* initialisation]: env e takes o_e =        */
                                /* floor(u * cap / 2^32) moves from its      */
                                /* start cells before its first observation, */
                                /* u = word 0 of Philox counter (0, 0, env,  */
                                /* 3); move tau draws word tau % 4 of        */
                                /* counter (tau / 4, agent, env, 4); its     */
                                /* episode clock starts at o_e (its first    */
                                /* episode ends cap - o_e steps later), at   */
                                /* create and at every hase_reset            */
#define HASE_EXPORT_STATE 64u  /* also write the true state [Sec. 3.3,      */
                                /* modes 2, 4, 5]: after every step the cell */
                                /* of every agent and the episode clock of   */
                                /* every env (the observed state: on a done  */
                                /* step, the reset one)                      */
#define HASE_SKIP_OBS 128u      /* write no decentralized observation        */
                                /* (obs_words = 0) [Sec. 3.3, modes 3-6];    */
                                /* obs_teams still chooses whose sightlines  */
                                /* feed HASE_EXPORT_CENTRAL.  Modes: 1 none, */
                                /* 2 EXPORT_STATE, 3 SKIP_OBS|EXPORT_CENTRAL,*/
                                /* 4 3 + EXPORT_STATE, 5 SKIP_OBS|EXPORT_    */
                                /* STATE, 6 SKIP_OBS (rewards and done only) */
#define HASE_EXPORT_FOG 256u    /* also write the fog of war [Sec. 3.3, the  */
                                /* discovery-map layer of Sec. 4, the diff   */
                                /* sweep of Sec. 5]: a cell is discovered    */
                                /* once an observing agent of the unit has   */
                                /* seen it (in its window; visible with      */
                                /* HASE_OBS_LOS) in the current episode.     */
                                /* Per env U units -- 1 (all observing       */
                                /* agents) or, with HASE_FOG_PER_AGENT, one  */
                                /* per observing agent, seekers first --     */
                                /* each two planes of S rows (bit x =        */
                                /* column x): discovered, newly discovered   */
                                /* in this step.  A reset starts a new map.  */
#define HASE_FOG_PER_AGENT 512u /* one fog unit per observing agent          */
#define HASE_CHUNKED_STEP 1024u /* step kernel forms (identical outputs):    */
#define HASE_STREAM_STEP 2048u  /* chunked -- all warps of a CTA meet at a   */
                                /* barrier every chunk of steps -- or        */
                                /* streaming -- the dynamics write an on-chip */
                                /* trajectory ring that the output warps read */
                                /* behind progress counters.  The streaming  */
                                /* form applies to seekers = ceil(A/2), no   */
                                /* line of sight, no HASE_EXPORT_CENTRAL or  */
                                /* HASE_EXPORT_FOG, ring_steps >= 160; by    */
                                /* default it runs when the batch needs more */
                                /* CTAs than the GPU has SMs.  These flags   */
                                /* force one form (not both)                 */
#define HASE_POOL_ALLOC 8u      /* buffers from the device's stream-ordered  */
                                /* pool (allocated on the create stream,     */
                                /* returned by hase_destroy on the stream of */
                                /* the handle's last call)                   */

/* Observation emitters (hase_env_desc.obs_teams). */
#define HASE_OBS_SEEKERS 1u
#define HASE_OBS_HIDERS 2u
#define HASE_OBS_LOS 4u     /* line of sight [Sec. 3.1]: a window cell is seen   */
                            /* iff every cell strictly between it and the agent  */
                            /* on the discrete line (rnd(i dx/n), rnd(i dy/n)),  */
                            /* i = 1..n-1, n = max(|dx|,|dy|), rnd rounding      */
                            /* halves away from zero, is in the grid and free;   */
                            /* unseen cells read 0 in all three planes           */

/* One environment's parameters.  Seekers are agents 0..n_seekers-1, hiders
 * n_seekers..n_agents-1.  obs_teams = 0 writes no observation and feeds no
 * centralized one (with no HASE_EXPORT_STATE: the paper's "void output"
 * mode). */
typedef struct hase_env_desc {
    uint32_t side;        /* grid side S, 2..HASE_MAX_SIDE                   */
    uint32_t n_agents;    /* A, 1..HASE_MAX_AGENTS, A <= S*S                 */
    uint32_t n_seekers;   /* 0..A                                            */
    uint32_t r_seek;      /* seeker view radius 0..HASE_MAX_RADIUS           */
    uint32_t r_hide;      /* hider view radius 0..HASE_MAX_RADIUS            */
    uint32_t cap;         /* episode length (steps), 1..2^31-1               */
    uint32_t density_thr; /* obstacle iff Philox word < density_thr          */
    uint32_t obs_teams;   /* HASE_OBS_SEEKERS | HASE_OBS_HIDERS              */
} hase_env_desc;

typedef struct hase_config {
    uint32_t n_envs;             /* number of environments >= 1                */
    uint32_t env_id_base;        /* global index of env 0 (Philox counters)    */
    uint64_t seed;               /* Philox key = (seed & 0xffffffff, seed>>32) */
    const hase_env_desc *envs;   /* host array of n_desc descriptors           */
    uint32_t n_desc;             /* 1 (broadcast) or n_envs                    */
    uint32_t ring_steps;         /* output ring length in steps >= 1           */
    uint32_t flags;              /* HASE_EXPORT_*                              */
    uint32_t steps_per_launch;   /* steps fused per kernel launch, 0 = auto    */
    uint32_t chunk_steps;        /* steps per on-chip chunk (1..64), 0 = auto  */
    uint32_t emit_warps;         /* output warps per CTA (1..12), 0 = auto     */
    uint32_t max_group_envs;     /* envs packed per CTA (1..64), 0 = auto      */
    uint32_t smem_cap;           /* dynamic shared memory per CTA in bytes     */
                                 /* (16384..221184), 0 = 221184: smaller caps  */
                                 /* pack fewer envs per CTA and drop window    */
                                 /* tables, so that more CTAs fit on an SM     */
    const uint64_t *env_seeds;   /* NULL, or one Philox seed per env (host     */
                                 /* array of n_envs): env e draws with its own */
                                 /* key instead of `seed`                      */
    const uint32_t *env_ids;     /* NULL, or the env id of every env in the    */
                                 /* Philox counters (host array of n_envs)     */
                                 /* instead of env_id_base + e.  With both, one */
                                 /* handle holds envs of several independent  */
                                 /* runs, each bit for bit as if run alone     */
} hase_config;

/* Sizes and per-env offsets of one ring slot.  The offset arrays are host
 * arrays owned by the handle (n_envs + 1 entries each, valid until
 * hase_destroy). */
typedef struct hase_layout {
    uint32_t n_envs;
    uint32_t ring_steps;
    uint64_t agents;         /* reward / action entries per slot            */
    uint64_t obs_words;      /* uint64 observation words per slot           */
    uint64_t unp_bytes;      /* unpacked observation bytes per slot         */
    const uint64_t *agent_off;
    const uint64_t *obs_off;
    const uint64_t *unp_off;
    uint64_t central_words;  /* centralized observation words per slot     */
    const uint64_t *central_off; /* env e at central_off[e]: [4][side] words */
    uint64_t fog_words;      /* fog-of-war words per slot                   */
    const uint64_t *fog_off; /* env e at fog_off[e]: [U][2][side] words     */
} hase_layout;

typedef struct hase_handle hase_handle;

/* Summary of a run of steps (hase_digest), all exact integers. */
typedef struct hase_digest_out {
    uint64_t digest;     /* sum mod 2^64 over steps s and obs words j of     */
                         /* splitmix64(obs[s][j] ^ (s * obs_words + j))     */
    uint64_t episodes;   /* done bits over the steps and envs                */
    int64_t reward_sum;  /* rewards over the steps and agents                */
    uint32_t gen_error;  /* the handle's error word, 0 = none: bit 0 the     */
                         /* world generation failed, bit 1 a bounded wait of */
                         /* the streaming step ran out, bit 2 a CTA's shared-*/
                         /* memory plan exceeded its launch (bits 1-2: the   */
                         /* outputs are incomplete)                          */
    uint32_t pad;
} hase_digest_out;

/* Create a batch on the current CUDA device: validates the configuration,
 * allocates every buffer, generates the worlds (a0) and writes the step -1
 * observation, all on `stream` (a cudaStream_t, NULL = legacy default).
 * [Sec. 3.2: a grid world with blocking tiles, here seeded Bernoulli maps;
 * Sec. 4.2: the generated world is kept as the pristine template; Sec. 3.3:
 * a vectorized batch of independent environments.]
 * Returns HASE_EINVAL for a bad configuration, HASE_ENOMEM when device
 * memory runs out, HASE_ECUDA for other CUDA errors; *out is NULL then. */
hase_status hase_create(const hase_config *cfg, void *stream, hase_handle **out);

/* Back to t = 0: start cells, episode counters 0 (with HASE_DESYNC_START:
 * the offsets, and the moves taken before the first observation), step -1
 * observation.  [Sec. 4.2: a reset restores the pristine
 * initial state.] */
hase_status hase_reset(hase_handle *h, void *stream);

/* Enqueue n_steps steps (a1-a9) of every environment on `stream`.
 * Asynchronous; n_steps = 0 is a no-op; HASE_EINVAL when the step counter
 * would pass 2^34.  A bounded wait of the streaming step kernel that ran out
 * is reported later by hase_sync as HASE_ETIMEOUT.  [Sec. 3.1: one
 * transition of the Dec-POMDP -- joint action, next state, per-agent
 * observation and reward; Sec. 3.3: every environment of the batch.] */
hase_status hase_step(hase_handle *h, uint32_t n_steps, void *stream);

/* Device pointers of the output rings (NULL when the output is not kept),
 * owned by the handle, valid until hase_destroy.  [Sec. 4.3: the outputs are
 * exposed in place, without a copy (the paper's zero-copy bridge, here in
 * device memory).]
 *   obs:     packed planes, and the uint8 unpacked ones  [Sec. 3.3, mode 1]
 *   reward:  int32 per agent                             [Sec. 3.1, R]
 *   done:    uint8 per env, 3 on the truncating step     [Sec. 4.2]
 *   actions: uint8 per agent (HASE_EXPORT_ACTIONS)       [Sec. 4.1: random
 *            actions are drawn inside the step] */
hase_status hase_obs_ptr(hase_handle *h, uint64_t **packed, uint8_t **unpacked);
hase_status hase_reward_ptr(hase_handle *h, int32_t **reward);
hase_status hase_done_ptr(hase_handle *h, uint8_t **done);
hase_status hase_actions_ptr(hase_handle *h, uint8_t **actions);
/* The centralized-observation ring (HASE_EXPORT_CENTRAL; NULL without it).
 * [Sec. 3.3, mode 3.] */
hase_status hase_central_ptr(hase_handle *h, uint64_t **central);
/* The true-state rings (HASE_EXPORT_STATE; NULL without it): cells
 * [ring_steps][agents] and ep_t [ring_steps][n_envs].  [Sec. 3.3, modes 2,
 * 4, 5.] */
hase_status hase_state_ptr(hase_handle *h, uint16_t **cells, uint32_t **ep_t);
/* The fog-of-war ring (HASE_EXPORT_FOG; NULL without it).  [Sec. 3.3 and
 * the discovery-map layer of Sec. 4; the newly discovered plane is the diff
 * sweep of Sec. 5.] */
hase_status hase_fog_ptr(hase_handle *h, uint64_t **fog);
/* Sizes and per-env offsets of a ring slot.  [Sec. 4.1: the arena's per-env
 * strides, here per-env offsets into each output.] */
hase_status hase_layout_get(hase_handle *h, hase_layout *out);

/* The same n_steps as one CUDA graph: the first call for a given n_steps
 * captures the launches hase_step would enqueue (on an internal stream) and
 * instantiates them; every call then launches the graph on `stream`.  The
 * kernels read the step counter from device memory, so one graph serves
 * every replay.  The capture allocates host-side graph objects only, and
 * must not itself run inside another stream capture.  Graphs are freed by
 * hase_destroy.  Not in the paper: a launch-overhead device of this engine. */
hase_status hase_step_graph(hase_handle *h, uint32_t n_steps, void *stream);

/* Reduce the outputs of the last n_steps steps (1 <= n_steps <= ring_steps,
 * n_steps <= steps taken), s = 0 being the oldest of them, into *out
 * (device memory, overwritten) and, when agent_rew is not NULL, the
 * per-agent reward sums into agent_rew (device, int64 [agents]).  Enqueued
 * on `stream`; uses the handle's own scratch, so two calls on one handle must
 * not overlap.  splitmix64 is the output function of Steele, Lea and Flood
 * (OOPSLA 2014).  Not in the paper: a result summary for serving and tests. */
hase_status hase_digest(hase_handle *h, uint32_t n_steps, hase_digest_out *out, int64_t *agent_rew,
                        void *stream);

/* hase_digest over steps [first_step, first_step + n_steps) (all still in
 * the ring) of envs [env_first, env_first + env_count): the digest index of
 * an observation word is s * W + j, with W the range's words per slot and j
 * the word's place inside the range, so that envs of several independent
 * runs sharing a handle (hase_config.env_seeds, env_ids) each get the digest
 * of their run alone.  agent_rew: per-agent sums of the range's agents.
 * Same scratch rule as hase_digest.  Not in the paper: the result summary of
 * one served request. */
hase_status hase_digest_range(hase_handle *h, uint64_t first_step, uint32_t n_steps, uint32_t env_first,
                              uint32_t env_count, hase_digest_out *out, int64_t *agent_rew, void *stream);

/* hase_digest without any allocation: the same reduction and results, with
 * the partial sums of its first pass in a fixed device array of the library
 * (256 partial sums of 3 words, 6 KiB) instead of the handle's scratch.  The
 * first pass runs at most 256 blocks that stride over the outputs, so a
 * digest of any length fits the array.  Nothing in that array needs to start
 * at zero (every slot read is written first in the same call).  The first
 * call on a device looks up the array's address (cudaGetSymbolAddress, with
 * the handle's device current) and keeps it for the process: make that call
 * before any stream capture, and not across a cudaDeviceReset of the device
 * (the kept address would then be stale).  Calls that overlap in time -- on
 * any handle or stream of the device -- race on the one array; serialise
 * them.  The paper has no counterpart: a scratch-free form of the run
 * summary for callers that may not allocate. */
hase_status hase_digest_noalloc(hase_handle *h, uint32_t n_steps, hase_digest_out *out, int64_t *agent_rew,
                                void *stream);

/* Steps taken since create / reset (the t of the action counters).
 * [Sec. 3.1: the time index of the transition.] */
hase_status hase_step_count(hase_handle *h, uint64_t *t);

/* Checkpoint: the dynamic state (positions, episode counters, step count,
 * fog-of-war maps) as an opaque host blob.  hase_get_state with buf = NULL
 * stores the size in *size.  Both synchronize `stream`.  Not in the paper
 * (its closest relative is the pristine template of Sec. 4.2). */
hase_status hase_get_state(hase_handle *h, void *buf, size_t *size, void *stream);
hase_status hase_set_state(hase_handle *h, const void *buf, size_t size, void *stream);

/* Read back the pristine obstacle grid of env e (side*side bytes, row
 * major, 1 = obstacle) and the start cells (x, y per agent).  Synchronous.
 * [Sec. 3.2: the generated world.] */
hase_status hase_get_world(hase_handle *h, uint32_t e, uint8_t *grid, int32_t *start_xy);

/* Wait for all work the handle enqueued; HASE_ETIMEOUT when a bounded wait
 * of the streaming step kernel ran out (its outputs are then incomplete),
 * HASE_ECUDA when a CTA found its shared-memory plan larger than its launch
 * and returned without stepping (an internal sizing error: the host sizes
 * every launch by the same plan), HASE_EINVAL when the world generation
 * failed.  Not in the paper. */
hase_status hase_sync(hase_handle *h);

/* Number of CTAs and dynamic shared memory of one step launch, and the
 * fused steps per launch (for reports and the autotuner).  Not in the paper. */
hase_status hase_launch_info(hase_handle *h, uint32_t *ctas, uint32_t *threads,
                             uint32_t *smem_bytes, uint32_t *steps_per_launch);

/* Free every buffer of the handle (NULL: no-op).  Not in the paper. */
void hase_destroy(hase_handle *h);
/* The message of the handle's last failure (NULL: of the last failed
 * hase_create), owned by the library.  Not in the paper. */
const char *hase_last_error(const hase_handle *h);

#ifdef __cplusplus
}
#endif

#endif
