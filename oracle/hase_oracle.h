/*
 * hase_oracle.h -- plain single-threaded C oracle of the batched
 * hide-and-seek environment step (Hide-And-Seek-Engine, arxiv 2604.27162).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this library: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA engine.
 *
 * What it computes (paper section in brackets; open points are fixed by the
 * readings listed in the design notes of the repository):
 *   a0 generation  -- start cells, Bernoulli obstacle grid with the start
 *                     cells forced free, kept as the pristine template
 *                     [Sec. 3.2 blocking tiles; Sec. 4.2 pristine templating]
 *   a1 actions     -- Philox4x32-10 (Salmon et al., SC'11) keyed by the seed,
 *                     counter (t>>2, agent, env, 0), word t&3, mapped to
 *                     {stay,N,S,E,W} by a multiply-shift [Sec. 4.1: random
 *                     actions are part of the step]
 *   a2/a3 moves    -- bounded grid, blocking obstacles, no entry into any
 *                     currently occupied cell, equal targets: lowest index wins
 *                     [Sec. 3.2 collision models]
 *   a5 obs         -- decentralized square window of radius r, three planes
 *                     (obstacle incl. out-of-bounds, ally excl. self,
 *                     opponent), packed LSB-first into uint64 words
 *                     [Sec. 3.3 observability mode 1]
 *   a6 reward      -- +#hiders seen by any seeker to every seeker, -1 to each
 *                     seen hider (Chebyshev distance <= the seeker radius)
 *   a7/a8 done     -- truncation at the episode cap, same-step auto-reset to
 *                     the pristine start cells [Sec. 4.2]
 * Every loop is naive and in index order; there is no bit trick, blocking or
 * reordering beyond what these definitions state.
 */
#ifndef HASE_ORACLE_H
#define HASE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One environment's parameters.  Seekers are agents 0..n_seekers-1, hiders
 * the rest.  obs_teams: bit 0 = seekers emit observations, bit 1 = hiders. */
typedef struct ho_env {
    uint32_t side;        /* grid side S (S x S cells)                        */
    uint32_t n_agents;    /* A                                                 */
    uint32_t n_seekers;   /* 0..A                                              */
    uint32_t r_seek;      /* seeker view radius                                */
    uint32_t r_hide;      /* hider view radius                                 */
    uint32_t cap;         /* episode length in steps (truncation)              */
    uint32_t density_thr; /* cell is an obstacle iff its Philox word < thr     */
    uint32_t obs_teams;   /* bit0 seekers emit obs, bit1 hiders emit obs,      */
                          /* bit2 line of sight masks the windows           */
} ho_env;

typedef struct ho_world ho_world;

/* Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11). */
void ho_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Action of `agent` of global env `env_id` at global step t (0 stay, 1 N,
 * 2 S, 3 E, 4 W). */
uint32_t ho_action(uint64_t seed, uint64_t t, uint32_t agent, uint32_t env_id);

/* Pure transition of one environment (a2+a3): positions x,y (A each), actions
 * act (A each) on an S x S grid (row-major, 1 = obstacle).  Writes the new
 * positions to nx, ny.  Exposed so tests can drive it with chosen actions. */
void ho_move(uint32_t S, const uint8_t *grid, uint32_t A, const int32_t *x,
             const int32_t *y, const uint8_t *act, int32_t *nx, int32_t *ny);

/* Pure reward of one environment (a6) for positions x,y. */
void ho_reward(uint32_t A, uint32_t n_seekers, uint32_t r_seek, const int32_t *x,
               const int32_t *y, int32_t *rew);

/* Pure observation of agent `a` (a5): writes 3*W words (W = words per plane).
 * r is the agent's radius; W must be >= ceil((2r+1)^2 / 64). */
void ho_observe_agent(uint32_t S, const uint8_t *grid, uint32_t A, uint32_t n_seekers,
                      const int32_t *x, const int32_t *y, uint32_t a, uint32_t r,
                      uint32_t W, uint32_t los, uint64_t *out);

/* Line of sight (Section 3.1): window cell (dx, dy) of an agent at (x, y) is
 * visible iff every cell strictly between them on the discrete line is inside
 * the grid and free; the line's cells are (rnd(i dx / n), rnd(i dy / n)),
 * i = 1 .. n-1, n = max(|dx|, |dy|), rnd rounding halves away from zero. */
int ho_visible(uint32_t S, const uint8_t *grid, int32_t x, int32_t y, int32_t dx, int32_t dy);

/* World of n_envs environments with global ids env_id_base + e.  envs holds
 * n_desc entries: 1 (broadcast to every env) or n_envs.  Returns NULL on an
 * invalid parameter (message from ho_error()). */
ho_world *ho_create(uint32_t n_envs, uint32_t env_id_base, uint64_t seed,
                    const ho_env *envs, uint32_t n_desc);
void ho_destroy(ho_world *w);
const char *ho_error(void);

/* Back to t = 0 and the pristine state (start cells, ep_t = 0, episode 0;
 * with the desynchronised start, ep_t = the env's drawn offset). */
void ho_reset(ho_world *w);

/* Centralized observation of the current state (Section 3.3, observability
 * mode 3), every env in order: four planes (0 seen by some observing agent,
 * 1 seen obstacles, 2 seen seekers, 3 seen hiders), each S rows of
 * ceil(S / 64) words, bit x % 64 of word x / 64 of row y = cell (x, y).
 * ho_central_words gives the words of all envs. */
uint64_t ho_central_words(const ho_world *w);
/* The same for one env given its grid and agent cells (out: 4 S ceil(S/64)). */
void ho_central_one(uint32_t side, const uint8_t *grid, uint32_t A, uint32_t n_seekers, uint32_t r_seek,
                    uint32_t r_hide, uint32_t obs_teams, const int32_t *x, const int32_t *y, uint64_t *out);
void ho_central(const ho_world *w, uint64_t *out);

/* Desynchronised start on (1) or off (0), then ho_reset.  With it on, env e
 * takes o_e = floor(u * cap / 2^32) steps of its dynamics from the start
 * cells before its first observation, u = word 0 of the Philox block of
 * counter (0, 0, env id, 3), and its episode clock starts at o_e (Section
 * 3.3, last paragraph). */
void ho_set_desync(ho_world *w, int on);

/* Action of pre-step tau (0 <= tau < o_e) of the desynchronised start: word
 * tau % 4 of the Philox block of counter (tau / 4, agent, env id, 4). */
uint32_t ho_prestep_action(uint64_t seed, uint32_t tau, uint32_t agent, uint32_t env_id);

/* Per-step output sizes: agents (rewards/actions), packed obs words and
 * unpacked obs bytes of one step over all envs. */
void ho_sizes(const ho_world *w, uint64_t *agents, uint64_t *obs_words, uint64_t *unp_bytes);

/* Prefix offsets (n_envs + 1 entries each) of every env inside one step's
 * agent, obs-word and unpacked-byte slices; words_per_plane has n_envs
 * entries. */
void ho_offsets(const ho_world *w, uint64_t *agent_off, uint64_t *obs_off,
                uint64_t *unp_off, uint32_t *words_per_plane);

/* Observation of the current state (the "step -1" observation after create
 * or reset).  unp may be NULL. */
void ho_observe(const ho_world *w, uint64_t *obs, uint8_t *unp);

/* One step of every env at the world's step counter t, then t += 1.
 * Any output pointer may be NULL. */
void ho_step(ho_world *w, uint64_t *obs, int32_t *rew, uint8_t *done, uint8_t *act,
             uint8_t *unp);

/* State read-out for invariant checks.  Positions are per agent (agent_off),
 * counters per env.  Any pointer may be NULL. */
void ho_state(const ho_world *w, int32_t *x, int32_t *y, int32_t *sx, int32_t *sy,
              uint32_t *ep_t, uint32_t *ep_idx, uint64_t *t);

/* Obstacle grid of env e (side*side bytes, row-major). */
/* Fog of war (Sec. 3.3, the discovery-map layer of Sec. 4, the diff sweep
 * of Sec. 5): unit j of an env is the j-th observing agent (per_agent) or
 * all observing agents; a cell is discovered once a unit's agent has seen it
 * in the current episode.  ho_fog_update applies one step to one env's
 * byte maps ([units][side][side]; start != 0 on an episode's first
 * observation); ho_set_fog turns the world's maps on (1 global, 2 per agent)
 * and restarts it; ho_fog packs them per env as [units][2][side] rows
 * (discovered, newly discovered). */
uint32_t ho_fog_units(uint32_t A, uint32_t n_seekers, uint32_t obs_teams, uint32_t per_agent);
void ho_fog_update(uint32_t side, const uint8_t *grid, uint32_t A, uint32_t n_seekers, uint32_t r_seek,
                   uint32_t r_hide, uint32_t obs_teams, uint32_t per_agent, const int32_t *ax,
                   const int32_t *ay, uint32_t start, uint8_t *disc, uint8_t *fresh);
void ho_set_fog(ho_world *w, int mode);
uint64_t ho_fog_words(const ho_world *w);
void ho_fog(const ho_world *w, uint64_t *out);

/* True state of the current step (Sec. 3.3, modes 2, 4, 5): cells[agent] =
 * x | y << 6, ep_t[env] = steps into the current episode. */
void ho_true_state(const ho_world *w, uint16_t *cells, uint32_t *ep_t);
void ho_grid(const ho_world *w, uint32_t e, uint8_t *out);

/* Overwrite the dynamic state (positions, counters, t).  Used by tests that
 * start from a chosen state. */
void ho_set_state(ho_world *w, const int32_t *x, const int32_t *y,
                  const uint32_t *ep_t, const uint32_t *ep_idx, uint64_t t);

/* Run n_steps steps and fold the outputs into a per-run result: the sum of
 * each agent's rewards (agents entries), the number of finished episodes and
 * the order-independent observation digest
 *   sum over steps s and obs words j of splitmix64(word ^ (s * words + j))
 * (mod 2^64), s counted from the first step of this call, words the
 * per-step obs word count, splitmix64 the finaliser of Steele, Lea and
 * Flood (OOPSLA 2014). */
void ho_run_digest(ho_world *w, uint64_t n_steps, int64_t *rew_sum, uint64_t *episodes,
                   uint64_t *digest);

uint64_t ho_splitmix64(uint64_t z);

#ifdef __cplusplus
}
#endif

#endif
