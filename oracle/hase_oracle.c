/*
 * hase_oracle.c -- plain single-threaded C oracle of the batched
 * hide-and-seek environment step (Hide-And-Seek-Engine, arxiv 2604.27162).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  It shares no code
 * with the CUDA engine.  Every function follows its definition literally with
 * naive loops: environments in index order, agents in index order, the
 * observation window cell by cell.
 *
 * Paper passages followed (section / table of the paper):
 *   Sec. 3.1   Dec-POMDP framing: one state, per-agent actions, observations
 *              and rewards.
 *   Sec. 3.2   "Collision Models": blocking tiles are impassable.
 *   Sec. 3.3   observability mode 1, "Decentralized Observation (No State)":
 *              each agent sees only its own sight window; modes 2-5 add the
 *              centralized observation and the true state (ho_central,
 *              ho_true_state).
 *   Sec. 4.1   random actions are generated inside the step (1/3 to 1/2 of
 *              the paper's runtime).
 *   Sec. 4.2   pristine-grid templating: a reset restores the immutable
 *              initial state.
 *   Table A.1  workload shape: 1024 environments, 1 / 5 / 10 agents.
 * Points the paper leaves open are fixed by the readings recorded in the
 * repository's design notes (Philox keying, multiply-shift action mapping,
 * Bernoulli threshold, start-cell redraw, simultaneous moves with
 * lowest-index-wins, out-of-bounds reads as obstacle, same-step auto-reset).
 */
#include "hase_oracle.h"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

struct ho_world {
    uint32_t n_envs;
    uint32_t env_id_base;
    uint64_t seed;
    uint64_t t;             /* global step counter                     */
    ho_env *env;            /* n_envs                                  */
    uint64_t *agent_off;    /* n_envs + 1                              */
    uint64_t *obs_off;      /* n_envs + 1 (uint64 words)               */
    uint64_t *unp_off;      /* n_envs + 1 (bytes)                      */
    uint32_t *wpp;          /* words per plane, n_envs                 */
    uint8_t **grid;         /* n_envs grids of side*side bytes         */
    int32_t *sx, *sy;       /* pristine start cells, per agent         */
    int32_t *x, *y;         /* current positions, per agent            */
    uint32_t *ep_t;         /* steps into the current episode, per env */
    uint32_t *ep_idx;       /* finished episodes, per env              */
    int desync;             /* episode clocks start at a drawn offset  */
    int fog;                /* 0 off, 1 global, 2 per-agent discovery  */
    uint64_t *fog_off;      /* n_envs + 1 (bytes of the fog maps)      */
    uint8_t *disc, *fresh;  /* discovery maps and their newest cells   */
};

static char g_err[256];
const char *ho_error(void) { return g_err; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds; each round multiplies counter      */
/* words 0 and 2 by the two published multipliers, and the new counter is    */
/* (hi(w2*M1) ^ c1 ^ k0, lo(w2*M1), hi(w0*M0) ^ c3 ^ k1, lo(w0*M0)).  Between */
/* rounds the key is bumped by the two Weyl constants.                       */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void ho_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* floor(u * n / 2^32): maps a uniform 32-bit word onto 0..n-1. */
static uint32_t mulhi32(uint32_t u, uint32_t n) {
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

static void philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    ho_philox4x32_10(ctr, key, out);
}

/* Stream 0: actions.  One Philox block serves four consecutive steps. */
uint32_t ho_action(uint64_t seed, uint64_t t, uint32_t agent, uint32_t env_id) {
    uint32_t out[4];
    philox_words(seed, (uint32_t)(t >> 2), agent, env_id, 0u, out);
    return mulhi32(out[t & 3u], 5u);
}

/* Action -> displacement.  x is the column, y the row, origin top-left. */
static const int32_t DX[5] = {0, 0, 0, 1, -1}; /* stay, N, S, E, W */
static const int32_t DY[5] = {0, -1, 1, 0, 0};

/* ------------------------------------------------------------------------ */
/* a2 + a3: simultaneous moves.  A move is valid when the action is not      */
/* "stay", the target is inside the grid, is not an obstacle and is not the */
/* current cell of any agent.  Among valid movers with the same target the   */
/* lowest agent index moves; every other agent stays.                        */
/* ------------------------------------------------------------------------ */
void ho_move(uint32_t S, const uint8_t *grid, uint32_t A, const int32_t *x,
             const int32_t *y, const uint8_t *act, int32_t *nx, int32_t *ny) {
    int32_t *tx = (int32_t *)malloc(sizeof(int32_t) * (A ? A : 1));
    int32_t *ty = (int32_t *)malloc(sizeof(int32_t) * (A ? A : 1));
    uint8_t *ok = (uint8_t *)malloc(A ? A : 1);
    for (uint32_t a = 0; a < A; ++a) {
        tx[a] = x[a] + DX[act[a]];
        ty[a] = y[a] + DY[act[a]];
        ok[a] = 1;
        if (act[a] == 0) ok[a] = 0;
        if (tx[a] < 0 || ty[a] < 0 || tx[a] >= (int32_t)S || ty[a] >= (int32_t)S) ok[a] = 0;
        if (ok[a] && grid[(size_t)ty[a] * S + (size_t)tx[a]] != 0) ok[a] = 0;
        if (ok[a]) {
            for (uint32_t b = 0; b < A; ++b) {
                if (x[b] == tx[a] && y[b] == ty[a]) ok[a] = 0;
            }
        }
    }
    for (uint32_t a = 0; a < A; ++a) {
        int moves = ok[a];
        for (uint32_t b = 0; b < a && moves; ++b) {
            if (ok[b] && tx[b] == tx[a] && ty[b] == ty[a]) moves = 0;
        }
        nx[a] = moves ? tx[a] : x[a];
        ny[a] = moves ? ty[a] : y[a];
    }
    free(tx);
    free(ty);
    free(ok);
}

/* ------------------------------------------------------------------------ */
/* a6: a hider is seen when some seeker is within Chebyshev distance r_seek. */
/* Each seen hider gets -1, every seeker gets +(number of seen hiders).     */
/* ------------------------------------------------------------------------ */
static int32_t iabs32(int32_t v) { return v < 0 ? -v : v; }

void ho_reward(uint32_t A, uint32_t n_seekers, uint32_t r_seek, const int32_t *x,
               const int32_t *y, int32_t *rew) {
    int32_t n_seen = 0;
    for (uint32_t h = n_seekers; h < A; ++h) {
        int seen = 0;
        for (uint32_t s = 0; s < n_seekers; ++s) {
            int32_t dx = iabs32(x[h] - x[s]);
            int32_t dy = iabs32(y[h] - y[s]);
            int32_t cheb = dx > dy ? dx : dy;
            if (cheb <= (int32_t)r_seek) seen = 1;
        }
        rew[h] = seen ? -1 : 0;
        n_seen += seen;
    }
    for (uint32_t s = 0; s < n_seekers && s < A; ++s) rew[s] = n_seen;
}

/* ------------------------------------------------------------------------ */
/* a5: decentralized observation of agent a.  Window cell (dx, dy), both in  */
/* -r..r, is bit k = (dy + r) * (2r + 1) + (dx + r) of each plane; bit k     */
/* lives in word k / 64 at position k % 64.  Plane 0: obstacle or outside    */
/* the grid.  Plane 1: an agent of a's team other than a.  Plane 2: an agent */
/* of the other team.                                                        */
/* ------------------------------------------------------------------------ */
/* Line of sight (Section 3.1: the observation is a line-of-sight projection
 * of the true state).  Reading: window cell (dx, dy) is visible from the
 * agent's cell iff every cell strictly between them on the discrete line is
 * inside the grid and free of obstacles; with n = max(|dx|, |dy|) those cells
 * are (rnd(i dx / n), rnd(i dy / n)) for i = 1 .. n-1, rnd rounding halves
 * away from zero. */
static int32_t rnd_div(int32_t p, int32_t n) {
    return p >= 0 ? (2 * p + n) / (2 * n) : -((-2 * p + n) / (2 * n));
}

int ho_visible(uint32_t S, const uint8_t *grid, int32_t x, int32_t y, int32_t dx, int32_t dy) {
    int32_t n = abs(dx) > abs(dy) ? abs(dx) : abs(dy);
    for (int32_t i = 1; i < n; ++i) {
        int32_t cx = x + rnd_div(i * dx, n);
        int32_t cy = y + rnd_div(i * dy, n);
        if (cx < 0 || cy < 0 || cx >= (int32_t)S || cy >= (int32_t)S) return 0;
        if (grid[(size_t)cy * S + (size_t)cx]) return 0;
    }
    return 1;
}

void ho_observe_agent(uint32_t S, const uint8_t *grid, uint32_t A, uint32_t n_seekers,
                      const int32_t *x, const int32_t *y, uint32_t a, uint32_t r,
                      uint32_t W, uint32_t los, uint64_t *out) {
    int32_t R = (int32_t)r;
    int32_t D = 2 * R + 1;
    int team_a = a < n_seekers ? 0 : 1;
    for (uint32_t i = 0; i < 3 * W; ++i) out[i] = 0;
    for (int32_t dy = -R; dy <= R; ++dy) {
        for (int32_t dx = -R; dx <= R; ++dx) {
            uint32_t k = (uint32_t)((dy + R) * D + (dx + R));
            uint64_t bit = (uint64_t)1 << (k % 64);
            uint32_t word = k / 64;
            int32_t cx = x[a] + dx;
            int32_t cy = y[a] + dy;
            if (los && !ho_visible(S, grid, x[a], y[a], dx, dy)) continue;  /* hidden: all planes 0 */
            if (cx < 0 || cy < 0 || cx >= (int32_t)S || cy >= (int32_t)S) {
                out[0 * W + word] |= bit;
                continue;
            }
            if (grid[(size_t)cy * S + (size_t)cx]) out[0 * W + word] |= bit;
            for (uint32_t b = 0; b < A; ++b) {
                if (b == a) continue;
                if (x[b] != cx || y[b] != cy) continue;
                int team_b = b < n_seekers ? 0 : 1;
                if (team_b == team_a)
                    out[1 * W + word] |= bit;
                else
                    out[2 * W + word] |= bit;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* World creation (a0).                                                      */
/* ------------------------------------------------------------------------ */
static uint32_t emits(const ho_env *p, uint32_t a) {
    uint32_t team = a < p->n_seekers ? 0u : 1u;
    return (p->obs_teams >> team) & 1u;
}

static uint32_t radius_of(const ho_env *p, uint32_t a) {
    return a < p->n_seekers ? p->r_seek : p->r_hide;
}

/* Centralized observation (Section 3.3, observability mode 3: all agents'
 * sightlines fused into one shared partial observation).  Reading: one
 * tensor per env over its whole grid with four planes -- 0 cells seen by
 * some observing agent (inside its window; with line of sight, visible to
 * it), 1 seen obstacles, 2 seen seekers, 3 seen hiders.  Plane p, row y,
 * bit x of word x / 64 is cell (x, y); S rows of ceil(S / 64) words. */
void ho_central_one(uint32_t side, const uint8_t *grid, uint32_t A, uint32_t n_seekers, uint32_t r_seek,
                    uint32_t r_hide, uint32_t obs_teams, const int32_t *ax, const int32_t *ay, uint64_t *out) {
    const int32_t S = (int32_t)side;
    const uint32_t rw = (side + 63u) / 64u;
    const uint32_t los = (obs_teams >> 2) & 1u;
    for (uint64_t i = 0; i < 4ull * S * rw; ++i) out[i] = 0;
    for (int32_t y = 0; y < S; ++y) {
        for (int32_t x = 0; x < S; ++x) {
            int seen = 0;
            for (uint32_t a = 0; a < A && !seen; ++a) {
                const uint32_t team = a < n_seekers ? 0u : 1u;
                if (!((obs_teams >> team) & 1u)) continue;
                const int32_t r = (int32_t)(team ? r_hide : r_seek);
                const int32_t dx = x - ax[a], dy = y - ay[a];
                if (dx < -r || dx > r || dy < -r || dy > r) continue;
                if (los && !ho_visible(side, grid, ax[a], ay[a], dx, dy)) continue;
                seen = 1;
            }
            if (!seen) continue;
            const uint64_t bit = (uint64_t)1 << (x % 64);
            const uint64_t at = (uint64_t)y * rw + (uint64_t)(x / 64);
            out[0 * S * rw + at] |= bit;
            if (grid[(size_t)y * S + (size_t)x]) out[1 * S * rw + at] |= bit;
            for (uint32_t b = 0; b < A; ++b) {
                if (ax[b] != x || ay[b] != y) continue;
                out[(b < n_seekers ? 2 : 3) * S * rw + at] |= bit;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Fog of war (Section 3.3 and the observation-layer table of Section 4: a   */
/* discovery map, per agent or global, where seen cells stay marked -- the   */
/* paper notes that visibility is monotone, "once seen, always seen"; and    */
/* the "diff sweep" variant of Section 5, which touches only newly           */
/* discovered tiles).  Unit j of an env is the j-th observing agent          */
/* (per_agent) or all observing agents together.                             */
/* ------------------------------------------------------------------------ */
uint32_t ho_fog_units(uint32_t A, uint32_t n_seekers, uint32_t obs_teams, uint32_t per_agent) {
    if (!per_agent) return 1u;
    uint32_t n = 0;
    for (uint32_t a = 0; a < A; ++a) {
        const uint32_t team = a < n_seekers ? 0u : 1u;
        if ((obs_teams >> team) & 1u) ++n;
    }
    return n;
}

/* Whether agent a sees cell (x, y): inside its (2r+1)^2 window and, with
 * line of sight, visible from it. */
static int agent_sees(uint32_t side, const uint8_t *grid, int32_t ax, int32_t ay, int32_t r, uint32_t los,
                      int32_t x, int32_t y) {
    const int32_t dx = x - ax, dy = y - ay;
    if (dx < -r || dx > r || dy < -r || dy > r) return 0;
    return !los || ho_visible(side, grid, ax, ay, dx, dy);
}

/* One update of one env's maps (side*side bytes per unit, row major).  A
 * cell is discovered once some agent of the unit has seen it in the current
 * episode; an episode's first observation (start != 0: after create, reset
 * or an auto-reset) begins with an empty map.  fresh marks the cells that
 * this update discovered. */
void ho_fog_update(uint32_t side, const uint8_t *grid, uint32_t A, uint32_t n_seekers, uint32_t r_seek,
                   uint32_t r_hide, uint32_t obs_teams, uint32_t per_agent, const int32_t *ax,
                   const int32_t *ay, uint32_t start, uint8_t *disc, uint8_t *fresh) {
    const uint32_t los = (obs_teams >> 2) & 1u;
    const uint64_t cells = (uint64_t)side * side;
    const uint32_t units = ho_fog_units(A, n_seekers, obs_teams, per_agent);
    for (uint32_t u = 0; u < units; ++u) {
        uint8_t *d = disc + u * cells;
        uint8_t *f = fresh + u * cells;
        for (int32_t y = 0; y < (int32_t)side; ++y) {
            for (int32_t x = 0; x < (int32_t)side; ++x) {
                int seen = 0;
                uint32_t k = 0; /* index among the observing agents */
                for (uint32_t a = 0; a < A && !seen; ++a) {
                    const uint32_t team = a < n_seekers ? 0u : 1u;
                    if (!((obs_teams >> team) & 1u)) continue;
                    const uint32_t mine = !per_agent || k == u;
                    k += 1;
                    if (!mine) continue;
                    const int32_t r = (int32_t)(team ? r_hide : r_seek);
                    seen = agent_sees(side, grid, ax[a], ay[a], r, los, x, y);
                }
                const size_t c = (size_t)y * side + (size_t)x;
                const uint8_t before = start ? 0 : d[c];
                d[c] = (uint8_t)(before | seen);
                f[c] = (uint8_t)(seen && !before);
            }
        }
    }
}

static void fog_env(ho_world *w, uint32_t e, uint32_t start) {
    const ho_env *p = &w->env[e];
    const uint64_t base = w->agent_off[e];
    ho_fog_update(p->side, w->grid[e], p->n_agents, p->n_seekers, p->r_seek, p->r_hide, p->obs_teams,
                  w->fog == 2, &w->x[base], &w->y[base], start, w->disc + w->fog_off[e],
                  w->fresh + w->fog_off[e]);
}

static void central_env(const ho_world *w, uint32_t e, uint64_t *out) {
    const ho_env *p = &w->env[e];
    const uint64_t base = w->agent_off[e];
    ho_central_one(p->side, w->grid[e], p->n_agents, p->n_seekers, p->r_seek, p->r_hide, p->obs_teams,
                   &w->x[base], &w->y[base], out);
}

uint64_t ho_central_words(const ho_world *w) {
    uint64_t n = 0;
    for (uint32_t e = 0; e < w->n_envs; ++e) n += 4ull * w->env[e].side * ((w->env[e].side + 63u) / 64u);
    return n;
}

void ho_central(const ho_world *w, uint64_t *out) {
    uint64_t off = 0;
    for (uint32_t e = 0; e < w->n_envs; ++e) {
        central_env(w, e, out + off);
        off += 4ull * w->env[e].side * ((w->env[e].side + 63u) / 64u);
    }
}


static uint32_t words_per_plane(const ho_env *p) {
    uint32_t wmax = 0;
    for (uint32_t a = 0; a < p->n_agents; ++a) {
        if (!emits(p, a)) continue;
        uint32_t D = 2 * radius_of(p, a) + 1;
        uint32_t w = (D * D + 63) / 64;
        if (w > wmax) wmax = w;
    }
    return wmax;
}

static uint32_t obs_agents(const ho_env *p) {
    uint32_t n = 0;
    for (uint32_t a = 0; a < p->n_agents; ++a) n += emits(p, a);
    return n;
}

static uint64_t unp_bytes(const ho_env *p) {
    uint64_t n = 0;
    for (uint32_t a = 0; a < p->n_agents; ++a) {
        if (!emits(p, a)) continue;
        uint64_t D = 2 * radius_of(p, a) + 1;
        n += 3 * D * D;
    }
    return n;
}

/* Start cells (stream 2): agent a draws cell = floor(u * S^2 / 2^32) from
 * counter (attempt, a, env, 2), word 0, redrawing with attempt + 1 while the
 * cell equals an earlier agent's.  Obstacles (stream 1): cell c is blocked
 * iff word c % 4 of counter (c / 4, 0, env, 1) is below density_thr.  Start
 * cells are then forced free.  Both are fixed for the life of the world. */
static void generate_env(ho_world *w, uint32_t e) {
    const ho_env *p = &w->env[e];
    uint32_t S = p->side;
    uint32_t env_id = w->env_id_base + e;
    uint64_t base = w->agent_off[e];
    uint32_t *cells = (uint32_t *)malloc(sizeof(uint32_t) * (p->n_agents ? p->n_agents : 1));
    for (uint32_t a = 0; a < p->n_agents; ++a) {
        uint32_t attempt = 0;
        for (;;) {
            uint32_t out[4];
            philox_words(w->seed, attempt, a, env_id, 2u, out);
            uint32_t cell = mulhi32(out[0], S * S);
            int dup = 0;
            for (uint32_t b = 0; b < a; ++b) {
                if (cells[b] == cell) dup = 1;
            }
            if (!dup) {
                cells[a] = cell;
                break;
            }
            attempt += 1;
        }
        w->sx[base + a] = (int32_t)(cells[a] % S);
        w->sy[base + a] = (int32_t)(cells[a] / S);
    }
    uint8_t *g = w->grid[e];
    for (uint32_t c = 0; c < S * S; ++c) {
        uint32_t out[4];
        philox_words(w->seed, c / 4u, 0u, env_id, 1u, out);
        g[c] = out[c % 4u] < p->density_thr ? 1 : 0;
    }
    for (uint32_t a = 0; a < p->n_agents; ++a) g[cells[a]] = 0;
    free(cells);
}

static int check_env(const ho_env *p) {
    if (p->side < 1 || p->side > 255) {
        snprintf(g_err, sizeof g_err, "side %u outside 1..255", p->side);
        return 0;
    }
    if (p->n_agents < 1 || p->n_agents > 256 || p->n_agents > p->side * p->side) {
        snprintf(g_err, sizeof g_err, "n_agents %u outside 1..min(256, side^2)", p->n_agents);
        return 0;
    }
    if (p->n_seekers > p->n_agents) {
        snprintf(g_err, sizeof g_err, "n_seekers %u > n_agents %u", p->n_seekers, p->n_agents);
        return 0;
    }
    if (p->r_seek > 7 || p->r_hide > 7) {
        snprintf(g_err, sizeof g_err, "view radius above 7");
        return 0;
    }
    if (p->cap < 1) {
        snprintf(g_err, sizeof g_err, "episode cap must be >= 1");
        return 0;
    }
    if (p->obs_teams > 7) {
        snprintf(g_err, sizeof g_err, "obs_teams %u: bits 0-2 only", p->obs_teams);
        return 0;
    }
    return 1;
}

ho_world *ho_create(uint32_t n_envs, uint32_t env_id_base, uint64_t seed,
                    const ho_env *envs, uint32_t n_desc) {
    if (n_desc != 1 && n_desc != n_envs) {
        snprintf(g_err, sizeof g_err, "n_desc must be 1 or n_envs");
        return NULL;
    }
    for (uint32_t i = 0; i < n_desc; ++i) {
        if (!check_env(&envs[i])) return NULL;
    }
    ho_world *w = (ho_world *)calloc(1, sizeof(ho_world));
    w->n_envs = n_envs;
    w->env_id_base = env_id_base;
    w->seed = seed;
    w->env = (ho_env *)malloc(sizeof(ho_env) * (n_envs ? n_envs : 1));
    for (uint32_t e = 0; e < n_envs; ++e) w->env[e] = envs[n_desc == 1 ? 0 : e];
    w->agent_off = (uint64_t *)calloc(n_envs + 1, sizeof(uint64_t));
    w->obs_off = (uint64_t *)calloc(n_envs + 1, sizeof(uint64_t));
    w->unp_off = (uint64_t *)calloc(n_envs + 1, sizeof(uint64_t));
    w->wpp = (uint32_t *)calloc(n_envs ? n_envs : 1, sizeof(uint32_t));
    for (uint32_t e = 0; e < n_envs; ++e) {
        const ho_env *p = &w->env[e];
        w->wpp[e] = words_per_plane(p);
        w->agent_off[e + 1] = w->agent_off[e] + p->n_agents;
        w->obs_off[e + 1] = w->obs_off[e] + (uint64_t)obs_agents(p) * 3u * w->wpp[e];
        w->unp_off[e + 1] = w->unp_off[e] + unp_bytes(p);
    }
    uint64_t n_ag = w->agent_off[n_envs];
    size_t na = (size_t)(n_ag ? n_ag : 1);
    w->sx = (int32_t *)malloc(sizeof(int32_t) * na);
    w->sy = (int32_t *)malloc(sizeof(int32_t) * na);
    w->x = (int32_t *)malloc(sizeof(int32_t) * na);
    w->y = (int32_t *)malloc(sizeof(int32_t) * na);
    w->ep_t = (uint32_t *)calloc(n_envs ? n_envs : 1, sizeof(uint32_t));
    w->ep_idx = (uint32_t *)calloc(n_envs ? n_envs : 1, sizeof(uint32_t));
    w->grid = (uint8_t **)calloc(n_envs ? n_envs : 1, sizeof(uint8_t *));
    for (uint32_t e = 0; e < n_envs; ++e) {
        w->grid[e] = (uint8_t *)malloc((size_t)w->env[e].side * w->env[e].side);
        generate_env(w, e);
    }
    ho_reset(w);
    return w;
}

void ho_destroy(ho_world *w) {
    if (!w) return;
    for (uint32_t e = 0; e < w->n_envs; ++e) free(w->grid[e]);
    free(w->grid);
    free(w->env);
    free(w->agent_off);
    free(w->obs_off);
    free(w->unp_off);
    free(w->wpp);
    free(w->sx);
    free(w->sy);
    free(w->x);
    free(w->y);
    free(w->ep_t);
    free(w->ep_idx);
    free(w->fog_off);
    free(w->disc);
    free(w->fresh);
    free(w);
}

/* Desynchronised start (Section 3.3, last paragraph: the envs of a batch are
 * stepped stochastically at initialisation so that they do not all end their
 * episodes together).  Reading: env e draws an offset o_e = floor(u * cap /
 * 2^32), u = word 0 of the Philox block of counter (0, 0, env id, 3), and
 * takes o_e steps of its dynamics (a1 actions, a2/a3 moves) from its start
 * cells before its first observation.  Those steps draw their actions from a
 * stream of their own -- pre-step tau uses word tau % 4 of counter
 * (tau / 4, agent, env id, 4) -- and give no reward, observation or fog
 * update; the env's episode clock starts at o_e, so its first episode ends
 * after cap - o_e more steps (o_e < cap: no episode ends while pre-stepping),
 * and every later episode starts from the start cells.  The action stream of
 * the steps themselves (stream 0, counter t) is untouched. */
static uint32_t start_offset(const ho_world *w, uint32_t e) {
    const uint32_t ctr[4] = {0u, 0u, w->env_id_base + e, 3u};
    const uint32_t key[2] = {(uint32_t)(w->seed & 0xffffffffu), (uint32_t)(w->seed >> 32)};
    uint32_t out[4];
    ho_philox4x32_10(ctr, key, out);
    return mulhi32(out[0], w->env[e].cap);
}

/* Stream 4: the action of pre-step tau of the desynchronised start. */
uint32_t ho_prestep_action(uint64_t seed, uint32_t tau, uint32_t agent, uint32_t env_id) {
    uint32_t out[4];
    philox_words(seed, tau >> 2, agent, env_id, 4u, out);
    return mulhi32(out[tau & 3u], 5u);
}

/* n pre-steps of env e: actions of stream 4, then the simultaneous moves. */
static void prestep_env(ho_world *w, uint32_t e, uint32_t n) {
    const ho_env *p = &w->env[e];
    const uint32_t A = p->n_agents, env_id = w->env_id_base + e;
    const uint64_t base = w->agent_off[e];
    uint8_t act[256];
    int32_t nx[256], ny[256];
    for (uint32_t tau = 0; tau < n; ++tau) {
        for (uint32_t a = 0; a < A; ++a) act[a] = (uint8_t)ho_prestep_action(w->seed, tau, a, env_id);
        ho_move(p->side, w->grid[e], A, &w->x[base], &w->y[base], act, nx, ny);
        for (uint32_t a = 0; a < A; ++a) {
            w->x[base + a] = nx[a];
            w->y[base + a] = ny[a];
        }
    }
}

void ho_set_desync(ho_world *w, int on) {
    w->desync = on ? 1 : 0;
    ho_reset(w);
}

void ho_reset(ho_world *w) {
    w->t = 0;
    for (uint32_t e = 0; e < w->n_envs; ++e) {
        w->ep_t[e] = w->desync ? start_offset(w, e) : 0;
        w->ep_idx[e] = 0;
        for (uint64_t i = w->agent_off[e]; i < w->agent_off[e + 1]; ++i) {
            w->x[i] = w->sx[i];
            w->y[i] = w->sy[i];
        }
        if (w->desync) prestep_env(w, e, w->ep_t[e]);
        if (w->fog) fog_env(w, e, 1u);
    }
}

/* Fog-of-war maps on (mode 1 global, 2 per agent) or off (0); restarts the
 * world like ho_reset, so the maps begin with the first observation. */
void ho_set_fog(ho_world *w, int mode) {
    free(w->fog_off);
    free(w->disc);
    free(w->fresh);
    w->fog_off = NULL;
    w->disc = w->fresh = NULL;
    w->fog = mode == 1 || mode == 2 ? mode : 0;
    if (w->fog) {
        w->fog_off = (uint64_t *)calloc(w->n_envs + 1, sizeof(uint64_t));
        for (uint32_t e = 0; e < w->n_envs; ++e) {
            const ho_env *p = &w->env[e];
            w->fog_off[e + 1] = w->fog_off[e] + (uint64_t)ho_fog_units(p->n_agents, p->n_seekers, p->obs_teams,
                                                                       w->fog == 2) *
                                                    p->side * p->side;
        }
        const uint64_t n = w->fog_off[w->n_envs];
        w->disc = (uint8_t *)calloc(n ? n : 1, 1);
        w->fresh = (uint8_t *)calloc(n ? n : 1, 1);
    }
    ho_reset(w);
}

/* Words of ho_fog: per env [units][2][side][ceil(side / 64)]. */
uint64_t ho_fog_words(const ho_world *w) {
    if (!w->fog) return 0;
    uint64_t n = 0;
    for (uint32_t e = 0; e < w->n_envs; ++e) {
        const ho_env *p = &w->env[e];
        n += (uint64_t)ho_fog_units(p->n_agents, p->n_seekers, p->obs_teams, w->fog == 2) * 2u * p->side *
             ((p->side + 63u) / 64u);
    }
    return n;
}

/* The maps of the current step, packed: per env and unit the discovery map
 * then the newly discovered cells, each side rows of bits (bit x of row y
 * = cell (x, y)). */
void ho_fog(const ho_world *w, uint64_t *out) {
    uint64_t o = 0;
    for (uint32_t e = 0; w->fog && e < w->n_envs; ++e) {
        const ho_env *p = &w->env[e];
        const uint32_t S = p->side, rw = (S + 63u) / 64u;
        const uint32_t units = ho_fog_units(p->n_agents, p->n_seekers, p->obs_teams, w->fog == 2);
        for (uint32_t u = 0; u < units; ++u) {
            for (uint32_t q = 0; q < 2; ++q) {
                const uint8_t *m = (q ? w->fresh : w->disc) + w->fog_off[e] + (uint64_t)u * S * S;
                for (uint32_t y = 0; y < S; ++y) {
                    for (uint32_t k = 0; k < rw; ++k) out[o + (uint64_t)y * rw + k] = 0;
                    for (uint32_t x = 0; x < S; ++x)
                        if (m[(size_t)y * S + x]) out[o + (uint64_t)y * rw + x / 64] |= (uint64_t)1 << (x % 64);
                }
                o += (uint64_t)S * rw;
            }
        }
    }
}

void ho_sizes(const ho_world *w, uint64_t *agents, uint64_t *obs_words, uint64_t *unp) {
    if (agents) *agents = w->agent_off[w->n_envs];
    if (obs_words) *obs_words = w->obs_off[w->n_envs];
    if (unp) *unp = w->unp_off[w->n_envs];
}

void ho_offsets(const ho_world *w, uint64_t *agent_off, uint64_t *obs_off,
                uint64_t *unp_off, uint32_t *wpp) {
    for (uint32_t e = 0; e <= w->n_envs; ++e) {
        if (agent_off) agent_off[e] = w->agent_off[e];
        if (obs_off) obs_off[e] = w->obs_off[e];
        if (unp_off) unp_off[e] = w->unp_off[e];
        if (wpp && e < w->n_envs) wpp[e] = w->wpp[e];
    }
}

/* Observation of every emitting agent of env e into its slice; the unpacked
 * form repeats each plane bit k as one byte at (plane * D*D + k). */
static void observe_env(const ho_world *w, uint32_t e, uint64_t *obs, uint8_t *unp) {
    const ho_env *p = &w->env[e];
    uint64_t base = w->agent_off[e];
    uint32_t W = w->wpp[e];
    uint64_t oi = w->obs_off[e];
    uint64_t ui = w->unp_off[e];
    uint64_t tmp[3 * 4];
    for (uint32_t a = 0; a < p->n_agents; ++a) {
        if (!emits(p, a)) continue;
        uint32_t r = radius_of(p, a);
        ho_observe_agent(p->side, w->grid[e], p->n_agents, p->n_seekers, &w->x[base],
                         &w->y[base], a, r, W, (p->obs_teams >> 2) & 1u, tmp);
        if (obs) {
            for (uint32_t i = 0; i < 3 * W; ++i) obs[oi + i] = tmp[i];
        }
        oi += 3u * W;
        uint32_t D = 2 * r + 1;
        if (unp) {
            for (uint32_t pl = 0; pl < 3; ++pl) {
                for (uint32_t k = 0; k < D * D; ++k) {
                    uint64_t word = tmp[pl * W + k / 64];
                    unp[ui + (uint64_t)pl * D * D + k] = (uint8_t)((word >> (k % 64)) & 1u);
                }
            }
        }
        ui += 3u * (uint64_t)D * D;
    }
}

void ho_observe(const ho_world *w, uint64_t *obs, uint8_t *unp) {
    for (uint32_t e = 0; e < w->n_envs; ++e) observe_env(w, e, obs, unp);
}

/* One step of one env: a1 actions, a2/a3 moves, a6 reward on the moved
 * positions, a7 episode counter and truncation, a8 same-step auto-reset, a5
 * observation of the (possibly reset) state. */
static void step_env(ho_world *w, uint32_t e, uint64_t *obs, int32_t *rew, uint8_t *done,
                     uint8_t *act_out, uint8_t *unp) {
    const ho_env *p = &w->env[e];
    uint32_t A = p->n_agents;
    uint64_t base = w->agent_off[e];
    uint32_t env_id = w->env_id_base + e;
    uint8_t act[256] = {0};
    int32_t nx[256], ny[256], r[256];
    for (uint32_t a = 0; a < A; ++a) act[a] = (uint8_t)ho_action(w->seed, w->t, a, env_id);
    ho_move(p->side, w->grid[e], A, &w->x[base], &w->y[base], act, nx, ny);
    for (uint32_t a = 0; a < A; ++a) {
        w->x[base + a] = nx[a];
        w->y[base + a] = ny[a];
    }
    ho_reward(A, p->n_seekers, p->r_seek, &w->x[base], &w->y[base], r);
    w->ep_t[e] += 1;
    uint8_t d = 0;
    if (w->ep_t[e] == p->cap) {
        d = 3; /* bit 0 done, bit 1 truncated */
        w->ep_t[e] = 0;
        w->ep_idx[e] += 1;
        for (uint32_t a = 0; a < A; ++a) {
            w->x[base + a] = w->sx[base + a];
            w->y[base + a] = w->sy[base + a];
        }
    }
    if (rew) {
        for (uint32_t a = 0; a < A; ++a) rew[base + a] = r[a];
    }
    if (act_out) {
        for (uint32_t a = 0; a < A; ++a) act_out[base + a] = act[a];
    }
    if (done) done[e] = d;
    if (obs || unp) observe_env(w, e, obs, unp);
    if (w->fog) fog_env(w, e, d != 0);
}

void ho_step(ho_world *w, uint64_t *obs, int32_t *rew, uint8_t *done, uint8_t *act,
             uint8_t *unp) {
    for (uint32_t e = 0; e < w->n_envs; ++e) step_env(w, e, obs, rew, done, act, unp);
    w->t += 1;
}

void ho_state(const ho_world *w, int32_t *x, int32_t *y, int32_t *sx, int32_t *sy,
              uint32_t *ep_t, uint32_t *ep_idx, uint64_t *t) {
    uint64_t n = w->agent_off[w->n_envs];
    for (uint64_t i = 0; i < n; ++i) {
        if (x) x[i] = w->x[i];
        if (y) y[i] = w->y[i];
        if (sx) sx[i] = w->sx[i];
        if (sy) sy[i] = w->sy[i];
    }
    for (uint32_t e = 0; e < w->n_envs; ++e) {
        if (ep_t) ep_t[e] = w->ep_t[e];
        if (ep_idx) ep_idx[e] = w->ep_idx[e];
    }
    if (t) *t = w->t;
}

/* True-state record (Sec. 3.3, observability modes 2, 4 and 5: the
 * environment also returns the omniscient game state).  The dynamic part of
 * the state: every agent's cell, x | y << 6, agents in handle order, and
 * every env's episode clock; the static part (obstacles, start cells) is
 * read with ho_grid / ho_state. */
void ho_true_state(const ho_world *w, uint16_t *cells, uint32_t *ep_t) {
    uint64_t n = w->agent_off[w->n_envs];
    for (uint64_t i = 0; i < n; ++i) cells[i] = (uint16_t)((uint32_t)w->x[i] | ((uint32_t)w->y[i] << 6));
    for (uint32_t e = 0; e < w->n_envs; ++e) ep_t[e] = w->ep_t[e];
}

void ho_grid(const ho_world *w, uint32_t e, uint8_t *out) {
    memcpy(out, w->grid[e], (size_t)w->env[e].side * w->env[e].side);
}

void ho_set_state(ho_world *w, const int32_t *x, const int32_t *y, const uint32_t *ep_t,
                  const uint32_t *ep_idx, uint64_t t) {
    uint64_t n = w->agent_off[w->n_envs];
    for (uint64_t i = 0; i < n; ++i) {
        if (x) w->x[i] = x[i];
        if (y) w->y[i] = y[i];
    }
    for (uint32_t e = 0; e < w->n_envs; ++e) {
        if (ep_t) w->ep_t[e] = ep_t[e];
        if (ep_idx) w->ep_idx[e] = ep_idx[e];
    }
    w->t = t;
}

/* splitmix64 output function (Steele, Lea, Flood, OOPSLA 2014): add the
 * golden gamma, then two xor-shift-multiply rounds and a final xor-shift. */
uint64_t ho_splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void ho_run_digest(ho_world *w, uint64_t n_steps, int64_t *rew_sum, uint64_t *episodes,
                   uint64_t *digest) {
    uint64_t n_ag = w->agent_off[w->n_envs];
    uint64_t n_words = w->obs_off[w->n_envs];
    uint64_t *obs = (uint64_t *)malloc(sizeof(uint64_t) * (n_words ? n_words : 1));
    int32_t *rew = (int32_t *)malloc(sizeof(int32_t) * (n_ag ? n_ag : 1));
    uint8_t *done = (uint8_t *)malloc(w->n_envs ? w->n_envs : 1);
    uint64_t dig = 0, eps = 0;
    for (uint64_t i = 0; i < n_ag; ++i) rew_sum[i] = 0;
    for (uint64_t s = 0; s < n_steps; ++s) {
        ho_step(w, obs, rew, done, NULL, NULL);
        for (uint64_t i = 0; i < n_ag; ++i) rew_sum[i] += rew[i];
        for (uint32_t e = 0; e < w->n_envs; ++e) eps += (done[e] & 1u);
        for (uint64_t j = 0; j < n_words; ++j) dig += ho_splitmix64(obs[j] ^ (s * n_words + j));
    }
    *episodes = eps;
    *digest = dig;
    free(obs);
    free(rew);
    free(done);
}
