/*
 * hase_serve.h -- rollout server on top of the batched step (hase.h).
 *
 * Not in the paper: the paper's engine serves one training process; this is
 * the serving form of the same step.  Clients submit rollout requests (each
 * a batch of identical environments run for a horizon, under its own seed)
 * from any thread while the server runs; a worker thread owns the GPU work:
 *
 *   admission   requests leave the submission queue in arrival order while
 *               the in-flight limit allows; every request larger than the
 *               whole memory budget is rejected with HASE_ENOMEM;
 *   batching    the admitted requests of a round (at most 256) are sorted
 *               by horizon and cut into batches of similar horizons (the
 *               longest at most twice the shortest) and at most
 *               max_batch_envs envs; requests of more than max_batch_envs / 32
 *               envs fill the GPU alone and get a handle of their own; a batch
 *               is admitted while its device bytes fit the budget (else its
 *               requests go back to the front of the queue) and becomes ONE
 *               handle (hase_config.env_seeds, env_ids: every env keeps its
 *               request's seed and request-local env id), so the requests of
 *               a batch share every step launch;
 *   stepping    each batch runs on one of a pool of CUDA streams (batches
 *               overlap on the device); its steps are enqueued up to each
 *               request's horizon in turn, each followed by that request's
 *               digest (hase_digest_range over its envs and horizon) and a
 *               32-byte copy of it to pinned memory, so a request finishes
 *               when its own horizon is reached;
 *   retirement  a request's result is ready when its copy has landed; a
 *               batch's memory goes back to the budget when its last request
 *               is done.
 * A request's result does not depend on what else runs: its environments,
 * seed, env ids and step counter are its own.
 */
#ifndef HASE_SERVE_H
#define HASE_SERVE_H

#include "hase.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hase_request {
    double arrival;       /* hase_serve: seconds after the start of the run,    */
                          /* non-decreasing; ignored by hase_server_submit      */
    uint64_t seed;        /* Philox key of the request                          */
    uint32_t n_envs;      /* environments of the request, >= 1                  */
    uint32_t steps;       /* horizon: steps of every environment, >= 1          */
    hase_env_desc desc;   /* shared by all environments of the request          */
} hase_request;

typedef struct hase_request_result {
    double submitted;     /* seconds since the server started: submission,      */
    double admitted;      /* admission into a batch,                            */
    double finished;      /* and when the worker saw the request's results      */
    uint64_t digest;      /* hase_digest_out of all of the request's steps      */
    uint64_t episodes;
    int64_t reward_sum;
    uint64_t bytes;       /* device memory charged to the request               */
    uint32_t status;      /* hase_status of the request                         */
    uint32_t batch_size;  /* requests that shared the request's batch           */
} hase_request_result;

/* Device bytes of a request with `steps` steps of output ring (its rings,
 * per-env state, keys and its share of a handle's fixed buffers).  A batch
 * is charged the sum over its requests with steps = the batch's longest
 * horizon (one ring length per handle). */
uint64_t hase_request_bytes(const hase_request *r);

/* ---------------------------------------------------------------------- */
/* The server.                                                             */
/* ---------------------------------------------------------------------- */
typedef struct hase_server hase_server;

typedef struct hase_server_config {
    uint64_t budget_bytes;   /* device memory the admitted batches may hold    */
    uint32_t n_streams;      /* CUDA streams batches are spread over (1..64)   */
    uint32_t max_inflight;   /* admitted, unfinished requests at most (>= 1)   */
    uint32_t queue_capacity; /* submitted, not yet admitted requests at most   */
                             /* (>= 1); submissions beyond get HASE_EBUSY      */
    uint32_t max_batch_envs; /* envs of one batch at most (0 = 16384)          */
    uint32_t max_batch;      /* requests of one batch at most (0 = 256; 1 = no */
                             /* sharing: every request its own handle)         */
    uint32_t pad;
} hase_server_config;

/* Start a server on the current CUDA device (its worker thread makes it
 * current).  HASE_EINVAL for a bad configuration, HASE_ECUDA when the
 * streams or result buffers cannot be created. */
hase_status hase_server_create(const hase_server_config *cfg, hase_server **out);

/* Queue one request (thread-safe); *id receives its id.  HASE_EBUSY when the
 * queue holds queue_capacity requests, HASE_ESTATE after
 * hase_server_shutdown, HASE_EINVAL for an invalid request.  A request that
 * can never fit the budget is accepted and finishes with HASE_ENOMEM. */
hase_status hase_server_submit(hase_server *s, const hase_request *r, uint64_t *id);

/* Wait up to timeout_s seconds (0: do not wait) for request `id` and, when it
 * has finished, store its result in *res (res->status: the request's own
 * status) and forget it.  HASE_ETIMEOUT when it has not finished in time,
 * HASE_EINVAL for an unknown or already collected id.  Thread-safe. */
hase_status hase_server_poll(hase_server *s, uint64_t id, double timeout_s, hase_request_result *res);

/* Counters of the server so far. */
typedef struct hase_serve_stats {
    double makespan;          /* wall seconds from start to the last result    */
    uint64_t peak_bytes;      /* largest sum of admitted batches' bytes        */
    uint32_t peak_inflight;   /* most requests in flight at once               */
    uint32_t rejected;        /* requests larger than the whole budget         */
    uint64_t batches;         /* batches (handles) created                     */
    uint64_t requests;        /* requests finished                             */
} hase_serve_stats;
hase_status hase_server_stats(hase_server *s, hase_serve_stats *out);

/* Stop taking submissions, finish every queued and admitted request, and
 * stop the worker (results stay pollable).  HASE_ECUDA when the device
 * failed during the run.  Idempotent. */
hase_status hase_server_shutdown(hase_server *s);

/* hase_server_shutdown, then free the server (NULL: no-op). */
void hase_server_destroy(hase_server *s);

/* ---------------------------------------------------------------------- */
/* Replay of a request list through a server.                              */
/* ---------------------------------------------------------------------- */
typedef struct hase_serve_config {
    uint64_t budget_bytes; /* device memory the admitted batches may hold      */
    uint32_t n_streams;    /* CUDA streams (1..64)                             */
    uint32_t max_inflight; /* admitted, unfinished requests at most (>= 1)     */
    double time_scale;     /* wall seconds per arrival second (0 = all at once) */
    uint32_t max_batch;    /* requests of one batch at most (0 = 256)          */
    uint32_t pad;
} hase_serve_config;

/* Serve n requests on the current device: a server receives request i at
 * arrival * time_scale seconds after the start (from the calling thread),
 * and the call returns when every one has finished.  res[i] receives request
 * i's result (times since the start).  Returns HASE_EINVAL for a bad
 * configuration, HASE_ECUDA when the device fails; per-request failures are
 * reported in res[i].status only. */
hase_status hase_serve(const hase_request *reqs, uint32_t n, const hase_serve_config *cfg,
                       hase_request_result *res, hase_serve_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* HASE_SERVE_H */
