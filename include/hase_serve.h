/*
 * hase_serve.h -- rollout server on top of the batched step (hase.h).
 *
 * Not in the paper: the paper's engine serves one training process; this is
 * the serving form of the same step.  A stream of rollout requests (each a
 * batch of identical environments run for a horizon) arrives over time; the
 * server keeps every admitted request's environments and outputs resident in
 * device memory, admits requests in arrival order while their bytes fit the
 * memory budget, runs them concurrently on a pool of CUDA streams (work of
 * requests that arrive while others run overlaps on the device), and returns
 * each request's digest (hase_digest over all of its steps) with its
 * admission and completion times.  A request's result does not depend on what
 * else runs: its environments, seed and step counter are its own.
 */
#ifndef HASE_SERVE_H
#define HASE_SERVE_H

#include "hase.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hase_request {
    double arrival;       /* seconds after the start of the run, non-decreasing */
    uint64_t seed;        /* Philox key of the request                          */
    uint32_t n_envs;      /* environments of the request, >= 1                  */
    uint32_t steps;       /* horizon: steps of every environment, >= 1          */
    hase_env_desc desc;   /* shared by all environments of the request          */
} hase_request;

typedef struct hase_serve_config {
    uint64_t budget_bytes; /* device memory the admitted requests may hold      */
    uint32_t n_streams;    /* CUDA streams the requests are spread over (1..64) */
    uint32_t max_inflight; /* admitted, unfinished requests at most (>= 1)      */
    double time_scale;     /* wall seconds per arrival second (0 = all at once) */
} hase_serve_config;

typedef struct hase_request_result {
    double admitted;      /* wall seconds since the start of hase_serve         */
    double finished;      /* when the server saw the request's results          */
    uint64_t digest;      /* hase_digest_out of all of the request's steps      */
    uint64_t episodes;
    int64_t reward_sum;
    uint64_t bytes;       /* device memory charged to the request               */
    uint32_t status;      /* hase_status of the request                         */
    uint32_t pad;
} hase_request_result;

typedef struct hase_serve_stats {
    double makespan;          /* wall seconds from start to the last result    */
    uint64_t peak_bytes;      /* largest sum of admitted requests' bytes       */
    uint32_t peak_inflight;   /* most requests in flight at once               */
    uint32_t rejected;        /* requests larger than the whole budget         */
} hase_serve_stats;

/* Device bytes a request is charged at admission (its output rings over its
 * horizon, the per-env state and the handle's scratch). */
uint64_t hase_request_bytes(const hase_request *r);

/* Serve n requests (arrival order) on the current device and return when
 * every one has finished.  res[i] receives request i's result; requests
 * larger than the budget get HASE_ENOMEM and are not run.  Returns
 * HASE_EINVAL for a bad configuration, HASE_ECUDA when the device fails;
 * per-request failures are reported in res[i].status only. */
hase_status hase_serve(const hase_request *reqs, uint32_t n, const hase_serve_config *cfg,
                       hase_request_result *res, hase_serve_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* HASE_SERVE_H */
