/*
 * zmc_server.h — a request loop that serves scans with continuous batching.
 *
 * Each request is one scan (zmc_scan_desc, host memory): direct Monte Carlo
 * of Eq. 1 over its parameter grid (Sec. 2), with the same random stream,
 * sums and statistics as zmc_scan_ex, so its results do not depend on what
 * else is being served (bit-identical to the same scan alone with the same
 * tile configuration; the configuration depends only on the request).
 *
 * A scheduler thread owns the GPU.  Requests wait in a queue and are admitted
 * at every step boundary while a slot is free and the device-memory budget
 * covers their lists, partial sums and output buffers.  Each step is one
 * persistent launch per precision over tiles taken from all admitted requests
 * (shortest remaining work first, with a share of every step reserved for the
 * oldest request so large scans keep moving); partial sums stay on the device
 * between steps.  Grids too large for one chunk are streamed: each chunk of
 * grid points is finalized as soon as its tiles are done and copied into the
 * caller's host arrays by a copier thread, on a separate stream, while later
 * steps compute (the scheduler never waits for a copy, so pageable output
 * arrays do not hold up the planning of the next step).  The paper cuts grids
 * into batches for its GPUs (Sec. 2); this is that cut, made dynamic on one
 * GPU.
 *
 * Conventions as in zmc.h.  All calls are thread-safe.
 */
#ifndef ZMC_SERVER_H_
#define ZMC_SERVER_H_

#include "zmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zmc_server zmc_server;

typedef struct zmc_server_opts {
  int max_active;          /* requests admitted at once (slots); default 128    */
  double step_ms;          /* target GPU time of one step; default 10 ms         */
  int64_t chunk_units;     /* unit-splits (points x trials x splits) per device
                              chunk of one request; default 2^22                 */
  int fail_alloc_every;    /* test hook: every k-th device allocation fails
                              (ZMC_ENOMEM for that request); 0 = off            */
} zmc_server_opts;

typedef struct zmc_server_stats {
  int64_t submitted, completed, cancelled, failed;
  int64_t queued, active;          /* now                                     */
  int64_t max_queued;              /* peak queue length                       */
  int64_t steps;                   /* persistent launches issued (steps)      */
  int64_t evaluations;             /* of completed requests                   */
  double busy_ms;                  /* GPU time of all steps (CUDA events)     */
  double evals_per_s;              /* evaluations / busy time                 */
  double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> done, completed ones   */
  size_t mem_in_use, mem_peak;     /* device bytes held for requests          */
} zmc_server_stats;

/* Defaults into *opts. */
int zmc_server_opts_init(zmc_server_opts* opts);

/* Start a server on the current device with a device-memory budget in bytes
 * (requests whose footprint exceeds the whole budget are refused at submit
 * with ZMC_ENOMEM).  opts may be NULL for defaults. */
int zmc_server_create(size_t mem_budget_bytes, const zmc_server_opts* opts,
                      zmc_server** out);

/*
 * Queue one scan.  d->mem must be ZMC_MEM_HOST: the lists, bounds and lengths
 * are copied before the call returns; the output arrays in *o (host memory,
 * count entries each; errw/s1/s2 optional) must stay valid until the ticket
 * is done.  When the request completes, o->total_ms holds its latency
 * (submit -> results in host memory) and o->tile_* its tile configuration.
 * *ticket identifies the request in the calls below.
 */
int zmc_submit(zmc_server* s, const zmc_scan_desc* d, zmc_scan_out* o, uint64_t* ticket);

/* *done = 1 once the request finished (completed, failed or cancelled).
 * ZMC_ENOTFOUND for an unknown ticket. */
int zmc_poll(zmc_server* s, uint64_t ticket, int* done);

/* Wait up to timeout_ms (< 0: no limit) for the request; returns its final
 * status (ZMC_OK, ZMC_ECANCELED, ZMC_ENOMEM, ZMC_ECUDA, ...), ZMC_ETIMEDOUT
 * if it is still running, ZMC_ENOTFOUND for an unknown ticket. */
int zmc_wait(zmc_server* s, uint64_t ticket, int timeout_ms);

/* Cancel a queued or running request (its outputs are left untouched);
 * ZMC_OK if it was cancelled, ZMC_EBUSY if it had already finished. */
int zmc_cancel(zmc_server* s, uint64_t ticket);

int zmc_server_stats_get(zmc_server* s, zmc_server_stats* st);

/* Cancel what is left, stop the scheduler, free everything. */
int zmc_server_destroy(zmc_server* s);

#ifdef __cplusplus
}
#endif

#endif /* ZMC_SERVER_H_ */
