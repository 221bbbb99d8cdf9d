/*
 * zmc_batch.h — many scans in one persistent launch.
 *
 * Each scan is the direct Monte Carlo evaluation of Eq. 1 over its own
 * parameter grid (Sec. 2), exactly as zmc_scan_ex computes it: the same random
 * stream, the same per-unit sums, the same statistics, so a scan's results in
 * a batch are bit-identical to the same scan run alone with the same tile
 * configuration.  The paper runs batches of one grid on one GPU each (Sec. 2);
 * here scans of different integrands, dimensions, grid sizes and sample counts
 * share one launch: their work is cut into block-sized tiles, ordered longest
 * first, and taken by resident blocks from a device counter.
 *
 * Conventions as in zmc.h (status codes, zmc_last_error, C grid order).
 */
#ifndef ZMC_BATCH_H_
#define ZMC_BATCH_H_

#include "zmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zmc_batch zmc_batch;

/* zmc_batch_create flags */
enum {
  ZMC_BATCH_GRAPH = 1   /* capture one run into a CUDA graph; runs replay it */
};

typedef struct zmc_batch_info {
  int scans;
  int precisions;          /* persistent launches per run (one per precision) */
  int64_t tiles;
  int64_t evaluations;     /* sum over scans of count * T * S                  */
  int grid;                /* resident blocks of the persistent launch        */
  int block;
  size_t scratch_bytes;    /* device memory the batch holds                   */
  int graph;               /* 1 when runs replay a captured CUDA graph         */
  int launches_per_run;    /* kernels one run launches                        */
} zmc_batch_info;

/*
 * Plan a batch of n scans whose lists and outputs are DEVICE memory
 * (d[i].mem == ZMC_MEM_DEVICE, o[i].mean/err/... device pointers; o[i] gets
 * the tile configuration of scan i).  Allocates the batch's scratch (scan
 * arguments, tile list, partial sums) and, with ZMC_BATCH_GRAPH, captures one
 * run into a CUDA graph.  The caller's buffers must stay valid while the batch
 * exists.  Tile overrides in d[i] are honoured (lanes, splits; the block size
 * of a batch is 256).  Returns ZMC_EINVAL for n < 1 or any invalid scan.
 */
int zmc_batch_create(const zmc_scan_desc* d, zmc_scan_out* o, int n, int flags,
                     zmc_batch** out);

/* Enqueue one run of the batch on `stream` (NULL = CUDA default stream). */
int zmc_batch_run(zmc_batch* b, void* stream);

int zmc_batch_info_get(const zmc_batch* b, zmc_batch_info* info);

/* Free the batch (waits for its device work first). */
int zmc_batch_destroy(zmc_batch* b);

/*
 * One-shot batch: n scans, all host memory or all device memory (as d[i].mem
 * says), one persistent launch per precision present, synchronous.  With
 * ZMC_F_TIMINGS in d[0].flags, o[0].kernel_ms / finalize_ms / total_ms hold
 * the batch's event times.
 */
int zmc_scan_batch(const zmc_scan_desc* d, int n, zmc_scan_out* o);

#ifdef __cplusplus
}
#endif

#endif /* ZMC_BATCH_H_ */
