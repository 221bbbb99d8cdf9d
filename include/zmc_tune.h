/*
 * zmc_tune.h — the library's own tile autotuner.
 *
 * The sampling kernels are parametrised by the lanes that share one
 * (grid point, trial) sample range, the threads per block, and the sample
 * groups each lane sums (which fixes how many ranges a unit is split into).
 * zmc_autotune times candidate configurations of one scan on the current GPU
 * (CUDA events, on a bounded slice of the scan) and records the fastest for
 * the scan's class: (precision, integrand, N, floor(log2 S)).  The planners of
 * zmc_scan_ex, zmc_batch_create, zmc_scan_batch and the server use a recorded
 * class entry whenever a descriptor leaves its tiles at 0; without one they
 * use fixed rules.  Tuning changes which sums are formed in which order, so
 * results agree across configurations within the parity tolerances, and are
 * bit-identical only for the same configuration.
 *
 * With the environment variable ZMC_AUTOTUNE_CACHE set to a file path, the
 * table is read from that file on first use and rewritten after each tune.
 */
#ifndef ZMC_TUNE_H_
#define ZMC_TUNE_H_

#include "zmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zmc_tune_result {
  int lanes;               /* lanes per unit-split                          */
  int block;               /* threads per block (256 for batches)           */
  int groups_per_lane;     /* sample groups one lane sums, target           */
  int candidates;          /* configurations timed                          */
  double evals_per_s;      /* of the chosen configuration on the slice      */
  double default_evals_per_s; /* of the fixed-rule plan on the same slice   */
} zmc_tune_result;

/*
 * Tune the class of scan d (any memory kind; only its shape, integrand,
 * precision and lists are used; lists are copied to the device).  budget_ms
 * bounds the GPU time spent (>= 50).  Records and returns the winner.
 */
int zmc_autotune(const zmc_scan_desc* d, int budget_ms, zmc_tune_result* out);

/* The recorded entry for (precision, integrand, N, S), ZMC_ENOTFOUND if none. */
int zmc_autotune_lookup(int precision, int integrand_id, int N, int64_t samples,
                        zmc_tune_result* out);

/* Forget every recorded entry (the cache file, if any, is left alone). */
int zmc_autotune_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* ZMC_TUNE_H_ */
