/*
 * zmc_user.h — user-defined integrands, compiled at run time.
 *
 * The paper keeps the integrand in the user's hands: users define their own
 * integrands and the package compiles them for the GPU (Abstract; Sec. 1).
 * Here a user integrand is CUDA C source compiled with NVRTC into the same
 * sampling kernel as the built-in registry: the same grid decode, Philox
 * stream, box map, compensated sums, reductions and statistics, with the
 * user's g(y; x) evaluated per sample.  A kernel is compiled for each
 * (N, M, precision) the first time a scan needs it and kept for the process.
 *
 * The source defines one or both of
 *
 *   __device__ float  zmc_user_g32(const float* y, const float* x);   // FP32, FP32_KAHAN
 *   __device__ double zmc_user_g64(const double* y, const double* x); // FP64
 *
 * where y holds the sample's N box coordinates and x the grid point's M
 * parameters; ZMC_N and ZMC_M are compile-time constants in the source.
 * Registered ids (>= ZMC_G_USER_BASE) work with zmc_scan, zmc_scan_ex and
 * zmc_integrand_info_get; batches, the server and zmc_scan_noalloc take the
 * compiled-in registry only.
 *
 * NVRTC is loaded on first use (libnvrtc.so.13); without it registration
 * returns ZMC_ENOTFOUND.
 */
#ifndef ZMC_USER_H_
#define ZMC_USER_H_

#include "zmc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define ZMC_G_USER_BASE 1000
#define ZMC_MAX_USER_INTEGRANDS 64

/*
 * Register a user integrand for dimensions n_min..n_max (1..ZMC_MAX_N) and
 * any M.  The source is compiled at once (N = n_min, M = 1) to check it; on a
 * compile error the call returns ZMC_EINVAL and zmc_last_error() holds the
 * compiler's log.  *id receives the new integrand id.  Needs no GPU.
 */
int zmc_integrand_register(const char* name, const char* source, int n_min, int n_max,
                           int* id);

#ifdef __cplusplus
}
#endif

#endif /* ZMC_USER_H_ */
