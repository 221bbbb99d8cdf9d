/*
 * zmc.h — C ABI of the GB300 parameter-grid direct Monte Carlo library.
 *
 * The method (arXiv:1910.01965, "ZMCintegral-v5"): for every point x of a
 * Cartesian parameter grid built from M per-parameter value lists (Sec. 2),
 * estimate f(x) = \int dy g(y; x) over an N-dimensional box (Eq. 1) by the
 * direct (plain) Monte Carlo method (Sec. 1, Sec. 2), repeated over T
 * independent trials (Sec. 3.2), and return one value per grid point as a
 * multi-dimensional grid (Sec. 2).
 *
 * Conventions shared by every entry point:
 *  - Every call returns a zmc_status.  Nothing throws across the ABI.  On any
 *    error the outputs are left untouched and zmc_last_error() returns a
 *    message for the calling thread.
 *  - Grid order is C order over the lists: the flat index p has the last list
 *    varying fastest, as numpy's indexing='ij'.  Output arrays hold one FP64
 *    value per grid point in that order.
 *  - Random numbers: call j of grid point p in trial t is Philox4x32-10
 *    (Salmon et al., SC'11) with counter (j, t, p mod 2^32, p >> 32) and key
 *    (seed mod 2^32, seed >> 32).  Its four output words r0..r3 form the
 *    128-bit block r0 + r1 2^32 + r2 2^64 + r3 2^96, cut into five 23-bit
 *    fields (bits 23m .. 23m+22, m = 0..4).  Sample s, dimension k uses field
 *    i = s*N + k, i.e. field (i mod 5) of call floor(i/5); its value v
 *    becomes u = (2 v + 1) * 2^-24 and y_k = a_k + (b_k - a_k) * u.  The
 *    stream depends only on (seed, p, t, s, k), so any slice of the grid
 *    reproduces the full-grid values bit for bit.
 *  - Estimates: I_t = V * sum_s g / S with V = prod_k (b_k - a_k);
 *    mean = sum_t I_t / T; err = sqrt(sum_t (I_t - mean)^2 / (T (T-1)))
 *    (NaN when T = 1); errw = V * sqrt(mean_t[(s2_t - s1_t^2/S)/(S-1)]/(T S)),
 *    the pooled within-trial standard error (NaN when S = 1).
 *  - Host buffers belong to the caller; the library copies what it needs
 *    before returning.  Device buffers (ZMC_MEM_DEVICE) belong to the caller
 *    and must stay valid until the work enqueued on the stream completes.
 *  - One CUDA device: the current device of the calling thread.
 */
#ifndef ZMC_H_
#define ZMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZMC_ABI_VERSION 2
#define ZMC_MAX_N 8   /* integration dimensions   */
#define ZMC_MAX_M 16  /* parameters (value lists) */

typedef enum {
  ZMC_OK = 0,
  ZMC_EINVAL = 1,      /* an argument is out of range            */
  ZMC_ENOMEM = 2,      /* device or host memory could not be had */
  ZMC_ECUDA = 3,       /* a CUDA call failed                     */
  ZMC_ETIMEDOUT = 4,   /* a bounded wait ran out                 */
  ZMC_ECANCELED = 5,   /* the request was cancelled              */
  ZMC_EBUSY = 6,       /* the resource is in use                 */
  ZMC_ENOTFOUND = 7    /* unknown integrand id or ticket         */
} zmc_status;

/* The FP32 paths form each coordinate y and evaluate g in FP32 (cos/sin/exp on
 * the special-function unit), so a box far from the origin compared with its
 * width, or an integrand that cancels strongly, keeps only FP32's 24 bits;
 * ZMC_FP64 has no such limit.  Per sample the FP32 error is ~1e-7 of g. */
typedef enum {
  ZMC_FP64 = 0,        /* FP64 samples, integrand and sums                 */
  ZMC_FP32 = 1,        /* FP32 samples and integrand, plain FP32 lane sums  */
  ZMC_FP32_KAHAN = 2   /* FP32 samples and integrand, Kahan FP32 lane sums  */
} zmc_precision;       /* cross-lane reduction and the statistics: FP64    */

/* Integrand registry (compiled in).  x has M entries, y has N entries. */
enum {
  ZMC_G_CONST = 0,    /* g = 1                                      any M  */
  ZMC_G_COSPROD = 1,  /* g = prod_k cos(x_k y_k)                    M = N  */
  ZMC_G_GAUSS03 = 2,  /* g = exp(-sum_k (y_k - x_k)^2 / (2 0.3^2))  M = N  */
  ZMC_G_POLY = 3,     /* g = prod_k (1 + x_k y_k^2)                 M = N  */
  ZMC_G_OSC01 = 4,    /* g = cos(sum_k x_k y_k + 0.1 sum_k y_k^2)   M = N  */
  ZMC_G_SINSUM = 5,   /* g = sin(sum_k y_k + sum_l x_l)             any M  */
                      /*     (the test integrand of Eq. 2 and Eq. 4)       */
  ZMC_G_COUNT = 6
};

enum { ZMC_MEM_HOST = 0, ZMC_MEM_DEVICE = 1 };

/* zmc_scan_desc.flags */
enum {
  ZMC_F_TIMINGS = 1,  /* record CUDA-event timings into zmc_scan_out; the
                         call then waits for its work before returning   */
  ZMC_F_SYNC = 2,     /* wait for the enqueued work before returning      */
  ZMC_F_PLAN_ONLY = 4 /* validate and plan: fill the tile fields of the
                         output struct and return without computing      */
};

/*
 * One scan request.  Initialise with zmc_scan_desc_init() and set fields.
 *  integrand_id, N      registry id and dimension N in [1, ZMC_MAX_N]
 *  lo, hi               HOST arrays of N finite doubles, hi[k] > lo[k]
 *  M, list_len          M in [1, ZMC_MAX_M]; HOST array of M lengths >= 1;
 *                       the grid has P = prod list_len points (P < 2^62)
 *  list_vals            the M lists concatenated (sum list_len doubles);
 *                       host or device memory according to `mem`
 *  samples_per_point    S >= 1, with S * N <= 2^34 - 2^20
 *  trials               T in [1, 2^31)
 *  seed                 64-bit Philox key
 *  precision            a zmc_precision
 *  mem                  ZMC_MEM_HOST: list_vals and outputs are host memory
 *                       and the call is synchronous.  ZMC_MEM_DEVICE: they
 *                       are device memory and the call only enqueues work
 *                       on `stream` (unless flags ask to wait).
 *  first_index, count   the slice [first_index, first_index + count) of the
 *                       flat grid to evaluate; count = -1 means to the end.
 *                       count = 0 is a valid no-op.  Outputs hold `count`
 *                       entries, for the slice's points in order.
 *  stream               cudaStream_t to launch on; NULL is the CUDA default
 *                       (legacy) stream, as for other CUDA libraries
 *  workspace            optional device scratch of workspace_bytes bytes
 *                       (see zmc_workspace_size); NULL = the library takes
 *                       it from its stream-ordered memory pool
 *  tile_lanes, tile_splits, tile_block
 *                       0 = chosen by the planner/autotuner; otherwise
 *                       lanes per unit-split (power of two <= tile_block),
 *                       sample splits per (point, trial) unit, and threads
 *                       per block (64..512, multiple of 32)
 *  flags                ZMC_F_* bits
 *  chunk_points         zmc_scan_ex cuts the slice into chunks of this many
 *                       consecutive grid points (the batches of Sec. 2);
 *                       0 = chosen by the library: as many points as keep
 *                       one chunk's FP64 partial sums within 256 MiB and,
 *                       with host buffers, at most 1/8 of the slice (never
 *                       fewer than 2^20 points).  Every chunk uses the tile
 *                       plan of the whole call, so the results do not depend
 *                       on the chunking (bit for bit).  With host buffers and
 *                       more than one chunk, the device->host copy of chunk k
 *                       runs on a copy stream while chunk k+1 computes
 *                       (straight into the caller's arrays when they are
 *                       pinned, else through pinned staging buffers that the
 *                       library keeps for reuse).  >= 0; the server and the
 *                       batch calls ignore it.
 */
typedef struct zmc_scan_desc {
  int integrand_id;
  int N;
  const double* lo;
  const double* hi;
  int M;
  const int64_t* list_len;
  const double* list_vals;
  int64_t samples_per_point;
  int trials;
  uint64_t seed;
  int precision;
  int mem;
  int64_t first_index;
  int64_t count;
  void* stream;
  void* workspace;
  size_t workspace_bytes;
  int tile_lanes;
  int tile_splits;
  int tile_block;
  int flags;
  int64_t chunk_points;
} zmc_scan_desc;

/*
 * Outputs of one scan.  mean and err are required (count entries each);
 * errw, s1 and s2 are optional (NULL = not written).  s1 and s2 receive the
 * per-trial sums sum_s g and sum_s g^2, count*T entries, trial fastest.
 * All arrays are host or device memory according to desc->mem.
 * The remaining fields are written by the call: the tile configuration it
 * used, the number of chunks and, with ZMC_F_TIMINGS, CUDA-event times in
 * milliseconds (kernel_ms and finalize_ms summed over the chunks).
 */
typedef struct zmc_scan_out {
  double* mean;
  double* err;
  double* errw;
  double* s1;
  double* s2;
  int tile_lanes;
  int tile_splits;
  int tile_block;
  int launches;        /* kernels this call launched                      */
  float h2d_ms;        /* host->device copies (ZMC_MEM_HOST only)          */
  float kernel_ms;     /* the sampling kernel                              */
  float finalize_ms;   /* the cross-split reduction and statistics kernel  */
  float d2h_ms;        /* device->host copies (ZMC_MEM_HOST only) not
                          hidden behind the sampling of later chunks       */
  float total_ms;      /* first event to last event                        */
  int64_t chunks;      /* chunks the slice was cut into (see chunk_points) */
} zmc_scan_out;

typedef struct zmc_integrand_info {
  int id;
  char name[32];
  int m_rule;          /* 0: any M;  1: M must equal N                    */
} zmc_integrand_info;

typedef struct zmc_device_info {
  int device;
  int sm_count;
  int cc_major;
  int cc_minor;
  int max_threads_per_sm;
  int clock_khz;       /* reported maximum SM clock                       */
  size_t total_mem;
  char name[96];
} zmc_device_info;

/* ABI version (ZMC_ABI_VERSION of the built library). */
int zmc_version(void);

/* Message of the last failed call on this thread ("" if none).  The string
 * stays valid until the next call on the same thread. */
const char* zmc_last_error(void);

/* Fill a descriptor with defaults: FP32_KAHAN, host memory, the whole grid,
 * library stream, planner-chosen tiles, T = 1, S = 1.  Returns ZMC_OK, or
 * ZMC_EINVAL for a NULL pointer. */
int zmc_scan_desc_init(zmc_scan_desc* d);

/* Registry lookup; ZMC_ENOTFOUND for an unknown id. */
int zmc_integrand_info_get(int id, zmc_integrand_info* info);

/* Properties of the current device; ZMC_ECUDA when there is none. */
int zmc_device_info_get(zmc_device_info* info);

/*
 * Check a descriptor without touching a GPU: ZMC_OK if zmc_scan_ex would
 * accept it, else ZMC_EINVAL / ZMC_ENOTFOUND with zmc_last_error() set.
 * For ZMC_MEM_HOST the pointers are dereferenced only for lo, hi and list_len.
 */
int zmc_validate(const zmc_scan_desc* d);

/*
 * Device scratch that zmc_scan_ex needs for `d` with its tile configuration
 * (after planning): 16 bytes per (point, trial, split) of one chunk for the
 * FP64 partial sums, plus the device copy of the lists and of the outputs of
 * one chunk (two when the slice takes several chunks) when
 * d->mem == ZMC_MEM_HOST.  Touches no GPU when the tiles are given
 * explicitly; otherwise it may query the device for its SM count.
 */
int zmc_workspace_size(const zmc_scan_desc* d, size_t* bytes);

/*
 * The simple entry point (Sec. 2: a grid of parameters in, a grid of
 * integrals out).  All pointers are HOST memory; precision FP32_KAHAN;
 * the whole grid; synchronous.  out_mean and out_err hold P doubles.
 */
int zmc_scan(int integrand_id, int N, const double* lo, const double* hi,
             int M, const int64_t* list_len, const double* list_vals,
             int64_t samples_per_point, int trials, uint64_t seed,
             double* out_mean, double* out_err);

/* The general entry point: every option of zmc_scan_desc. */
int zmc_scan_ex(const zmc_scan_desc* d, zmc_scan_out* o);

/*
 * Raw random words of one unit's stream: out[i] = word (first_word + i) of
 * grid point p, trial t, under `seed`, where word w is output word (w mod 4)
 * of call floor(w/4) (the calls at the top of this file; the samples' 23-bit
 * fields are cut from these words).  out is HOST memory of nwords entries;
 * first_word + nwords <= 2^34, nwords <= 2^30.  Computed on the GPU by the
 * same Philox code the sampling kernels use.  Synchronous.
 */
int zmc_stream_words(uint64_t seed, int64_t p, int t, uint64_t first_word,
                     int64_t nwords, uint32_t* out);

/*
 * Device-side checks.  A library built with -DZMC_DEBUG=1 (libzmc_debug.so,
 * paper_1910_01965_gb300/build.py --debug) checks every grid index, list
 * digit and offset, staged-table slot, batch tile and partial-sum slot before
 * the access; a failed check skips the access and is recorded on the device
 * (nothing traps).  zmc_scan_ex then waits for its work and fails with
 * ZMC_ECUDA and a message if a check failed.  This call waits for the current
 * device, returns the number of failed checks recorded since the last call
 * (the first one's check code and index in *code and *index, either may be
 * NULL) and clears them; it returns -1 in a build without checks.  Check
 * codes: 1 grid index outside the slice, 2 list digit or offset out of range,
 * 3 staged-list slot beyond the shared memory, 4 partial-sum slot, 5 batch
 * tile, 6 finalize index.  The paper has no counterpart (a test aid).
 */
int64_t zmc_debug_failures(unsigned* code, long long* index);

/*
 * A scan that allocates nothing.  The paper has no counterpart: this serves
 * callers that cannot call cudaMalloc (or any allocator) when they scan —
 * code on a latency-critical path, where an allocation can wait on the
 * driver or synchronise the device; code inside a host framework that owns
 * all device memory through its own allocator and budget; hosts that fix
 * their device footprint at start-up.
 *
 * Same computation and kernels as zmc_scan_ex, and the same tile plan (the
 * autotuner's entry for the scan's class when the tiles are left open, else
 * the fixed rules), so the results equal zmc_scan_ex's bit for bit.
 * d->mem must be ZMC_MEM_DEVICE (lists and outputs in caller-owned device
 * memory), d->workspace NULL, and ZMC_F_TIMINGS unset; ZMC_F_SYNC is
 * honoured, and ZMC_F_PLAN_ONLY fills the tile fields and returns without
 * computing.  The slice is not chunked (chunk_points is ignored).  Work is
 * enqueued on d->stream (NULL = the CUDA default stream).
 *
 * Scratch: the FP64 partial sums live in a file-scope device array of
 * ZMC_NOALLOC_SCRATCH_BYTES (16 MiB).  A call whose partial sums
 * (points x trials x sample splits x 16 bytes) exceed it returns ZMC_EINVAL
 * with a message; scan a smaller slice (first_index, count) per call.
 * CUDA loads device code lazily: the first call on a device loads the module
 * that holds the array, which reserves its 16 MiB there, looks up its device
 * address (once per device, with that device current) and reads the
 * autotuner's cache file if ZMC_AUTOTUNE_CACHE names one.  That first call can
 * therefore allocate, wait on the driver, or fail with ZMC_ENOMEM/ZMC_ECUDA;
 * make it once at start-up (a small warm-up scan), before any stream capture.
 * Later calls on that device allocate nothing; the device holds the array
 * until the process exits.  All calls share the array and it keeps the last
 * call's contents; nothing in it needs clearing, but calls that overlap on
 * the GPU race on it.
 */
#define ZMC_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int zmc_scan_noalloc(const zmc_scan_desc* d, zmc_scan_out* o);

#ifdef __cplusplus
}
#endif

#endif /* ZMC_H_ */
