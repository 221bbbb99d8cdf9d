// zmc_runtime.h — host-side helpers shared by the runtime translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "zmc_internal.h"

namespace zmc {

struct TilePlan {
  int lanes = 32;   // threads summing one unit-split (power of two)
  int splits = 1;   // sample ranges per (point, trial) unit
  int block = 256;  // threads per block
};

// Byte offsets of each region inside one scan's device scratch.  The slice
// is cut into `chunks` chunks of `chunk_points` grid points; the partial sums
// hold one chunk, the host-memory output regions `nbuf` chunks each.
struct ScanLayout {
  size_t partial, partial_bytes;
  size_t vals, mean, err, errw, s1, s2;  // SIZE_MAX when not used
  size_t total;
  int64_t chunk_points = 0, chunks = 0;
  int nbuf = 1;
};

int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();
const char* last_error();

int validate(const zmc_scan_desc* d, int64_t* P_out, int64_t* count_out);
TilePlan plan_tiles(int N, int64_t S, int T, int64_t count, int sm_count, int threads_per_sm,
                    int lanes_req, int splits_req, int block_req, int precision);
// The tile plan of a scan on a device with `sm` SMs of `tps` threads each:
// an autotuner entry for the scan's class when the caller leaves the tiles
// open and one is recorded (memory reads only), else plan_tiles.
TilePlan plan_with(const zmc_scan_desc* d, int64_t count, int sm, int tps);
// plan_with for the current device (its properties from the device state),
// after loading the autotuner's cache file once.
int plan_for(const zmc_scan_desc* d, int64_t count, TilePlan* tp);
// User integrands compiled at run time (zmc_user.cu).
bool is_user_integrand(int id);
int user_validate(const zmc_scan_desc* d);
int user_info(int id, zmc_integrand_info* info);
int user_launch(const zmc_scan_desc* d, const ScanArgs& a, int block, int64_t grid, size_t smem,
                cudaStream_t stream);
// Tuned-table access (zmc_tune.cu).  tune_find reads memory only.
void tune_ensure_loaded();
bool tune_find(int prec, int gid, int N, int64_t S, int* lanes, int* block, int* gpl);
ScanLayout layout_for(const zmc_scan_desc* d, int64_t count, const TilePlan& tp);
int64_t chunk_points_for(const zmc_scan_desc* d, int64_t count, const TilePlan& tp);
double box_volume(const zmc_scan_desc* d);
void fill_scan_args(const zmc_scan_desc* d, int64_t count, const TilePlan& tp,
                    const double* vals_dev, double* partial_dev, ScanArgs* a);
int launch_scan_args(const zmc_scan_desc* d, const ScanArgs& a, const TilePlan& tp,
                     cudaStream_t stream);
int scan_ex(const zmc_scan_desc* d, zmc_scan_out* o);
// The current device's check words in ZMC_DEBUG builds (once its state is set
// up by an allocating entry point), else null.
unsigned long long* debug_words();
// ZMC_DEBUG builds: wait for the device, read and clear its check words;
// returns the failed checks since the last read (first failure in *code and
// *index), or -1 in release builds.
int64_t debug_take(unsigned* code, long long* index);

}  // namespace zmc
