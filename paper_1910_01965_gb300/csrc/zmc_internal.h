// zmc_internal.h — types shared by the runtime and the kernel translation units.
#pragma once

#include <cstdint>

#include "../../include/zmc.h"

namespace zmc {

// Philox4x32-10 constants (Salmon et al., SC'11).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Largest list staging in shared memory (doubles).
constexpr int kMaxSmemVals = 4096;

// ---------------------------------------------------------- debug checks --
// Builds with -DZMC_DEBUG=1 check every grid index, list digit and offset,
// staged-table slot, batch tile and partial-sum slot before the access.  A
// failed check skips the access (a safe index is used instead) and records
// itself in three device words [code of the first failure, its index, number
// of failures]; nothing traps.  Release builds compile the checks away.
#ifndef ZMC_DEBUG
#define ZMC_DEBUG 0
#endif
enum {
  kDbgGridIndex = 1,    // a unit's grid index outside the slice
  kDbgListOffset = 2,   // a mixed-radix digit or list offset out of range
  kDbgStagedTable = 3,  // a staged-list slot beyond the dynamic shared memory
  kDbgPartialSlot = 4,  // a partial-sum slot beyond the launch's unit-splits
  kDbgTile = 5,         // a batch tile or its scan out of range
  kDbgFinalize = 6      // a finalize index beyond its scan's points
};

// Everything one launch of the sampling kernel needs, passed by value.
// A "unit" is one (grid point, trial) pair; its S samples are cut into
// `splits` contiguous ranges of sample groups, and each range (a
// "unit-split") is summed by `lanes` threads of one block.
struct ScanArgs {
  int64_t first;        // first flat grid index of the slice
  int64_t count;        // grid points in the slice
  int64_t S;            // samples per unit
  int64_t ngroups;      // sample groups per unit: ceil(S / G)
  int64_t gps;          // sample groups per split: ceil(ngroups / splits)
  int64_t n_us;         // unit-splits: count * T * splits
  int32_t T;
  int32_t M;
  int32_t splits;
  int32_t lanes;        // power of two, <= blockDim.x
  int32_t lanes_log2;
  int32_t nvals;        // total list length
  int32_t stage_smem;   // 1: lists copied to shared memory first
  int32_t idx32;        // 1: every flat index of the slice is below 2^32
  int32_t gid;          // integrand id (batched launches dispatch on it)
  int32_t N;            // dimension
  const double* vals;   // device, the M lists concatenated
  int64_t len[ZMC_MAX_M];
  int32_t off[ZMC_MAX_M];
  double lo[ZMC_MAX_N];
  double hi[ZMC_MAX_N];
  uint32_t rk0[10];     // Philox round keys: key0 + r * W0
  uint32_t rk1[10];     // Philox round keys: key1 + r * W1
  double* partial;      // device, [n_us][2] FP64 (sum g, sum g^2)
  unsigned long long* dbg;  // device check words (ZMC_DEBUG builds), or null
};

struct FinalizeArgs {
  int64_t count;
  int64_t S;
  int32_t T;
  int32_t splits;
  double V;
  const double* partial;
  double* mean;
  double* err;
  double* errw;   // may be null
  double* s1;     // may be null, [count][T]
  double* s2;     // may be null, [count][T]
  unsigned long long* dbg = nullptr;  // device check words (ZMC_DEBUG builds)
};

// Each Philox call gives five 23-bit fields.  Samples per group G and calls
// per group C for dimension N (1..8): G samples use exactly G*N = 5*C
// consecutive fields, so a group starts and ends on call boundaries.
constexpr int kFieldsPerCall = 5;
constexpr int group_samples(int N) { return (N % 5 == 0) ? 1 : 5; }
constexpr int group_calls(int N) { return N * group_samples(N) / kFieldsPerCall; }

// Launches of one precision's sampling kernel for (integrand, N).
// Returns a CUDA error code (0 = success).
typedef int (*ScanLaunchFn)(const ScanArgs& a, int block, int64_t grid,
                            size_t smem, void* stream);

ScanLaunchFn scan_launcher(int precision, int integrand, int N);
int finalize_launch(const FinalizeArgs& a, void* stream);

// ------------------------------------------------------------- batches --
// One tile = the unit-splits one block sums at once, all of one scan.
struct BatchTile {
  int32_t scan;      // index into the batch's ScanArgs array
  int32_t units;     // unit-splits in this tile (<= block / lanes)
  int64_t first_us;  // first unit-split of the tile
};

struct BatchArgs {
  const ScanArgs* scans;          // [nscans], device
  const BatchTile* tiles;         // [ntiles], device, in the order they are taken
  int64_t ntiles;
  unsigned long long* counter;    // device; zeroed before each launch
  int32_t nscans = 0;             // entries of scans (checked in ZMC_DEBUG builds)
  unsigned long long* dbg = nullptr;  // device check words (ZMC_DEBUG builds)
};

struct FinalizeBatchArgs {
  const FinalizeArgs* fa;   // [nscans], device
  const int64_t* prefix;    // [nscans + 1], device: first flat output index of each scan
  int32_t nscans;
  int64_t total;            // prefix[nscans]
};

// Launch the persistent batched sampling kernel of one precision.
int batch_launch(int precision, const BatchArgs& b, int grid, int block, size_t smem,
                 void* stream);
// Blocks of the batched kernel that fit on one SM at `block` threads, `smem` bytes.
int batch_blocks_per_sm(int precision, int block, size_t smem, int* out);
int finalize_batch_launch(const FinalizeBatchArgs& a, void* stream);

int stream_words_launch(uint64_t seed, int64_t p, int t, uint64_t first_word,
                        int64_t nwords, uint32_t* out_dev, void* stream);

#ifdef __CUDACC__
#if ZMC_DEBUG
// Record a failed check (first failure's code and index, failure count).
__device__ __forceinline__ bool dbg_ok(unsigned long long* w, bool ok, unsigned code,
                                       long long index) {
  if (!ok && w) {
    if (atomicCAS(&w[0], 0ull, static_cast<unsigned long long>(code)) == 0ull)
      w[1] = static_cast<unsigned long long>(index);
    atomicAdd(&w[2], 1ull);
  }
  return ok;
}
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned v;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}
#define ZMC_CHECK(w, cond, code, index) \
  ::zmc::dbg_ok((w), (cond), (code), static_cast<long long>(index))
#else
#define ZMC_CHECK(w, cond, code, index) true
#endif
#endif  // __CUDACC__

}  // namespace zmc
