// zmc_finalize.cu — K2: per-point statistics from the unit-split partial sums,
// and the raw-stream kernel behind zmc_stream_words.
//
// For each grid point of the slice (one thread per point, consecutive threads
// on consecutive points so every output write is coalesced):
//   s1_t = sum over splits of sum g,  s2_t likewise for g^2 (fixed order),
//   I_t = V s1_t / S,  mean = sum_t I_t / T                (direct MC, Sec. 2)
//   err = sqrt(sum_t (I_t - mean)^2 / (T (T - 1)))         (trials, Sec. 3.2)
//   errw = V sqrt(mean_t[(s2_t - s1_t^2 / S) / (S - 1)] / (T S))
// all in FP64.
#include <cmath>
#include <cstdint>

#include "zmc_internal.h"
#include "zmc_philox.cuh"

namespace zmc {

// Point i's statistics from its 2 T splits partial sums at `part` (global or
// shared memory), summed in a fixed order.
__device__ __forceinline__ void finalize_point_from(const FinalizeArgs& a, int64_t i,
                                                    const double* part) {
  const double S = static_cast<double>(a.S);
  double sumI = 0.0, pooled = 0.0;
  for (int t = 0; t < a.T; ++t) {
    double s1 = 0.0, s2 = 0.0;
    const double* pt = part + 2 * static_cast<int64_t>(t) * a.splits;
    for (int k = 0; k < a.splits; ++k) {
      s1 += pt[2 * k];
      s2 += pt[2 * k + 1];
    }
    if (a.s1) a.s1[i * a.T + t] = s1;
    if (a.s2) a.s2[i * a.T + t] = s2;
    sumI += a.V * s1 / S;
    pooled += (s2 - s1 * s1 / S) / (S - 1.0);
  }
  const double mean = sumI / a.T;
  double dev2 = 0.0;
  if (a.T > 1) {
    for (int t = 0; t < a.T; ++t) {
      const double* pt = part + 2 * static_cast<int64_t>(t) * a.splits;
      double s1 = 0.0;
      for (int k = 0; k < a.splits; ++k) s1 += pt[2 * k];
      const double dI = a.V * s1 / S - mean;
      dev2 += dI * dI;
    }
  }
  a.mean[i] = mean;
  a.err[i] = a.T > 1 ? sqrt(dev2 / (static_cast<double>(a.T) * (a.T - 1))) : NAN;
  if (a.errw)
    a.errw[i] = a.S > 1 ? a.V * sqrt(pooled / a.T / (static_cast<double>(a.T) * S)) : NAN;
}

__device__ __forceinline__ void finalize_point(const FinalizeArgs& a, int64_t i) {
  finalize_point_from(a, i, a.partial + 2 * (i * a.T) * a.splits);
}

// The partial sums of a block's points are one contiguous range.  When it fits
// in shared memory (2 T splits <= 24 at 256 threads) the block first copies it
// with consecutive threads on consecutive doubles (coalesced reads), then each
// thread sums its own point from shared memory; otherwise each thread reads its
// point's sums from global memory.  The sums and their order are the same.
constexpr int kFinalizeStageDoubles = 6144;  // 48 KB

__global__ void finalize_kernel(const __grid_constant__ FinalizeArgs a) {
  __shared__ double stage[kFinalizeStageDoubles];
  const int64_t first = static_cast<int64_t>(blockIdx.x) * blockDim.x;
  const int64_t n = min(static_cast<int64_t>(blockDim.x), a.count - first);
  const int64_t per = 2 * static_cast<int64_t>(a.T) * a.splits;
  if (per * blockDim.x <= kFinalizeStageDoubles) {
    const double* src = a.partial + first * per;
    for (int64_t k = threadIdx.x; k < n * per; k += blockDim.x) stage[k] = src[k];
    __syncthreads();
    if (threadIdx.x < n) finalize_point_from(a, first + threadIdx.x, stage + threadIdx.x * per);
  } else if (threadIdx.x < n) {
    finalize_point(a, first + threadIdx.x);
  }
}

// Every point of every scan of a batch: thread i finds its scan by binary
// search over the prefix array (consecutive threads on consecutive points of
// one scan, so writes stay coalesced).
__global__ void finalize_batch_kernel(const __grid_constant__ FinalizeBatchArgs b) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= b.total) return;
  int lo = 0, hi = b.nscans - 1;
  while (lo < hi) {  // the last scan whose prefix is <= i
    const int mid = (lo + hi + 1) >> 1;
    if (b.prefix[mid] <= i) lo = mid; else hi = mid - 1;
  }
  const int64_t k = i - b.prefix[lo];
  if (ZMC_CHECK(b.fa[lo].dbg, k >= 0 && k < b.fa[lo].count, kDbgFinalize, i))
    finalize_point(b.fa[lo], k);
}

int finalize_batch_launch(const FinalizeBatchArgs& a, void* stream) {
  if (a.total <= 0) return 0;
  const int block = 256;
  const int64_t grid = (a.total + block - 1) / block;
  finalize_batch_kernel<<<static_cast<unsigned>(grid), block, 0,
                          static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

int finalize_launch(const FinalizeArgs& a, void* stream) {
  if (a.count <= 0) return 0;
  const int block = 256;
  const int64_t grid = (a.count + block - 1) / block;
  finalize_kernel<<<static_cast<unsigned>(grid), block, 0,
                    static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

// Raw words w = first_word + i of the stream of unit (p, t), through the same
// per-unit hoisted Philox as the sampling kernels.
struct WordsArgs {
  uint32_t rk0[10];
  uint32_t rk1[10];
  uint64_t p;
  uint32_t t;
  uint64_t first_word;
  int64_t n;
  uint32_t* out;
};

__global__ void stream_words_kernel(const __grid_constant__ WordsArgs a) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint64_t w = a.first_word + static_cast<uint64_t>(i);
  const PhiloxUnit u = philox_unit(a.rk0, a.rk1, a.p, a.t);
  uint32_t r[4];
  philox_call(u, a.rk0, a.rk1, static_cast<uint32_t>(w >> 2), r);
  a.out[i] = r[w & 3u];
}

int stream_words_launch(uint64_t seed, int64_t p, int t, uint64_t first_word,
                        int64_t nwords, uint32_t* out_dev, void* stream) {
  if (nwords <= 0) return 0;
  WordsArgs a;
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    a.rk0[r] = k0 + static_cast<uint32_t>(r) * kPhiloxW0;
    a.rk1[r] = k1 + static_cast<uint32_t>(r) * kPhiloxW1;
  }
  a.p = static_cast<uint64_t>(p);
  a.t = static_cast<uint32_t>(t);
  a.first_word = first_word;
  a.n = nwords;
  a.out = out_dev;
  const int block = 256;
  const int64_t grid = (nwords + block - 1) / block;
  stream_words_kernel<<<static_cast<unsigned>(grid), block, 0,
                        static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace zmc
