// zmc_scan_kernel.cuh — the sampling kernel (K1) and its building blocks.
//
// Direct Monte Carlo over a parameter grid (Eq. 1, Sec. 2): every unit
// (grid point p, trial t) sums g over its S samples.  The paper gives each
// grid point to one GPU thread that loops over all samples (Sec. 2, Fig. 1);
// here a unit's samples are cut into `splits` ranges and each range is summed
// by `lanes` threads, so that a grid of any shape fills all SMs.  Lane sums
// are reduced with warp shuffles and, for ranges wider than a warp, through
// shared memory, in a fixed order; each range writes one FP64 (sum g,
// sum g^2) pair.  The finalize kernel (K2) adds the ranges in order and forms
// the statistics.
//
// Sample groups: G = group_samples(N) consecutive samples use exactly
// C = group_calls(N) Philox calls (G*N = 5C fields), so a lane always works
// on whole groups and never shares a call with another lane.
#pragma once

#include <cstdint>

#include "zmc_integrands.cuh"
#include "zmc_internal.h"
#include "zmc_philox.cuh"

namespace zmc {

enum { kPrecFP64 = ZMC_FP64, kPrecFP32 = ZMC_FP32, kPrecFP32K = ZMC_FP32_KAHAN };

// Compile-time tuning knobs (defaults are the shipped configuration).
#ifndef ZMC_LB_THREADS
#define ZMC_LB_THREADS 512   // __launch_bounds__ maximum block size
#endif
#ifndef ZMC_LB_MIN_BLOCKS
#define ZMC_LB_MIN_BLOCKS 1  // __launch_bounds__ minimum resident blocks
#endif
// ZMC_CALLS_IN_FLIGHT, when defined, overrides every functor's kCallsInFlight
// (independent Philox calls per lane per loop block in the FP32 paths).

template <int PREC>
struct LaneAcc;

template <>
struct LaneAcc<kPrecFP64> {
  double s1 = 0.0, s2 = 0.0;
  __device__ __forceinline__ void add(double g) {
    s1 += g;
    s2 = fma(g, g, s2);
  }
  __device__ __forceinline__ void add2(double a, double b) {
    add(a);
    add(b);
  }
  template <int K>
  __device__ __forceinline__ void add_group(const double* v) {
#pragma unroll
    for (int i = 0; i < K; ++i) add(v[i]);
  }
  __device__ __forceinline__ double sum1() const { return s1; }
  __device__ __forceinline__ double sum2() const { return s2; }
};

template <>
struct LaneAcc<kPrecFP32> {
  float s1 = 0.0f, s2 = 0.0f;
  __device__ __forceinline__ void add(float g) {
    s1 += g;
    s2 = fmaf(g, g, s2);
  }
  __device__ __forceinline__ void add2(float a, float b) {
    add(a);
    add(b);
  }
  template <int K>
  __device__ __forceinline__ void add_group(const float* v) {
#pragma unroll
    for (int i = 0; i < K; ++i) add(v[i]);
  }
  __device__ __forceinline__ double sum1() const { return s1; }
  __device__ __forceinline__ double sum2() const { return s2; }
};

// Kahan-compensated FP32 sums: c carries the negated low part, so the lane's
// sum is s - c, taken in FP64.
template <>
struct LaneAcc<kPrecFP32K> {
  float s1 = 0.0f, c1 = 0.0f, s2 = 0.0f, c2 = 0.0f;
  __device__ __forceinline__ void add(float g) {
    const float y1 = g - c1;
    const float t1 = s1 + y1;
    c1 = (t1 - s1) - y1;
    s1 = t1;
    const float y2 = fmaf(g, g, -c2);
    const float t2 = s2 + y2;
    c2 = (t2 - s2) - y2;
    s2 = t2;
  }
  // Two samples: their plain FP32 pair sums enter the compensated sums (the
  // pair's own rounding is at the scale of one sample, not of the running
  // sum, which is what the compensation protects).
  __device__ __forceinline__ void add2(float a, float b) {
    const float u = a + b;
    const float v = fmaf(a, a, b * b);
    const float y1 = u - c1;
    const float t1 = s1 + y1;
    c1 = (t1 - s1) - y1;
    s1 = t1;
    const float y2 = v - c2;
    const float t2 = s2 + y2;
    c2 = (t2 - s2) - y2;
    s2 = t2;
  }
  // K samples at once (a sample group): their plain FP32 sums, formed in a
  // fixed order, enter the compensated sums in one step.
  template <int K>
  __device__ __forceinline__ void add_group(const float* v) {
    float u = v[0], w = v[0] * v[0];
#pragma unroll
    for (int i = 1; i < K; ++i) {
      u += v[i];
      w = fmaf(v[i], v[i], w);
    }
    const float y1 = u - c1;
    const float t1 = s1 + y1;
    c1 = (t1 - s1) - y1;
    s1 = t1;
    const float y2 = w - c2;
    const float t2 = s2 + y2;
    c2 = (t2 - s2) - y2;
    s2 = t2;
  }
  __device__ __forceinline__ double sum1() const {
    return static_cast<double>(s1) - static_cast<double>(c1);
  }
  __device__ __forceinline__ double sum2() const {
    return static_cast<double>(s2) - static_cast<double>(c2);
  }
};

// List that staged value `idx` belongs to.
__device__ __forceinline__ int list_of(const ScanArgs& a, int idx) {
  int k = 0;
  for (int i = 1; i < a.M; ++i)
    if (idx >= a.off[i]) k = i;
  return k;
}

// One mixed-radix digit: d = p mod L, p = p div L, in 32 bits when the whole
// slice's indices fit (the common case), else in 64.
__device__ __forceinline__ int64_t next_digit(const ScanArgs& a, int64_t& p, int64_t L) {
  if (a.idx32) {
    const uint32_t p32 = static_cast<uint32_t>(p), L32 = static_cast<uint32_t>(L);
    const uint32_t q = p32 / L32;
    p = q;
    return p32 - q * L32;
  }
  const int64_t q = p / L;
  const int64_t d = p - q * L;
  p = q;
  return d;
}

// Decode the flat grid index p (C order, last list fastest; Sec. 2: the grid
// is the Cartesian product of the lists) and hand the parameters to f.
// `table` is the block's staged per-value table (null when not staged) and
// `dimc` its per-dimension constants.
template <int N, class F>
__device__ __forceinline__ void load_params(const ScanArgs& a, const void* table,
                                            const float* dimc, int64_t p, F& f) {
  if constexpr (F::kTable) {
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      const int64_t d = next_digit(a, p, a.len[i]);
      int idx = a.off[i] + static_cast<int>(d);
      if (!ZMC_CHECK(a.dbg, d >= 0 && d < a.len[i] && idx < a.nvals, kDbgListOffset, idx))
        idx = 0;
      const float2 v = table ? static_cast<const float2*>(table)[idx]
                             : F::value(i, a.vals[idx], a.lo[i], a.hi[i]);
      f.load(i, v, &dimc[3 * i]);
    }
  } else if constexpr (F::kFixedM > 0) {
    // one compiled M: the parameters land in registers
    const double* vals = table ? static_cast<const double*>(table) : a.vals;
#pragma unroll
    for (int i = F::kFixedM - 1; i >= 0; --i) {
      const int64_t d = next_digit(a, p, a.len[i]);
      int64_t idx = a.off[i] + d;
      if (!ZMC_CHECK(a.dbg, d >= 0 && d < a.len[i] && idx < a.nvals, kDbgListOffset, idx))
        idx = 0;
      f.set_param(i, vals[idx]);
    }
    f.finish(a.lo, a.hi);
  } else if constexpr (F::kPerDim) {
    // M == N: parameter i pairs with dimension i.
    const double* vals = table ? static_cast<const double*>(table) : a.vals;
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      const int64_t d = next_digit(a, p, a.len[i]);
      int64_t idx = a.off[i] + d;
      if (!ZMC_CHECK(a.dbg, d >= 0 && d < a.len[i] && idx < a.nvals, kDbgListOffset, idx))
        idx = 0;
      f.set(i, vals[idx], a.lo[i], a.hi[i]);
    }
  } else {
    const double* vals = table ? static_cast<const double*>(table) : a.vals;
    for (int i = a.M - 1; i >= 0; --i) {
      const int64_t d = next_digit(a, p, a.len[i]);
      int64_t idx = a.off[i] + d;
      if (!ZMC_CHECK(a.dbg, d >= 0 && d < a.len[i] && idx < a.nvals, kDbgListOffset, idx))
        idx = 0;
      f.add(vals[idx]);
    }
    f.finish(a.lo, a.hi);
  }
}

// Stage the lists into shared memory: per-value FP32 constants for kTable
// functors, the FP64 values otherwise.  Every thread of the block calls it.
template <int N, class F>
__device__ __forceinline__ const void* stage_lists(const ScanArgs& a, double* smem,
                                                   float* dimc) {
  if constexpr (F::kTable) {
    if (threadIdx.x < N)
      F::dim(threadIdx.x, a.lo[threadIdx.x], a.hi[threadIdx.x], &dimc[3 * threadIdx.x]);
    if (a.stage_smem) {
      float2* tab = reinterpret_cast<float2*>(smem);
      for (int i = threadIdx.x; i < a.nvals; i += blockDim.x) {
        if (!ZMC_CHECK(a.dbg, (i + 1) * sizeof(float2) <= dynamic_smem_bytes(),
                       kDbgStagedTable, i))
          break;
        const int k = list_of(a, i);
        tab[i] = F::value(k, a.vals[i], a.lo[k], a.hi[k]);
      }
    }
    __syncthreads();
    return a.stage_smem ? smem : nullptr;
  } else {
    if (a.stage_smem) {
      for (int i = threadIdx.x; i < a.nvals; i += blockDim.x) {
        if (!ZMC_CHECK(a.dbg, (i + 1) * sizeof(double) <= dynamic_smem_bytes(),
                       kDbgStagedTable, i))
          break;
        smem[i] = a.vals[i];
      }
      __syncthreads();
      return smem;
    }
    return nullptr;
  }
}

// Sample g of a group whose C calls' words are r[0 .. 4C): its N unit values
// come from the group's fields g*N .. g*N + N - 1 (field e is field e mod 5
// of the group's call e / 5).
template <int N, class F>
__device__ __forceinline__ auto eval_sample(const F& f, const uint32_t* r, int g) {
  typename F::unit_t u[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int e = g * N + k;
    u[k] = field_unit<typename F::unit_t>(
        field23(r + 4 * (e / kFieldsPerCall), e % kFieldsPerCall));
  }
  return f.eval(u);
}

// Sum over the sample groups [q, q_end) with stride `step` (one lane).
//
// Order of the compensated additions (the same for every blocking choice
// below, so the single-scan and batched kernels agree bit for bit): with
// G = 5, each group's five samples enter in one step (LaneAcc::add_group), in
// group order; with G = 1, consecutive groups are paired and a last unpaired
// group enters alone.
template <int N, class F, int PREC>
__device__ __forceinline__ void lane_groups(const uint32_t* __restrict__ rk0,
                                            const uint32_t* __restrict__ rk1,
                                            const PhiloxUnit& pu, const F& f, uint32_t q,
                                            uint32_t q_end, uint32_t step,
                                            LaneAcc<PREC>& acc) {
  constexpr int G = group_samples(N);
  constexpr int C = group_calls(N);
  // Groups per loop block: about kCallsInFlight independent Philox chains
  // per lane (a group of C calls already has C).  The FP64 path is bound by
  // its FP64 arithmetic, not by the stream: one group at a time.
#ifdef ZMC_CALLS_IN_FLIGHT
  constexpr int kCalls = PREC == kPrecFP64 ? 1 : ZMC_CALLS_IN_FLIGHT;
#else
  constexpr int kCalls = PREC == kPrecFP64 ? 1 : F::kCallsInFlight;
#endif
  constexpr int kBlock = kCalls / C > 1 ? kCalls / C : 1;
  // M0 * j for the lane's calls, carried along by 64-bit adds: call c of
  // group q has j = q C + c; the product for q C advances with the lane's
  // stride and call c adds the constant M0 c to it.
  StridedProduct sp;
  sp.init(q * C, step * C);
  auto call = [&](int c, uint32_t* out) {
    uint32_t H, L;
    sp.at(c, H, L);
    philox_call_pre(pu, rk0, rk1, H, L, out);
  };
  // Draw the words of V consecutive groups of this lane.
  auto draw = [&](auto& r) {
    constexpr int V = sizeof(r) / sizeof(r[0]);
#pragma unroll
    for (int u = 0; u < V; ++u) {
#pragma unroll
      for (int c = 0; c < C; ++c) call(c, &r[u][4 * c]);
      sp.advance();
    }
  };
  if constexpr (G > 1) {
    constexpr int U = kBlock;
    using T = typename F::unit_t;
    auto consume = [&](const auto& r) {
      constexpr int V = sizeof(r) / sizeof(r[0]);
#pragma unroll
      for (int u = 0; u < V; ++u) {
        T v[G];
#pragma unroll
        for (int g = 0; g < G; ++g) v[g] = eval_sample<N>(f, r[u], g);
        acc.template add_group<G>(v);
      }
    };
    if constexpr (U == 1 && C > 2) {
      // One long group at a time: each call is drawn just before the first
      // sample that reads it, so a call's words die once its last sample is
      // evaluated (fewer live registers than drawing all C calls first).
      for (; q < q_end; q += step) {
        uint32_t r[4 * C];
        T v[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int c0 = g == 0 ? 0 : (g * N - 1) / kFieldsPerCall + 1;
          const int c1 = (g * N + N - 1) / kFieldsPerCall;
#pragma unroll
          for (int c = c0; c <= c1; ++c) call(c, &r[4 * c]);
          v[g] = eval_sample<N>(f, r, g);
        }
        acc.template add_group<G>(v);
        sp.advance();
      }
    } else {
      for (; q + (U - 1) * step < q_end; q += U * step) {
        uint32_t r[U][4 * C];
        draw(r);
        consume(r);
      }
      if constexpr (U > 1) {
        for (; q < q_end; q += step) {
          uint32_t r[1][4 * C];
          draw(r);
          consume(r);
        }
      }
    }
  } else {
    // G == 1: consecutive groups are paired; U groups (U/2 pairs) per block.
    constexpr int U = kBlock >= 2 ? kBlock & ~1 : 2;
    auto consume = [&](const auto& r) {
      constexpr int V = sizeof(r) / sizeof(r[0]);
#pragma unroll
      for (int u = 0; u < V; u += 2)
        acc.add2(eval_sample<N>(f, r[u], 0), eval_sample<N>(f, r[u + 1], 0));
    };
    for (; q + (U - 1) * step < q_end; q += U * step) {
      uint32_t r[U][4 * C];
      draw(r);
      consume(r);
    }
    // Fewer than U groups left: pairs, then a single group.
    if constexpr (U > 2) {
      for (; q + step < q_end; q += 2 * step) {
        uint32_t r[2][4 * C];
        draw(r);
        consume(r);
      }
    }
    if (q < q_end) {
      uint32_t r[1][4 * C];
      draw(r);
      acc.add(eval_sample<N>(f, r[0], 0));
    }
  }
}

// The ragged last group of a unit when G does not divide S: its valid samples
// enter one at a time.
template <int N, class F, int PREC>
__device__ __forceinline__ void lane_tail_group(const uint32_t* __restrict__ rk0,
                                                const uint32_t* __restrict__ rk1,
                                                const PhiloxUnit& pu, const F& f, uint32_t q,
                                                int valid, LaneAcc<PREC>& acc) {
  constexpr int G = group_samples(N);
  constexpr int C = group_calls(N);
  uint32_t r[4 * C];
#pragma unroll
  for (int c = 0; c < C; ++c) philox_call(pu, rk0, rk1, q * C + c, &r[4 * c]);
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (g < valid) acc.add(eval_sample<N>(f, r, g));
}

// Work of one lane for unit-split `us`: decode, prepare, sample, sum.
// rk0/rk1 are the ten Philox round keys (parameter space in the single-scan
// kernel, registers in the batched one).
template <int N, class F, int PREC>
__device__ __forceinline__ void unit_split_lane(const ScanArgs& a, const uint32_t* rk0,
                                                const uint32_t* rk1, const void* table,
                                                const float* dimc, int64_t us, int lane,
                                                LaneAcc<PREC>& acc) {
  constexpr int G = group_samples(N);
  const int64_t unit = us / a.splits;
  const int64_t split = us - unit * a.splits;
  const int64_t lp = unit / a.T;
  const uint32_t t = static_cast<uint32_t>(unit - lp * a.T);
  const int64_t p = a.first + lp;
  if (!ZMC_CHECK(a.dbg, us >= 0 && lp < a.count && split < a.splits, kDbgGridIndex, us))
    return;

  F f{};
  load_params<N>(a, table, dimc, p, f);
  if constexpr (!F::kUsesSamples) {
    // g does not depend on y: the stream is not drawn at all.
    const int64_t q0 = split * a.gps;
    const int64_t q1 = min(q0 + a.gps, a.ngroups);
    for (int64_t q = q0 + lane; q < q1; q += a.lanes) {
      const int64_t left = a.S - q * G;
      const int cnt = left < G ? static_cast<int>(left) : G;
      for (int g = 0; g < cnt; ++g) acc.add(f.eval(nullptr));
    }
  } else {
    const PhiloxUnit pu = philox_unit(rk0, rk1, static_cast<uint64_t>(p), t);
    const int64_t q0 = split * a.gps;
    const int64_t q1 = min(q0 + a.gps, a.ngroups);
    const int64_t nfull = a.S / G;
    const int64_t qf = min(q1, nfull);
    if (q0 + lane < qf)
      lane_groups<N, F, PREC>(rk0, rk1, pu, f, static_cast<uint32_t>(q0 + lane),
                              static_cast<uint32_t>(qf), static_cast<uint32_t>(a.lanes),
                              acc);
    if (G > 1) {
      const int valid = static_cast<int>(a.S - nfull * G);
      if (valid > 0 && nfull >= q0 && nfull < q1 && ((nfull - q0) & (a.lanes - 1)) == lane)
        lane_tail_group<N, F, PREC>(rk0, rk1, pu, f, static_cast<uint32_t>(nfull), valid, acc);
    }
  }
}

// Reduce (s1, s2) over the `lanes` threads of each unit-split, in a fixed
// order.  Every thread of the block must call it.  Lane 0 of the unit-split
// returns the totals.
__device__ __forceinline__ void reduce_unit_split(const ScanArgs& a, double& s1,
                                                  double& s2, double* red) {
  const int width = a.lanes < 32 ? a.lanes : 32;
  for (int m = width >> 1; m >= 1; m >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, m);
    s2 += __shfl_xor_sync(0xffffffffu, s2, m);
  }
  if (a.lanes > 32) {
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red[2 * warp] = s1;
      red[2 * warp + 1] = s2;
    }
    __syncthreads();
    if ((threadIdx.x & (a.lanes - 1)) == 0) {
      const int wpu = a.lanes >> 5;
      double t1 = red[2 * warp], t2 = red[2 * warp + 1];
      for (int w = 1; w < wpu; ++w) {
        t1 += red[2 * (warp + w)];
        t2 += red[2 * (warp + w) + 1];
      }
      s1 = t1;
      s2 = t2;
    }
  }
}

template <int N, class F, int PREC>
__global__ void __launch_bounds__(ZMC_LB_THREADS, ZMC_LB_MIN_BLOCKS)
scan_kernel(const __grid_constant__ ScanArgs a) {
  extern __shared__ double smem[];
  __shared__ double red[64];
  __shared__ float dimc[3 * ZMC_MAX_N];
  const void* table = stage_lists<N, F>(a, smem, dimc);
  const int lane = threadIdx.x & (a.lanes - 1);
  const int64_t us = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> a.lanes_log2) +
                     (threadIdx.x >> a.lanes_log2);
  LaneAcc<PREC> acc;
  if (us < a.n_us) unit_split_lane<N, F, PREC>(a, a.rk0, a.rk1, table, dimc, us, lane, acc);
  double s1 = acc.sum1(), s2 = acc.sum2();
  reduce_unit_split(a, s1, s2, red);
  if (lane == 0 && us < a.n_us && ZMC_CHECK(a.dbg, us >= 0, kDbgPartialSlot, us)) {
    a.partial[2 * us] = s1;
    a.partial[2 * us + 1] = s2;
  }
}

#ifndef __CUDACC_RTC__
template <int N, class F, int PREC>
int launch_scan(const ScanArgs& a, int block, int64_t grid, size_t smem, void* stream) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(scan_kernel<N, F, PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return static_cast<int>(e);
  }
  scan_kernel<N, F, PREC><<<static_cast<unsigned>(grid), block, smem,
                            static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}
#endif  // __CUDACC_RTC__

}  // namespace zmc
