// zmc_user_functor.cuh — functors around a run-time-compiled user integrand.
//
// Included only by the translation unit that NVRTC compiles for a user
// integrand (zmc_user.cu), after the user's source and with ZMC_N and ZMC_M
// defined.  They map the sample's unit values f = 1 + v 2^-23 to y exactly
// as the built-in functors do (FP32: y = W f + A; FP64: y = fma(b - a, u, a)
// with u = f - (1 - 2^-24)) and call the user's g.
#pragma once

#include "zmc_integrands.cuh"

namespace zmc {

template <int N>
struct UserF32 {
  static constexpr bool kPerDim = false;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 4;
  static constexpr int kFixedM = ZMC_M;
  using unit_t = float;
  float W[N], A[N], X[ZMC_M];
  __device__ void set_param(int i, double xi) { X[i] = static_cast<float>(xi); }
  __device__ void add(double) {}
  __device__ void finish(const double* lo, const double* hi) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double w = hi[k] - lo[k];
      W[k] = static_cast<float>(w);
      A[k] = static_cast<float>(lo[k] - w * kOneMinusHalfUlp);
    }
  }
  __device__ float eval(const float* f) const {
    float y[N];
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] = fmaf(W[k], f[k], A[k]);
    return zmc_user_g32(y, X);
  }
};

template <int N>
struct UserF64 {
  static constexpr bool kPerDim = false;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 4;
  static constexpr int kFixedM = ZMC_M;
  using unit_t = double;
  double w[N], a[N], X[ZMC_M];
  __device__ void set_param(int i, double xi) { X[i] = xi; }
  __device__ void add(double) {}
  __device__ void finish(const double* lo, const double* hi) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      a[k] = lo[k];
      w[k] = hi[k] - lo[k];
    }
  }
  __device__ double eval(const double* f) const {
    double y[N];
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] = fma(w[k], f[k] - kOneMinusHalfUlp, a[k]);
    return zmc_user_g64(y, X);
  }
};

}  // namespace zmc
