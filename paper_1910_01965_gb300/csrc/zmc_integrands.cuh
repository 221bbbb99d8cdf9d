// zmc_integrands.cuh — the compiled-in integrand registry, as device functors.
//
// Each functor evaluates g(y; x) (Eq. 1, Sec. 2) at one sample, reading the
// sample's N unit values f_k = 1 + v_k 2^-23 in [1, 2), one per dimension,
// where v_k is the sample's 23-bit random field for dimension k (five fields
// per Philox call; field23 below).  The box coordinate is
// u = f - (1 - 2^-24) = (2 v + 1) 2^-24, y = a + (b - a) u.
//
// Two families:
//  * FP64 functors (suffix 64, unit_t double) evaluate y and g in FP64, with
//    the affine steps folded into per-unit constants as below.
//  * FP32 functors (suffix 32, unit_t float) take f as a float built from
//    the field's bits, so y = (b - a) f + A with A = a - (b - a)(1 - 2^-24).
//    Everything affine in y that depends only on (x, box) is folded, in
//    FP64, into per-unit constants before the sample loop; each sample then
//    costs one FFMA per dimension before the integrand's own arithmetic.
//    cos/sin use the SFU (MUFU) approximations, exp uses ex2.approx.
//
// kCallsInFlight: independent Philox calls a lane keeps in flight per loop
// block in the FP32 paths (measured on GB300: eight for the Gaussian,
// cos-product and polynomial integrands, +1.6 % on the Gaussian at N = 4; four
// for the others, whose N <= 3 kernels lose 1 % with eight).  The FP64 path
// draws one group at a time (it is bound by its FP64 arithmetic).
// kFixedM > 0 marks a functor compiled for one number of parameters M (the
// run-time-compiled user integrands); it receives parameter i by set_param.
// `set(i, x_i, a_i, b_i)` receives parameter i and box side i (kPerDim: the
// integrand pairs x_k with y_k, M == N); `add(x_i)` receives parameters of the
// any-M integrands; `finish(lo, hi)` runs once after the parameters.  FP32
// functors with kTable take their constants from per-block tables instead
// (value / dim / load, below).
#pragma once

#include <cstdint>

namespace zmc {

constexpr double kOneMinusHalfUlp = 1.0 - 0x1p-24;     // 1 - 2^-24
constexpr double kGaussSigma = 0.3;
constexpr double kOscQuad = 0.1;
// sqrt(log2(e) / (2 sigma^2)) for sigma = 0.3: scales (y - x) so that
// exp(-(y-x)^2 / (2 sigma^2)) = 2^-(d^2).
constexpr double kGaussScale = 2.83107266762673;  // to double precision
// 1 / (2 sigma^2) for sigma = 0.3: the FP64 Gaussian multiplies instead of
// dividing (FP64 division is an iteration on GB300's narrow FP64 pipe); the
// two differ by at most one unit in the last place of the exponent.
constexpr double kGaussInvTwoSigma2 = 5.555555555555555;

// Field m (0..4) of one Philox call's four words: bits 23m .. 23m+22 of the
// 128-bit block r[0] + r[1] 2^32 + r[2] 2^64 + r[3] 2^96 (m is a constant
// wherever this is inlined, so the branch folds).
__device__ __forceinline__ uint32_t field23(const uint32_t* r, int m) {
  const int b = 23 * m, q = b >> 5, sh = b & 31;
  const uint32_t x = (sh + 23 <= 32) ? (r[q] >> sh) : __funnelshift_r(r[q], r[q + 1], sh);
  return x & 0x7fffffu;
}

// The unit value f = 1 + v 2^-23 of a 23-bit field v, built from bits (the
// mask above and the exponent below merge into one logic operation).
template <class T>
__device__ __forceinline__ T field_unit(uint32_t v);
template <>
__device__ __forceinline__ float field_unit<float>(uint32_t v) {
  return __uint_as_float(0x3f800000u | v);
}
template <>
__device__ __forceinline__ double field_unit<double>(uint32_t v) {
  return __longlong_as_double(
      static_cast<long long>(0x3FF0000000000000ull | (static_cast<uint64_t>(v) << 29)));
}

__device__ __forceinline__ float ex2_approx(float v) {
  float out;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(out) : "f"(v));
  return out;
}

// ------------------------------------------------------------------ FP64 --
// FP64 functors fold the affine steps in y into per-unit constants the same way
// the FP32 ones do: y = (b - a) f + A with A = a - (b - a)(1 - 2^-24), so each
// dimension costs one DFMA before the integrand's own arithmetic.  The result
// differs from forming u first by at most a unit in the last place of each
// coordinate.

template <int N>
struct Const64 {
  static constexpr bool kPerDim = false;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = false;
  static constexpr int kCallsInFlight = 1;
  static constexpr int kFixedM = 0;
  using unit_t = double;
  __device__ void add(double) {}
  __device__ void finish(const double*, const double*) {}
  __device__ double eval(const double*) const { return 1.0; }
};

// cos(x y) = cos(B f + C), B = x (b - a), C = x A.
template <int N>
struct CosProd64 {
  static constexpr bool kPerDim = true;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 1;
  static constexpr int kFixedM = 0;
  using unit_t = double;
  double B[N], C[N];
  __device__ void set(int i, double xi, double ai, double bi) {
    const double w = bi - ai;
    B[i] = xi * w;
    C[i] = xi * (ai - w * kOneMinusHalfUlp);
  }
  __device__ double eval(const double* f) const {
    double g = cos(fma(B[0], f[0], C[0]));
#pragma unroll
    for (int k = 1; k < N; ++k) g *= cos(fma(B[k], f[k], C[k]));
    return g;
  }
};

// y - x = W f + C, C = A - x.
template <int N>
struct Gauss64 {
  static constexpr bool kPerDim = true;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 1;
  static constexpr int kFixedM = 0;
  using unit_t = double;
  double W[N], C[N];
  __device__ void set(int i, double xi, double ai, double bi) {
    const double w = bi - ai;
    W[i] = w;
    C[i] = (ai - w * kOneMinusHalfUlp) - xi;
  }
  __device__ double eval(const double* f) const {
    double d = fma(W[0], f[0], C[0]);
    double q = d * d;
#pragma unroll
    for (int k = 1; k < N; ++k) {
      d = fma(W[k], f[k], C[k]);
      q = fma(d, d, q);
    }
    return exp(-q * kGaussInvTwoSigma2);
  }
};

template <int N>
struct Poly64 {
  static constexpr bool kPerDim = true;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 1;
  static constexpr int kFixedM = 0;
  using unit_t = double;
  double W[N], A[N], X[N];
  __device__ void set(int i, double xi, double ai, double bi) {
    const double w = bi - ai;
    W[i] = w;
    A[i] = ai - w * kOneMinusHalfUlp;
    X[i] = xi;
  }
  __device__ double eval(const double* f) const {
    double y = fma(W[0], f[0], A[0]);
    double g = fma(X[0] * y, y, 1.0);
#pragma unroll
    for (int k = 1; k < N; ++k) {
      y = fma(W[k], f[k], A[k]);
      g *= fma(X[k] * y, y, 1.0);
    }
    return g;
  }
};

template <int N>
struct Osc64 {
  static constexpr bool kPerDim = true;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 1;
  static constexpr int kFixedM = 0;
  using unit_t = double;
  double W[N], A[N], X[N];
  __device__ void set(int i, double xi, double ai, double bi) {
    const double w = bi - ai;
    W[i] = w;
    A[i] = ai - w * kOneMinusHalfUlp;
    X[i] = xi;
  }
  __device__ double eval(const double* f) const {
    double lin = 0.0, quad = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double y = fma(W[k], f[k], A[k]);
      lin = fma(X[k], y, lin);
      quad = fma(y, y, quad);
    }
    return cos(fma(kOscQuad, quad, lin));
  }
};

// sin(sum_k W_k f_k + C0), C0 = sum_k A_k + sum_l x_l.
template <int N>
struct SinSum64 {
  static constexpr bool kPerDim = false;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 1;
  static constexpr int kFixedM = 0;
  using unit_t = double;
  double xsum, W[N], C0;
  __device__ void add(double xi) { xsum += xi; }
  __device__ void finish(const double* lo, const double* hi) {
    double c = xsum;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double w = hi[k] - lo[k];
      W[k] = w;
      c += lo[k] - w * kOneMinusHalfUlp;
    }
    C0 = c;
  }
  __device__ double eval(const double* f) const {
    double s = C0;
#pragma unroll
    for (int k = 0; k < N; ++k) s = fma(W[k], f[k], s);
    return sin(s);
  }
};

// ------------------------------------------------------------------ FP32 --
// FP32 functors with a per-value table (kTable): while the lists are staged
// into shared memory each value x of list k becomes a float2 of per-value
// constants (value(k, x, a, b)), and each dimension gets up to three FP32
// per-dimension constants (dim(k, a, b, out)), both computed once per block in
// FP64.  A thread then sets up a unit with table lookups only (load()).

template <int N>
struct Const32 {
  static constexpr bool kPerDim = false;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = false;
  static constexpr int kCallsInFlight = 4;
  static constexpr int kFixedM = 0;
  using unit_t = float;
  __device__ void add(double) {}
  __device__ void finish(const double*, const double*) {}
  __device__ float eval(const float*) const { return 1.0f; }
};

// cos(x y) = cos(B f + C), B = x (b - a), C = x A.
template <int N>
struct CosProd32 {
  static constexpr bool kPerDim = true;
  static constexpr bool kTable = true;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 8;
  static constexpr int kFixedM = 0;
  using unit_t = float;
  float B[N], C[N];
  static __device__ float2 value(int, double x, double a, double b) {
    const double w = b - a;
    return make_float2(static_cast<float>(x * w),
                       static_cast<float>(x * (a - w * kOneMinusHalfUlp)));
  }
  static __device__ void dim(int, double, double, float*) {}
  __device__ void load(int k, float2 v, const float*) { B[k] = v.x; C[k] = v.y; }
  __device__ float eval(const float* f) const {
    float g = __cosf(fmaf(B[0], f[0], C[0]));
#pragma unroll
    for (int k = 1; k < N; ++k) g *= __cosf(fmaf(B[k], f[k], C[k]));
    return g;
  }
};

// exp(-(y-x)^2/(2 s^2)) per dimension = 2^-(d^2), d = c (y - x) = B f + C,
// B = c (b - a) per dimension, C = c (A - x) per value.
template <int N>
struct Gauss32 {
  static constexpr bool kPerDim = true;
  static constexpr bool kTable = true;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 8;
  static constexpr int kFixedM = 0;
  using unit_t = float;
  float B[N], C[N];
  static __device__ float2 value(int, double x, double a, double b) {
    const double w = b - a;
    return make_float2(static_cast<float>((a - w * kOneMinusHalfUlp - x) * kGaussScale), 0.f);
  }
  static __device__ void dim(int, double a, double b, float* out) {
    out[0] = static_cast<float>((b - a) * kGaussScale);
  }
  __device__ void load(int k, float2 v, const float* d) { B[k] = d[0]; C[k] = v.x; }
  __device__ float eval(const float* f) const {
    float d = fmaf(B[0], f[0], C[0]);
    float q = d * d;
#pragma unroll
    for (int k = 1; k < N; ++k) {
      d = fmaf(B[k], f[k], C[k]);
      q = fmaf(d, d, q);
    }
    return ex2_approx(-q);
  }
};

// prod (1 + x y^2), y = W f + A (per dimension), X = x (per value).
template <int N>
struct Poly32 {
  static constexpr bool kPerDim = true;
  static constexpr bool kTable = true;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 8;
  static constexpr int kFixedM = 0;
  using unit_t = float;
  float W[N], A[N], X[N];
  static __device__ float2 value(int, double x, double, double) {
    return make_float2(static_cast<float>(x), 0.f);
  }
  static __device__ void dim(int, double a, double b, float* out) {
    const double w = b - a;
    out[0] = static_cast<float>(w);
    out[1] = static_cast<float>(a - w * kOneMinusHalfUlp);
  }
  __device__ void load(int k, float2 v, const float* d) { W[k] = d[0]; A[k] = d[1]; X[k] = v.x; }
  __device__ float eval(const float* f) const {
    float y = fmaf(W[0], f[0], A[0]);
    float g = fmaf(X[0] * y, y, 1.0f);
#pragma unroll
    for (int k = 1; k < N; ++k) {
      y = fmaf(W[k], f[k], A[k]);
      g *= fmaf(X[k] * y, y, 1.0f);
    }
    return g;
  }
};

// cos(sum_k y_k (x_k + 0.1 y_k)), y = W f + A (per dimension), X = x.
template <int N>
struct Osc32 {
  static constexpr bool kPerDim = true;
  static constexpr bool kTable = true;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 4;
  static constexpr int kFixedM = 0;
  using unit_t = float;
  float W[N], A[N], X[N];
  static __device__ float2 value(int, double x, double, double) {
    return make_float2(static_cast<float>(x), 0.f);
  }
  static __device__ void dim(int, double a, double b, float* out) {
    const double w = b - a;
    out[0] = static_cast<float>(w);
    out[1] = static_cast<float>(a - w * kOneMinusHalfUlp);
  }
  __device__ void load(int k, float2 v, const float* d) { W[k] = d[0]; A[k] = d[1]; X[k] = v.x; }
  __device__ float eval(const float* f) const {
    float y = fmaf(W[0], f[0], A[0]);
    float ph = y * fmaf(static_cast<float>(kOscQuad), y, X[0]);
#pragma unroll
    for (int k = 1; k < N; ++k) {
      y = fmaf(W[k], f[k], A[k]);
      ph = fmaf(y, fmaf(static_cast<float>(kOscQuad), y, X[k]), ph);
    }
    return __cosf(ph);
  }
};

// sin(sum_k W_k f_k + C0), C0 = (sum_k A_k + sum_l x_l) reduced mod 2 pi in FP64.
template <int N>
struct SinSum32 {
  static constexpr bool kPerDim = false;
  static constexpr bool kTable = false;
  static constexpr bool kUsesSamples = true;
  static constexpr int kCallsInFlight = 4;
  static constexpr int kFixedM = 0;
  using unit_t = float;
  double xsum;
  float W[N], C0;
  __device__ void add(double xi) { xsum += xi; }
  __device__ void finish(const double* lo, const double* hi) {
    double c = xsum;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double w = hi[k] - lo[k];
      W[k] = static_cast<float>(w);
      c += lo[k] - w * kOneMinusHalfUlp;
    }
    const double two_pi = 6.283185307179586476925;
    c = c - two_pi * floor(c / two_pi);
    C0 = static_cast<float>(c);
  }
  __device__ float eval(const float* f) const {
    float s = C0;
#pragma unroll
    for (int k = 0; k < N; ++k) s = fmaf(W[k], f[k], s);
    return __sinf(s);
  }
};

}  // namespace zmc
