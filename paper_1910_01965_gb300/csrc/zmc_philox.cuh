// zmc_philox.cuh — device Philox4x32-10 stream for the sampling kernels.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32->64 multiplies whose high halves are XORed with the other counter
// words and the round key.  The stream of a unit (grid point p, trial t)
// uses counter (j, t, p mod 2^32, p >> 32) and key (seed mod 2^32,
// seed >> 32); j is the only word that varies along the stream.
//
// Because three of the four counter words are fixed per unit, round 1's
// second multiply and round 2's first multiply do not depend on j.  They are
// computed once per unit (PhiloxUnit) and the per-call work drops from 20 to
// 18 multiplies.  The outputs are bit-identical to the plain ten rounds.
#pragma once

#include <cstdint>

#include "zmc_internal.h"

namespace zmc {

__device__ __forceinline__ void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi,
                                          uint32_t& lo) {
  uint64_t prod;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(prod) : "r"(a), "r"(b));
  lo = static_cast<uint32_t>(prod);
  hi = static_cast<uint32_t>(prod >> 32);
}

// Per-unit constants of rounds 1 and 2.
struct PhiloxUnit {
  uint32_t a2;   // p_hi ^ rk1[0]           (round 1, XOR into word 2)
  uint32_t b0;   // lo(M1 * p_lo) ^ rk0[1]  (round 2, XOR into word 0)
  uint32_t b1;   // hi(M0 * c0') ^ rk1[1]   (round 2, XOR into word 2)
  uint32_t b2;   // lo(M0 * c0')            (round 2, word 3)
};

__device__ __forceinline__ PhiloxUnit philox_unit(const uint32_t* rk0,
                                                  const uint32_t* rk1,
                                                  uint64_t p, uint32_t t) {
  const uint32_t plo = static_cast<uint32_t>(p);
  const uint32_t phi = static_cast<uint32_t>(p >> 32);
  // Round 1, the j-independent half: (H1, L1) = mulhilo(M1, p_lo).
  uint32_t H1, L1;
  mulhilo32(kPhiloxM1, plo, H1, L1);
  const uint32_t c0 = H1 ^ t ^ rk0[0];  // round-1 output word 0
  const uint32_t c1 = L1;               // round-1 output word 1
  // Round 2, the j-independent half: mulhilo(M0, c0).
  uint32_t H0b, L0b;
  mulhilo32(kPhiloxM0, c0, H0b, L0b);
  PhiloxUnit u;
  u.a2 = phi ^ rk1[0];
  u.b0 = c1 ^ rk0[1];
  u.b1 = H0b ^ rk1[1];
  u.b2 = L0b;
  return u;
}

// (hi:lo) += (ahi:alo), a 64-bit add on the integer ALU.
__device__ __forceinline__ void add64(uint32_t& lo, uint32_t& hi, uint32_t alo, uint32_t ahi) {
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;"
      : "+r"(lo), "+r"(hi) : "r"(alo), "r"(ahi));
}

// Four words of the call whose round-1 product M0 * j is (H0:L0).  A lane
// walking j in fixed strides carries this product with one 64-bit add per
// call instead of a 32x32->64 multiply.
__device__ __forceinline__ void philox_call_pre(const PhiloxUnit& u,
                                                const uint32_t* __restrict__ rk0,
                                                const uint32_t* __restrict__ rk1,
                                                uint32_t H0, uint32_t L0, uint32_t* out) {
  // Round 1: words become (c0, c1, H0 ^ p_hi ^ k1, L0).
  const uint32_t c2 = H0 ^ u.a2;
  // Round 2: only mulhilo(M1, c2) depends on j.
  uint32_t H1, L1;
  mulhilo32(kPhiloxM1, c2, H1, L1);
  uint32_t x0 = H1 ^ u.b0;
  uint32_t x1 = L1;
  uint32_t x2 = L0 ^ u.b1;
  uint32_t x3 = u.b2;
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(kPhiloxM0, x0, hi0, lo0);
    mulhilo32(kPhiloxM1, x2, hi1, lo1);
    const uint32_t n0 = hi1 ^ x1 ^ rk0[r];
    const uint32_t n2 = hi0 ^ x3 ^ rk1[r];
    x0 = n0;
    x1 = lo1;
    x2 = n2;
    x3 = lo0;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

// Four words of call j of the unit's stream.
__device__ __forceinline__ void philox_call(const PhiloxUnit& u,
                                            const uint32_t* __restrict__ rk0,
                                            const uint32_t* __restrict__ rk1,
                                            uint32_t j, uint32_t* out) {
  uint32_t H0, L0;
  mulhilo32(kPhiloxM0, j, H0, L0);
  philox_call_pre(u, rk0, rk1, H0, L0, out);
}

// Round-1 products M0 * j for j = j0, j0 + stride, j0 + 2 stride, ...
struct StridedProduct {
  uint32_t lo, hi;    // M0 * j (current)
  uint32_t dlo, dhi;  // M0 * stride
  __device__ __forceinline__ void init(uint32_t j0, uint32_t stride) {
    mulhilo32(kPhiloxM0, j0, hi, lo);
    mulhilo32(kPhiloxM0, stride, dhi, dlo);
  }
  __device__ __forceinline__ void advance() { add64(lo, hi, dlo, dhi); }
  // M0 * (j + c) for a small constant c: M0 * j plus the constant M0 * c (a
  // 64-bit add of an immediate), so the calls of one group share one product.
  __device__ __forceinline__ void at(int c, uint32_t& H, uint32_t& L) const {
    const uint64_t v = ((static_cast<uint64_t>(hi) << 32) | lo) +
                       static_cast<uint64_t>(kPhiloxM0) * static_cast<uint64_t>(c);
    L = static_cast<uint32_t>(v);
    H = static_cast<uint32_t>(v >> 32);
  }
};

}  // namespace zmc
