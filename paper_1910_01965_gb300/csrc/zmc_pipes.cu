// zmc_pipes.cu — instruction-throughput probes behind include/zmc_pipes.h.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "../../include/zmc_pipes.h"
#include "zmc_philox.cuh"
#include "zmc_runtime.h"

namespace zmc {

constexpr int kChains = 8;

template <int PIPE>
__device__ __forceinline__ void pipe_step(uint32_t (&u)[kChains], float (&f)[kChains],
                                          double (&d)[kChains], uint64_t (&w)[kChains],
                                          uint64_t (&v)[kChains], uint64_t vab,
                                          uint32_t c1, uint32_t c2, float fa, float fb,
                                          double da, double db, const PhiloxUnit& pu,
                                          const uint32_t* rk0, const uint32_t* rk1) {
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    if constexpr (PIPE == ZMC_PIPE_FFMA) {
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(fa), "f"(fb));
    } else if constexpr (PIPE == ZMC_PIPE_IMAD) {
      asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(u[k]) : "r"(c1), "r"(c2));
    } else if constexpr (PIPE == ZMC_PIPE_IMAD_WIDE) {
      // the low word of the running value is the next multiplicand
      asm volatile("{ .reg .u32 t; cvt.u32.u64 t, %0; mad.wide.u32 %0, t, %1, %0; }"
                   : "+l"(w[k]) : "r"(c1));
    } else if constexpr (PIPE == ZMC_PIPE_IMAD_HI) {
      asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(u[k]) : "r"(c1), "r"(c2));
    } else if constexpr (PIPE == ZMC_PIPE_LOP3) {
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[k]) : "r"(c1), "r"(c2));
    } else if constexpr (PIPE == ZMC_PIPE_SHF) {
      asm volatile("shf.r.wrap.b32 %0, %0, %1, 9;" : "+r"(u[k]) : "r"(c1));
    } else if constexpr (PIPE == ZMC_PIPE_MUFU_RSQ) {
      asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f[k]));
    } else if constexpr (PIPE == ZMC_PIPE_MUFU_EX2) {
      asm volatile("{ .reg .f32 t; neg.f32 t, %0; ex2.approx.ftz.f32 %0, t; }" : "+f"(f[k]));
    } else if constexpr (PIPE == ZMC_PIPE_MUFU_COS) {
      asm volatile("cos.approx.ftz.f32 %0, %0;" : "+f"(f[k]));
    } else if constexpr (PIPE == ZMC_PIPE_MUFU_EX2LG2) {
      asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[k]));
      asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(f[k]));
    } else if constexpr (PIPE == ZMC_PIPE_DFMA) {
      asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[k]) : "d"(da), "d"(db));
    } else if constexpr (PIPE == ZMC_PIPE_FFMA2) {
      asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(v[k]) : "l"(vab));
    } else if constexpr (PIPE == ZMC_PIPE_WIDE_FFMA) {
      asm volatile("{ .reg .u32 t; cvt.u32.u64 t, %0; mad.wide.u32 %0, t, %1, %0; }"
                   : "+l"(w[k]) : "r"(c1));
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(fa), "f"(fb));
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(fa), "f"(fb));
    } else if constexpr (PIPE == ZMC_PIPE_WIDE_FFMA2) {
      asm volatile("{ .reg .u32 t; cvt.u32.u64 t, %0; mad.wide.u32 %0, t, %1, %0; }"
                   : "+l"(w[k]) : "r"(c1));
      asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(v[k]) : "l"(vab));
    } else if constexpr (PIPE == ZMC_PIPE_PHILOX) {
      uint32_t r[4];
      philox_call(pu, rk0, rk1, u[k], r);
      u[k] = r[0] ^ r[1] ^ r[2] ^ r[3];
    }
  }
}

// One 1024-thread block per SM: the launch asks for more than half of the
// SM's shared memory, so no second block can share an SM.
constexpr int kProbeSmem = 120 * 1024;

template <int PIPE>
__global__ void __launch_bounds__(1024, 1)
pipe_kernel(int iters, uint32_t seed, unsigned long long* cycles, uint32_t* sink) {
  uint32_t u[kChains];
  float f[kChains];
  double d[kChains];
  uint64_t w[kChains], v[kChains];
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    u[k] = tid * 2654435761u + k + seed;
    f[k] = 1.0f + 1e-3f * k + 1e-7f * (tid & 1023);
    d[k] = 1.0 + 1e-3 * k;
    w[k] = u[k];
    v[k] = (static_cast<uint64_t>(__float_as_uint(f[k] + 0.5f)) << 32) | __float_as_uint(f[k]);
  }
  uint32_t rk0[10], rk1[10];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk0[r] = seed + r * kPhiloxW0;
    rk1[r] = seed * 3u + r * kPhiloxW1;
  }
  const PhiloxUnit pu = philox_unit(rk0, rk1, tid, 0);
  const uint32_t c1 = 0x9E3779B9u ^ seed, c2 = 0x7f4a7c15u;
  const float fa = 0.99993f, fb = 7e-5f;
  const double da = 0.99993, db = 7e-5;
  // (0.99993, 0.99993) as a packed pair: v = v * 0.99993 + 0.99993 stays bounded
  const uint64_t vab = (static_cast<uint64_t>(__float_as_uint(fa)) << 32) | __float_as_uint(fa);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i)
    pipe_step<PIPE>(u, f, d, w, v, vab, c1, c2, fa, fb, da, db, pu, rk0, rk1);
  __syncthreads();
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    if constexpr (PIPE == ZMC_PIPE_FFMA || PIPE == ZMC_PIPE_MUFU_RSQ ||
                  PIPE == ZMC_PIPE_MUFU_EX2LG2 || PIPE == ZMC_PIPE_MUFU_EX2 ||
                  PIPE == ZMC_PIPE_MUFU_COS)
      acc ^= __float_as_uint(f[k]);
    else if constexpr (PIPE == ZMC_PIPE_DFMA)
      acc ^= static_cast<uint32_t>(__double_as_longlong(d[k]));
    else if constexpr (PIPE == ZMC_PIPE_IMAD_WIDE)
      acc ^= static_cast<uint32_t>(w[k]) ^ static_cast<uint32_t>(w[k] >> 32);
    else if constexpr (PIPE == ZMC_PIPE_FFMA2)
      acc ^= static_cast<uint32_t>(v[k]) ^ static_cast<uint32_t>(v[k] >> 32);
    else if constexpr (PIPE == ZMC_PIPE_WIDE_FFMA)
      acc ^= static_cast<uint32_t>(w[k]) ^ __float_as_uint(f[k]);
    else if constexpr (PIPE == ZMC_PIPE_WIDE_FFMA2)
      acc ^= static_cast<uint32_t>(w[k]) ^ static_cast<uint32_t>(v[k]) ^
             static_cast<uint32_t>(v[k] >> 32);
    else
      acc ^= u[k];
  }
  if (acc == 0x12345678u) sink[tid & 1023] = acc;  // keeps the chains alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(t1 - t0);
}

typedef void (*PipeKernel)(int, uint32_t, unsigned long long*, uint32_t*);

static PipeKernel pipe_kernel_for(int pipe) {
  switch (pipe) {
    case ZMC_PIPE_FFMA: return pipe_kernel<ZMC_PIPE_FFMA>;
    case ZMC_PIPE_IMAD: return pipe_kernel<ZMC_PIPE_IMAD>;
    case ZMC_PIPE_IMAD_WIDE: return pipe_kernel<ZMC_PIPE_IMAD_WIDE>;
    case ZMC_PIPE_IMAD_HI: return pipe_kernel<ZMC_PIPE_IMAD_HI>;
    case ZMC_PIPE_LOP3: return pipe_kernel<ZMC_PIPE_LOP3>;
    case ZMC_PIPE_SHF: return pipe_kernel<ZMC_PIPE_SHF>;
    case ZMC_PIPE_MUFU_RSQ: return pipe_kernel<ZMC_PIPE_MUFU_RSQ>;
    case ZMC_PIPE_MUFU_EX2: return pipe_kernel<ZMC_PIPE_MUFU_EX2>;
    case ZMC_PIPE_MUFU_COS: return pipe_kernel<ZMC_PIPE_MUFU_COS>;
    case ZMC_PIPE_MUFU_EX2LG2: return pipe_kernel<ZMC_PIPE_MUFU_EX2LG2>;
    case ZMC_PIPE_DFMA: return pipe_kernel<ZMC_PIPE_DFMA>;
    case ZMC_PIPE_PHILOX: return pipe_kernel<ZMC_PIPE_PHILOX>;
    case ZMC_PIPE_FFMA2: return pipe_kernel<ZMC_PIPE_FFMA2>;
    case ZMC_PIPE_WIDE_FFMA: return pipe_kernel<ZMC_PIPE_WIDE_FFMA>;
    case ZMC_PIPE_WIDE_FFMA2: return pipe_kernel<ZMC_PIPE_WIDE_FFMA2>;
    default: return nullptr;
  }
}

}  // namespace zmc

extern "C" int zmc_pipe_measure(int pipe, int iterations, zmc_pipe_result* out) {
  using namespace zmc;
  clear_error();
  PipeKernel k = pipe_kernel_for(pipe);
  if (!k) return fail(ZMC_EINVAL, "unknown pipe %d", pipe);
  if (!out) return fail(ZMC_EINVAL, "out is NULL");
  if (iterations < 1 || iterations > (1 << 24))
    return fail(ZMC_EINVAL, "iterations %d outside [1, 2^24]", iterations);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int block = 1024, blocks = sms;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kProbeSmem)) != cudaSuccess)
    return cuda_fail(e, "cudaFuncSetAttribute(probe smem)");
  unsigned long long* cyc = nullptr;
  uint32_t* sink = nullptr;
  if ((e = cudaMalloc(&cyc, blocks * sizeof(unsigned long long))) != cudaSuccess)
    return cuda_fail(e, "cudaMalloc(cycles)");
  if ((e = cudaMalloc(&sink, 1024 * sizeof(uint32_t))) != cudaSuccess) {
    cudaFree(cyc);
    return cuda_fail(e, "cudaMalloc(sink)");
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  k<<<blocks, block, kProbeSmem>>>(1, 1u, cyc, sink);  // warm-up
  e = cudaGetLastError();
  cudaEventRecord(a);
  if (e == cudaSuccess) {
    k<<<blocks, block, kProbeSmem>>>(iterations, 7u, cyc, sink);
    e = cudaGetLastError();
  }
  cudaEventRecord(b);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, a, b);
  unsigned long long* hc = new unsigned long long[blocks];
  if (e == cudaSuccess)
    e = cudaMemcpy(hc, cyc, blocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(cyc);
  cudaFree(sink);
  if (e != cudaSuccess) {
    delete[] hc;
    return cuda_fail(e, "pipe probe");
  }
  double mean_cyc = 0.0;
  for (int i = 0; i < blocks; ++i) mean_cyc += static_cast<double>(hc[i]);
  mean_cyc /= blocks;
  delete[] hc;
  const int per_step = (pipe == ZMC_PIPE_MUFU_EX2LG2 || pipe == ZMC_PIPE_FFMA2) ? 2 : 1;
  const double ops_per_block = static_cast<double>(block) * iterations * kChains * per_step;
  std::memset(out, 0, sizeof(*out));
  out->pipe = pipe;
  out->ops = static_cast<int64_t>(ops_per_block * blocks);
  out->ms = ms;
  out->ops_per_clk_per_sm = ops_per_block / mean_cyc;  // one block per SM
  out->ops_per_s = out->ops / (ms * 1e-3);
  out->clock_mhz = mean_cyc / (ms * 1e-3) / 1e6;
  return ZMC_OK;
}
