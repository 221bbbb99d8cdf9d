/*
 * zmc_pipes.h — instruction-throughput micro-benchmarks (measurement support).
 *
 * The sampling kernels are bound by the SM's issue slots and its integer,
 * FP32, SFU and FP64 pipes, not by memory: the method's arithmetic is a
 * counter-based random stream, an integrand and two running sums per sample
 * (direct Monte Carlo, Sec. 2), with outputs of 16 bytes per grid point.
 * These probes measure, on the running GPU and at its running clock, how many
 * operations of one kind an SM retires per clock, so that the kernels'
 * achieved rates can be stated against measured ceilings.
 *
 * Each probe launches one block of 1024 threads per SM; every thread runs 8
 * independent dependency chains of the probed operation in a loop.  clock64()
 * brackets the loop in each block; results are averaged over blocks.
 */
#ifndef ZMC_PIPES_H_
#define ZMC_PIPES_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ZMC_PIPE_FFMA = 0,       /* fma.rn.f32                                  */
  ZMC_PIPE_IMAD = 1,       /* mad.lo.u32                                  */
  ZMC_PIPE_IMAD_WIDE = 2,  /* mad.wide.u32, the multiplicand loop-varying  */
  ZMC_PIPE_IMAD_HI = 3,    /* mad.hi.u32                                  */
  ZMC_PIPE_LOP3 = 4,       /* lop3.b32 (three-input XOR)                   */
  ZMC_PIPE_SHF = 5,        /* shf.r.wrap.b32 (funnel shift)                */
  ZMC_PIPE_MUFU_RSQ = 6,   /* rsqrt.approx.ftz.f32 (SFU)                   */
  ZMC_PIPE_MUFU_EX2LG2 = 7,/* ex2.approx.ftz.f32 + lg2.approx.ftz.f32 (SFU) */
  ZMC_PIPE_DFMA = 8,       /* fma.rn.f64                                  */
  ZMC_PIPE_PHILOX = 9,     /* one Philox4x32-10 call of the sampling kernels */
  ZMC_PIPE_MUFU_EX2 = 10,  /* ex2.approx.ftz.f32 of a negated input (SFU)  */
  ZMC_PIPE_MUFU_COS = 11,  /* cos.approx.ftz.f32 (SFU, plus its scaling)   */
  ZMC_PIPE_FFMA2 = 12,     /* fma.rn.f32x2 (two FP32 FMAs per instruction) */
  /* Mixed probes, counted in wide multiplies: each step is one mad.wide.u32
   * plus two FP32 FMAs, as two scalar instructions or one packed one, to show
   * whether the FP32 work takes issue cycles from the wide multiplies. */
  ZMC_PIPE_WIDE_FFMA = 13,
  ZMC_PIPE_WIDE_FFMA2 = 14,
  ZMC_PIPE_COUNT = 15
} zmc_pipe;

typedef struct zmc_pipe_result {
  int pipe;
  double ops_per_clk_per_sm;  /* operations (lane-level) per SM per clock   */
  double ops_per_s;           /* whole-GPU operations per second            */
  double clock_mhz;           /* SM clock implied by cycles / elapsed time  */
  double ms;                  /* elapsed time of the probe kernel            */
  int64_t ops;                /* operations executed                         */
} zmc_pipe_result;

/* Run one probe on the current device (synchronous).  ZMC_EINVAL for an
 * unknown pipe, ZMC_ECUDA / ZMC_ENOMEM on CUDA failures. */
int zmc_pipe_measure(int pipe, int iterations, zmc_pipe_result* out);

#ifdef __cplusplus
}
#endif

#endif /* ZMC_PIPES_H_ */
