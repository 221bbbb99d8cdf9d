// zmc_scan_inst.cu — instantiates the sampling kernel for one precision and
// one integrand, N = 1..8.  Compiled once per (ZMC_INST_PREC, ZMC_INST_GID)
// pair so that the 144 kernels build in parallel.
#include "zmc_scan_kernel.cuh"

#ifndef ZMC_INST_PREC
#error "ZMC_INST_PREC must be defined"
#endif
#ifndef ZMC_INST_GID
#error "ZMC_INST_GID must be defined"
#endif

namespace zmc {

#if ZMC_INST_PREC == 0
#define ZMC_F(name) name##64
#else
#define ZMC_F(name) name##32
#endif

#if ZMC_INST_GID == 0
#define ZMC_FUNCTOR ZMC_F(Const)
#elif ZMC_INST_GID == 1
#define ZMC_FUNCTOR ZMC_F(CosProd)
#elif ZMC_INST_GID == 2
#define ZMC_FUNCTOR ZMC_F(Gauss)
#elif ZMC_INST_GID == 3
#define ZMC_FUNCTOR ZMC_F(Poly)
#elif ZMC_INST_GID == 4
#define ZMC_FUNCTOR ZMC_F(Osc)
#elif ZMC_INST_GID == 5
#define ZMC_FUNCTOR ZMC_F(SinSum)
#else
#error "unknown ZMC_INST_GID"
#endif

#define ZMC_ROW_NAME2(p, g) scan_row_p##p##_g##g
#define ZMC_ROW_NAME(p, g) ZMC_ROW_NAME2(p, g)

ScanLaunchFn ZMC_ROW_NAME(ZMC_INST_PREC, ZMC_INST_GID)(int N) {
  static const ScanLaunchFn row[8] = {
      &launch_scan<1, ZMC_FUNCTOR<1>, ZMC_INST_PREC>,
      &launch_scan<2, ZMC_FUNCTOR<2>, ZMC_INST_PREC>,
      &launch_scan<3, ZMC_FUNCTOR<3>, ZMC_INST_PREC>,
      &launch_scan<4, ZMC_FUNCTOR<4>, ZMC_INST_PREC>,
      &launch_scan<5, ZMC_FUNCTOR<5>, ZMC_INST_PREC>,
      &launch_scan<6, ZMC_FUNCTOR<6>, ZMC_INST_PREC>,
      &launch_scan<7, ZMC_FUNCTOR<7>, ZMC_INST_PREC>,
      &launch_scan<8, ZMC_FUNCTOR<8>, ZMC_INST_PREC>,
  };
  return (N >= 1 && N <= 8) ? row[N - 1] : nullptr;
}

}  // namespace zmc
