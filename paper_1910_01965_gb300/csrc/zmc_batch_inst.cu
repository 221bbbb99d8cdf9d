// zmc_batch_inst.cu — the persistent batched sampling kernel (K3) for one
// precision (compiled once per ZMC_INST_PREC).
//
// Many scans of different integrands, dimensions, grid sizes and sample counts
// run in one launch.  The host cuts every scan into tiles — the unit-splits one
// block sums at once, all of one scan — and orders them longest first.  Each
// resident block takes the next tile from a device counter (one atomicAdd by
// thread 0, no waiting on other blocks), stages that scan's lists or constant
// tables into shared memory when the scan changes, copies its Philox round
// keys into registers, and runs the same per-lane sampling and reduction code
// as the single-scan kernel, writing each unit-split's FP64 partial sums into
// that scan's slice of the batch's partial buffer.
// The batched bodies keep as many Philox calls in flight per lane as the
// single-scan kernel; the order of the compensated additions does not depend
// on the blocking in any case, so results stay bit-identical to solo runs.
#include "zmc_scan_kernel.cuh"

#ifndef ZMC_INST_PREC
#error "ZMC_INST_PREC must be defined"
#endif

namespace zmc {

#if ZMC_INST_PREC == 0
#define ZMC_BF(name) name##64
#else
#define ZMC_BF(name) name##32
#endif

// Resident blocks per SM the register allocation is held to: 2 x 256 threads
// (128 registers), so that the FP32 bodies do not spill; the largest bodies
// set the residency of the whole launch (measured: faster than 85 or 64).
#ifndef ZMC_BATCH_MIN_BLOCKS
#define ZMC_BATCH_MIN_BLOCKS 2
#endif

// One tile.  Not inlined: each (integrand, N) body gets its own register
// allocation instead of the union of all 48 bodies (one call per tile).
template <int N, class F, int PREC>
__device__ __noinline__ void batch_tile(const ScanArgs& a, const BatchTile& t, bool restage,
                                           double* smem, float* dimc, double* red) {
  // Lists / tables of this scan (kept when the previous tile was the same scan).
  const void* table = nullptr;
  if (restage) {
    table = stage_lists<N, F>(a, smem, dimc);
  } else {
    table = a.stage_smem ? static_cast<const void*>(smem) : nullptr;
  }
  uint32_t rk0[10], rk1[10];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk0[r] = a.rk0[r];
    rk1[r] = a.rk1[r];
  }
  const int lane = threadIdx.x & (a.lanes - 1);
  const int local = threadIdx.x >> a.lanes_log2;
  const bool active = local < t.units;
  const int64_t us = t.first_us + local;
  LaneAcc<PREC> acc;
  if (active) unit_split_lane<N, F, PREC>(a, rk0, rk1, table, dimc, us, lane, acc);
  double s1 = acc.sum1(), s2 = acc.sum2();
  reduce_unit_split(a, s1, s2, red);
  if (lane == 0 && active && ZMC_CHECK(a.dbg, us >= 0 && us < a.n_us, kDbgPartialSlot, us)) {
    a.partial[2 * us] = s1;
    a.partial[2 * us + 1] = s2;
  }
}

#define ZMC_CASE_N(gid, F, n)                                                        \
  case (gid)*8 + (n)-1:                                                              \
    batch_tile<n, F<n>, ZMC_INST_PREC>(a, t, restage, smem, dimc, red);              \
    break;
#define ZMC_CASES(gid, F)                                                            \
  ZMC_CASE_N(gid, F, 1) ZMC_CASE_N(gid, F, 2) ZMC_CASE_N(gid, F, 3)                  \
  ZMC_CASE_N(gid, F, 4) ZMC_CASE_N(gid, F, 5) ZMC_CASE_N(gid, F, 6)                  \
  ZMC_CASE_N(gid, F, 7) ZMC_CASE_N(gid, F, 8)

template <int PREC>
__global__ void __launch_bounds__(256, ZMC_BATCH_MIN_BLOCKS)
batch_kernel(const __grid_constant__ BatchArgs b) {
  extern __shared__ double smem[];
  __shared__ double red[64];
  __shared__ float dimc[3 * ZMC_MAX_N];
  __shared__ long long s_tile;
  int staged = -1;  // scan whose lists/tables are in shared memory
  for (;;) {
    if (threadIdx.x == 0) s_tile = static_cast<long long>(atomicAdd(b.counter, 1ull));
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= b.ntiles) break;
    const BatchTile t = b.tiles[tile];
    if (ZMC_CHECK(b.dbg, t.scan >= 0 && t.scan < b.nscans && t.units >= 0, kDbgTile, tile)) {
      const ScanArgs& a = b.scans[t.scan];
      const bool restage = t.scan != staged;
      staged = t.scan;
      switch (a.gid * 8 + a.N - 1) {
        ZMC_CASES(ZMC_G_CONST, ZMC_BF(Const))
        ZMC_CASES(ZMC_G_COSPROD, ZMC_BF(CosProd))
        ZMC_CASES(ZMC_G_GAUSS03, ZMC_BF(Gauss))
        ZMC_CASES(ZMC_G_POLY, ZMC_BF(Poly))
        ZMC_CASES(ZMC_G_OSC01, ZMC_BF(Osc))
        ZMC_CASES(ZMC_G_SINSUM, ZMC_BF(SinSum))
        default:
          break;
      }
    }
    __syncthreads();  // the tile is done before shared memory or s_tile is reused
  }
}

#define ZMC_BATCH_FN2(p) batch_launch_p##p
#define ZMC_BATCH_FN(p) ZMC_BATCH_FN2(p)
#define ZMC_BATCH_OCC2(p) batch_occupancy_p##p
#define ZMC_BATCH_OCC(p) ZMC_BATCH_OCC2(p)

int ZMC_BATCH_FN(ZMC_INST_PREC)(const BatchArgs& b, int grid, int block, size_t smem,
                                void* stream) {
  batch_kernel<ZMC_INST_PREC><<<grid, block, smem, static_cast<cudaStream_t>(stream)>>>(b);
  return static_cast<int>(cudaGetLastError());
}

int ZMC_BATCH_OCC(ZMC_INST_PREC)(int block, size_t smem, int* out) {
  return static_cast<int>(
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_kernel<ZMC_INST_PREC>, block,
                                                    smem));
}

}  // namespace zmc
