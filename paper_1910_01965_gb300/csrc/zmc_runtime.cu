// zmc_runtime.cu — the C ABI of include/zmc.h: validation, tile planning,
// device memory, launches, copies and timings.
//
// Memory: device scratch comes from the caller (zmc_scan_desc.workspace) or
// from CUDA's stream-ordered pool (cudaMallocAsync / cudaFreeAsync on the
// launch stream; the pool keeps freed blocks for reuse).  Streams: the
// caller's (NULL = the CUDA default stream); the library's own non-blocking
// stream serves only its synchronous helpers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "zmc_internal.h"
#include "zmc_runtime.h"
#include "zmc_trace.h"

namespace zmc {

ScanLaunchFn scan_row_p0_g0(int), scan_row_p0_g1(int), scan_row_p0_g2(int),
    scan_row_p0_g3(int), scan_row_p0_g4(int), scan_row_p0_g5(int);
ScanLaunchFn scan_row_p1_g0(int), scan_row_p1_g1(int), scan_row_p1_g2(int),
    scan_row_p1_g3(int), scan_row_p1_g4(int), scan_row_p1_g5(int);
ScanLaunchFn scan_row_p2_g0(int), scan_row_p2_g1(int), scan_row_p2_g2(int),
    scan_row_p2_g3(int), scan_row_p2_g4(int), scan_row_p2_g5(int);

ScanLaunchFn scan_launcher(int precision, int integrand, int N) {
  typedef ScanLaunchFn (*RowFn)(int);
  static const RowFn rows[3][ZMC_G_COUNT] = {
      {scan_row_p0_g0, scan_row_p0_g1, scan_row_p0_g2, scan_row_p0_g3, scan_row_p0_g4,
       scan_row_p0_g5},
      {scan_row_p1_g0, scan_row_p1_g1, scan_row_p1_g2, scan_row_p1_g3, scan_row_p1_g4,
       scan_row_p1_g5},
      {scan_row_p2_g0, scan_row_p2_g1, scan_row_p2_g2, scan_row_p2_g3, scan_row_p2_g4,
       scan_row_p2_g5},
  };
  if (precision < 0 || precision > 2 || integrand < 0 || integrand >= ZMC_G_COUNT)
    return nullptr;
  return rows[precision][integrand](N);
}

// ------------------------------------------------------------ last error --
static thread_local std::string g_last_error;

int fail(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  log_msg(1, "status %d: %s", status, buf);
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(ZMC_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(ZMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_last_error.clear(); }
const char* last_error() { return g_last_error.c_str(); }

// ---------------------------------------------------------- device state --
struct DeviceState {
  bool init = false;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;  // device->host copies of chunked scans
  cudaDeviceProp prop{};
  unsigned long long* dbg = nullptr;   // check words (ZMC_DEBUG builds)
};

static std::mutex g_mu;
static DeviceState g_dev[64];

int device_state(DeviceState** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(ZMC_ECUDA, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& s = g_dev[dev];
  if (!s.init) {
    e = cudaGetDeviceProperties(&s.prop, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
    e = cudaStreamCreateWithFlags(&s.copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
#if ZMC_DEBUG
    e = cudaMalloc(reinterpret_cast<void**>(&s.dbg), 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s.dbg, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "debug check words");
#endif
    // Keep freed stream-ordered allocations in the pool for reuse.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s.init = true;
  }
  *out = &s;
  return ZMC_OK;
}

unsigned long long* debug_words() {
#if ZMC_DEBUG
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  return g_dev[dev].init ? g_dev[dev].dbg : nullptr;
#else
  return nullptr;
#endif
}

int64_t debug_take(unsigned* code, long long* index) {
#if ZMC_DEBUG
  unsigned long long* w = debug_words();
  if (!w) return 0;
  unsigned long long h[3] = {0, 0, 0};
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(w, 0, sizeof(h)) != cudaSuccess)
    return 0;
  if (code) *code = static_cast<unsigned>(h[0]);
  if (index) *index = static_cast<long long>(h[1]);
  if (h[2]) log_msg(1, "device-side check %u failed %llu times (first index %lld)",
                    static_cast<unsigned>(h[0]), h[2], static_cast<long long>(h[1]));
  return static_cast<int64_t>(h[2]);
#else
  (void)code;
  (void)index;
  return -1;
#endif
}

// ------------------------------------------------------------ validation --
static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int validate(const zmc_scan_desc* d, int64_t* P_out, int64_t* count_out) {
  if (!d) return fail(ZMC_EINVAL, "descriptor is NULL");
  const bool user = is_user_integrand(d->integrand_id);
  if (!user && (d->integrand_id < 0 || d->integrand_id >= ZMC_G_COUNT))
    return fail(ZMC_ENOTFOUND, "unknown integrand id %d", d->integrand_id);
  if (d->N < 1 || d->N > ZMC_MAX_N)
    return fail(ZMC_EINVAL, "N = %d outside [1, %d]", d->N, ZMC_MAX_N);
  if (d->M < 1 || d->M > ZMC_MAX_M)
    return fail(ZMC_EINVAL, "M = %d outside [1, %d]", d->M, ZMC_MAX_M);
  if (user) {
    const int ur = user_validate(d);
    if (ur != ZMC_OK) return ur;
  }
  const bool m_is_n = !user && d->integrand_id != ZMC_G_CONST &&
                      d->integrand_id != ZMC_G_SINSUM;
  if (m_is_n && d->M != d->N)
    return fail(ZMC_EINVAL, "integrand %d needs M == N (got M = %d, N = %d)",
                d->integrand_id, d->M, d->N);
  if (!d->lo || !d->hi) return fail(ZMC_EINVAL, "lo/hi is NULL");
  for (int k = 0; k < d->N; ++k) {
    if (!std::isfinite(d->lo[k]) || !std::isfinite(d->hi[k]) || !(d->hi[k] > d->lo[k]))
      return fail(ZMC_EINVAL, "box side %d is not finite with hi > lo", k);
  }
  if (!d->list_len) return fail(ZMC_EINVAL, "list_len is NULL");
  int64_t P = 1, nvals = 0;
  for (int i = 0; i < d->M; ++i) {
    const int64_t L = d->list_len[i];
    if (L < 1) return fail(ZMC_EINVAL, "list %d has length %lld < 1", i, (long long)L);
    if (P > (int64_t(1) << 62) / L) return fail(ZMC_EINVAL, "grid size overflows 2^62");
    P *= L;
    nvals += L;
    if (nvals > (int64_t(1) << 30)) return fail(ZMC_EINVAL, "lists hold more than 2^30 values");
  }
  if (!d->list_vals) return fail(ZMC_EINVAL, "list_vals is NULL");
  const int64_t S = d->samples_per_point;
  if (S < 1) return fail(ZMC_EINVAL, "samples_per_point = %lld < 1", (long long)S);
  // The word index s*N + k must leave the call index (word / 4) and the
  // in-kernel group counters inside 32 bits.
  const int64_t kMaxWords = (int64_t(1) << 34) - (int64_t(1) << 20);
  if (S > kMaxWords / d->N)
    return fail(ZMC_EINVAL, "samples_per_point * N exceeds 2^34 - 2^20");
  if (d->trials < 1) return fail(ZMC_EINVAL, "trials = %d < 1", d->trials);
  if (d->precision < ZMC_FP64 || d->precision > ZMC_FP32_KAHAN)
    return fail(ZMC_EINVAL, "unknown precision %d", d->precision);
  if (d->mem != ZMC_MEM_HOST && d->mem != ZMC_MEM_DEVICE)
    return fail(ZMC_EINVAL, "unknown memory kind %d", d->mem);
  if (d->first_index < 0 || d->first_index > P)
    return fail(ZMC_EINVAL, "first_index %lld outside [0, P = %lld]",
                (long long)d->first_index, (long long)P);
  int64_t count = d->count;
  if (count < 0) count = P - d->first_index;
  if (count > P - d->first_index)
    return fail(ZMC_EINVAL, "slice [%lld, %lld + %lld) exceeds P = %lld",
                (long long)d->first_index, (long long)d->first_index, (long long)count,
                (long long)P);
  if (d->trials > 0 && count > (int64_t(1) << 56) / d->trials)
    return fail(ZMC_EINVAL, "count * trials too large");
  if (d->tile_block != 0 &&
      (d->tile_block < 64 || d->tile_block > 512 || d->tile_block % 32 != 0))
    return fail(ZMC_EINVAL, "tile_block %d must be a multiple of 32 in [64, 512]",
                d->tile_block);
  if (d->tile_lanes != 0) {
    const int blk = d->tile_block ? d->tile_block : 256;
    if (!is_pow2(d->tile_lanes) || d->tile_lanes > blk || blk % d->tile_lanes != 0)
      return fail(ZMC_EINVAL, "tile_lanes %d must be a power of two dividing the block",
                  d->tile_lanes);
  }
  if (d->tile_splits < 0) return fail(ZMC_EINVAL, "tile_splits %d < 0", d->tile_splits);
  if (d->chunk_points < 0)
    return fail(ZMC_EINVAL, "chunk_points %lld < 0", (long long)d->chunk_points);
  if (P_out) *P_out = P;
  if (count_out) *count_out = count;
  return ZMC_OK;
}

// --------------------------------------------------------------- planner --
// Lanes per unit-split: the largest power of two <= 32 that still leaves each
// lane >= ZMC_PLAN_LANE_GROUPS sample groups (64 for plain FP32 lane sums,
// whose rounding grows with their length), then doubled while the launch has
// fewer than ~16 waves of resident threads and each lane keeps >= 64 groups.
// Every lane ends with FP64 work (its sums converted and reduced across the
// unit-split's lanes) on GB300's narrow FP64 unit, so fewer, longer lanes are
// faster when the grid fills the GPU anyway: measured on the Gaussian
// 10^6-point scan (2^14 samples), 4 lanes of 819 groups +2.8 % over 32 lanes
// of 102.  Splits: enough to give ~16 waves of resident threads, never fewer
// than 64 groups per lane.  Block: 256 threads.
#ifndef ZMC_PLAN_LANE_GROUPS
#define ZMC_PLAN_LANE_GROUPS 512
#endif
TilePlan plan_tiles(int N, int64_t S, int T, int64_t count, int sm_count,
                    int threads_per_sm, int lanes_req, int splits_req, int block_req,
                    int precision) {
  TilePlan tp;
  const int G = group_samples(N);
  const int64_t Q = (S + G - 1) / G;
  tp.block = block_req ? block_req : 256;
  int lanes = lanes_req;
  const int64_t units = std::max<int64_t>(1, count * T);
  const int64_t want = int64_t(16) * std::max(1, sm_count) * std::max(256, threads_per_sm);
  if (!lanes) {
    const int64_t min_groups = precision == ZMC_FP32 ? 64 : ZMC_PLAN_LANE_GROUPS;
    lanes = 32;
    while (lanes > 1 && Q / lanes < min_groups) lanes >>= 1;
    while (lanes < 32 && units * lanes < want && Q / (2 * lanes) >= 64) lanes <<= 1;
    lanes = std::min(lanes, tp.block);
  }
  tp.lanes = lanes;
  int64_t splits = splits_req;
  if (!splits) {
    const int64_t base = units * lanes;
    splits = (want + base - 1) / base;
    const int64_t cap = std::max<int64_t>(1, Q / (int64_t(lanes) * 64));
    splits = std::max<int64_t>(1, std::min(splits, cap));
  }
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, Q));
  splits = std::min<int64_t>(splits, int64_t(1) << 30);
  tp.splits = static_cast<int>(splits);
  return tp;
}

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// ------------------------------------------------------------- chunking --
// zmc_scan_ex cuts a slice into chunks of consecutive grid points (the batches
// of Sec. 2), so that its device scratch stays bounded whatever the grid size:
// one chunk of FP64 partial sums (at most kChunkUnitSplits unit-splits,
// 256 MiB) and, with host buffers, two chunks of outputs whose device->host
// copies overlap the next chunk's sampling.  Every chunk runs the tile plan
// of the whole call, so the results do not depend on the chunking.
constexpr int64_t kChunkUnitSplits = int64_t(1) << 24;
constexpr int64_t kHostChunkMinPoints = int64_t(1) << 20;
constexpr int64_t kHostChunks = 8;

int64_t chunk_points_for(const zmc_scan_desc* d, int64_t count, const TilePlan& tp) {
  if (count <= 0) return 1;
  if (d->chunk_points > 0) return std::min<int64_t>(d->chunk_points, count);
  const int64_t per_point = std::max<int64_t>(1, int64_t(d->trials) * tp.splits);
  int64_t cp = std::max<int64_t>(1, kChunkUnitSplits / per_point);
  if (d->mem == ZMC_MEM_HOST)
    cp = std::min(cp, std::max(kHostChunkMinPoints, (count + kHostChunks - 1) / kHostChunks));
  return std::min(cp, count);
}

ScanLayout layout_for(const zmc_scan_desc* d, int64_t count, const TilePlan& tp) {
  ScanLayout L{};
  int64_t nvals = 0;
  for (int i = 0; i < d->M; ++i) nvals += d->list_len[i];
  const int64_t cp = chunk_points_for(d, count, tp);
  L.chunk_points = cp;
  L.chunks = count > 0 ? (count + cp - 1) / cp : 0;
  L.nbuf = L.chunks > 1 ? 2 : 1;
  L.partial = 0;
  L.partial_bytes = static_cast<size_t>(cp) * d->trials * tp.splits * 2 * sizeof(double);
  size_t off = align256(std::max<size_t>(L.partial_bytes, 16));
  L.vals = L.mean = L.err = L.errw = L.s1 = L.s2 = SIZE_MAX;
  if (d->mem == ZMC_MEM_HOST) {
    L.vals = off;
    off = align256(off + static_cast<size_t>(nvals) * sizeof(double));
    const size_t pb = static_cast<size_t>(L.nbuf) * cp * sizeof(double);
    const size_t tb = pb * d->trials;
    L.mean = off; off = align256(off + pb);
    L.err = off;  off = align256(off + pb);
    L.errw = off; off = align256(off + pb);
    L.s1 = off;   off = align256(off + tb);
    L.s2 = off;   off = align256(off + tb);
  }
  L.total = off;
  return L;
}

TilePlan plan_with(const zmc_scan_desc* d, int64_t count, int sm, int tps) {
  // A class entry recorded by the autotuner, when the caller leaves tiles open.
  int tl = 0, tb = 0, tg = 0;
  if (!d->tile_lanes && !d->tile_splits && !d->tile_block &&
      tune_find(d->precision, d->integrand_id, d->N, d->samples_per_point, &tl, &tb, &tg)) {
    TilePlan tp;
    const int G = group_samples(d->N);
    const int64_t Q = (d->samples_per_point + G - 1) / G;
    int64_t splits = std::max<int64_t>(1, (Q + int64_t(tl) * tg - 1) / (int64_t(tl) * tg));
    // small grids: enough ranges for ~4 waves of resident threads
    const int64_t units = std::max<int64_t>(1, count * d->trials);
    const int64_t want = int64_t(4) * std::max(1, sm) * std::max(256, tps);
    if (units * splits * tl < want) {
      const int64_t more = (want + units * tl - 1) / (units * tl);
      splits = std::max(splits, std::min(more, std::max<int64_t>(1, Q / (int64_t(tl) * 64))));
    }
    tp.lanes = tl;
    tp.block = tb;
    tp.splits = static_cast<int>(std::min<int64_t>(splits, std::max<int64_t>(1, Q)));
    return tp;
  }
  return plan_tiles(d->N, d->samples_per_point, d->trials, count, sm, tps, d->tile_lanes,
                    d->tile_splits, d->tile_block, d->precision);
}

int plan_for(const zmc_scan_desc* d, int64_t count, TilePlan* tp) {
  int sm = 0, tps = 2048;
  const bool explicit_tiles = d->tile_lanes && d->tile_splits && d->tile_block;
  if (!explicit_tiles) {
    DeviceState* ds = nullptr;
    int rc = device_state(&ds);
    if (rc != ZMC_OK) return rc;
    sm = ds->prop.multiProcessorCount;
    tps = ds->prop.maxThreadsPerMultiProcessor;
  }
  if (!d->tile_lanes && !d->tile_splits && !d->tile_block) tune_ensure_loaded();
  *tp = plan_with(d, count, sm, tps);
  return ZMC_OK;
}

static void fill_round_keys(uint64_t seed, uint32_t* rk0, uint32_t* rk1) {
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk0[r] = k0 + static_cast<uint32_t>(r) * kPhiloxW0;
    rk1[r] = k1 + static_cast<uint32_t>(r) * kPhiloxW1;
  }
}

double box_volume(const zmc_scan_desc* d) {
  double V = 1.0;
  for (int k = 0; k < d->N; ++k) V *= d->hi[k] - d->lo[k];
  return V;
}

void fill_scan_args(const zmc_scan_desc* d, int64_t count, const TilePlan& tp,
                    const double* vals_dev, double* partial_dev, ScanArgs* a) {
  std::memset(a, 0, sizeof(*a));
  const int G = group_samples(d->N);
  a->first = d->first_index;
  a->count = count;
  a->S = d->samples_per_point;
  a->ngroups = (a->S + G - 1) / G;
  a->splits = tp.splits;
  a->gps = (a->ngroups + tp.splits - 1) / tp.splits;
  a->T = d->trials;
  a->M = d->M;
  a->n_us = count * d->trials * tp.splits;
  a->lanes = tp.lanes;
  int l2 = 0;
  while ((1 << l2) < tp.lanes) ++l2;
  a->lanes_log2 = l2;
  int64_t nv = 0;
  for (int i = 0; i < d->M; ++i) {
    a->len[i] = d->list_len[i];
    a->off[i] = static_cast<int32_t>(nv);
    nv += d->list_len[i];
  }
  a->nvals = static_cast<int32_t>(nv);
  a->stage_smem = nv <= kMaxSmemVals ? 1 : 0;
  a->idx32 = (d->first_index + count <= (int64_t(1) << 32)) ? 1 : 0;
  a->vals = vals_dev;
  for (int k = 0; k < d->N; ++k) {
    a->lo[k] = d->lo[k];
    a->hi[k] = d->hi[k];
  }
  fill_round_keys(d->seed, a->rk0, a->rk1);
  a->partial = partial_dev;
  a->dbg = debug_words();
  a->gid = d->integrand_id;
  a->N = d->N;
}

int launch_scan_args(const zmc_scan_desc* d, const ScanArgs& a, const TilePlan& tp,
                     cudaStream_t stream) {
  if (a.n_us == 0) return ZMC_OK;
  if (is_user_integrand(d->integrand_id)) {
    const int64_t per_block = tp.block / tp.lanes;
    const int64_t grid = (a.n_us + per_block - 1) / per_block;
    if (grid > 0x7fffffffLL) return fail(ZMC_EINVAL, "launch grid too large (%lld)", (long long)grid);
    const size_t smem = a.stage_smem ? static_cast<size_t>(a.nvals) * sizeof(double) : 0;
    return user_launch(d, a, tp.block, grid, smem, stream);
  }
  ScanLaunchFn fn = scan_launcher(d->precision, d->integrand_id, d->N);
  if (!fn) return fail(ZMC_ENOTFOUND, "no kernel for integrand %d, N %d", d->integrand_id, d->N);
  const int64_t per_block = tp.block / tp.lanes;
  const int64_t grid = (a.n_us + per_block - 1) / per_block;
  if (grid > 0x7fffffffLL) return fail(ZMC_EINVAL, "launch grid too large (%lld)", (long long)grid);
  const size_t smem = a.stage_smem ? static_cast<size_t>(a.nvals) * sizeof(double) : 0;
  int e = fn(a, tp.block, grid, smem, stream);
  if (e != 0) return cuda_fail(static_cast<cudaError_t>(e), "sampling kernel launch");
  return ZMC_OK;
}

// -------------------------------------------------------------- the scan --
// CUDA events of one call (ZMC_F_TIMINGS only; otherwise every call is a no-op).
struct EventSet {
  std::vector<cudaEvent_t> ev;
  bool on = false;
  int create(size_t n) {
    ev.assign(n, nullptr);
    for (auto& e : ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return cuda_fail(r, "cudaEventCreate");
    }
    on = true;
    return ZMC_OK;
  }
  void record(size_t i, cudaStream_t s) {
    if (on) cudaEventRecord(ev[i], s);
  }
  float ms(size_t a, size_t b) {
    float v = 0.0f;
    if (on) cudaEventElapsedTime(&v, ev[a], ev[b]);
    return v;
  }
  ~EventSet() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Host memory that the GPU can copy into asynchronously (page-locked, from
// cudaMallocHost / cudaHostAlloc / cudaHostRegister), first and last byte.
static bool is_pinned_host(const void* p, size_t bytes) {
  if (!p || bytes == 0) return true;
  auto pinned = [](const void* q) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return at.type == cudaMemoryTypeHost;
  };
  return pinned(p) && pinned(static_cast<const char*>(p) + bytes - 1);
}

// Page-locked staging buffers for chunked scans into pageable host arrays,
// kept for reuse across calls (a process-wide free list; each call holds its
// buffer for its duration, so concurrent calls never share one).
struct PinnedBuf {
  char* p = nullptr;
  size_t bytes = 0;
};
static std::mutex g_pin_mu;
static std::vector<PinnedBuf> g_pin_free;

static int pinned_take(size_t bytes, PinnedBuf* out) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (size_t i = 0; i < g_pin_free.size(); ++i)
      if (g_pin_free[i].bytes >= bytes) {
        *out = g_pin_free[i];
        g_pin_free.erase(g_pin_free.begin() + static_cast<long>(i));
        return ZMC_OK;
      }
  }
  PinnedBuf b;
  cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&b.p), bytes, cudaHostAllocDefault);
  if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc(staging)");
  b.bytes = bytes;
  *out = b;
  return ZMC_OK;
}

static void pinned_give(PinnedBuf b) {
  if (!b.p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(b);
  if (g_pin_free.size() > 4) {  // keep the four largest
    auto it = std::min_element(g_pin_free.begin(), g_pin_free.end(),
                               [](const PinnedBuf& x, const PinnedBuf& y) {
                                 return x.bytes < y.bytes;
                               });
    cudaFreeHost(it->p);
    g_pin_free.erase(it);
  }
}

// One output array of a chunk: where the finalize kernel wrote it on the
// device, where it goes on the host, and its length in doubles.
struct OutCopy {
  double* dst;
  const double* src;
  size_t n;
};

int scan_ex(const zmc_scan_desc* d, zmc_scan_out* o) {
  TraceRange trace("zmc_scan_ex");
  int64_t P = 0, count = 0;
  int rc = validate(d, &P, &count);
  if (rc != ZMC_OK) return rc;
  if (!o) return fail(ZMC_EINVAL, "output struct is NULL");
  const bool plan_only = (d->flags & ZMC_F_PLAN_ONLY) != 0;
  if (count > 0 && !plan_only && (!o->mean || !o->err))
    return fail(ZMC_EINVAL, "mean/err output is NULL");

  DeviceState* ds = nullptr;
  rc = device_state(&ds);
  if (rc != ZMC_OK) return rc;
  cudaStream_t stream = static_cast<cudaStream_t>(d->stream);  // NULL: default stream

  if (d->mem == ZMC_MEM_DEVICE && !plan_only) {
    const void* ptrs[6] = {d->list_vals, o->mean, o->err, o->errw, o->s1, o->s2};
    for (int i = 0; i < 6; ++i)
      if (ptrs[i] && !is_device_ptr(ptrs[i]))
        return fail(ZMC_EINVAL, "ZMC_MEM_DEVICE given a pointer that is not device memory");
  }

  TilePlan tp;
  rc = plan_for(d, count, &tp);
  if (rc != ZMC_OK) return rc;
  const ScanLayout L = layout_for(d, count, tp);

  o->tile_lanes = tp.lanes;
  o->tile_splits = tp.splits;
  o->tile_block = tp.block;
  o->chunks = L.chunks;
  o->launches = 0;
  o->h2d_ms = o->kernel_ms = o->finalize_ms = o->d2h_ms = o->total_ms = 0.0f;
  log_msg(2, "scan: integrand %d N %d precision %d, points [%lld, +%lld) x %d trials x %lld "
          "samples; tiles lanes %d splits %d block %d; %lld chunk(s) of %lld points; %s memory",
          d->integrand_id, d->N, d->precision, (long long)d->first_index, (long long)count,
          d->trials, (long long)d->samples_per_point, tp.lanes, tp.splits, tp.block,
          (long long)L.chunks, (long long)L.chunk_points, d->mem == ZMC_MEM_HOST ? "host" : "device");
  if (count == 0 || plan_only) return ZMC_OK;

  // Scratch: the caller's workspace or the stream-ordered pool.
  char* ws = static_cast<char*>(d->workspace);
  bool own_ws = false;
  if (ws) {
    if (d->workspace_bytes < L.total)
      return fail(ZMC_EINVAL, "workspace of %zu bytes is smaller than the %zu needed",
                  d->workspace_bytes, L.total);
  } else {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), L.total, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(workspace)");
    own_ws = true;
  }

  const bool host = d->mem == ZMC_MEM_HOST;
  const int64_t nch = L.chunks, cp = L.chunk_points, T = d->trials;
  // Several chunks with host buffers: results leave on the copy stream while
  // the next chunk samples, straight into the caller's arrays when they are
  // pinned, else through two pinned staging buffers.
  const bool piped = host && nch > 1;
  cudaStream_t cs = ds->copy_stream;
  bool direct = true;
  const size_t pb_all = static_cast<size_t>(count) * sizeof(double);
  if (piped)
    direct = is_pinned_host(o->mean, pb_all) && is_pinned_host(o->err, pb_all) &&
             is_pinned_host(o->errw, pb_all) && is_pinned_host(o->s1, pb_all * T) &&
             is_pinned_host(o->s2, pb_all * T);
  const size_t per_chunk_doubles =
      static_cast<size_t>(cp) * (2 + (o->errw ? 1 : 0) + (o->s1 ? T : 0) + (o->s2 ? T : 0));
  PinnedBuf stage;
  cudaEvent_t ready[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
  bool copies_enqueued = false;
  auto release = [&]() {
    if (copies_enqueued) cudaStreamSynchronize(cs);
    for (int b = 0; b < 2; ++b) {
      if (ready[b]) cudaEventDestroy(ready[b]);
      if (copied[b]) cudaEventDestroy(copied[b]);
    }
    pinned_give(stage);
    if (own_ws) cudaFreeAsync(ws, stream);
  };
  if (piped) {
    for (int b = 0; b < 2; ++b) {
      cudaError_t e = cudaEventCreateWithFlags(&ready[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
      if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "cudaEventCreate");
      }
    }
    if (!direct && (rc = pinned_take(2 * per_chunk_doubles * sizeof(double), &stage)) != ZMC_OK) {
      release();
      return rc;
    }
  }

  // Events: 0 start, 1 lists copied, then per chunk (sampling start, sampling
  // end, finalize end), then one after the last copy.
  EventSet ev;
  const bool timed = (d->flags & ZMC_F_TIMINGS) != 0;
  if (timed && (rc = ev.create(3 + 3 * static_cast<size_t>(nch))) != ZMC_OK) {
    release();
    return rc;
  }
  const size_t ev_last = 2 + 3 * static_cast<size_t>(nch);

  const double* vals_dev = d->list_vals;
  int64_t nvals = 0;
  for (int i = 0; i < d->M; ++i) nvals += d->list_len[i];
  ev.record(0, stream);
  if (host) {
    double* v = reinterpret_cast<double*>(ws + L.vals);
    cudaError_t e = cudaMemcpyAsync(v, d->list_vals, nvals * sizeof(double),
                                    cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(e, "cudaMemcpyAsync(lists)");
    }
    vals_dev = v;
  }
  ev.record(1, stream);

  // The outputs of chunk k (points [k cp, k cp + n) of the slice): on the
  // device (finalize's targets) and their host destinations.
  auto chunk_outputs = [&](int64_t k, int64_t n, int b, double* dev[5], OutCopy cps[5]) {
    const int64_t off = k * cp;
    if (!host) {
      dev[0] = o->mean + off;
      dev[1] = o->err + off;
      dev[2] = o->errw ? o->errw + off : nullptr;
      dev[3] = o->s1 ? o->s1 + off * T : nullptr;
      dev[4] = o->s2 ? o->s2 + off * T : nullptr;
      return;
    }
    const size_t bo = static_cast<size_t>(b) * cp;
    dev[0] = reinterpret_cast<double*>(ws + L.mean) + bo;
    dev[1] = reinterpret_cast<double*>(ws + L.err) + bo;
    dev[2] = o->errw ? reinterpret_cast<double*>(ws + L.errw) + bo : nullptr;
    dev[3] = o->s1 ? reinterpret_cast<double*>(ws + L.s1) + bo * T : nullptr;
    dev[4] = o->s2 ? reinterpret_cast<double*>(ws + L.s2) + bo * T : nullptr;
    double* hdst[5] = {o->mean + off, o->err + off, o->errw ? o->errw + off : nullptr,
                       o->s1 ? o->s1 + off * T : nullptr, o->s2 ? o->s2 + off * T : nullptr};
    const size_t len[5] = {size_t(n), size_t(n), size_t(n), size_t(n * T), size_t(n * T)};
    for (int i = 0; i < 5; ++i) cps[i] = {hdst[i], dev[i], hdst[i] ? len[i] : 0};
  };
  // Chunk k's outputs, copied by the GPU into staging buffer b, go to the
  // caller's pageable arrays.
  auto unstage = [&](int64_t k, int b) {
    const int64_t n = std::min(cp, count - k * cp);
    double* dev[5];
    OutCopy cps[5];
    chunk_outputs(k, n, b, dev, cps);
    const double* src = reinterpret_cast<const double*>(stage.p) + b * per_chunk_doubles;
    for (auto& c : cps) {
      if (!c.n) continue;
      std::memcpy(c.dst, src, c.n * sizeof(double));
      src += c.n;
    }
  };

  const double V = box_volume(d);
  for (int64_t k = 0; k < nch; ++k) {
    TraceRange chunk_trace("zmc_scan_ex chunk");
    const int64_t n = std::min(cp, count - k * cp);
    const int b = piped ? static_cast<int>(k & 1) : 0;
    log_msg(3, "chunk %lld/%lld: points [%lld, +%lld)%s", (long long)k, (long long)nch,
            (long long)(d->first_index + k * cp), (long long)n,
            piped ? (direct ? ", copied straight to pinned host arrays"
                            : ", copied through pinned staging") : "");
    zmc_scan_desc dc = *d;
    dc.first_index = d->first_index + k * cp;
    dc.count = n;
    ScanArgs a;
    fill_scan_args(&dc, n, tp, vals_dev, reinterpret_cast<double*>(ws + L.partial), &a);
    ev.record(2 + 3 * k, stream);
    rc = launch_scan_args(d, a, tp, stream);
    if (rc != ZMC_OK) {
      release();
      return rc;
    }
    ev.record(3 + 3 * k, stream);
    // output buffer b was last read by the copy of chunk k - 2
    if (piped && k >= 2) cudaStreamWaitEvent(stream, copied[b], 0);
    double* dev[5];
    OutCopy cps[5];
    chunk_outputs(k, n, b, dev, cps);
    FinalizeArgs f;
    f.count = n;
    f.S = d->samples_per_point;
    f.T = d->trials;
    f.splits = tp.splits;
    f.V = V;
    f.partial = a.partial;
    f.mean = dev[0];
    f.err = dev[1];
    f.errw = dev[2];
    f.s1 = dev[3];
    f.s2 = dev[4];
    int e2 = finalize_launch(f, stream);
    if (e2 != 0) {
      release();
      return cuda_fail(static_cast<cudaError_t>(e2), "finalize kernel launch");
    }
    o->launches += 2;
    ev.record(4 + 3 * k, stream);
    if (!host) continue;
    cudaStream_t cstream = piped ? cs : stream;
    if (piped) {
      cudaEventRecord(ready[b], stream);
      cudaStreamWaitEvent(cs, ready[b], 0);
    }
    double* sdst = piped && !direct
                       ? reinterpret_cast<double*>(stage.p) + b * per_chunk_doubles
                       : nullptr;
    for (auto& c : cps) {
      if (!c.n) continue;
      double* dst = sdst ? sdst : c.dst;
      cudaError_t e = cudaMemcpyAsync(dst, c.src, c.n * sizeof(double),
                                      cudaMemcpyDeviceToHost, cstream);
      if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "cudaMemcpyAsync(results)");
      }
      copies_enqueued = copies_enqueued || piped;
      if (sdst) sdst += c.n;
    }
    if (piped) {
      cudaEventRecord(copied[b], cs);
      // the previous chunk's staged results to the caller while this chunk runs
      if (!direct && k >= 1) {
        cudaError_t e = cudaEventSynchronize(copied[b ^ 1]);
        if (e != cudaSuccess) {
          release();
          return cuda_fail(e, "cudaEventSynchronize(chunk copy)");
        }
        unstage(k - 1, b ^ 1);
      }
    }
  }
  if (piped) {
    const int bl = static_cast<int>((nch - 1) & 1);
    if (!direct) {
      cudaError_t e = cudaEventSynchronize(copied[bl]);
      if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "cudaEventSynchronize(chunk copy)");
      }
      unstage(nch - 1, bl);
    }
    cudaStreamWaitEvent(stream, copied[bl], 0);  // the workspace outlives the copies
    copies_enqueued = false;  // ordered behind the stream: no wait on the copy stream
  }
  ev.record(ev_last, stream);
  release();

  if (host || timed || ZMC_DEBUG || (d->flags & ZMC_F_SYNC)) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  }
#if ZMC_DEBUG
  {
    unsigned code = 0;
    long long index = 0;
    const int64_t nfail = debug_take(&code, &index);
    if (nfail > 0)
      return fail(ZMC_ECUDA, "device-side check %u failed %lld times (first index %lld)",
                  code, static_cast<long long>(nfail), index);
  }
#endif
  if (timed) {
    o->h2d_ms = ev.ms(0, 1);
    for (int64_t k = 0; k < nch; ++k) {
      o->kernel_ms += ev.ms(2 + 3 * k, 3 + 3 * k);
      o->finalize_ms += ev.ms(3 + 3 * k, 4 + 3 * k);
    }
    o->d2h_ms = host ? ev.ms(4 + 3 * (nch - 1), ev_last) : 0.0f;
    o->total_ms = ev.ms(0, ev_last);
  }
  return ZMC_OK;
}

}  // namespace zmc

// ================================================================ C ABI ==
using namespace zmc;

extern "C" {

int zmc_version(void) { return ZMC_ABI_VERSION; }

const char* zmc_last_error(void) { return zmc::last_error(); }

int zmc_scan_desc_init(zmc_scan_desc* d) {
  if (!d) return fail(ZMC_EINVAL, "descriptor is NULL");
  std::memset(d, 0, sizeof(*d));
  d->samples_per_point = 1;
  d->trials = 1;
  d->precision = ZMC_FP32_KAHAN;
  d->mem = ZMC_MEM_HOST;
  d->count = -1;
  return ZMC_OK;
}

int zmc_integrand_info_get(int id, zmc_integrand_info* info) {
  static const char* names[ZMC_G_COUNT] = {"const", "cosprod", "gauss03",
                                           "poly", "osc01", "sinsum"};
  if (!info) return fail(ZMC_EINVAL, "info is NULL");
  if (is_user_integrand(id)) return user_info(id, info);
  if (id < 0 || id >= ZMC_G_COUNT) return fail(ZMC_ENOTFOUND, "unknown integrand id %d", id);
  std::memset(info, 0, sizeof(*info));
  info->id = id;
  std::snprintf(info->name, sizeof(info->name), "%s", names[id]);
  info->m_rule = (id == ZMC_G_CONST || id == ZMC_G_SINSUM) ? 0 : 1;
  return ZMC_OK;
}

int zmc_device_info_get(zmc_device_info* info) {
  if (!info) return fail(ZMC_EINVAL, "info is NULL");
  DeviceState* ds = nullptr;
  int rc = device_state(&ds);
  if (rc != ZMC_OK) return rc;
  int dev = 0;
  cudaGetDevice(&dev);
  std::memset(info, 0, sizeof(*info));
  info->device = dev;
  info->sm_count = ds->prop.multiProcessorCount;
  info->cc_major = ds->prop.major;
  info->cc_minor = ds->prop.minor;
  info->max_threads_per_sm = ds->prop.maxThreadsPerMultiProcessor;
  int clk = 0;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  info->clock_khz = clk;
  info->total_mem = ds->prop.totalGlobalMem;
  // the device name, cut to the field's 95 characters
  std::snprintf(info->name, sizeof(info->name), "%.95s", ds->prop.name);
  return ZMC_OK;
}

int zmc_validate(const zmc_scan_desc* d) {
  clear_error();
  return validate(d, nullptr, nullptr);
}

int zmc_workspace_size(const zmc_scan_desc* d, size_t* bytes) {
  clear_error();
  int64_t count = 0;
  int rc = validate(d, nullptr, &count);
  if (rc != ZMC_OK) return rc;
  if (!bytes) return fail(ZMC_EINVAL, "bytes is NULL");
  TilePlan tp;
  rc = plan_for(d, count, &tp);
  if (rc != ZMC_OK) return rc;
  *bytes = layout_for(d, count, tp).total;
  return ZMC_OK;
}

int zmc_scan_ex(const zmc_scan_desc* d, zmc_scan_out* o) {
  clear_error();
  return scan_ex(d, o);
}

int zmc_scan(int integrand_id, int N, const double* lo, const double* hi, int M,
             const int64_t* list_len, const double* list_vals, int64_t samples_per_point,
             int trials, uint64_t seed, double* out_mean, double* out_err) {
  clear_error();
  zmc_scan_desc d;
  zmc_scan_desc_init(&d);
  d.integrand_id = integrand_id;
  d.N = N;
  d.lo = lo;
  d.hi = hi;
  d.M = M;
  d.list_len = list_len;
  d.list_vals = list_vals;
  d.samples_per_point = samples_per_point;
  d.trials = trials;
  d.seed = seed;
  zmc_scan_out o;
  std::memset(&o, 0, sizeof(o));
  o.mean = out_mean;
  o.err = out_err;
  return scan_ex(&d, &o);
}

int64_t zmc_debug_failures(unsigned* code, long long* index) {
  unsigned c = 0;
  long long i = 0;
  const int64_t n = debug_take(&c, &i);
  if (code) *code = c;
  if (index) *index = i;
  return n;
}

int zmc_stream_words(uint64_t seed, int64_t p, int t, uint64_t first_word, int64_t nwords,
                     uint32_t* out) {
  clear_error();
  if (p < 0 || t < 0 || nwords < 0) return fail(ZMC_EINVAL, "negative p, t or nwords");
  if (nwords > 0 && !out) return fail(ZMC_EINVAL, "out is NULL");
  if (nwords > (int64_t(1) << 30)) return fail(ZMC_EINVAL, "nwords above 2^30");
  if (first_word + static_cast<uint64_t>(nwords) > (uint64_t(1) << 34))
    return fail(ZMC_EINVAL, "word index beyond 2^34");
  if (nwords == 0) return ZMC_OK;
  DeviceState* ds = nullptr;
  int rc = device_state(&ds);
  if (rc != ZMC_OK) return rc;
  uint32_t* dev = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dev), nwords * sizeof(uint32_t),
                                  ds->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(words)");
  int le = stream_words_launch(seed, p, t, first_word, nwords, dev, ds->stream);
  if (le != 0) {
    cudaFreeAsync(dev, ds->stream);
    return cuda_fail(static_cast<cudaError_t>(le), "stream words kernel launch");
  }
  e = cudaMemcpyAsync(out, dev, nwords * sizeof(uint32_t), cudaMemcpyDeviceToHost, ds->stream);
  cudaFreeAsync(dev, ds->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(words)");
  e = cudaStreamSynchronize(ds->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return ZMC_OK;
}

}  // extern "C"
