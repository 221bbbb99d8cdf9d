// zmc_batch.cu — host side of include/zmc_batch.h: batch planning, the tile
// list, scratch, persistent launches, the batched finalize and CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/zmc_batch.h"
#include "zmc_internal.h"
#include "zmc_runtime.h"
#include "zmc_trace.h"

namespace zmc {

int batch_launch_p0(const BatchArgs&, int, int, size_t, void*);
int batch_launch_p1(const BatchArgs&, int, int, size_t, void*);
int batch_launch_p2(const BatchArgs&, int, int, size_t, void*);
int batch_occupancy_p0(int, size_t, int*);
int batch_occupancy_p1(int, size_t, int*);
int batch_occupancy_p2(int, size_t, int*);

int batch_launch(int precision, const BatchArgs& b, int grid, int block, size_t smem,
                 void* stream) {
  switch (precision) {
    case 0: return batch_launch_p0(b, grid, block, smem, stream);
    case 1: return batch_launch_p1(b, grid, block, smem, stream);
    case 2: return batch_launch_p2(b, grid, block, smem, stream);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int batch_blocks_per_sm(int precision, int block, size_t smem, int* out) {
  switch (precision) {
    case 0: return batch_occupancy_p0(block, smem, out);
    case 1: return batch_occupancy_p1(block, smem, out);
    case 2: return batch_occupancy_p2(block, smem, out);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

constexpr int kBatchBlock = 256;
// Sample groups per lane that bound one tile's work (tiles stay short next to
// the whole batch, so the longest-first order balances the SMs).
constexpr int64_t kBatchGroupsPerLane = 1024;
// Lanes per unit-split: the largest power of two <= 32 leaving each lane at
// least this many sample groups (plain FP32 lane sums: 64).  Long lanes spend
// less of their time in the FP64 epilogue on GB300's narrow FP64 unit:
// measured, 512 against 64 makes the 2048 small scans of the serving mix 6 %
// faster in one launch and leaves the uneven 256-scan batch unchanged.
#ifndef ZMC_BATCH_LANE_GROUPS
#define ZMC_BATCH_LANE_GROUPS 512
#endif

TilePlan plan_batch_scan(const zmc_scan_desc* d) {
  TilePlan tp;
  const int G = group_samples(d->N);
  const int64_t Q = (d->samples_per_point + G - 1) / G;
  tp.block = kBatchBlock;
  int tl = 0, tb = 0, tg = 0;
  if (!d->tile_lanes && !d->tile_splits &&
      tune_find(d->precision, d->integrand_id, d->N, d->samples_per_point, &tl, &tb, &tg)) {
    // the autotuner's lanes and per-lane work; batches keep 256-thread blocks
    tp.lanes = std::min(tl, kBatchBlock);
    const int64_t per = int64_t(tp.lanes) * tg;
    tp.splits = static_cast<int>(std::min<int64_t>(std::max<int64_t>(1, (Q + per - 1) / per), Q));
    return tp;
  }
  int lanes = d->tile_lanes;
  if (!lanes) {
    const int64_t min_groups = d->precision == ZMC_FP32 ? 64 : ZMC_BATCH_LANE_GROUPS;
    lanes = 32;
    while (lanes > 1 && Q / lanes < min_groups) lanes >>= 1;
  }
  tp.lanes = std::min(lanes, kBatchBlock);
  int64_t splits = d->tile_splits;
  if (!splits) {
    const int64_t per = int64_t(tp.lanes) * kBatchGroupsPerLane;
    splits = std::max<int64_t>(1, (Q + per - 1) / per);
  }
  tp.splits = static_cast<int>(std::min<int64_t>(std::max<int64_t>(splits, 1), Q));
  return tp;
}

struct PrecGroup {
  int precision = -1;
  int64_t tile_begin = 0, tile_end = 0;
  size_t smem = 0;
  int grid = 0;
  unsigned long long* counter = nullptr;
};

}  // namespace zmc

struct zmc_batch {
  int n = 0;
  std::vector<zmc::ScanArgs> args;
  std::vector<zmc::FinalizeArgs> fargs;
  std::vector<int64_t> prefix;
  std::vector<zmc::PrecGroup> groups;
  char* dev = nullptr;
  size_t bytes = 0;
  zmc::ScanArgs* d_args = nullptr;
  zmc::BatchTile* d_tiles = nullptr;
  zmc::FinalizeArgs* d_fargs = nullptr;
  int64_t* d_prefix = nullptr;
  int64_t ntiles = 0;
  int64_t evals = 0;
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
};

namespace zmc {

static size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

// Enqueue one run.  `mid` (optional) is recorded between the sampling
// launches and the finalize.
static int enqueue_run(zmc_batch* b, cudaStream_t s, cudaEvent_t mid) {
  for (const PrecGroup& g : b->groups) {
    cudaError_t e = cudaMemsetAsync(g.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(tile counter)");
    BatchArgs ba;
    ba.scans = b->d_args;
    ba.tiles = b->d_tiles + g.tile_begin;
    ba.ntiles = g.tile_end - g.tile_begin;
    ba.counter = g.counter;
    ba.nscans = b->n;
    ba.dbg = debug_words();
    const int le = batch_launch(g.precision, ba, g.grid, kBatchBlock, g.smem, s);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "batched kernel launch");
  }
  if (mid) cudaEventRecord(mid, s);
  FinalizeBatchArgs fb;
  fb.fa = b->d_fargs;
  fb.prefix = b->d_prefix;
  fb.nscans = b->n;
  fb.total = b->prefix[b->n];
  const int fe = finalize_batch_launch(fb, s);
  if (fe != 0) return cuda_fail(static_cast<cudaError_t>(fe), "batched finalize launch");
  return ZMC_OK;
}

static void free_batch(zmc_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

static bool device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int batch_create(const zmc_scan_desc* d, zmc_scan_out* o, int n, int flags, zmc_batch** out) {
  if (!out) return fail(ZMC_EINVAL, "out is NULL");
  tune_ensure_loaded();
  if (n < 1 || !d || !o) return fail(ZMC_EINVAL, "a batch needs n >= 1 scans and outputs");
  std::vector<int64_t> counts(n);
  std::vector<TilePlan> plans(n);
  for (int i = 0; i < n; ++i) {
    int64_t P = 0;
    int rc = validate(&d[i], &P, &counts[i]);
    if (rc != ZMC_OK) return fail(rc, "scan %d: %s", i, last_error());
    if (d[i].mem != ZMC_MEM_DEVICE)
      return fail(ZMC_EINVAL, "scan %d: a batch object needs ZMC_MEM_DEVICE", i);
    if (is_user_integrand(d[i].integrand_id))
      return fail(ZMC_EINVAL, "scan %d: batches take the compiled-in integrands only", i);
    if (d[i].tile_block != 0 && d[i].tile_block != kBatchBlock)
      return fail(ZMC_EINVAL, "scan %d: batches run %d-thread blocks", i, kBatchBlock);
    if (counts[i] > 0 && (!o[i].mean || !o[i].err))
      return fail(ZMC_EINVAL, "scan %d: mean/err output is NULL", i);
    const void* ptrs[6] = {d[i].list_vals, o[i].mean, o[i].err, o[i].errw, o[i].s1, o[i].s2};
    for (int k = 0; k < 6; ++k)
      if (ptrs[k] && !device_ptr(ptrs[k]))
        return fail(ZMC_EINVAL, "scan %d: a pointer is not device memory", i);
    plans[i] = plan_batch_scan(&d[i]);
  }

  zmc_batch* b = new (std::nothrow) zmc_batch();
  if (!b) return fail(ZMC_ENOMEM, "host allocation failed");
  b->n = n;
  b->args.resize(n);
  b->fargs.resize(n);
  b->prefix.assign(n + 1, 0);

  // Per-scan unit-splits, tiles and partial-sum offsets.
  std::vector<int64_t> n_us(n), ntiles(n), per_block(n);
  std::vector<size_t> part_off(n);
  size_t part_bytes = 0;
  for (int i = 0; i < n; ++i) {
    n_us[i] = counts[i] * d[i].trials * plans[i].splits;
    per_block[i] = kBatchBlock / plans[i].lanes;
    ntiles[i] = (n_us[i] + per_block[i] - 1) / per_block[i];
    part_off[i] = part_bytes;
    part_bytes += a256(static_cast<size_t>(n_us[i]) * 16);
    b->ntiles += ntiles[i];
    b->evals += counts[i] * d[i].trials * d[i].samples_per_point;
    b->prefix[i + 1] = b->prefix[i] + counts[i];
    o[i].tile_lanes = plans[i].lanes;
    o[i].tile_splits = plans[i].splits;
    o[i].tile_block = kBatchBlock;
    o[i].launches = 0;
  }

  // Device layout: args | tiles | finalize args | prefix | counters | partials.
  const size_t off_args = 0;
  const size_t off_tiles = a256(off_args + sizeof(ScanArgs) * n);
  const size_t off_fargs = a256(off_tiles + sizeof(BatchTile) * b->ntiles);
  const size_t off_prefix = a256(off_fargs + sizeof(FinalizeArgs) * n);
  const size_t off_cnt = a256(off_prefix + sizeof(int64_t) * (n + 1));
  const size_t off_part = a256(off_cnt + 3 * 256);
  b->bytes = off_part + std::max<size_t>(part_bytes, 256);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->dev), b->bytes);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "cudaMalloc(batch scratch)");
  }
  b->d_args = reinterpret_cast<ScanArgs*>(b->dev + off_args);
  b->d_tiles = reinterpret_cast<BatchTile*>(b->dev + off_tiles);
  b->d_fargs = reinterpret_cast<FinalizeArgs*>(b->dev + off_fargs);
  b->d_prefix = reinterpret_cast<int64_t*>(b->dev + off_prefix);
  double* part = reinterpret_cast<double*>(b->dev + off_part);

  for (int i = 0; i < n; ++i) {
    double* pi = reinterpret_cast<double*>(reinterpret_cast<char*>(part) + part_off[i]);
    fill_scan_args(&d[i], counts[i], plans[i], d[i].list_vals, pi, &b->args[i]);
    FinalizeArgs& f = b->fargs[i];
    f.count = counts[i];
    f.S = d[i].samples_per_point;
    f.T = d[i].trials;
    f.splits = plans[i].splits;
    f.V = box_volume(&d[i]);
    f.partial = pi;
    f.mean = o[i].mean;
    f.err = o[i].err;
    f.errw = o[i].errw;
    f.s1 = o[i].s1;
    f.s2 = o[i].s2;
    f.dbg = b->args[i].dbg;
  }

  // Tiles: grouped by precision; within a group the scans with the longest
  // tiles come first, each scan's tiles in order.
  std::vector<BatchTile> tiles;
  tiles.reserve(static_cast<size_t>(b->ntiles));
  int dev = 0, sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  for (int prec = 0; prec < 3; ++prec) {
    std::vector<int> order;
    for (int i = 0; i < n; ++i)
      if (d[i].precision == prec && ntiles[i] > 0) order.push_back(i);
    if (order.empty()) continue;
    // Longest tiles first: work per tile ~ unit-splits x samples per split x N.
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      const int Gx = group_samples(d[x].N), Gy = group_samples(d[y].N);
      const double cx = static_cast<double>(per_block[x]) * Gx *
                        (((d[x].samples_per_point + Gx - 1) / Gx + plans[x].splits - 1) /
                         plans[x].splits) * d[x].N;
      const double cy = static_cast<double>(per_block[y]) * Gy *
                        (((d[y].samples_per_point + Gy - 1) / Gy + plans[y].splits - 1) /
                         plans[y].splits) * d[y].N;
      return cx > cy;
    });
    PrecGroup g;
    g.precision = prec;
    g.tile_begin = static_cast<int64_t>(tiles.size());
    for (int i : order) {
      for (int64_t k = 0; k < ntiles[i]; ++k) {
        BatchTile t;
        t.scan = i;
        t.first_us = k * per_block[i];
        t.units = static_cast<int32_t>(std::min<int64_t>(per_block[i], n_us[i] - t.first_us));
        tiles.push_back(t);
      }
      if (b->args[i].stage_smem)
        g.smem = std::max(g.smem, static_cast<size_t>(b->args[i].nvals) * sizeof(double));
    }
    g.tile_end = static_cast<int64_t>(tiles.size());
    g.counter = reinterpret_cast<unsigned long long*>(b->dev + off_cnt + 256 * prec);
    int per_sm = 0;
    const int oe = batch_blocks_per_sm(prec, kBatchBlock, g.smem, &per_sm);
    if (oe != 0 || per_sm < 1) {
      free_batch(b);
      return cuda_fail(static_cast<cudaError_t>(oe ? oe : cudaErrorInvalidConfiguration),
                       "batched kernel occupancy");
    }
    const int64_t want = static_cast<int64_t>(per_sm) * std::max(sm, 1);
    g.grid = static_cast<int>(std::max<int64_t>(1, std::min(want, g.tile_end - g.tile_begin)));
    b->groups.push_back(g);
  }

  std::vector<int64_t> prefix = b->prefix;
  struct Up { void* dst; const void* src; size_t n; } ups[4] = {
      {b->d_args, b->args.data(), sizeof(ScanArgs) * n},
      {b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size()},
      {b->d_fargs, b->fargs.data(), sizeof(FinalizeArgs) * n},
      {b->d_prefix, prefix.data(), sizeof(int64_t) * (n + 1)}};
  for (auto& u : ups) {
    if (!u.n) continue;
    e = cudaMemcpy(u.dst, u.src, u.n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e, "cudaMemcpy(batch tables)");
    }
  }
  b->launches = static_cast<int>(b->groups.size()) + 1;

  if (flags & ZMC_BATCH_GRAPH) {
    e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e, "graph capture");
    }
    int rc = enqueue_run(b, b->capture, nullptr);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->capture, &g);
    if (rc != ZMC_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      free_batch(b);
      return rc != ZMC_OK ? rc : cuda_fail(e, "cudaStreamEndCapture");
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  *out = b;
  return ZMC_OK;
}

int batch_run(zmc_batch* b, cudaStream_t s, cudaEvent_t mid) {
  if (!b) return fail(ZMC_EINVAL, "batch is NULL");
  if (b->exec && !mid) {
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return ZMC_OK;
  }
  return enqueue_run(b, s, mid);
}

}  // namespace zmc

using namespace zmc;

extern "C" {

int zmc_batch_create(const zmc_scan_desc* d, zmc_scan_out* o, int n, int flags,
                     zmc_batch** out) {
  clear_error();
  TraceRange trace("zmc_batch_create");
  const int rc = batch_create(d, o, n, flags, out);
  if (rc == ZMC_OK)
    log_msg(2, "batch: %d scans, %lld tiles, %lld evaluations, %d launches per run%s", n,
            (long long)(*out)->ntiles, (long long)(*out)->evals, (*out)->launches,
            (*out)->exec ? ", CUDA graph" : "");
  return rc;
}

int zmc_batch_run(zmc_batch* b, void* stream) {
  clear_error();
  TraceRange trace("zmc_batch_run");
  return batch_run(b, static_cast<cudaStream_t>(stream), nullptr);
}

int zmc_batch_info_get(const zmc_batch* b, zmc_batch_info* info) {
  clear_error();
  if (!b || !info) return fail(ZMC_EINVAL, "batch or info is NULL");
  std::memset(info, 0, sizeof(*info));
  info->scans = b->n;
  info->precisions = static_cast<int>(b->groups.size());
  info->tiles = b->ntiles;
  info->evaluations = b->evals;
  info->grid = b->groups.empty() ? 0 : b->groups[0].grid;
  info->block = kBatchBlock;
  info->scratch_bytes = b->bytes;
  info->graph = b->exec ? 1 : 0;
  info->launches_per_run = b->launches;
  return ZMC_OK;
}

int zmc_batch_destroy(zmc_batch* b) {
  clear_error();
  if (!b) return ZMC_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_batch(b);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  return ZMC_OK;
}

int zmc_scan_batch(const zmc_scan_desc* d, int n, zmc_scan_out* o) {
  clear_error();
  if (n < 1 || !d || !o) return fail(ZMC_EINVAL, "a batch needs n >= 1 scans and outputs");
  const int mem = d[0].mem;
  for (int i = 0; i < n; ++i)
    if (d[i].mem != mem) return fail(ZMC_EINVAL, "all scans of a batch share one memory kind");
  cudaStream_t s = static_cast<cudaStream_t>(d[0].stream);
  const bool timed = (d[0].flags & ZMC_F_TIMINGS) != 0;

  std::vector<zmc_scan_desc> dd(d, d + n);
  std::vector<zmc_scan_out> oo(o, o + n);
  std::vector<int64_t> counts(n, 0);
  char* stage = nullptr;
  std::vector<size_t> off_vals(n), off_out(n);
  if (mem == ZMC_MEM_HOST) {
    // Stage lists and outputs on the device in one stream-ordered block.
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
      int64_t P = 0;
      int rc = validate(&d[i], &P, &counts[i]);
      if (rc != ZMC_OK) return fail(rc, "scan %d: %s", i, last_error());
      int64_t nv = 0;
      for (int k = 0; k < d[i].M; ++k) nv += d[i].list_len[k];
      off_vals[i] = total;
      total = a256(total + nv * sizeof(double));
      off_out[i] = total;
      total = a256(total + counts[i] * sizeof(double) * (3 + 2 * d[i].trials));
    }
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&stage), std::max<size_t>(total, 256), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(batch staging)");
    for (int i = 0; i < n; ++i) {
      int64_t nv = 0;
      for (int k = 0; k < d[i].M; ++k) nv += d[i].list_len[k];
      double* v = reinterpret_cast<double*>(stage + off_vals[i]);
      e = cudaMemcpyAsync(v, d[i].list_vals, nv * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) {
        cudaFreeAsync(stage, s);
        return cuda_fail(e, "cudaMemcpyAsync(lists)");
      }
      dd[i].list_vals = v;
      dd[i].mem = ZMC_MEM_DEVICE;
      double* ob = reinterpret_cast<double*>(stage + off_out[i]);
      const int64_t c = counts[i], T = d[i].trials;
      oo[i].mean = ob;
      oo[i].err = ob + c;
      oo[i].errw = o[i].errw ? ob + 2 * c : nullptr;
      oo[i].s1 = o[i].s1 ? ob + 3 * c : nullptr;
      oo[i].s2 = o[i].s2 ? ob + 3 * c + c * T : nullptr;
    }
    // the lists must be on the device before the batch tables point at them
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFreeAsync(stage, s);
      return cuda_fail(e, "cudaStreamSynchronize");
    }
  }

  zmc_batch* b = nullptr;
  int rc = batch_create(dd.data(), oo.data(), n, 0, &b);
  if (rc != ZMC_OK) {
    if (stage) cudaFreeAsync(stage, s);
    return rc;
  }
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (timed)
    for (auto& x : ev) cudaEventCreate(&x);
  if (timed) cudaEventRecord(ev[0], s);
  rc = batch_run(b, s, timed ? ev[1] : nullptr);
  if (timed) cudaEventRecord(ev[2], s);
  if (rc == ZMC_OK && mem == ZMC_MEM_HOST) {
    for (int i = 0; i < n && rc == ZMC_OK; ++i) {
      const size_t pb = counts[i] * sizeof(double), tb = pb * d[i].trials;
      struct Cp { void* dst; const void* src; size_t n; } cps[5] = {
          {o[i].mean, oo[i].mean, pb}, {o[i].err, oo[i].err, pb}, {o[i].errw, oo[i].errw, pb},
          {o[i].s1, oo[i].s1, tb}, {o[i].s2, oo[i].s2, tb}};
      for (auto& c : cps) {
        if (!c.dst || !c.n) continue;
        cudaError_t e = cudaMemcpyAsync(c.dst, c.src, c.n, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
          rc = cuda_fail(e, "cudaMemcpyAsync(results)");
          break;
        }
      }
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (rc == ZMC_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  for (int i = 0; i < n; ++i) {
    o[i].tile_lanes = oo[i].tile_lanes;
    o[i].tile_splits = oo[i].tile_splits;
    o[i].tile_block = oo[i].tile_block;
    o[i].launches = 0;
  }
  o[0].launches = b->launches;
  if (timed && rc == ZMC_OK) {
    cudaEventElapsedTime(&o[0].kernel_ms, ev[0], ev[1]);
    cudaEventElapsedTime(&o[0].finalize_ms, ev[1], ev[2]);
    cudaEventElapsedTime(&o[0].total_ms, ev[0], ev[2]);
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  free_batch(b);
  if (stage) {
    cudaFreeAsync(stage, s);
    cudaStreamSynchronize(s);
  }
  return rc;
}

}  // extern "C"
