// zmc_tune.cu — the tile autotuner of include/zmc_tune.h and the table the
// planners consult.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/zmc_tune.h"
#include "zmc_internal.h"
#include "zmc_runtime.h"

namespace zmc {

struct TuneEntry {
  int lanes = 32, block = 256, gpl = 1024;
  double evals_per_s = 0, default_evals_per_s = 0;
};

static std::mutex g_tune_mu;
static std::map<uint64_t, TuneEntry> g_tune;
static bool g_tune_loaded = false;

static int sbucket(int64_t S) {
  int b = 0;
  while (b < 62 && (int64_t(1) << (b + 1)) <= S) ++b;
  return b;
}

static uint64_t tune_key(int prec, int gid, int N, int64_t S) {
  return static_cast<uint64_t>(prec) | (static_cast<uint64_t>(gid) << 4) |
         (static_cast<uint64_t>(N) << 8) | (static_cast<uint64_t>(sbucket(S)) << 16);
}

static const char* cache_path() { return std::getenv("ZMC_AUTOTUNE_CACHE"); }

// Read the cache file once (caller holds g_tune_mu).
static void load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* p = cache_path();
  if (!p) return;
  FILE* f = std::fopen(p, "r");
  if (!f) return;
  unsigned long long key;
  TuneEntry e;
  while (std::fscanf(f, "%llx %d %d %d %lf %lf", &key, &e.lanes, &e.block, &e.gpl,
                     &e.evals_per_s, &e.default_evals_per_s) == 6)
    g_tune[key] = e;
  std::fclose(f);
}

static void save_locked() {
  const char* p = cache_path();
  if (!p) return;
  FILE* f = std::fopen(p, "w");
  if (!f) return;
  for (const auto& kv : g_tune)
    std::fprintf(f, "%llx %d %d %d %.6e %.6e\n", static_cast<unsigned long long>(kv.first),
                 kv.second.lanes, kv.second.block, kv.second.gpl, kv.second.evals_per_s,
                 kv.second.default_evals_per_s);
  std::fclose(f);
}

void tune_ensure_loaded() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_locked();
}

// In-memory lookup only (no file access, no allocation).
bool tune_find(int prec, int gid, int N, int64_t S, int* lanes, int* block, int* gpl) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(prec, gid, N, S));
  if (it == g_tune.end()) return false;
  *lanes = it->second.lanes;
  *block = it->second.block;
  *gpl = it->second.gpl;
  return true;
}

static int tune(const zmc_scan_desc* d0, int budget_ms, zmc_tune_result* out) {
  int64_t P = 0, count = 0;
  int rc = validate(d0, &P, &count);
  if (rc != ZMC_OK) return rc;
  if (!out) return fail(ZMC_EINVAL, "out is NULL");
  if (budget_ms < 50) return fail(ZMC_EINVAL, "budget_ms below 50");
  if (count == 0) return fail(ZMC_EINVAL, "nothing to tune: the slice is empty");
  tune_ensure_loaded();
  const int64_t T = d0->trials, S = d0->samples_per_point;
  const double target = 4.0e9;  // evaluations per timed run
  const int64_t count_t = std::max<int64_t>(
      1, std::min<int64_t>(count, static_cast<int64_t>(target / (double(T) * S))));
  int64_t nvals = 0;
  for (int i = 0; i < d0->M; ++i) nvals += d0->list_len[i];

  cudaStream_t s = nullptr;
  double* buf = nullptr;
  const size_t bytes = (nvals + 2 * count_t) * sizeof(double);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), bytes, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(tune buffers)");
  e = cudaMemcpyAsync(buf, d0->list_vals, nvals * sizeof(double),
                      d0->mem == ZMC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                      s);
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s);
    return cuda_fail(e, "cudaMemcpyAsync(tune lists)");
  }
  zmc_scan_desc d = *d0;
  d.mem = ZMC_MEM_DEVICE;
  d.list_vals = buf;
  d.count = count_t;
  d.stream = s;
  d.workspace = nullptr;
  d.flags = ZMC_F_TIMINGS;
  zmc_scan_out o{};
  o.mean = buf + nvals;
  o.err = buf + nvals + count_t;

  const int G = group_samples(d.N);
  const int64_t Q = (S + G - 1) / G;
  double spent = 0;
  auto run = [&](int lanes, int splits, int block, double* evals_per_s) -> int {
    d.tile_lanes = lanes;
    d.tile_splits = splits;
    d.tile_block = block;
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      int r = scan_ex(&d, &o);
      if (r != ZMC_OK) return r;
      spent += o.total_ms;
      best = std::min(best, o.kernel_ms + o.finalize_ms);
    }
    *evals_per_s = double(count_t) * T * S / (best * 1e-3);
    return ZMC_OK;
  };

  // The fixed-rule plan first (its tiles become the fallback winner).
  zmc_tune_result res{};
  double dflt = 0;
  d.tile_lanes = d.tile_splits = d.tile_block = 0;
  rc = scan_ex(&d, &o);
  if (rc == ZMC_OK) rc = run(o.tile_lanes, o.tile_splits, o.tile_block, &dflt);
  if (rc != ZMC_OK) {
    cudaFreeAsync(buf, s);
    return rc;
  }
  TuneEntry best;
  best.lanes = o.tile_lanes;
  best.block = o.tile_block;
  best.gpl = static_cast<int>(std::max<int64_t>(
      1, (Q + int64_t(o.tile_lanes) * o.tile_splits - 1) / (int64_t(o.tile_lanes) * o.tile_splits)));
  best.evals_per_s = dflt;
  best.default_evals_per_s = dflt;
  int tried = 1;
  // Candidates: the long lanes the planner favours (each lane's FP64 epilogue
  // runs on the narrow FP64 unit) down to the wide ones of small grids.
  const int lanes_c[] = {1, 2, 4, 8, 16, 32, 64, 128};
  const int block_c[] = {256, 128, 512};
  const int gpl_c[] = {1024, 256, 4096, 8192};
  for (int gpl : gpl_c) {
    for (int block : block_c) {
      for (int lanes : lanes_c) {
        if (spent > budget_ms) break;
        if (lanes > block || Q / lanes < 16) continue;
        const int64_t splits64 = std::max<int64_t>(1, (Q + int64_t(lanes) * gpl - 1) / (int64_t(lanes) * gpl));
        const int splits = static_cast<int>(std::min<int64_t>(splits64, Q));
        double v = 0;
        rc = run(lanes, splits, block, &v);
        if (rc != ZMC_OK) {
          cudaFreeAsync(buf, s);
          return rc;
        }
        ++tried;
        if (v > best.evals_per_s * 1.01) {
          best.lanes = lanes;
          best.block = block;
          best.gpl = gpl;
          best.evals_per_s = v;
        }
      }
    }
  }
  cudaFreeAsync(buf, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(d0->precision, d0->integrand_id, d0->N, S)] = best;
    save_locked();
  }
  res.lanes = best.lanes;
  res.block = best.block;
  res.groups_per_lane = best.gpl;
  res.candidates = tried;
  res.evals_per_s = best.evals_per_s;
  res.default_evals_per_s = dflt;
  *out = res;
  return ZMC_OK;
}

}  // namespace zmc

using namespace zmc;

extern "C" {

int zmc_autotune(const zmc_scan_desc* d, int budget_ms, zmc_tune_result* out) {
  clear_error();
  return tune(d, budget_ms, out);
}

int zmc_autotune_lookup(int precision, int integrand_id, int N, int64_t samples,
                        zmc_tune_result* out) {
  clear_error();
  if (!out) return fail(ZMC_EINVAL, "out is NULL");
  tune_ensure_loaded();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(precision, integrand_id, N, samples));
  if (it == g_tune.end()) return fail(ZMC_ENOTFOUND, "no tuned entry for this class");
  std::memset(out, 0, sizeof(*out));
  out->lanes = it->second.lanes;
  out->block = it->second.block;
  out->groups_per_lane = it->second.gpl;
  out->evals_per_s = it->second.evals_per_s;
  out->default_evals_per_s = it->second.default_evals_per_s;
  return ZMC_OK;
}

int zmc_autotune_reset(void) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  g_tune_loaded = true;  // do not reload the file after an explicit reset
  return ZMC_OK;
}

}  // extern "C"
