// zmc_server.cu — the request loop of include/zmc_server.h.
//
// One scheduler thread owns the GPU.  A step:
//   1. admit queued requests while a slot is free and the memory budget
//      covers them (lists, one chunk of partial sums, output buffers);
//   2. pick tiles from the admitted requests (shortest remaining work first,
//      a quarter of the step reserved for the oldest request) up to the step's
//      evaluation budget;
//   3. upload the step's scan arguments and tiles, launch one persistent
//      sampling kernel per precision, then one batched finalize for every
//      chunk whose last tiles are in this step;
//   4. while the step runs, hand the previous step's finished chunks to the
//      copier thread, which copies them into the callers' host arrays on a
//      second stream (a copy into pageable memory holds the calling thread
//      until it is done, so it never runs on the scheduler thread);
//   5. wait for the step; a request is done when the copier has put its last
//      chunk in host memory.
// A chunk's output buffer on the device is finalized into again only after
// the copier has copied its previous contents out (the scheduler does not
// pick the tiles that would complete a chunk while its buffer is busy).
// No kernel waits on anything; every host wait is on a CUDA event of work
// already enqueued, or a condition variable with a deadline.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/zmc_server.h"
#include "zmc_internal.h"
#include "zmc_runtime.h"
#include "zmc_trace.h"

namespace zmc {

TilePlan plan_batch_scan(const zmc_scan_desc* d);
constexpr int kServeBlock = 256;

using Clock = std::chrono::steady_clock;

static size_t s256(size_t v) { return (v + 255) & ~size_t(255); }

struct Request {
  uint64_t id = 0;
  // owned copies of the inputs
  zmc_scan_desc d{};
  std::vector<double> lo, hi, vals;
  std::vector<int64_t> len;
  zmc_scan_out* user_out = nullptr;
  zmc_scan_out o{};  // the caller's output pointers
  int64_t count = 0;
  TilePlan tp;
  int64_t chunk_points = 0, nchunks = 0;
  size_t bytes = 0;
  double evals_total = 0, evals_left = 0;
  int64_t seq = 0;  // admission order
  Clock::time_point t_submit, t_done;
  // device state
  char* dev = nullptr;
  double* d_vals = nullptr;
  double* d_part = nullptr;
  double* d_out[2] = {nullptr, nullptr};
  size_t out_doubles = 0;  // per buffer
  // copier thread state: d_out[b] is being copied out; chunks in the
  // caller's host arrays; copy jobs queued or running; a failed copy
  std::atomic<bool> buf_busy[2];
  std::atomic<int64_t> delivered{0};
  std::atomic<int> jobs{0};
  std::atomic<int> copy_status{ZMC_OK};
  // progress of the current chunk
  int64_t chunk = 0, chunk_first = 0, chunk_count = 0;
  int64_t chunk_units = 0, chunk_tiles = 0, next_tile = 0;
  ScanArgs args{};
  Request() {
    buf_busy[0].store(false);
    buf_busy[1].store(false);
  }
  // shared with API threads (under the server mutex)
  int status = ZMC_OK;
  bool done = false;
  std::atomic<bool> cancel{false};
};

struct ChunkDone {
  std::shared_ptr<Request> r;
  int64_t chunk, first, count;
  int buf;
};

}  // namespace zmc

struct zmc_server {
  zmc_server_opts opts{};
  size_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<zmc::Request>> queue;
  std::map<uint64_t, std::shared_ptr<zmc::Request>> all;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread thread;
  uint64_t wake = 0;  // bumped by the copier when a copy job ends (under mu)
  // copier thread: device->host copies of finished chunks, in order
  std::thread copier;
  std::mutex cmu;
  std::condition_variable ccv;
  std::deque<zmc::ChunkDone> cjobs;
  bool cstop = false;
  // scheduler-owned
  std::vector<std::shared_ptr<zmc::Request>> active;
  int64_t seq = 0;
  cudaStream_t compute = nullptr, copy = nullptr;
  // Two steps may be in flight: each has its own pinned staging buffer and
  // events; the device copy of the step tables is shared, because a step's
  // upload is ordered after the previous step's kernels on the same stream.
  cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_end[2] = {nullptr, nullptr};
  char* h_stage[2] = {nullptr, nullptr};  // pinned upload staging
  char* d_stage = nullptr;                // device copy of the step tables
  size_t stage_bytes = 0;
  int64_t tile_cap = 0;
  unsigned long long* d_counters = nullptr;
  double rate = 3e8;  // evaluations per ms, running estimate
  int64_t alloc_count = 0;
  // stats (under mu)
  int64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, max_queued = 0;
  int64_t steps = 0;
  double evals_done = 0, busy_ms = 0;
  size_t mem_in_use = 0, mem_peak = 0;
  std::vector<double> latencies;
};

namespace zmc {

// ----------------------------------------------------------- lifecycle --
static void finish_request(zmc_server* s, const std::shared_ptr<Request>& r, int status) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->done) return;
  r->status = status;
  r->done = true;
  r->t_done = Clock::now();
  if (status == ZMC_OK) {
    const double ms =
        std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    s->latencies.push_back(ms);
    s->completed++;
    s->evals_done += r->evals_total;
    r->user_out->total_ms = static_cast<float>(ms);
    r->user_out->tile_lanes = r->tp.lanes;
    r->user_out->tile_splits = r->tp.splits;
    r->user_out->tile_block = r->tp.block;
  } else if (status == ZMC_ECANCELED) {
    s->cancelled++;
  } else {
    s->failed++;
  }
  // The input copies are not needed any more; a finished ticket keeps only
  // its status (so a long-running server does not accumulate the lists).
  std::vector<double>().swap(r->vals);
  std::vector<double>().swap(r->lo);
  std::vector<double>().swap(r->hi);
  std::vector<int64_t>().swap(r->len);
  s->cv_done.notify_all();
}

static void release_device(zmc_server* s, Request* r) {
  if (r->dev) {
    cudaFreeAsync(r->dev, s->compute);
    r->dev = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    s->mem_in_use -= r->bytes;
  }
}

// Set up chunk `c` of r: its points, unit-splits, tiles and scan arguments.
static void start_chunk(Request* r, int64_t c) {
  r->chunk = c;
  r->chunk_first = r->d.first_index + c * r->chunk_points;
  r->chunk_count = std::min(r->chunk_points, r->d.first_index + r->count - r->chunk_first);
  r->chunk_units = r->chunk_count * r->d.trials * r->tp.splits;
  const int64_t per_block = kServeBlock / r->tp.lanes;
  r->chunk_tiles = (r->chunk_units + per_block - 1) / per_block;
  r->next_tile = 0;
  zmc_scan_desc dc = r->d;
  dc.first_index = r->chunk_first;
  dc.count = r->chunk_count;
  fill_scan_args(&dc, r->chunk_count, r->tp, r->d_vals, r->d_part, &r->args);
}

// Admission: device memory for lists, one chunk of partials, output buffers.
static int admit_one(zmc_server* s, const std::shared_ptr<Request>& r) {
  const bool inject = s->opts.fail_alloc_every > 0 &&
                      (++s->alloc_count % s->opts.fail_alloc_every) == 0;
  cudaError_t e = inject ? cudaErrorMemoryAllocation
                         : cudaMallocAsync(reinterpret_cast<void**>(&r->dev), r->bytes, s->compute);
  if (e != cudaSuccess) {
    cudaGetLastError();
    r->dev = nullptr;
    return e == cudaErrorMemoryAllocation ? ZMC_ENOMEM : ZMC_ECUDA;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->mem_in_use += r->bytes;
    s->mem_peak = std::max(s->mem_peak, s->mem_in_use);
  }
  size_t off = 0;
  r->d_vals = reinterpret_cast<double*>(r->dev + off);
  off = s256(off + r->vals.size() * sizeof(double));
  r->d_part = reinterpret_cast<double*>(r->dev + off);
  off = s256(off + static_cast<size_t>(r->chunk_points) * r->d.trials * r->tp.splits * 16);
  const int nbuf = r->nchunks > 1 ? 2 : 1;
  for (int b = 0; b < nbuf; ++b) {
    r->d_out[b] = reinterpret_cast<double*>(r->dev + off);
    off = s256(off + r->out_doubles * sizeof(double));
  }
  e = cudaMemcpyAsync(r->d_vals, r->vals.data(), r->vals.size() * sizeof(double),
                      cudaMemcpyHostToDevice, s->compute);
  if (e != cudaSuccess) return ZMC_ECUDA;
  r->seq = s->seq++;
  start_chunk(r.get(), 0);
  return ZMC_OK;
}

// Copy a finished chunk (its finalize has completed) from its device output
// buffer into the caller's host arrays.  Runs on the copier thread: a copy
// into pageable memory returns only when it is done.
static int copy_chunk_now(zmc_server* s, const ChunkDone& c) {
  Request* r = c.r.get();
  const int64_t off = c.first - r->d.first_index;
  const int64_t n = c.count, T = r->d.trials;
  double* base = r->d_out[c.buf];
  struct Cp { double* dst; const double* src; size_t n; } cps[5] = {
      {r->o.mean ? r->o.mean + off : nullptr, base, static_cast<size_t>(n)},
      {r->o.err ? r->o.err + off : nullptr, base + n, static_cast<size_t>(n)},
      {r->o.errw ? r->o.errw + off : nullptr, base + 2 * n, static_cast<size_t>(n)},
      {r->o.s1 ? r->o.s1 + off * T : nullptr, base + 3 * n, static_cast<size_t>(n * T)},
      {r->o.s2 ? r->o.s2 + off * T : nullptr, base + 3 * n + n * T, static_cast<size_t>(n * T)}};
  for (auto& cp : cps) {
    if (!cp.dst || !cp.n) continue;
    cudaError_t e = cudaMemcpyAsync(cp.dst, cp.src, cp.n * sizeof(double),
                                    cudaMemcpyDeviceToHost, s->copy);
    if (e != cudaSuccess) return ZMC_ECUDA;
  }
  return cudaStreamSynchronize(s->copy) == cudaSuccess ? ZMC_OK : ZMC_ECUDA;
}

static void copier_loop(zmc_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    ChunkDone c;
    {
      std::unique_lock<std::mutex> lk(s->cmu);
      s->ccv.wait(lk, [&] { return s->cstop || !s->cjobs.empty(); });
      if (s->cjobs.empty()) return;
      c = s->cjobs.front();
      s->cjobs.pop_front();
    }
    Request* r = c.r.get();
    if (!r->cancel.load()) {
      if (copy_chunk_now(s, c) == ZMC_OK)
        r->delivered.fetch_add(1);
      else
        r->copy_status.store(ZMC_ECUDA);
    }
    r->buf_busy[c.buf].store(false);
    r->jobs.fetch_sub(1);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->wake++;
    }
    s->cv_work.notify_one();
  }
}

// Hand a finished chunk to the copier thread.
static void copy_chunk(zmc_server* s, const ChunkDone& c) {
  Request* r = c.r.get();
  r->buf_busy[c.buf].store(true);
  r->jobs.fetch_add(1);
  {
    std::lock_guard<std::mutex> lk(s->cmu);
    s->cjobs.push_back(c);
  }
  s->ccv.notify_one();
}

// Wait until the copier has no job of r queued or running (it skips the
// jobs of cancelled requests, and a running copy ends by itself).
static void drain_jobs(Request* r) {
  while (r->jobs.load() > 0) std::this_thread::sleep_for(std::chrono::microseconds(50));
}

struct StepPick {
  std::shared_ptr<Request> r;
  int64_t tile_begin, tile_end;
  bool completes_chunk;
};

// A launched step: its staging slot, work and the chunks it finalizes.
struct Step {
  int slot = 0;
  double evals = 0;
  std::vector<ChunkDone> completing;
};

// Wait for a launched step, account its GPU time and enqueue the host copies
// of the chunks it finalized (on the copy stream, overlapping later steps).
static void retire_step(zmc_server* s, Step& st) {
  cudaEventSynchronize(s->ev_end[st.slot]);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, s->ev_start[st.slot], s->ev_end[st.slot]);
  if (ms > 0.05f && st.evals > 0) s->rate = 0.7 * s->rate + 0.3 * (st.evals / ms);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->busy_ms += ms;
    s->steps++;
  }
  for (auto& c : st.completing) {
    Request* r = c.r.get();
    if (r->done || r->cancel.load()) continue;
    copy_chunk(s, c);
  }
}

// ------------------------------------------------------------ one step --
static void run_loop(zmc_server* s) {
  cudaSetDevice(s->device);
  // Steps are pipelined two deep: after launching step k the scheduler
  // retires step k-1 (waits for it, enqueues its copies) and then plans step
  // k+1 while step k runs, so the GPU does not idle during host work.
  std::deque<Step> inflight;
  int slot = 0;
  for (;;) {
    // 1. queue -> active, cancellations, stop.
    bool stopping;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      stopping = s->stop;
      if (!stopping && s->queue.empty() && s->active.empty() && inflight.empty())
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      stopping = s->stop;
    }
    const uint64_t wake_seen = [&] {
      std::lock_guard<std::mutex> lk(s->mu);
      return s->wake;
    }();
    // cancelled or stopping: queued requests end now
    {
      std::vector<std::shared_ptr<Request>> ended;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto it = s->queue.begin(); it != s->queue.end();) {
          if (stopping || (*it)->cancel.load()) {
            ended.push_back(*it);
            it = s->queue.erase(it);
          } else {
            ++it;
          }
        }
      }
      for (auto& r : ended) finish_request(s, r, ZMC_ECANCELED);
    }
    // admit in arrival order while slots and budget allow
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (stopping || s->queue.empty() ||
            static_cast<int>(s->active.size()) >= s->opts.max_active)
          break;
        if (s->mem_in_use + s->queue.front()->bytes > s->budget) break;
        r = s->queue.front();
        s->queue.pop_front();
      }
      const int rc = admit_one(s, r);
      if (rc != ZMC_OK) {
        release_device(s, r.get());
        finish_request(s, r, rc);
      } else {
        log_msg(2, "server: admitted request %llu (integrand %d N %d, %lld points in %lld "
                "chunk(s), %zu device bytes)", (unsigned long long)r->id, r->d.integrand_id,
                r->d.N, (long long)r->count, (long long)r->nchunks, r->bytes);
        s->active.push_back(r);
      }
    }
    if (stopping && s->active.empty()) {
      while (!inflight.empty()) {
        retire_step(s, inflight.front());
        inflight.pop_front();
      }
      return;
    }
    // 2. pick tiles (skip cancelled requests and those with every tile launched)
    std::vector<StepPick> picks;
    double budget = std::max(1.0, s->opts.step_ms * s->rate);
    int64_t tiles_used = 0;
    {
      std::vector<std::shared_ptr<Request>> ready;
      for (auto& r : s->active)
        if (!r->cancel.load() && !stopping && r->next_tile < r->chunk_tiles)
          ready.push_back(r);
      std::shared_ptr<Request> oldest;
      for (auto& r : ready)
        if (!oldest || r->seq < oldest->seq) oldest = r;
      std::stable_sort(ready.begin(), ready.end(), [](const std::shared_ptr<Request>& a,
                                                      const std::shared_ptr<Request>& b) {
        return a->evals_left < b->evals_left;
      });
      if (oldest) {  // the oldest first, with a quarter of the step
        ready.erase(std::find(ready.begin(), ready.end(), oldest));
        ready.insert(ready.begin(), oldest);
      }
      double left = budget;
      for (size_t i = 0; i < ready.size() && tiles_used < s->tile_cap; ++i) {
        Request* r = ready[i].get();
        const int G = group_samples(r->d.N);
        const int64_t per_block = kServeBlock / r->tp.lanes;
        const int64_t groups = (r->args.ngroups + r->tp.splits - 1) / r->tp.splits;
        const double tile_evals = static_cast<double>(per_block) * groups * G;
        const double allot = (i == 0 && ready.size() > 1) ? std::max(budget * 0.25, tile_evals)
                                                         : left;
        if (i > 0 && left < tile_evals) break;
        int64_t k = static_cast<int64_t>(allot / tile_evals);
        k = std::max<int64_t>(1, std::min(k, r->chunk_tiles - r->next_tile));
        k = std::min(k, s->tile_cap - tiles_used);
        // the chunk's output buffer still holds an earlier chunk being copied
        // out: run all but its last tile now, finalize it in a later step
        if (r->next_tile + k == r->chunk_tiles && r->buf_busy[r->chunk % 2].load()) --k;
        if (k <= 0) continue;
        StepPick p{ready[i], r->next_tile, r->next_tile + k, r->next_tile + k == r->chunk_tiles};
        r->next_tile += k;
        tiles_used += k;
        left -= k * tile_evals;
        r->evals_left -= k * tile_evals;
        picks.push_back(p);
        if (left <= 0) break;
      }
    }
    // 3. upload and launch the step
    if (!picks.empty()) {
      TraceRange step_trace("zmc_server step");
      Step st;
      st.slot = slot;
      const int nsc = static_cast<int>(picks.size());
      std::vector<FinalizeArgs> fa;
      std::vector<int64_t> prefix(1, 0);
      char* h = s->h_stage[slot];
      ScanArgs* h_args = reinterpret_cast<ScanArgs*>(h);
      const size_t off_tiles = s256(sizeof(ScanArgs) * s->opts.max_active);
      BatchTile* h_tiles = reinterpret_cast<BatchTile*>(h + off_tiles);
      const size_t off_fa = s256(off_tiles + sizeof(BatchTile) * s->tile_cap);
      FinalizeArgs* h_fa = reinterpret_cast<FinalizeArgs*>(h + off_fa);
      const size_t off_pre = s256(off_fa + sizeof(FinalizeArgs) * s->opts.max_active);
      int64_t* h_pre = reinterpret_cast<int64_t*>(h + off_pre);
      // tiles grouped by precision, in pick order
      int64_t nt = 0;
      int64_t gbeg[3] = {0, 0, 0}, gend[3] = {0, 0, 0};
      size_t gsmem[3] = {0, 0, 0};
      for (int prec = 0; prec < 3; ++prec) {
        gbeg[prec] = nt;
        for (int i = 0; i < nsc; ++i) {
          Request* r = picks[i].r.get();
          if (r->d.precision != prec) continue;
          const int64_t per_block = kServeBlock / r->tp.lanes;
          for (int64_t t = picks[i].tile_begin; t < picks[i].tile_end; ++t) {
            BatchTile bt;
            bt.scan = i;
            bt.first_us = t * per_block;
            bt.units = static_cast<int32_t>(std::min(per_block, r->chunk_units - bt.first_us));
            h_tiles[nt++] = bt;
          }
          if (r->args.stage_smem)
            gsmem[prec] = std::max(gsmem[prec], static_cast<size_t>(r->args.nvals) * 8);
        }
        gend[prec] = nt;
      }
      for (int i = 0; i < nsc; ++i) {
        Request* r = picks[i].r.get();
        h_args[i] = r->args;
        const int G = group_samples(r->d.N);
        const int64_t per_block = kServeBlock / r->tp.lanes;
        const int64_t groups = (r->args.ngroups + r->tp.splits - 1) / r->tp.splits;
        st.evals += static_cast<double>(picks[i].tile_end - picks[i].tile_begin) *
                    per_block * groups * G;
        if (picks[i].completes_chunk) {
          const int buf = static_cast<int>(r->chunk % 2);
          FinalizeArgs f;
          const int64_t n = r->chunk_count, T = r->d.trials;
          double* base = r->d_out[buf];
          f.count = n;
          f.S = r->d.samples_per_point;
          f.T = r->d.trials;
          f.splits = r->tp.splits;
          f.V = box_volume(&r->d);
          f.partial = r->d_part;
          f.mean = base;
          f.err = base + n;
          f.errw = r->o.errw ? base + 2 * n : nullptr;
          f.s1 = r->o.s1 ? base + 3 * n : nullptr;
          f.s2 = r->o.s2 ? base + 3 * n + n * T : nullptr;
          f.dbg = r->args.dbg;
          fa.push_back(f);
          prefix.push_back(prefix.back() + n);
          st.completing.push_back(ChunkDone{picks[i].r, r->chunk, r->chunk_first, n, buf});
        }
      }
      for (size_t k = 0; k < fa.size(); ++k) h_fa[k] = fa[k];
      for (size_t k = 0; k < prefix.size(); ++k) h_pre[k] = prefix[k];
      const size_t upload = off_pre + prefix.size() * sizeof(int64_t);
      cudaError_t e = cudaMemcpyAsync(s->d_stage, h, upload, cudaMemcpyHostToDevice, s->compute);
      int rc = e == cudaSuccess ? ZMC_OK : ZMC_ECUDA;
      cudaEventRecord(s->ev_start[slot], s->compute);
      for (int prec = 0; prec < 3 && rc == ZMC_OK; ++prec) {
        if (gend[prec] == gbeg[prec]) continue;
        unsigned long long* cnt = s->d_counters + 32 * prec;
        cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s->compute);
        BatchArgs ba;
        ba.scans = reinterpret_cast<const ScanArgs*>(s->d_stage);
        ba.tiles = reinterpret_cast<const BatchTile*>(s->d_stage + off_tiles) + gbeg[prec];
        ba.ntiles = gend[prec] - gbeg[prec];
        ba.counter = cnt;
        ba.nscans = nsc;
        ba.dbg = debug_words();
        int per_sm = 1, sm = 1;
        batch_blocks_per_sm(prec, kServeBlock, gsmem[prec], &per_sm);
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, s->device);
        const int64_t grid = std::max<int64_t>(
            1, std::min<int64_t>(static_cast<int64_t>(per_sm) * sm, ba.ntiles));
        if (batch_launch(prec, ba, static_cast<int>(grid), kServeBlock, gsmem[prec],
                         s->compute) != 0)
          rc = ZMC_ECUDA;
      }
      if (rc == ZMC_OK && !fa.empty()) {
        FinalizeBatchArgs fb;
        fb.fa = reinterpret_cast<const FinalizeArgs*>(s->d_stage + off_fa);
        fb.prefix = reinterpret_cast<const int64_t*>(s->d_stage + off_pre);
        fb.nscans = static_cast<int32_t>(fa.size());
        fb.total = prefix.back();
        if (finalize_batch_launch(fb, s->compute) != 0) rc = ZMC_ECUDA;
      }
      cudaEventRecord(s->ev_end[slot], s->compute);
      if (rc != ZMC_OK) {
        for (auto& p : picks) p.r->cancel.store(true);  // fail what the step carried
        cudaStreamSynchronize(s->compute);
        for (auto& p : picks) {
          release_device(s, p.r.get());
          finish_request(s, p.r, ZMC_ECUDA);
        }
        s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                       [](const std::shared_ptr<Request>& r) { return r->done; }),
                        s->active.end());
      } else {
        // the next chunk of a request may be picked by the next step: its
        // tiles run after this step's finalize on the same stream
        for (auto& c : st.completing) {
          Request* r = c.r.get();
          if (c.chunk + 1 < r->nchunks) start_chunk(r, c.chunk + 1);
        }
        log_msg(3, "server step: %d request(s), %lld tiles, %.3g evaluations, %zu chunk(s) "
                "finalized", nsc, (long long)nt, st.evals, st.completing.size());
        inflight.push_back(std::move(st));
        slot ^= 1;
      }
      // 4. keep one step queued behind the running one
      while (inflight.size() >= 2) {
        retire_step(s, inflight.front());
        inflight.pop_front();
      }
    } else if (!inflight.empty()) {
      retire_step(s, inflight.front());
      inflight.pop_front();
    } else if (!s->active.empty()) {
      // nothing to launch: wait (briefly) for the copier to deliver a chunk
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5),
                          [&] { return s->wake != wake_seen || s->stop || !s->queue.empty(); });
    }
    // 5. requests whose last chunk reached host memory, failed copies, and
    // cancellations (their copy jobs drained first: the copier never writes
    // into a finished request's arrays or reads its freed buffers)
    std::vector<std::shared_ptr<Request>> keep;
    for (auto& r : s->active) {
      const int cst = r->copy_status.load();
      if (r->cancel.load() || stopping || cst != ZMC_OK) {
        r->cancel.store(true);
        drain_jobs(r.get());
        cudaStreamSynchronize(s->compute);
        release_device(s, r.get());
        finish_request(s, r, cst != ZMC_OK ? cst : ZMC_ECANCELED);
        continue;
      }
      if (r->delivered.load() == r->nchunks) {
        release_device(s, r.get());
        finish_request(s, r, ZMC_OK);
        continue;
      }
      keep.push_back(r);
    }
    s->active.swap(keep);
  }
}

}  // namespace zmc

using namespace zmc;

extern "C" {

int zmc_server_opts_init(zmc_server_opts* o) {
  if (!o) return fail(ZMC_EINVAL, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->max_active = 128;
  o->step_ms = 10.0;
  o->chunk_units = int64_t(1) << 22;
  o->fail_alloc_every = 0;
  return ZMC_OK;
}

int zmc_server_create(size_t mem_budget_bytes, const zmc_server_opts* opts, zmc_server** out) {
  clear_error();
  if (!out) return fail(ZMC_EINVAL, "out is NULL");
  zmc_server_opts o;
  zmc_server_opts_init(&o);
  if (opts) o = *opts;
  if (o.max_active < 1 || o.max_active > 4096 || !(o.step_ms > 0) || o.chunk_units < 1024 ||
      o.fail_alloc_every < 0)
    return fail(ZMC_EINVAL, "server options out of range");
  if (mem_budget_bytes < (size_t(1) << 20)) return fail(ZMC_EINVAL, "budget below 1 MiB");
  tune_ensure_loaded();
  zmc_server* s = new (std::nothrow) zmc_server();
  if (!s) return fail(ZMC_ENOMEM, "host allocation failed");
  s->opts = o;
  s->budget = mem_budget_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  s->tile_cap = int64_t(1) << 20;
  s->stage_bytes = s256(sizeof(ScanArgs) * o.max_active) + s256(sizeof(BatchTile) * s->tile_cap) +
                   s256(sizeof(FinalizeArgs) * o.max_active) +
                   s256(sizeof(int64_t) * (o.max_active + 1));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  for (int k = 0; k < 2; ++k) {
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev_start[k]);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev_end[k]);
    if (e == cudaSuccess)
      e = cudaHostAlloc(reinterpret_cast<void**>(&s->h_stage[k]), s->stage_bytes, 0);
  }
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_stage), s->stage_bytes);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_counters), 3 * 256);
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "server set-up");
    if (s->d_counters) cudaFree(s->d_counters);
    if (s->d_stage) cudaFree(s->d_stage);
    for (int k = 0; k < 2; ++k) {
      if (s->h_stage[k]) cudaFreeHost(s->h_stage[k]);
      if (s->ev_start[k]) cudaEventDestroy(s->ev_start[k]);
      if (s->ev_end[k]) cudaEventDestroy(s->ev_end[k]);
    }
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    delete s;
    return rc;
  }
  s->copier = std::thread(copier_loop, s);
  s->thread = std::thread(run_loop, s);
  *out = s;
  return ZMC_OK;
}

int zmc_submit(zmc_server* s, const zmc_scan_desc* d, zmc_scan_out* o, uint64_t* ticket) {
  clear_error();
  if (!s || !d || !o || !ticket) return fail(ZMC_EINVAL, "NULL argument");
  int64_t P = 0, count = 0;
  int rc = validate(d, &P, &count);
  if (rc != ZMC_OK) return rc;
  if (d->mem != ZMC_MEM_HOST) return fail(ZMC_EINVAL, "served requests use ZMC_MEM_HOST");
  if (is_user_integrand(d->integrand_id))
    return fail(ZMC_EINVAL, "the server takes the compiled-in integrands only");
  if (d->tile_block != 0 && d->tile_block != kServeBlock)
    return fail(ZMC_EINVAL, "served requests run %d-thread blocks", kServeBlock);
  if (count > 0 && (!o->mean || !o->err)) return fail(ZMC_EINVAL, "mean/err output is NULL");
  auto r = std::make_shared<Request>();
  r->d = *d;
  r->lo.assign(d->lo, d->lo + d->N);
  r->hi.assign(d->hi, d->hi + d->N);
  r->len.assign(d->list_len, d->list_len + d->M);
  int64_t nv = 0;
  for (int i = 0; i < d->M; ++i) nv += d->list_len[i];
  r->vals.assign(d->list_vals, d->list_vals + nv);
  r->d.lo = r->lo.data();
  r->d.hi = r->hi.data();
  r->d.list_len = r->len.data();
  r->d.list_vals = nullptr;  // device copy at admission
  r->d.stream = nullptr;
  r->d.workspace = nullptr;
  r->user_out = o;
  r->o = *o;
  r->count = count;
  r->tp = plan_batch_scan(d);
  const int64_t per_point = int64_t(d->trials) * r->tp.splits;
  r->chunk_points = std::max<int64_t>(1, std::min<int64_t>(count, s->opts.chunk_units / per_point));
  r->nchunks = count > 0 ? (count + r->chunk_points - 1) / r->chunk_points : 0;
  const int64_t T = d->trials;
  r->out_doubles = static_cast<size_t>(r->chunk_points) * (3 + 2 * T);
  const int nbuf = r->nchunks > 1 ? 2 : 1;
  r->bytes = s256(nv * sizeof(double)) + s256(static_cast<size_t>(r->chunk_points) * per_point * 16) +
             nbuf * s256(r->out_doubles * sizeof(double));
  r->evals_total = static_cast<double>(count) * T * d->samples_per_point;
  r->evals_left = r->evals_total;
  r->t_submit = Clock::now();
  if (r->bytes > s->budget)
    return fail(ZMC_ENOMEM, "request needs %zu bytes, more than the server's budget of %zu",
                r->bytes, s->budget);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return fail(ZMC_EBUSY, "server is stopping");
  r->id = s->next_id++;
  s->all[r->id] = r;
  s->submitted++;
  if (count == 0) {  // nothing to compute
    r->done = true;
    r->status = ZMC_OK;
    o->total_ms = 0.0f;
    s->completed++;
    *ticket = r->id;
    return ZMC_OK;
  }
  s->queue.push_back(r);
  s->max_queued = std::max<int64_t>(s->max_queued, static_cast<int64_t>(s->queue.size()));
  *ticket = r->id;
  s->cv_work.notify_one();
  return ZMC_OK;
}

int zmc_poll(zmc_server* s, uint64_t ticket, int* done) {
  clear_error();
  if (!s || !done) return fail(ZMC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(ZMC_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  *done = it->second->done ? 1 : 0;
  return ZMC_OK;
}

int zmc_wait(zmc_server* s, uint64_t ticket, int timeout_ms) {
  clear_error();
  if (!s) return fail(ZMC_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(ZMC_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  std::shared_ptr<Request> r = it->second;
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, [&] { return r->done; });
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                  [&] { return r->done; })) {
    return fail(ZMC_ETIMEDOUT, "ticket %llu still running after %d ms",
                (unsigned long long)ticket, timeout_ms);
  }
  if (r->status != ZMC_OK) return fail(r->status, "ticket %llu ended with status %d",
                                       (unsigned long long)ticket, r->status);
  return ZMC_OK;
}

int zmc_cancel(zmc_server* s, uint64_t ticket) {
  clear_error();
  if (!s) return fail(ZMC_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(ZMC_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  if (it->second->done) return fail(ZMC_EBUSY, "ticket %llu already finished", (unsigned long long)ticket);
  it->second->cancel.store(true);
  s->cv_work.notify_one();
  return ZMC_OK;
}

int zmc_server_stats_get(zmc_server* s, zmc_server_stats* st) {
  clear_error();
  if (!s || !st) return fail(ZMC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->cancelled = s->cancelled;
  st->failed = s->failed;
  st->queued = static_cast<int64_t>(s->queue.size());
  int64_t act = 0;
  for (auto& kv : s->all)
    if (!kv.second->done) ++act;
  st->active = act - st->queued;
  st->max_queued = s->max_queued;
  st->steps = s->steps;
  st->evaluations = static_cast<int64_t>(s->evals_done);
  st->busy_ms = s->busy_ms;
  st->evals_per_s = s->busy_ms > 0 ? s->evals_done / (s->busy_ms * 1e-3) : 0.0;
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      const size_t i = static_cast<size_t>(q * (v.size() - 1) + 0.5);
      return v[std::min(i, v.size() - 1)];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->max_ms = v.back();
    double m = 0;
    for (double x : v) m += x;
    st->mean_ms = m / v.size();
  }
  st->mem_in_use = s->mem_in_use;
  st->mem_peak = s->mem_peak;
  return ZMC_OK;
}

int zmc_server_destroy(zmc_server* s) {
  clear_error();
  if (!s) return ZMC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->thread.joinable()) s->thread.join();
  {
    std::lock_guard<std::mutex> lk(s->cmu);
    s->cstop = true;
  }
  s->ccv.notify_all();
  if (s->copier.joinable()) s->copier.join();
  cudaStreamSynchronize(s->compute);
  cudaStreamSynchronize(s->copy);
  cudaFree(s->d_counters);
  cudaFree(s->d_stage);
  for (int k = 0; k < 2; ++k) {
    cudaFreeHost(s->h_stage[k]);
    cudaEventDestroy(s->ev_start[k]);
    cudaEventDestroy(s->ev_end[k]);
  }
  cudaStreamDestroy(s->compute);
  cudaStreamDestroy(s->copy);
  delete s;
  return ZMC_OK;
}

}  // extern "C"
