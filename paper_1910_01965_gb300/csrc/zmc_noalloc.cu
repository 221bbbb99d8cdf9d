// zmc_noalloc.cu — zmc_scan_noalloc: a scan that allocates no memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the moment they
// want a scan: code on a latency-critical path, where an allocation can wait
// on the driver or synchronise the device; code inside a host framework that
// owns all device memory through its own allocator and accounts every byte
// against a budget; and hosts that fix their device footprint at start-up.
// For them this entry point runs the same sampling and finalize kernels as
// zmc_scan_ex, with the only scratch a scan needs — the FP64 partial sums of
// each (grid point, trial, sample range) — in a file-scope device array of
// fixed size instead of an allocation.  The caller still passes the lists and
// the outputs in device memory.
//
// The array is kNoAllocScratchBytes (16 MiB, 2^20 partial-sum pairs).  CUDA
// loads a library's device code lazily, so the array is reserved on a device
// when the first call there loads this module: that first call (which also
// looks up the array's address and reads the autotuner's cache file, if one is
// named) may allocate, wait on the driver or fail with ZMC_ENOMEM, and callers
// with a fixed footprint should make it once at start-up, before any stream
// capture.  Later calls allocate nothing, and the device keeps the array until
// the process exits.  All calls share it and it keeps the last call's
// contents; nothing in it needs to start at zero (the sampling kernel writes
// every slot the finalize kernel reads), but calls that overlap on the GPU
// race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "zmc_internal.h"
#include "zmc_runtime.h"
#include "zmc_trace.h"

namespace zmc {

constexpr size_t kNoAllocScratchBytes = ZMC_NOALLOC_SCRATCH_BYTES;
constexpr size_t kNoAllocScratchDoubles = kNoAllocScratchBytes / sizeof(double);

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of the array, looked up once per device with that device
// current.  In host code `g_noalloc_scratch` names a host-side stand-in, not
// device memory, so only this address may be handed to a kernel.  Each call
// checks that the recorded address is still device memory of the current
// device (a pointer-attribute query, no allocation) and looks it up again if
// not, e.g. after cudaDeviceReset gave the device a new context.
struct NoAllocSlot {
  bool ready = false;
  double* ptr = nullptr;
};
static std::mutex g_noalloc_mu;
static NoAllocSlot g_noalloc_slot[64];

static bool still_mapped(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

static int noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(ZMC_ECUDA, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocSlot& s = g_noalloc_slot[dev];
  if (s.ready && !still_mapped(s.ptr, dev)) s.ready = false;
  if (!s.ready) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    s.ptr = static_cast<double*>(p);
    s.ready = true;
  }
  *out = s.ptr;
  return ZMC_OK;
}

static bool device_accessible(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static int scan_noalloc(const zmc_scan_desc* d, zmc_scan_out* o) {
  TraceRange trace("zmc_scan_noalloc");
  int64_t P = 0, count = 0;
  int rc = validate(d, &P, &count);
  if (rc != ZMC_OK) return rc;
  if (!o) return fail(ZMC_EINVAL, "output struct is NULL");
  if (d->mem != ZMC_MEM_DEVICE)
    return fail(ZMC_EINVAL, "zmc_scan_noalloc needs ZMC_MEM_DEVICE lists and outputs");
  if (is_user_integrand(d->integrand_id))  // loading their code would allocate
    return fail(ZMC_EINVAL, "zmc_scan_noalloc takes the compiled-in integrands only");
  if (d->workspace)
    return fail(ZMC_EINVAL, "zmc_scan_noalloc takes no workspace (its scratch is built in)");
  if (d->flags & ZMC_F_TIMINGS)
    return fail(ZMC_EINVAL, "zmc_scan_noalloc does not record timings");
  const bool plan_only = (d->flags & ZMC_F_PLAN_ONLY) != 0;
  if (count > 0 && !plan_only && (!o->mean || !o->err))
    return fail(ZMC_EINVAL, "mean/err output is NULL");
  const void* ptrs[6] = {d->list_vals, o->mean, o->err, o->errw, o->s1, o->s2};
  for (int i = 0; i < 6 && !plan_only; ++i)
    if (ptrs[i] && !device_accessible(ptrs[i]))
      return fail(ZMC_EINVAL, "zmc_scan_noalloc given a pointer that is not device memory");

  // The tile plan zmc_scan_ex would make (the autotuner's entry for the
  // scan's class, else the fixed rules) from the device's SM count: an
  // attribute query and memory reads, no allocation.
  int dev = 0, sm = 0, tps = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&tps, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (!d->tile_lanes && !d->tile_splits && !d->tile_block) tune_ensure_loaded();
  const TilePlan tp = plan_with(d, count, sm, tps);
  const double need = static_cast<double>(count) * d->trials * tp.splits * 2 * sizeof(double);
  if (need > static_cast<double>(kNoAllocScratchBytes))
    return fail(ZMC_EINVAL,
                "zmc_scan_noalloc: %.0f bytes of partial sums (points x trials x splits x 16) "
                "exceed its %zu-byte scratch; scan a smaller slice per call",
                need, kNoAllocScratchBytes);

  o->tile_lanes = tp.lanes;
  o->tile_splits = tp.splits;
  o->tile_block = tp.block;
  o->launches = 0;
  o->chunks = count > 0 ? 1 : 0;
  o->h2d_ms = o->kernel_ms = o->finalize_ms = o->d2h_ms = o->total_ms = 0.0f;
  if (count == 0 || plan_only) return ZMC_OK;

  double* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc != ZMC_OK) return rc;

  cudaStream_t stream = static_cast<cudaStream_t>(d->stream);
  ScanArgs a;
  fill_scan_args(d, count, tp, d->list_vals, scratch, &a);
  rc = launch_scan_args(d, a, tp, stream);
  if (rc != ZMC_OK) return rc;

  FinalizeArgs f;
  f.count = count;
  f.S = d->samples_per_point;
  f.T = d->trials;
  f.splits = tp.splits;
  f.V = box_volume(d);
  f.partial = scratch;
  f.mean = o->mean;
  f.err = o->err;
  f.errw = o->errw;
  f.s1 = o->s1;
  f.s2 = o->s2;
  f.dbg = a.dbg;
  const int fe = finalize_launch(f, stream);
  if (fe != 0) return cuda_fail(static_cast<cudaError_t>(fe), "finalize kernel launch");
  o->launches = 2;
  if (d->flags & ZMC_F_SYNC) {
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  }
  return ZMC_OK;
}

}  // namespace zmc

extern "C" int zmc_scan_noalloc(const zmc_scan_desc* d, zmc_scan_out* o) {
  zmc::clear_error();
  return zmc::scan_noalloc(d, o);
}
