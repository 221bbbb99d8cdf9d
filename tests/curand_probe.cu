// curand_probe.cu — test-only: Philox4x32-10 blocks from cuRAND's own device
// implementation (curand_Philox4x32_10 in curand_kernel.h), to pin the
// oracle's and the library's Philox against a third-party implementation.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void probe_kernel(const uint32_t* ctr, const uint32_t* key, int n, uint32_t* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
  uint4 o = curand_Philox4x32_10(c, k);
  out[4 * i] = o.x;
  out[4 * i + 1] = o.y;
  out[4 * i + 2] = o.z;
  out[4 * i + 3] = o.w;
}

extern "C" int curand_probe_philox(const uint32_t* ctr, const uint32_t* key, int n,
                                   uint32_t* out) {
  uint32_t *dc, *dk, *dout;
  if (cudaMalloc(&dc, 16 * (size_t)n) || cudaMalloc(&dk, 8 * (size_t)n) ||
      cudaMalloc(&dout, 16 * (size_t)n))
    return 1;
  cudaMemcpy(dc, ctr, 16 * (size_t)n, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, key, 8 * (size_t)n, cudaMemcpyHostToDevice);
  probe_kernel<<<(n + 127) / 128, 128>>>(dc, dk, n, dout);
  cudaError_t e = cudaMemcpy(out, dout, 16 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 2;
}
