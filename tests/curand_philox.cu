// Test helper: curand's device Philox4x32-10 (a library routine) on a list of
// counters and keys, to pin the oracle's and the library's implementations.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4* ctr, const uint2* key, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox(const unsigned* h_ctr, const unsigned* h_key, unsigned* h_out, int n) {
  uint4 *d_ctr = nullptr, *d_out = nullptr;
  uint2* d_key = nullptr;
  cudaError_t e = cudaMalloc(&d_ctr, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_key, sizeof(uint2) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMemcpy(d_ctr, h_ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_key, h_key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    curand_philox_kernel<<<(n + 127) / 128, 128>>>(d_ctr, d_key, d_out, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h_out, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  cudaFree(d_ctr);
  cudaFree(d_key);
  cudaFree(d_out);
  return (int)e;
}
