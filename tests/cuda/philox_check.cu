// Test helper: the library's device Philox4x32-10 next to cuRAND's block
// function on the same counters and keys.
#include <curand_kernel.h>

#include "md_device.cuh"

__global__ void k_philox_pair(const uint4* ctr, const uint2* key, uint4* mine, uint4* ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  mine[i] = md::philox4x32_10(ctr[i], key[i]);
  ref[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int philox_pair(const unsigned* ctr, const unsigned* key, unsigned* mine,
                           unsigned* ref, int n) {
  uint4 *dc, *dm, *dr;
  uint2* dk;
  if (cudaMalloc(&dc, 16 * n) || cudaMalloc(&dm, 16 * n) || cudaMalloc(&dr, 16 * n) ||
      cudaMalloc(&dk, 8 * n))
    return -1;
  cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, key, 8 * n, cudaMemcpyHostToDevice);
  k_philox_pair<<<(n + 127) / 128, 128>>>(dc, dk, dm, dr, n);
  cudaError_t e = cudaDeviceSynchronize();
  cudaMemcpy(mine, dm, 16 * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(ref, dr, 16 * n, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dm);
  cudaFree(dr);
  cudaFree(dk);
  return e == cudaSuccess ? 0 : -2;
}
