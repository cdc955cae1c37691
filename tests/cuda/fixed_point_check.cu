// Exhaustive check of the library's FP32 -> int64 fixed-point conversion
// (dsp::to_fixed, integer operations on the IEEE-754 fields) against CUDA's
// own conversion of x * 2^32 with round to nearest even, over all 2^32 bit
// patterns. Built and run by the GPU tests only.
#include <cuda_runtime.h>

#include "../../paper_1802_06215_b300/csrc/common.cuh"

__global__ void fixed_point_check_kernel(unsigned long long* bad, unsigned int* first) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long nbad = 0;
  unsigned int lo = 0xFFFFFFFFu;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32);
       i += stride) {
    const float x = __uint_as_float((unsigned int)i);
    const long long want = __float2ll_rn(__fmul_rn(x, 4294967296.0f));
    if (dsp::to_fixed(x) != want) {
      ++nbad;
      lo = min(lo, (unsigned int)i);
    }
  }
  if (nbad) {
    atomicAdd(bad, nbad);
    atomicMin(first, lo);
  }
}

// Returns 0 and the number of mismatching patterns and the smallest one
// (0xFFFFFFFF if none), or a CUDA error code.
extern "C" int fixed_point_check(unsigned long long* n_bad, unsigned int* first_bad) {
  unsigned long long* d_bad = nullptr;
  unsigned int* d_first = nullptr;
  cudaError_t e = cudaMalloc(&d_bad, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&d_first, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(d_bad, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d_first, 0xFF, sizeof(unsigned int));
  if (e == cudaSuccess) {
    fixed_point_check_kernel<<<148 * 8, 256>>>(d_bad, d_first);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(n_bad, d_bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(first_bad, d_first, sizeof(unsigned int), cudaMemcpyDeviceToHost);
  cudaFree(d_bad);
  cudaFree(d_first);
  return (int)e;
}
