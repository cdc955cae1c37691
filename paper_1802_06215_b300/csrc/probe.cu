// ALU throughput probe: eight independent chains of 32-bit integer ops per
// thread (xor then add, two instructions per chain step), enough warps per SM
// to hide latency. Used to measure the integer issue rate the expansion
// kernel's roofline is compared with.
#include <cuda_runtime.h>

#include "model.hpp"

namespace dsp {
namespace {

__global__ void __launch_bounds__(256) alu_probe_kernel(uint32_t* sink, int iters) {
  uint32_t a = threadIdx.x, b = blockIdx.x, c = a ^ 0x9E3779B9u, d = b + 0x7F4A7C15u;
  uint32_t e = a + 11u, f = b ^ 0x85EBCA6Bu, g = a * 3u, h = b * 5u;
  const uint32_t k = blockIdx.x * 0x2545F491u + 1u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      a = (a ^ k) + b;
      b = (b ^ k) + c;
      c = (c ^ k) + d;
      d = (d ^ k) + e;
      e = (e ^ k) + f;
      f = (f ^ k) + g;
      g = (g ^ k) + h;
      h = (h ^ k) + a;
    }
  }
  uint32_t r = a ^ b ^ c ^ d ^ e ^ f ^ g ^ h;
  if (r == 0x12345678u) sink[0] = r;
}

}  // namespace
}  // namespace dsp

extern "C" dsp_status dsp_alu_probe(uint32_t* sink, int32_t iters, double* ops_per_launch, void* stream) {
  if (!sink || iters < 1 || !ops_per_launch) return dsp::fail(DSP_E_INVALID, "dsp_alu_probe: bad argument");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = sms * 8, block = 256;
  dsp::alu_probe_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(sink, iters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dsp::cuda_fail(e, "dsp_alu_probe");
  *ops_per_launch = (double)grid * block * (double)iters * 16.0 * 8.0 * 2.0;
  return DSP_OK;
}
