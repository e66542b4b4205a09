// Arithmetic peak of the device for the roofline of ALU-bound kernels.
//
// The multiple Arnoldi path (Sec. III-B, Eq. EQ-LS-MULTIPLE) runs its block
// products in FP64, which GB300 executes at a small fraction of its FP32
// rate, so their roofline is the FP64 FMA throughput, not HBM. This kernel
// measures it: every thread runs 8 or 16 independent FMA chains (enough to
// cover the FMA latency), the grid fills every SM several times over, and
// the results are stored so that no chain can be removed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "gsk_ctx.h"

namespace gsk {
namespace {

template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T* out) {
  T a[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) a[i] = T(1) + T(threadIdx.x + i) * T(1e-6);
  const T m = T(0.999999), c = T(1e-7);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 64 / CH; ++u)
#pragma unroll
      for (int i = 0; i < CH; ++i) a[i] = fma(a[i], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < CH; ++i) s += a[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace gsk

extern "C" int gsk_alu_peak(int32_t precision, int32_t n_rep, double* tflops, void* stream) {
  using namespace gsk;
  if (!tflops || n_rep < 1 || (precision != GSK_FP64 && precision != GSK_MIXED)) return GSK_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GSK_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = sms * 8, block = 256;
  const int iters = precision == GSK_FP64 ? 4096 : 65536;   // about a millisecond per launch
  void* out = nullptr;
  const size_t bytes = (size_t)grid * block * sizeof(double);
  if (cudaMalloc(&out, bytes) != cudaSuccess) return GSK_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = GSK_OK;
  double best = 0.0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = GSK_ECUDA;
  // 8 and 16 independent chains per thread (64 FMAs per iteration either way),
  // the better of the two
  for (int r = 0; r <= 2 * n_rep && rc == GSK_OK; ++r) {      // launch 0 warms up
    const bool ch16 = (r & 1) != 0;
    cudaEventRecord(e0, s);
    if (precision == GSK_FP64) {
      if (ch16) k_fma_chains<double, 16><<<grid, block, 0, s>>>(iters, static_cast<double*>(out));
      else k_fma_chains<double, 8><<<grid, block, 0, s>>>(iters, static_cast<double*>(out));
    } else {
      if (ch16) k_fma_chains<float, 16><<<grid, block, 0, s>>>(iters, static_cast<float*>(out));
      else k_fma_chains<float, 8><<<grid, block, 0, s>>>(iters, static_cast<float*>(out));
    }
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = GSK_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 64.0 * iters * (double)grid * block;
    if (r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == GSK_OK) *tflops = best;
  return rc;
}
