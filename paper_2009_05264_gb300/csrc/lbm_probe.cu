// Arithmetic-peak probes for the benchmark's rooflines: the FP64 and FP32 fused multiply-add
// rate this GPU sustains in a plain (non-tensor) kernel.  Not part of the paper's method; the
// FP64 step is bounded by the FP64 pipe, whose nominal rate is a datasheet figure, so the
// benchmark measures it instead.
#include <cuda_runtime.h>

#include "lbm_internal.h"
#include "pplbm.h"

namespace pplbm {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread: enough to cover the pipe latency

// Every thread runs kChains independent chains of `iters` FMAs each; the result is stored
// so that the compiler keeps every FMA.
template <typename Real>
__global__ void __launch_bounds__(256) fma_probe_kernel(Real* out, int iters, Real m, Real c) {
  Real a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = Real(threadIdx.x + 1) * Real(1e-6) + Real(k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  Real s = Real(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename Real>
lbm_status probe(int64_t iters, cudaStream_t s, double* flops_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LBM_ECUDA;
  const int threads = 256, blocks = sms * 8;
  Real* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(Real) * (size_t)threads * blocks, s) != cudaSuccess) return LBM_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  lbm_status st = LBM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = LBM_ECUDA;
  const Real m = Real(0.999999), c = Real(1e-7);
  if (st == LBM_OK) {
    fma_probe_kernel<Real><<<blocks, threads, 0, s>>>(out, (int)(iters / 8 > 0 ? iters / 8 : 1), m, c);  // warm-up
    cudaEventRecord(e0, s);
    fma_probe_kernel<Real><<<blocks, threads, 0, s>>>(out, (int)iters, m, c);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f))
      st = LBM_ECUDA;
    else
      *flops_per_s = 2.0 * kChains * (double)iters * threads * blocks / (ms * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) st = LBM_ECUDA;
  return st;
}

}  // namespace
}  // namespace pplbm

extern "C" lbm_status lbm_probe_fma_rate(int32_t fp64, int64_t iters, void* cuda_stream, double* flops_per_s) {
  if (!flops_per_s || iters < 1 || iters > (1ll << 30) || (fp64 != 0 && fp64 != 1)) return LBM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return fp64 ? pplbm::probe<double>(iters, s, flops_per_s) : pplbm::probe<float>(iters, s, flops_per_s);
}
