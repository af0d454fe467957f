// dg2_peak.cu -- measured FP64 arithmetic peak of the current GPU
// (dg2_fp64_fma_peak), the denominator of the FP64 stage kernels' roofline.
//
// The FP64 DG2 kernels are bound by the FP64 pipe, not by HBM.  This kernel
// measures that pipe's throughput on the same device: every thread runs
// kChains independent chains of fused multiply-adds a <- a * b + c (b just
// below 1, so each chain converges and never overflows or goes subnormal), so
// the pipe sees independent FP64 FMAs back to back.  One FMA is counted as two
// floating-point operations, the convention of the FLOP counts it is compared
// with (an addition and a multiplication each one).
#include <cuda_runtime.h>

#include <string>

#include "../../include/dg2.h"

namespace dg2 {
void set_error_text(const std::string& s);  // dg2_api.cu
}

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// Written only when a chain ends on an impossible value, so the compiler keeps the
// arithmetic without the kernel needing an output buffer.
__device__ double g_peak_sink;

__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0) g_peak_sink = s;
}

int peak_fail(int code, const std::string& msg) {
  dg2::set_error_text(msg);
  return code;
}

}  // namespace

extern "C" int dg2_fp64_fma_peak(int blocks_per_sm, int iters, void* cuda_stream, double* gflops,
                                 double* ms) {
  if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || !gflops)
    return peak_fail(DG2_E_ARG, "need 1 <= blocks_per_sm <= 8, iters >= 1 and gflops");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return peak_fail(DG2_E_CUDA, "no current CUDA device");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return peak_fail(DG2_E_CUDA, "cudaEventCreate failed");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return peak_fail(DG2_E_CUDA, "cudaEventCreate failed");
  }
  const int blocks = sms * blocks_per_sm;
  // one untimed launch (clocks up, code loaded), then the timed one
  fma_chains_kernel<<<blocks, kThreads, 0, st>>>(iters, 0.9999999, 1e-3);
  cudaEventRecord(e0, st);
  fma_chains_kernel<<<blocks, kThreads, 0, st>>>(iters, 0.9999999, 1e-3);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess)
    return peak_fail(DG2_E_CUDA, std::string("FP64 peak kernel failed: ") + cudaGetErrorString(e));
  const double flops = 2.0 * kChains * (double)iters * kThreads * blocks;
  *gflops = flops / (t * 1e-3) / 1e9;
  if (ms) *ms = t;
  return DG2_OK;
}
