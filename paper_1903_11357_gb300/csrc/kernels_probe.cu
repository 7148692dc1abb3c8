// FP64 FMA issue-rate probe (no paper counterpart): the denominator of the roofline of the FP64 kernels.
// One CTA of 16 warps per SM, each thread running 8 independent FMA chains; the per-SM rate is taken from
// the CTA's own clock64 cycles, the GPU-wide rate from the launch's CUDA-event time.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.h"

namespace {

constexpr int PROBE_THREADS = 512;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fp64(int iters, double* sink, long long* cycles) {
  double a[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = 1e-3 * threadIdx.x + c;
  const double x = 1.0000001, y = 1e-9;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = fma(a[c], x, y);
  }
  __syncthreads();
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += a[c];
  if (s == 12345.678) sink[threadIdx.x] = s;   // keeps the chains alive; never true for these inputs
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" int dgasm_probe_fp64(int* nsm, double* fma_per_clk_per_sm, double* tflops) {
  using namespace dgasm;
  clear_error();
  if (!nsm || !fma_per_clk_per_sm || !tflops) return set_error(DGASM_EINVAL, "dgasm_probe_fp64: NULL argument");
  int dev = 0, sms = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DevBuf sink, cyc;
  DG_TRY(sink.alloc(sizeof(double) * PROBE_THREADS));
  DG_TRY(cyc.alloc(sizeof(long long) * sms));
  cudaEvent_t e0, e1;
  DG_CUDA(cudaEventCreate(&e0));
  DG_CUDA(cudaEventCreate(&e1));
  const int iters = 1 << 14;
  k_probe_fp64<<<sms, PROBE_THREADS>>>(64, sink.as<double>(), cyc.as<long long>());   // warm-up
  cudaEventRecord(e0);
  k_probe_fp64<<<sms, PROBE_THREADS>>>(iters, sink.as<double>(), cyc.as<long long>());
  cudaEventRecord(e1);
  cudaError_t ce = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_error((int)ce, "dgasm_probe_fp64");
  std::vector<long long> h(sms);
  DG_CUDA(cudaMemcpy(h.data(), cyc.ptr, sizeof(long long) * sms, cudaMemcpyDeviceToHost));
  std::sort(h.begin(), h.end());
  const double fmas_per_cta = (double)iters * PROBE_CHAINS * PROBE_THREADS;
  *nsm = sms;
  *fma_per_clk_per_sm = fmas_per_cta / (double)h[sms / 2];   // median SM
  *tflops = 2.0 * fmas_per_cta * sms / (ms * 1e-3) / 1e12;
  return DGASM_OK;
}
