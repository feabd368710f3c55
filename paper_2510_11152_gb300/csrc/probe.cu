// probe.cu -- measured float64 FMA throughput of the current device.
//
// GB300 runs float64 at a small fraction of its float32 rate, so the float64 kernels of the mixed-
// precision solve (the refinement residual above all) can be bound by the FP64 pipe rather than by
// HBM. Their roofline needs the pipe's real rate on the machine at hand, not a nominal figure: this
// file times a kernel of independent DFMA chains with CUDA events and reports FLOP/s (an FMA counts
// as two operations). No counterpart in the paper.
#include <cuda_runtime.h>

#include <string>

#include "../../include/fas.h"

namespace fasmg {
void set_last_error(const std::string& msg);  // fas_api.cu
namespace {

constexpr int kChains = 8;     // independent FMA chains per thread (hides the DFMA latency)
constexpr int kIters = 8192;   // FMAs per chain

__device__ double g_probe_sink;  // keeps the chains' results alive

__global__ void __launch_bounds__(256) k_dfma_chains(double x, double y) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5678) g_probe_sink = s;  // never true for the arguments used; the compiler cannot know
}

}  // namespace
}  // namespace fasmg

extern "C" fas_status fas_probe_fp64_rate(double* tflops) {
  using namespace fasmg;
  if (!tflops) {
    set_last_error("fas_probe_fp64_rate: null argument");
    return FAS_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, 0);
    k_dfma_chains<<<blocks, threads>>>(0.999999, 1e-7);
    cudaEventRecord(e1, 0);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;  // the first launch is a warm-up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("fas_probe_fp64_rate: ") + cudaGetErrorString(e));
    return FAS_ECUDA;
  }
  const double flops = 2.0 * kChains * (double)kIters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return FAS_OK;
}
