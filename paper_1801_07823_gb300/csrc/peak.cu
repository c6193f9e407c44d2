// Measured FP64 FMA throughput of the device (the denominator of the FP64
// kernels' roofline): one CTA of 16 warps per SM, each thread running four
// independent chains of dependent FMAs.  On GB300 every shape from one warp
// and one chain per sub-partition up runs at the same rate, so the figure is
// the pipe's sustained rate at the current clock (about 4 flop/clk/SM).
#include "sw_internal.h"

namespace {

constexpr int kChains = 4;
constexpr int kIters = 20000;

__global__ void k_fma_peak(double* out, int iters, double a, double b) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3 + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

int sw_fp64_peak(sw_ctx* c, double* tflops) {
  if (!c || !tflops) return SW_ERR_ARG;
  return guarded(c, [&] {
    int sms = 0;
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    constexpr int kThreadsPeak = 512;
    double* out = nullptr;
    SW_CUDA(cudaMalloc(&out, (size_t)sms * kThreadsPeak * sizeof(double)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) {
      k_fma_peak<<<sms, kThreadsPeak, 0, c->stream>>>(out, kIters / 10, 0.999999, 1e-9);  // warm-up
      sw_count_launch();
      cudaEventRecord(e0, c->stream);
      k_fma_peak<<<sms, kThreadsPeak, 0, c->stream>>>(out, kIters, 0.999999, 1e-9);
      sw_count_launch();
      cudaEventRecord(e1, c->stream);
      err = cudaEventSynchronize(e1);
      if (err == cudaSuccess) err = cudaGetLastError();
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(out, "FP64 peak scratch");
    SW_CUDA(err);
    SW_REQUIRE(ms > 0.f, SW_ERR_CUDA, "FP64 peak kernel took no time");
    const double flop = 2.0 * kChains * (double)kIters * sms * kThreadsPeak;
    *tflops = flop / (ms * 1e-3) / 1e12;
    return SW_OK;
  });
}
