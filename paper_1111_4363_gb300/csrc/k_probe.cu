// Measured FMA throughput of this GPU: the denominators of the FP64- and FP32-pipe rooflines.
//
// Every thread runs kChains independent FMA chains for `iters` iterations, so the pipe, not the
// dependent-FMA latency, is the limit; the grid is one full wave of resident CTAs on every SM.  The result is
// written to memory only when the chains cancel to a value that cannot occur, so the compiler keeps
// the work and the store costs nothing.
#include <cuda_runtime.h>

#include "../../include/leastaction.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, R a, R b, R* sink) {
  R x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (R)(threadIdx.x + c) * (R)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (R)-12345.678) sink[blockIdx.x] = s;
}

// One full wave: as many CTAs as fit on all SMs at once, so that no SM runs a tail of extra CTAs.
template <typename R>
cudaError_t time_probe(int sms, int iters, cudaStream_t s, double* tflops) {
  R* sink = nullptr;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<R>, kThreads, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int blocks = sms * per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) {
    // warm-up launch (clocks up, code loaded), then the timed one
    k_fma_probe<R><<<blocks, kThreads, 0, s>>>(iters / 4, (R)0.999, (R)1e-4, sink);
    cudaEventRecord(e0, s);
    k_fma_probe<R><<<blocks, kThreads, 0, s>>>(iters, (R)0.999, (R)1e-4, sink);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
  }
  if (err == cudaSuccess) err = cudaGetLastError();
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess)
    *tflops = 2.0 * kChains * (double)iters * blocks * kThreads / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return err;
}

}  // namespace

extern "C" la_status la_fma_peaks(double* fp64_tflops, double* fp32_tflops, int* sm_count, void* cuda_stream) {
  if (!fp64_tflops || !fp32_tflops || !sm_count) return LA_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return LA_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // about 10-20 ms each at the expected rates (FP64 ~1.2 TFLOP/s, FP32 ~75 TFLOP/s)
  if (time_probe<double>(sms, 1 << 11, s, fp64_tflops) != cudaSuccess ||
      time_probe<float>(sms, 1 << 17, s, fp32_tflops) != cudaSuccess) {
    cudaGetLastError();
    return LA_ECUDA;
  }
  *sm_count = sms;
  return LA_OK;
}
