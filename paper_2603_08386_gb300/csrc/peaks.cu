// Pipe throughput microbenchmarks (ddhf_measure_pipes): the denominators of
// the rooflines that bound the NDFT and comb kernels, measured on the device
// that runs them instead of derived from unit counts and clocks.
//
// Each kernel runs kChains independent dependency chains per thread for
// `iters` steps over a grid that fills every SM (8 blocks of 256 threads per
// SM), so the pipe, not the chain latency, sets the rate. Results are stored
// under a data-dependent test that never holds, so nothing is eliminated.
#include <string.h>

#include "ddhf_internal.cuh"

namespace ddhf {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) k_pipe_ffma(float a, float b, int iters, float *sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.2345f) sink[threadIdx.x] = s;
}

// paired FMAs: one f32x2 instruction updates two accumulators (FFMA2)
__global__ void __launch_bounds__(kThreads) k_pipe_ffma2(float a, float b, int iters,
                                                         float *sink) {
  float2 x[kChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)threadIdx.x, (float)c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == -1.2345f) sink[threadIdx.x] = s;
}

// special-function unit: sin.approx and lg2.approx chains (the hardware
// instructions behind __sinf and the comb's base-2 logarithm)
template <int OP>
__global__ void __launch_bounds__(kThreads) k_pipe_mufu(int iters, float *sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 0.001f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      float r;
      if (OP == 0)
        asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
      else
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
      x[c] = r + 1.5f;  // keeps lg2's argument positive and sin's bounded
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.2345f) sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace ddhf

using namespace ddhf;

extern "C" ddhf_status ddhf_measure_pipes(ddhf_pipe_peaks *out, int32_t iters,
                                          ddhf_stream stream) {
  if (!out || iters < 1 || iters > (1 << 24)) return DDHF_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  int dev = 0, nsm = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
    return DDHF_ERR_CUDA;
  out->sm_count = nsm;
  out->sm_clock_max_mhz = khz / 1000;
  cudaStream_t s = (cudaStream_t)stream;
  float *sink = nullptr;
  // a sink in device memory that the kernels never write (their test never
  // holds); allocated here because this is a measurement call, not a hot path
  if (cudaMalloc(&sink, kThreads * sizeof(float)) != cudaSuccess) return DDHF_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ddhf_status st = DDHF_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = DDHF_ERR_CUDA;
  const dim3 grid(nsm * kBlocksPerSm), block(kThreads);
  const double threads = (double)grid.x * kThreads;
  for (int k = 0; k < 4 && st == DDHF_OK; ++k) {
    float ms = 0.f;
    for (int rep = 0; rep < 2 && st == DDHF_OK; ++rep) {  // the first launch warms up
      if (cudaEventRecord(e0, s) != cudaSuccess) st = DDHF_ERR_CUDA;
      switch (k) {
        case 0: k_pipe_ffma<<<grid, block, 0, s>>>(0.9999f, 1e-4f, iters, sink); break;
        case 1: k_pipe_ffma2<<<grid, block, 0, s>>>(0.9999f, 1e-4f, iters, sink); break;
        case 2: k_pipe_mufu<0><<<grid, block, 0, s>>>(iters, sink); break;
        default: k_pipe_mufu<1><<<grid, block, 0, s>>>(iters, sink); break;
      }
      if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        st = DDHF_ERR_CUDA;
    }
    if (st != DDHF_OK) break;
    const double ops = threads * kChains * (double)iters * (k == 1 ? 2.0 : 1.0);
    const double rate = ops / (ms * 1e-3);
    out->elapsed_ms[k] = ms;
    if (k == 0) out->ffma_per_s = rate;
    else if (k == 1) out->ffma2_lane_per_s = rate;
    else if (k == 2) out->sin_approx_per_s = rate;
    else out->lg2_approx_per_s = rate;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}
