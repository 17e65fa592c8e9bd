// Accuracy of the library's sincospi_reduced against CUDA's sincospif on
// |x| <= 1: prints the largest differences in units of the last place of
// sincospif's result (a float at most 1 ulp from the exact value).
#include <cstdio>
#include <cmath>
#include "ddhf_internal.cuh"

__global__ void k_check(int n, unsigned seed, float *err_s, float *err_c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned h = (unsigned)i * 2654435761u + seed;
  h ^= h >> 13;
  h *= 0x5bd1e995u;
  h ^= h >> 15;
  float x = -1.f + 2.f * ((h >> 8) * (1.f / 16777216.f));
  if (i < 4096) x = -1.f + i * (2.f / 4095.f);  // a uniform grid incl. the quarter turns
  float s1, c1, s2, c2;
  sincospif(x, &s1, &c1);
  ddhf::sincospi_reduced(x, s2, c2);
  const float us = fmaxf(fabsf(s1), 1e-30f), uc = fmaxf(fabsf(c1), 1e-30f);
  // ulp of the reference value
  const float ulp_s = fmaxf(nextafterf(us, INFINITY) - us, 1.4e-45f);
  const float ulp_c = fmaxf(nextafterf(uc, INFINITY) - uc, 1.4e-45f);
  // near zero compare in absolute units of 2^-24 (the values are phasor parts)
  err_s[i] = fabsf(s2 - s1) / fmaxf(ulp_s, 5.96e-8f);
  err_c[i] = fabsf(c2 - c1) / fmaxf(ulp_c, 5.96e-8f);
}

int main() {
  const int n = 1 << 24;
  float *es, *ec;
  cudaMalloc(&es, n * sizeof(float));
  cudaMalloc(&ec, n * sizeof(float));
  k_check<<<(n + 255) / 256, 256>>>(n, 12345u, es, ec);
  float *hs = new float[n], *hc = new float[n];
  cudaMemcpy(hs, es, n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(hc, ec, n * sizeof(float), cudaMemcpyDeviceToHost);
  float ms = 0.f, mc = 0.f;
  for (int i = 0; i < n; ++i) {
    ms = fmaxf(ms, hs[i]);
    mc = fmaxf(mc, hc[i]);
  }
  printf("max_sin_ulp %.3f max_cos_ulp %.3f err %s\n", ms, mc,
         cudaGetErrorString(cudaGetLastError()));
  return 0;
}
