// Comb-scoring kernel (Eq. 7-11) over spectra stored in global memory, one
// warp per active pixel (ddhf_comb_score).
#include "comb.cuh"

namespace ddhf {
namespace {

// ------------------------------------------------------------------ comb

template <int NW>
__global__ void k_comb(const float *__restrict__ P, int64_t cap_px, const uint32_t *__restrict__ active,
                       const uint64_t *__restrict__ counters, CombConst cc, float *log_sf, float *snr,
                       int32_t *f0, uint8_t *mask, int warp_bytes, uint32_t *flags) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *base = reinterpret_cast<unsigned char *>(smem4) + warp * warp_bytes;
  float *Pw = reinterpret_cast<float *>(base);
  unsigned char *scratch = base + ((cc.N * 4 + 15) & ~15);
  const int64_t n_active = (int64_t)counters[2];
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = wid; a < n_active && a < cap_px; a += nwarps) {
    for (int j = lane; j < cc.N; j += 32) Pw[j] = P[a * cc.N + j];
    __syncwarp();
    CombOut o = comb_warp<NW>(Pw, cc, scratch);
    if (lane == 0) {
      if (o.bad) atomicOr(flags, DDHF_FLAG_INTERNAL);
      if (log_sf) log_sf[a] = o.log_sf;
      if (snr) snr[a] = o.snr;
      if (f0) f0[a] = o.w;
      mask[active[a]] = o.rotor;
    }
    __syncwarp();
  }
}

}  // namespace

ddhf_status launch_comb(Ctx *c, const float *P, int64_t cap_px, float *log_sf, float *snr,
                        int32_t *f0, uint8_t *mask, cudaStream_t s, int slot) {
  const Slot &sl = c->slots[slot];
  const int nw = (c->comb.bw + 31) / 32;
  const int wpb = 4;
  const int warp_bytes = ((c->grid.n_bins * 4 + 15) & ~15) +
                         ((CombScratch::bytes(c->grid.n_bins, nw <= 1 ? 1 : 8) + 15) & ~15);
  const size_t smem = (size_t)warp_bytes * wpb;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(mask, 0, c->npx, s));
  const int blocks = c->num_sms * 4;
#define DDHF_COMB_CASE(NWV)                                                                    \
  {                                                                                            \
    auto kern = k_comb<NWV>;                                                                   \
    DDHF_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                          (int)smem));                                         \
    kern<<<blocks, wpb * 32, smem, s>>>(P, cap_px, sl.active, sl.counters,   \
                                        c->comb, log_sf, snr, f0, mask, warp_bytes, c->flags);           \
  }
  if (nw <= 1) DDHF_COMB_CASE(1)
  else DDHF_COMB_CASE(8)
#undef DDHF_COMB_CASE
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

}  // namespace ddhf
