// Comb-scoring kernel (Eq. 7-11) over spectra stored in global memory, one
// warp per active pixel (ddhf_comb_score).
#include "comb.cuh"

namespace ddhf {
namespace {

// ------------------------------------------------------------------ comb

// Rows of P start every `ld` floats. The row is copied to shared memory with
// all of a lane's loads in flight at once (16-byte loads when the rows are
// 16-byte aligned), then scored by comb_warp.
// 4 warps per block; the fast variant is held to 64 registers so that 8 blocks
// fit on an SM with its 6.9 KB of shared memory per warp at 750 bins.
template <int NW>
__global__ void __launch_bounds__(128, NW == 0 ? 8 : 1) k_comb(const float *__restrict__ P, int64_t ld, int64_t cap_px,
                       const uint32_t *__restrict__ active, const uint64_t *__restrict__ counters,
                       CombConst cc, float *log_sf, float *snr, int32_t *f0, uint8_t *mask,
                       int warp_bytes, uint32_t *flags) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *base = reinterpret_cast<unsigned char *>(smem4) + warp * warp_bytes;
  float *Pw = reinterpret_cast<float *>(base);
  unsigned char *scratch = base + ((cc.N * 4 + 15) & ~15);
  const int64_t n_active = (int64_t)counters[2];
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(P) & 15) == 0);
  const int N = cc.N;
  for (int64_t a = wid; a < n_active && a < cap_px; a += nwarps) {
    const float *row = P + a * ld;
    if (vec && lane == 0 && a + nwarps < n_active && a + nwarps < cap_px) {
      // the warp's next row into L2 while this one is scored
      const float *nxt = P + (a + nwarps) * ld;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(nxt),
                   "r"((uint32_t)(((N + 3) / 4) * 16))
                   : "memory");
    }
    if (vec) {
      const float4 *r4 = reinterpret_cast<const float4 *>(row);
      const int n4 = (N + 3) / 4;
      for (int i0 = 0; i0 < n4; i0 += 32 * 8) {
        float4 t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + 32 * u + lane;
          t[u] = i < n4 ? __ldcs(r4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + 32 * u + lane;
          if (i < n4) reinterpret_cast<float4 *>(Pw)[i] = t[u];
        }
      }
    } else {
      for (int j0 = 0; j0 < N; j0 += 32 * 8) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + 32 * u + lane;
          t[u] = j < N ? __ldcs(row + j) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + 32 * u + lane;
          if (j < N) Pw[j] = t[u];
        }
      }
    }
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
                        int32_t *f0, uint8_t *mask, cudaStream_t s, int slot, int64_t ld) {
  const Slot &sl = c->slots[slot];
  const int variant = comb_variant(c->comb);
  const int wpb = 4;
  const int warp_bytes = ((c->grid.n_bins * 4 + 15) & ~15) +
                         ((comb_scratch_bytes(c->grid.n_bins, variant) + 15) & ~15);
  const size_t smem = (size_t)warp_bytes * wpb;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(mask, 0, c->npx, s));
#define DDHF_COMB_CASE(NWV)                                                                    \
  {                                                                                            \
    auto kern = k_comb<NWV>;                                                                   \
    DDHF_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                          (int)smem));                                         \
    int occ = 0;                                                                               \
    DDHF_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem)); \
    if (occ < 1) {                                                                             \
      c->last_error = "comb kernel does not fit on an SM (shared memory)";                     \
      return DDHF_ERR_UNSUPPORTED;                                                             \
    }                                                                                          \
    kern<<<c->num_sms * occ, wpb * 32, smem, s>>>(P, ld > 0 ? ld : c->grid.n_bins, cap_px,     \
                                                  sl.active, sl.counters, c->comb, log_sf, snr, \
                                                  f0, mask, warp_bytes, c->flags);             \
  }
  if (variant == 0) DDHF_COMB_CASE(0)
  else if (variant == 1) DDHF_COMB_CASE(1)
  else DDHF_COMB_CASE(8)
#undef DDHF_COMB_CASE
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

}  // namespace ddhf
