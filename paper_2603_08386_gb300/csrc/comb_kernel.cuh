// The comb-scoring kernel (Eq. 7-11) over spectra in global memory, one warp
// per active pixel, and its launcher. Two input forms:
//   real     rows of P (FP32 powers) in active-list order, row a at P + a * ld;
//   complex  rows of F (FP32 complex sums, float2) by pixel key, the row of
//            active pixel a at F + active[a] * ld; the kernel forms
//            P_j = |F_j|^2 as it loads the row (the sliding-window state).
// comb.cu instantiates the real form, comb_cplx.cu the complex one.
#pragma once

#include "comb.cuh"

namespace ddhf {

// The row is copied to shared memory with all of a lane's loads in flight at
// once (16-byte loads when the rows are 16-byte aligned), then scored by
// comb_warp; with spec_smem = 0 (real input only: the register form on
// 16-byte aligned rows, or the generic comb on a spectrum too large for
// shared memory) comb_warp reads the row in global memory and shared memory
// holds its scratch alone. 4 warps per block; the register form of the fast variant is held
// to 80 registers (6 blocks, 24 warps per SM; its 7.4 KB of shared memory per
// warp at 750 bins would allow 7), the shared-memory form to 64.
template <int NW, bool CPLX>
__global__ void __launch_bounds__(128, NW == 2 ? 6 : (NW == 3 ? 8 : 1)) k_comb(const float *__restrict__ P, int64_t ld, int64_t cap_px,
                       const uint32_t *__restrict__ active, const uint64_t *__restrict__ counters,
                       unsigned long long *cursor, CombConst cc, float *log_sf, float *snr,
                       int32_t *f0, uint8_t *mask, int warp_bytes, int spec_smem, uint32_t *flags) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *base = reinterpret_cast<unsigned char *>(smem4) + warp * warp_bytes;
  float *Pw = reinterpret_cast<float *>(base);
  unsigned char *scratch = base + (spec_smem ? ((cc.N * 4 + 15) & ~15) : 0);
  const int64_t n_active = (int64_t)counters[2];
  const bool vec = (ld % (CPLX ? 2 : 4) == 0) && ((reinterpret_cast<uintptr_t>(P) & 15) == 0);
  const int N = cc.N;
  // a row in floats: N powers, or N complex values
  const int64_t ldf = CPLX ? 2 * ld : ld;
  const int row_floats = CPLX ? 2 * N : N;
  // pixels are taken one at a time from a counter that the launcher zeroes
  // (the cost of a pixel varies with its flatness test and its evaluated
  // candidates, so warps that drew costly pixels take fewer of them); the
  // next index is fetched while the current pixel is scored
  unsigned long long next = 0;
  if (lane == 0) next = atomicAdd(cursor, 1ull);
  for (int64_t a = (int64_t)__shfl_sync(0xffffffffu, next, 0); a < n_active && a < cap_px;
       a = (int64_t)__shfl_sync(0xffffffffu, next, 0)) {
    if (lane == 0) next = atomicAdd(cursor, 1ull);
    const float *row = P + (CPLX ? (int64_t)active[a] : a) * ldf;
    if (!CPLX && !spec_smem) {
      // a spectrum too large for shared memory is scored where it is
      CombOut o = comb_warp<NW>(row, cc, scratch);
      if (!ddhf_check(o.w < 0 || (o.w >= cc.w_lo && o.w <= cc.w_hi), flags)) o.rotor = 0;
      if (lane == 0) {
        if (o.bad) atomicOr(flags, DDHF_FLAG_INTERNAL);
        if (log_sf) log_sf[a] = o.log_sf;
        if (snr) snr[a] = o.snr;
        if (f0) f0[a] = o.w;
        mask[active[a]] = o.rotor;
      }
      __syncwarp();
      continue;
    }
    if (vec) {
      const float4 *r4 = reinterpret_cast<const float4 *>(row);
      const int n4 = (row_floats + 3) / 4;
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
          if (i < n4) {
            if (CPLX) {
              // two complex bins 2i, 2i + 1; P = re^2 + im^2, products rounded first
              const float p0 = __fadd_rn(__fmul_rn(t[u].x, t[u].x), __fmul_rn(t[u].y, t[u].y));
              const float p1 = __fadd_rn(__fmul_rn(t[u].z, t[u].z), __fmul_rn(t[u].w, t[u].w));
              Pw[2 * i] = p0;
              if (2 * i + 1 < N) Pw[2 * i + 1] = p1;
            } else {
              reinterpret_cast<float4 *>(Pw)[i] = t[u];
            }
          }
        }
      }
    } else {
      for (int j0 = 0; j0 < N; j0 += 32 * 8) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + 32 * u + lane;
          if (CPLX) {
            const float re = j < N ? __ldcs(row + 2 * j) : 0.f;
            const float im = j < N ? __ldcs(row + 2 * j + 1) : 0.f;
            t[u] = __fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im));
          } else {
            t[u] = j < N ? __ldcs(row + j) : 0.f;
          }
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
    if (!ddhf_check(o.w < 0 || (o.w >= cc.w_lo && o.w <= cc.w_hi), flags)) o.rotor = 0;
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

// Score the active pixels of slot `slot` (ld: row stride in floats, or in
// complex values for CPLX); clears `mask` first.
template <bool CPLX>
ddhf_status launch_comb_t(Ctx *c, const float *P, int64_t cap_px, float *log_sf, float *snr,
                          int32_t *f0, uint8_t *mask, cudaStream_t s, int slot, int64_t ld) {
  const Slot &sl = c->slots[slot];
  int variant = comb_variant(c->comb);
  if (variant == 0) variant = comb_fast_form(c->comb);
  // 4 warps per block with the spectrum in shared memory when it fits; large
  // spectra (the generic comb) take fewer warps per block, then leave the
  // spectrum in global memory
  int max_smem = 0;
  DDHF_CUDA_TRY(c, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                          c->device));
  const int scratch_b = (comb_scratch_bytes(c->comb, variant) + 15) & ~15;
  const int spec_b = (c->grid.n_bins * 4 + 15) & ~15;
  int wpb = 4, spec_smem = 1;
  // the register form reads its rows where they are when they are 16-byte
  // aligned (each lane loads its 96 contiguous bytes; the row stays in L1)
  const int64_t ldv = ld > 0 ? ld : c->grid.n_bins;
  if (variant == 2 && !CPLX && ldv % 4 == 0 && (reinterpret_cast<uintptr_t>(P) & 15) == 0)
    spec_smem = 0;
  while (spec_smem && wpb > 1 && (spec_b + scratch_b) * wpb > max_smem) wpb >>= 1;
  if (spec_smem && (spec_b + scratch_b) * wpb > max_smem) {
    spec_smem = 0;
    if (CPLX || scratch_b > max_smem) {
      c->last_error = "comb scratch does not fit in shared memory for this grid and comb";
      return DDHF_ERR_UNSUPPORTED;
    }
  }
  const int warp_bytes = (spec_smem ? spec_b : 0) + scratch_b;
  const size_t smem = (size_t)warp_bytes * wpb;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(mask, 0, c->npx, s));
  // the pixel counter of this launch: word 6 of the slot's counters (unused
  // by the binning), so that the combs of different windows never share one
  unsigned long long *cursor = reinterpret_cast<unsigned long long *>(sl.counters + 6);
  DDHF_CUDA_TRY(c, cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s));
#define DDHF_COMB_CASE(NWV)                                                                    \
  {                                                                                            \
    auto kern = k_comb<NWV, CPLX>;                                                             \
    DDHF_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                          (int)smem));                                         \
    int occ = 0;                                                                               \
    DDHF_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem)); \
    if (occ < 1) {                                                                             \
      c->last_error = "comb kernel does not fit on an SM (shared memory)";                     \
      return DDHF_ERR_UNSUPPORTED;                                                             \
    }                                                                                          \
    kern<<<c->num_sms * occ, wpb * 32, smem, s>>>(P, ld > 0 ? ld : c->grid.n_bins, cap_px,     \
                                                  sl.active, sl.counters, cursor, c->comb, log_sf, snr, \
                                                  f0, mask, warp_bytes, spec_smem, c->flags);  \
  }
  if (variant == 2) DDHF_COMB_CASE(2)
  else if (variant == 3) DDHF_COMB_CASE(3)
  else if (variant == 1) DDHF_COMB_CASE(1)
  else DDHF_COMB_CASE(8)
#undef DDHF_COMB_CASE
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

}  // namespace ddhf
