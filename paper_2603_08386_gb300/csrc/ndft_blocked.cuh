// Per-pixel non-uniform DFT power (Sec. 3.3 Eq. 6, P_k = |F_k|^2), the
// comb-scoring kernel (Eq. 7-11) and the fused persistent kernel.
//
// Phases are exact: the phase of event tau at bin j is the integer residue
// r = (a_j * tau) mod D in units of 1/D cycles (64-bit products, Barrett
// reduction), and only that residue is converted to floating point.
//
// Forms (see DDHF_FORM_* in ddhf.h):
//   plain kernels   one warp per active pixel, lane l owns bins l + 32m; the
//                   events are broadcast by warp shuffles; the residue is
//                   advanced from bin to bin by an exact modular step.
//   BLOCKED         bins j = 32b + r. With A[b][k] = p_k e^{-2 pi i a_{32b}
//                   tau_k / D} and B[k][r] = u_k^r, u_k = e^{-2 pi i da tau_k
//                   / D}, F[32b + r] = sum_k A[b][k] B[k][r]: a complex matrix
//                   product per pixel whose factors are generated from two
//                   exact seeds per event (A rows by the step u_k^32, B by
//                   u_k). The product is accumulated with three real
//                   multiplications per term (T1 = sum Ar Br, T2 = sum Ai Bi,
//                   T3 = sum (Ar+Ai)(Br+Bi); Re F = T1 - T2, Im F = T3 - T1
//                   - T2). Lanes hold a TB x 4 tile of (b, r) accumulators;
//                   events are generated 16 at a time into shared memory by
//                   16 "B" lanes and 16 "A" lanes. Light pixels take one warp,
//                   heavy pixels a whole block (events split over warps,
//                   partial sums reduced in a fixed order), heavy first.
#pragma once

#include "comb.cuh"
#include "ddhf_internal.cuh"

namespace ddhf {
namespace blocked {

constexpr int kGenChunk = 16;

__device__ __forceinline__ void raise_flag(uint32_t *flags, uint32_t f) { atomicOr(flags, f); }

// ---------------------------------------------------------------- blocked

// Bank-conflict-free row stride (float4 units) of one lane group's A rows.
template <int TB>
struct ALayout {
  static constexpr int kGroup = (TB % 4 == 0) ? TB + 1 : TB;  // stride between lane groups
  static constexpr int kEvent = 4 * kGroup + 1;               // stride between events
};
constexpr int kBEvent = 25;  // float4 per event of B: [8 rg][3 comps] + 1 pad

template <int TB>
struct WarpLayout {
  // float4 offsets within a warp's staging area
  static constexpr int kB = 0;
  static constexpr int kA = kGenChunk * kBEvent;
  static constexpr int kStageF4 = kA + kGenChunk * ALayout<TB>::kEvent;
};

// Generate the A and B factors of events [0, ne) of one chunk (ev points at
// the chunk's first event). Lanes 0-15 write B rows, lanes 16-31 A rows.
template <int TB>
__device__ __forceinline__ void gen_chunk(const uint32_t *__restrict__ evp, int ne,
                                          const GridConst &g, uint64_t arow_mod, float4 *stage) {
  const int lane = threadIdx.x & 31;
  const int e = lane & 15;
  if (e >= ne) return;
  const uint32_t w = evp[e];
  const uint64_t tau = w & 0x7fffffffu;
  if (lane < 16) {
    const uint64_t r = mod_barrett(g.da_mod * tau, g.denom, g.barrett);
    const float2 u = phasor_of_residue(r, g.two_over_denom);
    float2 z = make_float2(1.f, 0.f);
    float4 *dst = stage + WarpLayout<TB>::kB + e * kBEvent;
#pragma unroll
    for (int rg = 0; rg < 8; ++rg) {
      float br[4], bi[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        br[q] = z.x;
        bi[q] = z.y;
        z = cmul(z, u);
      }
      dst[rg * 3 + 0] = make_float4(br[0], br[1], br[2], br[3]);
      dst[rg * 3 + 1] = make_float4(bi[0], bi[1], bi[2], bi[3]);
      dst[rg * 3 + 2] = make_float4(__fadd_rn(br[0], bi[0]), __fadd_rn(br[1], bi[1]),
                                    __fadd_rn(br[2], bi[2]), __fadd_rn(br[3], bi[3]));
    }
  } else {
    const uint64_t r0 = mod_barrett(arow_mod * tau, g.denom, g.barrett);
    const uint64_t rs = mod_barrett(g.da32_mod * tau, g.denom, g.barrett);
    float2 s = phasor_of_residue(r0, g.two_over_denom);
    if (w & kSignBit) {
      s.x = -s.x;
      s.y = -s.y;
    }
    const float2 v = phasor_of_residue(rs, g.two_over_denom);
    float4 *dst = stage + WarpLayout<TB>::kA + e * ALayout<TB>::kEvent;
#pragma unroll
    for (int bg = 0; bg < 4; ++bg) {
#pragma unroll
      for (int i = 0; i < TB; ++i) {
        dst[bg * ALayout<TB>::kGroup + i] = make_float4(s.x, s.y, __fadd_rn(s.x, s.y), 0.f);
        s = cmul(s, v);
      }
    }
  }
}

template <int TB>
struct Acc {
  float t1[TB][4], t2[TB][4], t3[TB][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < TB; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) t1[i][q] = t2[i][q] = t3[i][q] = 0.f;
  }
};

template <int TB>
__device__ __forceinline__ void gemm_chunk(int ne, const float4 *stage, Acc<TB> &acc) {
  const int lane = threadIdx.x & 31;
  const int bg = lane >> 3, rg = lane & 7;
  const float4 *sb = stage + WarpLayout<TB>::kB + rg * 3;
  const float4 *sa = stage + WarpLayout<TB>::kA + bg * ALayout<TB>::kGroup;
  for (int e = 0; e < ne; ++e) {
    const float4 br = sb[e * kBEvent + 0];
    const float4 bi = sb[e * kBEvent + 1];
    const float4 bs = sb[e * kBEvent + 2];
    const float brr[4] = {br.x, br.y, br.z, br.w};
    const float bii[4] = {bi.x, bi.y, bi.z, bi.w};
    const float bss[4] = {bs.x, bs.y, bs.z, bs.w};
#pragma unroll
    for (int i = 0; i < TB; ++i) {
      const float4 a = sa[e * ALayout<TB>::kEvent + i];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc.t1[i][q] = __fmaf_rn(a.x, brr[q], acc.t1[i][q]);
        acc.t2[i][q] = __fmaf_rn(a.y, bii[q], acc.t2[i][q]);
        acc.t3[i][q] = __fmaf_rn(a.z, bss[q], acc.t3[i][q]);
      }
    }
  }
}

// Accumulate events [e_begin, e_end) of a pixel in steps of `estep` chunks
// (warp w of a block takes chunks w, w + nw, ...).
template <int TB>
__device__ __forceinline__ void accumulate(const uint32_t *__restrict__ evp, int cnt, int chunk0,
                                           int chunk_step, const GridConst &g, uint64_t arow_mod,
                                           float4 *stage, Acc<TB> &acc) {
  for (int c0 = chunk0 * kGenChunk; c0 < cnt; c0 += chunk_step * kGenChunk) {
    const int ne = min(kGenChunk, cnt - c0);
    gen_chunk<TB>(evp + c0, ne, g, arow_mod, stage);
    __syncwarp();
    gemm_chunk<TB>(ne, stage, acc);
    __syncwarp();
  }
}

// Power of the lane's tile into Pw (row-major bins, float4 per lane row).
template <int TB>
__device__ __forceinline__ void finalize_tile(const Acc<TB> &acc, float *Pw, int row_base) {
  const int lane = threadIdx.x & 31;
  const int bg = lane >> 3, rg = lane & 7;
#pragma unroll
  for (int i = 0; i < TB; ++i) {
    float pv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float fr = __fsub_rn(acc.t1[i][q], acc.t2[i][q]);
      const float fi = __fsub_rn(__fsub_rn(acc.t3[i][q], acc.t1[i][q]), acc.t2[i][q]);
      pv[q] = __fmaf_rn(fr, fr, __fmul_rn(fi, fi));
    }
    const int row = row_base + bg * TB + i;
    *reinterpret_cast<float4 *>(Pw + row * 32 + rg * 4) = make_float4(pv[0], pv[1], pv[2], pv[3]);
  }
}

struct BlockedArgs {
  const SlotView *views;
  int slot0;                 // first slot of the light-pixel range
  int n_slots;
  int64_t npx;
  const uint64_t *heavy;     // heavy work items (slot << 32 | active index)
  const uint32_t *n_heavy;   // count of heavy items
  uint32_t heavy_cap;        // capacity of the heavy list
  uint32_t *cursors;         // [0] heavy cursor, [1] light cursor
  GridConst g;
  CombConst cc;
  float *P;                  // spectra (write mode), rows in active order of slot 0
  int64_t ld;                // row stride of P in floats (>= N)
  int64_t cap_px;
  int heavy_min;
  int warp_bytes;            // per-warp shared memory (bytes)
  int pw_offset;             // byte offset of the spectrum buffer inside a warp's area
  uint32_t *flags;
};

// One pixel's spectrum into Pw (fused: all passes, N padded) or streamed to P.
template <int TB, bool FUSED>
__device__ __forceinline__ void pixel_spectrum_warp(const BlockedArgs &A, const uint32_t *evp,
                                                    int cnt, int64_t prow, float4 *stage,
                                                    float *Pw) {
  const int lane = threadIdx.x & 31;
  const GridConst &g = A.g;
  const int rows_per_pass = 4 * TB;
  for (int b0 = 0; b0 < g.nbr; b0 += rows_per_pass) {
    const uint64_t arow_mod = (g.a0 + (uint64_t)(32 * b0) * g.da) % g.denom;
    Acc<TB> acc;
    acc.zero();
    accumulate<TB>(evp, cnt, 0, 1, g, arow_mod, stage, acc);
    if (FUSED) {
      finalize_tile<TB>(acc, Pw, b0);
    } else {
      finalize_tile<TB>(acc, Pw, 0);
      __syncwarp();
      const int j_begin = 32 * b0, j_end = min(g.N, 32 * (b0 + rows_per_pass));
      for (int j = j_begin + lane; j < j_end; j += 32) A.P[prow * A.ld + j] = Pw[j - j_begin];
    }
    __syncwarp();
  }
}

template <int NW>
__device__ __forceinline__ void store_scores(const BlockedArgs &A, const SlotView &v, int64_t a,
                                             uint32_t key, const CombOut &o) {
  if ((threadIdx.x & 31) == 0) {
    if (o.bad) atomicOr(A.flags, DDHF_FLAG_INTERNAL);
    v.log_sf[a] = o.log_sf;
    v.snr[a] = o.snr;
    v.f0[a] = o.w;
    v.mask[key] = o.rotor;
  }
}

template <int TB, int NW, bool FUSED>
__global__ void k_blocked(BlockedArgs A) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int warp_f4 = A.warp_bytes / 16;
  float4 *stage = smem4 + warp * warp_f4;
  float *Pw = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(stage) + A.pw_offset);
  __shared__ uint32_t s_item;

  // ---------------- heavy pixels: one block each, events split over warps
  const uint32_t n_heavy = min(*A.n_heavy, A.heavy_cap);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&A.cursors[0], 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= n_heavy) break;
    const uint64_t it = A.heavy[item];
    const int slot = (int)(it >> 32);
    const int64_t a = (int64_t)(uint32_t)it;
    const SlotView v = A.views[slot];
    const uint32_t key = v.active[a];
    const uint32_t o0 = v.offsets[key];
    const int cnt = (int)(v.offsets[key + 1] - o0);
    const int rows_per_pass = 4 * TB;
    bool overflow = !FUSED && a >= A.cap_px;
    if (overflow) {
      if (threadIdx.x == 0) raise_flag(A.flags, DDHF_FLAG_CAPACITY);
      continue;
    }
    for (int b0 = 0; b0 < A.g.nbr; b0 += rows_per_pass) {
      const uint64_t arow_mod = (A.g.a0 + (uint64_t)(32 * b0) * A.g.da) % A.g.denom;
      Acc<TB> acc;
      acc.zero();
      accumulate<TB>(v.ev + o0, cnt, warp, nw, A.g, arow_mod, stage, acc);
      // partial sums of this warp -> its staging area, [comp][i][q][lane]
      float *part = reinterpret_cast<float *>(stage);
#pragma unroll
      for (int i = 0; i < TB; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          part[((0 * TB + i) * 4 + q) * 32 + lane] = acc.t1[i][q];
          part[((1 * TB + i) * 4 + q) * 32 + lane] = acc.t2[i][q];
          part[((2 * TB + i) * 4 + q) * 32 + lane] = acc.t3[i][q];
        }
      __syncthreads();
      if (warp == 0) {
        for (int w2 = 1; w2 < nw; ++w2) {
          const float *op = reinterpret_cast<const float *>(smem4 + w2 * warp_f4);
#pragma unroll
          for (int i = 0; i < TB; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc.t1[i][q] = __fadd_rn(acc.t1[i][q], op[((0 * TB + i) * 4 + q) * 32 + lane]);
              acc.t2[i][q] = __fadd_rn(acc.t2[i][q], op[((1 * TB + i) * 4 + q) * 32 + lane]);
              acc.t3[i][q] = __fadd_rn(acc.t3[i][q], op[((2 * TB + i) * 4 + q) * 32 + lane]);
            }
        }
        if (FUSED) {
          finalize_tile<TB>(acc, Pw, b0);
        } else {
          finalize_tile<TB>(acc, Pw, 0);
          __syncwarp();
          const int j_begin = 32 * b0, j_end = min(A.g.N, 32 * (b0 + rows_per_pass));
          for (int j = j_begin + lane; j < j_end; j += 32) A.P[a * A.ld + j] = Pw[j - j_begin];
        }
        __syncwarp();
      }
      __syncthreads();
    }
    if (FUSED && warp == 0) {
      CombOut o = comb_warp<NW>(Pw, A.cc, reinterpret_cast<unsigned char *>(stage));
      store_scores<NW>(A, v, a, key, o);
    }
    __syncthreads();
  }

  // ---------------- light pixels: one warp each, virtual index over slots x pixels
  const int64_t total = (int64_t)A.n_slots * A.npx;
  constexpr int kGrab = 4;
  for (;;) {
    uint32_t v0 = 0;
    if (lane == 0) v0 = atomicAdd(&A.cursors[1], (uint32_t)kGrab);
    v0 = __shfl_sync(0xffffffffu, v0, 0);
    if ((int64_t)v0 >= total) break;
    for (int q = 0; q < kGrab; ++q) {
      const int64_t vi = (int64_t)v0 + q;
      if (vi >= total) break;
      const int slot = A.slot0 + (int)(vi / A.npx);
      const int64_t a = vi - (int64_t)(slot - A.slot0) * A.npx;
      const SlotView v = A.views[slot];
      if (a >= (int64_t)v.counters[2]) continue;
      const uint32_t key = v.active[a];
      const uint32_t o0 = v.offsets[key];
      const int cnt = (int)(v.offsets[key + 1] - o0);
      if (cnt >= A.heavy_min) continue;
      if (!FUSED && a >= A.cap_px) {
        if (lane == 0) raise_flag(A.flags, DDHF_FLAG_CAPACITY);
        continue;
      }
      pixel_spectrum_warp<TB, FUSED>(A, v.ev + o0, cnt, a, stage, Pw);
      if (FUSED) {
        CombOut o = comb_warp<NW>(Pw, A.cc, reinterpret_cast<unsigned char *>(stage));
        store_scores<NW>(A, v, a, key, o);
      }
    }
  }
}

template <int TB>
int blocked_warp_bytes(const Ctx *c, bool fused, int NW, int *pw_offset) {
  const int stage = WarpLayout<TB>::kStageF4 * 16;
  const int nbr = (int)c->gconst.nbr;
  const int pw = fused ? ((nbr + 4 * TB - 1) / (4 * TB)) * 4 * TB * 32 * 4 : 4 * TB * 32 * 4;
  int scratch = stage;
  const int partial = 3 * TB * 4 * 32 * 4;
  if (partial > scratch) scratch = partial;
  if (fused) {
    int cb = comb_scratch_bytes(c->grid.n_bins, NW);
    if (cb > scratch) scratch = cb;
  }
  scratch = (scratch + 15) & ~15;
  *pw_offset = scratch;
  return scratch + pw;
}

template <int TB, int NW, bool FUSED>
ddhf_status launch_blocked_t(Ctx *c, int n_slots, float *P, int64_t cap_px, cudaStream_t s,
                             int slot0 = 0, int64_t ld = 0) {
  BlockedArgs A{};
  A.views = c->d_views;
  A.slot0 = slot0;
  A.n_slots = n_slots;
  A.npx = c->npx;
  A.heavy = c->work;
  A.n_heavy = c->qctl + 0;
  A.heavy_cap = (uint32_t)std::min<int64_t>(c->heavy_cap, 0xffffffffll);
  A.cursors = c->qctl + 1;
  A.g = c->gconst;
  A.cc = c->comb;
  A.P = P;
  A.ld = ld > 0 ? ld : c->gconst.N;
  A.cap_px = cap_px;
  A.heavy_min = c->tuning.heavy_min;
  A.warp_bytes = blocked_warp_bytes<TB>(c, FUSED, NW, &A.pw_offset);
  A.flags = c->flags;
  const int wpb = c->tuning.warps_per_block;
  const size_t smem = (size_t)A.warp_bytes * wpb;
  auto kern = k_blocked<TB, NW, FUSED>;
  DDHF_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
  int occ = 0;
  DDHF_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem));
  if (occ < 1) {
    c->last_error = "blocked kernel does not fit on an SM (shared memory)";
    return DDHF_ERR_UNSUPPORTED;
  }
  int bps = c->tuning.blocks_per_sm > 0 ? std::min(occ, c->tuning.blocks_per_sm) : occ;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(c->qctl + 1, 0, 2 * sizeof(uint32_t), s));
  kern<<<c->num_sms * bps, wpb * 32, smem, s>>>(A);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

template <bool FUSED>
ddhf_status launch_blocked_any(Ctx *c, int n_slots, float *P, int64_t cap_px, cudaStream_t s,
                               int slot0 = 0, int64_t ld = 0) {
  const int nbr = c->gconst.nbr;
  int tb = std::min(8, (nbr + 3) / 4);
  tb = tb <= 2 ? tb : tb <= 4 ? 4 : tb <= 6 ? 6 : 8;
  if (c->tuning.rows_per_lane > 0) tb = c->tuning.rows_per_lane;
  // fused: the fast comb where it applies, else the generic one with 8 mask words
  const int variant = comb_variant(c->comb);
#define DDHF_TB_CASE(T)                                                           \
  case T:                                                                         \
    if constexpr (!FUSED) {                                                       \
      return launch_blocked_t<T, 1, false>(c, n_slots, P, cap_px, s, slot0, ld);  \
    } else {                                                                      \
      if (variant == 0)                                                           \
        return launch_blocked_t<T, 0, true>(c, n_slots, P, cap_px, s, slot0, ld); \
      return launch_blocked_t<T, 8, true>(c, n_slots, P, cap_px, s, slot0, ld);   \
    }
  switch (tb) {
    DDHF_TB_CASE(1)
    DDHF_TB_CASE(2)
    DDHF_TB_CASE(4)
    DDHF_TB_CASE(6)
    DDHF_TB_CASE(8)
  }
#undef DDHF_TB_CASE
  return DDHF_ERR_UNSUPPORTED;
}


}  // namespace blocked
}  // namespace ddhf
