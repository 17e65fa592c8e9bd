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
//                   - T2). Lanes hold a TB x 4 tile of (b, r) accumulators,
//                   updated by paired FMAs; events are generated 16 at a time
//                   into shared memory, two lanes per event. Light pixels take one warp,
//                   heavy pixels a whole block (events split over warps,
//                   partial sums reduced in a fixed order), heavy first.
#pragma once

#include "comb.cuh"
#include "ddhf_internal.cuh"

namespace ddhf {
namespace blocked {

constexpr int kGenChunk = 16;

// (a of bin 32 b) mod D = (a0 + 32 b da) mod D, for b < 2^11 (the operand of
// the reduction stays below 2^43).
__device__ __forceinline__ uint64_t arow_residue(const GridConst &g, int b) {
  return mod_barrett(g.a0_mod + (uint64_t)b * g.da32_mod, g.denom, g.barrett);
}

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

// Generate the A and B factors of the events of one chunk; w is the event
// word of event e = lane % 16, active when e < the chunk's event count. Two
// lanes per event run the same code: lane e (half 0) writes B columns
// r = 0..15 and A rows 0..2TB-1, lane e + 16 (half 1) B columns 16..31 and A
// rows 2TB..4TB-1. The step phasors u = e^{-2 pi i da tau / D} (columns) and
// v = u^32 (rows) and each lane's first A row come from exact seeds
// (residues); half 1's first column u^16 is u squared four times (one exact
// seed fewer; its error stays near that of the 16 chain steps it replaces).
// Each lane steps in two interleaved chains.
// arow_mod[h]: (a of the first A row of half h) mod D.
template <int TB>
__device__ __forceinline__ void gen_chunk(uint32_t w, bool active, const GridConst &g,
                                          const uint64_t (&arow_mod)[2], float4 *stage) {
  const int lane = threadIdx.x & 31;
  const int e = lane & 15, half = lane >> 4;
  const uint64_t tau = w & 0x7fffffffu;
  // the two lanes of an event make one step phasor each (half 0: u, half 1:
  // v = u^32) and swap them; each makes its own first A row, and half 1 its
  // first B column u^16 (half 0 starts at u^0 = 1)
  const uint64_t ra = mod_barrett((half ? g.da32_mod : g.da_mod) * tau, g.denom, g.barrett);
  const uint64_t rs = mod_barrett(arow_mod[half] * tau, g.denom, g.barrett);
  const float2 pa = phasor_of_residue(ra, g.two_over_denom);
  const float2 pb = make_float2(__shfl_xor_sync(0xffffffffu, pa.x, 16),
                                __shfl_xor_sync(0xffffffffu, pa.y, 16));
  if (!active) return;
  const float2 u = half ? pb : pa;
  const float2 v = half ? pa : pb;
  float2 s = phasor_of_residue(rs, g.two_over_denom);
  const float2 q2 = cmul(u, u), q4 = cmul(q2, q2), q8 = cmul(q4, q4), q16 = cmul(q8, q8);
  float2 z = half ? q16 : make_float2(1.f, 0.f);
  if (w & kSignBit) {
    s.x = -s.x;
    s.y = -s.y;
  }
  // columns: two interleaved chains (even and odd r) stepped by u^2
  const float2 u2 = cmul(u, u);
  float2 za = z, zb = cmul(z, u);
  float4 *dstb = stage + WarpLayout<TB>::kB + e * kBEvent + half * 4 * 3;
#pragma unroll
  for (int rg = 0; rg < 4; ++rg) {
    const float2 zc = cmul(za, u2), zd = cmul(zb, u2);
    const float br[4] = {za.x, zb.x, zc.x, zd.x};
    const float bi[4] = {za.y, zb.y, zc.y, zd.y};
    if (rg < 3) {
      za = cmul(zc, u2);
      zb = cmul(zd, u2);
    }
    dstb[rg * 3 + 0] = make_float4(br[0], bi[0], br[1], bi[1]);
    dstb[rg * 3 + 1] = make_float4(br[2], bi[2], br[3], bi[3]);
    dstb[rg * 3 + 2] = make_float4(__fadd_rn(br[0], bi[0]), __fadd_rn(br[1], bi[1]),
                                   __fadd_rn(br[2], bi[2]), __fadd_rn(br[3], bi[3]));
  }
  // rows: two interleaved chains (even and odd row) stepped by v^2
  const float2 v2 = cmul(v, v);
  float2 sa = s, sb = cmul(s, v);
  float4 *dsta = stage + WarpLayout<TB>::kA + e * ALayout<TB>::kEvent +
                 half * 2 * ALayout<TB>::kGroup;
#pragma unroll
  for (int k = 0; k < 2 * TB; k += 2) {
    const float ssa = __fadd_rn(sa.x, sa.y), ssb = __fadd_rn(sb.x, sb.y);
    dsta[(k / TB) * ALayout<TB>::kGroup + k % TB] = make_float4(sa.x, sa.y, ssa, ssa);
    dsta[((k + 1) / TB) * ALayout<TB>::kGroup + (k + 1) % TB] = make_float4(sb.x, sb.y, ssb, ssb);
    if (k + 2 < 2 * TB) {
      sa = cmul(sa, v2);
      sb = cmul(sb, v2);
    }
  }
}

// Accumulators of a lane's TB x 4 tile, in float2 pairs so that one paired
// FMA (FFMA2, each element rounded on its own) updates two of them:
// t12[i][q] = (T1, T2) of bin (i, q), t3[i][h] = (T3 of bin (i, 2h), of (i, 2h+1)).
// Shared-memory operands come in matching pairs: A rows as (Ar, Ai, Ar+Ai,
// Ar+Ai), B columns as (Br0, Bi0, Br1, Bi1), (Br2, Bi2, Br3, Bi3),
// (Br0+Bi0, .., Br3+Bi3).
template <int TB>
struct Acc {
  float2 t12[TB][4], t3[TB][2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < TB; ++i) {
#pragma unroll
      for (int q = 0; q < 4; ++q) t12[i][q] = make_float2(0.f, 0.f);
      t3[i][0] = t3[i][1] = make_float2(0.f, 0.f);
    }
  }
  // component c (0: T1, 1: T2, 2: T3) of bin (i, q)
  __device__ __forceinline__ float &at(int c, int i, int q) {
    if (c == 0) return t12[i][q].x;
    if (c == 1) return t12[i][q].y;
    return (q & 1) ? t3[i][q >> 1].y : t3[i][q >> 1].x;
  }
  __device__ __forceinline__ float get(int c, int i, int q) const {
    if (c == 0) return t12[i][q].x;
    if (c == 1) return t12[i][q].y;
    return (q & 1) ? t3[i][q >> 1].y : t3[i][q >> 1].x;
  }
};

// Events [e_lo, e_hi) of the staged chunk into the lane's tile.
template <int TB>
__device__ __forceinline__ void gemm_range(int e_lo, int e_hi, const float4 *stage, Acc<TB> &acc) {
  const int lane = threadIdx.x & 31;
  const int bg = lane >> 3, rg = lane & 7;
  const float4 *sb = stage + WarpLayout<TB>::kB + rg * 3;
  const float4 *sa = stage + WarpLayout<TB>::kA + bg * ALayout<TB>::kGroup;
  for (int e = e_lo; e < e_hi; ++e) {
    const float4 b01 = sb[e * kBEvent + 0];
    const float4 b23 = sb[e * kBEvent + 1];
    const float4 bs = sb[e * kBEvent + 2];
    const float2 bri[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                           make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
    const float2 bss[2] = {make_float2(bs.x, bs.y), make_float2(bs.z, bs.w)};
#pragma unroll
    for (int i = 0; i < TB; ++i) {
      const float4 a = sa[e * ALayout<TB>::kEvent + i];
      const float2 axy = make_float2(a.x, a.y), ass = make_float2(a.z, a.w);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc.t12[i][q] = __ffma2_rn(axy, bri[q], acc.t12[i][q]);
#pragma unroll
      for (int h = 0; h < 2; ++h) acc.t3[i][h] = __ffma2_rn(ass, bss[h], acc.t3[i][h]);
    }
  }
}

template <int TB>
__device__ __forceinline__ void gemm_chunk(int ne, const float4 *stage, Acc<TB> &acc) {
  gemm_range<TB>(0, ne, stage, acc);
}

// Accumulate events [e_begin, e_end) of a pixel in steps of `estep` chunks
// (warp w of a block takes chunks w, w + nw, ...).
template <int TB>
__device__ __forceinline__ void accumulate(const uint32_t *__restrict__ evp, int cnt, int chunk0,
                                           int chunk_step, const GridConst &g,
                                           const uint64_t (&arow_mod)[2],
                                           float4 *stage, Acc<TB> &acc) {
  const int e = threadIdx.x & 15;
  const int step = chunk_step * kGenChunk;
  int c0 = chunk0 * kGenChunk;
  uint32_t w = c0 + e < cnt ? evp[c0 + e] : 0u;
  for (; c0 < cnt; c0 += step) {
    const int ne = min(kGenChunk, cnt - c0);
    gen_chunk<TB>(w, e < ne, g, arow_mod, stage);
    __syncwarp();
    const int c1 = c0 + step;  // the next chunk's event word, loaded ahead
    w = c1 + e < cnt ? evp[c1 + e] : 0u;
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
      const float t1 = acc.get(0, i, q), t2 = acc.get(1, i, q), t3 = acc.get(2, i, q);
      const float fr = __fsub_rn(t1, t2);
      const float fi = __fsub_rn(__fsub_rn(t3, t1), t2);
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
  int vec_store;             // P and ld 16-byte aligned
  int64_t cap_px;
  int heavy_min;
  int skip_min;              // > 0: pixels with at least this many events are left to the
                             // hybrid grid path (their rows are written there)
  int warp_bytes;            // per-warp shared memory (bytes)
  int pw_offset;             // byte offset of the spectrum buffer inside a warp's area
  uint32_t *flags;
  int64_t ev_cap;            // events each slot's event array holds (CSR bound)
};

// Bins [j_begin, j_end) of spectrum row `prow` from Pw (bin j_begin at Pw[0])
// to P, by 16-byte stores when rows are 16-byte aligned (j_begin is a
// multiple of 32).
__device__ __forceinline__ void store_row(const BlockedArgs &A, int64_t prow, int j_begin,
                                          int j_end, const float *Pw) {
  const int lane = threadIdx.x & 31;
  float *dst = A.P + prow * A.ld + j_begin;
  int j0 = j_begin;
  if (A.vec_store) {
    const int n4 = (j_end - j_begin) >> 2;
    for (int i = lane; i < n4; i += 32)
      reinterpret_cast<float4 *>(dst)[i] = reinterpret_cast<const float4 *>(Pw)[i];
    j0 = j_begin + 4 * n4;
  }
  for (int j = j0 + lane; j < j_end; j += 32) dst[j - j_begin] = Pw[j - j_begin];
}

// One pixel's spectrum into Pw (fused: all passes, N padded) or streamed to P.
template <int TB, bool FUSED>
__device__ __forceinline__ void pixel_spectrum_warp(const BlockedArgs &A, const uint32_t *evp,
                                                    int cnt, int64_t prow, float4 *stage,
                                                    float *Pw) {
  const int lane = threadIdx.x & 31;
  const GridConst &g = A.g;
  const int rows_per_pass = 4 * TB;
  for (int b0 = 0; b0 < g.nbr; b0 += rows_per_pass) {
    const uint64_t arow_mod[2] = {arow_residue(g, b0), arow_residue(g, b0 + 2 * TB)};
    Acc<TB> acc;
    acc.zero();
    accumulate<TB>(evp, cnt, 0, 1, g, arow_mod, stage, acc);
    if (FUSED) {
      finalize_tile<TB>(acc, Pw, b0);
    } else {
      finalize_tile<TB>(acc, Pw, 0);
      __syncwarp();
      const int j_begin = 32 * b0, j_end = min(g.N, 32 * (b0 + rows_per_pass));
      store_row(A, prow, j_begin, j_end, Pw);
    }
    __syncwarp();
  }
}

// Power of the lane's tile straight to spectrum row `prow` (bin rows from b0):
// lane (bg, rg) holds bins 32 (b0 + bg TB + i) + 4 rg + q, so each store of
// the warp covers four whole 128-byte rows; bins at or beyond N are not written.
template <int TB>
__device__ __forceinline__ void store_tile(const BlockedArgs &A, const Acc<TB> &acc, int64_t prow,
                                           int b0) {
  const int lane = threadIdx.x & 31;
  const int bg = lane >> 3, rg = lane & 7;
  const int N = A.g.N;
  float *dst = A.P + prow * A.ld;
#pragma unroll
  for (int i = 0; i < TB; ++i) {
    float pv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float t1 = acc.get(0, i, q), t2 = acc.get(1, i, q), t3 = acc.get(2, i, q);
      const float fr = __fsub_rn(t1, t2);
      const float fi = __fsub_rn(__fsub_rn(t3, t1), t2);
      pv[q] = __fmaf_rn(fr, fr, __fmul_rn(fi, fi));
    }
    const int j = 32 * (b0 + bg * TB + i) + 4 * rg;
    if (A.vec_store && j + 3 < N) {
      *reinterpret_cast<float4 *>(dst + j) = make_float4(pv[0], pv[1], pv[2], pv[3]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (j + q < N) dst[j + q] = pv[q];
    }
  }
}

// Light pixels of one slot, spectra to global memory. A warp takes runs of
// `run` consecutive active pixels and, when their event lists follow one
// another in memory (the CSR order of the binning), streams the run's events
// through the 16-event factor chunks in that order: the factors of an event do
// not depend on its pixel, so one chunk serves the end of one pixel and the
// start of the next, and a pixel's tile is stored and cleared as soon as its
// last event is in. Events of pixels outside the run's light set (heavy ones,
// pixels left to the hybrid path, inactive pixels) are skipped chunk-wise.
// Runs whose lists are not in order (caller-built lists) are streamed one
// pixel at a time. The run length is 16 pixels when there are at least eight
// such runs per warp of the grid, and halves (down to one pixel) until there
// are: on a sparse window the warps then share the pixels evenly instead of a
// few runs of heavy-tailed pixels setting the kernel's time. A pixel's events
// are accumulated in the same order whatever the run length, so the spectra
// do not depend on it.
template <int TB>
__device__ __forceinline__ void light_stream(const BlockedArgs &A, float4 *stage) {
  const int lane = threadIdx.x & 31;
  const int e = lane & 15;
  const GridConst &g = A.g;
  const SlotView &v = A.views[A.slot0];
  const int64_t n_act = (int64_t)v.counters[2];
  const int rows_per_pass = 4 * TB;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int run = 16;
  while (run > 1 && (int64_t)run * n_warps * 8 > n_act) run >>= 1;
  for (;;) {
    uint32_t a0 = 0;
    if (lane == 0) a0 = atomicAdd(&A.cursors[1], (uint32_t)run);
    a0 = __shfl_sync(0xffffffffu, a0, 0);
    if ((int64_t)a0 >= n_act) break;
    // lane q < run: pixel a0 + q of the run, its event range and whether it is light
    const int64_t aq = (int64_t)a0 + lane;
    uint32_t q_lo = 0, q_hi = 0;
    bool q_ok = false;
    if (lane < run && aq < n_act) {
      const uint32_t key = v.active[aq];
      q_lo = v.offsets[key];
      q_hi = v.offsets[key + 1];
      const int cnt = (int)(q_hi - q_lo);
      q_ok = cnt < A.heavy_min && !(A.skip_min > 0 && cnt >= A.skip_min) &&
             ddhf_check((int64_t)q_hi <= A.ev_cap, A.flags);
      if (q_ok && aq >= A.cap_px) {
        raise_flag(A.flags, DDHF_FLAG_CAPACITY);
        q_ok = false;
      }
    }
    uint32_t okm = __ballot_sync(0xffffffffu, q_ok);
    if (!okm) continue;
    // in order: every light pixel's list starts at or after the previous one's end
    const uint32_t lower = okm & lanemask_lt();
    const int prev = lower ? 31 - __clz(lower) : -1;
    const uint32_t prev_end = __shfl_sync(0xffffffffu, q_hi, prev < 0 ? 0 : prev);
    const bool bad = q_ok && (q_hi < q_lo || (prev >= 0 && q_lo < prev_end));
    const bool in_order = !__any_sync(0xffffffffu, bad);
    // the whole run at once, or (lists out of order) one pixel at a time
    for (uint32_t todo = okm; todo;) {
      const uint32_t sub = in_order ? todo : (todo & (0u - todo));
      todo &= ~sub;
      const uint32_t e_end = __shfl_sync(0xffffffffu, q_hi, 31 - __clz(sub));
      for (int b0 = 0; b0 < g.nbr; b0 += rows_per_pass) {
        const uint64_t arow_mod[2] = {arow_residue(g, b0), arow_residue(g, b0 + 2 * TB)};
        // the staged chunk holds events [c0, cend); wn: word of event cend + e
        uint32_t c0 = 0, cend = 0, wn = 0;
        bool have_wn = false;
        for (uint32_t rem = sub; rem; rem &= rem - 1) {
          const int p = __ffs(rem) - 1;
          const uint32_t pe0 = __shfl_sync(0xffffffffu, q_lo, p);
          const uint32_t pe1 = __shfl_sync(0xffffffffu, q_hi, p);
          Acc<TB> acc;
          acc.zero();
          for (uint32_t pos = pe0; pos < pe1;) {
            if (pos >= cend) {  // stage the chunk that starts at pos
              const uint32_t w =
                  have_wn && pos == cend ? wn : (pos + e < e_end ? v.ev[pos + e] : 0u);
              c0 = pos;
              cend = min(c0 + (uint32_t)kGenChunk, e_end);
              __syncwarp();  // the previous chunk's products are done
              gen_chunk<TB>(w, c0 + e < cend, g, arow_mod, stage);
              __syncwarp();
              wn = cend + e < e_end ? v.ev[cend + e] : 0u;
              have_wn = true;
            }
            const uint32_t e1 = min(pe1, cend);
            gemm_range<TB>((int)(pos - c0), (int)(e1 - c0), stage, acc);
            pos = e1;
          }
          store_tile<TB>(A, acc, (int64_t)a0 + p, b0);
        }
        __syncwarp();
      }
    }
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
__global__ void __launch_bounds__(256, TB == 6 ? 2 : 1) k_blocked(BlockedArgs A) {
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
    if (A.skip_min > 0 && cnt >= A.skip_min) continue;
    if (!ddhf_check((int64_t)o0 + cnt <= A.ev_cap, A.flags)) continue;
    const int rows_per_pass = 4 * TB;
    bool overflow = !FUSED && a >= A.cap_px;
    if (overflow) {
      if (threadIdx.x == 0) raise_flag(A.flags, DDHF_FLAG_CAPACITY);
      continue;
    }
    for (int b0 = 0; b0 < A.g.nbr; b0 += rows_per_pass) {
      const uint64_t arow_mod[2] = {arow_residue(A.g, b0), arow_residue(A.g, b0 + 2 * TB)};
      Acc<TB> acc;
      acc.zero();
      accumulate<TB>(v.ev + o0, cnt, warp, nw, A.g, arow_mod, stage, acc);
      // partial sums of this warp -> its staging area, [comp][i][q][lane]
      float *part = reinterpret_cast<float *>(stage);
#pragma unroll
      for (int i = 0; i < TB; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          part[((0 * TB + i) * 4 + q) * 32 + lane] = acc.get(0, i, q);
          part[((1 * TB + i) * 4 + q) * 32 + lane] = acc.get(1, i, q);
          part[((2 * TB + i) * 4 + q) * 32 + lane] = acc.get(2, i, q);
        }
      __syncthreads();
      if (warp == 0) {
        for (int w2 = 1; w2 < nw; ++w2) {
          const float *op = reinterpret_cast<const float *>(smem4 + w2 * warp_f4);
#pragma unroll
          for (int i = 0; i < TB; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float &x1 = acc.at(0, i, q), &x2 = acc.at(1, i, q);
              float &x3 = acc.at(2, i, q);
              x1 = __fadd_rn(x1, op[((0 * TB + i) * 4 + q) * 32 + lane]);
              x2 = __fadd_rn(x2, op[((1 * TB + i) * 4 + q) * 32 + lane]);
              x3 = __fadd_rn(x3, op[((2 * TB + i) * 4 + q) * 32 + lane]);
            }
        }
        if (FUSED) {
          finalize_tile<TB>(acc, Pw, b0);
        } else {
          finalize_tile<TB>(acc, Pw, 0);
          __syncwarp();
          const int j_begin = 32 * b0, j_end = min(A.g.N, 32 * (b0 + rows_per_pass));
          store_row(A, a, j_begin, j_end, Pw);
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

  if constexpr (!FUSED) {
    light_stream<TB>(A, stage);
    return;
  }

  // ---------------- light pixels: one warp each, virtual index over slots x pixels.
  // A warp grabs kGrab consecutive virtual pixels; lanes 0..kGrab-1 fetch
  // their metadata in parallel, then the warp takes the pixels in order.
  const int64_t total = (int64_t)A.n_slots * A.npx;
  constexpr int kGrab = 4;
  for (;;) {
    uint32_t v0 = 0;
    if (lane == 0) v0 = atomicAdd(&A.cursors[1], (uint32_t)kGrab);
    v0 = __shfl_sync(0xffffffffu, v0, 0);
    if ((int64_t)v0 >= total) break;
    int m_slot = A.slot0, m_cnt = -1;
    int64_t m_a = 0;
    uint32_t m_key = 0, m_o0 = 0;
    const uint32_t *m_ev = nullptr;
    if (lane < kGrab) {
      const int64_t vi = (int64_t)v0 + lane;
      if (vi < total) {
        const int64_t q = A.n_slots == 1 ? 0 : vi / A.npx;
        m_slot = A.slot0 + (int)q;
        m_a = vi - q * A.npx;
        const SlotView &v = A.views[m_slot];
        if (m_a < (int64_t)v.counters[2]) {
          m_key = v.active[m_a];
          m_o0 = v.offsets[m_key];
          m_cnt = (int)(v.offsets[m_key + 1] - m_o0);
          m_ev = v.ev + m_o0;
        }
      }
    }
    for (int q = 0; q < kGrab; ++q) {
      const int cnt = __shfl_sync(0xffffffffu, m_cnt, q);
      const int slot = __shfl_sync(0xffffffffu, m_slot, q);
      const int64_t a = __shfl_sync(0xffffffffu, m_a, q);
      const uint32_t key = __shfl_sync(0xffffffffu, m_key, q);
      const uint32_t *evp = reinterpret_cast<const uint32_t *>(
          __shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(m_ev), q));
      if (cnt < 0 || cnt >= A.heavy_min) continue;  // inactive, past the end, or heavy
      if (A.skip_min > 0 && cnt >= A.skip_min) continue;  // hybrid grid path
      if (!FUSED && a >= A.cap_px) {
        if (lane == 0) raise_flag(A.flags, DDHF_FLAG_CAPACITY);
        continue;
      }
      pixel_spectrum_warp<TB, FUSED>(A, evp, cnt, a, stage, Pw);
      if (FUSED) {
        CombOut o = comb_warp<NW>(Pw, A.cc, reinterpret_cast<unsigned char *>(stage));
        store_scores<NW>(A, A.views[slot], a, key, o);
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
    int cb = comb_scratch_bytes(c->comb, NW);
    if (cb > scratch) scratch = cb;
  }
  scratch = (scratch + 15) & ~15;
  if (!fused) {
    // the tile of one pass is written after that pass's last GEMM step and
    // streamed out before the next generation step: it shares the staging area
    *pw_offset = 0;
    return scratch > pw ? scratch : pw;
  }
  *pw_offset = scratch;
  return scratch + pw;
}

template <int TB, int NW, bool FUSED>
ddhf_status launch_blocked_t(Ctx *c, int n_slots, float *P, int64_t cap_px, cudaStream_t s,
                             int slot0 = 0, int64_t ld = 0, int skip_min = 0) {
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
  A.vec_store = (A.ld % 4 == 0) && (reinterpret_cast<uintptr_t>(P) % 16 == 0);
  A.cap_px = cap_px;
  A.heavy_min = c->tuning.heavy_min;
  A.skip_min = skip_min;
  A.warp_bytes = blocked_warp_bytes<TB>(c, FUSED, NW, &A.pw_offset);
  A.flags = c->flags;
  A.ev_cap = std::max<int64_t>(c->max_events, 1);
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

// One kernel instantiation per rows-per-lane choice TB, for comb variant NW.
template <int NW, bool FUSED>
ddhf_status launch_blocked_tb(Ctx *c, int n_slots, float *P, int64_t cap_px, cudaStream_t s,
                              int slot0, int64_t ld, int skip_min) {
  const int nbr = c->gconst.nbr;
  int tb = std::min(8, (nbr + 3) / 4);
  tb = tb <= 2 ? tb : tb <= 4 ? 4 : tb <= 6 ? 6 : 8;
  if (c->tuning.rows_per_lane > 0) tb = c->tuning.rows_per_lane;
  switch (tb) {
    case 1: return launch_blocked_t<1, NW, FUSED>(c, n_slots, P, cap_px, s, slot0, ld,
                                                    skip_min);
    case 2: return launch_blocked_t<2, NW, FUSED>(c, n_slots, P, cap_px, s, slot0, ld,
                                                    skip_min);
    case 4: return launch_blocked_t<4, NW, FUSED>(c, n_slots, P, cap_px, s, slot0, ld,
                                                    skip_min);
    case 6: return launch_blocked_t<6, NW, FUSED>(c, n_slots, P, cap_px, s, slot0, ld,
                                                    skip_min);
    case 8: return launch_blocked_t<8, NW, FUSED>(c, n_slots, P, cap_px, s, slot0, ld,
                                                    skip_min);
  }
  return DDHF_ERR_UNSUPPORTED;
}

// The fused kernels with the generic comb (1 or 8 mask words) are
// instantiated in their own translation unit.
extern template ddhf_status launch_blocked_tb<1, true>(Ctx *, int, float *, int64_t, cudaStream_t,
                                                       int, int64_t, int);
extern template ddhf_status launch_blocked_tb<8, true>(Ctx *, int, float *, int64_t, cudaStream_t,
                                                       int, int64_t, int);

template <bool FUSED>
ddhf_status launch_blocked_any(Ctx *c, int n_slots, float *P, int64_t cap_px, cudaStream_t s,
                               int slot0 = 0, int64_t ld = 0, int skip_min = 0) {
  if constexpr (!FUSED) {
    return launch_blocked_tb<1, false>(c, n_slots, P, cap_px, s, slot0, ld, skip_min);
  } else {
    // the comb variant of the spectrum size: fast, or generic with 1 or 8 mask words
    switch (comb_variant(c->comb)) {
      case 0: return launch_blocked_tb<0, true>(c, n_slots, P, cap_px, s, slot0, ld, 0);
      case 1: return launch_blocked_tb<1, true>(c, n_slots, P, cap_px, s, slot0, ld, 0);
      default: return launch_blocked_tb<8, true>(c, n_slots, P, cap_px, s, slot0, ld, 0);
    }
  }
}

}  // namespace blocked
}  // namespace ddhf
