// Warp-level spectral flatness and median-normalised harmonic comb (Sec. 3.4,
// Eq. 7-11) on one pixel's power spectrum held in shared memory.
//
// The FP32 evaluation order is fixed so that the result is a function of the
// spectrum bits alone: window maxima are exact; N(w) = (((0 + m_1) + m_2) +
// ...) / M_valid with every operation rounded on its own; the complement
// median is an exact order statistic (mean of the two middle values as
// (a + b) * 0.5f for an even count); SNR = N(w) / B. The best candidate is the
// largest SNR, the smallest w on ties.
//
// The median of the complement of H(w) is found without sorting per
// candidate. Removing |H(w)| <= h_max = M(2d+1) bins moves the complement's
// middle ranks by at most h_max in the full order, so one exact selection of
// the band of full ranks [lo_r, lo_r + bw) around N/2 per pixel suffices:
// for each candidate, the number of removed bins below the band and the set
// of removed band positions (a bit mask) locate the complement median inside
// the band by a find-nth-zero-bit.
#pragma once

#include "ddhf_internal.cuh"

namespace ddhf {

// Per-warp comb scratch layout (bytes), aliased onto the NDFT staging area.
//   [0, 2048)       band values (f32[256]) and band indices (i32[256])
//   [2048, 6144)    selection histogram (u32[1024])
//   [6144, 6656)    selection candidates (u64[64])
//   from 2048, after the selection: window maxima f32[N], below-band prefix
//   counts u16[N+1], band masks per window centre u32[N][NW]
struct CombScratch {
  static constexpr int kBand = 0;
  static constexpr int kHist = 2048;
  static constexpr int kCand = 6144;
  static constexpr int kSelEnd = 6656;
  static constexpr int kPhase2 = 2048;
  __host__ __device__ static int preb_off(int N) { return kPhase2 + 4 * N; }
  __host__ __device__ static int wmask_off(int N) {
    return preb_off(N) + ((2 * (N + 1) + 15) & ~15);
  }
  __host__ __device__ static int bytes(int N, int NW) {
    int p2 = wmask_off(N) + 4 * N * NW;
    p2 = (p2 + 15) & ~15;
    return p2 > kSelEnd ? p2 : kSelEnd;
  }
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

template <typename T>
__device__ __forceinline__ T warp_excl_scan(T v, T &total) {
  const int lane = threadIdx.x & 31;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  total = __shfl_sync(0xffffffffu, inc, 31);
  return inc - v;
}

// Bitonic sort (ascending) of S = 2^k u64 keys in shared memory by one warp.
__device__ __forceinline__ void warp_sort_u64(uint64_t *a, int S) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= S; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < S; i += 32) {
        int p = i ^ j;
        if (p > i) {
          uint64_t x = a[i], y = a[p];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[p] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Composite key of bin j: float bits (P >= 0, so bit order = value order)
// above the index, giving the (value, index) total order.
__device__ __forceinline__ uint64_t bin_key(const float *Pw, int j) {
  return ((uint64_t)__float_as_uint(Pw[j]) << 16) | (uint32_t)j;
}

// Exact key at full rank R (0-based) by 8-bit radix select over the 48-bit keys.
__device__ __noinline__ static uint64_t select_rank_slow(const float *Pw, int N, int R, uint32_t *hist) {
  const int lane = threadIdx.x & 31;
  uint64_t prefix = 0, pmask = 0;
  int r = R;
  for (int shift = 40; shift >= 0; shift -= 8) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    for (int j = lane; j < N; j += 32) {
      uint64_t key = bin_key(Pw, j);
      if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255], 1u);
    }
    __syncwarp();
    uint32_t h[8], s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      h[q] = hist[lane * 8 + q];
      s += h[q];
    }
    uint32_t tot;
    uint32_t ex = warp_excl_scan<uint32_t>(s, tot);
    bool own = (uint32_t)r >= ex && (uint32_t)r < ex + s;
    uint32_t ball = __ballot_sync(0xffffffffu, own);
    int src = __ffs(ball) - 1;
    int g = 0;
    uint32_t below = 0;
    if (lane == src) {
      uint32_t c = ex;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if ((uint32_t)r >= c && (uint32_t)r < c + h[q]) {
          g = lane * 8 + q;
          below = c;
        }
        c += h[q];
      }
    }
    g = __shfl_sync(0xffffffffu, g, src);
    below = __shfl_sync(0xffffffffu, below, src);
    prefix |= (uint64_t)g << shift;
    pmask |= (uint64_t)0xFF << shift;
    r -= (int)below;
    __syncwarp();
  }
  return prefix;
}

struct CombOut {
  float log_sf;
  float snr;
  int32_t w;
  uint8_t rotor;
  uint8_t bad;  // an index check failed (never expected; reported as a device flag)
};

// Bitonic sort (ascending) of 64 u64 keys held two per lane (element i = lane
// + 32 s in register v[s]) by warp shuffles.
__device__ __forceinline__ void warp_sort64_regs(uint64_t &v0, uint64_t &v1) {
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll 1
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {
        if (v0 > v1) {  // k = 64: the whole sequence ascends
          const uint64_t t = v0;
          v0 = v1;
          v1 = t;
        }
      } else {
        const bool lower = (lane & j) == 0;
        const uint64_t o0 = __shfl_xor_sync(0xffffffffu, v0, j);
        const uint64_t o1 = __shfl_xor_sync(0xffffffffu, v1, j);
        const bool up0 = (lane & k) == 0, up1 = ((lane + 32) & k) == 0;
        const uint64_t mn0 = v0 < o0 ? v0 : o0, mx0 = v0 < o0 ? o0 : v0;
        const uint64_t mn1 = v1 < o1 ? v1 : o1, mx1 = v1 < o1 ? o1 : v1;
        v0 = (lower == up0) ? mn0 : mx0;
        v1 = (lower == up1) ? mn1 : mx1;
      }
    }
  }
}

// Mean-scaled linear bucket of a power value (monotone in the value).
__device__ __forceinline__ int lin_bucket(float v, float scale) {
  return (int)fminf(__fmul_rn(v, scale), 1023.f);
}

// 512 linear buckets (the fast path's histogram).
__device__ __forceinline__ int lin_bucket512(float v, float scale) {
  return (int)fminf(__fmul_rn(v, scale), 511.f);
}

// Smallest float v >= 0 with lin_bucket512(v, scale) >= g, for 1 <= g <= 511;
// -1 when the search does not settle (the caller then takes an exact path).
__device__ __forceinline__ float bucket_low(int g, float scale) {
  float v = __fdiv_rn((float)g, scale);
  if (!(v > 0.f) || !(v < __int_as_float(0x7f800000))) return -1.f;
  for (int it = 0; it < 8 && v > 0.f &&
                   lin_bucket512(__uint_as_float(__float_as_uint(v) - 1u), scale) >= g;
       ++it)
    v = __uint_as_float(__float_as_uint(v) - 1u);
  for (int it = 0; it < 8 && lin_bucket512(v, scale) < g; ++it)
    v = __uint_as_float(__float_as_uint(v) + 1u);
  const bool ok = lin_bucket512(v, scale) >= g &&
                  (v == 0.f || lin_bucket512(__uint_as_float(__float_as_uint(v) - 1u), scale) < g);
  return ok ? v : -1.f;
}

__device__ __forceinline__ float snr_of(float nw, float B) {
  return B > 0.f ? __fdiv_rn(nw, B) : (nw > 0.f ? __int_as_float(0x7f800000) : 0.f);
}

// Natural log of a normal float, ln x = log2(x) ln 2, with the hardware base-2
// logarithm (PTX lg2.approx, flush-to-zero form; its inputs here are >= 1e-30).
__device__ __forceinline__ float ln_normal(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return __fmul_rn(r, 0.693147180559945309f);
}

// N(w) = s / M_valid (Eq. 8); a power-of-two divisor is an exact scaling.
__device__ __forceinline__ float comb_nw(float s, int mv) {
  return ((mv & (mv - 1)) == 0) ? __fmul_rn(s, __int_as_float((127 - (__ffs(mv) - 1)) << 23))
                                : __fdiv_rn(s, (float)mv);
}

// Eq. 7-11 for the spectrum Pw[0..N) (shared memory) by the calling warp.
// scratch: CombScratch::bytes(N, NW) bytes of shared memory (16-byte aligned).
template <int NW>
__device__ __forceinline__ CombOut comb_warp_generic(const float *Pw, const CombConst &cc,
                                                     unsigned char *scratch) {
  const int lane = threadIdx.x & 31;
  const int N = cc.N;
  CombOut out;
  // ---- Eq. 7: spectral flatness, ln SF = mean(ln P) - ln(mean P)
  float slog = 0.f, sum = 0.f;
  for (int j = lane; j < N; j += 32) {
    float v = Pw[j];
    slog = __fadd_rn(slog, ln_normal(fmaxf(v, 1e-30f)));
    sum = __fadd_rn(sum, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    slog = __fadd_rn(slog, __shfl_xor_sync(0xffffffffu, slog, o));
    sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, o));
  }
  const float fN = (float)N;
  out.log_sf = sum > 0.f ? __fsub_rn(__fdiv_rn(slog, fN), __logf(__fdiv_rn(sum, fN))) : 0.f;
  out.snr = 0.f;
  out.w = -1;
  out.rotor = 0;
  out.bad = 0;
  if (!(out.log_sf <= cc.ln_tau_sf) || cc.w_hi < cc.w_lo) return out;
  bool bad = false;

  float *bandv = reinterpret_cast<float *>(scratch + CombScratch::kBand);
  int32_t *bandj = reinterpret_cast<int32_t *>(scratch + CombScratch::kBand + 1024);
  uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + CombScratch::kHist);
  uint64_t *cand = reinterpret_cast<uint64_t *>(scratch + CombScratch::kCand);
  const int lo_r = cc.lo_r, bw = cc.bw, hi_r = cc.lo_r + cc.bw - 1;

  // ---- band of full ranks [lo_r, hi_r] in (value, index) order.
  // 1024 linear buckets over [0, 2 * mean): the band usually falls into a few
  // buckets holding ~bw + 2 values, which are then sorted exactly.
  const float scale = __fdiv_rn(512.f, __fdiv_rn(sum, fN));
#pragma unroll 4
  for (int q = 0; q < 32; ++q) hist[q * 32 + lane] = 0;
  __syncwarp();
  for (int j = lane; j < N; j += 32) atomicAdd(&hist[lin_bucket(Pw[j], scale)], 1u);
  __syncwarp();
  uint32_t lsum = 0;
#pragma unroll 4
  for (int q = 0; q < 32; ++q) lsum += hist[lane * 32 + ((q + lane) & 31)];  // rotated: no conflicts
  uint32_t tot;
  const uint32_t lex = warp_excl_scan<uint32_t>(lsum, tot);
  int gsel[2];
  uint32_t gbelow[2], gcount[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const uint32_t R = t == 0 ? (uint32_t)lo_r : (uint32_t)hi_r;
    int src = __ffs(__ballot_sync(0xffffffffu, R >= lex && R < lex + lsum)) - 1;
    if (src < 0) {
      src = 0;
      bad = true;
    }
    const uint32_t base = __shfl_sync(0xffffffffu, lex, src);
    const uint32_t h = hist[src * 32 + lane];
    uint32_t t2;
    const uint32_t ex = warp_excl_scan<uint32_t>(h, t2) + base;
    const bool own = R >= ex && R < ex + h;
    int s2 = __ffs(__ballot_sync(0xffffffffu, own)) - 1;
    if (s2 < 0) {
      s2 = 0;
      bad = true;
    }
    gsel[t] = src * 32 + s2;
    gbelow[t] = __shfl_sync(0xffffffffu, ex, s2);
    gcount[t] = __shfl_sync(0xffffffffu, h, s2);
  }
  const uint32_t cand_below = gbelow[0];
  const uint32_t ncand = gbelow[1] + gcount[1] - cand_below;
  __syncwarp();
  if (ncand <= 64) {
    uint32_t run = 0;
    for (int j0 = 0; j0 < N; j0 += 32) {
      const int j = j0 + lane;
      bool in = false;
      uint64_t key = 0;
      if (j < N) {
        const float v = Pw[j];
        const int g = lin_bucket(v, scale);
        in = g >= gsel[0] && g <= gsel[1];
        key = ((uint64_t)__float_as_uint(v) << 16) | (uint32_t)j;
      }
      const uint32_t b = __ballot_sync(0xffffffffu, in);
      if (in) cand[run + __popc(b & lanemask_lt())] = key;
      run += __popc(b);
    }
    __syncwarp();
    uint64_t v2[2];
    v2[0] = lane < (int)ncand ? cand[lane] : ~0ull;
    v2[1] = lane + 32 < (int)ncand ? cand[lane + 32] : ~0ull;
    warp_sort64_regs(v2[0], v2[1]);
    // sorted element i sits in lane i % 32, register i / 32
    for (int b0 = 0; b0 < bw; b0 += 32) {
      const int i = lo_r - (int)cand_below + b0 + lane;
      const int ic = i < 0 ? 0 : (i > 63 ? 63 : i);
      if (b0 + lane < bw && ic != i) bad = true;
      const uint64_t k0 = __shfl_sync(0xffffffffu, v2[0], ic & 31);
      const uint64_t k1 = __shfl_sync(0xffffffffu, v2[1], ic & 31);
      const uint64_t key = ic < 32 ? k0 : k1;
      if (b0 + lane < bw) {
        bandv[b0 + lane] = __uint_as_float((uint32_t)(key >> 16));
        bandj[b0 + lane] = (int32_t)(key & 0xFFFF);
      }
    }
  } else {
    const uint64_t klo = select_rank_slow(Pw, N, lo_r, hist);
    const uint64_t khi = select_rank_slow(Pw, N, hi_r, hist);
    uint64_t *buf = reinterpret_cast<uint64_t *>(scratch + CombScratch::kHist);
    int S = 32;
    while (S < bw) S <<= 1;
    uint32_t run = 0;
    for (int j0 = 0; j0 < N; j0 += 32) {
      const int j = j0 + lane;
      const uint64_t key = j < N ? bin_key(Pw, j) : ~0ull;
      const bool in = j < N && key >= klo && key <= khi;
      const uint32_t b = __ballot_sync(0xffffffffu, in);
      if (in) buf[run + __popc(b & lanemask_lt())] = key;
      run += __popc(b);
    }
    for (int i = (int)run + lane; i < S; i += 32) buf[i] = ~0ull;
    __syncwarp();
    warp_sort_u64(buf, S);
    for (int b = lane; b < bw; b += 32) {
      const uint64_t key = buf[b];
      bandv[b] = __uint_as_float((uint32_t)(key >> 16));
      bandj[b] = (int32_t)(key & 0xFFFF);
    }
  }
  __syncwarp();
  const uint64_t key_lo = ((uint64_t)__float_as_uint(bandv[0]) << 16) | (uint32_t)bandj[0];

  // ---- per-bin prefix of below-band counts, window maxima, per-centre band masks
  const int d = cc.d;
  float *wmax = reinterpret_cast<float *>(scratch + CombScratch::kPhase2);
  uint16_t *preb = reinterpret_cast<uint16_t *>(scratch + CombScratch::preb_off(N));
  uint32_t *wmask = reinterpret_cast<uint32_t *>(scratch + CombScratch::wmask_off(N));
  {
    uint32_t run = 0;
    for (int j0 = 0; j0 <= N; j0 += 32) {
      const int j = j0 + lane;
      const bool below = j < N && bin_key(Pw, j) < key_lo;
      const uint32_t b = __ballot_sync(0xffffffffu, below);
      if (j <= N) preb[j] = (uint16_t)(run + __popc(b & lanemask_lt()));
      run += __popc(b);
    }
  }
  for (int c = d + lane; c <= N - 1 - d; c += 32) {
    float mx = Pw[c - d];
    if (d <= 4) {
#pragma unroll
      for (int i = 1; i <= 8; ++i)  // fixed trip count: independent loads
        if (i <= 2 * d) mx = fmaxf(mx, Pw[c - d + i]);
    } else {
      for (int i = 1; i <= 2 * d; ++i) mx = fmaxf(mx, Pw[c - d + i]);
    }
    wmax[c] = mx;
  }
  for (int i = lane; i < N * NW; i += 32) wmask[i] = 0;
  __syncwarp();
  for (int b = lane; b < bw; b += 32) {
    const int jb = bandj[b];
    for (int c = max(0, jb - d); c <= min(N - 1, jb + d); ++c)
      atomicOr(&wmask[c * NW + (b >> 5)], 1u << (b & 31));
  }
  __syncwarp();

  // ---- Eq. 8-10 for every candidate fundamental, one candidate per lane
  float best = 0.f;
  int bestw = -1;
  const int L = N - 1 - d;
  for (int w = cc.w_lo + lane; w <= cc.w_hi; w += 32) {
    // M_valid = min(M, floor(L / w)) without an integer division
    int mv = __float2int_rz(__fdiv_rz((float)L, (float)w));
    if ((mv + 1) * w <= L) ++mv;
    if (mv * w > L) --mv;
    mv = min(mv, cc.M);
    float s = 0.f;
    uint32_t mask[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) mask[q] = 0;
    int below = 0, c0 = 0;
    for (int m = 1; m <= mv; ++m) {
      c0 += w;
      s = __fadd_rn(s, wmax[c0]);
#pragma unroll
      for (int q = 0; q < NW; ++q) mask[q] |= wmask[c0 * NW + q];
      below += (int)preb[c0 + d + 1] - (int)preb[c0 - d];
    }
    int h;
    if (w >= 2 * d + 1) {
      h = mv * (2 * d + 1);
    } else {  // overlapping windows: their union is one contiguous range
      h = (mv - 1) * w + 2 * d + 1;
      below = (int)preb[mv * w + d + 1] - (int)preb[w - d];
    }
    const int c = N - h;
    if (c <= 0) continue;
    const float nw = ((mv & (mv - 1)) == 0) ? __fmul_rn(s, 1.0f / (float)mv)
                                            : __fdiv_rn(s, (float)mv);
    const int base = lo_r - below;
    float v[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      int t = (k == 0 ? (c - 1) / 2 : c / 2) - base;
      int pos = -1;
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        if (pos < 0) {
          const uint32_t free_bits = ~mask[q];
          const int nfree = __popc(free_bits);
          if (t >= 0 && t < nfree) pos = q * 32 + (int)__fns(free_bits, 0, t + 1);
          else t -= nfree;
        }
      }
      if (pos < 0 || pos >= bw) {
        pos = 0;
        bad = true;
      }
      v[k] = bandv[pos];
    }
    const float B = (c & 1) ? v[0] : __fmul_rn(__fadd_rn(v[0], v[1]), 0.5f);
    const float snr = snr_of(nw, B);
    if (bestw < 0 || snr > best) {
      best = snr;
      bestw = w;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int ow = __shfl_xor_sync(0xffffffffu, bestw, o);
    if (ow >= 0 && (bestw < 0 || ob > best || (ob == best && ow < bestw))) {
      best = ob;
      bestw = ow;
    }
  }
  out.bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
  out.snr = bestw >= 0 ? best : 0.f;
  out.w = bestw;
  out.rotor = (bestw >= 0 && best >= cc.tau_comb) ? 1 : 0;
  __syncwarp();
  return out;
}


// ------------------------------------------------------------------------
// Fast variant for N <= 1024 bins and a median band of at most 32 ranks.
//
// Same results as comb_warp_generic, bit for bit, with fewer instructions:
//  * 512 linear buckets over [0, 2 mean) are filled in the same pass as the
//    log sum of Eq. 7 (the Eq. 7 sums take 4-bin groups per lane);
//  * the buckets holding ranks lo_r and hi_r bound the candidate set, which is
//    extracted in one pass and sorted in registers as 32-bit keys (value bits
//    relative to the smallest candidate, above the 10-bit bin index);
//  * with (T, tj) the value and bin at rank lo_r, a bin lies below the band
//    exactly when P < T, or P == T at a smaller bin index, so the bins of a
//    window below the band are counted from the spectrum directly, with no
//    prefix array;
//  * one window maximum per window centre and one code byte per bin (band
//    position, below or above the band), from which a candidate's band mask
//    and count of bins below the band are gathered; the complement median is
//    picked from the band values by a shuffle.
// Pixels whose candidates do not fit (more than 64, or a value range above
// 2^22 ulps) take an exact radix selection of the band instead.
// Eq. 8-10 are evaluated in two phases. Every complement median lies between
// the first and last band values T <= B <= T_hi, so LB = N_max / T_hi (the
// largest N(w) over candidates) is a lower bound on the best SNR, and a
// candidate with N(w) / T < LB can neither win nor tie. Phase 1 computes
// N(w) for all candidates; phase 2 runs the exact median and division only
// for the candidates that survive this test (or for all of them when more
// than 64 survive).
// Scratch layout (bytes from the scratch base, 16-byte aligned):
//   [0, R)   R = max(5N, 2048): histogram u32[512] during selection, then the
//            candidate values u32[64] and indices u16[64] (and the fallback's
//            radix histogram), then the window maxima f32[N] and, from 4N,
//            one code byte per bin: its band position 0..31, 32 below the
//            band, 64 above it
//   [R, R + 128)  surviving candidates u16[64]
struct CombFast {
  __host__ __device__ static int rec_bytes(int N) { return 5 * N > 2048 ? 5 * N : 2048; }
  __host__ __device__ static int list_off(int N) { return (rec_bytes(N) + 15) & ~15; }
  __host__ __device__ static int bytes(int N) { return list_off(N) + 128; }
  static constexpr int kMaxN = 1024;
  static constexpr int kMaxBand = 32;
  static constexpr int kMaxList = 64;
};

// Bitonic sort (ascending) of 32 keys, one per lane.
__device__ __forceinline__ uint32_t warp_sort32_u32(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
      const bool lower = (lane & j) == 0, up = (lane & k) == 0;
      const uint32_t mn = min(v, o), mx = max(v, o);
      v = (lower == up) ? mn : mx;
    }
  }
  return v;
}

// Bitonic sort (ascending) of 64 keys, element i = lane + 32 s in v[s].
__device__ __forceinline__ void warp_sort64_u32(uint32_t &v0, uint32_t &v1) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint32_t o0 = __shfl_xor_sync(0xffffffffu, v0, j);
      const uint32_t o1 = __shfl_xor_sync(0xffffffffu, v1, j);
      const bool lower = (lane & j) == 0;
      const bool up0 = k == 32 ? true : (lane & k) == 0;
      const bool up1 = k == 32 ? false : (lane & k) == 0;
      const uint32_t mn0 = min(v0, o0), mx0 = max(v0, o0);
      const uint32_t mn1 = min(v1, o1), mx1 = max(v1, o1);
      v0 = (lower == up0) ? mn0 : mx0;
      v1 = (lower == up1) ? mn1 : mx1;
    }
  }
  const uint32_t a = min(v0, v1), b = max(v0, v1);  // k = 64, j = 32
  v0 = a;
  v1 = b;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const uint32_t o0 = __shfl_xor_sync(0xffffffffu, v0, j);
    const uint32_t o1 = __shfl_xor_sync(0xffffffffu, v1, j);
    const bool lower = (lane & j) == 0;
    v0 = lower ? min(v0, o0) : max(v0, o0);
    v1 = lower ? min(v1, o1) : max(v1, o1);
  }
}

// Bitonic sort (ascending) of 32 u64 keys, one per lane.
__device__ __forceinline__ uint64_t warp_sort32_u64(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
      const bool lower = (lane & j) == 0, up = (lane & k) == 0;
      const uint64_t mn = v < o ? v : o, mx = v < o ? o : v;
      v = (lower == up) ? mn : mx;
    }
  }
  return v;
}

// Position of the k-th (0-based) set bit of x, or -1.
__device__ __forceinline__ int nth_set_bit(uint32_t x, int k) {
  int pos = 0;
  int c = __popc(x & 0xFFFFu);
  if (k >= c) { k -= c; x >>= 16; pos += 16; }
  c = __popc(x & 0xFFu);
  if (k >= c) { k -= c; x >>= 8; pos += 8; }
  c = __popc(x & 0xFu);
  if (k >= c) { k -= c; x >>= 4; pos += 4; }
  c = __popc(x & 0x3u);
  if (k >= c) { k -= c; x >>= 2; pos += 2; }
  c = (int)(x & 1u);
  if (k >= c) { k -= c; x >>= 1; pos += 1; }
  return (k == 0 && (x & 1u)) ? pos : -1;
}

// The band of full ranks [lo_r, hi_r] (bw <= 32 ranks) of Pw[0..N) in the
// (value, index) order, exactly, by radix selection of its two ends: lane p
// gets the value bits and bin of rank lo_r + p. Returns true when the count
// found disagrees with bw (an internal error). Kept out of line: it runs only
// for spectra whose middle ranks the histogram cannot separate.
__device__ __noinline__ static bool comb_band_exact(const float *Pw, int N, int lo_r, int hi_r,
                                                    int bw, uint32_t *hist, uint32_t &bv_bits,
                                                    int &bj) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const uint64_t klo = select_rank_slow(Pw, N, lo_r, hist);
  const uint64_t khi = select_rank_slow(Pw, N, hi_r, hist);
  uint64_t key = ~0ull;
  uint32_t run = 0;
  for (int j0 = 0; j0 < N; j0 += 32) {
    const int j = j0 + lane;
    const uint64_t k = j < N ? bin_key(Pw, j) : ~0ull;
    const bool in = j < N && k >= klo && k <= khi;
    const uint32_t bi = __ballot_sync(0xffffffffu, in);
    const uint32_t slot = run + __popc(bi & lt);
#pragma unroll 1
    for (uint32_t m = bi; m; m &= m - 1) {  // lane `slot` receives the key
      const int srcl = __ffs(m) - 1;
      const uint64_t kk = __shfl_sync(0xffffffffu, k, srcl);
      const uint32_t sl = __shfl_sync(0xffffffffu, slot, srcl);
      if ((uint32_t)lane == sl) key = kk;
    }
    run += __popc(bi);
  }
  key = warp_sort32_u64(key);
  bv_bits = (uint32_t)(key >> 16);
  bj = (int)(key & 0xFFFFu);
  return (int)run != bw;
}

// Bin j (value v) lies below the band that starts at (T, tj) in the
// (value, index) order.
__device__ __forceinline__ bool below_band(float v, int j, float T, int tj) {
  return v < T || (v == T && j < tj);
}

// Window maxima and bin codes for any half-width d (the d = 3 case has an
// inline quad version); out of line.
__device__ __noinline__ static void comb_records_any_d(const float *Pw, int N, int d, float T,
                                                       int tj, float *rec, uint8_t *code) {
  const int lane = threadIdx.x & 31;
  for (int c = lane; c < N; c += 32) {
    float mx = 0.f;
    if (c >= d && c <= N - 1 - d) {
      mx = Pw[c - d];
      for (int i = 1; i <= 2 * d; ++i) mx = fmaxf(mx, Pw[c - d + i]);
    }
    rec[c] = mx;
    code[c] = below_band(Pw[c], c, T, tj) ? 32u : 64u;
  }
}

__device__ __forceinline__ CombOut comb_warp_fast(const float *Pw, const CombConst &cc,
                                                  unsigned char *scratch) {
  const int lane = threadIdx.x & 31;
  const int N = cc.N;
  const uint32_t lt = lanemask_lt();
  uint32_t *hist = reinterpret_cast<uint32_t *>(scratch);
  uint16_t *list = reinterpret_cast<uint16_t *>(scratch + CombFast::list_off(N));
  const float4 *P4 = reinterpret_cast<const float4 *>(Pw);
  const int ng = (N + 3) >> 2;  // 4-bin groups, the last one possibly partial
  CombOut out;
  out.snr = 0.f;
  out.w = -1;
  out.rotor = 0;
  out.bad = 0;
  bool bad = false;

  // ---- Eq. 7 sums (fixed order: 4-bin groups lane-strided, then a
  // butterfly) and the histogram
#pragma unroll
  for (int q = 0; q < 4; ++q)
    reinterpret_cast<uint4 *>(hist)[q * 32 + lane] = make_uint4(0u, 0u, 0u, 0u);
  // full 4-bin groups, then the (at most 3) tail bins in the lane owning
  // group N / 4, in bin order
  const int nfull = N >> 2;
  const int tail_lane = nfull & 31;
  const int jt = nfull << 2;
  float sum = 0.f;
  for (int q = lane; q < nfull; q += 32) {
    const float4 v = P4[q];
    sum = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(sum, v.x), v.y), v.z), v.w);
  }
  if (lane == tail_lane)
    for (int j = jt; j < N; ++j) sum = __fadd_rn(sum, Pw[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, o));
  const float fN = (float)N;
  const float scale = __fdiv_rn(256.f, __fdiv_rn(sum, fN));
  __syncwarp();
  float slog = 0.f;
  for (int q = lane; q < nfull; q += 32) {
    const float4 v = P4[q];
    slog = __fadd_rn(slog, ln_normal(fmaxf(v.x, 1e-30f)));
    slog = __fadd_rn(slog, ln_normal(fmaxf(v.y, 1e-30f)));
    slog = __fadd_rn(slog, ln_normal(fmaxf(v.z, 1e-30f)));
    slog = __fadd_rn(slog, ln_normal(fmaxf(v.w, 1e-30f)));
    atomicAdd(&hist[lin_bucket512(v.x, scale)], 1u);
    atomicAdd(&hist[lin_bucket512(v.y, scale)], 1u);
    atomicAdd(&hist[lin_bucket512(v.z, scale)], 1u);
    atomicAdd(&hist[lin_bucket512(v.w, scale)], 1u);
  }
  if (lane == tail_lane) {
    for (int j = jt; j < N; ++j) {
      const float v = Pw[j];
      slog = __fadd_rn(slog, ln_normal(fmaxf(v, 1e-30f)));
      atomicAdd(&hist[lin_bucket512(v, scale)], 1u);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) slog = __fadd_rn(slog, __shfl_xor_sync(0xffffffffu, slog, o));
  out.log_sf = sum > 0.f ? __fsub_rn(__fdiv_rn(slog, fN), __logf(__fdiv_rn(sum, fN))) : 0.f;
  if (!(out.log_sf <= cc.ln_tau_sf) || cc.w_hi < cc.w_lo) return out;
  __syncwarp();

  // ---- buckets of ranks lo_r and hi_r; lane l owns buckets [16 l, 16 l + 16)
  const int lo_r = cc.lo_r, bw = cc.bw, hi_r = cc.lo_r + cc.bw - 1;
  uint32_t lsum = 0;
  {
    const uint4 *h4 = reinterpret_cast<const uint4 *>(hist) + lane * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 t = h4[(q + (lane >> 1)) & 3];  // rotated: no bank conflicts
      lsum += t.x + t.y + t.z + t.w;
    }
  }
  uint32_t tot;
  const uint32_t lex = warp_excl_scan<uint32_t>(lsum, tot);
  if (tot != (uint32_t)N) bad = true;
  int gsel[2];
  uint32_t gbelow[2], gcount[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const uint32_t R = t == 0 ? (uint32_t)lo_r : (uint32_t)hi_r;
    int src = __ffs(__ballot_sync(0xffffffffu, R >= lex && R < lex + lsum)) - 1;
    if (src < 0) {
      src = 0;
      bad = true;
    }
    const uint32_t base = __shfl_sync(0xffffffffu, lex, src);
    const uint32_t h = lane < 16 ? hist[src * 16 + lane] : 0u;
    uint32_t t2;
    const uint32_t ex = warp_excl_scan<uint32_t>(h, t2) + base;
    int s2 = __ffs(__ballot_sync(0xffffffffu, R >= ex && R < ex + h)) - 1;
    if (s2 < 0) {
      s2 = 0;
      bad = true;
    }
    gsel[t] = src * 16 + s2;
    gbelow[t] = __shfl_sync(0xffffffffu, ex, s2);
    gcount[t] = __shfl_sync(0xffffffffu, h, s2);
  }
  const int cb = (int)gbelow[0];  // bins in buckets below the candidates
  const int ncand = (int)(gbelow[1] + gcount[1]) - cb;
  bool slow = ncand > 64 || bad;
  __syncwarp();

  // ---- the band: lane p < bw holds the bin at full rank lo_r + p
  float bv = 0.f;  // its value
  int bj = 0;      // its bin
  float T = 0.f;   // band start in the (value, index) order: (T, tj)
  int tj = 0;
  if (!slow) {
    uint32_t *cv = hist;                                         // u32[64]
    uint16_t *cj = reinterpret_cast<uint16_t *>(scratch + 256);  // u16[64]
    // candidates are the bins with vlo <= P < vhi, the value bounds of buckets
    // gsel[0] .. gsel[1] (exact: checked against the bucket function)
    const float vlo = gsel[0] == 0 ? 0.f : bucket_low(gsel[0], scale);
    const float vhi = gsel[1] >= 511 ? __int_as_float(0x7f800000) : bucket_low(gsel[1] + 1, scale);
    if (vlo < 0.f || vhi < 0.f) slow = true;
    uint32_t run = 0;
    for (int q0 = 0; q0 < ng; q0 += 32) {
      const int q = q0 + lane;
      const float4 v = q < ng ? P4[q] : make_float4(-1.f, -1.f, -1.f, -1.f);
      const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = 4 * q + u;
        const bool in = e[u] >= vlo && e[u] < vhi && j < N;
        const uint32_t bi = __ballot_sync(0xffffffffu, in);
        if (in) {
          const uint32_t slot = run + __popc(bi & lt);
          if (slot < 64) {
            cv[slot] = __float_as_uint(e[u]);
            cj[slot] = (uint16_t)j;
          }
        }
        run += __popc(bi);
      }
    }
    if ((int)run != ncand) slow = true;
    __syncwarp();
    const bool in0 = lane < ncand, in1 = lane + 32 < ncand;
    const uint32_t b0 = in0 ? cv[lane] : 0xFFFFFFFFu;
    const uint32_t b1 = in1 ? cv[lane + 32] : 0xFFFFFFFFu;
    const uint32_t j0v = in0 ? cj[lane] : 0u;
    const uint32_t j1v = in1 ? cj[lane + 32] : 0u;
    const uint32_t mn = __reduce_min_sync(0xffffffffu, min(b0, b1));
    const uint32_t mx = __reduce_max_sync(0xffffffffu, max(in0 ? b0 : 0u, in1 ? b1 : 0u));
    if (slow || mx - mn >= (1u << 22)) {
      slow = true;
    } else {
      uint32_t k0 = in0 ? (((b0 - mn) << 10) | j0v) : 0xFFFFFFFFu;
      uint32_t k1 = in1 ? (((b1 - mn) << 10) | j1v) : 0xFFFFFFFFu;
      if (ncand <= 32) {
        k0 = warp_sort32_u32(k0);
      } else {
        warp_sort64_u32(k0, k1);
      }
      // sorted element i sits in lane i % 32, register i / 32; band position
      // p is sorted element p0 + p
      const int p0 = lo_r - cb;
      const int i = p0 + lane;
      const int src = i & 31;
      const uint32_t kk0 = __shfl_sync(0xffffffffu, k0, src);
      const uint32_t kk1 = __shfl_sync(0xffffffffu, k1, src);
      const uint32_t key = i < 32 ? kk0 : kk1;
      if (lane < bw && i >= ncand) bad = true;
      bv = __uint_as_float((key >> 10) + mn);
      bj = (int)(key & 1023u);
      T = __shfl_sync(0xffffffffu, bv, 0);
      tj = __shfl_sync(0xffffffffu, bj, 0);
    }
    __syncwarp();
  }
  if (slow) {
    // exact band [lo_r, hi_r] by radix selection (a rare, out-of-line path)
    uint32_t bvu = 0u;
    bad |= comb_band_exact(Pw, N, lo_r, hi_r, bw, hist, bvu, bj);
    bv = __uint_as_float(bvu);
    T = __shfl_sync(0xffffffffu, bv, 0);
    tj = __shfl_sync(0xffffffffu, bj, 0);
    __syncwarp();
  }

  // ---- window maxima: rec[c] = max of P over [c - d, c + d]; bin codes
  const int d = cc.d;
  float *rec = reinterpret_cast<float *>(scratch);
  uint8_t *code = scratch + 4 * N;
  if (d == 3) {
    // centre quads 4q .. 4q + 3: bins 4q - 4 .. 4q + 7 by three 16-byte loads
    const int nq4 = N >> 2;  // quads whose bins 4q .. 4q + 3 are all < N
    for (int q = lane; q < ng; q += 32) {
      float b[12];  // b[i] = P[4q - 4 + i]
      if (q >= 1 && q + 1 < nq4) {
        const float4 x = P4[q - 1], y = P4[q], z = P4[q + 1];
        b[0] = x.x; b[1] = x.y; b[2] = x.z; b[3] = x.w;
        b[4] = y.x; b[5] = y.y; b[6] = y.z; b[7] = y.w;
        b[8] = z.x; b[9] = z.y; b[10] = z.z; b[11] = z.w;
      } else {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
          const int j = 4 * q - 4 + i;
          b[i] = (j >= 0 && j < N) ? Pw[j] : 0.f;
        }
      }
      const float mid = fmaxf(fmaxf(b[4], b[5]), fmaxf(b[6], b[7]));  // 4q .. 4q+3
      const float l1 = fmaxf(b[2], b[3]), r1 = fmaxf(b[8], b[9]);
      const float w0 = fmaxf(mid, fmaxf(b[1], l1));   // 4q-3 .. 4q+3
      const float w1 = fmaxf(mid, fmaxf(l1, b[8]));   // 4q-2 .. 4q+4
      const float w2 = fmaxf(mid, fmaxf(b[3], r1));   // 4q-1 .. 4q+5
      const float w3 = fmaxf(mid, fmaxf(r1, b[10]));  // 4q   .. 4q+6
      const int j0 = 4 * q;
      const uint32_t k0 = below_band(b[4], j0, T, tj) ? 32u : 64u;
      const uint32_t k1 = below_band(b[5], j0 + 1, T, tj) ? 32u : 64u;
      const uint32_t k2 = below_band(b[6], j0 + 2, T, tj) ? 32u : 64u;
      const uint32_t k3 = below_band(b[7], j0 + 3, T, tj) ? 32u : 64u;
      if (q < nq4) {
        reinterpret_cast<float4 *>(rec)[q] = make_float4(w0, w1, w2, w3);
        reinterpret_cast<uint32_t *>(code)[q] = k0 | (k1 << 8) | (k2 << 16) | (k3 << 24);
      } else {  // the partial last quad
        const float wv[4] = {w0, w1, w2, w3};
        const uint32_t kv[4] = {k0, k1, k2, k3};
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j0 + u < N) {
            rec[j0 + u] = wv[u];
            code[j0 + u] = (uint8_t)kv[u];
          }
      }
    }
  } else {
    comb_records_any_d(Pw, N, d, T, tj, rec, code);
  }
  __syncwarp();
  if (lane < bw) code[bj] = (uint8_t)lane;
  __syncwarp();

  // ---- Eq. 8-10, phase 1: N(w) of every candidate and the largest one.
  // When every candidate has M_valid = M and a non-empty complement (always
  // for h_min >= M and N > M(2d+1)), N(w) is a plain sum over M windows.
  const int L = N - 1 - d;
  const int M = cc.M;
  const int n_cand = cc.w_hi - cc.w_lo + 1;
  const bool uniform = M * cc.w_hi <= L && N > M * (2 * d + 1);
  // In the uniform case with at most 256 candidates, lane l keeps the window
  // sums of its candidates l + 32 k in registers for the survivor pass.
  constexpr int kSlots = 8;
  const bool in_regs = uniform && n_cand <= 32 * kSlots;
  float sv[kSlots];
  float maxnw = 0.f;
  if (in_regs) {
    float maxs = 0.f;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      sv[k] = 0.f;
      if (32 * k < n_cand) {
        const int i = 32 * k + lane;
        const int w = cc.w_lo + i;
        if (i < n_cand) {
          float s = 0.f;
          int c0 = 0;
#pragma unroll 4
          for (int m = 0; m < M; ++m) {
            c0 += w;
            s = __fadd_rn(s, rec[c0]);
          }
          sv[k] = s;
          maxs = fmaxf(maxs, s);  // same order as N(w): a common scaling
        }
      }
    }
    maxnw = comb_nw(maxs, M);
  } else if (uniform) {
    for (int i0 = 0; i0 < n_cand; i0 += 32) {
      const int w = cc.w_lo + i0 + lane;
      if (i0 + lane < n_cand) {
        float s = 0.f;
        int c0 = 0;
#pragma unroll 4
        for (int m = 0; m < M; ++m) {
          c0 += w;
          s = __fadd_rn(s, rec[c0]);
        }
        maxnw = fmaxf(maxnw, s);
      }
    }
    maxnw = comb_nw(maxnw, M);
  } else {
    for (int i0 = 0; i0 < n_cand; i0 += 32) {
      const int w = cc.w_lo + i0 + lane;
      if (i0 + lane < n_cand) {
        int mv = M;
        while (mv * w > L) --mv;
        const int h = w >= 2 * d + 1 ? mv * (2 * d + 1) : (mv - 1) * w + 2 * d + 1;
        float s = 0.f;
        int c0 = 0;
        for (int m = 1; m <= mv; ++m) {
          c0 += w;
          s = __fadd_rn(s, rec[c0]);
        }
        if (N - h > 0) maxnw = fmaxf(maxnw, comb_nw(s, mv));
      }
    }
  }
  maxnw = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(maxnw)));  // >= 0
  const float Thi = __shfl_sync(0xffffffffu, bv, bw - 1);
  const float LB = snr_of(maxnw, Thi);
  // keep w when N(w) >= thr; thr <= LB T (1 - 2^-20) (1 + 2^-23), so a
  // dropped candidate has N(w) / T < LB (1 - 2^-21) and SNR(w) < LB
  // (LB and LB T normal and finite, so that the relative rounding bounds hold)
  const float lbt = __fmul_rn(LB, T);
  const bool prune = T > 0.f && LB >= 0x1p-126f && LB < __int_as_float(0x7f800000) &&
                     lbt >= 0x1p-100f && lbt < __int_as_float(0x7f800000);
  const float thr = prune ? __fmul_rn(lbt, 1.0f - 0x1p-20f) : 0.f;

  // ---- surviving candidates, in increasing w
  int n_items = n_cand;
  bool use_list = false;
  if (prune) {
    uint32_t run = 0;
    if (in_regs) {
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        if (32 * k < n_cand) {
          const int i = 32 * k + lane;
          const bool keep = i < n_cand && comb_nw(sv[k], M) >= thr;
          const uint32_t b = __ballot_sync(0xffffffffu, keep);
          const uint32_t slot = run + __popc(b & lt);
          if (keep && slot < (uint32_t)CombFast::kMaxList) list[slot] = (uint16_t)(cc.w_lo + i);
          run += __popc(b);
        }
      }
    } else {
      for (int i0 = 0; i0 < n_cand; i0 += 32) {
        const int w = cc.w_lo + i0 + lane;
        bool keep = false;
        if (i0 + lane < n_cand) {
          int mv = M;
          if (!uniform)
            while (mv * w > L) --mv;
          float s = 0.f;
          int c0 = 0;
#pragma unroll 4
          for (int m = 1; m <= mv; ++m) {
            c0 += w;
            s = __fadd_rn(s, rec[c0]);
          }
          keep = comb_nw(s, mv) >= thr;
        }
        const uint32_t b = __ballot_sync(0xffffffffu, keep);
        const uint32_t slot = run + __popc(b & lt);
        if (keep && slot < (uint32_t)CombFast::kMaxList) list[slot] = (uint16_t)w;
        run += __popc(b);
      }
    }
    if (run <= (uint32_t)CombFast::kMaxList) {
      use_list = true;
      n_items = (int)run;
    }
    __syncwarp();
  }

  // ---- phase 2: exact SNR of the surviving candidates, 32 at a time, one
  // per lane. The band mask of H(w) and its bins below the band are gathered
  // from the bin codes by a group of g lanes per candidate (g the largest
  // power of two with nk g <= 32; each lane takes every g-th bin of H(w)) and
  // combined within the group, then handed to the candidate's lane.
  const uint32_t outside = bw >= 32 ? 0u : (0xFFFFFFFFu << bw);
  float best = 0.f;
  int bestw = -1;
  for (int i0 = 0; i0 < n_items; i0 += 32) {
    const int nk = min(32, n_items - i0);
    const int wl = lane < nk ? (use_list ? (int)list[i0 + lane] : cc.w_lo + i0 + lane) : 1;
    const int g = nk > 16 ? 1 : nk > 8 ? 2 : nk > 4 ? 4 : nk > 2 ? 8 : nk > 1 ? 16 : 32;
    const int gk = lane / g, gs = lane - gk * g;
    const int wk = __shfl_sync(0xffffffffu, wl, gk < nk ? gk : 0);
    uint32_t gmask = 0u;
    int gbelow = 0;
    if (gk < nk) {
      int mvk = M;
      while (mvk * wk > L) --mvk;
      if (wk >= 2 * d + 1) {
        for (int m = 1; m <= mvk; ++m) {
          for (int i = gs - d; i <= d; i += g) {
            const uint32_t k = code[m * wk + i];
            gmask |= __funnelshift_lc(0u, 1u, k);  // 1 << k, 0 for k >= 32
            gbelow += (int)((k >> 5) & 1u);
          }
        }
      } else {  // overlapping windows: one range
        for (int j = wk - d + gs; j <= mvk * wk + d; j += g) {
          const uint32_t k = code[j];
          gmask |= __funnelshift_lc(0u, 1u, k);
          gbelow += (int)((k >> 5) & 1u);
        }
      }
    }
    for (int o = g >> 1; o > 0; o >>= 1) {
      gmask |= __shfl_xor_sync(0xffffffffu, gmask, o);
      gbelow += __shfl_xor_sync(0xffffffffu, gbelow, o);
    }
    const int lead = lane * g < 32 ? lane * g : 0;
    const uint32_t my_mask = __shfl_sync(0xffffffffu, gmask, lead);
    const int my_below = __shfl_sync(0xffffffffu, gbelow, lead);
    const bool ok = lane < nk;
    const int w = wl;
    int pos0 = 0, pos1 = 0, c = 0, mv = 1;
    float s = 0.f;
    if (ok) {
      mv = M;
      while (mv * w > L) --mv;
      int c0 = 0;
#pragma unroll 4
      for (int m = 1; m <= mv; ++m) {
        c0 += w;
        s = __fadd_rn(s, rec[c0]);
      }
      const int h = w >= 2 * d + 1 ? mv * (2 * d + 1) : (mv - 1) * w + 2 * d + 1;
      c = N - h;
      if (c > 0) {
        const int t = (c - 1) / 2 - (lo_r - my_below);
        const uint32_t freeb = ~(my_mask | outside);
        pos0 = t >= 0 ? nth_set_bit(freeb, t) : -1;
        if (pos0 < 0) {
          pos0 = 0;
          bad = true;
        }
        const uint32_t rest = pos0 >= 31 ? 0u : (freeb & (0xFFFFFFFEu << pos0));
        pos1 = (c & 1) ? pos0 : __ffs(rest) - 1;
        if (pos1 < 0) {
          pos1 = 0;
          bad = true;
        }
      }
    }
    const float v0 = __shfl_sync(0xffffffffu, bv, pos0);
    const float v1 = __shfl_sync(0xffffffffu, bv, pos1);
    if (ok && c > 0) {
      const float B = (c & 1) ? v0 : __fmul_rn(__fadd_rn(v0, v1), 0.5f);
      const float snr = snr_of(comb_nw(s, mv), B);
      if (bestw < 0 || snr > best || (snr == best && w < bestw)) {
        best = snr;
        bestw = w;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int ow = __shfl_xor_sync(0xffffffffu, bestw, o);
    if (ow >= 0 && (bestw < 0 || ob > best || (ob == best && ow < bestw))) {
      best = ob;
      bestw = ow;
    }
  }
  out.bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
  out.snr = bestw >= 0 ? best : 0.f;
  out.w = bestw;
  out.rotor = (bestw >= 0 && best >= cc.tau_comb) ? 1 : 0;
  __syncwarp();
  return out;
}

// Which comb variant a context uses: 0 = fast (N <= 1024, band <= 32),
// otherwise the generic one with NW mask words per centre.
__host__ __device__ inline int comb_variant(const CombConst &cc) {
  if (cc.N <= CombFast::kMaxN && cc.bw <= CombFast::kMaxBand && cc.M * (2 * cc.d + 1) <= 32)
    return 0;
  return cc.bw <= 32 ? 1 : 8;
}

__host__ __device__ inline int comb_scratch_bytes(int N, int variant) {
  return variant == 0 ? CombFast::bytes(N) : CombScratch::bytes(N, variant);
}

// Eq. 7-11 for one pixel's spectrum Pw[0..N) in shared memory by the calling
// warp; scratch: comb_scratch_bytes(N, NW) bytes (16-byte aligned).
template <int NW>
__device__ __forceinline__ CombOut comb_warp(const float *Pw, const CombConst &cc,
                                             unsigned char *scratch) {
  if constexpr (NW == 0) return comb_warp_fast(Pw, cc, scratch);
  else return comb_warp_generic<NW>(Pw, cc, scratch);
}

}  // namespace ddhf
