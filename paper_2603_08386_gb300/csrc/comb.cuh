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

__device__ __forceinline__ float snr_of(float nw, float B) {
  return B > 0.f ? __fdiv_rn(nw, B) : (nw > 0.f ? __int_as_float(0x7f800000) : 0.f);
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
    slog = __fadd_rn(slog, __logf(fmaxf(v, 1e-30f)));
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
//  * 2048 linear buckets over [0, 2 mean), two 16-bit counts per word, are
//    filled in the same pass as the log sum of Eq. 7;
//  * the buckets holding ranks lo_r and hi_r bound the candidate set; one pass
//    extracts the candidates and writes the prefix count of bins in lower
//    buckets (the "below" prefix), so the band is extended downwards to the
//    first candidate: band position p = full rank cb + p, cb = bins in lower
//    buckets, and the band covers full ranks [cb, hi_r] (at most 32);
//  * candidates are sorted in registers as 32-bit keys (value bits relative
//    to the smallest candidate, above the 10-bit bin index);
//  * per window centre one float2 record {window maximum, band mask};
//  * the complement median is picked from the band values by a shuffle.
// Pixels whose candidates do not fit (more than 64, band wider than 32, or
// value range above 2^22 ulps) take an exact radix selection of the band
// [lo_r, hi_r] instead, with the same record layout.
// Scratch layout (bytes from the scratch base, 16-byte aligned):
//   [0, R)   R = max(8N, 4096): histogram u32[1024] during selection, then the
//            candidate values u32[64] and indices u16[64] (and the fallback's
//            radix histogram and keys), then the window records float2[N]
//   [R, R + 2(N+1))  below prefix u16[N+1]
struct CombFast {
  __host__ __device__ static int rec_bytes(int N) { return 8 * N > 4096 ? 8 * N : 4096; }
  __host__ __device__ static int preb_off(int N) { return (rec_bytes(N) + 15) & ~15; }
  __host__ __device__ static int bytes(int N) { return preb_off(N) + ((2 * (N + 1) + 15) & ~15); }
  static constexpr int kMaxN = 1024;
  static constexpr int kMaxBand = 32;
};

__device__ __forceinline__ int bucket2048(float v, float scale) {
  return (int)fminf(__fmul_rn(v, scale), 2047.f);
}

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

__device__ __forceinline__ CombOut comb_warp_fast(const float *Pw, const CombConst &cc,
                                                  unsigned char *scratch) {
  const int lane = threadIdx.x & 31;
  const int N = cc.N;
  const uint32_t lt = lanemask_lt();
  uint32_t *hist = reinterpret_cast<uint32_t *>(scratch);
  uint16_t *preb = reinterpret_cast<uint16_t *>(scratch + CombFast::preb_off(N));
  CombOut out;
  out.snr = 0.f;
  out.w = -1;
  out.rotor = 0;
  out.bad = 0;
  bool bad = false;

  // ---- Eq. 7 sums (fixed order: lane-strided, then a butterfly) + histogram
#pragma unroll
  for (int q = 0; q < 8; ++q)
    reinterpret_cast<uint4 *>(hist)[q * 32 + lane] = make_uint4(0u, 0u, 0u, 0u);
  float sum = 0.f;
#pragma unroll 4
  for (int j = lane; j < N; j += 32) sum = __fadd_rn(sum, Pw[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, o));
  const float fN = (float)N;
  const float scale = __fdiv_rn(1024.f, __fdiv_rn(sum, fN));
  __syncwarp();
  float slog = 0.f;
#pragma unroll 4
  for (int j = lane; j < N; j += 32) {
    const float v = Pw[j];
    slog = __fadd_rn(slog, __logf(fmaxf(v, 1e-30f)));
    const int g = bucket2048(v, scale);
    atomicAdd(&hist[g >> 1], 1u << ((g & 1) << 4));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) slog = __fadd_rn(slog, __shfl_xor_sync(0xffffffffu, slog, o));
  out.log_sf = sum > 0.f ? __fsub_rn(__fdiv_rn(slog, fN), __logf(__fdiv_rn(sum, fN))) : 0.f;
  if (!(out.log_sf <= cc.ln_tau_sf) || cc.w_hi < cc.w_lo) return out;
  __syncwarp();

  // ---- buckets of ranks lo_r and hi_r. Lane l owns words [32 l, 32 l + 32)
  // (buckets [64 l, 64 l + 64)); both 16-bit halves are summed in one word.
  const int lo_r = cc.lo_r, hi_r = cc.lo_r + cc.bw - 1;
  uint32_t acc = 0;
  {
    const uint4 *h4 = reinterpret_cast<const uint4 *>(hist) + lane * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 t = h4[(q + lane) & 7];  // rotated: no bank conflicts
      acc += t.x + t.y + t.z + t.w;
    }
  }
  const uint32_t lsum = (acc & 0xFFFFu) + (acc >> 16);
  uint32_t tot;
  const uint32_t lex = warp_excl_scan<uint32_t>(lsum, tot);
  if (tot != (uint32_t)N) bad = true;
  int gb[2];
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
    const uint32_t wv = hist[src * 32 + lane];
    const uint32_t c0 = wv & 0xFFFFu, c1 = wv >> 16;
    uint32_t t2;
    const uint32_t ex = warp_excl_scan<uint32_t>(c0 + c1, t2) + base;
    const bool own = R >= ex && R < ex + c0 + c1;
    int s2 = __ffs(__ballot_sync(0xffffffffu, own)) - 1;
    if (s2 < 0) {
      s2 = 0;
      bad = true;
    }
    const bool first = R < ex + c0;  // meaningful in lane s2
    const uint32_t gsel = (uint32_t)(src * 64 + 2 * lane) + (first ? 0u : 1u);
    const uint32_t gbl = first ? ex : ex + c0;
    const uint32_t gct = first ? c0 : c1;
    gb[t] = (int)__shfl_sync(0xffffffffu, gsel, s2);
    gbelow[t] = __shfl_sync(0xffffffffu, gbl, s2);
    gcount[t] = __shfl_sync(0xffffffffu, gct, s2);
  }
  int cb = (int)gbelow[0];
  const int ncand = (int)(gbelow[1] + gcount[1]) - cb;
  int bwe = hi_r - cb + 1;  // band positions: full ranks [cb, hi_r]
  bool slow = ncand > 64 || bwe > CombFast::kMaxBand || bad;
  __syncwarp();

  // ---- candidates (bins of buckets gb[0]..gb[1]) and the below prefix
  uint32_t *cv = hist;                                         // u32[64]
  uint16_t *cj = reinterpret_cast<uint16_t *>(scratch + 256);  // u16[64]
  float bv = 0.f;  // band value at position lane (lane < bwe)
  int bj = 0;      // its bin
  if (!slow) {
    const int g0 = gb[0];
    const uint32_t gspan = (uint32_t)(gb[1] - gb[0]);
    uint32_t run = 0, runb = 0;
    for (int j0 = 0; j0 <= N; j0 += 32) {
      const int j = j0 + lane;
      const float v = j < N ? Pw[j] : 0.f;
      const int g = bucket2048(v, scale);
      const bool in = j < N && (uint32_t)(g - g0) <= gspan;
      const bool below = j < N && g < g0;
      const uint32_t bi = __ballot_sync(0xffffffffu, in);
      const uint32_t bb = __ballot_sync(0xffffffffu, below);
      if (in) {
        const uint32_t slot = run + __popc(bi & lt);
        if (slot < 64) {
          cv[slot] = __float_as_uint(v);
          cj[slot] = (uint16_t)j;
        }
      }
      if (j <= N) preb[j] = (uint16_t)(runb + __popc(bb & lt));
      run += __popc(bi);
      runb += __popc(bb);
    }
    if ((int)run != ncand || (int)runb != cb) bad = true;
    __syncwarp();
    const bool in0 = lane < ncand, in1 = lane + 32 < ncand;
    const uint32_t b0 = in0 ? cv[lane] : 0xFFFFFFFFu;
    const uint32_t b1 = in1 ? cv[lane + 32] : 0xFFFFFFFFu;
    const uint32_t j0v = in0 ? cj[lane] : 0u;
    const uint32_t j1v = in1 ? cj[lane + 32] : 0u;
    const uint32_t mn = __reduce_min_sync(0xffffffffu, min(b0, b1));
    const uint32_t mx = __reduce_max_sync(0xffffffffu, max(in0 ? b0 : 0u, in1 ? b1 : 0u));
    if (mx - mn >= (1u << 22)) {
      slow = true;
    } else {
      uint32_t k0 = in0 ? (((b0 - mn) << 10) | j0v) : 0xFFFFFFFFu;
      uint32_t k1 = in1 ? (((b1 - mn) << 10) | j1v) : 0xFFFFFFFFu;
      if (ncand <= 32) {
        k0 = warp_sort32_u32(k0);
      } else {
        warp_sort64_u32(k0, k1);
      }
      bv = __uint_as_float((k0 >> 10) + mn);
      bj = (int)(k0 & 1023u);
    }
    __syncwarp();
  }
  if (slow) {
    // exact band [lo_r, hi_r] by radix selection; prefix of bins below it
    uint32_t *h256 = hist;
    const uint64_t klo = select_rank_slow(Pw, N, lo_r, h256);
    const uint64_t khi = select_rank_slow(Pw, N, hi_r, h256);
    uint64_t key = ~0ull;
    uint32_t run = 0, runb = 0;
    for (int j0 = 0; j0 <= N; j0 += 32) {
      const int j = j0 + lane;
      const uint64_t k = j < N ? bin_key(Pw, j) : ~0ull;
      const bool in = j < N && k >= klo && k <= khi;
      const bool below = j < N && k < klo;
      const uint32_t bi = __ballot_sync(0xffffffffu, in);
      const uint32_t bb = __ballot_sync(0xffffffffu, below);
      const uint32_t slot = run + __popc(bi & lt);
      // one band key per lane: lane `slot` receives it
#pragma unroll 1
      for (uint32_t m = bi; m; m &= m - 1) {
        const int srcl = __ffs(m) - 1;
        const uint64_t kk = __shfl_sync(0xffffffffu, k, srcl);
        const uint32_t sl = __shfl_sync(0xffffffffu, slot, srcl);
        if ((uint32_t)lane == sl) key = kk;
      }
      if (j <= N) preb[j] = (uint16_t)(runb + __popc(bb & lt));
      run += __popc(bi);
      runb += __popc(bb);
    }
    if ((int)run != cc.bw) bad = true;
    key = warp_sort32_u64(key);
    bv = __uint_as_float((uint32_t)(key >> 16));
    bj = (int)(key & 0xFFFFu);
    cb = lo_r;
    bwe = cc.bw;
    __syncwarp();
  }

  // ---- window records {max of P over [c - d, c + d], band mask of the window}
  const int d = cc.d;
  float2 *rec = reinterpret_cast<float2 *>(scratch);
  if (d == 3) {
    // centre pairs (2q, 2q + 1): bins 2q - 4 .. 2q + 5 by five 8-byte loads
    const float2 *P2 = reinterpret_cast<const float2 *>(Pw);
    const int npair = (N + 1) >> 1;
    for (int q = lane; q < npair; q += 32) {
      float2 a[5];
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        const int pi = q - 2 + u;  // pair index of bins 2 pi, 2 pi + 1
        if (pi >= 0 && 2 * pi + 1 < N) a[u] = P2[pi];
        else a[u] = make_float2(pi >= 0 && 2 * pi < N ? Pw[2 * pi] : 0.f, 0.f);
      }
      // bins: a[0] = (2q-4, 2q-3), a[1] = (2q-2, 2q-1), a[2] = (2q, 2q+1),
      //       a[3] = (2q+2, 2q+3), a[4] = (2q+4, 2q+5)
      const float mid = fmaxf(fmaxf(fmaxf(a[1].x, a[1].y), fmaxf(a[2].x, a[2].y)),
                              fmaxf(a[3].x, a[3].y));  // 2q-2 .. 2q+3
      const float w0 = fmaxf(mid, a[0].y);             // 2q-3 .. 2q+3
      const float w1 = fmaxf(mid, a[4].x);             // 2q-2 .. 2q+4
      if (2 * q + 1 < N) {
        reinterpret_cast<float4 *>(rec)[q] = make_float4(w0, 0.f, w1, 0.f);
      } else {
        rec[2 * q] = make_float2(w0, 0.f);
      }
    }
  } else {
    for (int c = lane; c < N; c += 32) {
      float mx = 0.f;
      if (c >= d && c <= N - 1 - d) {
        mx = Pw[c - d];
        for (int i = 1; i <= 2 * d; ++i) mx = fmaxf(mx, Pw[c - d + i]);
      }
      rec[c] = make_float2(mx, 0.f);
    }
  }
  __syncwarp();
  if (lane < bwe) {
    uint32_t *recw = reinterpret_cast<uint32_t *>(rec);
    const int c_lo = max(0, bj - d), c_hi = min(N - 1, bj + d);
    for (int c = c_lo; c <= c_hi; ++c) atomicOr(&recw[2 * c + 1], 1u << lane);
  }
  __syncwarp();

  // ---- Eq. 8-10 for every candidate fundamental, one per lane
  const uint32_t outside = bwe >= 32 ? 0u : (0xFFFFFFFFu << bwe);
  float best = 0.f;
  int bestw = -1;
  const int L = N - 1 - d;
  for (int w0 = cc.w_lo; w0 <= cc.w_hi; w0 += 32) {
    const int w = w0 + lane;
    const bool ok = w <= cc.w_hi;
    int pos0 = 0, pos1 = 0, c = 0, mv = 1;
    float s = 0.f;
    if (ok) {
      mv = cc.M;
      while (mv * w > L) --mv;
      uint32_t mask = outside;
      int below = 0, cc0 = 0;
#pragma unroll 4
      for (int m = 1; m <= mv; ++m) {
        cc0 += w;
        const float2 r = rec[cc0];
        s = __fadd_rn(s, r.x);
        mask |= __float_as_uint(r.y);
        below += (int)preb[cc0 + d + 1] - (int)preb[cc0 - d];
      }
      int h;
      if (w >= 2 * d + 1) {
        h = mv * (2 * d + 1);
      } else {  // overlapping windows: their union is one contiguous range
        h = (mv - 1) * w + 2 * d + 1;
        below = (int)preb[mv * w + d + 1] - (int)preb[w - d];
      }
      c = N - h;
      if (c > 0) {
        const int t = (c - 1) / 2 - (cb - below);
        const uint32_t freeb = ~mask;
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
      const float nw = ((mv & (mv - 1)) == 0) ? __fmul_rn(s, 1.0f / (float)mv)
                                              : __fdiv_rn(s, (float)mv);
      const float B = (c & 1) ? v0 : __fmul_rn(__fadd_rn(v0, v1), 0.5f);
      const float snr = snr_of(nw, B);
      if (bestw < 0 || snr > best) {
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
__host__ __device__ inline int comb_variant(int N, int bw) {
  if (N <= CombFast::kMaxN && bw <= CombFast::kMaxBand) return 0;
  return bw <= 32 ? 1 : 8;
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
