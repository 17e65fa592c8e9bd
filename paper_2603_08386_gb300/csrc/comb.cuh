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
//   [2048, 6144)    selection histogram (u32[1024]); later window maxima f32[N]
//   [6144, 6656)    selection candidates (u64[64])
//   after wmax      below-band ballot words and their prefix counts (u32 each)
struct CombScratch {
  static constexpr int kBand = 0;
  static constexpr int kHist = 2048;
  static constexpr int kCand = 6144;
  static constexpr int kSelEnd = 6656;
  static constexpr int kPhase2 = 2048;
  // ballot words cover bins 0..N inclusive (a count "below bin N" is a query)
  __host__ __device__ static int words(int N) { return N / 32 + 1; }
  __host__ __device__ static int bytes(int N, int) {
    int p2 = kPhase2 + 4 * N + 8 * words(N);
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
__device__ __forceinline__ void warp_sort64_regs(uint64_t (&v)[2]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {
        if (v[0] > v[1]) {  // k = 64: the whole sequence ascends
          uint64_t t = v[0];
          v[0] = v[1];
          v[1] = t;
        }
      } else {
#pragma unroll
        for (int sidx = 0; sidx < 2; ++sidx) {
          const int i = lane + 32 * sidx;
          const uint64_t o = __shfl_xor_sync(0xffffffffu, v[sidx], j);
          const bool up = (i & k) == 0;
          const bool lower = (i & j) == 0;
          const uint64_t mn = v[sidx] < o ? v[sidx] : o;
          const uint64_t mx = v[sidx] < o ? o : v[sidx];
          v[sidx] = (lower == up) ? mn : mx;
        }
      }
    }
  }
}

// Mean-scaled linear bucket of a power value (monotone in the value).
__device__ __forceinline__ int lin_bucket(float v, float scale) {
  return (int)fminf(__fmul_rn(v, scale), 1023.f);
}

// Number of bins j' < j below the band (from the ballot words and their prefix).
__device__ __forceinline__ int below_before(const uint32_t *bwords, const uint32_t *bbase, int j) {
  const int w = j >> 5, b = j & 31;
  return (int)bbase[w] + __popc(bwords[w] & ((1u << b) - 1u));
}

// Eq. 8 numerator sum and its division by M_valid, in the fixed FP32 order.
__device__ __forceinline__ float comb_nw(const float *wmax, int w, int mv) {
  float s = 0.f;
  for (int m = 1; m <= mv; ++m) s = __fadd_rn(s, wmax[m * w]);
  if ((mv & (mv - 1)) == 0) return __fmul_rn(s, 1.0f / (float)mv);  // exact: power of two
  return __fdiv_rn(s, (float)mv);
}

__device__ __forceinline__ float snr_of(float nw, float B) {
  return B > 0.f ? __fdiv_rn(nw, B) : (nw > 0.f ? __int_as_float(0x7f800000) : 0.f);
}

// Eq. 7-11 for the spectrum Pw[0..N) (shared memory) by the calling warp.
// scratch: CombScratch::bytes(N, NW) bytes of shared memory (16-byte aligned).
template <int NW>
__device__ CombOut comb_warp(const float *Pw, const CombConst &cc, unsigned char *scratch) {
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
#pragma unroll
  for (int q = 0; q < 32; ++q) hist[q * 32 + lane] = 0;
  __syncwarp();
  for (int j = lane; j < N; j += 32) atomicAdd(&hist[lin_bucket(Pw[j], scale)], 1u);
  __syncwarp();
  uint32_t lsum = 0;
#pragma unroll 8
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
    warp_sort64_regs(v2);
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
  const float v_lo = bandv[0], v_hi = bandv[bw - 1];
  const uint64_t key_lo = ((uint64_t)__float_as_uint(v_lo) << 16) | (uint32_t)bandj[0];

  // ---- window maxima, below-band ballot words
  const int d = cc.d;
  float *wmax = reinterpret_cast<float *>(scratch + CombScratch::kPhase2);
  uint32_t *bwords = reinterpret_cast<uint32_t *>(scratch + CombScratch::kPhase2 + 4 * N);
  uint32_t *bbase = bwords + CombScratch::words(N);
  for (int c = d + lane; c <= N - 1 - d; c += 32) {
    float mx = Pw[c - d];
    for (int i = 1; i <= 2 * d; ++i) mx = fmaxf(mx, Pw[c - d + i]);
    wmax[c] = mx;
  }
  {
    uint32_t run = 0;
    const int nwd = CombScratch::words(N);
    for (int w = 0; w < nwd; ++w) {
      const int j = w * 32 + lane;
      const bool below = j < N && bin_key(Pw, j) < key_lo;
      const uint32_t b = __ballot_sync(0xffffffffu, below);
      if (lane == 0) {
        bwords[w] = b;
        bbase[w] = run;
      }
      run += __popc(b);
    }
  }
  __syncwarp();

  // ---- Eq. 8 for every candidate, then the exact Eq. 9-10 only where the
  // bounds v_lo <= B(w) <= v_hi leave w a chance to be the maximum.
  float nmax = 0.f;
  for (int w = cc.w_lo + lane; w <= cc.w_hi; w += 32) {
    const int mv = min(cc.M, (N - 1 - d) / w);
    nmax = fmaxf(nmax, comb_nw(wmax, w, mv));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
  const float lb_max = snr_of(nmax, v_hi);
  const float pre = (v_lo > 0.f && v_hi > 0.f) ? __fmul_rn(__fdiv_rn(v_lo, v_hi), 0.999f) : 0.f;
  float best = -1.f;
  int bestw = -1;
  for (int w0 = cc.w_lo; w0 <= cc.w_hi; w0 += 32) {
    const int wl = w0 + lane;
    float nwl = 0.f;
    bool surv = false;
    if (wl <= cc.w_hi) {
      const int mv = min(cc.M, (N - 1 - d) / wl);
      nwl = comb_nw(wmax, wl, mv);
      if (nwl >= __fmul_rn(nmax, pre)) surv = !(snr_of(nwl, v_lo) < lb_max);
    }
    uint32_t sb = __ballot_sync(0xffffffffu, surv);
    while (sb) {
      const int src = __ffs(sb) - 1;
      sb &= sb - 1;
      const int w = w0 + src;
      const float nw = __shfl_sync(0xffffffffu, nwl, src);
      const int mv = min(cc.M, (N - 1 - d) / w);
      int h, below;
      if (w >= 2 * d + 1) {
        h = mv * (2 * d + 1);
        int bl = 0;
        for (int m = lane + 1; m <= mv; m += 32) {
          const int c = m * w;
          bl += below_before(bwords, bbase, c + d + 1) - below_before(bwords, bbase, c - d);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bl += __shfl_xor_sync(0xffffffffu, bl, o);
        below = bl;
      } else {
        h = (mv - 1) * w + 2 * d + 1;
        below = below_before(bwords, bbase, mv * w + d + 1) - below_before(bwords, bbase, w - d);
      }
      const int c = N - h;
      if (c <= 0) continue;
      uint32_t mask[NW];
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        const int b = q * 32 + lane;
        bool inside = false;
        if (b < bw) {
          const int jb = bandj[b];
          if (w >= 2 * d + 1) {
            const int m = (jb + d) / w;
            inside = m >= 1 && m <= mv && jb + d - m * w <= 2 * d;
          } else {
            inside = jb >= w - d && jb <= mv * w + d;
          }
        }
        mask[q] = __ballot_sync(0xffffffffu, inside);
      }
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
  }
  if (bestw < 0) bad = true;  // the maximiser always survives the bounds
  out.bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
  out.snr = bestw >= 0 ? best : 0.f;
  out.w = bestw;
  out.rotor = (bestw >= 0 && best >= cc.tau_comb) ? 1 : 0;
  __syncwarp();
  return out;
}

}  // namespace ddhf
