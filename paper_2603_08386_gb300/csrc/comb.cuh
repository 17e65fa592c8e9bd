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
  return (int)fminf(fmaxf(__fmul_rn(v, scale), 0.f), 1023.f);
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

// Approximate reciprocal (PTX rcp.approx, flush-to-zero form).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Base-2 logarithm of a normal float (PTX lg2.approx, flush-to-zero form).
__device__ __forceinline__ float lg2_normal(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
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
// Fast variants for N <= 1024 bins, a median band of at most 32 ranks and at
// most 32 bins in a candidate's harmonic windows (M (2d+1) <= 32).
//
// Same results as comb_warp_generic, bit for bit, with far fewer
// instructions per pixel:
//  * the log sum of Eq. 7 (base 2, scaled by ln 2 once) shares its pass with
//    a histogram of 768 buckets linear in P over [0, 1.5 mean) (values above
//    go to the last);
//  * the buckets holding ranks lo_r and hi_r bound the candidate bins; at
//    most 64 candidates (about 31 on C3's spectra) are compacted into shared
//    memory and sorted in registers as 32-bit keys (value bits relative to
//    the smallest candidate, above the 10-bit bin index), so that lane p
//    holds the bin of full rank lo_r + p;
//  * one window maximum per centre (Eq. 8), then N(w) for every candidate,
//    kept in shared memory;
//  * candidates are evaluated one at a time by the whole warp: lane i <
//    |H(w)| tests bin i of H(w) against the band start (bins below the band),
//    lane p < bw tests whether the band's p-th bin lies in H(w); two ballots
//    then locate the complement's middle ranks in the band, and SNR = N(w) /
//    B by a correctly rounded division. The candidate with the largest N(w)
//    goes first: its SNR bounds the best one from below, and since every
//    complement median is at least the band start T, a candidate with
//    N(w) / T below that bound can neither win nor tie (on C3's spectra
//    fewer than two candidates per pixel are evaluated on average); the rest
//    follow in increasing w.
// Two forms share these steps. The register form (512 < N <= 768, M = 4,
// d = 3: Table 2's comb on the 750-bin grid) gives each lane 24 consecutive
// bins in registers, so every per-bin pass is a fixed, fully unrolled
// sequence and the window maxima come from registers and six shuffles. The
// shared-memory form takes any other size within the limits.
// Pixels whose candidates do not fit (more than 64, or a value range above
// 2^22 ulps) take an exact radix selection of the band instead.
// Scratch (bytes from the scratch base, 16-byte aligned):
//   [0, 3072)   histogram u32[768]; once the band's buckets are located, over
//               it: candidate value bits u32[64] at 0 and their bins u16[64]
//               at 256; once the band is in registers: N(w) of candidate
//               w_lo + i, f32[n_cand] (-1: complement empty), when it fits
//   [3072, +16 ceil(N/4))  window maxima f32[N]
//   then N(w), when it does not fit over the histogram
struct CombFast {
  static constexpr int kBuckets = 768;
  static constexpr int kHist = 0;
  static constexpr int kHistBytes = 3072;
  static constexpr int kCandV = 0;
  static constexpr int kCandJ = 256;
  static constexpr int kRec = 3072;
  __host__ __device__ static int rec_end(int N) { return kRec + ((4 * N + 15) & ~15); }
  __host__ __device__ static int nw_off(int N, int n_cand) {
    return 4 * n_cand <= kHistBytes ? 0 : rec_end(N);
  }
  __host__ __device__ static int bytes(int N, int n_cand) {
    const int nc = n_cand > 0 ? n_cand : 0;
    const int e = nw_off(N, nc) + 4 * nc;
    return ((e > rec_end(N) ? e : rec_end(N)) + 15) & ~15;
  }
  static constexpr int kMaxN = 1024;
  static constexpr int kMaxBand = 32;
  static constexpr int kMaxCand = 64;
};

// The register form's shape: bins per lane, and the comb it is written for.
struct CombReg {
  static constexpr int kBPL = 24;
  static constexpr int kM = 4;
  static constexpr int kD = 3;
  // every candidate then has all M windows and a non-empty complement
  __host__ __device__ static bool fits(const CombConst &cc) {
    return cc.N > 16 * kBPL && cc.N <= 32 * kBPL && cc.M == kM && cc.d == kD &&
           kM * cc.w_hi <= cc.N - 1 - kD && cc.N > kM * (2 * kD + 1) &&
           cc.w_hi - cc.w_lo + 1 <= 256;
  }
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

// Window maxima rec[c] = max of P over [c - d, c + d] for any half-width d;
// out of line (the d = 3 case has inline versions).
__device__ __noinline__ static void comb_records_any_d(const float *Pw, int N, int d,
                                                       float *rec) {
  const int lane = threadIdx.x & 31;
  for (int c = d + lane; c <= N - 1 - d; c += 32) {
    float mx = Pw[c - d];
    for (int i = 1; i <= 2 * d; ++i) mx = fmaxf(mx, Pw[c - d + i]);
    rec[c] = mx;
  }
}

// 768 linear buckets over [0, 1.5 mean) (the fast forms' histogram, with
// scale = 512 / mean): x = v scale clamped to at most 767, bucket floor(x),
// taken by adding 2^23 rounded down (the float bits then hold floor(x) in the
// low mantissa bits), so no float-to-integer conversion runs on the
// special-function pipe. Monotone in v >= 0, so the bins of a bucket range
// are a range of full ranks, and bucket g0 <= g <= g1 exactly when g0 <= x <
// g1 + 1. Any input (a negative value, NaN) still gives an index in [0, 1023]
// (a histogram word index below 512: inside the scratch).
__device__ __forceinline__ float bucket_x(float v, float scale) {
  return fminf(__fmul_rn(v, scale), 767.f);
}
__device__ __forceinline__ uint32_t bucket_bits(float v, float scale) {
  return __float_as_uint(__fadd_rd(bucket_x(v, scale), 0x1p23f));  // 0x4B000000 + g
}
__device__ __forceinline__ int bucket_of(float v, float scale) {
  return (int)(bucket_bits(v, scale) & 1023u);
}

// Add one to the bucket whose bucket_bits are ybits in the histogram at
// shared address hist_sa (one counter per bucket).
__device__ __forceinline__ void hist_add(uint32_t hist_sa, uint32_t ybits) {
  const uint32_t a = hist_sa + ((ybits & 1023u) << 2);
  asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a) : "memory");
}

// M_valid(w) = #{m <= M : m w + d <= N - 1}, the in-band harmonics (a prefix).
__device__ __forceinline__ int comb_mvalid(int w, int M, int L) {
  int mv = M;
  while (mv > 0 && mv * w > L) --mv;
  return mv;
}

// N(w) of Eq. 8 from the window maxima, or -1 when w's complement is empty
// (KM, KD: the comb's M and d when known at compile time, else 0).
template <int KM, int KD>
__device__ __forceinline__ float comb_cand_nw(const float *rec, int w, const CombConst &cc,
                                              bool uniform) {
  const int M = KM ? KM : cc.M, d = KD ? KD : cc.d, N = cc.N;
  const int L = N - 1 - d;
  const int mv = uniform ? M : comb_mvalid(w, M, L);
  const int h = w >= 2 * d + 1 ? mv * (2 * d + 1) : (mv - 1) * w + 2 * d + 1;
  if (N - h <= 0) return -1.f;
  float s = rec[w];  // 0 + m_1, exact
  if (KM && uniform) {
#pragma unroll
    for (int m = 2; m <= KM; ++m) s = __fadd_rn(s, rec[m * w]);
    return comb_nw(s, KM);
  }
#pragma unroll 4
  for (int m = 2; m <= mv; ++m) s = __fadd_rn(s, rec[m * w]);
  return comb_nw(s, mv);
}

// The buckets holding full ranks lo_r and hi_r in the histogram; lane l owns
// buckets [24 l, 24 l + 24). Returns the first and last candidate bucket, the
// bins below the first (cb) and the candidate count.
struct BandBuckets {
  int g0, g1, cb, ncand;
};
__device__ __forceinline__ BandBuckets comb_locate(const uint32_t *hist, int N, int lo_r,
                                                   int hi_r, bool &bad) {
  const int lane = threadIdx.x & 31;
  uint32_t lsum;
  {
    const uint4 *h4 = reinterpret_cast<const uint4 *>(hist) + lane * 6;
    uint32_t s2 = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const uint4 t = h4[(q + (lane >> 2)) % 6];  // rotated: no bank conflicts
      s2 += t.x + t.y + t.z + t.w;
    }
    lsum = s2;
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
    const uint32_t h = lane < 24 ? hist[src * 24 + lane] : 0u;
    uint32_t t2;
    const uint32_t ex = warp_excl_scan<uint32_t>(h, t2) + base;
    int s2 = __ffs(__ballot_sync(0xffffffffu, R >= ex && R < ex + h)) - 1;
    if (s2 < 0) {
      s2 = 0;
      bad = true;
    }
    gsel[t] = src * 24 + s2;
    gbelow[t] = __shfl_sync(0xffffffffu, ex, s2);
    gcount[t] = __shfl_sync(0xffffffffu, h, s2);
  }
  BandBuckets r;
  r.g0 = gsel[0];
  r.g1 = gsel[1];
  r.cb = (int)gbelow[0];
  r.ncand = (int)(gbelow[1] + gcount[1]) - r.cb;
  return r;
}

// The band from the ncand <= 64 compacted candidates (value bits cv, bins
// cj; element i in lane i % 32, register i / 32): sorted as 32-bit keys,
// lane p < bw takes full rank lo_r + p (value bv, bin bj). Returns false
// (warp-uniform) when the values span 2^22 ulps or more, so that the exact
// selection must run instead.
__device__ __forceinline__ bool comb_band_sorted(const unsigned char *scratch, int ncand,
                                                 int lo_r, int cb, int bw, float &bv, int &bj,
                                                 bool &bad) {
  const int lane = threadIdx.x & 31;
  const uint32_t *cv = reinterpret_cast<const uint32_t *>(scratch + CombFast::kCandV);
  const uint16_t *cj = reinterpret_cast<const uint16_t *>(scratch + CombFast::kCandJ);
  const bool in0 = lane < ncand, in1 = lane + 32 < ncand;
  const uint32_t b0 = in0 ? cv[lane] : 0xFFFFFFFFu;
  const uint32_t b1 = in1 ? cv[lane + 32] : 0xFFFFFFFFu;
  const uint32_t mn = __reduce_min_sync(0xffffffffu, min(b0, b1));
  const uint32_t mx = __reduce_max_sync(0xffffffffu, max(in0 ? b0 : 0u, in1 ? b1 : 0u));
  if (mx - mn >= (1u << 22)) return false;
  uint32_t k0 = in0 ? (((b0 - mn) << 10) | (uint32_t)cj[lane]) : 0xFFFFFFFFu;
  uint32_t k1 = in1 ? (((b1 - mn) << 10) | (uint32_t)cj[lane + 32]) : 0xFFFFFFFFu;
  if (ncand <= 32) k0 = warp_sort32_u32(k0);
  else warp_sort64_u32(k0, k1);
  // band position p is sorted element i = lo_r - cb + p (lane i % 32, register i / 32)
  const int i = lo_r - cb + lane;
  const uint32_t kk0 = __shfl_sync(0xffffffffu, k0, i & 31);
  const uint32_t kk1 = __shfl_sync(0xffffffffu, k1, i & 31);
  const uint32_t kk = i < 32 ? kk0 : kk1;
  if (lane < bw && (i < 0 || i >= ncand)) bad = true;
  bv = __uint_as_float((kk >> 10) + mn);
  bj = (int)(kk & 1023u);
  return true;
}

// N(w) of every candidate into nws[], the largest and its candidate index
// (the first of equal maxima; -1 / INT_MAX when every complement is empty).
// KM, KD > 0 (the register form): the comb's M and d, with every candidate
// known to have all M windows and a non-empty complement (CombReg::fits).
template <int KM, int KD>
__device__ __forceinline__ void comb_nw_all(const float *rec, float *nws, const CombConst &cc,
                                            bool uniform, float &maxnw, int &maxi) {
  const int lane = threadIdx.x & 31;
  const int n_cand = cc.w_hi - cc.w_lo + 1;
  maxnw = -1.f;
  maxi = 0x7fffffff;
  if (KM) {
    // every candidate has all KM windows and a non-empty complement: N(w) is
    // a plain sum of KM window maxima
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
      const int i = lane + 32 * k;
      if (32 * k >= n_cand) break;
      if (i < n_cand) {
        const int w = cc.w_lo + i;
        float sm = rec[w];
#pragma unroll
        for (int m = 2; m <= KM; ++m) sm = __fadd_rn(sm, rec[m * w]);
        const float nw = comb_nw(sm, KM);
        nws[i] = nw;
        if (nw > maxnw) {
          maxnw = nw;
          maxi = i;
        }
      }
    }
  } else {
    for (int i = lane; i < n_cand; i += 32) {
      const float nw = comb_cand_nw<0, 0>(rec, cc.w_lo + i, cc, uniform);
      nws[i] = nw;
      if (nw > maxnw) {
        maxnw = nw;
        maxi = i;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float on = __shfl_xor_sync(0xffffffffu, maxnw, o);
    const int oi = __shfl_xor_sync(0xffffffffu, maxi, o);
    if (on > maxnw || (on == maxnw && oi < maxi)) {
      maxnw = on;
      maxi = oi;
    }
  }
}

// Eq. 9-10 for the candidates, each by the whole warp: the one with the
// largest N(w) first, then, in increasing w, those that the first one's SNR
// does not rule out (see the description above). Lane i of a disjoint H(w)
// (w >= 2d + 1) takes bin (1 + i / (2d+1)) w + i % (2d+1) - d; of an
// overlapping one, bin w - d + i. Band lane p's bin lies in H(w) when it is
// within d of m w for some m <= M_valid. bv, bj: the band value and bin of
// lane p. KM, KD as for comb_cand_nw.
template <int KM, int KD>
__device__ __forceinline__ void comb_best(const float *Pw, const float *nws, const CombConst &cc,
                                          bool uniform, float maxnw, int maxi, float bv, int bj,
                                          float &best, int &bestw, bool &bad) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const int N = cc.N, M = KM ? KM : cc.M, d = KD ? KD : cc.d, lo_r = cc.lo_r, bw = cc.bw;
  const int n_cand = cc.w_hi - cc.w_lo + 1;
  const float T = __shfl_sync(0xffffffffu, bv, 0);  // band start (T, tj)
  const int tj = __shfl_sync(0xffffffffu, bj, 0);
  const int span = 2 * d + 1;
  const int lane_m = 1 + lane / span, lane_o = lane % span - d;
  const bool band_lane = lane < bw;
  // SNR of candidate w with N(w) = nw
  auto eval = [&](int w, float nw) -> float {
    const int mv = (KM || uniform) ? M : comb_mvalid(w, M, N - 1 - d);
    const bool disjoint = w >= span;
    const int h = disjoint ? mv * span : (mv - 1) * w + span;
    const int c = N - h;
    // bins of H(w) below the band
    const int j = disjoint ? lane_m * w + lane_o : w - d + lane;
    const bool blw = lane < h && below_band(Pw[lane < h ? j : 0], j, T, tj);
    const int below = __popc(__ballot_sync(0xffffffffu, blw));
    // band positions inside H(w)
    bool rm = false;
    if (KM) {
#pragma unroll
      for (int m = 1; m <= KM; ++m) rm |= (uint32_t)(bj - m * w + d) <= (uint32_t)(2 * d);
    } else {
      for (int m = 1; m <= mv; ++m) rm |= (uint32_t)(bj - m * w + d) <= (uint32_t)(2 * d);
    }
    const bool fr = band_lane && !rm;
    const uint32_t fb = __ballot_sync(0xffffffffu, fr);
    const int rank = __popc(fb & lt);
    const int t = (c - 1) / 2 - (lo_r - below);
    int pos0 = __ffs(__ballot_sync(0xffffffffu, fr && rank == t)) - 1;
    int pos1 = (c & 1) ? pos0 : __ffs(__ballot_sync(0xffffffffu, fr && rank == t + 1)) - 1;
    if (pos0 < 0 || pos1 < 0) {
      pos0 = pos1 = 0;
      bad = true;
    }
    const float v0 = __shfl_sync(0xffffffffu, bv, pos0);
    const float v1 = __shfl_sync(0xffffffffu, bv, pos1);
    const float B = (c & 1) ? v0 : __fmul_rn(__fadd_rn(v0, v1), 0.5f);
    return snr_of(nw, B);
  };
  best = 0.f;
  bestw = -1;
  const int wstar = maxnw >= 0.f ? cc.w_lo + maxi : -1;
  float thr = 0.f;
  if (wstar >= 0) {
    best = eval(wstar, maxnw);
    bestw = wstar;
    // keep w when N(w) >= thr: thr <= best T (1 - 2^-20) (1 + 2^-23), so a
    // dropped candidate has N(w) / T < best (1 - 2^-21) and SNR(w) < best
    // (best and best T normal and finite, so that the rounding bounds hold)
    const float bt = __fmul_rn(best, T);
    const bool prune = T > 0.f && best >= 0x1p-126f && best < __int_as_float(0x7f800000) &&
                       bt >= 0x1p-100f && bt < __int_as_float(0x7f800000);
    thr = prune ? __fmul_rn(bt, 1.0f - 0x1p-20f) : 0.f;
  }
  for (int i0 = 0; i0 < n_cand; i0 += 32) {
    const int i = i0 + lane;
    const float nwl = i < n_cand ? nws[i] : -1.f;
    uint32_t sm = __ballot_sync(0xffffffffu, nwl >= 0.f && nwl >= thr && cc.w_lo + i != wstar);
    while (sm) {
      const int src = __ffs(sm) - 1;
      sm &= sm - 1;
      const int w = cc.w_lo + i0 + src;
      const float snr = eval(w, __shfl_sync(0xffffffffu, nwl, src));
      if (snr > best || (snr == best && w < bestw)) {
        best = snr;
        bestw = w;
      }
    }
  }
}

__device__ __forceinline__ CombOut comb_out(float best, int bestw, bool bad, float log_sf,
                                            const CombConst &cc) {
  CombOut out;
  out.log_sf = log_sf;
  out.bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
  out.snr = bestw >= 0 ? best : 0.f;
  out.w = bestw;
  out.rotor = (bestw >= 0 && best >= cc.tau_comb) ? 1 : 0;
  return out;
}

// The shared-memory form (any size within the fast limits).
__device__ __forceinline__ CombOut comb_warp_fast_smem(const float *Pw, const CombConst &cc,
                                                       unsigned char *scratch) {
  const int lane = threadIdx.x & 31;
  const int N = cc.N;
  uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + CombFast::kHist);
  const uint32_t hist_sa = (uint32_t)__cvta_generic_to_shared(hist);
  const float4 *P4 = reinterpret_cast<const float4 *>(Pw);
  const int ng = (N + 3) >> 2;  // 4-bin groups, the last one possibly partial
  CombOut out;
  out.snr = 0.f;
  out.w = -1;
  out.rotor = 0;
  out.bad = 0;
  bool bad = false;

  // ---- Eq. 7 sums (fixed order: 4-bin groups lane-strided, the (at most 3)
  // tail bins in the lane owning group N / 4, then a butterfly); the
  // histogram only for a pixel that passes the flatness test
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
  const float scale = __fdiv_rn(512.f, __fdiv_rn(sum, fN));
  __syncwarp();
  float sl2 = 0.f;  // sum of log2 max(P, 1e-30)
  for (int q = lane; q < nfull; q += 32) {
    const float4 v = P4[q];
    sl2 = __fadd_rn(sl2, lg2_normal(fmaxf(v.x, 1e-30f)));
    sl2 = __fadd_rn(sl2, lg2_normal(fmaxf(v.y, 1e-30f)));
    sl2 = __fadd_rn(sl2, lg2_normal(fmaxf(v.z, 1e-30f)));
    sl2 = __fadd_rn(sl2, lg2_normal(fmaxf(v.w, 1e-30f)));
  }
  if (lane == tail_lane)
    for (int j = jt; j < N; ++j) sl2 = __fadd_rn(sl2, lg2_normal(fmaxf(Pw[j], 1e-30f)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sl2 = __fadd_rn(sl2, __shfl_xor_sync(0xffffffffu, sl2, o));
  const float slog = __fmul_rn(sl2, 0.693147180559945309f);
  out.log_sf = sum > 0.f ? __fsub_rn(__fdiv_rn(slog, fN), __logf(__fdiv_rn(sum, fN))) : 0.f;
  if (!(out.log_sf <= cc.ln_tau_sf) || cc.w_hi < cc.w_lo) return out;
#pragma unroll
  for (int q = 0; q < CombFast::kHistBytes / 512; ++q)
    reinterpret_cast<uint4 *>(hist)[q * 32 + lane] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  for (int q = lane; q < nfull; q += 32) {
    const float4 v = P4[q];
    hist_add(hist_sa, bucket_bits(v.x, scale));
    hist_add(hist_sa, bucket_bits(v.y, scale));
    hist_add(hist_sa, bucket_bits(v.z, scale));
    hist_add(hist_sa, bucket_bits(v.w, scale));
  }
  if (lane == tail_lane)
    for (int j = jt; j < N; ++j) hist_add(hist_sa, bucket_bits(Pw[j], scale));
  __syncwarp();

  // ---- the band: lane p < bw holds the bin at full rank lo_r + p
  const int lo_r = cc.lo_r, bw = cc.bw, hi_r = cc.lo_r + cc.bw - 1;
  const BandBuckets bb = comb_locate(hist, N, lo_r, hi_r, bad);
  bool slow = bb.ncand > CombFast::kMaxCand || bad;
  float bv = 0.f;  // its value
  int bj = 0;      // its bin
  if (!slow) {
    // this lane's candidates: bit 4k + u for element u of group lane + 32 k
    const uint32_t g0 = (uint32_t)bb.g0, gspan = (uint32_t)(bb.g1 - bb.g0);
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int q = lane + 32 * k;
      if (32 * k < ng && q < ng) {
        const float4 v = P4[q];
        const int j = 4 * q;
        m |= ((uint32_t)(bucket_of(v.x, scale) - g0) <= gspan ? 1u : 0u) << (4 * k);
        m |= ((uint32_t)(bucket_of(v.y, scale) - g0) <= gspan && j + 1 < N ? 1u : 0u)
             << (4 * k + 1);
        m |= ((uint32_t)(bucket_of(v.z, scale) - g0) <= gspan && j + 2 < N ? 1u : 0u)
             << (4 * k + 2);
        m |= ((uint32_t)(bucket_of(v.w, scale) - g0) <= gspan && j + 3 < N ? 1u : 0u)
             << (4 * k + 3);
      }
    }
    uint32_t nsel;
    uint32_t off = warp_excl_scan<uint32_t>((uint32_t)__popc(m), nsel);
    if ((int)nsel != bb.ncand) slow = true;  // uniform (a reduction)
    if (!slow) {
      uint32_t *cv = reinterpret_cast<uint32_t *>(scratch + CombFast::kCandV);
      uint16_t *cj = reinterpret_cast<uint16_t *>(scratch + CombFast::kCandJ);
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int j = 4 * (lane + 32 * (b >> 2)) + (b & 3);
        cv[off] = __float_as_uint(Pw[j]);
        cj[off] = (uint16_t)j;
        ++off;
      }
      __syncwarp();
      if (!comb_band_sorted(scratch, bb.ncand, lo_r, bb.cb, bw, bv, bj, bad)) slow = true;
      __syncwarp();
    }
  }
  if (slow) {
    // exact band [lo_r, hi_r] by radix selection (a rare, out-of-line path)
    uint32_t bvu = 0u;
    __syncwarp();
    bad |= comb_band_exact(Pw, N, lo_r, hi_r, bw, hist, bvu, bj);
    bv = __uint_as_float(bvu);
    __syncwarp();
  }

  // ---- window maxima: rec[c] = max of P over [c - d, c + d] (centres
  // d .. N-1-d are the ones read)
  const int d = cc.d;
  float *rec = reinterpret_cast<float *>(scratch + CombFast::kRec);
  if (d == 3) {
    // centre quads 4q .. 4q + 3: bins 4q - 4 .. 4q + 7 by three 16-byte loads
    for (int q = lane; q < ng; q += 32) {
      float b[12];  // b[i] = P[4q - 4 + i]
      if (q >= 1 && q + 1 < nfull) {
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
      if (q < nfull) {
        reinterpret_cast<float4 *>(rec)[q] = make_float4(w0, w1, w2, w3);
      } else {  // the partial last quad
        const float wv[4] = {w0, w1, w2, w3};
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j0 + u < N) rec[j0 + u] = wv[u];
      }
    }
  } else {
    comb_records_any_d(Pw, N, d, rec);
  }
  __syncwarp();

  // ---- Eq. 8-10. When every candidate has M_valid = M and a non-empty
  // complement (always for h_min >= M and N > M(2d+1)), N(w) is a plain sum
  // over M windows.
  const bool uniform = cc.M * cc.w_hi <= N - 1 - d && N > cc.M * (2 * d + 1);
  float *nws = reinterpret_cast<float *>(scratch + CombFast::nw_off(N, cc.w_hi - cc.w_lo + 1));
  float maxnw;
  int maxi;
  comb_nw_all<0, 0>(rec, nws, cc, uniform, maxnw, maxi);
  __syncwarp();
  float best;
  int bestw;
  comb_best<0, 0>(Pw, nws, cc, uniform, maxnw, maxi, bv, bj, best, bestw, bad);
  out = comb_out(best, bestw, bad, out.log_sf, cc);
  __syncwarp();
  return out;
}

// The register form: 512 < N <= 768 bins, M = 4, d = 3. Lane l holds bins
// [24 l, 24 l + 24) in v[0..5] (bins at or beyond N as zeros); the lane's own
// sums run in bin order, then a butterfly. The zeros of the last lanes add
// nothing to the sum, lg2(1e-30) each to the log sum and one each to bucket 0
// of the histogram; both are taken back out, so the results are those of the
// N bins.
__device__ __forceinline__ CombOut comb_warp_fast_regs(const float *Pw, const CombConst &cc,
                                                       unsigned char *scratch) {
  constexpr int kB = CombReg::kBPL, kM = CombReg::kM, kD = CombReg::kD;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const int N = cc.N;
  uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + CombFast::kHist);
  const uint32_t hist_sa = (uint32_t)__cvta_generic_to_shared(hist);
  CombOut out;
  out.snr = 0.f;
  out.w = -1;
  out.rotor = 0;
  out.bad = 0;
  bool bad = false;
  // ---- the lane's 24 bins
  const int base = kB * lane;
  const int nval = min(max(N - base, 0), kB);  // bins of this lane below N
  float v[kB];
  {
    const float4 *P4 = reinterpret_cast<const float4 *>(Pw) + base / 4;
#pragma unroll
    for (int k = 0; k < kB / 4; ++k) {
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (4 * k < nval) {
        t = P4[k];
        const int r = nval - 4 * k;  // the group may run past N: those bins become zeros
        if (r < 4) {
          if (r < 2) t.y = 0.f;
          if (r < 3) t.z = 0.f;
          t.w = 0.f;
        }
      }
      v[4 * k] = t.x;
      v[4 * k + 1] = t.y;
      v[4 * k + 2] = t.z;
      v[4 * k + 3] = t.w;
    }
  }
  // ---- Eq. 7 sums; the histogram only for a pixel that passes the flatness test
  float sum = 0.f;
#pragma unroll
  for (int i = 0; i < kB; ++i) sum = __fadd_rn(sum, v[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, o));
  // 512 / mean; any positive scale gives exact buckets (the histogram and the
  // candidate test use the same one), so an approximate reciprocal will do
  const float scale = __fmul_rn(512.f * (float)N, rcp_approx(sum));
  __syncwarp();
  float sl2 = 0.f;
#pragma unroll
  for (int i = 0; i < kB; ++i) sl2 = __fadd_rn(sl2, lg2_normal(fmaxf(v[i], 1e-30f)));
  const int npad = kB - nval;
  if (npad > 0) sl2 = __fmaf_rn(-(float)npad, lg2_normal(1e-30f), sl2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sl2 = __fadd_rn(sl2, __shfl_xor_sync(0xffffffffu, sl2, o));
  const float slog = __fmul_rn(sl2, 0.693147180559945309f);
  out.log_sf = sum > 0.f ? __fsub_rn(__fmul_rn(slog, cc.inv_N), __logf(__fmul_rn(sum, cc.inv_N)))
                         : 0.f;
  if (!(out.log_sf <= cc.ln_tau_sf) || cc.w_hi < cc.w_lo) return out;
#pragma unroll
  for (int q = 0; q < CombFast::kHistBytes / 512; ++q)
    reinterpret_cast<uint4 *>(hist)[q * 32 + lane] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
#pragma unroll
  for (int i = 0; i < kB; ++i) hist_add(hist_sa, bucket_bits(v[i], scale));
  if (npad > 0) atomicSub(&hist[0], (uint32_t)npad);  // bucket 0 is the low half of word 0
  __syncwarp();

  // ---- window maxima of the lane's centres from its bins and three bins of
  // each neighbour: b[i] = P[base - 3 + i], i = 0..29; centres 4k .. 4k+3 of
  // the lane need b[4k .. 4k+9]
  float *rec = reinterpret_cast<float *>(scratch + CombFast::kRec);
  {
    float lft[kD], rgt[kD];
#pragma unroll
    for (int i = 0; i < kD; ++i) {
      lft[i] = __shfl_up_sync(0xffffffffu, v[kB - kD + i], 1);
      rgt[i] = __shfl_down_sync(0xffffffffu, v[i], 1);
    }
    float4 *r4 = reinterpret_cast<float4 *>(rec) + base / 4;
#pragma unroll
    for (int k = 0; k < kB / 4; ++k) {
      float b[10];
#pragma unroll
      for (int i = 0; i < 10; ++i) {
        const int src = 4 * k + i - kD;  // bin of the lane, -3 .. 26
        b[i] = src < 0 ? lft[src + kD] : (src >= kB ? rgt[src - kB] : v[src]);
      }
      const float mid = fmaxf(fmaxf(b[3], b[4]), fmaxf(b[5], b[6]));
      const float l1 = fmaxf(b[1], b[2]), r1 = fmaxf(b[7], b[8]);
      const float w0 = fmaxf(mid, fmaxf(b[0], l1));
      const float w1 = fmaxf(mid, fmaxf(l1, b[7]));
      const float w2 = fmaxf(mid, fmaxf(b[2], r1));
      const float w3 = fmaxf(mid, fmaxf(r1, b[9]));
      if (4 * k < nval) r4[k] = make_float4(w0, w1, w2, w3);
    }
  }

  // ---- the band: lane p < bw holds the bin at full rank lo_r + p
  const int lo_r = cc.lo_r, bw = cc.bw, hi_r = cc.lo_r + cc.bw - 1;
  const BandBuckets bb = comb_locate(hist, N, lo_r, hi_r, bad);
  bool slow = bb.ncand > CombFast::kMaxCand || bad;
  float bv = 0.f;
  int bj = 0;
  if (!slow) {
    // the lane's candidates as a bit mask over its 24 bins (read back from
    // shared memory, so that its registers are free for the selection), then
    // compacted in bin order
    uint32_t *cv = reinterpret_cast<uint32_t *>(scratch + CombFast::kCandV);
    uint16_t *cj = reinterpret_cast<uint16_t *>(scratch + CombFast::kCandJ);
    const float x0 = (float)bb.g0, x1 = (float)(bb.g1 + 1);
    const float4 *P4 = reinterpret_cast<const float4 *>(Pw) + base / 4;
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < kB / 4; ++k) {
      const float4 t = 4 * k < nval ? P4[k] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float e[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float x = bucket_x(e[u], scale);
        m |= (x >= x0 && x < x1 ? 1u : 0u) << (4 * k + u);
      }
    }
    m &= nval >= kB ? 0xFFFFFFu : (nval > 0 ? (1u << nval) - 1u : 0u);
    uint32_t run;
    uint32_t off = warp_excl_scan<uint32_t>((uint32_t)__popc(m), run);
    if ((int)run == bb.ncand) {
      while (m) {
        const int bi = __ffs(m) - 1;
        m &= m - 1;
        cv[off] = __float_as_uint(Pw[base + bi]);
        cj[off] = (uint16_t)(base + bi);
        ++off;
      }
    }
    __syncwarp();
    if ((int)run != bb.ncand) slow = true;  // uniform (a warp total)
    if (!slow && !comb_band_sorted(scratch, bb.ncand, lo_r, bb.cb, bw, bv, bj, bad)) slow = true;
    __syncwarp();
  }
  if (slow) {
    uint32_t bvu = 0u;
    __syncwarp();
    bad |= comb_band_exact(Pw, N, lo_r, hi_r, bw, hist, bvu, bj);
    bv = __uint_as_float(bvu);
    __syncwarp();
  }
  __syncwarp();

  // ---- Eq. 8-10
  const bool uniform = kM * cc.w_hi <= N - 1 - kD && N > kM * (2 * kD + 1);
  float *nws = reinterpret_cast<float *>(scratch + CombFast::nw_off(N, cc.w_hi - cc.w_lo + 1));
  float maxnw;
  int maxi;
  comb_nw_all<kM, kD>(rec, nws, cc, uniform, maxnw, maxi);
  __syncwarp();
  float best;
  int bestw;
  comb_best<kM, kD>(Pw, nws, cc, uniform, maxnw, maxi, bv, bj, best, bestw, bad);
  out = comb_out(best, bestw, bad, out.log_sf, cc);
  __syncwarp();
  return out;
}

__device__ __forceinline__ CombOut comb_warp_fast(const float *Pw, const CombConst &cc,
                                                  unsigned char *scratch) {
  if (CombReg::fits(cc)) return comb_warp_fast_regs(Pw, cc, scratch);
  return comb_warp_fast_smem(Pw, cc, scratch);
}

// Which comb variant a context uses: 0 = fast (N <= 1024, band <= 32; the
// register or shared-memory form, chosen at run time), otherwise the generic
// one with NW mask words per centre. A kernel that scores every pixel of one
// context can instead take the fast form itself: 2 = register form, 3 =
// shared-memory form (comb_fast_form).
__host__ __device__ inline int comb_variant(const CombConst &cc) {
  if (cc.N <= CombFast::kMaxN && cc.bw <= CombFast::kMaxBand && cc.M * (2 * cc.d + 1) <= 32)
    return 0;
  return cc.bw <= 32 ? 1 : 8;
}

__host__ __device__ inline int comb_fast_form(const CombConst &cc) {
  return CombReg::fits(cc) ? 2 : 3;
}

__host__ __device__ inline int comb_scratch_bytes(const CombConst &cc, int variant) {
  return (variant == 0 || variant == 2 || variant == 3)
             ? CombFast::bytes(cc.N, cc.w_hi - cc.w_lo + 1)
             : CombScratch::bytes(cc.N, variant);
}

// Eq. 7-11 for one pixel's spectrum Pw[0..N) in shared memory by the calling
// warp; scratch: comb_scratch_bytes(cc, NW) bytes (16-byte aligned).
template <int NW>
__device__ __forceinline__ CombOut comb_warp(const float *Pw, const CombConst &cc,
                                             unsigned char *scratch) {
  if constexpr (NW == 0) return comb_warp_fast(Pw, cc, scratch);
  else if constexpr (NW == 2) return comb_warp_fast_regs(Pw, cc, scratch);
  else if constexpr (NW == 3) return comb_warp_fast_smem(Pw, cc, scratch);
  else return comb_warp_generic<NW>(Pw, cc, scratch);
}

}  // namespace ddhf
