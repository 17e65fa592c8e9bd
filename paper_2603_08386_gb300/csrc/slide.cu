// Sliding-window spectra: Eq. 6 kept up to date event by event.
//
// Sec. 3.3 notes that the direct NDFT can take the contribution of each event
// on its own as it arrives. Here a window of length T slides over one event
// stream: every push of the events of [t_prev, t_end) adds their terms and
// subtracts the terms of the events that leave [t_end - T, t_end), so a hop
// costs (events in + events out) x n_bins terms instead of the whole window's.
//
// State, per pixel k of the context's sensor:
//   F_k[j] = sum over the window's events of p e^{-2 pi i a_j (t - t_b) / denom}
//            (FP32 complex, t_b = the stream's first time, row stride ldF),
//   n_k    = the window's event count (int32).
// |F_k[j]|^2 is Eq. 6's P over the window: the phase origin of Eq. 6 (the
// window start t0) and t_b differ by the factor e^{-2 pi i a_j (t0 - t_b) /
// denom}, of modulus one. As in the batch kernels, the phase of a term is the
// exact integer residue (a_j tau) mod denom, here with tau = (t - t_b) mod
// denom, so an event that leaves subtracts exactly the phasor it added.
//
// The events of the window are kept in a device ring, in push order: a 32-bit
// word (pixel key, polarity -1 in bit 31, kDropKey for events that were not
// added) and the int64 timestamp. The host keeps each push's ring range and
// time span [t_lo, t_hi); a push scans the ranges of the pushes with
// t_lo < t_end - T and selects the events with t_end_prev - T <= t < t_end - T,
// so events may arrive in any order within a push. A push's ring space is
// reused once t_hi <= t_end_prev - T.
//
// Per push: one kernel writes the new events into the ring and packs the
// delta (pixel key; tau | sign bit, the sign of an expiring event flipped)
// with kDropKey for unselected entries; the binning sort groups the delta by
// pixel (stable: within a pixel, events that leave come first, in ring order,
// then events that enter, in input order); a persistent kernel adds each
// touched pixel's delta sum to F_k (pixels with many delta events by a whole
// block, the others by one warp each; every pixel by exactly one group, so
// the result is deterministic).
//
// Precision: each push rounds F_k once more, so after R pushes F carries up to
// R rounding steps of 2^-24 |F|. Every rebuild_every pushes the state is
// recomputed: F and n are cleared and every event still in the window is
// added again, which bounds that drift.
//
// Detection: the pixels with n_k >= n_min (ascending) become the context's
// active list (slot 0); the comb kernel reads their rows of F and forms
// P = |F|^2 as it loads them (the same rounding as ddhf_slide_spectra), and
// the labelling and box kernels of ddhf_detect follow.
#include <string.h>

#include <algorithm>
#include <deque>
#include <new>

#include "ddhf_internal.cuh"

#define DDHF_TRY_S(x)                  \
  do {                                 \
    ddhf_status st__ = (x);            \
    if (st__ != DDHF_OK) return st__;  \
  } while (0)

namespace ddhf {

struct SlideBatch {
  int64_t start, n, t_lo, t_hi;
};

struct SlideState {
  int64_t T = 0, t_begin = 0, t_end = 0, cap = 0;
  int rebuild_every = 0, since = 0;
  int tpl = 8;
  int64_t ldF = 0;
  float2 *F = nullptr;
  int32_t *cnt = nullptr;
  uint32_t *ring_key = nullptr;
  int64_t *ring_t = nullptr;
  uint32_t *dk = nullptr, *dv = nullptr;  // packed delta [cap]
  Slot delta;                             // the delta grouped by pixel
  uint64_t *heavy = nullptr;              // [npx] heavy delta pixels
  uint32_t *ctl = nullptr;                // [4] heavy count, heavy grab, light grab, -
  uint64_t *stat = nullptr;               // [4] added, dropped, expired, in window
  std::deque<SlideBatch> batches;
  int64_t used = 0, tail = 0;
  int64_t pushes = 0, rebuilds = 0;
};

namespace {

constexpr int kSlideThreads = 256;
constexpr int kSlideWarps = kSlideThreads / 32;
constexpr int kSlideHeavy = 256;  // delta events from which a block takes the pixel
constexpr int kSlideGrab = 4;     // light pixels per grab
constexpr unsigned kFull = 0xffffffffu;

struct PackArgs {
  const int16_t *x, *y;
  const int64_t *t;
  const int8_t *p;
  int64_t n_new;
  int64_t t_lo_new, t_end;  // new events kept: t_lo_new <= t < t_end
  int64_t cut_prev, cut;    // ring events leaving: cut_prev <= t < cut
  int rebuild;              // ring events re-added: t >= cut
  int64_t scan_start, n_scan, tail, cap;
  int W, H, pol01, row0;
  int64_t t_begin;
  uint64_t denom, barrett;
};

__device__ __forceinline__ uint32_t tau_of(int64_t t, const PackArgs &A) {
  return (uint32_t)mod_barrett((uint64_t)(t - A.t_begin), A.denom, A.barrett);
}

// Ring entries to scan (delta positions [0, n_scan)), then the new events
// (positions n_scan + i), which are also written into the ring at tail + i.
__global__ void __launch_bounds__(256) k_slide_pack(PackArgs A, uint32_t *__restrict__ ring_key,
                                                    int64_t *__restrict__ ring_t,
                                                    uint32_t *__restrict__ dk,
                                                    uint32_t *__restrict__ dv,
                                                    int32_t *__restrict__ cnt,
                                                    uint64_t *__restrict__ stat) {
  const int64_t total = A.n_scan + A.n_new;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool added = false, dropped = false, expired = false;
    if (i < A.n_scan) {
      int64_t pos = A.scan_start + i;
      if (pos >= A.cap) pos -= A.cap;
      const uint32_t rk = ring_key[pos];
      const int64_t t = ring_t[pos];
      uint32_t key = kDropKey, val = 0;
      if (rk != kDropKey) {
        expired = t >= A.cut_prev && t < A.cut;
        const bool keep = A.rebuild ? t >= A.cut : expired;
        if (keep) {
          key = rk & 0x7fffffffu;
          const bool neg = (rk & kSignBit) != 0;
          val = tau_of(t, A) | ((A.rebuild ? neg : !neg) ? kSignBit : 0u);
          atomicAdd(&cnt[key], A.rebuild ? 1 : -1);
        }
      }
      dk[i] = key;
      dv[i] = val;
    } else if (i < total) {
      const int64_t e = i - A.n_scan;
      const int xx = A.x[e], yy = A.y[e] - A.row0;
      const int64_t t = A.t[e];
      const int pp = A.p[e];
      const bool okp = A.pol01 ? (pp == 0 || pp == 1) : (pp == 1 || pp == -1);
      const bool neg = A.pol01 ? (pp == 0) : (pp == -1);
      const bool ok = okp && xx >= 0 && xx < A.W && yy >= 0 && yy < A.H && t >= A.t_lo_new &&
                      t < A.t_end;
      const uint32_t key = (uint32_t)(yy * A.W + xx);
      int64_t pos = A.tail + e;
      if (pos >= A.cap) pos -= A.cap;
      ring_key[pos] = ok ? (key | (neg ? kSignBit : 0u)) : kDropKey;
      ring_t[pos] = t;
      dk[i] = ok ? key : kDropKey;
      dv[i] = ok ? (tau_of(t, A) | (neg ? kSignBit : 0u)) : 0u;
      if (ok) atomicAdd(&cnt[key], 1);
      added = ok;
      dropped = !ok;
    }
    const uint32_t na = __popc(__ballot_sync(kFull, added));
    const uint32_t nd = __popc(__ballot_sync(kFull, dropped));
    const uint32_t nx = __popc(__ballot_sync(kFull, expired));
    if (lane == 0) {
      if (na) atomicAdd((unsigned long long *)&stat[0], (unsigned long long)na);
      if (nd) atomicAdd((unsigned long long *)&stat[1], (unsigned long long)nd);
      if (nx) atomicAdd((unsigned long long *)&stat[2], (unsigned long long)nx);
      if (na != nx)
        atomicAdd((unsigned long long *)&stat[3], (unsigned long long)((int64_t)na - (int64_t)nx));
    }
  }
}

struct UpdArgs {
  const uint32_t *ev, *offsets, *active;
  const uint64_t *counters;  // [2] = pixels touched by the delta
  const uint64_t *heavy;     // heavy items, low 32 bits = index into active
  const uint32_t *ctl;       // ctl[0] = heavy count
  uint32_t *grab;            // [0] heavy, [1] light
  float2 *F;
  int64_t ldF;
  int64_t n_heavy_cap;
  GridConst g;
};

// Partial sums over the packed events ev[e0, e1) at bins j0 + lane + 32 m,
// m < TPL, as two rotation chains of TPL / 2 bins: chain A starts at bin
// j0 + lane, chain B at bin j0 + lane + 32 TPL / 2. Per event: the exact
// residues of both first bins and of a 32-bin step, their phasors, then
// TPL / 2 - 1 rotations of both chains at once in paired FP32 instructions
// (real parts of A and B in one float2, imaginary parts in another):
//   re' = re ur - im ui,  im' = re ui + im ur,  each element rounded on its own.
// accR[m] = (A_m, B_m) real sums, accI[m] the imaginary ones.
template <int TPL>
__device__ __forceinline__ void slide_terms(const uint32_t *__restrict__ ev, int64_t e0,
                                            int64_t e1, uint64_t a_mod_a, uint64_t a_mod_b,
                                            const GridConst &g, float2 (&accR)[TPL / 2],
                                            float2 (&accI)[TPL / 2], int lane) {
  for (int64_t c0 = e0; c0 < e1; c0 += 32) {
    const uint32_t mine = (c0 + lane < e1) ? ev[c0 + lane] : 0u;
    const int ne = (int)(e1 - c0 < 32 ? e1 - c0 : 32);
    for (int e = 0; e < ne; ++e) {
      const uint32_t w = __shfl_sync(kFull, mine, e);
      const uint64_t tau = w & 0x7fffffffu;
      const float2 za =
          phasor_of_residue(mod_barrett(a_mod_a * tau, g.denom, g.barrett), g.two_over_denom);
      const float2 zb =
          phasor_of_residue(mod_barrett(a_mod_b * tau, g.denom, g.barrett), g.two_over_denom);
      const float2 u =
          phasor_of_residue(mod_barrett(g.da32_mod * tau, g.denom, g.barrett), g.two_over_denom);
      const float sg = (w & kSignBit) ? -1.f : 1.f;
      float2 R = make_float2(sg * za.x, sg * zb.x), I = make_float2(sg * za.y, sg * zb.y);
      const float2 UR = make_float2(u.x, u.x), UI = make_float2(u.y, u.y);
      const float2 NUI = make_float2(-u.y, -u.y);
#pragma unroll
      for (int m = 0; m < TPL / 2; ++m) {
        accR[m] = __fadd2_rn(accR[m], R);
        accI[m] = __fadd2_rn(accI[m], I);
        if (m + 1 < TPL / 2) {
          const float2 t1 = __fmul2_rn(R, UR), t2 = __fmul2_rn(R, UI);
          R = __ffma2_rn(I, NUI, t1);
          I = __ffma2_rn(I, UR, t2);
        }
      }
    }
  }
}

__device__ __forceinline__ uint64_t first_bin_mod(const GridConst &g, int j) {
  return mod_barrett(g.a0 + (uint64_t)j * g.da, g.denom, g.barrett);
}

template <int TPL>
__device__ void slide_pixel_warp(const UpdArgs &A, uint32_t k, int64_t e0, int64_t e1,
                                 int lane) {
  constexpr int HALF = TPL / 2;
  const int N = A.g.N;
  float2 *Fk = A.F + (int64_t)k * A.ldF;
  for (int j0 = 0; j0 < N; j0 += 32 * TPL) {
    float2 accR[HALF], accI[HALF];
#pragma unroll
    for (int m = 0; m < HALF; ++m) accR[m] = accI[m] = make_float2(0.f, 0.f);
    slide_terms<TPL>(A.ev, e0, e1, first_bin_mod(A.g, j0 + lane),
                     first_bin_mod(A.g, j0 + lane + 32 * HALF), A.g, accR, accI, lane);
#pragma unroll
    for (int m = 0; m < HALF; ++m) {
      const int ja = j0 + lane + 32 * m, jb = ja + 32 * HALF;
      if (ja < N) {
        const float2 f = Fk[ja];
        Fk[ja] = make_float2(__fadd_rn(f.x, accR[m].x), __fadd_rn(f.y, accI[m].x));
      }
      if (jb < N) {
        const float2 f = Fk[jb];
        Fk[jb] = make_float2(__fadd_rn(f.x, accR[m].y), __fadd_rn(f.y, accI[m].y));
      }
    }
  }
}

// A whole block on one pixel: warp w sums the w-th eighth of the events; the
// eight partials of each bin are added in warp order through shared memory,
// chain A's bins first, then chain B's.
template <int TPL>
__device__ void slide_pixel_block(const UpdArgs &A, uint32_t k, int64_t e0, int64_t e1,
                                  float2 *red) {
  constexpr int HALF = TPL / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = A.g.N;
  const int64_t n = e1 - e0;
  const int64_t lo = e0 + n * warp / kSlideWarps, hi = e0 + n * (warp + 1) / kSlideWarps;
  float2 *Fk = A.F + (int64_t)k * A.ldF;
  for (int j0 = 0; j0 < N; j0 += 32 * TPL) {
    float2 accR[HALF], accI[HALF];
#pragma unroll
    for (int m = 0; m < HALF; ++m) accR[m] = accI[m] = make_float2(0.f, 0.f);
    slide_terms<TPL>(A.ev, lo, hi, first_bin_mod(A.g, j0 + lane),
                     first_bin_mod(A.g, j0 + lane + 32 * HALF), A.g, accR, accI, lane);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
      for (int m = 0; m < HALF; ++m)
        red[warp * 32 * HALF + 32 * m + lane] =
            c == 0 ? make_float2(accR[m].x, accI[m].x) : make_float2(accR[m].y, accI[m].y);
      __syncthreads();
      for (int b = threadIdx.x; b < 32 * HALF; b += kSlideThreads) {
        const int j = j0 + 32 * HALF * c + b;  // slot 32 m + lane: bin j0 + lane + 32 m (+ chain)
        if (j < N) {
          float2 sm = red[b];
          for (int w = 1; w < kSlideWarps; ++w) {
            sm.x = __fadd_rn(sm.x, red[w * 32 * HALF + b].x);
            sm.y = __fadd_rn(sm.y, red[w * 32 * HALF + b].y);
          }
          const float2 f = Fk[j];
          Fk[j] = make_float2(__fadd_rn(f.x, sm.x), __fadd_rn(f.y, sm.y));
        }
      }
      __syncthreads();
    }
  }
}

// Persistent: blocks take heavy delta pixels first, then warps take the
// others in grabs of kSlideGrab.
template <int TPL>
__global__ void __launch_bounds__(kSlideThreads, 3) k_slide_update(UpdArgs A) {
  __shared__ float2 red[kSlideWarps * 32 * (TPL / 2)];
  __shared__ uint32_t item;
  const int lane = threadIdx.x & 31;
  const int64_t nh = (int64_t)A.ctl[0];
  const uint32_t n_heavy = (uint32_t)(nh < A.n_heavy_cap ? nh : A.n_heavy_cap);
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(&A.grab[0], 1u);
    __syncthreads();
    const uint32_t h = item;
    __syncthreads();
    if (h >= n_heavy) break;
    const uint32_t k = A.active[(uint32_t)A.heavy[h]];
    slide_pixel_block<TPL>(A, k, A.offsets[k], A.offsets[k + 1], red);
  }
  const uint64_t n_touched = A.counters[2];
  for (;;) {
    uint32_t a0 = 0;
    if (lane == 0) a0 = atomicAdd(&A.grab[1], (uint32_t)kSlideGrab);
    a0 = __shfl_sync(kFull, a0, 0);
    if ((uint64_t)a0 >= n_touched) break;
    for (int i = 0; i < kSlideGrab; ++i) {
      const uint64_t a = (uint64_t)a0 + i;
      if (a >= n_touched) break;
      const uint32_t k = A.active[a];
      const uint32_t e0 = A.offsets[k], e1 = A.offsets[k + 1];
      if ((int64_t)(e1 - e0) >= kSlideHeavy) continue;  // a block's
      slide_pixel_warp<TPL>(A, k, e0, e1, lane);
    }
  }
}

// (n_k << 32 | 1) for pixels with n_k >= n_min, else 0; entry npx is 0.
__global__ void k_slide_flag(const int32_t *__restrict__ cnt, uint64_t *__restrict__ packed,
                             int64_t npx, int n_min) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= npx;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v = 0;
    if (k < npx) {
      const int32_t n = cnt[k];
      if (n >= n_min) v = ((uint64_t)(uint32_t)n << 32) | 1u;
    }
    packed[k] = v;
  }
}

// Active list (ascending keys) and the slot counters from the scanned flags.
__global__ void k_slide_list(const int32_t *__restrict__ cnt, const uint64_t *__restrict__ scanned,
                             uint32_t *__restrict__ active, uint64_t *__restrict__ counters,
                             const uint64_t *__restrict__ stat, int64_t npx, int n_min,
                             int64_t n_bins) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= npx;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t v = scanned[k];
    if (k < npx) {
      if (cnt[k] >= n_min) active[(uint32_t)v] = (uint32_t)k;
    } else {
      counters[0] = stat[3];  // events in the window
      counters[1] = 0;
      counters[2] = (uint32_t)v;  // active pixels
      counters[3] = stat[3];
      counters[4] = 0;
      counters[5] = (v >> 32) * (uint64_t)n_bins;  // terms of a full evaluation
    }
  }
}

// P[a * ld + j] = |F_k[j]|^2 for the a-th active pixel k, one warp per row.
__global__ void __launch_bounds__(256) k_slide_power(const float2 *__restrict__ F, int64_t ldF,
                                                     const uint32_t *__restrict__ active,
                                                     const uint64_t *__restrict__ counters,
                                                     float *__restrict__ P, int64_t ld,
                                                     int64_t cap_px, int N, uint32_t *flags) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_active = (int64_t)counters[2];
  for (int64_t a = wid; a < n_active; a += nw) {
    if (a >= cap_px) {
      if (lane == 0) atomicOr(flags, DDHF_FLAG_CAPACITY);
      break;
    }
    const float2 *Fk = F + (int64_t)active[a] * ldF;
    float *Pa = P + a * ld;
    for (int j = lane; j < N; j += 32) {
      const float2 f = Fk[j];
      Pa[j] = __fadd_rn(__fmul_rn(f.x, f.x), __fmul_rn(f.y, f.y));
    }
  }
}

ddhf_status sfail(Ctx *c, ddhf_status st, const char *msg) {
  c->last_error = msg;
  return st;
}

template <typename T>
ddhf_status salloc(Ctx *c, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    c->last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return DDHF_ERR_CUDA;
  }
  *p = static_cast<T *>(q);
  return DDHF_OK;
}

// Bins per lane per pass: the largest of 24, 16, 8 with the fewest padded bins.
int choose_tpl(int N) {
  int best = 24;
  int64_t best_pad = -1;
  for (int t : {24, 16, 8}) {
    const int64_t span = 32 * t;
    const int64_t pad = ceil_div(N, span) * span;
    if (best_pad < 0 || pad < best_pad) {
      best = t;
      best_pad = pad;
    }
  }
  return best;
}

ddhf_status launch_update(Ctx *c, SlideState *S, cudaStream_t s) {
  UpdArgs A{S->delta.ev, S->delta.offsets, S->delta.active, S->delta.counters, S->heavy,
            S->ctl,      S->ctl + 1,       S->F,           S->ldF,           c->npx,
            c->gconst};
#define DDHF_SLIDE_CASE(TPLV)                                                                 \
  {                                                                                           \
    int occ = 0;                                                                              \
    DDHF_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_slide_update<TPLV>, \
                                                                   kSlideThreads, 0));        \
    occ = std::max(occ, 1);                                                                   \
    k_slide_update<TPLV><<<c->num_sms * occ, kSlideThreads, 0, s>>>(A);                       \
  }
  if (S->tpl == 24) DDHF_SLIDE_CASE(24)
  else if (S->tpl == 16) DDHF_SLIDE_CASE(16)
  else DDHF_SLIDE_CASE(8)
#undef DDHF_SLIDE_CASE
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

// Active list of the window (slot 0) from the counts.
ddhf_status slide_active(Ctx *c, SlideState *S, cudaStream_t s) {
  const int64_t npx = c->npx;
  const unsigned pb = (unsigned)std::min<int64_t>(ceil_div(npx + 1, 256), c->num_sms * 8);
  k_slide_flag<<<pb, 256, 0, s>>>(S->cnt, c->packed, npx, c->params.n_min);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  DDHF_TRY_S(launch_scan_u64(c, c->packed, c->packed, npx + 1, s));
  Slot &sl = c->slots[0];
  k_slide_list<<<pb, 256, 0, s>>>(S->cnt, c->packed, sl.active, sl.counters, S->stat, npx,
                                  c->params.n_min, c->grid.n_bins);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  c->binned = false;  // slot 0's per-pixel event list no longer matches its active list
  return DDHF_OK;
}

ddhf_status slide_power(Ctx *c, SlideState *S, float *P, int64_t ld, int64_t cap_px,
                        cudaStream_t s) {
  const int64_t rows = std::max<int64_t>(1, std::min<int64_t>(c->npx, cap_px));
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(rows, 8), c->num_sms * 8);
  k_slide_power<<<blocks, 256, 0, s>>>(S->F, S->ldF, c->slots[0].active, c->slots[0].counters,
                                       P, ld, cap_px, c->grid.n_bins, c->flags);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

}  // namespace

void slide_free(Ctx *c) {
  SlideState *S = c->slide;
  if (!S) return;
  auto F = [](void *p) {
    if (p) cudaFree(p);
  };
  F(S->F);
  F(S->cnt);
  F(S->ring_key);
  F(S->ring_t);
  F(S->dk);
  F(S->dv);
  F(S->delta.ev);
  F(S->delta.offsets);
  F(S->delta.active);
  F(S->delta.counters);
  F(S->heavy);
  F(S->ctl);
  F(S->stat);
  delete S;
  c->slide = nullptr;
}

}  // namespace ddhf

using namespace ddhf;

extern "C" {

ddhf_status ddhf_slide_begin(ddhf_ctx *h, int64_t window_us, int64_t t_begin_us,
                             int64_t capacity, int32_t rebuild_every) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (window_us < 1 || capacity < 1 || capacity > c->max_events || capacity >= (1ll << 31) ||
      rebuild_every < 0)
    return sfail(c, DDHF_ERR_INVALID_ARG,
                 "need window_us >= 1, 1 <= capacity <= min(max_events, 2^31 - 1), "
                 "rebuild_every >= 0");
  if (c->slide) {
    cudaDeviceSynchronize();
    slide_free(c);
  }
  SlideState *S = new (std::nothrow) SlideState();
  if (!S) return sfail(c, DDHF_ERR_CUDA, "host allocation failed");
  c->slide = S;
  S->T = window_us;
  S->t_begin = t_begin_us;
  S->t_end = t_begin_us;
  S->cap = capacity;
  S->rebuild_every = rebuild_every;
  S->tpl = choose_tpl(c->grid.n_bins);
  S->ldF = ((int64_t)c->grid.n_bins + 31) & ~(int64_t)31;
  const int64_t npx = c->npx;
  ddhf_status st = DDHF_OK;
#define A(ptr, n) \
  if (st == DDHF_OK) st = salloc(c, &(ptr), (size_t)(n))
  A(S->F, npx * S->ldF);
  A(S->cnt, npx);
  A(S->ring_key, capacity);
  A(S->ring_t, capacity);
  A(S->dk, capacity);
  A(S->dv, capacity);
  A(S->delta.ev, capacity);
  A(S->delta.offsets, npx + 1);
  A(S->delta.active, npx);
  A(S->delta.counters, 8);
  A(S->heavy, npx);
  A(S->ctl, 4);
  A(S->stat, 4);
#undef A
  if (st == DDHF_OK) {
    cudaError_t e = cudaMemset(S->F, 0, (size_t)npx * S->ldF * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(S->cnt, 0, npx * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(S->stat, 0, 4 * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMemset(S->delta.counters, 0, 8 * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      c->last_error = std::string("slide state: ") + cudaGetErrorString(e);
      st = DDHF_ERR_CUDA;
    }
  }
  if (st != DDHF_OK) slide_free(c);
  return st;
}

ddhf_status ddhf_slide_end(ddhf_ctx *h) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!c->slide) return sfail(c, DDHF_ERR_STATE, "no sliding window");
  cudaDeviceSynchronize();
  slide_free(c);
  return DDHF_OK;
}

ddhf_status ddhf_slide_push(ddhf_ctx *h, const int16_t *x, const int16_t *y, const int64_t *t_us,
                            const int8_t *p, int64_t n, int64_t t_end_us, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  SlideState *S = c->slide;
  if (!S) return sfail(c, DDHF_ERR_STATE, "no sliding window (ddhf_slide_begin)");
  if (n < 0 || (n > 0 && (!x || !y || !t_us || !p)) || t_end_us < S->t_end)
    return sfail(c, DDHF_ERR_INVALID_ARG, "bad events or t_end before the previous t_end");
  const int64_t cut_prev = S->t_end - S->T, cut = t_end_us - S->T;
  // ring space of pushes whose events all left at an earlier push
  while (!S->batches.empty() && S->batches.front().t_hi <= cut_prev) {
    S->used -= S->batches.front().n;
    S->batches.pop_front();
  }
  if (S->used + n > S->cap)
    return sfail(c, DDHF_ERR_CAPACITY, "ring capacity exceeded (events of the window + push)");
  const bool rebuild = S->rebuild_every > 0 && S->since + 1 >= S->rebuild_every;
  int64_t n_scan = 0;
  if (rebuild) {
    n_scan = S->used;
  } else {
    for (const SlideBatch &b : S->batches) {
      if (b.t_lo >= cut) break;
      n_scan += b.n;
    }
  }
  const int64_t scan_start = S->batches.empty() ? S->tail : S->batches.front().start;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(S->ctl, 0, 4 * sizeof(uint32_t), s));
  if (rebuild) {
    DDHF_CUDA_TRY(c, cudaMemsetAsync(S->F, 0, (size_t)c->npx * S->ldF * sizeof(float2), s));
    DDHF_CUDA_TRY(c, cudaMemsetAsync(S->cnt, 0, c->npx * sizeof(int32_t), s));
  }
  const GridConst &g = c->gconst;
  PackArgs A{x,        y,          t_us,       p,         n,      std::max(S->t_end, cut),
             t_end_us, cut_prev,   cut,        rebuild,   scan_start, n_scan,
             S->tail,  S->cap,     c->W,       c->H,      c->params.polarity_01, c->row0,
             S->t_begin, g.denom,  g.barrett};
  const int64_t total = n_scan + n;
  if (total > 0) {
    const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(total, 256), c->num_sms * 16);
    k_slide_pack<<<blocks, 256, 0, s>>>(A, S->ring_key, S->ring_t, S->dk, S->dv, S->cnt,
                                        S->stat);
    DDHF_CUDA_TRY(c, cudaGetLastError());
  }
  DDHF_TRY_S(bin_packed(c, S->delta, S->dk, S->dv, total, 1, kSlideHeavy, S->heavy, S->ctl,
                        c->npx, s));
  DDHF_TRY_S(launch_update(c, S, s));
  if (n > 0) {
    S->batches.push_back(SlideBatch{S->tail, n, S->t_end, t_end_us});
    S->used += n;
    S->tail = (S->tail + n) % S->cap;
  }
  S->t_end = t_end_us;
  S->pushes += 1;
  if (rebuild) {
    S->rebuilds += 1;
    S->since = 0;
  } else {
    S->since += 1;
  }
  return DDHF_OK;
}

ddhf_status ddhf_slide_spectra(ddhf_ctx *h, float *P, int64_t cap_px, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  SlideState *S = c->slide;
  if (!S) return sfail(c, DDHF_ERR_STATE, "no sliding window (ddhf_slide_begin)");
  if (cap_px < 0 || (cap_px > 0 && !P)) return sfail(c, DDHF_ERR_INVALID_ARG, "bad P");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  DDHF_TRY_S(slide_active(c, S, s));
  if (cap_px > 0) DDHF_TRY_S(slide_power(c, S, P, c->grid.n_bins, cap_px, s));
  return DDHF_OK;
}

ddhf_status ddhf_slide_detect(ddhf_ctx *h, ddhf_box *boxes, int32_t cap, int32_t *n_boxes_dev,
                              uint8_t *mask_out, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  SlideState *S = c->slide;
  if (!S) return sfail(c, DDHF_ERR_STATE, "no sliding window (ddhf_slide_begin)");
  if (!n_boxes_dev || cap < 0 || (cap > 0 && !boxes))
    return sfail(c, DDHF_ERR_INVALID_ARG, "bad box arguments");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  Slot &sl = c->slots[0];
  DDHF_TRY_S(slide_active(c, S, s));
  DDHF_TRY_S(launch_comb_cplx(c, S->F, S->ldF, sl.log_sf, sl.snr, sl.f0, sl.mask, s));
  DDHF_TRY_S(launch_label(c, sl.mask, sl.labels, sl.counters + 7, s));
  DDHF_TRY_S(launch_boxes(c, sl.labels, boxes, cap, sl.nbox, s));
  DDHF_CUDA_TRY(c, cudaMemcpyAsync(n_boxes_dev, sl.nbox, sizeof(int32_t),
                                   cudaMemcpyDeviceToDevice, s));
  if (mask_out)
    DDHF_CUDA_TRY(c, cudaMemcpyAsync(mask_out, sl.mask, c->npx, cudaMemcpyDeviceToDevice, s));
  return DDHF_OK;
}

ddhf_status ddhf_slide_get_stats(ddhf_ctx *h, ddhf_slide_stats *out) {
  if (!h || !out) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  SlideState *S = c->slide;
  if (!S) return sfail(c, DDHF_ERR_STATE, "no sliding window (ddhf_slide_begin)");
  DDHF_CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
  uint64_t st[4], dc[8];
  DDHF_CUDA_TRY(c, cudaMemcpy(st, S->stat, sizeof(st), cudaMemcpyDeviceToHost));
  DDHF_CUDA_TRY(c, cudaMemcpy(dc, S->delta.counters, sizeof(dc), cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  out->t_end_us = S->t_end;
  out->pushes = S->pushes;
  out->rebuilds = S->rebuilds;
  out->n_added = (int64_t)st[0];
  out->n_dropped = (int64_t)st[1];
  out->n_expired = (int64_t)st[2];
  out->n_window = (int64_t)st[3];
  out->last_delta = (int64_t)dc[0];
  out->last_pixels = (int64_t)dc[2];
  out->ring_used = S->used;
  return DDHF_OK;
}

}  // extern "C"
