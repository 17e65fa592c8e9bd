// Spectra of heavy pixels through a uniform time grid (the NUFFT route that
// the footnote to Sec. 3.3 sets aside for the tens of events of a typical
// pixel; the heavy tail of a busy window has pixels with thousands).
//
// For a pixel with events (tau_k, p_k), Eq. 6 at bin j is
//   F_j = sum_k p_k e^{-2 pi i a_j tau_k / D},  a_j = a0 + j da.
// With the centre bin J = floor(N / 2), a_c = a0 + J da and m = j - J:
//   F_j = sum_k q_k e^{-2 pi i m nu tau_k},  q_k = p_k e^{-2 pi i a_c tau_k / D},
// nu = da / D cycles per us: a type-1 non-uniform transform over |m| <= N/2
// (Dutt and Rokhlin's problem). Each event is spread onto a grid of spacing s
// us (t_g = (g - 3) s, s = floor(D / (2 da N)), so the band |m nu s| <= 1/4 is
// at most half the grid's Nyquist band) with the "exponential of semicircle"
// kernel of Barnett, Magland and af Klinteberg (SIAM J. Sci. Comput. 2019),
//   psi(z) = exp(beta (sqrt(1 - (2 z / w)^2) - 1)),  |z| <= w / 2,  w = 8,
//   beta = 2.30 w,
// c_g = sum_k q_k psi(g - 3 - tau_k / s). By Poisson summation
//   sum_g c_g e^{-2 pi i m nu t_g} = sum_k q_k sum_l psi^(kappa_m + l)
//                                    e^{-2 pi i (kappa_m + l) tau_k / s},
// kappa_m = m nu s, so F_j = S_j / psi^(kappa_m) up to the aliased terms l != 0
// (relative size ~1e-7 at w = 8). S_j is a product of the pixel's G grid
// values with one table E[g][j] = e^{-2 pi i m nu t_g} / psi^(kappa_m) shared by
// every pixel: a dense complex matrix product [pixels x G] x [G x N], done
// here with three real multiplications per term as in the blocked form.
// Phases of q_k and of E come from exact integer residues; psi^ is a
// quadrature on the host in FP64.
//
// Kernels: k_hyb_list (pixels with at least thr events), k_hyb_table (E),
// k_hyb_spread (one block per pixel, its warps on contiguous shares of the
// events, four event groups per warp into four copies of the grid in shared
// memory, so that no two lanes add to the same word and the sum order is
// fixed), k_hyb_grid (64 pixels x 128 bins per block tile,
// K = grid rows in chunks of 16 staged by cp.async in two buffers, 4 x 8
// outputs per thread updated by paired FMAs).
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include "ddhf_internal.cuh"

namespace ddhf {
namespace hybrid {

constexpr int kW = 8;          // grid points per event
constexpr int kOff = kW / 2 - 1;  // grid row g holds time (g - kOff) s
constexpr double kBeta = 2.30 * kW;
constexpr int kTileP = 64, kTileB = 128, kKC = 16;
constexpr int kGemmThreads = 256;
constexpr int kSpreadWarps = 8;
constexpr int kCopies = 32 / kW;  // event groups per warp step
constexpr int kCopyPad = 8;       // float2 between grid copies: the four groups of a
                                  // step fall on alternate halves of the banks

constexpr uint32_t kFrontMin = 1024;  // pixels listed first (taken first by the spread)

// The kernel in grid steps z, |z| <= w / 2, from the hardware reciprocal
// square root and base-2 exponential: relative error ~1e-7 near the peak and
// ~1e-6 at the edges, where the kernel is below e^-10. With FP32 sums this
// puts the spectra 2-3e-6 of the peak power from Eq. 6 (the route's own
// aliasing error is ~1e-7).
__device__ __forceinline__ float es_kernel(float z) {
  const float x = __fmul_rn(z, 2.0f / kW);
  const float r = fmaxf(__fsub_rn(1.0f, __fmul_rn(x, x)), 0.0f);
  const float sq = r > 0.0f ? __fmul_rn(r, rsqrtf(r)) : 0.0f;
  return __expf((float)kBeta * (sq - 1.0f));
}

// Entry h of the hybrid list: pixels with at least kFrontMin events are
// stored from the front (count[0] of them), the others from the back.
__device__ __forceinline__ uint32_t list_at(const uint32_t *list, const uint32_t *count,
                                            int64_t cap, int64_t h) {
  const uint32_t nf = count[0];
  return h < (int64_t)nf ? list[h] : list[cap - 1 - (h - (int64_t)nf)];
}

__device__ __forceinline__ int64_t list_size(const uint32_t *count, int64_t cap) {
  return min((int64_t)count[0] + (int64_t)count[1], cap);
}

// Active indices a of the slot's pixels with at least thr events, the
// heaviest (>= kFrontMin) at the front so that they are spread first.
__global__ void k_hyb_list(const uint32_t *__restrict__ active, const uint32_t *__restrict__ offsets,
                           const uint64_t *__restrict__ counters, int thr, uint32_t *list,
                           uint32_t *count, int64_t cap, uint32_t *flags) {
  const int64_t n_act = (int64_t)counters[2];
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n_act;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = base + threadIdx.x;
    uint32_t cnt = 0;
    if (a < n_act) {
      const uint32_t k = active[a];
      cnt = offsets[k + 1] - offsets[k];
    }
    const bool take = a < n_act && cnt >= (uint32_t)thr;
    const bool front = take && cnt >= kFrontMin;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool mine = side == 0 ? front : (take && !front);
      const uint32_t bal = __ballot_sync(0xffffffffu, mine);
      uint32_t pos0 = 0;
      if (lane == 0 && bal) pos0 = atomicAdd(count + side, (uint32_t)__popc(bal));
      pos0 = __shfl_sync(0xffffffffu, pos0, 0);
      if (mine) {
        const int64_t pos = pos0 + __popc(bal & ((1u << lane) - 1u));
        if (pos < cap) list[side == 0 ? pos : cap - 1 - pos] = (uint32_t)a;
        else atomicOr(flags, DDHF_FLAG_INTERNAL);
      }
    }
  }
}

struct TableArgs {
  GridConst g;
  int G, Gp, np, J;
  uint64_t ds_mod;   // (da s) mod D
  const float *dec;  // [N] 1 / psi^(kappa_m)
  float2 *eri;       // [Gp][np]
  float *es;         // [Gp][np]
};

// E[g][j] = dec_j e^{-2 pi i r / D}, r = (m (g - kOff) da s) mod D; zero
// outside g < G, j < N.
__global__ void k_hyb_table(TableArgs T) {
  const int64_t total = (int64_t)T.Gp * T.np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(i / T.np), j = (int)(i - (int64_t)g * T.np);
    float2 e = make_float2(0.f, 0.f);
    if (g < T.G && j < T.g.N) {
      const int64_t D = (int64_t)T.g.denom;
      int64_t u = ((int64_t)(j - T.J) * (int64_t)(g - kOff)) % D;
      if (u < 0) u += D;
      const uint64_t r = mod_barrett((uint64_t)u * T.ds_mod, T.g.denom, T.g.barrett);
      const float2 z = phasor_of_residue(r, T.g.two_over_denom);
      const float dj = T.dec[j];
      e = make_float2(__fmul_rn(z.x, dj), __fmul_rn(z.y, dj));
    }
    T.eri[i] = e;
    T.es[i] = __fadd_rn(e.x, e.y);
  }
}

struct SpreadArgs {
  GridConst g;
  const uint32_t *ev, *offsets, *active;
  const uint32_t *list;
  const uint32_t *count;
  uint64_t ac_mod;  // a_c mod D
  uint32_t s;       // grid spacing (us)
  float inv_s;
  int Gp;
  int64_t cap_h;    // row stride of C (pixels)
  float4 *C;        // [Gp][cap_h]: (cr, ci, cr + ci, cr + ci)
  uint32_t *cursor; // next list entry to take (zeroed before the launch)
};

// One block per listed pixel (blocks take pixels from a counter); warp w of
// nw takes the w-th contiguous share of the pixel's events. Lane l of a
// 32-event chunk prepares event l (its phasor q and grid position; the next
// chunk's event word is loaded meanwhile). Lane (e, i) = (l / 8, l % 8) then
// evaluates the kernel for events 4 t + e, t < 8, of the chunk (independent
// work, kept in registers) and adds q psi to the warp's copy e of grid rows
// i0 + i, one step t at a time. The nw x 4 copies are summed in a fixed order
// (warp, then copy) and cleared for the next pixel.
__global__ void __launch_bounds__(kSpreadWarps * 32) k_hyb_spread(SpreadArgs A) {
  extern __shared__ float2 sm2[];
  __shared__ uint32_t s_item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int cs = A.Gp + kCopyPad;  // stride of one grid copy
  float2 *acc = sm2 + (int64_t)warp * kCopies * cs;
  const int ncopy = nw * kCopies;
  // the list holds at most cap_h entries (an overflow raised DDHF_FLAG_INTERNAL)
  const uint32_t n_h = (uint32_t)list_size(A.count, A.cap_h);
  const int grp = lane / kW, ii = lane % kW;
  constexpr int kSteps = 32 / kCopies;
  for (int i = threadIdx.x; i < ncopy * cs; i += blockDim.x) sm2[i] = make_float2(0.f, 0.f);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.cursor, 1u);
    __syncthreads();  // also orders the clearing below before this pixel's sums
    const uint32_t h = s_item;
    __syncthreads();
    if (h >= n_h) break;
    const uint32_t a = list_at(A.list, A.count, A.cap_h, h);
    const uint32_t key = A.active[a];
    const uint32_t p0 = A.offsets[key], p1 = A.offsets[key + 1];
    const uint32_t n = p1 - p0;
    const uint32_t o0 = p0 + (uint32_t)((uint64_t)n * warp / nw);
    const uint32_t o1 = p0 + (uint32_t)((uint64_t)n * (warp + 1) / nw);
    uint32_t wnext = o0 + lane < o1 ? A.ev[o0 + lane] : 0u;
    for (uint32_t c0 = o0; c0 < o1; c0 += 32) {
      const int ne = (int)min(32u, o1 - c0);
      const uint32_t w = wnext;
      wnext = c0 + 32 + lane < o1 ? A.ev[c0 + 32 + lane] : 0u;
      float qx = 0.f, qy = 0.f, fr = 0.f;
      uint32_t i0 = 0;
      if (lane < ne) {
        const uint32_t tau = w & 0x7fffffffu;
        const uint64_t r = mod_barrett(A.ac_mod * (uint64_t)tau, A.g.denom, A.g.barrett);
        const float2 z = phasor_of_residue(r, A.g.two_over_denom);
        const float sg = (w & kSignBit) ? -1.f : 1.f;
        qx = sg * z.x;
        qy = sg * z.y;
        i0 = tau / A.s;
        fr = __fmul_rn((float)(tau - i0 * A.s), A.inv_s);
      }
      float vx[kSteps], vy[kSteps];
      uint32_t vg[kSteps];
#pragma unroll
      for (int t = 0; t < kSteps; ++t) {
        const int src = kCopies * t + grp;
        const float ex = __shfl_sync(0xffffffffu, qx, src);
        const float ey = __shfl_sync(0xffffffffu, qy, src);
        const float ef = __shfl_sync(0xffffffffu, fr, src);
        vg[t] = __shfl_sync(0xffffffffu, i0, src);
        const float psi = src < ne ? es_kernel(__fsub_rn((float)(ii - kOff), ef)) : 0.f;
        vx[t] = __fmul_rn(ex, psi);
        vy[t] = __fmul_rn(ey, psi);
      }
#pragma unroll
      for (int t = 0; t < kSteps; ++t) {
        if (kCopies * t + grp < ne) {
          float2 &cg = acc[grp * cs + vg[t] + ii];
          cg.x = __fadd_rn(cg.x, vx[t]);
          cg.y = __fadd_rn(cg.y, vy[t]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int g = threadIdx.x; g < A.Gp; g += blockDim.x) {
      float2 v = sm2[g];
      sm2[g] = make_float2(0.f, 0.f);
      for (int cpy = 1; cpy < ncopy; ++cpy) {
        const float2 u = sm2[cpy * cs + g];
        sm2[cpy * cs + g] = make_float2(0.f, 0.f);
        v.x = __fadd_rn(v.x, u.x);
        v.y = __fadd_rn(v.y, u.y);
      }
      const float sum = __fadd_rn(v.x, v.y);
      A.C[(int64_t)g * A.cap_h + h] = make_float4(v.x, v.y, sum, sum);
    }
  }
}

struct GridArgs {
  const float4 *C;    // [Gp][cap_h]
  const float2 *eri;  // [Gp][np]
  const float *es;    // [Gp][np]
  const uint32_t *list;
  const uint32_t *count;
  int64_t cap_h;
  int Gp, np, N;
  float *P;
  int64_t ld;
  int vec_store;      // P and ld allow 8-byte stores
  int64_t cap_px;
  uint32_t *flags;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Shared-memory stage: A [kKC][64] float4, B [kKC][64] float4 (128 (Er, Ei)
// pairs), S [kKC][32] float4 (128 Er + Ei).
constexpr int kStageA = kKC * kTileP;  // float4
constexpr int kStageB = kKC * kTileB / 2;
constexpr int kStageS = kKC * kTileB / 4;
constexpr int kStageF4 = kStageA + kStageB + kStageS;
constexpr size_t kGemmSmem = 2 * kStageF4 * sizeof(float4);

__device__ __forceinline__ void load_stage(const GridArgs &A, float4 *st, int64_t p0, int b0,
                                           int k0) {
  const int t = threadIdx.x;
  // A: kKC rows of 64 float4
  for (int i = t; i < kStageA; i += kGemmThreads) {
    const int kk = i / kTileP, c = i % kTileP;
    cp_async16(st + i, A.C + (int64_t)(k0 + kk) * A.cap_h + p0 + c);
  }
  float4 *sb = st + kStageA;
  for (int i = t; i < kStageB; i += kGemmThreads) {
    const int kk = i / (kTileB / 2), c = i % (kTileB / 2);
    cp_async16(sb + i, reinterpret_cast<const float4 *>(A.eri + (int64_t)(k0 + kk) * A.np + b0) + c);
  }
  float4 *ss = sb + kStageB;
  for (int i = t; i < kStageS; i += kGemmThreads) {
    const int kk = i / (kTileB / 4), c = i % (kTileB / 4);
    cp_async16(ss + i, reinterpret_cast<const float4 *>(A.es + (int64_t)(k0 + kk) * A.np + b0) + c);
  }
}

// Thread (ty, tx): pixels 4 ty + p (p < 4), bins 2 tx + 32 q + {0, 1} (q < 4).
// t12[p][2q + e] = (T1, T2) of bin 2tx + 32q + e; t3[p][q] = (T3, T3) of the
// bin pair.
__global__ void __launch_bounds__(kGemmThreads, 1) k_hyb_grid(GridArgs A) {
  extern __shared__ float4 gsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ty = warp * 2 + (lane >> 4), tx = lane & 15;
  const int64_t n_h = list_size(A.count, A.cap_h);
  const int nbt = A.np / kTileB;
  const int64_t n_tiles = ((n_h + kTileP - 1) / kTileP) * nbt;
  const int nk = A.Gp / kKC;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t p0 = (tile / nbt) * kTileP;
    const int b0 = (int)(tile % nbt) * kTileB;
    float2 t12[4][8], t3[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
#pragma unroll
      for (int e = 0; e < 8; ++e) t12[p][e] = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q) t3[p][q] = make_float2(0.f, 0.f);
    }
    load_stage(A, gsm, p0, b0, 0);
    cp_async_commit();
    for (int kc = 0; kc < nk; ++kc) {
      if (kc + 1 < nk) load_stage(A, gsm + ((kc + 1) & 1) * kStageF4, p0, b0, (kc + 1) * kKC);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      const float4 *sa = gsm + (kc & 1) * kStageF4;
      const float4 *sb = sa + kStageA;
      const float2 *ss = reinterpret_cast<const float2 *>(sb + kStageB);
#pragma unroll 4
      for (int kk = 0; kk < kKC; ++kk) {
        float4 av[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) av[p] = sa[kk * kTileP + 4 * ty + p];
        float4 bv[4];
        float2 sv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          bv[q] = sb[kk * (kTileB / 2) + tx + 16 * q];
          sv[q] = ss[kk * (kTileB / 2) + tx + 16 * q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float2 cri = make_float2(av[p].x, av[p].y), css = make_float2(av[p].z, av[p].w);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            t12[p][2 * q] = __ffma2_rn(cri, make_float2(bv[q].x, bv[q].y), t12[p][2 * q]);
            t12[p][2 * q + 1] = __ffma2_rn(cri, make_float2(bv[q].z, bv[q].w), t12[p][2 * q + 1]);
            t3[p][q] = __ffma2_rn(css, sv[q], t3[p][q]);
          }
        }
      }
      __syncthreads();
    }
    // epilogue: P = (T1 - T2)^2 + (T3 - T1 - T2)^2 per bin
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t h = p0 + 4 * ty + p;
      if (h >= n_h) continue;
      const int64_t a = (int64_t)list_at(A.list, A.count, A.cap_h, h);
      if (a >= A.cap_px) {
        atomicOr(A.flags, DDHF_FLAG_CAPACITY);
        continue;
      }
      float *row = A.P + a * A.ld;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float pw[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float t1 = t12[p][2 * q + e].x, t2 = t12[p][2 * q + e].y;
          const float t3v = e ? t3[p][q].y : t3[p][q].x;
          const float fr = __fsub_rn(t1, t2);
          const float fi = __fsub_rn(__fsub_rn(t3v, t1), t2);
          pw[e] = __fmaf_rn(fr, fr, __fmul_rn(fi, fi));
        }
        const int j = b0 + 2 * tx + 32 * q;
        if (A.vec_store && j + 1 < A.N) {
          *reinterpret_cast<float2 *>(row + j) = make_float2(pw[0], pw[1]);
        } else {
          if (j < A.N) row[j] = pw[0];
          if (j + 1 < A.N) row[j + 1] = pw[1];
        }
      }
    }
  }
}

// psi^(kappa) = int psi(z) e^{-2 pi i kappa z} dz over |z| <= w/2 (even
// kernel, real transform), with z = (w/2) sin(theta): composite Simpson in
// theta on [-pi/2, pi/2], where the integrand is smooth.
double es_transform(double kappa) {
  const int n = 2048;
  const double h = M_PI / n, half = 0.5 * kW;
  double sum = 0.0;
  for (int i = 0; i <= n; ++i) {
    const double th = -0.5 * M_PI + i * h;
    const double f = exp(kBeta * (cos(th) - 1.0)) * cos(th) * half *
                     cos(2.0 * M_PI * kappa * half * sin(th));
    const double wgt = (i == 0 || i == n) ? 1.0 : (i & 1) ? 4.0 : 2.0;
    sum += wgt * f;
  }
  return sum * h / 3.0;
}

}  // namespace hybrid

using namespace hybrid;

int64_t hybrid_spacing(const ddhf_grid &g) {
  const double s = floor((double)g.denom / (2.0 * (double)g.da * (double)g.n_bins));
  return s >= 1.0 ? (int64_t)s : 0;
}

// Grid spacing, rows and pixel threshold of a window; false when the window
// does not take the route (grid spacing below 1 us, or G outside [16, 1024]).
// s and G are written either way.
bool hybrid_geometry(const ddhf_grid &g, int64_t window_us, int hybrid_min, int64_t *s,
                     int64_t *G, int64_t *thr) {
  *s = hybrid_spacing(g);
  *G = (*s >= 1 && window_us >= 1) ? (window_us - 1) / *s + kW : 0;
  *thr = std::max<int64_t>(std::max(hybrid_min, 16), ceil_div(*G, 2));
  return *s >= 1 && hybrid_min > 0 && window_us >= 1 && *G >= 16 && *G <= kHybMaxG;
}

// 1 / psi^(kappa_m) for the bins of grid g at spacing s: kappa_m = (j - J) da
// s / D with J = floor(N / 2); psi^ is even, so one quadrature per |m|.
void hybrid_dec_factors(const ddhf_grid &g, int64_t s, float *dec) {
  const int N = g.n_bins, J = N / 2;
  std::vector<float> by_abs_m(std::max(J, N - 1 - J) + 1);
  for (size_t am = 0; am < by_abs_m.size(); ++am) {
    const double kappa = (double)am * (double)g.da * (double)s / (double)g.denom;
    by_abs_m[am] = (float)(1.0 / es_transform(kappa));
  }
  for (int j = 0; j < N; ++j) dec[j] = by_abs_m[std::abs(j - J)];
}

HybridPlan hybrid_plan(const Ctx *c, int64_t window_us, int hybrid_min) {
  HybridPlan p{};
  int64_t G = 0;
  if (!hybrid_geometry(c->grid, window_us, hybrid_min, &p.s, &G, &p.thr)) {
    p.thr = 0;
    return p;
  }
  p.G = (int)G;
  p.Gp = (int)ceil_div(G, kKC) * kKC;
  const int64_t cap = std::min<int64_t>(c->npx, c->max_events / p.thr + 1);
  p.cap_h = ceil_div(cap, kTileP) * kTileP;
  p.ok = (int64_t)p.Gp * p.cap_h <= c->hyb_celems && p.cap_h <= c->hyb_list_cap;
  return p;
}

ddhf_status hybrid_alloc(Ctx *c) {
  if (c->hyb_c) return DDHF_OK;
  if (hybrid_spacing(c->grid) < 1) return DDHF_OK;  // the grid never takes this path
  const int N = c->grid.n_bins;
  c->hyb_np = ceil_div(N, kTileB) * kTileB;
  c->hyb_celems = 4 * std::max<int64_t>(c->max_events, 1) + (int64_t)kTileP * kHybMaxG;
  c->hyb_list_cap = ceil_div(std::min<int64_t>(c->npx, c->max_events / 16 + 1), kTileP) * kTileP;
  auto al = [&](void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) c->last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  bool ok = al((void **)&c->hyb_c, (size_t)c->hyb_celems * sizeof(float4)) &&
            al((void **)&c->hyb_eri, (size_t)kHybMaxG * c->hyb_np * sizeof(float2)) &&
            al((void **)&c->hyb_es, (size_t)kHybMaxG * c->hyb_np * sizeof(float)) &&
            al((void **)&c->hyb_dec, (size_t)N * sizeof(float)) &&
            al((void **)&c->hyb_list, (size_t)c->hyb_list_cap * sizeof(uint32_t));
  if (ok) {
    std::vector<float> dec(N);
    hybrid_dec_factors(c->grid, hybrid_spacing(c->grid), dec.data());
    ok = cudaMemcpy(c->hyb_dec, dec.data(), N * sizeof(float), cudaMemcpyHostToDevice) ==
         cudaSuccess;
    if (!ok) c->last_error = "hybrid: copy of the deconvolution factors failed";
  }
  if (!ok) {
    hybrid_free(c);
    cudaGetLastError();
    return DDHF_ERR_CUDA;
  }
  return DDHF_OK;
}

void hybrid_free(Ctx *c) {
  for (void *p : {(void *)c->hyb_c, (void *)c->hyb_eri, (void *)c->hyb_es, (void *)c->hyb_dec,
                  (void *)c->hyb_list})
    if (p) cudaFree(p);
  c->hyb_c = nullptr;
  c->hyb_eri = nullptr;
  c->hyb_es = nullptr;
  c->hyb_dec = nullptr;
  c->hyb_list = nullptr;
}

ddhf_status launch_hybrid(Ctx *c, int slot, const HybridPlan &hp, float *P, int64_t cap_px,
                          int64_t ld, cudaStream_t s) {
  const Slot &sl = c->slots[slot];
  uint32_t *count = c->qctl + 12;  // [0] front (heaviest), [1] back
  DDHF_CUDA_TRY(c, cudaMemsetAsync(count, 0, 2 * sizeof(uint32_t), s));
  k_hyb_list<<<c->num_sms * 8, 256, 0, s>>>(sl.active, sl.offsets, sl.counters, (int)hp.thr,
                                            c->hyb_list, count, hp.cap_h, c->flags);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  const GridConst &g = c->gconst;
  TableArgs T{};
  T.g = g;
  T.G = hp.G;
  T.Gp = hp.Gp;
  T.np = (int)c->hyb_np;
  T.J = g.N / 2;
  T.ds_mod = (uint64_t)(((unsigned __int128)g.da * (uint64_t)hp.s) % g.denom);
  T.dec = c->hyb_dec;
  T.eri = c->hyb_eri;
  T.es = c->hyb_es;
  const int64_t tot = (int64_t)hp.Gp * T.np;
  k_hyb_table<<<(int)std::min<int64_t>(ceil_div(tot, 256), (int64_t)c->num_sms * 16), 256, 0, s>>>(T);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  SpreadArgs S{};
  S.g = g;
  S.ev = sl.ev;
  S.offsets = sl.offsets;
  S.active = sl.active;
  S.list = c->hyb_list;
  S.count = count;
  S.ac_mod = (uint64_t)(((unsigned __int128)g.a0 + (unsigned __int128)(g.N / 2) * g.da) % g.denom);
  S.s = (uint32_t)hp.s;
  S.inv_s = (float)(1.0 / (double)hp.s);
  S.Gp = hp.Gp;
  S.cap_h = hp.cap_h;
  S.C = c->hyb_c;
  S.cursor = c->qctl + 14;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(S.cursor, 0, sizeof(uint32_t), s));
  // warps per pixel: up to 8, with their grid copies within 192 KiB
  const int cs = hp.Gp + kCopyPad;
  const int nw = std::max(1, std::min(kSpreadWarps, (192 * 1024) / (kCopies * cs * 8)));
  const size_t ssm = (size_t)nw * kCopies * cs * sizeof(float2);
  DDHF_CUDA_TRY(c, cudaFuncSetAttribute(k_hyb_spread, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)ssm));
  int occ = 0;
  DDHF_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hyb_spread, nw * 32,
                                                                 ssm));
  k_hyb_spread<<<c->num_sms * std::max(occ, 1), nw * 32, ssm, s>>>(S);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  GridArgs Gd{};
  Gd.C = c->hyb_c;
  Gd.eri = c->hyb_eri;
  Gd.es = c->hyb_es;
  Gd.list = c->hyb_list;
  Gd.count = count;
  Gd.cap_h = hp.cap_h;
  Gd.Gp = hp.Gp;
  Gd.np = (int)c->hyb_np;
  Gd.N = g.N;
  Gd.P = P;
  Gd.ld = ld;
  Gd.vec_store = (ld % 2 == 0) && (reinterpret_cast<uintptr_t>(P) % 8 == 0);
  Gd.cap_px = cap_px;
  Gd.flags = c->flags;
  DDHF_CUDA_TRY(c, cudaFuncSetAttribute(k_hyb_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kGemmSmem));
  int gocc = 0;
  DDHF_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gocc, k_hyb_grid, kGemmThreads,
                                                                 kGemmSmem));
  k_hyb_grid<<<c->num_sms * std::max(gocc, 1), kGemmThreads, kGemmSmem, s>>>(Gd);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

}  // namespace ddhf

extern "C" ddhf_status ddhf_hybrid_geometry(const ddhf_grid *grid, int64_t window_us,
                                            int32_t hybrid_min, int64_t *s_us, int32_t *rows,
                                            int32_t *threshold, float *dec) {
  if (!grid || grid->a0 < 0 || grid->da <= 0 || grid->denom <= 0 ||
      grid->denom >= ((int64_t)1 << 31) || grid->n_bins < 1 || grid->n_bins > 16384 ||
      window_us < 1 || window_us >= ((int64_t)1 << 31) || hybrid_min < 1)
    return DDHF_ERR_INVALID_ARG;
  int64_t s = 0, G = 0, thr = 0;
  const bool ok = ddhf::hybrid_geometry(*grid, window_us, hybrid_min, &s, &G, &thr);
  if (s_us) *s_us = s;
  if (rows) *rows = (int32_t)std::min<int64_t>(G, INT32_MAX);
  if (threshold) *threshold = ok ? (int32_t)thr : 0;
  if (dec && s >= 1) ddhf::hybrid_dec_factors(*grid, s, dec);
  return ok ? DDHF_OK : DDHF_ERR_UNSUPPORTED;
}
