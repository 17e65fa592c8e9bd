// Soft comb score and its adjoint (the differentiation pattern; the paper has
// no soft score, this builds on Eq. 6 and the comb idea of Eq. 8-10):
//
//   f_hq = h f0 + q delta,  h = 1..n_h, q = -Q..Q
//   G_hq = exp(-(q delta)^2 / (2 sigma_h^2)),  Z_h = sum_q G_hq
//   S    = sum_h w_h (sum_q G_hq P(f_hq) / Z_h) / B
//
// with P(f) = |F(f)|^2, F(f) = sum_k p_k exp(-2 pi i f (tau_k - tau_c)), B a
// constant background per pixel. The adjoint uses
// dP/df = 2 Re(conj(F) D), D = sum_k (-2 pi i (tau_k - tau_c)) p_k exp(...).
//
// One warp per pixel; lanes hold events (32 per chunk). For each harmonic h
// the phasor of event k at q = -Q is seeded exactly: the frequency, an
// integer number of micro-Hz (f0 and delta rounded to 1 uHz), is split into
// integer mHz (exact residue of a * tau mod 1e9, as in the grid NDFT) plus a
// sub-mHz remainder, and the constant window-centre phase is reduced exactly
// in integers (tau_c in half-microseconds); no FP64 arithmetic runs per
// harmonic or per event. The next q values follow by rotation with
// e^{-2 pi i delta (tau - tau_c)}. F and D for the 2Q+1
// frequencies are accumulated per lane and reduced over the warp in a fixed
// order. Per-pixel gradient contributions to w and sigma are written to a
// workspace and summed over pixels by a fixed-order reduction, so every
// output is deterministic.
#include "ddhf_internal.cuh"

namespace ddhf {

namespace {

constexpr int kSoftMaxQ = 8;   // 2Q+1 <= 17 frequencies per harmonic
constexpr int kSoftMaxH = 8;
constexpr float kTwoPi = 6.28318530717958647692f;

struct SoftArgs {
  const uint32_t *ev;
  const uint32_t *offsets;
  const uint32_t *pixels;  // pixel keys
  int64_t n_px;
  const float *f0;
  const float *w;
  const float *sigma;
  const float *B;
  int n_h, Q;
  int64_t delta_uhz;       // evaluation step in micro-Hz
  float delta_hz;          // the same step in Hz
  int64_t tc2;             // 2 tau_c in half-microseconds (tau_c relative to the window start)
  float *S;                // forward output [n_px]
  const float *gS;         // backward input [n_px]
  float *g_f0;             // backward output [n_px]
  float *g_f;              // backward output [n_px][n_h][2Q+1], nullable
  float *part;             // backward workspace [n_px][2 n_h]
  int backward;
  uint64_t barrett;        // floor((2^64-1) / 1e9)
  int64_t npx;             // keys at or beyond it are skipped (DDHF_FLAG_INPUT)
  uint32_t *flags;
  uint32_t *cursor;        // next pixel to take (zeroed before each launch)
};

template <bool BWD>
__global__ void __launch_bounds__(256) k_softcomb(SoftArgs A) {
  const int lane = threadIdx.x & 31;
  const uint64_t D9 = 1000000000ull;
  const int nq = 2 * A.Q + 1;
  // pixels are taken one at a time from a counter (a pixel's cost grows with
  // its events, which are heavy-tailed); the next index is fetched while the
  // current pixel is processed
  uint32_t next = 0;
  if (lane == 0) next = atomicAdd(A.cursor, 1u);
  for (int64_t a = __shfl_sync(0xffffffffu, next, 0); a < A.n_px;
       a = __shfl_sync(0xffffffffu, next, 0)) {
    if (lane == 0) next = atomicAdd(A.cursor, 1u);
    const uint32_t key = A.pixels[a];
    // a key off the sensor has no events: S = 0, zero gradients, flagged
    const bool key_ok = (int64_t)key < A.npx;
    if (!key_ok && lane == 0) atomicOr(A.flags, DDHF_FLAG_INPUT);
    const uint32_t o0 = key_ok ? A.offsets[key] : 0u;
    const int cnt = key_ok ? (int)(A.offsets[key + 1] - o0) : 0;
    // f0 in integer micro-Hz: every frequency h f0 + q delta is then an exact
    // integer number of micro-Hz, split into integer mHz (exact residue
    // a tau mod 1e9, as in the grid NDFT) plus a remainder below 1 mHz
    const int64_t f0u = __double2ll_rn((double)A.f0[a] * 1e6);
    const float Bv = A.B[a];
    float S = 0.f, g0 = 0.f;
    for (int h = 1; h <= A.n_h; ++h) {
      const int64_t fbu = (int64_t)h * f0u - (int64_t)A.Q * A.delta_uhz;  // q = -Q
      int64_t fm = fbu / 1000, rem = fbu - fm * 1000;
      if (rem < 0) {
        rem += 1000;
        fm -= 1;
      }
      const uint64_t am = mod_barrett((uint64_t)(fm < 0 ? -fm : fm), D9, A.barrett);
      const uint64_t ai = (fm < 0 && am != 0) ? D9 - am : am;        // fm mod 1e9
      const float fr = __fmul_rn((float)rem, 1e-6f);                 // Hz, in [0, 1e-3)
      // constant phase f tau_c in cycles: (fbu * tc2 / 2e12) mod 1, exactly in
      // integers (fbu mod 2e12 < 2^41, tc2 < 2^21)
      const int64_t P2 = 2000000000000ll;
      int64_t fmod2 = fbu % P2;
      if (fmod2 < 0) fmod2 += P2;
      const int64_t cm = (int64_t)(((uint64_t)fmod2 * (uint64_t)A.tc2) % (uint64_t)P2);
      const float cff = __fmul_rn((float)cm, 5e-13f);
      float Fr[2 * kSoftMaxQ + 1], Fi[2 * kSoftMaxQ + 1];
      float Dr[2 * kSoftMaxQ + 1], Di[2 * kSoftMaxQ + 1];
#pragma unroll
      for (int q = 0; q < 2 * kSoftMaxQ + 1; ++q) Fr[q] = Fi[q] = Dr[q] = Di[q] = 0.f;
      for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int k = c0 + lane;
        if (k < cnt) {
          const uint32_t wv = A.ev[o0 + k];
          const uint64_t tau = wv & 0x7fffffffu;
          const float sg = (wv & kSignBit) ? -1.f : 1.f;
          const uint64_t r = mod_barrett(ai * tau, D9, A.barrett);
          float x = __fmul_rn((float)(uint32_t)r, 1e-9f);  // r < 1e9, tau < 2^31: 32-bit
          x = __fadd_rn(x, __fmul_rn(__fmul_rn(fr, (float)(uint32_t)tau), 1e-6f));
          x = __fsub_rn(x, cff);
          x = __fsub_rn(x, rintf(x));                                 // [-0.5, 0.5] cycles
          float sn, cs;
          sincospi_reduced(2.f * x, sn, cs);
          float zr = sg * cs, zi = -sg * sn;
          const float tt = __fmul_rn((float)((int64_t)(2 * tau) - A.tc2), 0.5e-6f);  // s
          float ss, sc;
          float xs = __fmul_rn(A.delta_hz, tt);  // cycles, folded to [-1/2, 1/2]
          xs = __fsub_rn(xs, rintf(xs));
          sincospi_reduced(2.f * xs, ss, sc);
          const float ur = sc, ui = -ss;
          const float wtt = kTwoPi * tt;
#pragma unroll
          for (int q = 0; q < 2 * kSoftMaxQ + 1; ++q) {
            if (q < nq) {
              Fr[q] += zr;
              Fi[q] += zi;
              if (BWD) {
                Dr[q] = __fmaf_rn(wtt, zi, Dr[q]);   // D += -2 pi i tt z
                Di[q] = __fmaf_rn(-wtt, zr, Di[q]);
              }
              const float nr = __fmaf_rn(zr, ur, -__fmul_rn(zi, ui));
              const float ni = __fmaf_rn(zr, ui, __fmul_rn(zi, ur));
              zr = nr;
              zi = ni;
            }
          }
        }
      }
      // warp reduction in a fixed order
#pragma unroll
      for (int q = 0; q < 2 * kSoftMaxQ + 1; ++q) {
        if (q < nq) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            Fr[q] += __shfl_xor_sync(0xffffffffu, Fr[q], o);
            Fi[q] += __shfl_xor_sync(0xffffffffu, Fi[q], o);
            if (BWD) {
              Dr[q] += __shfl_xor_sync(0xffffffffu, Dr[q], o);
              Di[q] += __shfl_xor_sync(0xffffffffu, Di[q], o);
            }
          }
        }
      }
      const float sgm = A.sigma[h - 1], wh = A.w[h - 1];
      float Z = 0.f, Ac = 0.f, Ad = 0.f, Cc = 0.f, Ec = 0.f;
#pragma unroll
      for (int q = 0; q < 2 * kSoftMaxQ + 1; ++q) {
        if (q < nq) {
          const float qd = __fmul_rn((float)(q - A.Q), A.delta_hz);
          const float G = expf(-(qd * qd) / (2.f * sgm * sgm));
          const float P = Fr[q] * Fr[q] + Fi[q] * Fi[q];
          Z += G;
          Ac += G * P;
          if (BWD) {
            const float Pd = 2.f * (Fr[q] * Dr[q] + Fi[q] * Di[q]);
            Ad += G * Pd;
            Cc += G * P * qd * qd;
            Ec += G * qd * qd;
          }
        }
      }
      S += wh * (Ac / Z) / Bv;
      if (BWD && A.g_f) {
        // per evaluation frequency: g dS/df_hq = g w_h G_hq P'(f_hq) / (Z_h B),
        // written by lane q (every lane holds the reduced sums)
        const float gs = A.gS[a];
        float *out = A.g_f + (a * A.n_h + (h - 1)) * (int64_t)nq;
#pragma unroll
        for (int q = 0; q < 2 * kSoftMaxQ + 1; ++q) {
          if (q < nq && lane == q) {
            const float qd = __fmul_rn((float)(q - A.Q), A.delta_hz);
            const float G = expf(-(qd * qd) / (2.f * sgm * sgm));
            const float Pd = 2.f * (Fr[q] * Dr[q] + Fi[q] * Di[q]);
            out[q] = gs * (wh * G * Pd / (Z * Bv));
          }
        }
      }
      if (BWD) {
        g0 += wh * (float)h * (Ad / Z) / Bv;
        if (lane == 0) {
          const float gs = A.gS[a];
          A.part[a * 2 * A.n_h + (h - 1)] = gs * ((Ac / Z) / Bv);
          A.part[a * 2 * A.n_h + A.n_h + (h - 1)] =
              gs * (wh / (Bv * sgm * sgm * sgm) * (Cc / Z - (Ac / Z) * (Ec / Z)));
        }
      }
    }
    if (lane == 0) {
      if (BWD)
        A.g_f0[a] = A.gS[a] * g0;
      else
        A.S[a] = S;
    }
  }
}

// out[c] = sum_a part[a][c] for c < ncol, fixed order (block-wide tree).
__global__ void k_col_sum(const float *part, int64_t n_rows, int ncol, float *out) {
  __shared__ float sh[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int64_t a = threadIdx.x; a < n_rows; a += blockDim.x) s += part[a * ncol + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// Median of each spectrum row (the mean of the two middle values for an even
// count), exact, one warp per row: the two middle ranks are selected by an
// 8-bit radix select over the (value, index) keys.
__device__ uint64_t select_key(const float *Pr, int N, int R, uint32_t *hist) {
  const int lane = threadIdx.x & 31;
  uint64_t prefix = 0, pmask = 0;
  int r = R;
  for (int shift = 40; shift >= 0; shift -= 8) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    for (int j = lane; j < N; j += 32) {
      const uint64_t key = ((uint64_t)__float_as_uint(Pr[j]) << 16) | (uint32_t)j;
      if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255], 1u);
    }
    __syncwarp();
    uint32_t hv[8], s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      hv[q] = hist[lane * 8 + q];
      s += hv[q];
    }
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    const uint32_t ex = inc - s;
    const bool own = (uint32_t)r >= ex && (uint32_t)r < ex + s;
    int src = __ffs(__ballot_sync(0xffffffffu, own)) - 1;
    src = src < 0 ? 0 : src;
    int g = 0;
    uint32_t below = 0;
    if (lane == src) {
      uint32_t c = ex;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if ((uint32_t)r >= c && (uint32_t)r < c + hv[q]) {
          g = lane * 8 + q;
          below = c;
        }
        c += hv[q];
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

__global__ void k_row_median(const float *P, int64_t rows, int N, float *med) {
  __shared__ uint32_t hist[8][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = wid; a < rows; a += nwarps) {
    const float *Pr = P + a * N;
    const uint64_t k1 = select_key(Pr, N, (N - 1) / 2, hist[warp]);
    float v = __uint_as_float((uint32_t)(k1 >> 16));
    if ((N & 1) == 0) {
      const uint64_t k2 = select_key(Pr, N, N / 2, hist[warp]);
      v = __fmul_rn(__fadd_rn(v, __uint_as_float((uint32_t)(k2 >> 16))), 0.5f);
    }
    if (lane == 0) med[a] = v;
  }
}

}  // namespace
}  // namespace ddhf

using namespace ddhf;

extern "C" ddhf_status ddhf_softcomb(ddhf_ctx *h, int64_t n_px, const uint32_t *pixels,
                                     const float *f0, int32_t n_h, int32_t Q, double delta_hz,
                                     double tau_c_us, const float *w, const float *sigma,
                                     const float *B, float *S, const float *grad_S,
                                     float *grad_f0, float *grad_w, float *grad_sigma,
                                     float *grad_f, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!c->binned) {
    c->last_error = "no binned window";
    return DDHF_ERR_STATE;
  }
  if (n_px < 0 || n_px > c->npx || n_h < 1 || n_h > kSoftMaxH || Q < 0 || Q > kSoftMaxQ ||
      !(delta_hz >= 1e-6) || !(delta_hz < 1e6) || !(tau_c_us >= 0.0) ||
      !(tau_c_us < (double)(1 << 20)) ||
      (n_px > 0 && (!pixels || !f0 || !w || !sigma || !B))) {
    c->last_error = "softcomb: bad arguments";
    return DDHF_ERR_INVALID_ARG;
  }
  const bool bwd = grad_S != nullptr;
  if (!bwd && !S) {
    c->last_error = "softcomb: need S (forward) or grad_S (backward)";
    return DDHF_ERR_INVALID_ARG;
  }
  if (bwd && (!grad_f0 || !grad_w || !grad_sigma)) {
    c->last_error = "softcomb: backward needs grad_f0, grad_w, grad_sigma";
    return DDHF_ERR_INVALID_ARG;
  }
  if (n_px == 0) return DDHF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  SoftArgs A;
  A.ev = c->slots[0].ev;
  A.offsets = c->slots[0].offsets;
  A.pixels = pixels;
  A.n_px = n_px;
  A.f0 = f0;
  A.w = w;
  A.sigma = sigma;
  A.B = B;
  A.n_h = n_h;
  A.Q = Q;
  A.delta_uhz = llround(delta_hz * 1e6);
  A.delta_hz = (float)delta_hz;
  A.tc2 = llround(2.0 * tau_c_us);
  A.S = S;
  A.gS = grad_S;
  A.g_f0 = grad_f0;
  A.g_f = bwd ? grad_f : nullptr;
  A.part = c->soft_part;  // [n_px][2 n_h] then the 2 n_h column sums
  A.backward = bwd;
  A.barrett = ~0ull / 1000000000ull;
  A.npx = c->npx;
  A.flags = c->flags;
  A.cursor = c->qctl + 4;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(A.cursor, 0, sizeof(uint32_t), s));
  const int blocks = (int)std::min<int64_t>(ceil_div(n_px, 8), (int64_t)c->num_sms * 16);
  if (bwd) {
    k_softcomb<true><<<blocks, 256, 0, s>>>(A);
    k_col_sum<<<2 * n_h, 256, 0, s>>>(A.part, n_px, 2 * n_h, A.part + n_px * 2 * n_h);
    DDHF_CUDA_TRY(c, cudaMemcpyAsync(grad_w, A.part + n_px * 2 * n_h, n_h * sizeof(float),
                                     cudaMemcpyDeviceToDevice, s));
    DDHF_CUDA_TRY(c, cudaMemcpyAsync(grad_sigma, A.part + n_px * 2 * n_h + n_h,
                                     n_h * sizeof(float), cudaMemcpyDeviceToDevice, s));
  } else {
    k_softcomb<false><<<blocks, 256, 0, s>>>(A);
  }
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

extern "C" ddhf_status ddhf_spectrum_median(ddhf_ctx *h, const float *P, int64_t rows,
                                            float *median, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (rows < 0 || (rows > 0 && (!P || !median))) {
    c->last_error = "spectrum_median: bad arguments";
    return DDHF_ERR_INVALID_ARG;
  }
  if (rows == 0) return DDHF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const int blocks = (int)std::min<int64_t>(ceil_div(rows, 8), (int64_t)c->num_sms * 8);
  k_row_median<<<blocks, 256, 0, s>>>(P, rows, c->grid.n_bins, median);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}
