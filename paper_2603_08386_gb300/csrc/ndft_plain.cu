// Plain one-warp-per-pixel NDFT forms (Sec. 3.3 Eq. 6, P_k = |F_k|^2) used as
// the per-pixel baseline and for the precision study:
//   SINCOS   exact integer phase per term, advanced from bin to bin by an
//            exact modular step, then FP32 sincospi per term;
//   RECUR    exact seed and step phasors per event and lane, then a complex
//            rotation per bin (re-seeded every TPL bins);
//   KAHAN    SINCOS with compensated summation;
//   NAIVE32  FP32 phase 2 pi f t from the absolute timestamp (shows the loss
//            of precision that the exact reduction avoids);
//   F64      exact phase, FP64 sincospi and FP64 accumulation (check path).
// Lane l owns bins j0 + l + 32m (m < TPL); events are broadcast by shuffles.
#include "ddhf_internal.cuh"

namespace ddhf {

ddhf_status launch_blocked_spectrum(Ctx *c, float *P, int64_t cap_px, cudaStream_t s);
ddhf_status launch_hybrid_spectrum(Ctx *c, float *P, int64_t cap_px, cudaStream_t s);

namespace {

constexpr int kPlainThreads = 256;

__device__ __forceinline__ void raise_flag(uint32_t *flags, uint32_t f) { atomicOr(flags, f); }

// ------------------------------------------------------------------ plain

template <int FORM, int TPL>
__global__ void __launch_bounds__(kPlainThreads) k_plain(const uint32_t *__restrict__ ev,
                                                         const uint32_t *__restrict__ offsets,
                                                         const uint32_t *__restrict__ active,
                                                         const uint64_t *__restrict__ counters,
                                                         GridConst g, int64_t t0, float *__restrict__ P,
                                                         int64_t cap_px, uint32_t *flags) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_active = (int64_t)counters[2];
  const uint32_t D = (uint32_t)g.denom;
  const int N = g.N;
  for (int64_t a = wid; a < n_active; a += nwarps) {
    if (a >= cap_px) {
      if (lane == 0) raise_flag(flags, DDHF_FLAG_CAPACITY);
      break;
    }
    const uint32_t k = active[a];
    const uint32_t o0 = offsets[k];
    const int cnt = (int)(offsets[k + 1] - o0);
    for (int j0 = 0; j0 < N; j0 += 32 * TPL) {
      // per-lane bins j = j0 + lane + 32 m, m < TPL
      const uint64_t a_first = g.a0 + (uint64_t)(j0 + lane) * g.da;
      const uint64_t a_first_mod = a_first % g.denom;
      float re[TPL], im[TPL], cre[TPL], cim[TPL];
      double dre[TPL], dim[TPL];
#pragma unroll
      for (int m = 0; m < TPL; ++m) {
        re[m] = im[m] = cre[m] = cim[m] = 0.f;
        dre[m] = dim[m] = 0.0;
      }
      for (int c0 = 0; c0 < cnt; c0 += 32) {
        const uint32_t mine = (c0 + lane < cnt) ? ev[o0 + c0 + lane] : 0u;
        const int ne = min(32, cnt - c0);
        for (int e = 0; e < ne; ++e) {
          const uint32_t w = __shfl_sync(0xffffffffu, mine, e);
          const uint64_t tau = w & 0x7fffffffu;
          const float sgn = (w & kSignBit) ? -1.f : 1.f;
          if (FORM == DDHF_FORM_NAIVE32) {
            const float tsec = (float)((int64_t)tau + t0) * 1e-6f;
#pragma unroll
            for (int m = 0; m < TPL; ++m) {
              const float f = (float)(g.a0 + (uint64_t)(j0 + lane + 32 * m) * g.da) *
                              (1e6f / (float)g.denom);  // cycles per second
              const float th = 6.2831853f * f * tsec;
              float s, c;
              sincosf(th, &s, &c);
              re[m] += sgn * c;
              im[m] -= sgn * s;
            }
            continue;
          }
          uint32_t r = (uint32_t)mod_barrett(a_first_mod * tau, g.denom, g.barrett);
          const uint32_t step = (uint32_t)mod_barrett(g.da32_mod * tau, g.denom, g.barrett);
          if (FORM == DDHF_FORM_RECUR) {
            float2 z = phasor_of_residue(r, g.two_over_denom);
            const float2 u = phasor_of_residue(step, g.two_over_denom);
            z.x *= sgn;
            z.y *= sgn;
#pragma unroll
            for (int m = 0; m < TPL; ++m) {
              re[m] += z.x;
              im[m] += z.y;
              z = cmul(z, u);
            }
          } else {
#pragma unroll
            for (int m = 0; m < TPL; ++m) {
              if (FORM == DDHF_FORM_F64) {
                double s, c;
                double x = 2.0 * (double)r / (double)D;
                if (x > 1.0) x -= 2.0;
                sincospi(x, &s, &c);
                dre[m] += (double)sgn * c;
                dim[m] -= (double)sgn * s;
              } else {
                const float2 z = phasor_of_residue(r, g.two_over_denom);
                if (FORM == DDHF_FORM_KAHAN) {
                  float yr = sgn * z.x - cre[m];
                  float tr = re[m] + yr;
                  cre[m] = (tr - re[m]) - yr;
                  re[m] = tr;
                  float yi = sgn * z.y - cim[m];
                  float ti = im[m] + yi;
                  cim[m] = (ti - im[m]) - yi;
                  im[m] = ti;
                } else {
                  re[m] += sgn * z.x;
                  im[m] += sgn * z.y;
                }
              }
              r += step;
              if (r >= D) r -= D;
            }
          }
        }
      }
#pragma unroll
      for (int m = 0; m < TPL; ++m) {
        const int j = j0 + lane + 32 * m;
        if (j < N) {
          float pv;
          if (FORM == DDHF_FORM_F64)
            pv = (float)(dre[m] * dre[m] + dim[m] * dim[m]);
          else
            pv = re[m] * re[m] + im[m] * im[m];
          P[a * (int64_t)N + j] = pv;
        }
      }
    }
  }
}

template <int FORM>
ddhf_status launch_plain_form(Ctx *c, float *P, int64_t cap_px, cudaStream_t s) {
  const Slot &sl = c->slots[0];
  const int blocks = c->num_sms * 8;
  const int N = c->grid.n_bins;
  if (N <= 32 * 8)
    k_plain<FORM, 8><<<blocks, kPlainThreads, 0, s>>>(sl.ev, sl.offsets, sl.active,
                                                      sl.counters, c->gconst,
                                                      sl.t0, P, cap_px, c->flags);
  else
    k_plain<FORM, 16><<<blocks, kPlainThreads, 0, s>>>(sl.ev, sl.offsets, sl.active,
                                                       sl.counters, c->gconst,
                                                       sl.t0, P, cap_px, c->flags);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

}  // namespace

ddhf_status launch_spectrum(Ctx *c, int form, float *P, int64_t cap_px, cudaStream_t s) {
  switch (form) {
    case DDHF_FORM_SINCOS: return launch_plain_form<DDHF_FORM_SINCOS>(c, P, cap_px, s);
    case DDHF_FORM_RECUR: return launch_plain_form<DDHF_FORM_RECUR>(c, P, cap_px, s);
    case DDHF_FORM_NAIVE32: return launch_plain_form<DDHF_FORM_NAIVE32>(c, P, cap_px, s);
    case DDHF_FORM_KAHAN: return launch_plain_form<DDHF_FORM_KAHAN>(c, P, cap_px, s);
    case DDHF_FORM_F64: return launch_plain_form<DDHF_FORM_F64>(c, P, cap_px, s);
    case DDHF_FORM_BLOCKED: return launch_blocked_spectrum(c, P, cap_px, s);
    case DDHF_FORM_HYBRID: return launch_hybrid_spectrum(c, P, cap_px, s);
    default:
      c->last_error = "unknown NDFT form";
      return DDHF_ERR_INVALID_ARG;
  }
}

}  // namespace ddhf
