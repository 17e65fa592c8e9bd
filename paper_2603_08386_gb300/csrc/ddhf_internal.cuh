// Internal declarations of libddhf: the context, workspace layout, device
// helpers and the launch functions each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/ddhf.h"

namespace ddhf {

constexpr int kMaxDigitBits = 11;  // at most 2048 bins per radix pass
constexpr int kBinThreads = 256;   // threads of a histogram block (one chunk)
constexpr int kScatThreads = 512;  // threads of a scatter block (one chunk, 16 warps)
constexpr int kScatItems = 16;     // consecutive 32-event rows per scatter warp
constexpr int kBinChunk = kScatThreads * kScatItems;  // 8192 events
constexpr int kMaxBandWords = 8;   // comb rank band up to 256 positions
constexpr uint32_t kSignBit = 0x80000000u;
constexpr size_t kCanaryBytes = 256;        // guard region on each side of a buffer
constexpr unsigned char kCanaryByte = 0xA5;
constexpr uint32_t kDropKey = 0xffffffffu;  // pre-packed sort input: pair not kept

// Invariant checks of the debug build (-DDDHF_BOUNDS_CHECK, made by
// build(debug=True)): a failed check raises DDHF_FLAG_INTERNAL and the caller
// skips the work item (never a trap or an assert). Release builds compile the
// checks away.
#ifdef DDHF_BOUNDS_CHECK
__device__ __forceinline__ bool ddhf_check(bool ok, uint32_t *flags) {
  if (!ok) atomicOr(flags, DDHF_FLAG_INTERNAL);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool ddhf_check(bool, uint32_t *) { return true; }
#endif

// Per-window binning output and per-pixel results (one "slot" per window).
struct Slot {
  uint32_t *ev = nullptr;       // [max_events] packed events, pixel-major
  uint32_t *offsets = nullptr;  // [npx + 1]
  uint32_t *active = nullptr;   // [npx] active pixel keys, ascending
  uint64_t *counters = nullptr; // [8] n_valid, n_dropped, n_active, n_in, n_heavy, terms,
                                // comb pixel cursor, n_rotor
  uint8_t *mask = nullptr;      // [npx] rotor mask
  int32_t *labels = nullptr;    // [npx]
  float *log_sf = nullptr;      // [npx] per active pixel (active-list order)
  float *snr = nullptr;         // [npx]
  int32_t *f0 = nullptr;        // [npx]
  int32_t *nbox = nullptr;      // [1]
  int64_t t0 = 0, window_us = 0;
};

// Device-visible view of the per-slot arrays for the persistent kernel.
struct SlotView {
  const uint32_t *ev;
  const uint32_t *offsets;
  const uint32_t *active;
  const uint64_t *counters;
  uint8_t *mask;
  float *log_sf;
  float *snr;
  int32_t *f0;
  int64_t t0;
};

// Parameters of the comb stage derived once from ddhf_params and the grid.
struct CombConst {
  int32_t N;        // bins
  int32_t M, d, h_min;
  int32_t w_lo;     // first candidate fundamental: max(1, d)
  int32_t w_hi;     // last candidate with M_valid >= h_min
  int32_t lo_r;     // first full rank of the median band
  int32_t bw;       // band width (positions)
  float ln_tau_sf;  // log(tau_sf) in FP32
  float tau_comb;
  float inv_N;      // 1 / N in FP32
};

struct GridConst {
  uint64_t a0, da, denom;
  uint64_t barrett;   // floor((2^64 - 1) / denom)
  uint64_t a0_mod;    // a0 mod denom
  uint64_t da_mod;    // da mod denom
  uint64_t da32_mod;  // 32 da mod denom
  int32_t N;
  int32_t nbr;        // b-rows of the blocked form: ceil(N / 32)
  float two_over_denom;
};

// The grid requirements of include/ddhf.h: a0 >= 0, da > 0, 0 < denom <
// 2^31, 1 <= n_bins <= 16384, and the last A row's frequency (bin n_bins - 1
// rounded up to a 32-bin row) below 2^32.
inline bool grid_ok(const ddhf_grid *g) {
  if (!g || g->a0 < 0 || g->da <= 0 || g->denom <= 0 || g->denom >= ((int64_t)1 << 31) ||
      g->n_bins < 1 || g->n_bins > 16384)
    return false;
  return (double)g->a0 + (double)g->da * (g->n_bins - 1 + 31) < 4294967296.0;
}

// Residues and reduction constants of a valid grid (one derivation shared by
// the context and the no-allocation entry point, so both evaluate the same
// phases).
inline GridConst make_grid_const(const ddhf_grid &g) {
  GridConst k;
  k.a0 = (uint64_t)g.a0;
  k.da = (uint64_t)g.da;
  k.denom = (uint64_t)g.denom;
  k.barrett = ~0ull / (uint64_t)g.denom;
  k.a0_mod = (uint64_t)g.a0 % (uint64_t)g.denom;
  k.da_mod = (uint64_t)g.da % (uint64_t)g.denom;
  k.da32_mod = ((uint64_t)g.da * 32ull) % (uint64_t)g.denom;
  k.N = g.n_bins;
  k.nbr = (g.n_bins + 31) / 32;
  k.two_over_denom = (float)(2.0 / (double)g.denom);
  return k;
}

struct SlideState;  // sliding-window spectra (slide.cu)

// Hybrid spectra (ndft_hybrid.cu): the grid rows a window needs, at most
// kHybMaxG, and the event-count threshold of the pixels that take the path.
constexpr int kHybMaxG = 1024;
constexpr int kHybDefaultMin = 64;  // DDHF_FORM_HYBRID when the tuning sets none
struct HybridPlan {
  bool ok = false;
  int64_t s = 0;      // grid spacing (us)
  int G = 0, Gp = 0;  // grid rows, rounded up to the K chunk
  int64_t thr = 0;    // pixels with at least thr events
  int64_t cap_h = 0;  // pixel capacity (column stride of the coefficient matrix)
};

struct Ctx {
  int W = 0, H = 0;
  int row0 = 0;  // sensor row of row 0 (a row band of a larger sensor)
  int64_t npx = 0;
  ddhf_grid grid{};
  ddhf_params params{};
  ddhf_tuning tuning{};
  int64_t max_events = 0;
  int max_windows = 0;
  int device = 0, num_sms = 0;
  int key_bits = 0, npass = 0;
  int digit_bits[3] = {0, 0, 0};
  int64_t nchunks = 0;
  // sort scratch
  uint32_t *keysA = nullptr, *valsA = nullptr, *keysB = nullptr, *valsB = nullptr;
  uint32_t *hist = nullptr;      // [2048 * nchunks]
  uint32_t *scan_part = nullptr; // block partials of the scans
  uint32_t *seg_lo = nullptr, *seg_hi = nullptr;  // [npx]
  uint64_t *packed = nullptr;    // [npx + 1]
  // per-window slots
  std::vector<Slot> slots;
  SlotView *d_views = nullptr;   // [max_windows]
  // work queue of the persistent kernel
  uint64_t *work = nullptr;      // [heavy_cap] heavy items (slot << 32 | active index)
  int64_t heavy_cap = 0;
  uint32_t *qctl = nullptr;      // [16] queue counters: [0] heavy count, [1-2] spectrum cursors,
                                 // [4] soft-comb cursor, [8] kept events of a binning, [9]
                                 // label count, [12-13] hybrid lists, [14] hybrid cursor
  // labelling / boxes scratch
  int32_t *box_root = nullptr;   // [npx]
  int32_t *box_tmp = nullptr;    // [npx * 6]
  uint32_t *flags = nullptr;     // [1] DDHF_FLAG_* bits
  // workspace buffers with guard bytes (kCanaryBytes of kCanaryByte before
  // and after each), checked by ddhf_get_stats
  struct Guarded {
    void *user;        // the pointer the kernels use
    size_t bytes;      // its size
  };
  std::vector<Guarded> guarded;
  float *soft_part = nullptr;    // [16 * npx + 16] soft-comb gradient partials
  float *pbuf = nullptr;         // [npx * pbuf_ld] spectra of one window (unfused detection)
  float *pbuf2 = nullptr;        // a second one for overlapped windows (tuning.overlap)
  cudaStream_t aux_stream = nullptr;  // comb kernels of overlapped windows
  cudaEvent_t ov_spec[2] = {nullptr, nullptr}, ov_comb[2] = {nullptr, nullptr};
  cudaEvent_t ov_fork = nullptr, ov_join = nullptr;
  int64_t pbuf_ld = 0;           // row stride of pbuf: n_bins rounded up to 4 floats
  CombConst comb{};
  GridConst gconst{};
  cudaStream_t last_stream = nullptr;
  bool binned = false;
  std::string last_error;
  // stage timing (tracing)
  bool timing = false;
  bool timing_recorded = false;
  bool timing_fused = true;
  int timing_windows = 0;
  // host-input detection (ddhf_detect_batch_host): two device staging sets
  // for one window's raw events, a copy stream and its events, and the
  // device box buffer of one window
  void *hstage[2] = {nullptr, nullptr};  // x int16, y int16, t int64, p int8 each
  int64_t hstage_cap = 0;                // events per window of a staging set
  int hstage_windows = 0;                // windows per staging set
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t h_ready[2] = {nullptr, nullptr}, h_free[2] = {nullptr, nullptr}, h_start = nullptr;
  cudaEvent_t h_win[32] = {};  // per staged window (2 sets of up to 16): its copy is done
  ddhf_box *hbox = nullptr;
  int32_t *hnbox = nullptr;
  int64_t hbox_cap = 0;                  // boxes the device box buffer holds
  int32_t hnbox_cap = 0;
  cudaEvent_t stage_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> win_ev;  // 5 per window (unfused path)
  // graph cache of ddhf_detect_batch
  int64_t graph_kernels = 0;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<uint8_t> graph_key;
  SlideState *slide = nullptr;  // ddhf_slide_begin .. ddhf_slide_end
  int loop_limit = 1 << 24;     // iterations of the bounded device loops (ddhf_set_loop_limit)
  // hybrid spectra (allocated once tuning.hybrid_min > 0 or DDHF_FORM_HYBRID is used)
  float4 *hyb_c = nullptr;       // [hyb_celems] grid coefficients (cr, ci, cr+ci, cr+ci)
  int64_t hyb_celems = 0;
  float2 *hyb_eri = nullptr;     // [kHybMaxG][hyb_np] table E of the grid product
  float *hyb_es = nullptr;       // [kHybMaxG][hyb_np] Re E + Im E
  float *hyb_dec = nullptr;      // [n_bins] deconvolution factors
  uint32_t *hyb_list = nullptr;  // [hyb_list_cap] active indices of the window's hybrid pixels
  int64_t hyb_list_cap = 0;
  int64_t hyb_np = 0;            // n_bins rounded up to the bin tile (128)
};

// ---------------------------------------------------------------- helpers

// An NVTX range (shown by profilers on the host timeline) around the launches
// of one stage; free when no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

#define DDHF_CUDA_TRY(ctx, call)                                                   \
  do {                                                                             \
    cudaError_t err__ = (call);                                                    \
    if (err__ != cudaSuccess) {                                                    \
      (ctx)->last_error = std::string(#call) + ": " + cudaGetErrorString(err__);   \
      return DDHF_ERR_CUDA;                                                        \
    }                                                                              \
  } while (0)

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// (x mod D) for x < 2^64 with a precomputed Barrett factor m = floor(2^64/D).
__device__ __forceinline__ uint64_t mod_barrett(uint64_t x, uint64_t D, uint64_t m) {
  uint64_t q = __umul64hi(x, m);
  uint64_t r = x - q * D;
  if (r >= D) r -= D;
  if (r >= D) r -= D;
  return r;
}

// sin(pi x) and cos(pi x) for |x| <= 1: x = y + q/2 with q = rint(2x) (the
// subtraction is exact), then sin(pi y) = y P(y^2) and cos(pi y) = 1 + y^2 C(y^2)
// on |y| <= 1/4 with polynomials fitted by weighted least squares (relative
// error, FP64) and rounded to FP32 (paper_2603_08386_gb300/fit_sincospi.py
// regenerates them); the quadrant q mod 4 swaps and negates.
// q is rounded by adding 1.5 * 2^23 (|2x| <= 2: round to nearest even, as
// rint does), whose float bits then hold q mod 4 in their lowest bits, so
// no conversion runs on the special-function pipe.
// Error within 2 ulp of the exact values (checked against sincospif).
__device__ __forceinline__ void sincospi_reduced(float x, float &s, float &c) {
  const float mq = __fadd_rn(__fmul_rn(2.f, x), 0x1.8p23f);
  const float q = __fsub_rn(mq, 0x1.8p23f);
  const float y = __fmaf_rn(-0.5f, q, x);
  const float t = __fmul_rn(y, y);
  float p = 0.0810556039f;
  p = __fmaf_rn(p, t, -0.599208117f);
  p = __fmaf_rn(p, t, 2.55016279f);
  p = __fmaf_rn(p, t, -5.16771269f);
  p = __fmaf_rn(p, t, 3.14159274f);
  const float sy = __fmul_rn(y, p);
  float k = 0.231556028f;
  k = __fmaf_rn(k, t, -1.33507168f);
  k = __fmaf_rn(k, t, 4.05870819f);
  k = __fmaf_rn(k, t, -4.93480206f);
  const float cy = __fmaf_rn(k, t, 1.f);
  const int iq = __float_as_int(mq) & 3;  // 0: (sy, cy), 1: (cy, -sy), 2: (-sy, -cy), 3: (-cy, sy)
  const float s0 = (iq & 1) ? cy : sy, c0 = (iq & 1) ? sy : cy;
  s = (iq & 2) ? -s0 : s0;
  c = (iq == 1 || iq == 2) ? -c0 : c0;
}

// e^{-2 pi i r / D} for an exact residue 0 <= r < D, via sin/cos(pi x) of the
// half-open turn x = 2r/D folded to [-1, 1]. D < 2^31, so r converts from 32
// bits (the same rounding as from 64 bits, without a 64-bit conversion, which
// runs on the FP64 pipe).
__device__ __forceinline__ float2 phasor_of_residue(uint64_t r, float two_over_denom) {
  float x = __fmul_rn((float)(uint32_t)r, two_over_denom);
  if (x > 1.0f) x = __fsub_rn(x, 2.0f);
  float s, c;
  sincospi_reduced(x, s, c);
  return make_float2(c, -s);
}

// Complex product with a fixed rounding sequence (no compiler contraction), so
// every kernel that generates the same phasors gets the same bits.
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)),
                     __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

// ---------------------------------------------------------- launch entry points
// bin.cu
ddhf_status bin_window(Ctx *c, int slot, const int16_t *x, const int16_t *y, const int64_t *t,
                       const int8_t *p, int64_t n, int64_t t0, int64_t win, cudaStream_t s);
ddhf_status bin_packed(Ctx *c, Slot &sl, const uint32_t *keys, const uint32_t *vals, int64_t n,
                       int n_min, int heavy_min, uint64_t *heavy_list, uint32_t *heavy_count,
                       int64_t heavy_cap, cudaStream_t s);
ddhf_status launch_scan_u32(Ctx *c, const uint32_t *in, uint32_t *out, int64_t n,
                            cudaStream_t s);
ddhf_status launch_scan_u64(Ctx *c, const uint64_t *in, uint64_t *out, int64_t n,
                            cudaStream_t s);
// slide.cu
void slide_free(Ctx *c);
// ndft_hybrid.cu
int64_t hybrid_spacing(const ddhf_grid &g);
HybridPlan hybrid_plan(const Ctx *c, int64_t window_us, int hybrid_min);
ddhf_status hybrid_alloc(Ctx *c);
void hybrid_free(Ctx *c);
ddhf_status launch_hybrid(Ctx *c, int slot, const HybridPlan &hp, float *P, int64_t cap_px,
                          int64_t ld, cudaStream_t s);
// ndft.cu
ddhf_status launch_spectrum(Ctx *c, int form, float *P, int64_t cap_px, cudaStream_t s);
ddhf_status launch_spectrum_slot(Ctx *c, int slot, float *P, int64_t cap_px, cudaStream_t s,
                                 int64_t ld);
ddhf_status launch_comb(Ctx *c, const float *P, int64_t cap_px, float *log_sf, float *snr,
                        int32_t *f0, uint8_t *mask, cudaStream_t s, int slot = 0,
                        int64_t ld = 0);
// comb_cplx.cu: the comb on complex rows F (row of active pixel a at
// F + active[a] * ldF) of slot 0's active list
ddhf_status launch_comb_cplx(Ctx *c, const float2 *F, int64_t ldF, float *log_sf, float *snr,
                             int32_t *f0, uint8_t *mask, cudaStream_t s);
ddhf_status launch_fused(Ctx *c, int n_slots, bool write_p, float *P, int64_t cap_px,
                         cudaStream_t s);
void set_bin_attributes();
// ccl.cu
ddhf_status launch_label(Ctx *c, const uint8_t *mask, int32_t *labels, uint64_t *n_fg,
                         cudaStream_t s);
ddhf_status launch_box_f0(Ctx *c, int slot, const ddhf_box *boxes, const int32_t *n_boxes,
                          int32_t cap, int32_t *f0_out, float *snr_out, float *med_hz,
                          cudaStream_t s);
ddhf_status launch_components(Ctx *c, const int32_t *labels, int32_t row0, ddhf_component *out,
                              int32_t cap, int32_t *n_out, cudaStream_t s);
ddhf_status launch_boxes(Ctx *c, const int32_t *labels, ddhf_box *boxes, int32_t cap,
                         int32_t *n_boxes, cudaStream_t s);

}  // namespace ddhf

struct ddhf_ctx {
  ddhf::Ctx c;
};
