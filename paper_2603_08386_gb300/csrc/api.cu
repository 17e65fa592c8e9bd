// C ABI of libddhf (declarations and contracts in include/ddhf.h): context
// creation, workspace layout, argument checks and the launch sequences of the
// per-window pipeline (Sec. 3.5) and its batched form.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>

#include "ddhf_internal.cuh"

namespace ddhf {
namespace {

__global__ void k_copy_counted(uint32_t *dst, const uint32_t *src, const uint64_t *count,
                               int64_t cap, uint32_t *flags) {
  const int64_t n = (int64_t)*count;
  if (blockIdx.x == 0 && threadIdx.x == 0 && n > cap) atomicOr(flags, DDHF_FLAG_CAPACITY);
  const int64_t m = n < cap ? n : cap;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_copy_counts(int64_t *dst, const uint64_t *counters) {
  if (threadIdx.x < 4) dst[threadIdx.x] = (int64_t)counters[threadIdx.x];
}

// Injected allocation failure (ddhf_debug_fail_alloc_after): while armed, the
// countdown reaches 0 at the allocation that fails.
std::atomic<int> g_fail_alloc_countdown{-1};

template <typename T>
ddhf_status dev_alloc(Ctx *c, T **p, size_t count) {
  void *q = nullptr;
  int left = g_fail_alloc_countdown.load();
  while (left >= 0 && !g_fail_alloc_countdown.compare_exchange_weak(left, left - 1)) {
  }
  if (left == 0) {
    c->last_error = "cudaMalloc: out of memory (injected failure)";
    return DDHF_ERR_CUDA;
  }
  // [kCanaryBytes guard][buffer, rounded up to 256 bytes][kCanaryBytes guard]
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  const size_t body = (bytes + 255) & ~(size_t)255;
  cudaError_t e = cudaMalloc(&q, body + 2 * kCanaryBytes);
  if (e == cudaSuccess) e = cudaMemset(q, kCanaryByte, kCanaryBytes);
  unsigned char *user = static_cast<unsigned char *>(q) + kCanaryBytes;
  if (e == cudaSuccess) e = cudaMemset(user + bytes, kCanaryByte, body - bytes + kCanaryBytes);
  if (e != cudaSuccess) {
    if (q) cudaFree(q);
    c->last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return DDHF_ERR_CUDA;
  }
  c->guarded.push_back(Ctx::Guarded{user, bytes});
  *p = reinterpret_cast<T *>(user);
  return DDHF_OK;
}

// Free a workspace buffer: through its guard region when dev_alloc made it.
void dev_free(Ctx *c, void *p) {
  if (!p) return;
  for (size_t i = 0; i < c->guarded.size(); ++i)
    if (c->guarded[i].user == p) {
      cudaFree(static_cast<unsigned char *>(p) - kCanaryBytes);
      c->guarded[i] = c->guarded.back();
      c->guarded.pop_back();
      return;
    }
  cudaFree(p);
}

// Guard check: every byte of the regions listed must still be kCanaryByte.
constexpr int kGuardBatch = 64;
struct GuardList {
  const unsigned char *p[kGuardBatch];
  uint32_t len[kGuardBatch];
  int n;
};
__global__ void k_check_guards(GuardList g, uint32_t *flags) {
  const int r = blockIdx.x;
  if (r >= g.n) return;
  bool bad = false;
  for (uint32_t i = threadIdx.x; i < g.len[r]; i += blockDim.x) bad |= g.p[r][i] != kCanaryByte;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, DDHF_FLAG_INTERNAL);
}

// Launch the guard check over every guarded buffer (head and tail regions).
cudaError_t check_guards(Ctx *c, cudaStream_t s) {
  GuardList g{};
  for (const Ctx::Guarded &b : c->guarded) {
    const unsigned char *u = static_cast<const unsigned char *>(b.user);
    const size_t body = (b.bytes + 255) & ~(size_t)255;
    const unsigned char *regions[2] = {u - kCanaryBytes, u + b.bytes};
    const size_t lens[2] = {kCanaryBytes, body - b.bytes + kCanaryBytes};
    for (int k = 0; k < 2; ++k) {
      g.p[g.n] = regions[k];
      g.len[g.n] = (uint32_t)lens[k];
      if (++g.n == kGuardBatch) {
        k_check_guards<<<kGuardBatch, 128, 0, s>>>(g, c->flags);
        g.n = 0;
      }
    }
  }
  if (g.n) k_check_guards<<<g.n, 128, 0, s>>>(g, c->flags);
  return cudaGetLastError();
}

#define DDHF_TRY(x)                      \
  do {                                   \
    ddhf_status st__ = (x);              \
    if (st__ != DDHF_OK) return st__;    \
  } while (0)

void free_all(Ctx *c) {
  slide_free(c);
  hybrid_free(c);
  auto F = [c](void *p) { dev_free(c, p); };
  F(c->keysA);
  F(c->valsA);
  F(c->keysB);
  F(c->valsB);
  F(c->hist);
  F(c->scan_part);
  F(c->seg_lo);
  F(c->seg_hi);
  F(c->packed);
  for (auto &s : c->slots) {
    F(s.ev);
    F(s.offsets);
    F(s.active);
    F(s.counters);
    F(s.mask);
    F(s.labels);
    F(s.log_sf);
    F(s.snr);
    F(s.f0);
    F(s.nbox);
  }
  c->slots.clear();
  F(c->d_views);
  F(c->work);
  F(c->qctl);
  F(c->box_root);
  F(c->box_tmp);
  F(c->flags);
  F(c->soft_part);
  F(c->pbuf);
  F(c->pbuf2);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  c->aux_stream = nullptr;
  for (cudaEvent_t *e : {&c->ov_spec[0], &c->ov_spec[1], &c->ov_comb[0], &c->ov_comb[1],
                         &c->ov_fork, &c->ov_join})
    if (*e) {
      cudaEventDestroy(*e);
      *e = nullptr;
    }
  F(c->hstage[0]);
  F(c->hstage[1]);
  F(c->hbox);
  F(c->hnbox);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  c->copy_stream = nullptr;
  for (cudaEvent_t *e : {&c->h_ready[0], &c->h_ready[1], &c->h_free[0], &c->h_free[1],
                         &c->h_start})
    if (*e) {
      cudaEventDestroy(*e);
      *e = nullptr;
    }
  for (cudaEvent_t &e : c->h_win)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  for (auto &e : c->stage_ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : c->win_ev)
    if (e) cudaEventDestroy(e);
  c->win_ev.clear();
}

void drop_graph(Ctx *c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  c->graph_key.clear();
}

ddhf_status fail(Ctx *c, ddhf_status st, const char *msg) {
  if (c) c->last_error = msg;
  return st;
}

int ceil_log2(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v) ++b;
  return b;
}

void derive_constants(Ctx *c) {
  const ddhf_grid &g = c->grid;
  c->gconst = make_grid_const(g);
  CombConst &cc = c->comb;
  const ddhf_params &p = c->params;
  const int N = g.n_bins;
  cc.N = N;
  cc.M = p.M;
  cc.d = p.d;
  cc.h_min = p.h_min;
  cc.w_lo = std::max(1, p.d);
  // largest w with M_valid(w) = min(M, (N-1-d)/w) >= h_min
  int whi = cc.w_lo - 1;
  if (N - 1 - p.d >= 1) {
    const int hm = std::min(p.h_min, p.M);
    if (p.h_min <= p.M && hm >= 1) whi = (N - 1 - p.d) / p.h_min;
  }
  cc.w_hi = whi;
  const int hmax = p.M * (2 * p.d + 1);
  int lo = (N - hmax - 1) / 2;
  if (N - hmax - 1 < 0) lo = 0;
  int hi = (N + hmax) / 2;
  if (hi > N - 1) hi = N - 1;
  cc.lo_r = lo;
  cc.bw = hi - lo + 1;
  cc.ln_tau_sf = (float)log((double)p.tau_sf);
  cc.inv_N = (float)(1.0 / (double)N);
  cc.tau_comb = p.tau_comb;
}

ddhf_status check_params(const ddhf_params *p) {
  if (!p) return DDHF_ERR_INVALID_ARG;
  if (p->M < 1 || p->d < 0 || p->h_min < 1 || p->n_min < 1 || p->A_min < 0 || !(p->alpha >= 0.0))
    return DDHF_ERR_INVALID_ARG;
  if (p->M * (2 * p->d + 1) > 254) return DDHF_ERR_UNSUPPORTED;
  if (!(p->tau_sf > 0.f) || !(p->tau_comb >= 0.f)) return DDHF_ERR_INVALID_ARG;
  return DDHF_OK;
}

ddhf_status check_window(Ctx *c, const void *x, const void *y, const void *t, const void *p,
                         int64_t n, int64_t window_us) {
  if (n < 0 || n > c->max_events) return fail(c, DDHF_ERR_INVALID_ARG, "n out of [0, max_events]");
  if (n > 0 && (!x || !y || !t || !p)) return fail(c, DDHF_ERR_INVALID_ARG, "null event array");
  if (window_us <= 0 || window_us >= ((int64_t)1 << 31))
    return fail(c, DDHF_ERR_INVALID_ARG, "window_us out of (0, 2^31)");
  return DDHF_OK;
}

ddhf_status write_views(Ctx *c) {
  std::vector<SlotView> v(c->max_windows);
  for (int i = 0; i < c->max_windows; ++i) {
    const Slot &s = c->slots[i];
    v[i] = SlotView{s.ev, s.offsets, s.active, s.counters, s.mask, s.log_sf, s.snr, s.f0};
  }
  DDHF_CUDA_TRY(c, cudaMemcpy(c->d_views, v.data(), sizeof(SlotView) * v.size(),
                              cudaMemcpyHostToDevice));
  return DDHF_OK;
}

// Binning of one window into a slot, appending its heavy pixels to the queue.
ddhf_status bin_into(Ctx *c, int slot, const int16_t *x, const int16_t *y, const int64_t *t,
                     const int8_t *p, int64_t n, int64_t t0, int64_t win, cudaStream_t s) {
  return bin_window(c, slot, x, y, t, p, n, t0, win, s);
}

// Stage event: an external event node while the stream is being captured into
// a graph, a plain record otherwise.
cudaError_t record_event(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  if (cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
  return cudaEventRecord(ev, s);
}

cudaError_t record_stage(Ctx *c, int i, cudaStream_t s) { return record_event(c->stage_ev[i], s); }

// ready (nullable): per window, an event that `s` waits for before binning it
// (the host-buffer path: that window's copy).
ddhf_status run_detect(Ctx *c, const ddhf_window *wins, int nw, ddhf_box *boxes, int32_t cap,
                       int32_t *n_boxes_dev, uint8_t *masks_out, cudaStream_t s,
                       const cudaEvent_t *ready = nullptr) {
  if (c->timing) DDHF_CUDA_TRY(c, record_stage(c, 0, s));
  const bool fused = c->tuning.fuse != 0 || !c->pbuf;
  if (fused) {
    DDHF_CUDA_TRY(c, cudaMemsetAsync(c->qctl, 0, sizeof(uint32_t), s));  // heavy count
    for (int w = 0; w < nw; ++w) {
      const ddhf_window &W = wins[w];
      NvtxRange r("ddhf binning");
      DDHF_CUDA_TRY(c, cudaMemsetAsync(c->slots[w].mask, 0, c->npx, s));
      if (ready) DDHF_CUDA_TRY(c, cudaStreamWaitEvent(s, ready[w], 0));
      DDHF_TRY(bin_into(c, w, W.x, W.y, W.t_us, W.p, W.n, W.t0_us, W.window_us, s));
    }
    if (c->timing) DDHF_CUDA_TRY(c, record_stage(c, 1, s));
    {
      NvtxRange r("ddhf spectra + comb (fused)");
      DDHF_TRY(launch_fused(c, nw, true, nullptr, 0, s));
    }
  } else if (c->tuning.overlap && c->pbuf2 && nw > 1) {
    // per window as below, but the comb kernel of window w runs on the aux
    // stream while the main stream bins window w + 1 and computes its spectra
    // into the other buffer; a buffer is reused once the comb two windows
    // back has read it
    cudaStream_t b = c->aux_stream;
    DDHF_CUDA_TRY(c, cudaEventRecord(c->ov_fork, s));
    DDHF_CUDA_TRY(c, cudaStreamWaitEvent(b, c->ov_fork, 0));
    for (int w = 0; w < nw; ++w) {
      const ddhf_window &W = wins[w];
      float *buf = (w & 1) ? c->pbuf2 : c->pbuf;
      cudaEvent_t *we = c->timing ? &c->win_ev[5 * w] : nullptr;
      if (we) DDHF_CUDA_TRY(c, record_event(we[0], s));
      {
        NvtxRange r("ddhf binning");
        DDHF_CUDA_TRY(c, cudaMemsetAsync(c->qctl, 0, sizeof(uint32_t), s));
        if (ready) DDHF_CUDA_TRY(c, cudaStreamWaitEvent(s, ready[w], 0));
      DDHF_TRY(bin_into(c, w, W.x, W.y, W.t_us, W.p, W.n, W.t0_us, W.window_us, s));
      }
      if (we) DDHF_CUDA_TRY(c, record_event(we[1], s));
      if (w >= 2) DDHF_CUDA_TRY(c, cudaStreamWaitEvent(s, c->ov_comb[w & 1], 0));
      {
        NvtxRange r("ddhf spectra");
        DDHF_TRY(launch_spectrum_slot(c, w, buf, c->npx, s, c->pbuf_ld));
      }
      if (we) DDHF_CUDA_TRY(c, record_event(we[2], s));
      DDHF_CUDA_TRY(c, cudaEventRecord(c->ov_spec[w & 1], s));
      DDHF_CUDA_TRY(c, cudaStreamWaitEvent(b, c->ov_spec[w & 1], 0));
      Slot &sl = c->slots[w];
      if (we) DDHF_CUDA_TRY(c, record_event(we[3], b));
      {
        NvtxRange r("ddhf comb");
        DDHF_TRY(launch_comb(c, buf, c->npx, sl.log_sf, sl.snr, sl.f0, sl.mask, b, w,
                             c->pbuf_ld));
      }
      if (we) DDHF_CUDA_TRY(c, record_event(we[4], b));
      DDHF_CUDA_TRY(c, cudaEventRecord(c->ov_comb[w & 1], b));
    }
    DDHF_CUDA_TRY(c, cudaEventRecord(c->ov_join, b));
    DDHF_CUDA_TRY(c, cudaStreamWaitEvent(s, c->ov_join, 0));
  } else {
    // per window: binning (own heavy list), spectra into the context buffer, comb
    for (int w = 0; w < nw; ++w) {
      const ddhf_window &W = wins[w];
      cudaEvent_t *we = c->timing ? &c->win_ev[5 * w] : nullptr;
      if (we) DDHF_CUDA_TRY(c, record_event(we[0], s));
      {
        NvtxRange r("ddhf binning");
        DDHF_CUDA_TRY(c, cudaMemsetAsync(c->qctl, 0, sizeof(uint32_t), s));
        if (ready) DDHF_CUDA_TRY(c, cudaStreamWaitEvent(s, ready[w], 0));
      DDHF_TRY(bin_into(c, w, W.x, W.y, W.t_us, W.p, W.n, W.t0_us, W.window_us, s));
      }
      if (we) DDHF_CUDA_TRY(c, record_event(we[1], s));
      Slot &sl = c->slots[w];
      {
        NvtxRange r("ddhf spectra");
        DDHF_TRY(launch_spectrum_slot(c, w, c->pbuf, c->npx, s, c->pbuf_ld));
      }
      if (we) DDHF_CUDA_TRY(c, record_event(we[2], s));
      if (we) DDHF_CUDA_TRY(c, record_event(we[3], s));
      {
        NvtxRange r("ddhf comb");
        DDHF_TRY(launch_comb(c, c->pbuf, c->npx, sl.log_sf, sl.snr, sl.f0, sl.mask, s, w,
                             c->pbuf_ld));
      }
      if (we) DDHF_CUDA_TRY(c, record_event(we[4], s));
    }
  }
  c->timing_fused = fused;
  c->timing_windows = nw;
  if (c->timing) DDHF_CUDA_TRY(c, record_stage(c, 2, s));
  for (int w = 0; w < nw; ++w) {
    Slot &sl = c->slots[w];
    NvtxRange r("ddhf labels + boxes");
    DDHF_TRY(launch_label(c, sl.mask, sl.labels, sl.counters + 7, s));
    DDHF_TRY(launch_boxes(c, sl.labels, boxes + (int64_t)w * cap, cap, sl.nbox, s));
    DDHF_CUDA_TRY(c, cudaMemcpyAsync(n_boxes_dev + w, sl.nbox, sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, s));
    if (masks_out)
      DDHF_CUDA_TRY(c, cudaMemcpyAsync(masks_out + (int64_t)w * c->npx, sl.mask, c->npx,
                                       cudaMemcpyDeviceToDevice, s));
  }
  if (c->timing) {
    DDHF_CUDA_TRY(c, record_stage(c, 3, s));
    c->timing_recorded = true;
  }
  return DDHF_OK;
}

}  // namespace
}  // namespace ddhf

using namespace ddhf;

extern "C" {

const char *ddhf_status_string(ddhf_status s) {
  switch (s) {
    case DDHF_OK: return "ok";
    case DDHF_ERR_INVALID_ARG: return "invalid argument";
    case DDHF_ERR_CUDA: return "CUDA error";
    case DDHF_ERR_CAPACITY: return "capacity exceeded";
    case DDHF_ERR_TIMEOUT: return "device-side wait limit reached";
    case DDHF_ERR_UNSUPPORTED: return "unsupported configuration";
    case DDHF_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

ddhf_status ddhf_debug_corrupt_guard(ddhf_ctx *h, int32_t index) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (index < 0 || index >= (int32_t)c->guarded.size())
    return fail(c, DDHF_ERR_INVALID_ARG, "guard index out of range");
  const Ctx::Guarded &b = c->guarded[index];
  DDHF_CUDA_TRY(c, cudaMemset(static_cast<unsigned char *>(b.user) + b.bytes, 0, 1));
  return DDHF_OK;
}

ddhf_status ddhf_debug_fail_alloc_after(int32_t n) {
  if (n < -1) return DDHF_ERR_INVALID_ARG;
  g_fail_alloc_countdown.store(n);
  return DDHF_OK;
}

ddhf_status ddhf_default_params(ddhf_params *out) {
  if (!out) return DDHF_ERR_INVALID_ARG;
  out->tau_sf = 0.89f;
  out->tau_comb = 1.5f;
  out->M = 4;
  out->d = 3;
  out->h_min = 4;
  out->n_min = 6;
  out->A_min = 147;
  out->polarity_01 = 0;
  out->alpha = 19.05;
  return DDHF_OK;
}

ddhf_status ddhf_create(int32_t W, int32_t H, const ddhf_grid *grid, const ddhf_params *params,
                        int64_t max_events, int32_t max_windows, ddhf_ctx **out) {
  if (!out || !grid || !params) return DDHF_ERR_INVALID_ARG;
  *out = nullptr;
  if (W < 1 || H < 1 || W > 32767 || H > 32767 || (int64_t)W * H > ((int64_t)1 << 26))
    return DDHF_ERR_INVALID_ARG;
  if (max_events < 0 || max_events >= ((int64_t)1 << 31) || max_windows < 1 || max_windows > 4096)
    return DDHF_ERR_INVALID_ARG;
  if (!grid_ok(grid)) return DDHF_ERR_INVALID_ARG;
  ddhf_status ps = check_params(params);
  if (ps != DDHF_OK) return ps;
  ddhf_ctx *h = new (std::nothrow) ddhf_ctx();
  if (!h) return DDHF_ERR_CUDA;
  Ctx *c = &h->c;
  c->W = W;
  c->H = H;
  c->npx = (int64_t)W * H;
  c->grid = *grid;
  c->params = *params;
  c->max_events = max_events;
  c->max_windows = max_windows;
  c->tuning = ddhf_tuning{1024, 4, 0, 0, 0, 0, 0};
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete h;
    return DDHF_ERR_CUDA;
  }
  c->key_bits = std::max(1, ceil_log2(c->npx));
  c->npass = (c->key_bits + kMaxDigitBits - 1) / kMaxDigitBits;
  for (int i = 0, rem = c->key_bits; i < c->npass; ++i) {
    int b = (rem + (c->npass - i) - 1) / (c->npass - i);
    c->digit_bits[i] = b;
    rem -= b;
  }
  c->nchunks = std::max<int64_t>(1, ceil_div(max_events, kBinChunk));
  derive_constants(c);
  const int64_t npx = c->npx;
  const int64_t nev = std::max<int64_t>(max_events, 1);
  const int64_t hist_n = (int64_t)(1 << kMaxDigitBits) * c->nchunks;
  const int64_t scan_n = std::max<int64_t>(hist_n, 2 * (npx + 1));
  const int64_t heavy_cap = (int64_t)max_windows * std::min<int64_t>(npx, ceil_div(nev, 32));
  ddhf_status st = DDHF_OK;
#define A(ptr, n) \
  if (st == DDHF_OK) st = dev_alloc(c, &(ptr), (size_t)(n))
  A(c->keysA, nev);
  A(c->valsA, nev);
  A(c->keysB, nev);
  A(c->valsB, nev);
  A(c->hist, hist_n);
  A(c->scan_part, scan_n / 4000 + 256);
  A(c->seg_lo, npx);
  A(c->seg_hi, npx);
  A(c->packed, npx + 1);
  c->slots.resize(max_windows);
  for (int i = 0; i < max_windows && st == DDHF_OK; ++i) {
    Slot &s = c->slots[i];
    A(s.ev, nev);
    A(s.offsets, npx + 1);
    A(s.active, npx);
    A(s.counters, 8);
    A(s.mask, npx);
    A(s.labels, npx);
    A(s.log_sf, npx);
    A(s.snr, npx);
    A(s.f0, npx);
    A(s.nbox, 1);
    if (st == DDHF_OK) {
      cudaMemset(s.counters, 0, 8 * sizeof(uint64_t));
      cudaMemset(s.offsets, 0, (npx + 1) * sizeof(uint32_t));
      cudaMemset(s.mask, 0, npx);
    }
  }
  A(c->d_views, max_windows);
  c->heavy_cap = heavy_cap;
  A(c->work, heavy_cap);
  A(c->qctl, 16);
  A(c->box_root, npx);
  A(c->box_tmp, 15 * npx);
  A(c->flags, 1);
  A(c->soft_part, 16 * npx + 16);
  c->pbuf_ld = ((int64_t)grid->n_bins + 3) & ~(int64_t)3;  // 16-byte aligned rows
  if (grid->n_bins <= 4096) {
    A(c->pbuf, npx * c->pbuf_ld);
  } else if (st == DDHF_OK) {
    // a large grid's spectrum buffer (W*H rows of n_bins floats) is optional:
    // without it detection runs the fused kernel
    if (cudaMalloc(&c->pbuf, (size_t)npx * c->pbuf_ld * sizeof(float)) != cudaSuccess) {
      c->pbuf = nullptr;
      cudaGetLastError();
    }
  }
#undef A
  if (st == DDHF_OK) {
    cudaMemset(c->qctl, 0, 16 * sizeof(uint32_t));
    cudaMemset(c->flags, 0, sizeof(uint32_t));
    st = write_views(c);
  }
  if (st == DDHF_OK) {
    set_bin_attributes();
    if (cudaDeviceSynchronize() != cudaSuccess) st = DDHF_ERR_CUDA;
  }
  if (st != DDHF_OK) {
    free_all(c);
    delete h;
    return st;
  }
  *out = h;
  return DDHF_OK;
}

ddhf_status ddhf_destroy(ddhf_ctx *h) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  free_all(&h->c);
  delete h;
  return DDHF_OK;
}

ddhf_status ddhf_set_tuning(ddhf_ctx *h, const ddhf_tuning *t) {
  if (!h || !t) return DDHF_ERR_INVALID_ARG;
  const int r = t->rows_per_lane;
  if (t->heavy_min < 32 || (t->warps_per_block != 2 && t->warps_per_block != 4 &&
                            t->warps_per_block != 8) ||
      t->blocks_per_sm < 0 || t->blocks_per_sm > 32 ||
      !(r == 0 || r == 1 || r == 2 || r == 4 || r == 6 || r == 8) ||
      (t->fuse != 0 && t->fuse != 1) || (t->overlap != 0 && t->overlap != 1) ||
      t->hybrid_min < 0)
    return fail(&h->c, DDHF_ERR_INVALID_ARG, "tuning out of range");
  Ctx *c = &h->c;
  if (t->hybrid_min > 0) {
    const ddhf_status hs = hybrid_alloc(c);
    if (hs != DDHF_OK) return hs;
  }
  if (t->overlap && c->pbuf && !c->pbuf2) {
    // second spectrum buffer, a stream and events for overlapped windows
    if (cudaMalloc(&c->pbuf2, (size_t)c->npx * c->pbuf_ld * sizeof(float)) != cudaSuccess) {
      c->pbuf2 = nullptr;
      cudaGetLastError();
      return fail(c, DDHF_ERR_CUDA, "no memory for a second spectrum buffer");
    }
    int lo_prio = 0, hi_prio = 0;
    DDHF_CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    DDHF_CUDA_TRY(c, cudaStreamCreateWithPriority(&c->aux_stream, cudaStreamNonBlocking, hi_prio));
    for (cudaEvent_t *e : {&c->ov_spec[0], &c->ov_spec[1], &c->ov_comb[0], &c->ov_comb[1],
                           &c->ov_fork, &c->ov_join})
      DDHF_CUDA_TRY(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  c->tuning = *t;
  drop_graph(c);
  return DDHF_OK;
}

ddhf_status ddhf_set_loop_limit(ddhf_ctx *h, int32_t limit) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  if (limit < 1) return fail(&h->c, DDHF_ERR_INVALID_ARG, "loop limit < 1");
  h->c.loop_limit = limit;
  drop_graph(&h->c);
  return DDHF_OK;
}

ddhf_status ddhf_enable_stage_timing(ddhf_ctx *h, int32_t enable) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (enable && !c->stage_ev[0]) {
    for (auto &e : c->stage_ev) DDHF_CUDA_TRY(c, cudaEventCreate(&e));
    c->win_ev.assign(5 * (size_t)c->max_windows, nullptr);
    for (auto &e : c->win_ev) DDHF_CUDA_TRY(c, cudaEventCreate(&e));
  }
  if ((bool)enable != c->timing) drop_graph(c);
  c->timing = enable != 0;
  c->timing_recorded = false;
  return DDHF_OK;
}

ddhf_status ddhf_stage_times(ddhf_ctx *h, float *out_ms) {
  if (!h || !out_ms) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!c->timing || !c->timing_recorded) return fail(c, DDHF_ERR_STATE, "no timed detection");
  DDHF_CUDA_TRY(c, cudaEventSynchronize(c->stage_ev[3]));
  for (int i = 0; i < 5; ++i) out_ms[i] = 0.f;
  if (c->timing_fused) {
    for (int i = 0; i < 3; ++i)
      DDHF_CUDA_TRY(c, cudaEventElapsedTime(&out_ms[i], c->stage_ev[i], c->stage_ev[i + 1]));
  } else {
    for (int w = 0; w < c->timing_windows; ++w) {
      float b, sp, cb;
      const cudaEvent_t *we = &c->win_ev[5 * w];
      DDHF_CUDA_TRY(c, cudaEventElapsedTime(&b, we[0], we[1]));
      DDHF_CUDA_TRY(c, cudaEventElapsedTime(&sp, we[1], we[2]));
      DDHF_CUDA_TRY(c, cudaEventElapsedTime(&cb, we[3], we[4]));
      out_ms[0] += b;
      out_ms[3] += sp;
      out_ms[4] += cb;
    }
    out_ms[1] = out_ms[3] + out_ms[4];
    DDHF_CUDA_TRY(c, cudaEventElapsedTime(&out_ms[2], c->stage_ev[2], c->stage_ev[3]));
  }
  return DDHF_OK;
}

ddhf_status ddhf_set_params(ddhf_ctx *h, const ddhf_params *params) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  const ddhf_status st = check_params(params);
  if (st != DDHF_OK) return fail(c, st, "parameters out of range");
  c->params = *params;
  derive_constants(c);
  drop_graph(c);
  return DDHF_OK;
}

ddhf_status ddhf_get_tuning(const ddhf_ctx *h, ddhf_tuning *out) {
  if (!h || !out) return DDHF_ERR_INVALID_ARG;
  *out = h->c.tuning;
  return DDHF_OK;
}

ddhf_status ddhf_bin_events(ddhf_ctx *h, const int16_t *x, const int16_t *y, const int64_t *t_us,
                            const int8_t *p, int64_t n, int64_t t0_us, int64_t window_us,
                            ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  DDHF_TRY(check_window(c, x, y, t_us, p, n, window_us));
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(c->qctl, 0, sizeof(uint32_t), s));
  DDHF_TRY(bin_into(c, 0, x, y, t_us, p, n, t0_us, window_us, s));
  c->binned = true;
  return DDHF_OK;
}

ddhf_status ddhf_export_csr(ddhf_ctx *h, uint32_t *offsets, uint32_t *ev, int64_t cap_ev,
                            uint32_t *active, int64_t *counts, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!c->binned) return fail(c, DDHF_ERR_STATE, "no binned window");
  if (cap_ev < 0) return fail(c, DDHF_ERR_INVALID_ARG, "cap_ev < 0");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const Slot &sl = c->slots[0];
  const uint64_t *cnt = sl.counters;
  if (offsets)
    DDHF_CUDA_TRY(c, cudaMemcpyAsync(offsets, sl.offsets, (c->npx + 1) * sizeof(uint32_t),
                                     cudaMemcpyDeviceToDevice, s));
  if (ev) {
    k_copy_counted<<<c->num_sms * 4, 256, 0, s>>>(ev, sl.ev, cnt + 0, cap_ev, c->flags);
    DDHF_CUDA_TRY(c, cudaGetLastError());
  }
  if (active) {
    k_copy_counted<<<c->num_sms * 4, 256, 0, s>>>(active, sl.active, cnt + 2, c->npx, c->flags);
    DDHF_CUDA_TRY(c, cudaGetLastError());
  }
  if (counts) {
    k_copy_counts<<<1, 32, 0, s>>>(counts, cnt);
    DDHF_CUDA_TRY(c, cudaGetLastError());
  }
  return DDHF_OK;
}

ddhf_status ddhf_power_spectrum(ddhf_ctx *h, int32_t form, float *P, int64_t cap_px,
                                ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!c->binned) return fail(c, DDHF_ERR_STATE, "no binned window");
  if (!P || cap_px < 0) return fail(c, DDHF_ERR_INVALID_ARG, "bad spectrum buffer");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return launch_spectrum(c, form, P, cap_px, s);
}

ddhf_status ddhf_comb_score(ddhf_ctx *h, const float *P, int64_t cap_px, float *log_sf, float *snr,
                            int32_t *f0_bin, uint8_t *mask, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!c->binned) return fail(c, DDHF_ERR_STATE, "no binned window");
  if (!P || !mask || cap_px < 0) return fail(c, DDHF_ERR_INVALID_ARG, "null P or mask");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return launch_comb(c, P, cap_px, log_sf, snr, f0_bin, mask, s);
}

ddhf_status ddhf_label(ddhf_ctx *h, const uint8_t *mask, int32_t *labels, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!mask || !labels) return fail(c, DDHF_ERR_INVALID_ARG, "null mask or labels");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return launch_label(c, mask, labels, c->slots[0].counters + 7, s);
}

ddhf_status ddhf_boxes(ddhf_ctx *h, const int32_t *labels, ddhf_box *boxes, int32_t cap,
                       int32_t *n_boxes_dev, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!labels || !n_boxes_dev || cap < 0 || (cap > 0 && !boxes))
    return fail(c, DDHF_ERR_INVALID_ARG, "bad box arguments");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return launch_boxes(c, labels, boxes, cap, n_boxes_dev, s);
}

ddhf_status ddhf_set_row_offset(ddhf_ctx *h, int32_t row0) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (row0 < 0 || (int64_t)row0 + c->H > 32767)
    return fail(c, DDHF_ERR_INVALID_ARG, "row offset out of range");
  c->row0 = row0;
  drop_graph(c);
  return DDHF_OK;
}

ddhf_status ddhf_components(ddhf_ctx *h, const int32_t *labels, int32_t row0,
                            ddhf_component *comps, int32_t cap, int32_t *n_dev,
                            ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!labels || !n_dev || cap < 0 || (cap > 0 && !comps) || row0 < 0 ||
      (int64_t)row0 * c->W + c->npx > INT32_MAX)
    return fail(c, DDHF_ERR_INVALID_ARG, "bad component arguments");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return launch_components(c, labels, row0, comps, cap, n_dev, s);
}

ddhf_status ddhf_detect(ddhf_ctx *h, const int16_t *x, const int16_t *y, const int64_t *t_us,
                        const int8_t *p, int64_t n, int64_t t0_us, int64_t window_us,
                        ddhf_box *boxes, int32_t cap, int32_t *n_boxes_dev, uint8_t *mask_out,
                        ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  DDHF_TRY(check_window(c, x, y, t_us, p, n, window_us));
  if (!n_boxes_dev || cap < 0 || (cap > 0 && !boxes))
    return fail(c, DDHF_ERR_INVALID_ARG, "bad box arguments");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  ddhf_window w{x, y, t_us, p, n, t0_us, window_us};
  DDHF_TRY(run_detect(c, &w, 1, boxes, cap, n_boxes_dev, mask_out, s));
  c->binned = true;
  return DDHF_OK;
}

ddhf_status ddhf_detect_batch(ddhf_ctx *h, const ddhf_window *wins, int32_t n_windows,
                              ddhf_box *boxes, int32_t cap, int32_t *n_boxes_dev,
                              uint8_t *masks_out, int32_t use_graph, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!wins || n_windows < 1 || n_windows > c->max_windows)
    return fail(c, DDHF_ERR_INVALID_ARG, "n_windows out of [1, max_windows]");
  if (!n_boxes_dev || cap < 0 || (cap > 0 && !boxes))
    return fail(c, DDHF_ERR_INVALID_ARG, "bad box arguments");
  for (int w = 0; w < n_windows; ++w)
    DDHF_TRY(check_window(c, wins[w].x, wins[w].y, wins[w].t_us, wins[w].p, wins[w].n,
                          wins[w].window_us));
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  if (!use_graph) {
    DDHF_TRY(run_detect(c, wins, n_windows, boxes, cap, n_boxes_dev, masks_out, s));
    c->binned = true;
    return DDHF_OK;
  }
  // graph keyed by every argument value
  std::vector<uint8_t> key(sizeof(ddhf_window) * n_windows + 64);
  memcpy(key.data(), wins, sizeof(ddhf_window) * n_windows);
  uint8_t *tail = key.data() + sizeof(ddhf_window) * n_windows;
  memcpy(tail, &boxes, sizeof(boxes));
  memcpy(tail + 8, &cap, sizeof(cap));
  memcpy(tail + 16, &n_boxes_dev, sizeof(n_boxes_dev));
  memcpy(tail + 24, &masks_out, sizeof(masks_out));
  memcpy(tail + 32, &s, sizeof(s));
  if (!c->graph_exec || key != c->graph_key) {
    if (c->graph_exec) {
      cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
    }
    cudaStream_t cap_s = nullptr;
    DDHF_CUDA_TRY(c, cudaStreamCreateWithFlags(&cap_s, cudaStreamNonBlocking));
    // kernels read tuning-dependent attributes at launch; set them before capture
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap_s, cudaStreamCaptureModeThreadLocal);
    ddhf_status st = DDHF_OK;
    if (e == cudaSuccess) st = run_detect(c, wins, n_windows, boxes, cap, n_boxes_dev, masks_out, cap_s);
    cudaError_t e2 = cudaStreamEndCapture(cap_s, &graph);
    cudaStreamDestroy(cap_s);
    if (e != cudaSuccess || e2 != cudaSuccess || st != DDHF_OK) {
      if (graph) cudaGraphDestroy(graph);
      if (st == DDHF_OK) {
        c->last_error = std::string("graph capture: ") +
                        cudaGetErrorString(e != cudaSuccess ? e : e2);
        st = DDHF_ERR_CUDA;
      }
      return st;
    }
    size_t nn = 0;
    c->graph_kernels = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess) {
        for (size_t i = 0; i < nn; ++i) {
          cudaGraphNodeType ty;
          if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
            c->graph_kernels += 1;
        }
      }
    }
    e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->graph_exec = nullptr;
      c->last_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
      return DDHF_ERR_CUDA;
    }
    c->graph_key = key;
  }
  DDHF_CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, s));
  c->binned = true;
  return DDHF_OK;
}

// Windows per group of ddhf_detect_batch_host.
constexpr int kHostGroup = 16;
static_assert(2 * kHostGroup <= (int)(sizeof(Ctx::h_win) / sizeof(cudaEvent_t)),
              "one copy event per staged window");

// Stage sizes of one window's raw events: x, y int16, t int64, p int8.
static int64_t host_stage_bytes(int64_t n) {
  const int64_t a = (2 * n + 255) & ~(int64_t)255;
  return 2 * a + ((8 * n + 255) & ~(int64_t)255) + ((n + 255) & ~(int64_t)255);
}

ddhf_status ddhf_detect_batch_host(ddhf_ctx *h, const ddhf_window *wins, int32_t n_windows,
                                   ddhf_box *boxes_host, int32_t cap, int32_t *n_boxes_host,
                                   uint8_t *masks_host, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (!wins || n_windows < 1) return fail(c, DDHF_ERR_INVALID_ARG, "need at least one window");
  if (!n_boxes_host || cap < 0 || (cap > 0 && !boxes_host))
    return fail(c, DDHF_ERR_INVALID_ARG, "bad box arguments");
  for (int w = 0; w < n_windows; ++w)
    DDHF_TRY(check_window(c, wins[w].x, wins[w].y, wins[w].t_us, wins[w].p, wins[w].n,
                          wins[w].window_us));
  // windows go through in groups of G (up to kHostGroup, at most max_windows)
  // by the batched detection; the next group's events are copied meanwhile
  const int G = std::min<int>(std::min(n_windows, kHostGroup), c->max_windows);
  const int64_t per_win = host_stage_bytes(std::max<int64_t>(c->max_events, 1));
  // workspace: two staging sets of G windows, box buffers for G x cap (grown on demand)
  if (c->hstage_cap < c->max_events || c->hstage_windows < G) {
    for (auto &p : c->hstage) {
      if (p) cudaFree(p);
      p = nullptr;
      DDHF_CUDA_TRY(c, cudaMalloc(&p, (size_t)per_win * G));
    }
    c->hstage_cap = c->max_events;
    c->hstage_windows = G;
  }
  const int64_t box_need = (int64_t)std::max(cap, 1) * G;
  if (c->hbox_cap < box_need) {
    if (c->hbox) cudaFree(c->hbox);
    c->hbox = nullptr;
    DDHF_CUDA_TRY(c, cudaMalloc(&c->hbox, sizeof(ddhf_box) * box_need));
    c->hbox_cap = box_need;
  }
  if (c->hnbox_cap < G) {
    if (c->hnbox) cudaFree(c->hnbox);
    c->hnbox = nullptr;
    DDHF_CUDA_TRY(c, cudaMalloc(&c->hnbox, sizeof(int32_t) * G));
    c->hnbox_cap = G;
  }
  if (!c->copy_stream)
    DDHF_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  for (cudaEvent_t *e : {&c->h_ready[0], &c->h_ready[1], &c->h_free[0], &c->h_free[1],
                         &c->h_start})
    if (!*e) DDHF_CUDA_TRY(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  for (cudaEvent_t &e : c->h_win)
    if (!e) DDHF_CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaStream_t s = (cudaStream_t)stream;
  cudaStream_t cs = c->copy_stream;
  c->last_stream = s;
  // the copies are ordered after the caller's earlier work on `stream`
  DDHF_CUDA_TRY(c, cudaEventRecord(c->h_start, s));
  DDHF_CUDA_TRY(c, cudaStreamWaitEvent(cs, c->h_start, 0));
  const int64_t ab2 = (2 * c->hstage_cap + 255) & ~(int64_t)255;
  const int64_t ab8 = (8 * c->hstage_cap + 255) & ~(int64_t)255;
  ddhf_window dw[kHostGroup];
  // each window's binning waits only for its own copy, so the first group
  // starts once its first window is in
  for (int g0 = 0, k = 0; g0 < n_windows; g0 += G, ++k) {
    const int b = k & 1;
    const int ng = std::min(G, n_windows - g0);
    // group k's events into staging set b once group k - 2 has finished with it
    if (k >= 2) DDHF_CUDA_TRY(c, cudaStreamWaitEvent(cs, c->h_free[b], 0));
    for (int i = 0; i < ng; ++i) {
      const ddhf_window &W = wins[g0 + i];
      const int64_t n = W.n;
      char *base = static_cast<char *>(c->hstage[b]) + (int64_t)i * per_win;
      int16_t *dx = reinterpret_cast<int16_t *>(base);
      int16_t *dy = reinterpret_cast<int16_t *>(base + ab2);
      int64_t *dt = reinterpret_cast<int64_t *>(base + 2 * ab2);
      int8_t *dp = reinterpret_cast<int8_t *>(base + 2 * ab2 + ab8);
      if (n > 0) {
        DDHF_CUDA_TRY(c, cudaMemcpyAsync(dx, W.x, 2 * n, cudaMemcpyHostToDevice, cs));
        DDHF_CUDA_TRY(c, cudaMemcpyAsync(dy, W.y, 2 * n, cudaMemcpyHostToDevice, cs));
        DDHF_CUDA_TRY(c, cudaMemcpyAsync(dt, W.t_us, 8 * n, cudaMemcpyHostToDevice, cs));
        DDHF_CUDA_TRY(c, cudaMemcpyAsync(dp, W.p, n, cudaMemcpyHostToDevice, cs));
      }
      DDHF_CUDA_TRY(c, cudaEventRecord(c->h_win[b * kHostGroup + i], cs));
      dw[i] = W;
      dw[i].x = dx;
      dw[i].y = dy;
      dw[i].t_us = dt;
      dw[i].p = dp;
    }
    DDHF_TRY(run_detect(c, dw, ng, c->hbox, cap, c->hnbox, nullptr, s, &c->h_win[b * kHostGroup]));
    DDHF_CUDA_TRY(c, cudaEventRecord(c->h_free[b], s));
    if (cap > 0)
      DDHF_CUDA_TRY(c, cudaMemcpyAsync(boxes_host + (int64_t)g0 * cap, c->hbox,
                                       sizeof(ddhf_box) * cap * ng, cudaMemcpyDeviceToHost, s));
    DDHF_CUDA_TRY(c, cudaMemcpyAsync(n_boxes_host + g0, c->hnbox, sizeof(int32_t) * ng,
                                     cudaMemcpyDeviceToHost, s));
    if (masks_host)
      for (int i = 0; i < ng; ++i)
        DDHF_CUDA_TRY(c, cudaMemcpyAsync(masks_host + (int64_t)(g0 + i) * c->npx,
                                         c->slots[i].mask, c->npx, cudaMemcpyDeviceToHost, s));
  }
  c->binned = true;
  return DDHF_OK;
}

ddhf_status ddhf_export_scores(ddhf_ctx *h, int32_t slot, uint32_t *active, float *log_sf, float *snr,
                               int32_t *f0_bin, int64_t *counts, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (slot < 0 || slot >= c->max_windows) return fail(c, DDHF_ERR_INVALID_ARG, "slot out of range");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const Slot &sl = c->slots[slot];
  const uint64_t *cnt = sl.counters;
  if (active) k_copy_counted<<<c->num_sms * 4, 256, 0, s>>>(active, sl.active, cnt + 2, c->npx, c->flags);
  if (log_sf)
    k_copy_counted<<<c->num_sms * 4, 256, 0, s>>>(reinterpret_cast<uint32_t *>(log_sf),
                                                 reinterpret_cast<const uint32_t *>(sl.log_sf),
                                                 cnt + 2, c->npx, c->flags);
  if (snr)
    k_copy_counted<<<c->num_sms * 4, 256, 0, s>>>(reinterpret_cast<uint32_t *>(snr),
                                                 reinterpret_cast<const uint32_t *>(sl.snr),
                                                 cnt + 2, c->npx, c->flags);
  if (f0_bin)
    k_copy_counted<<<c->num_sms * 4, 256, 0, s>>>(reinterpret_cast<uint32_t *>(f0_bin),
                                                 reinterpret_cast<const uint32_t *>(sl.f0),
                                                 cnt + 2, c->npx, c->flags);
  if (counts) k_copy_counts<<<1, 32, 0, s>>>(counts, cnt);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

ddhf_status ddhf_box_frequencies(ddhf_ctx *h, int32_t slot, const ddhf_box *boxes,
                                 const int32_t *n_boxes_dev, int32_t cap, int32_t *f0_bin,
                                 float *snr, float *f0_hz_median, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (slot < 0 || slot >= c->max_windows) return fail(c, DDHF_ERR_INVALID_ARG, "slot out of range");
  if (cap < 0 || (cap > 0 && (!boxes || !n_boxes_dev || !f0_bin)))
    return fail(c, DDHF_ERR_INVALID_ARG, "boxes, n_boxes_dev and f0_bin are required");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return launch_box_f0(c, slot, boxes, n_boxes_dev, cap, f0_bin, snr, f0_hz_median, s);
}

ddhf_status ddhf_export_labels(ddhf_ctx *h, int32_t slot, int32_t *labels, ddhf_stream stream) {
  if (!h) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  if (slot < 0 || slot >= c->max_windows || !labels)
    return fail(c, DDHF_ERR_INVALID_ARG, "bad label export arguments");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  DDHF_CUDA_TRY(c, cudaMemcpyAsync(labels, c->slots[slot].labels, c->npx * sizeof(int32_t),
                                   cudaMemcpyDeviceToDevice, s));
  return DDHF_OK;
}

ddhf_status ddhf_get_stats(ddhf_ctx *h, ddhf_stats *out) {
  if (!h || !out) return DDHF_ERR_INVALID_ARG;
  Ctx *c = &h->c;
  DDHF_CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
  DDHF_CUDA_TRY(c, check_guards(c, c->last_stream));
  DDHF_CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
  uint64_t cnt[8];
  uint32_t flags = 0;
  int32_t nbox = 0;
  DDHF_CUDA_TRY(c, cudaMemcpy(cnt, c->slots[0].counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  DDHF_CUDA_TRY(c, cudaMemcpy(&flags, c->flags, sizeof(flags), cudaMemcpyDeviceToHost));
  DDHF_CUDA_TRY(c, cudaMemcpy(&nbox, c->slots[0].nbox, sizeof(nbox), cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  out->n_valid = (int64_t)cnt[0];
  out->n_dropped = (int64_t)cnt[1];
  out->n_active = (int64_t)cnt[2];
  out->n_in = (int64_t)cnt[3];
  out->terms = (int64_t)cnt[5];
  out->n_rotor = (int64_t)cnt[7];
  out->n_boxes = nbox;
  out->graph_kernels = c->graph_kernels;
  out->device_flags = flags;
  if (flags) DDHF_CUDA_TRY(c, cudaMemset(c->flags, 0, sizeof(uint32_t)));
  if (flags & DDHF_FLAG_INTERNAL) return fail(c, DDHF_ERR_CUDA, "internal consistency check failed");
  if (flags & DDHF_FLAG_INPUT)
    return fail(c, DDHF_ERR_INVALID_ARG, "a device array held a pixel key or label out of range");
  if (flags & DDHF_FLAG_TIMEOUT) return fail(c, DDHF_ERR_TIMEOUT, "device-side loop limit reached");
  if (flags & DDHF_FLAG_CAPACITY) return fail(c, DDHF_ERR_CAPACITY, "output capacity exceeded");
  return DDHF_OK;
}

const char *ddhf_last_error(const ddhf_ctx *h) { return h ? h->c.last_error.c_str() : ""; }

}  // extern "C"
