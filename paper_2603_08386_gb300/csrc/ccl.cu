// Segmentation-mask processing (Sec. 3.5): 8-connected component labelling,
// per-component bounding boxes, the A_min area filter and centroid merging
// with Eq. 12, repeated to a fixed point.
//
// Labelling is a lock-free union-find over the pixel grid: every foreground
// pixel unions itself with its foreground neighbours W, NW, N and NE; a union
// always hooks the larger root under the smaller one (compare-and-swap on the
// root's parent), so every parent index is smaller than its child and the
// final root of a component is its smallest linear index, whatever order the
// unions ran in. Boxes use the root index as a slot (atomic min/max/add),
// survivors of the area filter are collected, and one thread block merges
// them: all pairs satisfying Eq. 12 are unioned (smallest index as root),
// each group becomes its union box, the survivors are compacted in root
// order, and the round repeats until no pair is close. The result is sorted
// by (y0, x0, y1, x1, n_px) by rank counting.
#include "ddhf_internal.cuh"

namespace ddhf {

namespace {

// Every union-find loop below stops after `limit` iterations (the context's
// loop limit, 2^24 unless a test lowers it), raises DDHF_FLAG_TIMEOUT and
// returns an index that is still in range, so a run-out leaves wrong labels
// but no bad access.
__device__ __forceinline__ int find_root(int32_t *lab, int x, uint32_t *flags, int limit) {
  int it = 0;
  int p = lab[x];
  while (p != x) {
    int gp = lab[p];
    if (gp < p) lab[x] = gp;  // path halving; parents only move to smaller ancestors
    x = p;
    p = gp;
    if (++it > limit) {
      atomicOr(flags, DDHF_FLAG_TIMEOUT);
      break;
    }
  }
  return x;
}

__device__ __forceinline__ void unite(int32_t *lab, int a, int b, uint32_t *flags, int limit) {
  for (int it = 0; it < limit; ++it) {
    a = find_root(lab, a, flags, limit);
    b = find_root(lab, b, flags, limit);
    if (a == b) return;
    if (a < b) {
      int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(&lab[a], a, b) == a) return;
  }
  atomicOr(flags, DDHF_FLAG_TIMEOUT);
}

__global__ void k_label_init(const uint8_t *__restrict__ mask, int32_t *__restrict__ lab,
                             int64_t npx, uint64_t *n_fg) {
  uint32_t cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool fg = mask[i] != 0;
    lab[i] = fg ? (int32_t)i : -1;
    cnt += fg;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt && n_fg) atomicAdd((unsigned long long *)n_fg, cnt);
}

__global__ void k_label_union(const uint8_t *__restrict__ mask, int32_t *lab, int W, int H,
                              uint32_t *flags, int limit) {
  const int64_t npx = (int64_t)W * H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[i]) continue;
    const int x = (int)(i % W), y = (int)(i / W);
    // Only the unions that no other pixel's own unions imply: the pixel above,
    // when set, is joined to the one left of it and to the one right of it by
    // their left-neighbour unions, and to this pixel's left neighbour by that
    // neighbour's up-right union; the left neighbour, when set, is joined to
    // the pixel above it by its own up union. The components (and so the
    // minimum-index labels) are those of all eight-neighbour unions.
    const bool left = x > 0 && mask[i - 1];
    if (y > 0 && mask[i - W]) {
      unite(lab, (int)i, (int)(i - W), flags, limit);
    } else {
      if (left) unite(lab, (int)i, (int)(i - 1), flags, limit);
      else if (y > 0 && x > 0 && mask[i - W - 1]) unite(lab, (int)i, (int)(i - W - 1), flags, limit);
      if (y > 0 && x < W - 1 && mask[i - W + 1]) unite(lab, (int)i, (int)(i - W + 1), flags, limit);
    }
  }
}

// Root of x without writing any parent: during the compress pass every thread
// writes only its own pixel, so no stale path-halving write can overwrite a
// root that another thread has already stored.
__device__ __forceinline__ int find_root_ro(const int32_t *lab, int x, uint32_t *flags,
                                            int limit) {
  for (int it = 0; it < limit; ++it) {
    const int p = lab[x];
    if (p == x) return x;
    x = p;
  }
  atomicOr(flags, DDHF_FLAG_TIMEOUT);
  return x;
}

__global__ void k_label_compress(int32_t *lab, int64_t npx, uint32_t *flags, int limit) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (lab[i] >= 0) lab[i] = find_root_ro(lab, (int)i, flags, limit);
  }
}

// Box slots indexed by root pixel: x0, y0, x1, y1, n (5 arrays of npx int32).
__global__ void k_box_root_init(const int32_t *__restrict__ lab, int32_t *bx, int W, int64_t npx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (lab[i] == (int32_t)i) {
      bx[i] = (int32_t)(i % W);
      bx[npx + i] = (int32_t)(i / W);
      bx[2 * npx + i] = (int32_t)(i % W);
      bx[3 * npx + i] = (int32_t)(i / W);
      bx[4 * npx + i] = 0;
    }
  }
}

// Pixels of one component usually share a warp, so the bounds are first
// reduced among the lanes with the same root and one lane updates the slot.
// A label at or beyond npx (a caller's labels array) is skipped and raises
// DDHF_FLAG_INPUT.
__global__ void k_box_accum(const int32_t *__restrict__ lab, int32_t *bx, int W, int64_t npx,
                            uint32_t *flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npx; base += stride) {
    const int64_t i = base + threadIdx.x;
    int r = i < npx ? lab[i] : -1;
    if ((int64_t)r >= npx) {
      atomicOr(flags, DDHF_FLAG_INPUT);
      r = -1;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, r);
    if (r < 0) continue;
    const int x = (int)(i % W), y = (int)(i / W);
    const int xmin = __reduce_min_sync(peers, x);
    const int xmax = __reduce_max_sync(peers, x);
    const int ymax = __reduce_max_sync(peers, y);
    const int n = __popc(peers);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) {
      atomicMin(&bx[r], xmin);
      atomicMax(&bx[2 * npx + r], xmax);
      atomicMax(&bx[3 * npx + r], ymax);
      atomicAdd(&bx[4 * npx + r], n);
    }
  }
}

// Survivors of the area filter, appended as quintuples (order fixed later).
__global__ void k_box_collect(const int32_t *__restrict__ lab, const int32_t *__restrict__ bx,
                              int64_t npx, int A_min, int32_t *list, uint32_t *count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (lab[i] != (int32_t)i) continue;
    const int x0 = bx[i], y0 = bx[npx + i], x1 = bx[2 * npx + i], y1 = bx[3 * npx + i];
    const int64_t area = (int64_t)(x1 - x0 + 1) * (int64_t)(y1 - y0 + 1);
    if (area < A_min) continue;
    const uint32_t pos = atomicAdd(count, 1u);
    int32_t *o = list + 5 * (int64_t)pos;
    o[0] = x0;
    o[1] = y0;
    o[2] = x1;
    o[3] = y1;
    o[4] = bx[4 * npx + i];
  }
}

// Every component (no area filter), shifted to sensor coordinates.
__global__ void k_comp_collect(const int32_t *__restrict__ lab, const int32_t *__restrict__ bx,
                               int64_t npx, int W, int32_t row0, ddhf_component *out, int cap,
                               uint32_t *count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (lab[i] != (int32_t)i) continue;
    const uint32_t pos = atomicAdd(count, 1u);
    if ((int64_t)pos >= cap) continue;
    ddhf_component c;
    c.label = (int32_t)(i + (int64_t)row0 * W);
    c.x0 = bx[i];
    c.y0 = bx[npx + i] + row0;
    c.x1 = bx[2 * npx + i];
    c.y1 = bx[3 * npx + i] + row0;
    c.n_px = bx[4 * npx + i];
    out[pos] = c;
  }
}

// Eq. 12 in FP64, every product rounded on its own.
__device__ __forceinline__ bool eq12_close(const int32_t *a, const int32_t *b, double alpha) {
  const int64_t dx2 = (int64_t)(a[0] + a[2]) - (int64_t)(b[0] + b[2]);
  const int64_t dy2 = (int64_t)(a[1] + a[3]) - (int64_t)(b[1] + b[3]);
  int64_t m = a[2] - a[0] + 1;
  m = max(m, (int64_t)(a[3] - a[1] + 1));
  m = max(m, (int64_t)(b[2] - b[0] + 1));
  m = max(m, (int64_t)(b[3] - b[1] + 1));
  const double lhs = (double)(dx2 * dx2 + dy2 * dy2);
  const double s = __dmul_rn(__dmul_rn(2.0, alpha), (double)m);
  return lhs < __dmul_rn(s, s);
}

__device__ __forceinline__ int gfind(int32_t *par, int x, uint32_t *flags, int limit) {
  int p = par[x];
  for (int it = 0; p != x; ++it) {
    int gp = par[p];
    par[x] = gp;
    x = p;
    p = gp;
    if (it > limit) {
      atomicOr(flags, DDHF_FLAG_TIMEOUT);
      break;
    }
  }
  return x;
}

__device__ __forceinline__ void gunite(int32_t *par, int a, int b, uint32_t *flags, int limit) {
  for (int it = 0; it < limit; ++it) {
    a = gfind(par, a, flags, limit);
    b = gfind(par, b, flags, limit);
    if (a == b) return;
    if (a < b) {
      int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(&par[a], a, b) == a) return;
  }
  atomicOr(flags, DDHF_FLAG_TIMEOUT);
}

__device__ __forceinline__ bool box_less(const int32_t *a, const int32_t *b) {
  for (int k = 0; k < 5; ++k) {
    const int ka = k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 3 : k == 3 ? 2 : 4;  // y0, x0, y1, x1, n
    if (a[ka] != b[ka]) return a[ka] < b[ka];
  }
  return false;
}

constexpr int kMergeThreads = 1024;

__global__ void __launch_bounds__(kMergeThreads) k_box_merge(int32_t *list, int32_t *list2,
                                                             int32_t *par, int32_t *root,
                                                             const uint32_t *count,
                                                             double alpha, ddhf_box *out, int cap,
                                                             int32_t *n_out, uint32_t *flags,
                                                             int limit) {
  __shared__ int any;
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t s_base;
  int B = (int)*count;
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int round = 0; round <= B + 1; ++round) {
    for (int i = tid; i < B; i += bs) par[i] = i;
    if (tid == 0) any = 0;
    __syncthreads();
    const int64_t pairs = (int64_t)B * B;
    for (int64_t p = tid; p < pairs; p += bs) {
      const int i = (int)(p / B), j = (int)(p % B);
      if (j <= i) continue;
      if (eq12_close(list + 5 * (int64_t)i, list + 5 * (int64_t)j, alpha)) {
        any = 1;
        gunite(par, i, j, flags, limit);
      }
    }
    __syncthreads();
    if (!any) break;
    if (round == B + 1) {
      if (tid == 0) atomicOr(flags, DDHF_FLAG_TIMEOUT);
      break;
    }
    for (int i = tid; i < B; i += bs) root[i] = find_root_ro(par, i, flags, limit);
    __syncthreads();
    for (int i = tid; i < B; i += bs) par[i] = root[i];
    __syncthreads();
    for (int i = tid; i < B; i += bs) {
      if (par[i] == i) {
        int32_t *d = list2 + 5 * (int64_t)i;
        const int32_t *s = list + 5 * (int64_t)i;
        d[0] = s[0];
        d[1] = s[1];
        d[2] = s[2];
        d[3] = s[3];
        d[4] = 0;
      }
    }
    __syncthreads();
    for (int i = tid; i < B; i += bs) {
      const int r = par[i];
      int32_t *d = list2 + 5 * (int64_t)r;
      const int32_t *s = list + 5 * (int64_t)i;
      atomicMin(&d[0], s[0]);
      atomicMin(&d[1], s[1]);
      atomicMax(&d[2], s[2]);
      atomicMax(&d[3], s[3]);
      atomicAdd(&d[4], s[4]);
    }
    __syncthreads();
    // compact roots in index order into list
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < B; c0 += bs) {
      const int i = c0 + tid;
      const bool root = i < B && par[i] == i;
      const uint32_t bal = __ballot_sync(0xffffffffu, root);
      const int lane = tid & 31, warp = tid >> 5;
      if (lane == 0) warp_tot[warp] = __popc(bal);
      __syncthreads();
      uint32_t wpre = 0;
      for (int w2 = 0; w2 < warp; ++w2) wpre += warp_tot[w2];
      const uint32_t pos = s_base + wpre + __popc(bal & ((1u << lane) - 1));
      if (root) {
        int32_t *d = list + 5 * (int64_t)pos;
        const int32_t *s = list2 + 5 * (int64_t)i;
        for (int k = 0; k < 5; ++k) d[k] = s[k];
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t t = 0;
        for (int w2 = 0; w2 < (bs >> 5); ++w2) t += warp_tot[w2];
        s_base += t;
      }
      __syncthreads();
    }
    B = (int)s_base;
    __syncthreads();
  }
  for (int i = tid; i < B; i += bs) {
    const int32_t *bi = list + 5 * (int64_t)i;
    int rank = 0;
    for (int j = 0; j < B; ++j) {
      const int32_t *bj = list + 5 * (int64_t)j;
      if (box_less(bj, bi) || (j < i && !box_less(bi, bj))) ++rank;
    }
    if (rank < cap) {
      ddhf_box o;
      o.x0 = bi[0];
      o.y0 = bi[1];
      o.x1 = bi[2];
      o.y1 = bi[3];
      o.n_px = bi[4];
      out[rank] = o;
    }
  }
  if (tid == 0) {
    *n_out = B;
    if (B > cap) atomicOr(flags, DDHF_FLAG_CAPACITY);
  }
}

}  // namespace

ddhf_status launch_label(Ctx *c, const uint8_t *mask, int32_t *labels, uint64_t *nfg,
                         cudaStream_t s) {
  const int blocks = c->num_sms * 8;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(nfg, 0, sizeof(uint64_t), s));
  k_label_init<<<blocks, 256, 0, s>>>(mask, labels, c->npx, nfg);
  k_label_union<<<blocks, 256, 0, s>>>(mask, labels, c->W, c->H, c->flags, c->loop_limit);
  k_label_compress<<<blocks, 256, 0, s>>>(labels, c->npx, c->flags, c->loop_limit);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

// Dominant frequency of each box: block b scans the rows of box b; warp by
// warp, a row's active pixels are the run of the (ascending) active list
// between the keys y W + x0 and y W + x1, found by binary search. First pass:
// each rotor pixel offers (SNR bits, -active index) to a maximum (the
// strongest pixel) and is counted; then, when asked for, the lower median of
// the rotor pixels' dominant bins by a two-digit radix selection (bins below
// 2^14, 7 bits per pass, one more scan of the box per digit). A box without
// rotor pixels gets bin -1, SNR 0 and median 0 Hz.
__global__ void __launch_bounds__(256) k_box_f0(const uint32_t *__restrict__ active,
                                                const uint64_t *__restrict__ counters,
                                                const uint8_t *__restrict__ mask,
                                                const float *__restrict__ snr,
                                                const int32_t *__restrict__ f0,
                                                const ddhf_box *__restrict__ boxes,
                                                const int32_t *__restrict__ n_boxes, int32_t cap,
                                                int W, int H, int32_t *f0_out, float *snr_out,
                                                float *med_hz, int64_t g_a0, int64_t g_da,
                                                int64_t g_denom, uint32_t *flags) {
  __shared__ unsigned long long red[8];
  __shared__ uint32_t cnt[8];
  __shared__ uint32_t hist[128];
  __shared__ uint32_t sel[2];
  const int b = blockIdx.x;
  const int nb = min(*n_boxes, cap);
  if (b >= nb) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n_act = (int64_t)counters[2];
  const ddhf_box bx = boxes[b];
  const int x0 = max(bx.x0, 0), x1 = min(bx.x1, W - 1);
  const int y0 = max(bx.y0, 0), y1 = min(bx.y1, H - 1);
  // fn(i) for every rotor pixel i (active index) inside the box
  auto visit = [&](auto fn) {
    for (int y = y0 + warp; y <= y1 && x0 <= x1; y += 8) {
      const uint32_t lo = (uint32_t)((int64_t)y * W + x0), hi = (uint32_t)((int64_t)y * W + x1);
      int64_t l = 0, r = n_act;  // first index with active[i] >= lo
      while (l < r) {
        const int64_t m = (l + r) >> 1;
        if (active[m] < lo) l = m + 1;
        else r = m;
      }
      for (int64_t i = l + lane;; i += 32) {
        const bool in = i < n_act && active[i] <= hi;
        if (in && mask[active[i]]) fn(i);
        if (!__any_sync(0xffffffffu, in)) break;
      }
    }
  };
  unsigned long long best = 0ull;
  uint32_t n = 0;
  visit([&](int64_t i) {
    const unsigned long long v =
        ((unsigned long long)__float_as_uint(snr[i]) << 32) | (0xffffffffu - (uint32_t)i);
    best = v > best ? v : best;
    ++n;
  });
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, best, o);
    best = u > best ? u : best;
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  if (lane == 0) {
    red[warp] = best;
    cnt[warp] = n;
  }
  __syncthreads();
  best = red[0];
  n = cnt[0];
  for (int w = 1; w < 8; ++w) {
    best = red[w] > best ? red[w] : best;
    n += cnt[w];
  }
  if (threadIdx.x == 0) {
    if (best == 0ull) {
      f0_out[b] = -1;
      if (snr_out) snr_out[b] = 0.f;
    } else {
      const uint32_t i = 0xffffffffu - (uint32_t)best;
      f0_out[b] = f0[i];
      if (snr_out) snr_out[b] = snr[i];
    }
  }
  if (!med_hz) return;
  if (n == 0) {
    if (threadIdx.x == 0) med_hz[b] = 0.f;
    return;
  }
  // lower median: the element of rank (n - 1) / 2 of the dominant bins
  uint32_t rank = (n - 1) / 2, prefix = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int shift = pass == 0 ? 7 : 0;
    for (int k = threadIdx.x; k < 128; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    visit([&](int64_t i) {
      const uint32_t v = (uint32_t)f0[i];
      if (!ddhf_check(v < (1u << 14), flags)) return;
      if (pass == 1 && (v >> 7) != prefix) return;
      atomicAdd(&hist[(v >> shift) & 127u], 1u);
    });
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      int dsel = 127;
      for (int k = 0; k < 128; ++k) {
        if (rank < run + hist[k]) {
          dsel = k;
          break;
        }
        run += hist[k];
      }
      sel[0] = (uint32_t)dsel;
      sel[1] = rank - run;
    }
    __syncthreads();
    if (pass == 0) prefix = sel[0];
    else prefix = (prefix << 7) | sel[0];
    rank = sel[1];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    med_hz[b] = (float)((double)(g_a0 + (int64_t)prefix * g_da) * 1e6 / (double)g_denom);
}

ddhf_status launch_box_f0(Ctx *c, int slot, const ddhf_box *boxes, const int32_t *n_boxes,
                          int32_t cap, int32_t *f0_out, float *snr_out, float *med_hz,
                          cudaStream_t s) {
  const Slot &sl = c->slots[slot];
  // bin j at (a0 + j da) / denom cycles per microsecond
  if (cap > 0)
    k_box_f0<<<cap, 256, 0, s>>>(sl.active, sl.counters, sl.mask, sl.snr, sl.f0, boxes, n_boxes,
                                 cap, c->W, c->H, f0_out, snr_out, med_hz, c->grid.a0, c->grid.da,
                                 c->grid.denom, c->flags);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

ddhf_status launch_components(Ctx *c, const int32_t *labels, int32_t row0, ddhf_component *out,
                              int32_t cap, int32_t *n_out, cudaStream_t s) {
  const int blocks = c->num_sms * 8;
  const int64_t npx = c->npx;
  int32_t *bx = c->box_tmp;  // 5 * npx
  uint32_t *count = reinterpret_cast<uint32_t *>(n_out);
  DDHF_CUDA_TRY(c, cudaMemsetAsync(count, 0, sizeof(uint32_t), s));
  k_box_root_init<<<blocks, 256, 0, s>>>(labels, bx, c->W, npx);
  k_box_accum<<<blocks, 256, 0, s>>>(labels, bx, c->W, npx, c->flags);
  k_comp_collect<<<blocks, 256, 0, s>>>(labels, bx, npx, c->W, row0, out, cap, count);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

ddhf_status launch_boxes(Ctx *c, const int32_t *labels, ddhf_box *boxes, int32_t cap,
                         int32_t *n_boxes, cudaStream_t s) {
  const int blocks = c->num_sms * 8;
  const int64_t npx = c->npx;
  int32_t *bx = c->box_tmp;                  // 5 * npx
  int32_t *list = c->box_tmp + 5 * npx;      // 5 * npx
  int32_t *list2 = c->box_tmp + 10 * npx;    // 5 * npx
  int32_t *par = c->box_root;                // npx
  uint32_t *count = c->qctl + 9;
  DDHF_CUDA_TRY(c, cudaMemsetAsync(count, 0, sizeof(uint32_t), s));
  k_box_root_init<<<blocks, 256, 0, s>>>(labels, bx, c->W, npx);
  k_box_accum<<<blocks, 256, 0, s>>>(labels, bx, c->W, npx, c->flags);
  k_box_collect<<<blocks, 256, 0, s>>>(labels, bx, npx, c->params.A_min, list, count);
  k_box_merge<<<1, kMergeThreads, 0, s>>>(list, list2, par, bx, count, c->params.alpha, boxes,
                                          cap, n_boxes, c->flags, c->loop_limit);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

}  // namespace ddhf
