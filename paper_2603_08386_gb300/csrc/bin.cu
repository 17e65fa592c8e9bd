// Event binning (Sec. 3.5 "Event processing"): window + validity filter, a
// stable sort of the events by pixel key y*W + x into a per-pixel list, and
// the list of active pixels (at least n_min events, Table 2).
//
// Design: least-significant-digit radix sort over the key bits in 1-3 passes
// of <= 11 bits. Each pass is reduce-then-scan: a histogram kernel writes one
// count per (digit, chunk of 8192 events) in digit-major order, an exclusive
// scan of that table gives every (digit, chunk) its output offset, and a
// scatter kernel re-reads its chunk and places each element at
// offset + (its rank among equal digits earlier in the chunk). The in-chunk
// rank is computed warp by warp with one ballot per digit bit and per-warp digit
// counters in shared memory, so element order inside a digit is input order
// and every pass is stable; the chunk is staged in shared memory in digit
// order and written out in contiguous runs; no block waits on another block. The first pass
// reads the raw (x, y, t, p) arrays directly and packs each kept event into
// one 32-bit word: tau = t - t0 in bits 0-30, bit 31 set for polarity -1.
// Per-pixel counts come from segment boundaries of the sorted keys, and one
// 64-bit scan of (count << 32 | active flag) gives both the CSR offsets and
// the active-pixel list.
#include "ddhf_internal.cuh"

namespace ddhf {

namespace {

struct RawIn {
  const int16_t *x, *y;
  const int64_t *t;
  const int8_t *p;
  int64_t n;
  int64_t t0;
  uint64_t win;
  int W, H, pol01;
  int row0;  // sensor row of the context's row 0 (row bands)
  // pre-packed input instead of (x, y, t, p): key pk[e] (kDropKey = not kept)
  // and value pv[e] as the sort carries them
  const uint32_t *pk = nullptr, *pv = nullptr;
};

__device__ __forceinline__ bool load_raw(const RawIn &in, int64_t e, uint32_t &key,
                                         uint32_t &val) {
  if (in.pk) {
    key = in.pk[e];
    val = in.pv[e];
    return key != kDropKey;
  }
  int xx = in.x[e], yy = in.y[e] - in.row0;
  int64_t tt = in.t[e];
  int pp = in.p[e];
  bool okp = in.pol01 ? (pp == 0 || pp == 1) : (pp == 1 || pp == -1);
  bool neg = in.pol01 ? (pp == 0) : (pp == -1);
  uint64_t dt = (uint64_t)tt - (uint64_t)in.t0;
  bool ok = okp && xx >= 0 && xx < in.W && yy >= 0 && yy < in.H && tt >= in.t0 && dt < in.win;
  key = (uint32_t)(yy * in.W + xx);
  val = (uint32_t)dt | (neg ? kSignBit : 0u);
  return ok;
}

template <bool RAW>
__global__ void __launch_bounds__(kBinThreads) k_hist(RawIn raw, const uint32_t *__restrict__ kin,
                                                      const uint32_t *__restrict__ n_dev,
                                                      uint32_t *__restrict__ hist, int64_t nchunks,
                                                      int shift, int nb) {
  __shared__ uint32_t sh[1 << kMaxDigitBits];
  constexpr int kU = 8;  // elements per thread with their loads in flight together
  const int64_t n = RAW ? raw.n : (int64_t)*n_dev;
  const int64_t chunk = blockIdx.x;
  const int64_t c0 = chunk * kBinChunk;
  for (int d = threadIdx.x; d < nb; d += blockDim.x) sh[d] = 0;
  __syncthreads();
  const int64_t c1 = min(n, c0 + (int64_t)kBinChunk);
  if (!RAW && c1 - c0 == kBinChunk && (reinterpret_cast<uintptr_t>(kin) & 15) == 0) {
    // a whole chunk of sort words: 16-byte loads, 4 keys each, 8 per thread and step
    const uint4 *k4 = reinterpret_cast<const uint4 *>(kin + c0);
    for (int q = threadIdx.x; q < kBinChunk / 4; q += 2 * kBinThreads) {
      const uint4 a = k4[q];
      const uint4 b = k4[q + kBinThreads];
      const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 8; ++u) atomicAdd(&sh[(w[u] >> shift) & (uint32_t)(nb - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += blockDim.x) hist[(int64_t)d * nchunks + chunk] = sh[d];
    return;
  }
  for (int64_t base = c0 + threadIdx.x; base < c1; base += (int64_t)kBinThreads * kU) {
    uint32_t d[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t e = base + (int64_t)u * kBinThreads;
      d[u] = (uint32_t)nb;  // sentinel: not counted
      if (e < c1) {
        if (RAW) {
          uint32_t key, val;
          if (load_raw(raw, e, key, val)) d[u] = (key >> shift) & (uint32_t)(nb - 1);
        } else {
          d[u] = (kin[e] >> shift) & (uint32_t)(nb - 1);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (d[u] < (uint32_t)nb) atomicAdd(&sh[d[u]], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nb; d += blockDim.x) hist[(int64_t)d * nchunks + chunk] = sh[d];
}

// First pass over raw events: the histogram of the first digit per chunk, as
// k_hist, and each event packed into the (key, value) words the sort carries
// (key kDropKey for events that are not kept), so that the first scatter reads
// 8 bytes per event in two coalesced words. VEC: the arrays are aligned for
// loads of 4 consecutive events (x, y: 8 bytes, t: 2 x 16 bytes, p: 4 bytes).
template <bool VEC>
__global__ void __launch_bounds__(kBinThreads) k_hist_pack(RawIn raw, uint32_t *__restrict__ pk,
                                                           uint32_t *__restrict__ pv,
                                                           uint32_t *__restrict__ hist,
                                                           int64_t nchunks, int nb) {
  __shared__ uint32_t sh[1 << kMaxDigitBits];
  const int64_t n = raw.n;
  const int64_t chunk = blockIdx.x;
  const int64_t c0 = chunk * kBinChunk;
  for (int d = threadIdx.x; d < nb; d += blockDim.x) sh[d] = 0;
  __syncthreads();
  const int64_t c1 = min(n, c0 + (int64_t)kBinChunk);
  const uint32_t mask = (uint32_t)(nb - 1);
  // 4 consecutive events per thread and step; 8 steps cover the chunk
  for (int64_t e0 = c0 + 4 * (int64_t)threadIdx.x; e0 < c1; e0 += 4 * kBinThreads) {
    uint32_t key[4], val[4];
    bool kept[4];
    if (VEC && e0 + 4 <= c1) {
      const short4 xs = *reinterpret_cast<const short4 *>(raw.x + e0);
      const short4 ys = *reinterpret_cast<const short4 *>(raw.y + e0);
      const longlong2 t01 = *reinterpret_cast<const longlong2 *>(raw.t + e0);
      const longlong2 t23 = *reinterpret_cast<const longlong2 *>(raw.t + e0 + 2);
      const char4 ps = *reinterpret_cast<const char4 *>(raw.p + e0);
      const int xx[4] = {xs.x, xs.y, xs.z, xs.w}, yy[4] = {ys.x, ys.y, ys.z, ys.w};
      const int64_t tt[4] = {t01.x, t01.y, t23.x, t23.y};
      const int pp[4] = {(int8_t)ps.x, (int8_t)ps.y, (int8_t)ps.z, (int8_t)ps.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int xv = xx[u], yv = yy[u] - raw.row0;
        const bool okp = raw.pol01 ? (pp[u] == 0 || pp[u] == 1) : (pp[u] == 1 || pp[u] == -1);
        const bool neg = raw.pol01 ? (pp[u] == 0) : (pp[u] == -1);
        const uint64_t dt = (uint64_t)tt[u] - (uint64_t)raw.t0;
        kept[u] = okp && xv >= 0 && xv < raw.W && yv >= 0 && yv < raw.H && tt[u] >= raw.t0 &&
                  dt < raw.win;
        key[u] = (uint32_t)(yv * raw.W + xv);
        val[u] = (uint32_t)dt | (neg ? kSignBit : 0u);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        kept[u] = false;
        key[u] = 0u;
        val[u] = 0u;
        if (e0 + u < c1) kept[u] = load_raw(raw, e0 + u, key[u], val[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!kept[u]) key[u] = kDropKey;
      else atomicAdd(&sh[key[u] & mask], 1u);
    }
    if (VEC && e0 + 4 <= c1) {
      *reinterpret_cast<uint4 *>(pk + e0) = make_uint4(key[0], key[1], key[2], key[3]);
      *reinterpret_cast<uint4 *>(pv + e0) = make_uint4(val[0], val[1], val[2], val[3]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (e0 + u < c1) {
          pk[e0 + u] = key[u];
          pv[e0 + u] = val[u];
        }
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nb; d += blockDim.x) hist[(int64_t)d * nchunks + chunk] = sh[d];
}

// Exclusive scan in place of a[0..n) (n <= 2^kMaxDigitBits) by one block of
// kScatThreads threads; returns the total. Uses `tmp` (kScatThreads / 32 words).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t *a, int n, uint32_t *tmp) {
  constexpr int kPer = (1 << kMaxDigitBits) / kScatThreads;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = (n + kScatThreads - 1) / kScatThreads;  // <= kPer
  uint32_t v[kPer], s = 0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int j = t * per + i;
    v[i] = (i < per && j < n) ? a[j] : 0u;
    s += v[i];
  }
  uint32_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  uint32_t wpre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kScatThreads / 32; ++w) {
    const uint32_t x = tmp[w];
    if (w < warp) wpre += x;
    tot += x;
  }
  uint32_t run = wpre + inc - s;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int j = t * per + i;
    if (i < per && j < n) {
      a[j] = run;
      run += v[i];
    }
  }
  __syncthreads();
  return tot;
}

// Shared memory of k_scatter in 32-bit words: the ranking counters (16-bit,
// one per warp and digit) share their space with the staged chunk (keys and
// values), followed by two words per digit and the chunk's values in input
// order.
// Ranking chains per warp (counter tables, each over a contiguous group of the
// warp's rows): one; splitting the rows into two interleaved chains measured
// slower.
__host__ __device__ constexpr int scatter_chains(int) { return 1; }
__host__ __device__ constexpr int scatter_union_words(int nb) {
  return (kScatThreads / 32) * scatter_chains(nb) * nb / 2 > 2 * kBinChunk
             ? (kScatThreads / 32) * scatter_chains(nb) * nb / 2
             : 2 * kBinChunk;
}
__host__ __device__ constexpr int scatter_smem_bytes(int nb) {
  return (scatter_union_words(nb) + 2 * nb + kBinChunk) * 4;
}

// Asynchronous global -> shared copies (cp.async), `bytes` of `size` read.
__device__ __forceinline__ void cp_async16(uint32_t dst_sa, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst_sa), "l"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst_sa, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst_sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Stable scatter of one chunk of 8192 (key, value) elements. Warp w holds the
// chunk's keys [512 w, 512 (w + 1)) as 16 rows of 32 consecutive keys (lane l
// of row i: element 512 w + 32 i + l), so the order (warp, row, lane) is input
// order; the values go to shared memory in input order by asynchronous copies
// meanwhile. Ranking: row by row, each element's rank among the warp's earlier
// elements of its digit is a per-warp counter (shared memory, 16 bits) plus
// the number of lower lanes with the same digit (one ballot per digit bit);
// the lowest such lane advances the counter. One pass over the digits then
// turns the counters into the chunk positions (the digit's start in the
// chunk, from the histogram table, plus the counts of the earlier warps), the
// elements are staged in shared memory at their positions (the chunk in digit
// order), and the staged chunk is written out so that consecutive slots of one
// digit go to consecutive addresses, from the (digit, chunk)'s offset in the
// scanned table. DROP (first pass): the input has n_in elements, key kDropKey
// marks one that is not kept; otherwise all n_total elements are kept.
// n_total: kept elements of the whole array (the table's sum). BITS: digit
// width (nb = 2^BITS), a template argument so that the ballots unroll.
template <bool DROP, int BITS>
__global__ void __launch_bounds__(kScatThreads, 2) k_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, int64_t n_in,
    const uint32_t *__restrict__ n_total, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *__restrict__ hscan, int64_t nchunks,
    int shift, uint32_t *flags) {
  constexpr int kWarps = kScatThreads / 32;
  constexpr int nb = 1 << BITS;
  constexpr int kCh = scatter_chains(nb);            // counter tables per warp
  constexpr int kVW = kWarps * kCh;                   // virtual warps, in input order
  constexpr int kRows = kScatItems / kCh;             // rows per chain
  constexpr uint32_t mask = (uint32_t)(nb - 1);
  extern __shared__ uint32_t sm[];
  uint16_t *cnt = reinterpret_cast<uint16_t *>(sm);  // [kVW][nb], then chunk positions
  uint32_t *sk = sm;                                  // [kBinChunk] staged keys
  uint32_t *sv = sm + kBinChunk;                      // [kBinChunk] staged values
  uint32_t *lst = sm + scatter_union_words(nb);       // [nb] start of each digit in the chunk
  uint32_t *gofs = lst + nb;                          // [nb] output offset minus the start
  uint32_t *vbuf = gofs + nb;                         // [kBinChunk] values in input order
  __shared__ uint32_t scan_tmp[kWarps];
  const int64_t n = DROP ? n_in : (int64_t)*n_total;
  const int64_t chunk = blockIdx.x;
  const int64_t c0 = chunk * kBinChunk;
  if (c0 >= n) return;
  const int nloc = (int)min((int64_t)kBinChunk, n - c0);  // elements of this chunk
  // values -> vbuf (16-byte copies when the array is aligned for them)
  const uint32_t vbuf_sa = (uint32_t)__cvta_generic_to_shared(vbuf);
  if ((reinterpret_cast<uintptr_t>(vin) & 15) == 0) {
    for (int q = threadIdx.x; 4 * q < nloc; q += kScatThreads)
      cp_async16(vbuf_sa + 16 * q, vin + c0 + 4 * q, 4 * min(4, nloc - 4 * q));
  } else {
    for (int q = threadIdx.x; q < nloc; q += kScatThreads) cp_async4(vbuf_sa + 4 * q, vin + c0 + q);
  }
  const int64_t ncells = (int64_t)nb * nchunks;
  const uint32_t total = *n_total;
  for (int i = threadIdx.x; i < kVW * nb / 2; i += kScatThreads) sm[i] = 0;
  for (int d = threadIdx.x; d < nb; d += kScatThreads) {
    const int64_t cell = (int64_t)d * nchunks + chunk;
    const uint32_t b = hscan[cell];
    gofs[d] = b;
    lst[d] = (cell + 1 < ncells ? hscan[cell + 1] : total) - b;  // this chunk's count of d
  }
  __syncthreads();
  const uint32_t m = block_excl_scan(lst, nb, scan_tmp);  // kept elements of the chunk
  for (int d = threadIdx.x; d < nb; d += kScatThreads) gofs[d] -= lst[d];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1;
  uint16_t *my = cnt + warp * kCh * nb;  // chain h of this warp: my + h * nb
  const int wloc = warp * (32 * kScatItems) + lane;  // local index of row 0
  // ps: two 16-bit ranks (then chunk positions, < 8192) per register
  uint32_t kk[kScatItems], ps[kScatItems / 2], ok = 0;
#pragma unroll
  for (int i = 0; i < kScatItems; ++i) {
    const int l = wloc + 32 * i;
    const uint32_t key = l < nloc ? kin[c0 + l] : kDropKey;
    const bool kept = l < nloc && (!DROP || key != kDropKey);
    kk[i] = key;
    ok |= kept ? (1u << i) : 0u;
  }
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
#pragma unroll
    for (int h = 0; h < kCh; ++h) {
      const int i = h * kRows + j;  // row i of the warp, chain h
      const bool kept = (ok >> i) & 1u;
      const uint32_t d = (kk[i] >> shift) & mask;
      // lanes with the same digit (kept ones) or the other dropped lanes
      uint32_t peers = __ballot_sync(0xffffffffu, kept);
      if (!kept) peers = ~peers;
#pragma unroll
      for (int b = 0; b < BITS; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t bm = __ballot_sync(0xffffffffu, bit);
        peers &= bm ^ (bit - 1u);  // bm where the bit is set, ~bm where it is not
      }
      const uint32_t before = __popc(peers & lt);
      uint16_t *myh = my + h * nb;
      uint32_t c = 0;
      if (kept) c = myh[d];
      __syncwarp();
      if (kept && before == 0) myh[d] = (uint16_t)(c + __popc(peers));
      __syncwarp();
      const uint32_t r = c + before;
      ps[i / 2] = (i & 1) ? (ps[i / 2] | (r << 16)) : r;
    }
  }
  __syncthreads();
  // counters -> chunk positions: start of the digit plus the earlier warps' counts
  for (int d = threadIdx.x; d < nb; d += kScatThreads) {
    uint32_t run = lst[d];
#pragma unroll
    for (int w = 0; w < kVW; ++w) {
      const uint32_t v = cnt[w * nb + d];
      cnt[w * nb + d] = (uint16_t)run;
      run += v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScatItems; ++i)
    if ((ok >> i) & 1u)
      ps[i / 2] += (uint32_t)my[(i / kRows) * nb + ((kk[i] >> shift) & mask)] << (16 * (i & 1));
  cp_async_wait_all();
  __syncthreads();  // counters read, values arrived
#pragma unroll
  for (int i = 0; i < kScatItems; ++i) {
    const uint32_t pos = (ps[i / 2] >> (16 * (i & 1))) & 0xffffu;
    if (((ok >> i) & 1u) && ddhf_check(pos < (uint32_t)kBinChunk, flags)) {
      sk[pos] = kk[i];
      sv[pos] = vbuf[wloc + 32 * i];
    }
  }
  __syncthreads();
  // staged chunk out: consecutive slots of one digit go to consecutive addresses
  for (uint32_t sl = threadIdx.x; sl < m && sl < (uint32_t)kBinChunk; sl += kScatThreads) {
    const uint32_t key = sk[sl];
    const uint32_t dest = gofs[(key >> shift) & mask] + sl;
    if (dest < total) {  // always true when the counts agree with the table
      kout[dest] = key;
      vout[dest] = sv[sl];
    } else {
      ddhf_check(false, flags);
    }
  }
}

// Segment bounds of the sorted keys: seg_lo[k] = first index, seg_hi[k] = one
// past the last index of key k (both 0 for absent keys). Each thread takes 8
// consecutive keys (two 16-byte loads) and the keys on either side of them.
// Keys at or beyond npx (impossible for a correct sort) are not written.
__global__ void k_seg(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ n_dev,
                      uint32_t *__restrict__ seg_lo, uint32_t *__restrict__ seg_hi, int64_t npx,
                      uint32_t *flags) {
  const int64_t n = *n_dev;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 8 * g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = 8 * g;
    uint32_t k[10];  // k[0] = keys[i0 - 1], k[1..8] = keys[i0 .. i0 + 7], k[9] = keys[i0 + 8]
    if (i0 + 8 <= n) {
      const uint4 a = *reinterpret_cast<const uint4 *>(keys + i0);
      const uint4 b = *reinterpret_cast<const uint4 *>(keys + i0 + 4);
      k[1] = a.x; k[2] = a.y; k[3] = a.z; k[4] = a.w;
      k[5] = b.x; k[6] = b.y; k[7] = b.z; k[8] = b.w;
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) k[1 + u] = i0 + u < n ? keys[i0 + u] : 0xffffffffu;
    }
    k[0] = i0 > 0 ? keys[i0 - 1] : 0xffffffffu;
    k[9] = i0 + 8 < n ? keys[i0 + 8] : 0xffffffffu;
#pragma unroll
    for (int u = 1; u <= 8; ++u) {
      const int64_t i = i0 + u - 1;
      const uint32_t kk = k[u];
      if (i >= n) continue;
      if ((int64_t)kk >= npx) {
        ddhf_check(false, flags);
        continue;
      }
      if (i == 0 || k[u - 1] != kk) seg_lo[kk] = (uint32_t)i;
      if (i == n - 1 || k[u + 1] != kk) seg_hi[kk] = (uint32_t)(i + 1);
    }
  }
}

__global__ void k_pack(const uint32_t *__restrict__ seg_lo, const uint32_t *__restrict__ seg_hi,
                       uint64_t *__restrict__ packed, int64_t npx, int n_min) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= npx;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v = 0;
    if (k < npx) {
      uint32_t cnt = seg_hi[k] - seg_lo[k];
      v = ((uint64_t)cnt << 32) | (cnt >= (uint32_t)n_min ? 1u : 0u);
    }
    packed[k] = v;
  }
}

__global__ void k_finish(const uint64_t *__restrict__ scanned, const uint32_t *__restrict__ seg_lo,
                         const uint32_t *__restrict__ seg_hi, uint32_t *__restrict__ offsets,
                         uint32_t *__restrict__ active, uint64_t *__restrict__ counters,
                         int64_t npx, int n_min, int heavy_min, int64_t n_in, int64_t n_bins,
                         uint64_t *__restrict__ heavy_list, uint32_t *heavy_count,
                         uint32_t slot, int64_t heavy_cap, uint32_t *flags) {
  uint64_t terms = 0;
  uint32_t heavy = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= npx;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v = scanned[k];
    offsets[k] = (uint32_t)(v >> 32);
    if (k < npx) {
      uint32_t cnt = seg_hi[k] - seg_lo[k];
      if (cnt >= (uint32_t)n_min) {
        active[(uint32_t)v] = (uint32_t)k;
        terms += (uint64_t)cnt * (uint64_t)n_bins;
        if (cnt >= (uint32_t)heavy_min) {
          heavy += 1u;
          const uint32_t pos = atomicAdd(heavy_count, 1u);
          if ((int64_t)pos < heavy_cap)
            heavy_list[pos] = ((uint64_t)slot << 32) | (uint32_t)v;
          else
            atomicOr(flags, DDHF_FLAG_CAPACITY);
        }
      }
    } else {
      counters[0] = v >> 32;                       // n_valid
      counters[1] = (uint64_t)n_in - (v >> 32);    // n_dropped
      counters[2] = (uint32_t)v;                   // n_active
      counters[3] = (uint64_t)n_in;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    terms += __shfl_xor_sync(0xffffffffu, terms, o);
    heavy += __shfl_xor_sync(0xffffffffu, heavy, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (terms) atomicAdd((unsigned long long *)&counters[5], (unsigned long long)terms);
    if (heavy) atomicAdd((unsigned long long *)&counters[4], (unsigned long long)heavy);
  }
}

// ------------------------------------------------------------------ scans

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_sums, T &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : T(0);
    T si = s;
    for (int o = 1; o < 32; o <<= 1) {
      T u = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += u;
    }
    warp_sums[lane] = si - s;  // exclusive per warp
    if (lane == 31) warp_sums[32] = si;
  }
  __syncthreads();
  total = warp_sums[32];
  return inc - v + warp_sums[warp];
}

// Exclusive scan of each tile; tile totals go to part[blockIdx.x]. In place is allowed.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const T *in, T *out, T *part, int64_t n) {
  __shared__ T ws[33];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (t0 + i < n) ? in[t0 + i] : T(0);
    s += v[i];
  }
  T total;
  T ex = block_exclusive_scan<T>(s, ws, total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (t0 + i < n) out[t0 + i] = ex;
    ex += v[i];
  }
  if (threadIdx.x == 0 && part) part[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_add(T *out, const T *part, int64_t n) {
  const T add = part[blockIdx.x];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
    if (t0 + i < n) out[t0 + i] += add;
}

// Sum of each tile of in[] into part[tile].
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_sum(const T *in, T *part, int64_t n) {
  __shared__ T ws[33];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) v += (t0 + i < n) ? in[t0 + i] : T(0);
  T total;
  block_exclusive_scan<T>(v, ws, total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Exclusive scan of each tile offset by the sum of the tiles before it (summed
// by the block itself from part[]); the last tile writes the grand total.
// In place is allowed.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_prefixed(const T *in, T *out,
                                                                const T *part, int64_t n,
                                                                T *total_out) {
  __shared__ T ws[33];
  T pre = 0;
  for (int64_t j = threadIdx.x; j < (int64_t)blockIdx.x; j += kScanThreads) pre += part[j];
  T pre_total;
  block_exclusive_scan<T>(pre, ws, pre_total);
  __syncthreads();  // ws is reused below
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (t0 + i < n) ? in[t0 + i] : T(0);
    sum += v[i];
  }
  T tile_total;
  T ex = block_exclusive_scan<T>(sum, ws, tile_total) + pre_total;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (t0 + i < n) out[t0 + i] = ex;
    ex += v[i];
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    *total_out = pre_total + tile_total;
}

// Exclusive scan; up to kScanDirectTiles tiles by a tile-sum pass and one
// prefixed scan pass, beyond that recursively (scratch holds the per-level
// partials). When total is not null, the grand total is written there.
constexpr int64_t kScanDirectTiles = 4096;
template <typename T>
cudaError_t scan_rec(const T *in, T *out, int64_t n, T *scratch, T *total, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t nt = ceil_div(n, kScanTile);
  if (nt > 1 && nt <= kScanDirectTiles) {
    k_tile_sum<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, scratch, n);
    k_scan_prefixed<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, out, scratch, n, total);
    return cudaGetLastError();
  }
  k_scan_tile<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, out, nt > 1 ? scratch : total, n);
  if (nt > 1) {
    cudaError_t e = scan_rec<T>(scratch, scratch, nt, scratch + nt, total, s);
    if (e != cudaSuccess) return e;
    k_scan_add<T><<<(unsigned)nt, 256, 0, s>>>(out, scratch, n);
  }
  return cudaGetLastError();
}

}  // namespace

// Exclusive scan of a uint32 array (in place allowed) using the context scratch.
ddhf_status launch_scan_u32(Ctx *c, const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s) {
  DDHF_CUDA_TRY(c, scan_rec<uint32_t>(in, out, n, c->scan_part, nullptr, s));
  return DDHF_OK;
}

// The same for uint64 (the scratch holds n / 2048 + 64 words of 64 bits).
ddhf_status launch_scan_u64(Ctx *c, const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s) {
  DDHF_CUDA_TRY(c, scan_rec<uint64_t>(in, out, n, reinterpret_cast<uint64_t *>(c->scan_part),
                                      nullptr, s));
  return DDHF_OK;
}

// k_scatter for a digit width of `bits` (1..kMaxDigitBits).
template <bool DROP, int BITS = 1>
void launch_scatter(int bits, int64_t nch, cudaStream_t s, const uint32_t *kin,
                    const uint32_t *vin, int64_t n_in, const uint32_t *n_total, uint32_t *kout,
                    uint32_t *vout, const uint32_t *hscan, int shift, uint32_t *flags) {
  if constexpr (BITS <= kMaxDigitBits) {
    if (bits != BITS)
      return launch_scatter<DROP, BITS + 1>(bits, nch, s, kin, vin, n_in, n_total, kout, vout,
                                            hscan, shift, flags);
    k_scatter<DROP, BITS><<<(unsigned)nch, kScatThreads, scatter_smem_bytes(1 << BITS), s>>>(
        kin, vin, n_in, n_total, kout, vout, hscan, nch, shift, flags);
  }
}

template <bool DROP, int BITS = 1>
void scatter_attributes() {
  if constexpr (BITS <= kMaxDigitBits) {
    cudaFuncSetAttribute(k_scatter<DROP, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         scatter_smem_bytes(1 << BITS));
    scatter_attributes<DROP, BITS + 1>();
  }
}

ddhf_status bin_core(Ctx *c, Slot &sl, const RawIn &raw, int n_min, int heavy_min,
                     uint64_t *heavy_list, uint32_t *heavy_count, uint32_t slot_tag,
                     int64_t heavy_cap, cudaStream_t s) {
  const int64_t n = raw.n;
  const int64_t npx = c->npx;
  uint32_t *ntot = reinterpret_cast<uint32_t *>(c->qctl + 8);  // n_valid of this binning
  DDHF_CUDA_TRY(c, cudaMemsetAsync(ntot, 0, sizeof(uint32_t), s));
  DDHF_CUDA_TRY(c, cudaMemsetAsync(sl.counters, 0, 7 * sizeof(uint64_t), s));
  const int64_t nch = ceil_div(n, kBinChunk);
  uint32_t *kbuf[2] = {c->keysA, c->keysB};
  uint32_t *vbuf[2] = {c->valsA, c->valsB};
  int shift = 0;
  if (nch > 0) {
    for (int pass = 0; pass < c->npass; ++pass) {
      const int bits = c->digit_bits[pass];
      const int nb = 1 << bits;
      const bool last = pass == c->npass - 1;
      uint32_t *ko = kbuf[pass & 1];
      uint32_t *vo = last ? sl.ev : vbuf[pass & 1];
      const uint32_t *ki = pass ? kbuf[(pass - 1) & 1] : nullptr;
      const uint32_t *vi = pass ? vbuf[(pass - 1) & 1] : nullptr;
      // raw events are packed by the first histogram into the second buffer
      // pair (free until the second pass writes it) and sorted from there
      RawIn in = raw;
      if (pass == 0 && !raw.pk) {
        const bool vec = (reinterpret_cast<uintptr_t>(raw.x) % 8 == 0) &&
                         (reinterpret_cast<uintptr_t>(raw.y) % 8 == 0) &&
                         (reinterpret_cast<uintptr_t>(raw.t) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(raw.p) % 4 == 0);
        if (vec)
          k_hist_pack<true><<<(unsigned)nch, kBinThreads, 0, s>>>(raw, c->keysB, c->valsB,
                                                                  c->hist, nch, nb);
        else
          k_hist_pack<false><<<(unsigned)nch, kBinThreads, 0, s>>>(raw, c->keysB, c->valsB,
                                                                   c->hist, nch, nb);
        in.pk = c->keysB;
        in.pv = c->valsB;
      } else if (pass == 0) {
        k_hist<true><<<(unsigned)nch, kBinThreads, 0, s>>>(raw, nullptr, nullptr, c->hist, nch,
                                                           shift, nb);
      } else {
        k_hist<false><<<(unsigned)nch, kBinThreads, 0, s>>>(raw, ki, ntot, c->hist, nch, shift,
                                                            nb);
      }
      DDHF_CUDA_TRY(c, cudaGetLastError());
      // pass 0: the grand total of the table is the number of kept events
      DDHF_CUDA_TRY(c, scan_rec<uint32_t>(c->hist, c->hist, (int64_t)nb * nch, c->scan_part,
                                          pass == 0 ? ntot : nullptr, s));
      if (pass == 0)
        launch_scatter<true>(bits, nch, s, in.pk, in.pv, n, ntot, ko, vo, c->hist, shift,
                             c->flags);
      else
        launch_scatter<false>(bits, nch, s, ki, vi, n, ntot, ko, vo, c->hist, shift, c->flags);
      DDHF_CUDA_TRY(c, cudaGetLastError());
      shift += bits;
    }
  }
  const uint32_t *kfinal = kbuf[(c->npass - 1) & 1];
  DDHF_CUDA_TRY(c, cudaMemsetAsync(c->seg_lo, 0, npx * sizeof(uint32_t), s));
  DDHF_CUDA_TRY(c, cudaMemsetAsync(c->seg_hi, 0, npx * sizeof(uint32_t), s));
  const int sm_blocks = c->num_sms * 8;
  if (nch > 0) {
    k_seg<<<sm_blocks, 256, 0, s>>>(kfinal, ntot, c->seg_lo, c->seg_hi, npx, c->flags);
    DDHF_CUDA_TRY(c, cudaGetLastError());
  }
  unsigned pb = (unsigned)std::min<int64_t>(ceil_div(npx + 1, 256), sm_blocks);
  k_pack<<<pb, 256, 0, s>>>(c->seg_lo, c->seg_hi, c->packed, npx, n_min);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  DDHF_CUDA_TRY(c, scan_rec<uint64_t>(c->packed, c->packed, npx + 1,
                                      reinterpret_cast<uint64_t *>(c->scan_part), nullptr, s));
  k_finish<<<pb, 256, 0, s>>>(c->packed, c->seg_lo, c->seg_hi, sl.offsets, sl.active,
                              sl.counters, npx, n_min, heavy_min, n, c->grid.n_bins, heavy_list,
                              heavy_count, slot_tag, heavy_cap, c->flags);
  DDHF_CUDA_TRY(c, cudaGetLastError());
  return DDHF_OK;
}

ddhf_status bin_window(Ctx *c, int slot_i, const int16_t *x, const int16_t *y, const int64_t *t,
                       const int8_t *p, int64_t n, int64_t t0, int64_t win, cudaStream_t s) {
  Slot &sl = c->slots[slot_i];
  sl.t0 = t0;
  sl.window_us = win;
  RawIn raw{x, y, t, p, n, t0, (uint64_t)win, c->W, c->H, c->params.polarity_01, c->row0};
  return bin_core(c, sl, raw, c->params.n_min, c->tuning.heavy_min, c->work, c->qctl,
                  (uint32_t)slot_i, c->heavy_cap, s);
}

// Stable sort of pre-packed (key, value) pairs into a slot's per-pixel list;
// key kDropKey marks pairs that are not kept.
ddhf_status bin_packed(Ctx *c, Slot &sl, const uint32_t *keys, const uint32_t *vals, int64_t n,
                       int n_min, int heavy_min, uint64_t *heavy_list, uint32_t *heavy_count,
                       int64_t heavy_cap, cudaStream_t s) {
  RawIn raw{nullptr, nullptr, nullptr, nullptr, n, 0, 0, c->W, c->H, 0, 0, keys, vals};
  return bin_core(c, sl, raw, n_min, heavy_min, heavy_list, heavy_count, 0u, heavy_cap, s);
}

void set_bin_attributes() {
  scatter_attributes<true>();
  scatter_attributes<false>();
}

}  // namespace ddhf
