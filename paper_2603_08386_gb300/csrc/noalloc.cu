// ddhf_power_spectrum_noalloc: the BLOCKED NDFT power spectra computed from a
// per-pixel event list that the caller built and owns, with no device memory
// allocated by the library.
//
// Who needs it: callers that must not allocate device memory once they are
// running, e.g. a detector on a drone or another embedded real-time system
// that reserves all memory at start-up (cudaMalloc can synchronise the device
// and take milliseconds, which breaks a 33 ms frame budget), or a host program
// whose own memory manager owns the whole device. ddhf_create() allocates a
// workspace, so those callers cannot use the context-based entry points.
//
// The kernel's scratch (work-queue counters, the list of heavy pixels, the
// per-window view the persistent kernel reads) lives in one file-scope
// __device__ array of fixed size, present on every device that loads the
// library until the process exits. Host code only knows a stand-in for that
// symbol, so its device address is fetched once per device with
// cudaGetSymbolAddress(), during the first call made with that device
// current; that first call should therefore come before any stream capture.
// Every call shares the array: the counters are cleared at the start of each
// call, and two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "ndft_blocked.cuh"

namespace ddhf {
namespace {

constexpr int64_t kNoAllocMaxEvents = (int64_t)1 << 25;  // per call
constexpr int kNoAllocHeavyMin = 1024;                   // same default as a context
constexpr int64_t kNoAllocMaxHeavy = kNoAllocMaxEvents / kNoAllocHeavyMin;  // 32768
constexpr int kNoAllocWarps = 4;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  SlotView view;
  uint64_t counters[8];  // [2] = number of active pixels
  uint32_t qctl[4];      // [0] heavy count, [1] heavy cursor, [2] light cursor
  uint32_t flags;
  uint32_t pad[3];
  uint64_t heavy[kNoAllocMaxHeavy];  // heavy work items (slot 0 << 32 | active index)
};

// 256-byte aligned; 256 KiB of heavy items plus a small header.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_addr_mu;
NoAllocScratch *g_addr[kMaxDevices] = {};

__global__ void k_noalloc_prepare(NoAllocScratch *s, const uint32_t *ev, const uint32_t *offsets,
                                  const uint32_t *active, int64_t n_active) {
  if (threadIdx.x == 0) {
    s->view = SlotView{ev, offsets, active, s->counters, nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 8; ++i) s->counters[i] = 0;
    s->counters[2] = (uint64_t)n_active;
    for (int i = 0; i < 4; ++i) s->qctl[i] = 0;
    s->flags = 0;
  }
}

__global__ void k_noalloc_heavy(NoAllocScratch *s, const uint32_t *offsets, const uint32_t *active,
                                int64_t n_active) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_active;
       a += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = active[a];
    if (offsets[k + 1] - offsets[k] >= (uint32_t)kNoAllocHeavyMin) {
      const uint32_t pos = atomicAdd(&s->qctl[0], 1u);
      if ((int64_t)pos < kNoAllocMaxHeavy) s->heavy[pos] = (uint32_t)a;
    }
  }
}

template <int TB>
ddhf_status launch_noalloc(NoAllocScratch *sp, const GridConst &g, float *P, int64_t cap_px,
                           int64_t n_active, int num_sms, cudaStream_t s) {
  blocked::BlockedArgs A{};
  A.views = &sp->view;
  A.slot0 = 0;
  A.n_slots = 1;
  A.npx = n_active;  // light pixels: virtual index over the active list
  A.heavy = sp->heavy;
  A.n_heavy = &sp->qctl[0];
  A.heavy_cap = (uint32_t)kNoAllocMaxHeavy;
  A.cursors = &sp->qctl[1];
  A.g = g;
  A.cc = CombConst{};
  A.P = P;
  A.ld = g.N;
  A.vec_store = (A.ld % 4 == 0) && (reinterpret_cast<uintptr_t>(P) % 16 == 0);
  A.cap_px = cap_px;
  A.heavy_min = kNoAllocHeavyMin;
  const int stage = blocked::WarpLayout<TB>::kStageF4 * 16;
  const int partial = 3 * TB * 4 * 32 * 4;
  const int scratch = ((stage > partial ? stage : partial) + 15) & ~15;
  A.pw_offset = scratch;
  A.warp_bytes = scratch + 4 * TB * 32 * 4;
  A.flags = &sp->flags;
  const size_t smem = (size_t)A.warp_bytes * kNoAllocWarps;
  auto kern = blocked::k_blocked<TB, 1, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DDHF_ERR_CUDA;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kNoAllocWarps * 32, smem) !=
          cudaSuccess ||
      occ < 1)
    return DDHF_ERR_CUDA;
  kern<<<num_sms * occ, kNoAllocWarps * 32, smem, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? DDHF_OK : DDHF_ERR_CUDA;
}

}  // namespace
}  // namespace ddhf

using namespace ddhf;

extern "C" ddhf_status ddhf_power_spectrum_noalloc(const ddhf_grid *grid, const uint32_t *offsets,
                                                   const uint32_t *ev, int64_t n_events,
                                                   const uint32_t *active, int64_t n_active,
                                                   float *P, int64_t cap_px, ddhf_stream stream) {
  if (!grid || !offsets || !active || !P) return DDHF_ERR_INVALID_ARG;
  if (n_events < 0 || n_events > kNoAllocMaxEvents) return DDHF_ERR_INVALID_ARG;
  if (n_events > 0 && !ev) return DDHF_ERR_INVALID_ARG;
  if (n_active < 0 || n_active > ((int64_t)1 << 26) || cap_px < n_active)
    return DDHF_ERR_INVALID_ARG;
  if (grid->a0 < 0 || grid->da <= 0 || grid->denom <= 0 || grid->denom >= ((int64_t)1 << 31) ||
      grid->n_bins < 1 || grid->n_bins > 16384)
    return DDHF_ERR_INVALID_ARG;
  if ((double)grid->a0 + (double)grid->da * (grid->n_bins - 1 + 31) >= 4294967296.0)
    return DDHF_ERR_INVALID_ARG;
  int dev = 0, num_sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DDHF_ERR_CUDA;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DDHF_ERR_CUDA;
  NoAllocScratch *sp = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DDHF_ERR_CUDA;
      g_addr[dev] = static_cast<NoAllocScratch *>(p);
    }
    sp = g_addr[dev];
  }
  if (n_active == 0) return DDHF_OK;
  GridConst g;
  g.a0 = (uint64_t)grid->a0;
  g.da = (uint64_t)grid->da;
  g.denom = (uint64_t)grid->denom;
  g.barrett = ~0ull / (uint64_t)grid->denom;
  g.a0_mod = (uint64_t)grid->a0 % (uint64_t)grid->denom;
  g.da_mod = (uint64_t)grid->da % (uint64_t)grid->denom;
  g.da16_mod = ((uint64_t)grid->da * 16ull) % (uint64_t)grid->denom;
  g.da32_mod = ((uint64_t)grid->da * 32ull) % (uint64_t)grid->denom;
  g.N = grid->n_bins;
  g.nbr = (grid->n_bins + 31) / 32;
  g.two_over_denom = (float)(2.0 / (double)grid->denom);
  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_prepare<<<1, 32, 0, s>>>(sp, ev, offsets, active, n_active);
  const int blocks = (int)std::min<int64_t>(ceil_div(n_active, 256), (int64_t)num_sms * 8);
  k_noalloc_heavy<<<blocks, 256, 0, s>>>(sp, offsets, active, n_active);
  if (cudaGetLastError() != cudaSuccess) return DDHF_ERR_CUDA;
  int tb = std::min(8, (g.nbr + 3) / 4);
  tb = tb <= 2 ? tb : tb <= 4 ? 4 : tb <= 6 ? 6 : 8;
  switch (tb) {
    case 1: return launch_noalloc<1>(sp, g, P, cap_px, n_active, num_sms, s);
    case 2: return launch_noalloc<2>(sp, g, P, cap_px, n_active, num_sms, s);
    case 4: return launch_noalloc<4>(sp, g, P, cap_px, n_active, num_sms, s);
    case 6: return launch_noalloc<6>(sp, g, P, cap_px, n_active, num_sms, s);
    default: return launch_noalloc<8>(sp, g, P, cap_px, n_active, num_sms, s);
  }
}
