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
// per-window view the persistent kernel reads, the flags) lives in one
// file-scope __device__ array of fixed size, present on every device that
// loads the library until the process exits. Host code only knows a stand-in
// for that symbol, so its device address is fetched with
// cudaGetSymbolAddress() once per CUDA context (keyed by the context's
// process-unique id), during the first call made with that context current.
// That first call also loads every kernel this entry point can launch (all
// five rows-per-lane instantiations of the spectrum kernel and the helpers),
// so that under lazy module loading no later call, whatever its grid, loads
// code or allocates; it should therefore come before any stream capture and
// outside any frame budget. Every call shares the array: the counters and
// flags are cleared at the start of each call, and two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.
#include <cuda.h>

#include <mutex>

#include "ndft_blocked.cuh"

namespace ddhf {
namespace {

constexpr int64_t kNoAllocMaxEvents = (int64_t)1 << 25;  // per call
constexpr int kNoAllocHeavyMin = 1024;                   // same default as a context
constexpr int64_t kNoAllocMaxHeavy = kNoAllocMaxEvents / kNoAllocHeavyMin;  // 32768
constexpr int kNoAllocWarps = 4;
constexpr int kMaxContexts = 64;

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

// Heavy pixels (at least kNoAllocHeavyMin events) into the work list. With
// offsets that stay within the n_events <= kNoAllocMaxEvents events of the
// call the list cannot overflow; a pixel that does not fit (offsets beyond
// n_events) gets a row of NaN and raises DDHF_FLAG_CAPACITY.
__global__ void k_noalloc_heavy(NoAllocScratch *s, const uint32_t *offsets, const uint32_t *active,
                                int64_t n_active, float *P, int n_bins) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_active;
       a += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = active[a];
    if (offsets[k + 1] - offsets[k] >= (uint32_t)kNoAllocHeavyMin) {
      const uint32_t pos = atomicAdd(&s->qctl[0], 1u);
      if ((int64_t)pos < kNoAllocMaxHeavy) {
        s->heavy[pos] = (uint32_t)a;
      } else {
        atomicOr(&s->flags, DDHF_FLAG_CAPACITY);
        for (int j = 0; j < n_bins; ++j) P[a * n_bins + j] = __int_as_float(0x7fc00000);
      }
    }
  }
}

// The DDHF_FLAG_* bits this call raised, into the caller's word.
__global__ void k_noalloc_finish(const NoAllocScratch *s, uint32_t *flags_out) {
  if (threadIdx.x == 0) *flags_out = s->flags;
}

// Scratch address per CUDA context: (process-unique context id, address).
struct AddrEntry {
  unsigned long long ctx_id;
  NoAllocScratch *addr;
};
std::mutex g_addr_mu;
AddrEntry g_addr[kMaxContexts] = {};
int g_addr_n = 0;

typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the current context (0 when none is current or the query fails).
unsigned long long current_ctx_id() {
  static CtxGetIdFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetIdFn>(f);
    looked = true;
  }
  unsigned long long id = 0;
  if (!fn || fn(nullptr, &id) != CUDA_SUCCESS) return 0;
  return id;
}

template <int TB>
cudaError_t load_blocked() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, blocked::k_blocked<TB, 1, false>);
}

// The scratch address for the current context: looked up, and every kernel of
// this entry point loaded, on the context's first call.
ddhf_status scratch_for_current(NoAllocScratch **out) {
  std::lock_guard<std::mutex> lock(g_addr_mu);
  unsigned long long id = current_ctx_id();
  for (int i = 0; id != 0 && i < g_addr_n; ++i)
    if (g_addr[i].ctx_id == id) {
      *out = g_addr[i].addr;
      return DDHF_OK;
    }
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DDHF_ERR_CUDA;
  cudaFuncAttributes fa;
  if (load_blocked<1>() != cudaSuccess || load_blocked<2>() != cudaSuccess ||
      load_blocked<4>() != cudaSuccess || load_blocked<6>() != cudaSuccess ||
      load_blocked<8>() != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_noalloc_prepare) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_noalloc_heavy) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_noalloc_finish) != cudaSuccess)
    return DDHF_ERR_CUDA;
  if (id == 0) id = current_ctx_id();  // the symbol lookup made the primary context current
  if (id != 0 && g_addr_n < kMaxContexts) g_addr[g_addr_n++] = AddrEntry{id, static_cast<NoAllocScratch *>(p)};
  *out = static_cast<NoAllocScratch *>(p);
  return DDHF_OK;
}

template <int TB>
ddhf_status launch_noalloc(NoAllocScratch *sp, const GridConst &g, float *P, int64_t cap_px,
                           int64_t n_active, int64_t n_events, int num_sms, cudaStream_t s) {
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
  A.ev_cap = n_events;
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
                                                   float *P, int64_t cap_px, uint32_t *flags_dev,
                                                   ddhf_stream stream) {
  if (!grid || !offsets || !active || !P) return DDHF_ERR_INVALID_ARG;
  if (n_events < 0 || n_events > kNoAllocMaxEvents) return DDHF_ERR_INVALID_ARG;
  if (n_events > 0 && !ev) return DDHF_ERR_INVALID_ARG;
  if (n_active < 0 || n_active > ((int64_t)1 << 26) || cap_px < n_active)
    return DDHF_ERR_INVALID_ARG;
  if (!grid_ok(grid)) return DDHF_ERR_INVALID_ARG;
  int dev = 0, num_sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DDHF_ERR_CUDA;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DDHF_ERR_CUDA;
  NoAllocScratch *sp = nullptr;
  const ddhf_status ss = scratch_for_current(&sp);
  if (ss != DDHF_OK) return ss;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_active == 0) {
    if (flags_dev && cudaMemsetAsync(flags_dev, 0, sizeof(uint32_t), s) != cudaSuccess)
      return DDHF_ERR_CUDA;
    return DDHF_OK;
  }
  const GridConst g = make_grid_const(*grid);
  k_noalloc_prepare<<<1, 32, 0, s>>>(sp, ev, offsets, active, n_active);
  const int blocks = (int)std::min<int64_t>(ceil_div(n_active, 256), (int64_t)num_sms * 8);
  k_noalloc_heavy<<<blocks, 256, 0, s>>>(sp, offsets, active, n_active, P, g.N);
  if (cudaGetLastError() != cudaSuccess) return DDHF_ERR_CUDA;
  int tb = std::min(8, (g.nbr + 3) / 4);
  tb = tb <= 2 ? tb : tb <= 4 ? 4 : tb <= 6 ? 6 : 8;
  ddhf_status st;
  switch (tb) {
    case 1: st = launch_noalloc<1>(sp, g, P, cap_px, n_active, n_events, num_sms, s); break;
    case 2: st = launch_noalloc<2>(sp, g, P, cap_px, n_active, n_events, num_sms, s); break;
    case 4: st = launch_noalloc<4>(sp, g, P, cap_px, n_active, n_events, num_sms, s); break;
    case 6: st = launch_noalloc<6>(sp, g, P, cap_px, n_active, n_events, num_sms, s); break;
    default: st = launch_noalloc<8>(sp, g, P, cap_px, n_active, n_events, num_sms, s); break;
  }
  if (st != DDHF_OK) return st;
  if (flags_dev) {
    k_noalloc_finish<<<1, 32, 0, s>>>(sp, flags_dev);
    if (cudaGetLastError() != cudaSuccess) return DDHF_ERR_CUDA;
  }
  return DDHF_OK;
}
