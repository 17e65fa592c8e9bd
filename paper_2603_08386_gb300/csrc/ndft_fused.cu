// Instantiation of the persistent blocked NDFT kernel with spectral flatness
// and comb scoring fused into it (ddhf_detect, ddhf_detect_batch): spectra
// stay in shared memory.
#include "ndft_blocked.cuh"

namespace ddhf {
ddhf_status launch_fused(Ctx *c, int n_slots, bool, float *, int64_t, cudaStream_t s) {
  return blocked::launch_blocked_any<true>(c, n_slots, nullptr, 0, s);
}
}  // namespace ddhf
