// Instantiation of the persistent blocked NDFT kernel that writes spectra to
// global memory (ddhf_power_spectrum with DDHF_FORM_BLOCKED).
#include "ndft_blocked.cuh"

namespace ddhf {
ddhf_status launch_blocked_spectrum(Ctx *c, float *P, int64_t cap_px, cudaStream_t s) {
  return blocked::launch_blocked_any<false>(c, 1, P, cap_px, s);
}

// Spectra of one window slot (its heavy items must be the only ones queued).
ddhf_status launch_spectrum_slot(Ctx *c, int slot, float *P, int64_t cap_px, cudaStream_t s,
                                 int64_t ld) {
  return blocked::launch_blocked_any<false>(c, 1, P, cap_px, s, slot, ld);
}
}  // namespace ddhf
