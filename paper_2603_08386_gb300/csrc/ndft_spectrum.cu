// Instantiation of the persistent blocked NDFT kernel that writes spectra to
// global memory (ddhf_power_spectrum with DDHF_FORM_BLOCKED).
#include "ndft_blocked.cuh"

namespace ddhf {
ddhf_status launch_blocked_spectrum(Ctx *c, float *P, int64_t cap_px, cudaStream_t s) {
  return blocked::launch_blocked_any<false>(c, 1, P, cap_px, s);
}

// Pixels of slot `slot` with at least the plan's threshold of events through
// the hybrid grid path, the others through the blocked kernel; without a plan
// (hybrid_min 0, or a window whose grid does not fit) all through the latter.
ddhf_status spectrum_with_hybrid(Ctx *c, int slot, int hybrid_min, float *P, int64_t cap_px,
                                 cudaStream_t s, int64_t ld) {
  int skip = 0;
  if (hybrid_min > 0 && c->hyb_c) {
    const HybridPlan hp = hybrid_plan(c, c->slots[slot].window_us, hybrid_min);
    if (hp.ok) {
      const ddhf_status st = launch_hybrid(c, slot, hp, P, cap_px, ld, s);
      if (st != DDHF_OK) return st;
      skip = (int)hp.thr;
    }
  }
  return blocked::launch_blocked_any<false>(c, 1, P, cap_px, s, slot, ld, skip);
}

// Spectra of one window slot (its heavy items must be the only ones queued),
// with the tuning's hybrid threshold.
ddhf_status launch_spectrum_slot(Ctx *c, int slot, float *P, int64_t cap_px, cudaStream_t s,
                                 int64_t ld) {
  return spectrum_with_hybrid(c, slot, c->tuning.hybrid_min, P, cap_px, s, ld);
}

// ddhf_power_spectrum with DDHF_FORM_HYBRID: slot 0, rows of n_bins floats.
ddhf_status launch_hybrid_spectrum(Ctx *c, float *P, int64_t cap_px, cudaStream_t s) {
  const ddhf_status st = hybrid_alloc(c);
  if (st != DDHF_OK) return st;
  const int hm = c->tuning.hybrid_min > 0 ? c->tuning.hybrid_min : kHybDefaultMin;
  return spectrum_with_hybrid(c, 0, hm, P, cap_px, s, c->grid.n_bins);
}
}  // namespace ddhf
