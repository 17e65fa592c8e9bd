// Comb scoring (Eq. 7-11) of spectra stored as FP32 powers, one warp per
// active pixel (ddhf_comb_score and the unfused detection path).
#include "comb_kernel.cuh"

namespace ddhf {

ddhf_status launch_comb(Ctx *c, const float *P, int64_t cap_px, float *log_sf, float *snr,
                        int32_t *f0, uint8_t *mask, cudaStream_t s, int slot, int64_t ld) {
  return launch_comb_t<false>(c, P, cap_px, log_sf, snr, f0, mask, s, slot, ld);
}

}  // namespace ddhf
