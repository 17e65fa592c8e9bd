// Comb scoring (Eq. 7-11) of spectra held as complex sums F (the sliding
// window's state): the kernel squares |F_j| as it loads each row.
#include "comb_kernel.cuh"

namespace ddhf {

ddhf_status launch_comb_cplx(Ctx *c, const float2 *F, int64_t ldF, float *log_sf, float *snr,
                             int32_t *f0, uint8_t *mask, cudaStream_t s) {
  return launch_comb_t<true>(c, reinterpret_cast<const float *>(F), c->npx, log_sf, snr, f0,
                             mask, s, 0, ldF);
}

}  // namespace ddhf
