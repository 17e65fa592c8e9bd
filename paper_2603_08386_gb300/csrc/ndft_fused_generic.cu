// Instantiations of the fused persistent kernel (spectra + SF + comb) with
// the generic comb, for spectra of more than 1024 bins or wide median bands
// (1 or 8 band-mask words per window centre).
#include "ndft_blocked.cuh"

namespace ddhf {
namespace blocked {
template ddhf_status launch_blocked_tb<1, true>(Ctx *, int, float *, int64_t, cudaStream_t, int,
                                                int64_t, int);
template ddhf_status launch_blocked_tb<8, true>(Ctx *, int, float *, int64_t, cudaStream_t, int,
                                                int64_t, int);
}  // namespace blocked
}  // namespace ddhf
