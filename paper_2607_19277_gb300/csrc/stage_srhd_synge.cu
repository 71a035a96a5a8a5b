// Instantiations of the per-stage update kernel for the srhd physics module with the
// approximate Synge-gas EOS (Section 2.3.4).
#include "launch.h"
#include "stage_go.cuh"

namespace agile {

template <typename R>
static cudaError_t go_r(int lim, int flux, const StageArgs& a, cudaStream_t s) {
  if (flux != FLUX_TVDLF) return cudaErrorInvalidValue;   // srhd: TVDLF only (paper Table 1)
  return lim == LIM_MINMOD ? stage_go<SrhdSyngePhys, R, LIM_MINMOD, FLUX_TVDLF>(a, s)
                           : stage_go<SrhdSyngePhys, R, LIM_VANLEER, FLUX_TVDLF>(a, s);
}

cudaError_t launch_stage_srhd_synge(int real_bytes, int lim, int flux, const StageArgs& a,
                                    cudaStream_t s) {
  return real_bytes == 8 ? go_r<double>(lim, flux, a, s) : go_r<float>(lim, flux, a, s);
}

}  // namespace agile
