// Instantiations of the per-stage update kernel for the ffhd physics module (with and
// without hyperbolic thermal conduction).
#include "launch.h"
#include "stage_go.cuh"

namespace agile {

template <template <typename> class PT, typename R>
static cudaError_t go_r(int lim, int flux, const StageArgs& a, cudaStream_t s) {
  if (flux != FLUX_TVDLF) return cudaErrorInvalidValue;   // ffhd: TVDLF only (paper Table 1)
  return lim == LIM_MINMOD ? stage_go<PT, R, LIM_MINMOD, FLUX_TVDLF>(a, s)
                           : stage_go<PT, R, LIM_VANLEER, FLUX_TVDLF>(a, s);
}

cudaError_t launch_stage_ffhd(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s) {
  return real_bytes == 8 ? go_r<FfhdPhys, double>(lim, flux, a, s) : go_r<FfhdPhys, float>(lim, flux, a, s);
}

cudaError_t launch_stage_ffhd_htc(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s) {
  return real_bytes == 8 ? go_r<FfhdHtcPhys, double>(lim, flux, a, s)
                         : go_r<FfhdHtcPhys, float>(lim, flux, a, s);
}

}  // namespace agile
