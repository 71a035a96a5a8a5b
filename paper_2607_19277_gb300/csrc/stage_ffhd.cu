// Instantiations of the per-stage update kernel for the ffhd physics module.
#include "launch.h"
#include "stage_go.cuh"

namespace agile {

template <typename R>
static cudaError_t go_r(int lim, int flux, const StageArgs& a, cudaStream_t s) {
  if (flux != FLUX_TVDLF) return cudaErrorInvalidValue;   // ffhd: TVDLF only (paper Table 1)
  return lim == LIM_MINMOD ? stage_go<FfhdPhys, R, LIM_MINMOD, FLUX_TVDLF>(a, s)
                           : stage_go<FfhdPhys, R, LIM_VANLEER, FLUX_TVDLF>(a, s);
}

cudaError_t launch_stage_ffhd(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s) {
  return real_bytes == 8 ? go_r<double>(lim, flux, a, s) : go_r<float>(lim, flux, a, s);
}

}  // namespace agile
