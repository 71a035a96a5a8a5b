// Instantiations of the per-stage update kernel for the mhd module with resistivity.
#include "launch.h"
#include "stage_go.cuh"

namespace agile {

template <typename R>
static cudaError_t go_r(int lim, int flux, const StageArgs& a, cudaStream_t s) {
  if (lim == LIM_MINMOD)
    return flux == FLUX_HLL ? stage_go<MhdResPhys, R, LIM_MINMOD, FLUX_HLL>(a, s)
                            : stage_go<MhdResPhys, R, LIM_MINMOD, FLUX_TVDLF>(a, s);
  return flux == FLUX_HLL ? stage_go<MhdResPhys, R, LIM_VANLEER, FLUX_HLL>(a, s)
                          : stage_go<MhdResPhys, R, LIM_VANLEER, FLUX_TVDLF>(a, s);
}

cudaError_t launch_stage_mhd_res(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s) {
  return real_bytes == 8 ? go_r<double>(lim, flux, a, s) : go_r<float>(lim, flux, a, s);
}

}  // namespace agile
