// Instantiations of the per-stage update kernel for the hd physics module.
#include "kernels.cuh"
#include "launch.h"

namespace agile {

template <typename R, int LIM, int FLUX>
static cudaError_t go(const StageArgs& a, cudaStream_t s) {
  constexpr int MINB = sizeof(R) == 4 ? 2 : 1;   // CTAs per SM the register budget targets
  auto k = stage_kernel<HdPhys, R, LIM, FLUX, MINB>;
  const size_t smem = stage_smem_bytes<HdPhys, R>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  // persistent grid: as many CTAs as fit on the GPU at once, each looping over blocks
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int grid = a.nblk < MINB * sms ? a.nblk : MINB * sms;
  if (grid <= 0) return cudaSuccess;
  k<<<grid, 256, smem, s>>>(*static_cast<const CUtensorMap*>(a.tmap), a);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t go_r(int lim, int flux, const StageArgs& a, cudaStream_t s) {
  if (flux == FLUX_HLLC)   // hydrodynamics only (paper Table 1)
    return lim == LIM_MINMOD ? go<R, LIM_MINMOD, FLUX_HLLC>(a, s) : go<R, LIM_VANLEER, FLUX_HLLC>(a, s);
  if (lim == LIM_MINMOD)
    return flux == FLUX_HLL ? go<R, LIM_MINMOD, FLUX_HLL>(a, s) : go<R, LIM_MINMOD, FLUX_TVDLF>(a, s);
  return flux == FLUX_HLL ? go<R, LIM_VANLEER, FLUX_HLL>(a, s) : go<R, LIM_VANLEER, FLUX_TVDLF>(a, s);
}

cudaError_t launch_stage_hd(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s) {
  return real_bytes == 8 ? go_r<double>(lim, flux, a, s) : go_r<float>(lim, flux, a, s);
}

}  // namespace agile
