// Launch of the persistent per-stage update kernel for one physics trait and scheme.
#pragma once
#include "kernels.cuh"

namespace agile {

template <template <typename> class PT, typename R, int LIM, int FLUX>
static cudaError_t stage_go(const StageArgs& a, cudaStream_t s) {
  // CTAs per SM the register budget targets: 1 in FP64; in FP32 3 when three CTAs' shared
  // memory fits an SM (233472 bytes, 1 KB reserved per CTA), else 2
  constexpr size_t SMEM = stage_smem_bytes<PT, R>();
  constexpr int MINB = sizeof(R) == 8 ? 1 : (3 * (SMEM + 1024) <= 233472 ? 3 : 2);
  auto k = stage_kernel<PT, R, LIM, FLUX, MINB>;
  const size_t smem = SMEM;
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
  int grid = a.grid > 0 ? a.grid : MINB * sms;   // a tuned persistent grid, else the default
  if (grid > a.nblk) grid = a.nblk;
  if (grid <= 0) return cudaSuccess;
  StageArgs args = a;
  args.ppf.set(a.gamma, 0.0);
  args.fa = (float)a.a;
  args.fb = (float)a.b;
  args.combine = a.a != 0.0 ? 1 : 0;
  k<<<grid, 256, smem, s>>>(*static_cast<const CUtensorMap*>(args.tmap), args);
  return cudaGetLastError();
}

}  // namespace agile
