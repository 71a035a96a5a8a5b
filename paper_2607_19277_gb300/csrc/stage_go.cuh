// Launch of the persistent per-stage update kernel for one physics trait and scheme.
#pragma once
#include "kernels.cuh"

namespace agile {

// CTAs per SM a staging layout allows, by the shared memory of an SM (233472 bytes, 1 KB
// reserved per CTA) and the register budget it implies: FP32 three when three CTAs fit, else
// two; FP64 two when two CTAs fit (hydrodynamics, whose FP64 kernel fits 128 registers), else
// one (its full register budget).
template <template <typename> class PT, typename R, int RAW, int SFB>
constexpr int stage_minb() {
  constexpr size_t SMEM = stage_smem_bytes<PT, R, RAW, SFB>();
  if (sizeof(R) == 8) return 2 * (SMEM + 1024) <= 233472 ? 2 : 1;
  return 3 * (SMEM + 1024) <= 233472 ? 3 : (2 * (SMEM + 1024) <= 233472 ? 2 : 1);
}

template <template <typename> class PT, typename R, int LIM, int FLUX, int RAW, int SFB>
static cudaError_t stage_go_layout(const StageArgs& a, cudaStream_t s) {
  constexpr size_t SMEM = stage_smem_bytes<PT, R, RAW, SFB>();
  constexpr int MINB = stage_minb<PT, R, RAW, SFB>();
  auto k = stage_kernel<PT, R, LIM, FLUX, MINB, RAW, SFB>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
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
  k<<<grid, 256, SMEM, s>>>(*static_cast<const CUtensorMap*>(args.tmap), args);
  return cudaGetLastError();
}

// Staging layouts: STAGE_LAYOUT_RING4 = four raw slots, one flux buffer, two barriers per
// plane; STAGE_LAYOUT_RING5_DB = five raw slots, two flux buffers, one barrier per plane.
// The default (layout 0) takes the second where it keeps as many CTAs per SM as the first
// (FP32 stencils only; FP64 keeps the first).
template <template <typename> class PT, typename R, int LIM, int FLUX>
static cudaError_t stage_go(const StageArgs& a, cudaStream_t s) {
  if constexpr (sizeof(R) == 8) {
    return stage_go_layout<PT, R, LIM, FLUX, 4, 1>(a, s);
  } else {
    constexpr bool db_default = stage_minb<PT, R, 5, 2>() >= stage_minb<PT, R, 4, 1>();
    const bool db = a.layout == STAGE_LAYOUT_RING5_DB || (a.layout == 0 && db_default);
    return db ? stage_go_layout<PT, R, LIM, FLUX, 5, 2>(a, s) : stage_go_layout<PT, R, LIM, FLUX, 4, 1>(a, s);
  }
}

}  // namespace agile
