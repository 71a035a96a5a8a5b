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
// plane; STAGE_LAYOUT_RING5_DB = five raw slots, two flux buffers, one barrier per plane;
// STAGE_LAYOUT_RING3_DB = three raw slots, two flux buffers, one barrier per plane, the update
// reading its stage input from global memory (L2) instead of a raw slot. The default (layout
// 0) takes layout 2 where it keeps as many CTAs per SM as layout 1, else layout 1 (FP32
// stencils; FP64 keeps layout 1). Layout 3 is an autotuner choice: at equal CTAs per SM its
// global re-read of U_s costs about what its saved barrier gains (MHD 0.870 against 0.860 ms,
// FFHD 0.459 against 0.450 ms per 256^3 stage launch).
template <template <typename> class PT, typename R, int LIM, int FLUX>
static cudaError_t stage_go(const StageArgs& a, cudaStream_t s) {
  if constexpr (sizeof(R) == 8) {
    return stage_go_layout<PT, R, LIM, FLUX, 4, 1>(a, s);
  } else {
    constexpr int dflt = stage_minb<PT, R, 5, 2>() >= stage_minb<PT, R, 4, 1>() ? STAGE_LAYOUT_RING5_DB
                                                                                 : STAGE_LAYOUT_RING4;
    const int lay = a.layout == 0 ? dflt : a.layout;
    if (lay == STAGE_LAYOUT_RING5_DB) return stage_go_layout<PT, R, LIM, FLUX, 5, 2>(a, s);
    if (lay == STAGE_LAYOUT_RING3_DB) return stage_go_layout<PT, R, LIM, FLUX, 3, 2>(a, s);
    return stage_go_layout<PT, R, LIM, FLUX, 4, 1>(a, s);
  }
}

}  // namespace agile
