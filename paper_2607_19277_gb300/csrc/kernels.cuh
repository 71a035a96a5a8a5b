// Device kernels of the block update (sm_103a).
//
// stage_kernel is the per-stage macro-kernel (paper Section 2.1.3): one CTA per 16^3
// block, 256 threads, one thread per (x, y) column marching along z. Per plane it
// recovers primitives (interior from a per-thread register window, the x/y halo from the
// neighbours through the block's face table), reconstructs (PLM) and solves the Riemann
// problem at each x-, y- and z-face ONCE (x/y faces through shared memory, z faces kept
// in registers between planes), then forms -div F and the SSPRK stage combine. The
// paper's OpenACC version recomputes each face from both sides; here every face flux is
// evaluated once.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "agile_internal.h"
#include "pair.cuh"
#include "physics.cuh"

namespace agile {

enum : int { STAGE_LAYOUT_RING4 = 1, STAGE_LAYOUT_RING5_DB = 2, STAGE_LAYOUT_RING3_DB = 3 };

struct StageArgs {
  const void* Us;           // stage input state (with aux)
  const void* Un;           // U^n for the combine (a != 0)
  void* Uout;               // stage output
  const BlockDesc* bd;
  const void* gs;           // ghost slots
  void* fr;                 // flux registers (nullptr: none)
  const double* dtch;       // device [dt, c_h]
  double a, b;              // U_out = a U^n + b (U_s + dt L(U_s))
  double gamma;
  double glm_alpha;
  int glm_post;             // multiply psi of the output by exp(-dt/2 c_h alpha / min dx)
  int nblk;
  int* status;
  unsigned long long* speeds;   // fused reduction of [max sum_d s_d/dx_d, max s_d] per solve, or nullptr
  const void* tmap;             // host CUtensorMap of the pool Us, or of W for a physics with a
                                // primitive-recovery pass (x, y, z, block*var)
  const void* W = nullptr;      // primitives (and auxiliaries) of Us, per block as Us, from the
                                // recovery pass (physics with prim_pass_of), else unused
  const void* WG = nullptr;     // the same for the ghost slots
  const int* solve_of;          // solve index of each block (batched solves), nullptr = one solve
  int* work;                    // block counter of this launch (zeroed before it), dynamic scheduling
  int grid = 0;                 // persistent CTAs of the launch (0: CTAs-per-SM target x SMs)
  double htc_kappa0 = 0.0;      // ffhd with conduction: kappa_par = htc_kappa0 T^(5/2)
  int layout = 0;               // staging layout (STAGE_LAYOUT_*), 0: the default for the physics
  double eta = 0.0;             // resistive mhd: uniform resistivity
  const int* wl = nullptr;      // work list: pool block of each of the nblk work items (nullptr: identity)
  // FP32 copies of the equation parameters and the combine weights, formed on the host at
  // launch (stage_go), so that the FP32 kernel never forms them from the FP64 fields (the
  // compiler may recompute such values at every use instead of holding them in registers)
  PhysParamsT<float> ppf;
  float fa = 0.0f, fb = 0.0f;
  int combine = 0;
};

// Conserved + auxiliary values of the cell (x, y, z) of block b in the halo view: the
// interior, a same-level neighbour's interior, a physical boundary image or a ghost slot.
template <class P, typename R>
__device__ __forceinline__ void load_cell(const R* __restrict__ U, const R* __restrict__ G,
                                          const int* src, int b, int x, int y, int z, R* u) {
  constexpr int NT = P::NV + P::NA;
  int f = -1;
  if (x < 0) f = 0;
  else if (x > NB - 1) f = 1;
  else if (y < 0) f = 2;
  else if (y > NB - 1) f = 3;
  else if (z < 0) f = 4;
  else if (z > NB - 1) f = 5;
  int q[3] = {x, y, z};
  int blk = b;
  if (f >= 0) {
    const int d = f >> 1, s = f & 1;
    const int sv = src[f];
    if (sv >= 0) {
      q[d] &= NB - 1;
      blk = sv;
    } else if (sv == SRC_OUTFLOW) {
      q[d] = s ? NB - 1 : 0;
    } else if (sv == SRC_REFLECT) {
      q[d] = s ? 2 * NB - 1 - q[d] : -1 - q[d];
      const R* p = U + (size_t)blk * NT * NCELL + q[2] * 256 + q[1] * 16 + q[0];
#pragma unroll
      for (int v = 0; v < NT; ++v) u[v] = p[(size_t)v * NCELL];
      if (P::IV >= 0) u[P::IV + d] = -u[P::IV + d];
      if (P::BOFF >= 0) u[P::BOFF + d] = -u[P::BOFF + d];
      return;
    } else {
      const int slot = SRC_SLOT0 - sv;
      const int layer = s ? q[d] - NB : q[d] + 2;
      const int t1 = d == 0 ? q[1] : q[0];
      const int t2 = d == 2 ? q[1] : q[2];
      const R* p = G + (size_t)slot * NT * 512 + layer * 256 + t2 * 16 + t1;
#pragma unroll
      for (int v = 0; v < NT; ++v) u[v] = p[(size_t)v * 512];
      return;
    }
  }
  const R* p = U + (size_t)blk * NT * NCELL + q[2] * 256 + q[1] * 16 + q[0];
#pragma unroll
  for (int v = 0; v < NT; ++v) u[v] = p[(size_t)v * NCELL];
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Signal speeds of one cell, s_d = max |lambda_+-| along d, evaluated in the stencil
// precision R (the SRHD primitive recovery inside is FP64 always); the maxima
// ssum = max sum_d s_d / dx_d and smax = max_d s_d are accumulated in R (a maximum is exact
// in any precision; the caller widens the result to FP64 once). dxr = dx rounded to R.
template <template <typename> class PT, typename R>
__device__ __forceinline__ void prim_speeds(const R* p, const PhysParamsT<R>& pp, const R* dxr, R& ssum,
                                            R& smax) {
  using P = PT<R>;
  R lm, lp;
  P::template lambdas<0>(p, lm, lp, pp);
  const R s0 = rmax(rabs(lm), rabs(lp));
  P::template lambdas<1>(p, lm, lp, pp);
  const R s1 = rmax(rabs(lm), rabs(lp));
  P::template lambdas<2>(p, lm, lp, pp);
  const R s2 = rmax(rabs(lm), rabs(lp));
  smax = rmax(smax, rmax(rmax(s0, s1), s2));
  const R acc = (s0 / dxr[0] + s1 / dxr[1]) + s2 / dxr[2];
  ssum = rmax(ssum, acc);
}
// The same from the conserved values (and auxiliaries) of the cell.
template <template <typename> class PT, typename R>
__device__ __forceinline__ void cell_speeds(const R* u, R* aux, const PhysParamsT<R>& pp,
                                            const R* dxr, R& ssum, R& smax, int& st) {
  using P = PT<R>;
  R p[P::NV];
  P::cons2prim(u, p, aux, pp, st);
  prim_speeds<PT, R>(p, pp, dxr, ssum, smax);
}

// Maxima of a and b over the CTA, widened to FP64 once and merged into out[0..1] (non-negative
// values: their FP64 bit patterns order like the values). The reduction runs in the values'
// own precision (a maximum is exact in any precision).
template <int NTHREADS, typename T>
__device__ __forceinline__ void block_max2(T a, T b, unsigned long long* out) {
  __shared__ T ra[NTHREADS / 32], rb[NTHREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = rmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = rmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    ra[w] = a;
    rb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T ma = ra[0], mb = rb[0];
    for (int i = 1; i < NTHREADS / 32; ++i) {
      ma = rmax(ma, ra[i]);
      mb = rmax(mb, rb[i]);
    }
    atomic_max_pos(out, (double)ma);
    atomic_max_pos(out + 1, (double)mb);
  }
}

// --------------------------------------------------------------------------- TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` polls and reports it (no endless spin).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
}
// Whole-box tile load (4-D tensor map: x, y, z, block*var) into shared memory.
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <typename R>
__device__ __forceinline__ void cp_async_elem(R* dst, const R* src) {
  if constexpr (sizeof(R) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Address of variable 0 of cell (x, y, z) in the halo view of block b and the variable
// stride there (same pointer rules as load_cell); *neg_d is the dimension whose normal
// components a reflecting boundary negates, or -1.
template <class P, typename R>
__device__ __forceinline__ const R* cell_addr(const R* __restrict__ U, const R* __restrict__ G,
                                              const int* src, int b, int x, int y, int z, int* vstride,
                                              int* neg_d) {
  constexpr int NT = P::NV + P::NA;
  int f = -1;
  if (x < 0) f = 0;
  else if (x > NB - 1) f = 1;
  else if (y < 0) f = 2;
  else if (y > NB - 1) f = 3;
  else if (z < 0) f = 4;
  else if (z > NB - 1) f = 5;
  int q[3] = {x, y, z};
  int blk = b;
  *neg_d = -1;
  *vstride = NCELL;
  if (f >= 0) {
    const int d = f >> 1, s = f & 1;
    const int sv = src[f];
    if (sv >= 0) {
      q[d] &= NB - 1;
      blk = sv;
    } else if (sv == SRC_OUTFLOW) {
      q[d] = s ? NB - 1 : 0;
    } else if (sv == SRC_REFLECT) {
      q[d] = s ? 2 * NB - 1 - q[d] : -1 - q[d];
      *neg_d = d;
    } else {
      const int slot = SRC_SLOT0 - sv;
      const int layer = s ? q[d] - NB : q[d] + 2;
      const int t1 = d == 0 ? q[1] : q[0];
      const int t2 = d == 2 ? q[1] : q[2];
      *vstride = 512;
      return G + (size_t)slot * NT * 512 + layer * 256 + t2 * 16 + t1;
    }
  }
  return U + (size_t)blk * NT * NCELL + q[2] * 256 + q[1] * 16 + q[0];
}

// x/y component swap used to evaluate a y-face with the x-face solver.
template <class P, typename R>
__device__ __forceinline__ void swap_xy(R* v, bool yd) {
  if constexpr (P::IV >= 0) {
    const R a = v[P::IV], c = v[P::IV + 1];
    v[P::IV] = yd ? c : a;
    v[P::IV + 1] = yd ? a : c;
  }
  if constexpr (P::BOFF >= 0) {
    const R e = v[P::BOFF], g = v[P::BOFF + 1];
    v[P::BOFF] = yd ? g : e;
    v[P::BOFF + 1] = yd ? e : g;
  }
}

// Variable that takes slot v when the x and y vector components are exchanged.
template <class P>
__host__ __device__ constexpr int swapv(int v) {
  return (P::IV >= 0 && v == P::IV)          ? P::IV + 1
         : (P::IV >= 0 && v == P::IV + 1)    ? P::IV
         : (P::BOFF >= 0 && v == P::BOFF)     ? P::BOFF + 1
         : (P::BOFF >= 0 && v == P::BOFF + 1) ? P::BOFF
                                              : v;
}

constexpr uint32_t WAIT_LIMIT = 1u << 22;   // ~0.1 s of polling per wait at most
constexpr int ST_ETIMEOUT = 4;

// Slot of plane p (-2 .. 17) in the primitive ring of three 20 x 20 planes: plane p + 3 takes
// the slot of plane p.
__device__ __forceinline__ int pslot(int p) { return (p + 3) % 3; }

// Shared memory of the stage kernel for one staging layout: RAW raw-plane slots the TMA fills
// (4: the ring holds planes k .. k+3 at plane k; 5: one more plane in flight; 3: planes k+2 ..
// k+4 only, the update of plane k then reading its stage input from global memory, where the
// TMA has just passed it through L2) and SFB buffers of the x/y face fluxes (2: the fluxes of
// plane k+1 are formed while those of plane k are still being read, so one CTA barrier per
// plane suffices).
template <template <typename> class PT, typename R, int RAW, int SFB>
struct StageSmem {
  static constexpr int NV = PT<R>::NV, NT = PT<R>::NV + PT<R>::NA;
  static constexpr size_t bars = 128;                                  // RAW mbarriers (+pad)
  static constexpr size_t raw = bars;                                  // [RAW][NT][256]
  static constexpr size_t ring = raw + sizeof(R) * RAW * NT * 256;     // [3][NT][20 x 20]
  static constexpr size_t fx = ring + sizeof(R) * 3 * NT * 400;        // [SFB][NV][16 x 16 + 16]
  static constexpr size_t fy = fx + sizeof(R) * SFB * NV * 272;        // [SFB][NV][17][16]
  static constexpr size_t total = fy + sizeof(R) * SFB * NV * 272;
};

// The per-stage macro-kernel. Plane k of a block is one iteration:
//   A. primitives of plane k+2 of this thread's own column (raw data from the TMA ring) into
//      the primitive ring;
//   B. primitives of the x/y halo of plane k+1, whose raw values this thread fetched with
//      cp.async into the ring's 20 x 20 frame one plane earlier (converted in place; the two
//      halves of the CTA take turns), and the fetch of plane k+2's halo;
//   C. the x- and y-face fluxes of plane k (ring plane k: interior and halo, complete since
//      the previous barrier) into shared memory, and the z-face flux at k+1/2 (ring planes
//      k .. k+2 of this column, carried to the next plane in registers);
//   -- CTA barrier --
//   D. flux divergence, SSPRK combine and store of cell (x, y, k);
//   -- CTA barrier, with one flux buffer only: the next plane's faces overwrite it --
// Raw planes arrive by TMA one or two planes ahead of their conversion.
template <template <typename> class PT, typename R, int LIM, int FLUX, int MINB, int RAW, int SFB>
__global__ void __launch_bounds__(256, MINB) stage_kernel(const __grid_constant__ CUtensorMap tmap,
                                                           StageArgs A) {
  static_assert(RAW >= 3 && RAW <= 5, "three to five raw slots");
  static_assert((RAW == 4) == (SFB == 1), "one flux buffer with four raw slots, two with three or five");
  using P = PT<R>;
  // primitives come from a recovery pass of their own (A.W, A.WG, and the tensor map over
  // A.W): the ring is filled with them as they are, and the update reads U_s from global
  constexpr bool PRIMIN = prim_pass_of<P>::value;
  constexpr bool US_GLOBAL = RAW == 3 || PRIMIN;   // the update reads U_s of its cell from global memory
  using S = StageSmem<PT, R, RAW, SFB>;
  constexpr int NV = P::NV, NA = P::NA, NT = NV + NA;
  // FP32 HD / MHD with HLL or TVDLF: x- and y-faces solved as packed pairs
  constexpr bool PAIRED = sizeof(R) == 4 && PairPhys<P>::OK && (FLUX == FLUX_HLL || FLUX == FLUX_TVDLF);
  constexpr int NAW = NA > 0 ? NA : 1;
  constexpr bool RESP = res_of<P>::value;   // resistive MHD sources
  // completions of raw slot s's barrier per block (planes -2 .. 17 = TMA sequence 0 .. 19)
  auto phases = [](int s) { return (20 + RAW - 1 - s) / RAW; };
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  R* sRaw = reinterpret_cast<R*>(smem_raw + S::raw);
  R* sP = reinterpret_cast<R*>(smem_raw + S::ring);
  R* sFx0 = reinterpret_cast<R*>(smem_raw + S::fx);
  R* sFy0 = reinterpret_cast<R*>(smem_raw + S::fy);

  const R* __restrict__ Us = static_cast<const R*>(A.Us);
  const R* __restrict__ Un = static_cast<const R*>(A.Un);
  R* __restrict__ Uo = static_cast<R*>(A.Uout);
  const R* __restrict__ G = static_cast<const R*>(A.gs);
  R* __restrict__ FR = static_cast<R*>(A.fr);
  // what the ring is filled from: U_s and its ghost slots, or their primitives
  const R* __restrict__ Rs = PRIMIN ? static_cast<const R*>(A.W) : Us;
  const R* __restrict__ Rg = PRIMIN ? static_cast<const R*>(A.WG) : G;

  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int warp = t >> 5;
  const int cell2 = ty * 16 + tx;
  const int cellp = (ty + 2) * 20 + tx + 2;   // this thread's cell in a 20 x 20 ring plane
  // Faces of the x/y pass: column fc of row fr, the two half-warps of warp w on rows
  // (w & 3) + 8 (w >> 2) and 4 rows further, which the 20-wide plane rows put 16 banks apart
  // (the four-cell stencil loads are free of bank conflicts).
  const int fc = tx;
  const int fr = (warp & 3) + 8 * (warp >> 2) + 4 * ((t >> 4) & 1);
  // x-face fluxes: [NV][16 rows][16] for faces 0..15 of each row, then [NV][16] for face 16
  const int fxr = tx < 15 ? cell2 + 1 : 256 + ty;   // this cell's right x-face
  // Halo cell of this thread: h < 64 x-faces, above y-faces; the half t >> 7 of the CTA owns
  // the halo of the planes of its parity.
  const int hh = t & 127;
  int hx, hy;
  {
    const int side = (hh >> 5) & 1, layer = (hh >> 4) & 1, rr = hh & 15;
    const int c = side ? NB + layer : layer - 2;
    if (hh < 64) { hx = c; hy = rr; } else { hx = rr; hy = c; }
  }
  const int hoff = (hy + 2) * 20 + hx + 2;
  if (t == 0) {
#pragma unroll
    for (int i = 0; i < RAW; ++i) mbar_init(bar + i, 1);
    fence_mbar_init();
  }
  __syncthreads();
  int st = 0;
  // Persistent loop: this CTA starts with block blockIdx.x and then takes the next free block
  // from the launch's counter; every block completes PHASES phases of each raw slot's barrier.
  __shared__ int s_next;
  __shared__ int s_src[6], s_slot[6];   // face sources / register slots of the current block
  __shared__ R s_kc[12];                // per-(solve, level) constants, formed by thread 0
  // Launch constants, and the per-(solve, level) constants of the current block: they are
  // recomputed only when the block's solve or level differs from the previous block's (a
  // CTA-uniform test), by one thread.
  PhysParamsT<R> pp;
  R ra, rb;
  if constexpr (sizeof(R) == 4) {
    pp = A.ppf;
    ra = A.fa;
    rb = A.fb;
  } else {
    pp.set(A.gamma, 0.0);
    ra = R(A.a);
    rb = R(A.b);
  }
  const bool combine = A.combine != 0;
  const bool glm_post = A.glm_post != 0;
  constexpr uint32_t PLANE_BYTES = (uint32_t)(sizeof(R) * NT * 256);
  int key_sv = -1, key_lev = -1;
  R idx = R(0), idy = R(0), idz = R(0), rdt = R(0), glm_fr = R(1);
  R rq4 = R(0);                        // 1 / tau = 1 / (4 dt) of the conduction relaxation
  const R kap0 = R(A.htc_kappa0);
  const R reta = R(A.eta);
  R dxr[3] = {R(0), R(0), R(0)};
  if (t == 0 && blockIdx.x < A.nblk) {
    const int b0 = A.wl ? A.wl[blockIdx.x] : (int)blockIdx.x;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      s_src[f] = A.bd[b0].src[f];
      s_slot[f] = A.bd[b0].slot[f];
    }
  }
  __syncthreads();
  const int* src = s_src;
  const int* slot = s_slot;
  // work item w is pool block b (the work list of a batch skips the blocks of detached solves)
  for (int w = blockIdx.x, jb = 0; w < A.nblk; ++jb) {
  const int b = A.wl ? A.wl[w] : w;
  const int sv = A.solve_of ? A.solve_of[b] : 0;
  unsigned long long* speeds = A.speeds ? A.speeds + 2 * sv : nullptr;
  const BlockDesc& bd = A.bd[b];
  if (sv != key_sv || bd.level != key_lev) {   // CTA-uniform: every thread takes it or none
    // one thread forms the constants in FP64 (divisions, the exp) and the CTA reads them
    // back, so the FP64 units see one thread's work per change instead of the CTA's
    if (t == 0) {
      const double* dtch = A.dtch + 2 * sv;
      const double dt = dtch[0], ch_ = dtch[1];
      s_kc[0] = R(1.0 / bd.dx[0]);
      s_kc[1] = R(1.0 / bd.dx[1]);
      s_kc[2] = R(1.0 / bd.dx[2]);
      s_kc[3] = R(dt);
      s_kc[4] = P::QV >= 0 ? R(0.25 / dt) : R(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) s_kc[5 + d] = R(bd.dx[d]);
      R fr = R(1);
      if (glm_post) {
        const double dxm = fmin(fmin(bd.dx[0], bd.dx[1]), bd.dx[2]);
        fr = R(exp(-0.5 * dt * ch_ * A.glm_alpha / dxm));
      }
      s_kc[8] = fr;
      PhysParamsT<R> q;
      q.set_ch(ch_);
      s_kc[9] = q.ch;
      s_kc[10] = q.ich;
      s_kc[11] = q.ch2;
    }
    __syncthreads();
    idx = s_kc[0];
    idy = s_kc[1];
    idz = s_kc[2];
    rdt = s_kc[3];
    rq4 = s_kc[4];
#pragma unroll
    for (int d = 0; d < 3; ++d) dxr[d] = s_kc[5 + d];
    glm_fr = s_kc[8];
    pp.ch = s_kc[9];
    pp.ich = s_kc[10];
    pp.ch2 = s_kc[11];
    key_sv = sv;
    key_lev = bd.level;
  }

  // plane p (-2 .. 17) -> TMA sequence q = p + 2, raw slot q % RAW, phase (q / RAW) of this block
  auto plane_tma = [&](int p) -> bool {   // does plane p come by TMA (else loaded directly)?
    if (p >= 0 && p < NB) return true;
    return src[p < 0 ? 4 : 5] >= 0;
  };
  auto issue = [&](int p) {               // thread 0 only
    const int q = p + 2;
    uint64_t* br = bar + (q % RAW);
    if (plane_tma(p)) {
      int blk = b, z = p;
      if (p < 0 || p >= NB) {
        blk = src[p < 0 ? 4 : 5];
        z = p & (NB - 1);
      }
      mbar_expect_tx(br, PLANE_BYTES);
      tma_load_4d(sRaw + (size_t)(q % RAW) * NT * 256, &tmap, br, 0, 0, z, blk * NT);
    } else {
      mbar_arrive(br);
    }
  };
  auto ring = [&](int p) -> R* { return sP + (size_t)pslot(p) * NT * 400; };
  // Primitive recovery of this thread's own column at plane p into the primitive ring.
  auto convert_own = [&](int p) {
    const int q = p + 2;
    R u[NT];
    if (plane_tma(p)) {
      if (!mbar_wait(bar + (q % RAW), ((q / RAW) + jb * phases(q % RAW)) & 1, WAIT_LIMIT)) st |= ST_ETIMEOUT;
      const R* r = sRaw + (size_t)(q % RAW) * NT * 256 + cell2;
#pragma unroll
      for (int v = 0; v < NT; ++v) u[v] = r[v * 256];
    } else {
      load_cell<P, R>(Rs, Rg, src, b, tx, ty, p, u);
    }
    R pr[NV], aux[NAW];
    if constexpr (NA > 0) {
#pragma unroll
      for (int i = 0; i < NA; ++i) aux[i] = u[NV + i];
    } else {
      aux[0] = R(0);
    }
    if constexpr (PRIMIN) {
#pragma unroll
      for (int v = 0; v < NV; ++v) pr[v] = u[v];
    } else {
      P::cons2prim(u, pr, aux, pp, st);
    }
    R* w = ring(p) + cellp;
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v * 400] = pr[v];
    if constexpr (NA > 0) {
#pragma unroll
      for (int i = 0; i < NA; ++i) w[(NV + i) * 400] = aux[i];
    }
  };
  // Halo source of this thread's halo cell: the address at plane 0 and the step per plane
  // (a plane of a block pool, or a row of a ghost slot), formed once per block.
  int hvs, hnd;
  const R* ha0 = cell_addr<P, R>(Rs, Rg, src, b, hx, hy, 0, &hvs, &hnd);
  ptrdiff_t hinc;
  {
    int vs1, nd1;
    hinc = cell_addr<P, R>(Rs, Rg, src, b, hx, hy, 1, &vs1, &nd1) - ha0;
  }
  auto halo_mine = [&](int p) { return (t >> 7) == (p & 1); };
  auto prefetch_halo = [&](int p) {       // raw values of the halo of plane p into its frame
    if (halo_mine(p)) {
      const R* a = ha0 + (ptrdiff_t)p * hinc;
      R* d = ring(p) + hoff;
#pragma unroll
      for (int v = 0; v < NT; ++v) cp_async_elem(d + v * 400, a + (size_t)v * hvs);
      cp_async_commit();
    }
  };
  auto convert_halo = [&](int p) {        // the same thread's fetch, converted in place
    if (PRIMIN && halo_mine(p)) {          // primitives already: a reflecting face's image only
      cp_async_wait_all();
      R* d = ring(p) + hoff;
      if constexpr (P::IV >= 0) {
        if (hnd >= 0) d[(P::IV + hnd) * 400] = -d[(P::IV + hnd) * 400];
      }
      if constexpr (P::BOFF >= 0) {
        if (hnd >= 0) d[(P::BOFF + hnd) * 400] = -d[(P::BOFF + hnd) * 400];
      }
    } else if (halo_mine(p)) {
      cp_async_wait_all();
      R* d = ring(p) + hoff;
      R u[NT], pr[NV], aux[NAW];
#pragma unroll
      for (int v = 0; v < NT; ++v) u[v] = d[v * 400];
      if (hnd >= 0) {
        if (P::IV >= 0) u[P::IV + hnd] = -u[P::IV + hnd];
        if (P::BOFF >= 0) u[P::BOFF + hnd] = -u[P::BOFF + hnd];
      }
      if constexpr (NA > 0) {
#pragma unroll
        for (int i = 0; i < NA; ++i) aux[i] = u[NV + i];
      } else {
        aux[0] = R(0);
      }
      P::cons2prim(u, pr, aux, pp, st);
#pragma unroll
      for (int v = 0; v < NV; ++v) d[v * 400] = pr[v];
    }
  };
  // z-face flux at k + 1/2 of this column. hz holds half the limited slope of plane k
  // (from the previous z-face, where plane k was the upper cell) and leaves with that of
  // plane k + 1, so each plane's z-slope is formed once.
  auto zface = [&](int k, R* f, R* hz) {
    R bq[NV], c[NV], d[NV], pl[NV], pr[NV];
    const R* r1 = ring(k) + cellp;
    const R* r2 = ring(k + 1) + cellp;
    const R* r3 = ring(k + 2) + cellp;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      bq[v] = r1[v * 400]; c[v] = r2[v * 400]; d[v] = r3[v * 400];
      const R h = v < P::NREC ? half_slope<R, LIM>(c[v] - bq[v], d[v] - c[v]) : R(0);
      pl[v] = bq[v] + hz[v];
      pr[v] = c[v] - h;
      hz[v] = h;
    }
    if constexpr (PAIRED) riemann_z_lr<P, FLUX>(pl, pr, f, pp);
    else riemann<P, R, 2, FLUX>(pl, pr, f, pp);
  };
  auto xface = [&](const R* C, int fi, int row, R* f) {  // x-face fi - 1/2 of row `row`
    R a[NV], bq[NV], c[NV], d[NV], pl[NV], pr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R* r = C + v * 400 + (row + 2) * 20 + fi;
      a[v] = r[0]; bq[v] = r[1]; c[v] = r[2]; d[v] = r[3];
    }
    plm<NV, R, LIM, P::NREC>(a, bq, c, d, pl, pr);
    riemann<P, R, 0, FLUX>(pl, pr, f, pp);
  };
  auto yface = [&](const R* C, int fj, int col, R* f) {  // y-face fj - 1/2 of column `col`
    R a[NV], bq[NV], c[NV], d[NV], pl[NV], pr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R* r = C + v * 400 + fj * 20 + col + 2;
      a[v] = r[0]; bq[v] = r[20]; c[v] = r[40]; d[v] = r[60];
    }
    plm<NV, R, LIM, P::NREC>(a, bq, c, d, pl, pr);
    riemann<P, R, 1, FLUX>(pl, pr, f, pp);
  };

  // ---- prologue: raw planes by TMA, halo fetches of planes 0 and 1, primitives of planes
  // -2 .. 1 of this column, the z-face at -1/2, the halo of plane 0
  if (t == 0) {
    fence_proxy_async();   // the previous block's reads of the ring precede these copies
    for (int p = -2; p <= RAW - 3; ++p) issue(p);
  }
  prefetch_halo(0);
  prefetch_halo(1);
  convert_own(-2);
  convert_own(-1);
  __syncthreads();   // raw slots of planes -2 and -1 are free
  if (t == 0) {
    fence_proxy_async();
    for (int p = RAW - 2; p <= (RAW == 3 ? 2 : 3); ++p) issue(p);
  }
  convert_own(0);
  R fzd[NV], fzu[NV], hz[NV];
  {  // z-slope of plane -1 from planes -2, -1 and 0 ... before plane 1 takes plane -2's slot
    const R* r0 = ring(-2) + cellp;
    const R* r1 = ring(-1) + cellp;
    const R* r2 = ring(0) + cellp;
#pragma unroll
    for (int v = 0; v < NV; ++v)
      hz[v] = v < P::NREC ? half_slope<R, LIM>(r1[v * 400] - r0[v * 400], r2[v * 400] - r1[v * 400]) : R(0);
  }
  convert_own(1);
  zface(-1, fzd, hz);
  if (FR && slot[4] >= 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) FR[((size_t)slot[4] * NV + v) * 256 + cell2] = fzd[v];
  }
  convert_halo(0);
  __syncthreads();   // plane 0 of the ring (interior and halo) is complete
  if (RAW == 3 && t == 0) {   // raw slots of planes 0 and 1, converted above
    fence_proxy_async();
    issue(3);
    issue(4);
  }

  R ssum = R(0), smax = R(0);

  R Tkm1 = R(0);   // conduction: T = p / rho of this column at plane k - 1
  R Bkm1[3] = {R(0), R(0), R(0)};   // resistivity: B of this column at plane k - 1
  for (int k = 0; k < NB; ++k) {
    R* sFx = sFx0 + (SFB == 2 ? (k & 1) : 0) * NV * 272;
    R* sFy = sFy0 + (SFB == 2 ? (k & 1) : 0) * NV * 272;
    if (RAW == 4 && t == 0 && k >= 1 && k + 3 <= NB + 1) {
      fence_proxy_async();
      issue(k + 3);   // raw slot of plane k-1, read by its update before the previous barrier
    }
    // ---- A, B
    if constexpr (P::QV >= 0) {   // plane k - 1 leaves the primitive ring now
      const R* r = ring(k - 1) + cellp;
      Tkm1 = rdiv(r[P::IE * 400], r[0]);
    }
    if constexpr (RESP) {
      const R* r = ring(k - 1) + cellp;
#pragma unroll
      for (int i = 0; i < 3; ++i) Bkm1[i] = r[(P::BOFF + i) * 400];
    }
    if (k + 2 <= NB + 1) convert_own(k + 2);
    if (k + 1 < NB) convert_halo(k + 1);
    if (k + 2 < NB) prefetch_halo(k + 2);
    // ---- C
    const R* Ck = ring(k);
    // conduction target kappa0 T^(5/2) b.grad T of cell (tx, ty, k) (Eq. 10): central
    // differences of T = p / rho over the face neighbours (x, y from the ring plane k with
    // its halo, z from ring plane k + 1 and the carried plane k - 1), b of the cell
    R htc_g = R(0);
    if constexpr (P::QV >= 0) {
      const R* C = Ck + cellp;
      auto T_at = [&](int o) { return rdiv(C[P::IE * 400 + o], C[o]); };
      const R* rp = ring(k + 1) + cellp;
      const R Tc = T_at(0);
      const R gx = (T_at(1) - T_at(-1)) * (R(0.5) * idx);
      const R gy = (T_at(20) - T_at(-20)) * (R(0.5) * idy);
      const R gz = (rdiv(rp[P::IE * 400], rp[0]) - Tkm1) * (R(0.5) * idz);
      const R bgrad = (C[P::BOFF * 400] * gx + C[(P::BOFF + 1) * 400] * gy) + C[(P::BOFF + 2) * 400] * gz;
      htc_g = kap0 * (Tc * Tc * rsqrt_(Tc)) * bgrad;
    }
    // resistive sources of cell (tx, ty, k) (Section 2.3.3): eta lap B for the induction
    // equation and eta (J.J + B.lap B) for the energy equation, J = curl B, from the face
    // neighbours (x, y from the ring plane k with its halo, z from ring plane k + 1 and the
    // carried plane k - 1): central differences and the 7-point Laplacian
    R rsrc[4] = {R(0), R(0), R(0), R(0)};
    if constexpr (RESP) {
      const R* C = Ck + cellp;
      const R* rp = ring(k + 1) + cellp;
      const R ix2 = idx * idx, iy2 = idy * idy, iz2 = idz * idz;
      const R hx = R(0.5) * idx, hy = R(0.5) * idy, hzz = R(0.5) * idz;
      R bc[3], lap[3], gx[3], gy[3], gz[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R* q = C + (P::BOFF + i) * 400;
        const R b0 = q[0], xp = q[1], xm = q[-1], yp = q[20], ym = q[-20];
        const R zp = rp[(P::BOFF + i) * 400], zm = Bkm1[i];
        bc[i] = b0;
        lap[i] = (((xp - b0) - (b0 - xm)) * ix2 + ((yp - b0) - (b0 - ym)) * iy2) + ((zp - b0) - (b0 - zm)) * iz2;
        gx[i] = (xp - xm) * hx;
        gy[i] = (yp - ym) * hy;
        gz[i] = (zp - zm) * hzz;
      }
      const R j0 = gy[2] - gz[1], j1 = gz[0] - gx[2], j2 = gx[1] - gy[0];
      const R jj = (j0 * j0 + j1 * j1) + j2 * j2;
      const R blap = (bc[0] * lap[0] + bc[1] * lap[1]) + bc[2] * lap[2];
#pragma unroll
      for (int i = 0; i < 3; ++i) rsrc[i] = reta * lap[i];
      rsrc[3] = reta * (jj + blap);
    }
    // U^n of cell (tx, ty, k) for the stage combine, loaded now so that the face work of
    // this phase covers its latency
    R unk[NV];
    if (combine) {
      const R* pn = Un + (size_t)b * NT * NCELL + (size_t)k * 256 + cell2;
#pragma unroll
      for (int v = 0; v < NV; ++v) unk[v] = __ldg(pn + (size_t)v * NCELL);
    }
    {
      R f[NV];
      if constexpr (PAIRED) {
        // the x-face fc - 1/2 of row fr and the y-face fr - 1/2 of column fc as one pair, the
        // y-face's states with x and y components exchanged
        f2 a[NV], bq[NV], c[NV], d[NV], pl[NV], pr[NV], fp[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const R* rx = Ck + v * 400 + (fr + 2) * 20 + fc;
          const R* ry = Ck + swapv<P>(v) * 400 + fr * 20 + fc + 2;
          a[v] = f2_of(rx[0], ry[0]);
          bq[v] = f2_of(rx[1], ry[20]);
          c[v] = f2_of(rx[2], ry[40]);
          d[v] = f2_of(rx[3], ry[60]);
        }
        plm2<NV, LIM, P::NREC>(a, bq, c, d, pl, pr);
        riemann2<P, FLUX>(pl, pr, fp, PairK(pp));
        // the flux buffers hold F / dx (the divergence then needs differences only); the
        // flux registers of the coarse-fine correction take the fluxes themselves
        const f2 kxy = f2_of(idx, idy);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          R sx, sy;
          f2_split(fp[v] * kxy, sx, sy);
          sFx[v * 272 + fr * 16 + fc] = sx;
          sFy[swapv<P>(v) * 272 + fr * 16 + fc] = sy;
        }
        if (FR && fc == 0 && slot[0] >= 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            R fx_, fy_;
            f2_split(fp[v], fx_, fy_);
            FR[((size_t)slot[0] * NV + v) * 256 + k * 16 + fr] = fx_;
          }
        }
        if (FR && fr == 0 && slot[2] >= 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            R fx_, fy_;
            f2_split(fp[v], fx_, fy_);
            FR[((size_t)slot[2] * NV + swapv<P>(v)) * 256 + k * 16 + fc] = fy_;
          }
        }
      } else {
        xface(Ck, fc, fr, f);
#pragma unroll
        for (int v = 0; v < NV; ++v) sFx[v * 272 + fr * 16 + fc] = f[v] * idx;
        if (FR && fc == 0 && slot[0] >= 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) FR[((size_t)slot[0] * NV + v) * 256 + k * 16 + fr] = f[v];
        }
        yface(Ck, fr, fc, f);
#pragma unroll
        for (int v = 0; v < NV; ++v) sFy[v * 272 + fr * 16 + fc] = f[v] * idy;
        if (FR && fr == 0 && slot[2] >= 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) FR[((size_t)slot[2] * NV + v) * 256 + k * 16 + fc] = f[v];
        }
      }
      // the 32 block-boundary faces, one warp per plane in turn, taken from the half of the
      // CTA that converts no halo in this plane (B converted plane k+1's halo in the half
      // (k+1) & 1), so that no warp carries both extra pieces of work between two barriers
      if (warp == 4 * (k & 1) + ((k >> 1) & 3)) {
        // lanes 0-15: x-face 16 - 1/2 of row r; lanes 16-31: y-face 16 - 1/2 of column r,
        // evaluated with the x-face solver on x/y-swapped states (no divergence)
        const int lane = t & 31, r = lane & 15;
        const bool yd = lane >= 16;
        const int base = yd ? 16 * 20 + r + 2 : (r + 2) * 20 + 16;
        const int stp = yd ? 20 : 1;
        R a[NV], bq[NV], c[NV], d[NV], pl[NV], pr[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const R* q = Ck + v * 400 + base;
          a[v] = q[0]; bq[v] = q[stp]; c[v] = q[2 * stp]; d[v] = q[3 * stp];
        }
        swap_xy<P, R>(a, yd);
        swap_xy<P, R>(bq, yd);
        swap_xy<P, R>(c, yd);
        swap_xy<P, R>(d, yd);
        plm<NV, R, LIM, P::NREC>(a, bq, c, d, pl, pr);
        riemann<P, R, 0, FLUX>(pl, pr, f, pp);
        swap_xy<P, R>(f, yd);
        const int fs = yd ? 1 : 0;
        R* dstp = yd ? sFy + 16 * 16 + r : sFx + 256 + r;
        const R ids = yd ? idy : idx;
#pragma unroll
        for (int v = 0; v < NV; ++v) dstp[v * 272] = f[v] * ids;
        const int sl = slot[1 + 2 * fs];
        if (FR && sl >= 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) FR[((size_t)sl * NV + v) * 256 + k * 16 + r] = f[v];
        }
      }
      zface(k, fzu, hz);
      if (FR && k == NB - 1 && slot[5] >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) FR[((size_t)slot[5] * NV + v) * 256 + cell2] = fzu[v];
      }
    }
    __syncthreads();
    if (RAW == 5 && t == 0 && k + 4 <= NB + 1) {
      fence_proxy_async();
      issue(k + 4);   // raw slot of plane k-1, whose update finished before this barrier
    }
    if (RAW == 3 && t == 0 && k + 5 <= NB + 1) {
      fence_proxy_async();
      issue(k + 5);   // raw slot of plane k+2, converted by every thread before this barrier
    }
    // ---- D: flux divergence and stage combine of cell (tx, ty, k)
    {
      const size_t cell = (size_t)k * 256 + cell2;
      const size_t base = (size_t)b * NT * NCELL + cell;
      // U_s of the cell: the raw TMA slot, or global memory (layout with three slots)
      const R* raw = US_GLOBAL ? Us + base : sRaw + (size_t)((k + 2) % RAW) * NT * 256 + cell2;
      constexpr int RSTR = US_GLOBAL ? NCELL : 256;
      R out[NV];
      if constexpr (P::SOURCE) {
        // all flux divergences first: the source needs those of other variables
        R L[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const R lx = sFx[v * 272 + fxr] - sFx[v * 272 + cell2];
          const R ly = sFy[v * 272 + (ty + 1) * 16 + tx] - sFy[v * 272 + ty * 16 + tx];
          const R lz = (fzu[v] - fzd[v]) * idz;
          L[v] = -((lx + ly) + lz);
          fzd[v] = fzu[v];
        }
        R pc[NV];
        const R* pk = Ck + cellp;
#pragma unroll
        for (int v = 0; v < NV; ++v) pc[v] = pk[v * 400];
        P::source(L, pc);
        if constexpr (P::QV >= 0) L[P::QV] = (htc_g - pc[P::QV]) * rq4;   // -(q - target) / tau
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          R val = raw[(size_t)v * RSTR];
          if (v < P::FROZEN) {
            val = val + rdt * L[v];
            if (combine) val = ra * unk[v] + rb * val;
          }
          out[v] = val;
        }
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const R lx = sFx[v * 272 + fxr] - sFx[v * 272 + cell2];
          const R ly = sFy[v * 272 + (ty + 1) * 16 + tx] - sFy[v * 272 + ty * 16 + tx];
          const R lz = (fzu[v] - fzd[v]) * idz;
          R L = -((lx + ly) + lz);
          if constexpr (RESP) {
            if (v >= P::BOFF && v < P::BOFF + 3) L = L + rsrc[v - P::BOFF];
            if (v == P::IE) L = L + rsrc[3];
          }
          R val = raw[(size_t)v * RSTR] + rdt * L;
          if (combine) val = ra * unk[v] + rb * val;
          out[v] = val;
          fzd[v] = fzu[v];
        }
      }
      if (P::GLM && glm_post) out[NV - 1] = out[NV - 1] * glm_fr;
#pragma unroll
      for (int v = 0; v < NV; ++v) Uo[base + (size_t)v * NCELL] = out[v];
      R auxk[NAW];
      if constexpr (NA > 0) {
        const R* pa = Ck + cellp;
#pragma unroll
        for (int i = 0; i < NA; ++i) {
          auxk[i] = pa[(NV + i) * 400];
          Uo[base + (size_t)(NV + i) * NCELL] = auxk[i];
        }
      } else {
        auxk[0] = R(0);
      }
      if (speeds) {
        R ad[NAW];
#pragma unroll
        for (int i = 0; i < NAW; ++i) ad[i] = auxk[i];
        cell_speeds<PT, R>(out, ad, pp, dxr, ssum, smax, st);
      }
    }
    if (SFB == 1) __syncthreads();   // the flux buffer and plane k's raw slot are reused next
  }
  if (speeds) block_max2<256>(ssum, smax, speeds);
  if (t == 0) {
    // every read of this block's face table happened before the last plane's barrier
    const int nx = A.work ? (int)gridDim.x + atomicAdd(A.work, 1) : w + (int)gridDim.x;
    s_next = nx;
    if (nx < A.nblk) {
      const int bn = A.wl ? A.wl[nx] : nx;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        s_src[f] = A.bd[bn].src[f];
        s_slot[f] = A.bd[bn].slot[f];
      }
    }
  }
  __syncthreads();       // ring, raw slots, flux buffers and reduction scratch are reused next
  w = s_next;
  }
  if (st) atomicOr(A.status, st);
}

template <template <typename> class PT, typename R, int RAW, int SFB>
constexpr size_t stage_smem_bytes() {
  return StageSmem<PT, R, RAW, SFB>::total;
}

}  // namespace agile
