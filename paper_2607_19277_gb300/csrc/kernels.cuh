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
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "physics.cuh"

namespace agile {

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
  unsigned long long* speeds;   // fused reduction of [max sum_d s_d/dx_d, max s_d] or nullptr
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
      u[1 + d] = -u[1 + d];
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

// Signal speeds of one cell in FP64: s_d = max |lambda_+-| along d.
template <template <typename> class PT>
__device__ __forceinline__ void cell_speeds(const double* u, double* aux, const PhysParams& pp,
                                            const double* dx, double& ssum, double& smax, int& st) {
  using P = PT<double>;
  double p[P::NV];
  P::cons2prim(u, p, aux, pp, st);
  double lm, lp, s;
  P::template lambdas<0>(p, lm, lp, pp);
  s = fmax(fabs(lm), fabs(lp));
  smax = fmax(smax, s);
  double acc = s / dx[0];
  P::template lambdas<1>(p, lm, lp, pp);
  s = fmax(fabs(lm), fabs(lp));
  smax = fmax(smax, s);
  acc = acc + s / dx[1];
  P::template lambdas<2>(p, lm, lp, pp);
  s = fmax(fabs(lm), fabs(lp));
  smax = fmax(smax, s);
  acc = acc + s / dx[2];
  ssum = fmax(ssum, acc);
}

template <int NTHREADS>
__device__ __forceinline__ void block_max2(double a, double b, unsigned long long* out) {
  __shared__ double ra[NTHREADS / 32], rb[NTHREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    ra[w] = a;
    rb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ma = ra[0], mb = rb[0];
    for (int i = 1; i < NTHREADS / 32; ++i) {
      ma = fmax(ma, ra[i]);
      mb = fmax(mb, rb[i]);
    }
    atomic_max_pos(out, ma);
    atomic_max_pos(out + 1, mb);
  }
}

template <template <typename> class PT, typename R, int LIM, int FLUX>
__global__ void __launch_bounds__(256) stage_kernel(StageArgs A) {
  using P = PT<R>;
  constexpr int NV = P::NV, NA = P::NA, NT = NV + NA;
  constexpr int NAW = NA > 0 ? NA : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sP = reinterpret_cast<R*>(smem_raw);      // [NV][20][20] primitives of plane k
  R* sFx = sP + NV * 400;                       // [NV][16][17] x-face fluxes
  R* sFy = sFx + NV * 272;                      // [NV][17][16] y-face fluxes

  const R* __restrict__ Us = static_cast<const R*>(A.Us);
  const R* __restrict__ Un = static_cast<const R*>(A.Un);
  R* __restrict__ Uo = static_cast<R*>(A.Uout);
  const R* __restrict__ G = static_cast<const R*>(A.gs);
  R* __restrict__ FR = static_cast<R*>(A.fr);

  const int b = blockIdx.x;
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const BlockDesc& bd = A.bd[b];
  int src[6], slot[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    src[f] = bd.src[f];
    slot[f] = bd.slot[f];
  }
  const double dt = A.dtch[0];
  PhysParams pp;
  pp.gamma = A.gamma;
  pp.ch = A.dtch[1];
  const R idx = R(1.0 / bd.dx[0]), idy = R(1.0 / bd.dx[1]), idz = R(1.0 / bd.dx[2]);
  const R rdt = R(dt);
  const R ra = R(A.a), rb = R(A.b);
  int st = 0;

  R W[4][NV];     // primitives of planes k-1 .. k+2 of this column
  R WA[4][NAW];   // auxiliaries recovered with them
  R fzd[NV], fzu[NV];

  auto load_prim = [&](int x, int y, int z, R* p, R* aux) {
    R u[NT];
    load_cell<P, R>(Us, G, src, b, x, y, z, u);
    R a_[NAW];
    if constexpr (NA > 0) {
#pragma unroll
      for (int i = 0; i < NA; ++i) a_[i] = u[NV + i];
    } else {
      a_[0] = R(0);
    }
    P::cons2prim(u, p, a_, pp, st);
#pragma unroll
    for (int i = 0; i < NAW; ++i) aux[i] = a_[i];
  };

  // Prologue: planes -2, -1, 0, 1 of this column and the z-face at -1/2.
#pragma unroll
  for (int i = 0; i < 4; ++i) load_prim(tx, ty, i - 2, W[i], WA[i]);
  {
    R pl[NV], pr[NV];
    plm<NV, R, LIM>(W[0], W[1], W[2], W[3], pl, pr);
    riemann<P, R, 2, FLUX>(pl, pr, fzd, pp);
  }
  if (FR && slot[4] >= 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) FR[((size_t)slot[4] * NV + v) * 256 + ty * 16 + tx] = fzd[v];
  }
  // shift in plane 2
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    W[0][v] = W[1][v];
    W[1][v] = W[2][v];
    W[2][v] = W[3][v];
  }
#pragma unroll
  for (int i = 0; i < NAW; ++i) {
    WA[0][i] = WA[1][i];
    WA[1][i] = WA[2][i];
    WA[2][i] = WA[3][i];
  }
  load_prim(tx, ty, 2, W[3], WA[3]);

  double ssum = 0.0, smax = 0.0;
  double dxd[3] = {bd.dx[0], bd.dx[1], bd.dx[2]};
  double glm_f = 1.0;
  if (A.glm_post) {
    const double dxm = fmin(fmin(bd.dx[0], bd.dx[1]), bd.dx[2]);
    glm_f = exp(-0.5 * dt * pp.ch * A.glm_alpha / dxm);
  }

  for (int k = 0; k < NB; ++k) {
    // 1. primitives of plane k into shared memory: own column + x/y halo
#pragma unroll
    for (int v = 0; v < NV; ++v) sP[v * 400 + (ty + 2) * 20 + tx + 2] = W[1][v];
    if (t < 128) {
      const int side = (t >> 5) & 1, layer = (t >> 4) & 1, r = t & 15;
      const int c = side ? NB + layer : layer - 2;
      int x, y;
      if (t < 64) { x = c; y = r; } else { x = r; y = c; }
      R p[NV], aux[NAW];
      load_prim(x, y, k, p, aux);
#pragma unroll
      for (int v = 0; v < NV; ++v) sP[v * 400 + (y + 2) * 20 + x + 2] = p[v];
    }
    __syncthreads();
    // 2. x- and y-face fluxes of plane k (17 x 16 each); warp 0 takes the 32 extra faces
    {
      R a[NV], bq[NV], c[NV], d[NV], pl[NV], pr[NV], f[NV];
      // x-face at tx - 1/2 of row ty
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const R* row = sP + v * 400 + (ty + 2) * 20 + tx;
        a[v] = row[0]; bq[v] = row[1]; c[v] = row[2]; d[v] = row[3];
      }
      plm<NV, R, LIM>(a, bq, c, d, pl, pr);
      riemann<P, R, 0, FLUX>(pl, pr, f, pp);
#pragma unroll
      for (int v = 0; v < NV; ++v) sFx[v * 272 + ty * 17 + tx] = f[v];
      if (FR && tx == 0 && slot[0] >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) FR[((size_t)slot[0] * NV + v) * 256 + k * 16 + ty] = f[v];
      }
      // y-face at ty - 1/2 of column tx
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const R* col = sP + v * 400 + ty * 20 + tx + 2;
        a[v] = col[0]; bq[v] = col[20]; c[v] = col[40]; d[v] = col[60];
      }
      plm<NV, R, LIM>(a, bq, c, d, pl, pr);
      riemann<P, R, 1, FLUX>(pl, pr, f, pp);
#pragma unroll
      for (int v = 0; v < NV; ++v) sFy[v * 272 + ty * 16 + tx] = f[v];
      if (FR && ty == 0 && slot[2] >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) FR[((size_t)slot[2] * NV + v) * 256 + k * 16 + tx] = f[v];
      }
      if (t < 32) {
        const int r = t & 15;
        if (t < 16) {   // x-face 16 - 1/2 of row r
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const R* row = sP + v * 400 + (r + 2) * 20 + 16;
            a[v] = row[0]; bq[v] = row[1]; c[v] = row[2]; d[v] = row[3];
          }
          plm<NV, R, LIM>(a, bq, c, d, pl, pr);
          riemann<P, R, 0, FLUX>(pl, pr, f, pp);
#pragma unroll
          for (int v = 0; v < NV; ++v) sFx[v * 272 + r * 17 + 16] = f[v];
          if (FR && slot[1] >= 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) FR[((size_t)slot[1] * NV + v) * 256 + k * 16 + r] = f[v];
          }
        } else {        // y-face 16 - 1/2 of column r
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const R* col = sP + v * 400 + 16 * 20 + r + 2;
            a[v] = col[0]; bq[v] = col[20]; c[v] = col[40]; d[v] = col[60];
          }
          plm<NV, R, LIM>(a, bq, c, d, pl, pr);
          riemann<P, R, 1, FLUX>(pl, pr, f, pp);
#pragma unroll
          for (int v = 0; v < NV; ++v) sFy[v * 272 + 16 * 16 + r] = f[v];
          if (FR && slot[3] >= 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) FR[((size_t)slot[3] * NV + v) * 256 + k * 16 + r] = f[v];
          }
        }
      }
      // z-face at k + 1/2 of this column
      plm<NV, R, LIM>(W[0], W[1], W[2], W[3], pl, pr);
      riemann<P, R, 2, FLUX>(pl, pr, fzu, pp);
      if (FR && k == NB - 1 && slot[5] >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) FR[((size_t)slot[5] * NV + v) * 256 + ty * 16 + tx] = fzu[v];
      }
    }
    __syncthreads();
    // 3. flux divergence and stage combine for cell (tx, ty, k)
    {
      const size_t cell = (size_t)k * 256 + ty * 16 + tx;
      const size_t base = (size_t)b * NT * NCELL + cell;
      R out[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const R lx = (sFx[v * 272 + ty * 17 + tx + 1] - sFx[v * 272 + ty * 17 + tx]) * idx;
        const R ly = (sFy[v * 272 + (ty + 1) * 16 + tx] - sFy[v * 272 + ty * 16 + tx]) * idy;
        const R lz = (fzu[v] - fzd[v]) * idz;
        const R L = -((lx + ly) + lz);
        R val = Us[base + (size_t)v * NCELL] + rdt * L;
        if (A.a != 0.0) val = ra * Un[base + (size_t)v * NCELL] + rb * val;
        out[v] = val;
      }
      if (P::BOFF >= 0 && A.glm_post) out[NV - 1] = R((double)out[NV - 1] * glm_f);
#pragma unroll
      for (int v = 0; v < NV; ++v) Uo[base + (size_t)v * NCELL] = out[v];
      if constexpr (NA > 0) {
#pragma unroll
        for (int i = 0; i < NA; ++i) Uo[base + (size_t)(NV + i) * NCELL] = WA[1][i];
      }
      if (A.speeds) {
        double ud[NV], ad[2];
#pragma unroll
        for (int v = 0; v < NV; ++v) ud[v] = (double)out[v];
        ad[0] = NA > 0 ? (double)WA[1][0] : 0.0;
        ad[1] = 0.0;
        cell_speeds<PT>(ud, ad, pp, dxd, ssum, smax, st);
      }
    }
    // 4. advance the column window
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      fzd[v] = fzu[v];
      W[0][v] = W[1][v];
      W[1][v] = W[2][v];
      W[2][v] = W[3][v];
    }
#pragma unroll
    for (int i = 0; i < NAW; ++i) {
      WA[0][i] = WA[1][i];
      WA[1][i] = WA[2][i];
      WA[2][i] = WA[3][i];
    }
    if (k + 3 <= NB + 1) load_prim(tx, ty, k + 3, W[3], WA[3]);
  }
  if (A.speeds) block_max2<256>(ssum, smax, A.speeds);
  if (st) atomicOr(A.status, st);
}

template <template <typename> class PT, typename R>
constexpr size_t stage_smem_bytes() {
  return sizeof(R) * (size_t)PT<R>::NV * (400 + 272 + 272);
}

}  // namespace agile
