// Non-update kernels: coarse-fine ghost slots (restriction, limited-linear prolongation),
// coarse-fine flux correction, global signal-speed reduction for the CFL step, GLM damping,
// Loehner estimator, regrid prolongation/restriction, state packing and conserved sums.
#include <math.h>

#include <type_traits>

#include "kernels.cuh"
#include "launch.h"

namespace agile {

int phys_nvar(int phys) {
  return phys == PH_MHD ? 9 : (phys == PH_FFHD ? 6 : (phys == PH_FFHD_HTC ? 7 : 5));
}
int phys_naux(int phys) { return phys == PH_SRHD || phys == PH_SRHD_SYNGE ? 2 : 0; }

// ------------------------------------------------------------------------------ helpers
template <typename R>
__device__ __forceinline__ R minmod_(R a, R b) {
  return (a > R(0) && b > R(0)) ? (a < b ? a : b) : ((a < R(0) && b < R(0)) ? (a > b ? a : b) : R(0));
}

// Mean of the 8 fine cells with lower corner (fx, fy, fz) of block fb; x fastest, then
// y, then z, added in that order and scaled by 1/8 (volume-average restriction).
template <typename R, int NT>
__device__ __forceinline__ void restrict8(const R* __restrict__ U, int fb, int fx, int fy, int fz,
                                          R* out) {
  const R* p = U + (size_t)fb * NT * NCELL + fz * 256 + fy * 16 + fx;
#pragma unroll
  for (int v = 0; v < NT; ++v) {
    const R* q = p + (size_t)v * NCELL;
    R s = q[0] + q[1];
    s = s + q[16];
    s = s + q[17];
    s = s + q[256];
    s = s + q[257];
    s = s + q[272];
    s = s + q[273];
    out[v] = s * R(0.125);
  }
}

// Value of cell (x, y, z) in the halo view of a COARSE block C as the prolongation sees it:
// the interior, and face ghosts from a same-level copy, a physical boundary or restriction
// of the finer neighbour. A face whose neighbour is still coarser is not available (false).
template <class P, typename R>
__device__ __forceinline__ bool coarse_view(const R* __restrict__ U, const BlockDesc* __restrict__ bd,
                                            int C, int x, int y, int z, R* u) {
  constexpr int NT = P::NV + P::NA;
  int f = -1;
  if (x < 0) f = 0;
  else if (x > NB - 1) f = 1;
  else if (y < 0) f = 2;
  else if (y > NB - 1) f = 3;
  else if (z < 0) f = 4;
  else if (z > NB - 1) f = 5;
  if (f >= 0) {
    const int kind = bd[C].kind[f];
    if (kind == FK_COARSER) return false;
    if (kind == FK_FINER) {
      const int d = f >> 1, s = f & 1;
      int q[3] = {x, y, z};
      const int t1 = d == 0 ? q[1] : q[0];
      const int t2 = d == 2 ? q[1] : q[2];
      const int fb = bd[C].nbr[f][(t1 >> 3) + 2 * (t2 >> 3)];
      int fq[3];
      fq[d] = s ? 0 : NB - 2;
      const int t1d = d == 0 ? 1 : 0, t2d = d == 2 ? 1 : 2;
      fq[t1d] = 2 * (t1 & 7);
      fq[t2d] = 2 * (t2 & 7);
      restrict8<R, NT>(U, fb, fq[0], fq[1], fq[2], u);
      return true;
    }
  }
  int src[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) src[i] = bd[C].src[i];
  load_cell<P, R>(U, (const R*)nullptr, src, C, x, y, z, u);
  return true;
}

// ------------------------------------------------------------------------------ ghost slots
template <template <typename> class PT, typename R>
__global__ void __launch_bounds__(256) ghost_kernel(const R* __restrict__ U, R* __restrict__ G,
                                                     const BlockDesc* __restrict__ bd,
                                                     const GhostTask* __restrict__ tasks) {
  using P = PT<R>;
  constexpr int NT = P::NV + P::NA;
  const GhostTask tk = tasks[blockIdx.x];
  const int d = tk.face >> 1, s = tk.face & 1;
  const int t1d = d == 0 ? 1 : 0, t2d = d == 2 ? 1 : 2;
  // prolongation: the slot's 2 x 16 x 16 fine ghost cells lie in one layer of 8 x 8 coarse
  // cells of block C; the value and the three limited slopes of each coarse cell are formed
  // once (256 threads: 64 cells x {value, slope along x, y, z}) and shared by its fine cells
  __shared__ R s_uc[NT][64], s_sig[3][NT][64];
  if (tk.kind != FK_FINER) {                 // CTA-uniform
    const int cl = threadIdx.x & 63, job = threadIdx.x >> 6;
    const int n = 8 * tk.par[d] + (s ? 0 : 7);              // the coarse layer along d
    const int a1 = 8 * tk.par[t1d] + (cl & 7), a2 = 8 * tk.par[t2d] + (cl >> 3);
    const int cx = d == 0 ? n : a1, cy = d == 1 ? n : (d == 0 ? a1 : a2), cz = d == 2 ? n : a2;
    const int C = tk.nbr[0];
    R uc[NT], up[NT], um[NT];
    coarse_view<P, R>(U, bd, C, cx, cy, cz, uc);
    if (job == 0) {
#pragma unroll
      for (int v = 0; v < NT; ++v) s_uc[v][cl] = uc[v];
    } else {
      const int ex = job == 1, ey = job == 2, ez = job == 3;   // the slope's direction
      const bool okp = coarse_view<P, R>(U, bd, C, cx + ex, cy + ey, cz + ez, up);
      const bool okm = coarse_view<P, R>(U, bd, C, cx - ex, cy - ey, cz - ez, um);
      R sig[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) sig[v] = (okp && okm) ? minmod_(up[v] - uc[v], uc[v] - um[v]) : R(0);
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        if (job == 1) s_sig[0][v][cl] = sig[v];
        else if (job == 2) s_sig[1][v][cl] = sig[v];
        else s_sig[2][v][cl] = sig[v];
      }
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < 512; c += 256) {
    const int layer = c >> 8, t2 = (c >> 4) & 15, t1 = c & 15;
    R out[NT];
    if (tk.kind == FK_FINER) {
      const int fb = tk.nbr[(t1 >> 3) + 2 * (t2 >> 3)];
      int fq[3];
      fq[d] = s ? 2 * layer : NB - 4 + 2 * layer;
      fq[t1d] = 2 * (t1 & 7);
      fq[t2d] = 2 * (t2 & 7);
      restrict8<R, NT>(U, fb, fq[0], fq[1], fq[2], out);
    } else {
      // fine ghost cell in neighbour-position-local fine coordinates f: u_C + sum_e of the
      // sign of its offset along e times sigma_e / 4
      int f3[3];
      f3[d] = s ? layer : NB - 2 + layer;
      f3[t1d] = t1;
      f3[t2d] = t2;
      R sg[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) sg[e] = (f3[e] & 1) ? R(1) : R(-1);
      const int cl = (t1 >> 1) + 8 * (t2 >> 1);
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        R acc = sg[0] * s_sig[0][v][cl];
        acc = acc + sg[1] * s_sig[1][v][cl];
        acc = acc + sg[2] * s_sig[2][v][cl];
        out[v] = s_uc[v][cl] + R(0.25) * acc;
      }
    }
    R* g = G + (size_t)tk.slot * NT * 512 + layer * 256 + t2 * 16 + t1;
#pragma unroll
    for (int v = 0; v < NT; ++v) g[(size_t)v * 512] = out[v];
  }
}

// ------------------------------------------------------------------------------ flux fix-up
// One CTA per coarse block: its coarse-fine faces are corrected one after the other (a
// cell on an edge between two such faces receives both corrections without a race).
// U += b dt (+/-)(F_coarse - mean of the 2x2 fine face fluxes) / dx on the adjacent cells.
template <typename R, int NV, int NT>
__global__ void __launch_bounds__(256) fixup_kernel(R* __restrict__ U, const R* __restrict__ FR,
                                                     const BlockDesc* __restrict__ bd,
                                                     const FixupTask* __restrict__ tasks, double b,
                                                     const double* __restrict__ dtch,
                                                     const int* __restrict__ solve_of) {
  const FixupTask& tk = tasks[blockIdx.x];
  const double dt = dtch[2 * (solve_of ? solve_of[tk.blk] : 0)];   // the block's solve
  const int t1 = threadIdx.x & 15, t2 = threadIdx.x >> 4;
  for (int j = 0; j < tk.nface; ++j) {
    const int face = tk.face[j];
    const int d = face >> 1, s = face & 1;
    const int t1d = d == 0 ? 1 : 0, t2d = d == 2 ? 1 : 2;
    int q[3];
    q[d] = s ? NB - 1 : 0;
    q[t1d] = t1;
    q[t2d] = t2;
    const size_t cell = (size_t)q[2] * 256 + q[1] * 16 + q[0];
    const int sf = tk.slot_f[j][(t1 >> 3) + 2 * (t2 >> 3)];
    const int a0 = 2 * (t1 & 7), b0 = 2 * (t2 & 7);
    const R w = R(b * dt / bd[tk.blk].dx[d]) * (s ? R(1) : R(-1));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R fc = FR[((size_t)tk.slot_c[j] * NV + v) * 256 + t2 * 16 + t1];
      const R* ff = FR + ((size_t)sf * NV + v) * 256;
      R avg = ff[b0 * 16 + a0] + ff[b0 * 16 + a0 + 1];
      avg = avg + ff[(b0 + 1) * 16 + a0];
      avg = avg + ff[(b0 + 1) * 16 + a0 + 1];
      avg = avg * R(0.25);
      R* u = U + ((size_t)tk.blk * NT + v) * NCELL + cell;
      *u = *u + w * (fc - avg);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ CFL speeds
template <template <typename> class PT, typename R>
__global__ void __launch_bounds__(256) speeds_kernel(const R* __restrict__ U,
                                                      const BlockDesc* __restrict__ bd,
                                                      const PhysParamsT<R> pp,   // formed on the host
                                                      unsigned long long* speeds, int* status,
                                                      const int* __restrict__ solve_of,
                                                      const int* __restrict__ wl) {
  using P = PT<R>;
  constexpr int NV = P::NV, NA = P::NA, NT = NV + NA;
  const int b = wl ? wl[blockIdx.x] : (int)blockIdx.x;
  const R dxr[3] = {R(bd[b].dx[0]), R(bd[b].dx[1]), R(bd[b].dx[2])};
  R ssum = R(0), smax = R(0);
  int st = 0;
  const R* base = U + (size_t)b * NT * NCELL;
  for (int c = threadIdx.x; c < NCELL; c += 256) {
    R u[NV], aux[2] = {R(0), R(0)};
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = base[(size_t)v * NCELL + c];
    if constexpr (NA > 0) aux[0] = base[(size_t)NV * NCELL + c];
    cell_speeds<PT, R>(u, aux, pp, dxr, ssum, smax, st);
  }
  block_max2<256>(ssum, smax, speeds + 2 * (solve_of ? solve_of[b] : 0));
  if (st) atomicOr(status, st);
}

__global__ void set_dt_kernel(const unsigned long long* speeds, double* dtch, double dt_host,
                              double cfl, int nsolve, double rate_floor) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsolve) return;
  const double smax = __longlong_as_double((long long)speeds[2 * i]);
  const double cmax = __longlong_as_double((long long)speeds[2 * i + 1]);
  dtch[2 * i] = dt_host > 0.0 ? dt_host : cfl / fmax(smax, rate_floor);
  dtch[2 * i + 1] = cmax;
}

// ------------------------------------------------------------------------------ GLM source
// One CTA per block: thread 0 forms the factor in FP64, the CTA scales psi in the stencil
// precision with 16-byte accesses (psi of a block is 4096 contiguous values).
template <typename R>
__global__ void __launch_bounds__(256) glm_decay_kernel(R* __restrict__ U, const BlockDesc* __restrict__ bd,
                                                         const double* __restrict__ dtch, double alpha,
                                                         const int* __restrict__ solve_of,
                                                         const int* __restrict__ wl) {
  __shared__ R s_f;
  const int b = wl ? wl[blockIdx.x] : (int)blockIdx.x;
  if (threadIdx.x == 0) {
    const double* dc = dtch + 2 * (solve_of ? solve_of[b] : 0);
    const double dxm = fmin(fmin(bd[b].dx[0], bd[b].dx[1]), bd[b].dx[2]);
    s_f = R(exp(-0.5 * dc[0] * dc[1] * alpha / dxm));
  }
  __syncthreads();
  const R f = s_f;
  using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
  constexpr int PER = 16 / sizeof(R);
  V* psi = reinterpret_cast<V*>(U + ((size_t)b * 9 + 8) * NCELL);
  for (int c = threadIdx.x; c < NCELL / PER; c += blockDim.x) {
    V v = psi[c];
    if constexpr (sizeof(R) == 4) {
      v.x *= f; v.y *= f; v.z *= f; v.w *= f;
    } else {
      v.x *= f; v.y *= f;
    }
    psi[c] = v;
  }
}

// ------------------------------------------------------------------------------ estimator
// One variable of cell (x, y, z) in the halo view of block b (the rules of load_cell: a
// same-level neighbour's interior, a physical boundary image with the normal vector
// components negated at a reflecting wall, or a ghost slot).
template <class P, typename R>
__device__ __forceinline__ R load_var(const R* __restrict__ U, const R* __restrict__ G, const int* src, int b,
                                      int x, int y, int z, int iv) {
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
  bool neg = false;
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
      neg = (P::IV >= 0 && iv == P::IV + d) || (P::BOFF >= 0 && iv == P::BOFF + d);
    } else {
      const int slot = SRC_SLOT0 - sv;
      const int layer = s ? q[d] - NB : q[d] + 2;
      const int t1 = d == 0 ? q[1] : q[0];
      const int t2 = d == 2 ? q[1] : q[2];
      return G[((size_t)slot * NT + iv) * 512 + layer * 256 + t2 * 16 + t1];
    }
  }
  const R v = U[((size_t)blk * NT + iv) * NCELL + q[2] * 256 + q[1] * 16 + q[0]];
  return neg ? -v : v;
}

// Loehner (1987) second-derivative estimate per cell and variable (axis terms only):
// E_u = sqrt(sum_d (u+ - 2u0 + u-)^2 / sum_d (|u+ - u0| + |u0 - u-| + eps (|u+| + 2|u0| + |u-|))^2),
// E = sum_u w_u E_u; every operation rounded on its own (no FMA) in this order. Per refinement
// variable the CTA stages the block's interior (coalesced) and its six face layers in shared
// memory; each thread keeps the running sums of its 16 cells in registers.
// Whether the nonzero value x became zero or subnormal in its FP32 copy f (a test on the
// bits of x, which keeps FP64 operations out of the FP32 screen).
template <typename R>
__device__ __forceinline__ bool below_fp32_normal(R x, float f) {
  bool nz;
  if constexpr (sizeof(R) == 8) nz = (__double_as_longlong(x) & 0x7fffffffffffffffLL) != 0;
  else nz = (__float_as_int(x) & 0x7fffffff) != 0;
  return nz && !(fabsf(f) >= 1.17549435e-38f);
}

template <template <typename> class PT, typename R>
__global__ void __launch_bounds__(256) estimate_kernel(const R* __restrict__ U, const R* __restrict__ G,
                                                        const BlockDesc* __restrict__ bd,
                                                        const int* __restrict__ vars,
                                                        const double* __restrict__ weights, int nvars,
                                                        double eps, double* __restrict__ emax,
                                                        const int* __restrict__ wl,
                                                        const double* __restrict__ tols,
                                                        const int* __restrict__ solve_of, double margin) {
  using P = PT<R>;
  constexpr int NT = P::NV + P::NA;
  const int b = wl ? wl[blockIdx.x] : (int)blockIdx.x;
  const int t = threadIdx.x;
  __shared__ int src[6];
  __shared__ R sI[NCELL];          // interior of the staged variable
  __shared__ R sF[6][256];         // its face layers: face f, cell (t1 + 16 t2) as in the ghost slots
  __shared__ double red[8];
  __shared__ int s_amb;
  if (t < 6) src[t] = bd[b].src[t];
  // one refinement variable of the block (interior and face layers) into shared memory
  auto stage = [&](int iv) {
    __syncthreads();               // src is set; the previous variable's reads are done
    const R* base = U + ((size_t)b * NT + iv) * NCELL;
#pragma unroll 4
    for (int c = t; c < NCELL; c += 256) sI[c] = base[c];
    for (int e = t; e < 6 * 256; e += 256) {
      const int f = e >> 8, d = f >> 1, s = f & 1, t1 = e & 15, t2 = (e >> 4) & 15;
      int q[3];
      q[d] = s ? NB : -1;
      q[d == 0 ? 1 : 0] = t1;
      q[d == 2 ? 1 : 2] = t2;
      sF[f][t2 * 16 + t1] = load_var<P, R>(U, G, src, b, q[0], q[1], q[2], iv);
    }
    __syncthreads();
  };
  // the three values of the stencil of cell c along d (face layers beyond the block)
  auto nbrs = [&](int c, int d, R& a, R& m) {
    const int x = c & 15, y = (c >> 4) & 15, z = c >> 8;
    const int pos = d == 0 ? x : (d == 1 ? y : z);
    const int st = d == 0 ? 1 : (d == 1 ? 16 : 256);
    const int t1 = d == 0 ? y : x, t2 = d == 2 ? y : z;
    a = pos < NB - 1 ? sI[c + st] : sF[2 * d + 1][t2 * 16 + t1];
    m = pos > 0 ? sI[c - st] : sF[2 * d][t2 * 16 + t1];
  };
  // maximum over the CTA of a non-negative value (every thread calls it)
  auto block_max = [&](double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    double mx = red[0];
    for (int i = 1; i < 8; ++i) mx = fmax(mx, red[i]);
    return mx;
  };

  if (tols) {
    // Screen for the refinement decision: the same estimate in FP32 for every cell. Each cell's
    // FP32 value lies within `margin` of the exact one (the caller's bound from eps and the
    // weights), so the FP32 block maximum lies within `margin` of the exact maximum. Where it
    // is farther than that from both thresholds (refine above tols[0], coarsen below tols[1]
    // of the block's solve), it leads to the same decision and is returned as it is;
    // otherwise (or on values outside the screen's range) the exact FP64 pass below decides.
    float etf[16];
    bool bad = false;
    const float epsf = (float)eps;
    for (int i = 0; i < nvars; ++i) {
      stage(vars[i]);
      const float wf = (float)weights[i];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = t + 256 * j;
        const float o = (float)sI[c];
        bool lost = below_fp32_normal(sI[c], o);
        float num = 0.0f, den = 0.0f, smag = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          R ar, mr;
          nbrs(c, d, ar, mr);
          const float a = (float)ar, m = (float)mr;
          lost |= below_fp32_normal(ar, a) || below_fp32_normal(mr, m);
          const float tt = (a - 2.0f * o) + m;
          const float sm = (fabsf(a) + 2.0f * fabsf(o)) + fabsf(m);
          const float q = (fabsf(a - o) + fabsf(o - m)) + epsf * sm;
          num += tt * tt;
          den += q * q;
          smag = fmaxf(smag, sm);
        }
        const float e = den > 0.0f ? sqrtf(num / den) : 0.0f;
        // outside the screen's range: non-finite, squares that could underflow or overflow,
        // or a nonzero value that FP32 sees as zero or subnormal
        bad |= !(e <= 1.5f) || (smag > 0.0f && smag < 1e-10f) || !(smag < 1e18f) || lost;
        etf[j] = i == 0 ? wf * e : etf[j] + wf * e;
      }
    }
    float bf = 0.0f;
#pragma unroll
    for (int j = 0; j < 16; ++j) bf = fmaxf(bf, etf[j]);
    if (t == 0) s_amb = 0;
    __syncthreads();
    if (bad) s_amb = 1;
    const double M = block_max((double)bf);   // its barriers also publish s_amb
    const int sv = solve_of ? solve_of[b] : 0;
    const double tr = tols[2 * sv], tc = tols[2 * sv + 1];
    const bool amb = s_amb || !(margin >= 0.0) || fabs(M - tr) <= margin || fabs(M - tc) <= margin;
    if (!amb) {                    // CTA-uniform
      if (t == 0) emax[b] = M;
      return;
    }
  }

  double etot[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) etot[j] = 0.0;
  for (int i = 0; i < nvars; ++i) {
    const double w = weights[i];
    stage(vars[i]);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = t + 256 * j;
      const double o = (double)sI[c];
      double num = 0.0, den = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        R ar, mr;
        nbrs(c, d, ar, mr);
        const double a = (double)ar, m = (double)mr;
        const double tt = __dadd_rn(__dsub_rn(a, __dmul_rn(2.0, o)), m);
        const double q = __dadd_rn(__dadd_rn(fabs(__dsub_rn(a, o)), fabs(__dsub_rn(o, m))),
                                   __dmul_rn(eps, __dadd_rn(__dadd_rn(fabs(a), __dmul_rn(2.0, fabs(o))),
                                                            fabs(m))));
        const double t2q = __dmul_rn(tt, tt), q2 = __dmul_rn(q, q);
        num = d == 0 ? t2q : __dadd_rn(num, t2q);
        den = d == 0 ? q2 : __dadd_rn(den, q2);
      }
      const double e = den > 0.0 ? __dsqrt_rn(__ddiv_rn(num, den)) : 0.0;
      const double we = __dmul_rn(w, e);
      etot[j] = i == 0 ? we : __dadd_rn(etot[j], we);
    }
  }
  double best = 0.0;
#pragma unroll
  for (int j = 0; j < 16; ++j) best = fmax(best, etot[j]);
  const double mx = block_max(best);
  if (t == 0) emax[b] = mx;
}

template <template <typename> class PT, typename R>
__global__ void __launch_bounds__(256) regrid_kernel(const R* __restrict__ Uold, const R* __restrict__ Gold,
                                                      const BlockDesc* __restrict__ bdold,
                                                      R* __restrict__ Unew,
                                                      const RegridSrc* __restrict__ srcs) {
  using P = PT<R>;
  constexpr int NT = P::NV + P::NA;
  const int nb = blockIdx.x;
  const RegridSrc rs = srcs[nb];
  R* out = Unew + (size_t)nb * NT * NCELL;
  if (rs.mode == 0) {
    const R* in = Uold + (size_t)rs.src[0] * NT * NCELL;
    for (int i = threadIdx.x; i < NT * NCELL; i += 256) out[i] = in[i];
    return;
  }
  for (int c = threadIdx.x; c < NCELL; c += 256) {
    const int x = c & 15, y = (c >> 4) & 15, z = c >> 8;
    R val[NT];
    if (rs.mode == 2) {
      const int o = (x >> 3) + 2 * (y >> 3) + 4 * (z >> 3);
      restrict8<R, NT>(Uold, rs.src[o], 2 * (x & 7), 2 * (y & 7), 2 * (z & 7), val);
    } else {
      const int P0 = rs.src[0];
      int src[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) src[i] = bdold[P0].src[i];
      const int fo[3] = {16 * (rs.octant & 1), 16 * ((rs.octant >> 1) & 1), 16 * (rs.octant >> 2)};
      const int f3[3] = {fo[0] + x, fo[1] + y, fo[2] + z};
      int cc[3];
      R sg[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        cc[e] = f3[e] >> 1;
        sg[e] = (f3[e] & 1) ? R(1) : R(-1);
      }
      R uc[NT], up[NT], um[NT], acc[NT];
      load_cell<P, R>(Uold, Gold, src, P0, cc[0], cc[1], cc[2], uc);
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        int pp[3] = {cc[0], cc[1], cc[2]}, mm[3] = {cc[0], cc[1], cc[2]};
        pp[e] += 1;
        mm[e] -= 1;
        load_cell<P, R>(Uold, Gold, src, P0, pp[0], pp[1], pp[2], up);
        load_cell<P, R>(Uold, Gold, src, P0, mm[0], mm[1], mm[2], um);
#pragma unroll
        for (int v = 0; v < NT; ++v) {
          const R sig = minmod_(up[v] - uc[v], uc[v] - um[v]);
          acc[v] = e == 0 ? sg[0] * sig : acc[v] + sg[e] * sig;
        }
      }
#pragma unroll
      for (int v = 0; v < NT; ++v) val[v] = uc[v] + R(0.25) * acc[v];
    }
#pragma unroll
    for (int v = 0; v < NT; ++v) out[(size_t)v * NCELL + c] = val[v];
  }
}

// ------------------------------------------------------------------------ recovery pass
// Primitives and auxiliaries of every cell of U_s (the work list's blocks, 16 CTAs of one
// z-plane each) and of its ghost slots (two CTAs of 256 cells each per slot) into W / WG,
// laid out as U_s / the slots are. One recovery per stored cell: the same function the stage
// kernel applies, on the same inputs, so the primitives are the same bit for bit. With
// speeds non-null (the first stage of a step) it also reduces the CFL maxima of the leaf
// cells per solve from these primitives, as the stage kernel's fused reduction would have
// from the same state at the end of the previous step.
template <template <typename> class PT, typename R>
__global__ void __launch_bounds__(256) prim_pass_kernel(const R* __restrict__ U, R* __restrict__ W,
                                                        const R* __restrict__ G, R* __restrict__ WG,
                                                        const int* __restrict__ wl, int nwork,
                                                        PhysParamsT<R> pp, int* status,
                                                        const BlockDesc* __restrict__ bd,
                                                        const int* __restrict__ solve_of,
                                                        unsigned long long* speeds) {
  using P = PT<R>;
  constexpr int NV = P::NV, NA = P::NA, NT = NV + NA;
  const int item = blockIdx.x;
  const R* src;
  R* dst;
  int vs;
  int b = -1;
  if (item < nwork * 16) {
    const int w = item >> 4, z = item & 15;
    b = wl ? wl[w] : w;
    const size_t off = (size_t)b * NT * NCELL + (size_t)z * 256 + threadIdx.x;
    src = U + off;
    dst = W + off;
    vs = NCELL;
  } else {
    const int j = item - nwork * 16;          // slot j / 2, cells (j % 2) * 256 ..
    const size_t off = (size_t)(j >> 1) * NT * 512 + (size_t)(j & 1) * 256 + threadIdx.x;
    src = G + off;
    dst = WG + off;
    vs = 512;
  }
  R u[NT], p[NV], aux[NA > 0 ? NA : 1];
#pragma unroll
  for (int v = 0; v < NT; ++v) u[v] = src[(size_t)v * vs];
  if constexpr (NA > 0) {
#pragma unroll
    for (int i = 0; i < NA; ++i) aux[i] = u[NV + i];
  } else {
    aux[0] = R(0);
  }
  int st = 0;
  P::cons2prim(u, p, aux, pp, st);
#pragma unroll
  for (int v = 0; v < NV; ++v) dst[(size_t)v * vs] = p[v];
#pragma unroll
  for (int i = 0; i < NA; ++i) dst[(size_t)(NV + i) * vs] = aux[i];
  if (st) atomicOr(status, st);
  if (speeds && b >= 0) {             // CTA-uniform: a pool plane, not a ghost slot
    const R dxr[3] = {R(bd[b].dx[0]), R(bd[b].dx[1]), R(bd[b].dx[2])};
    R ssum = R(0), smax = R(0);
    prim_speeds<PT, R>(p, pp, dxr, ssum, smax);
    block_max2<256>(ssum, smax, speeds + 2 * (solve_of ? solve_of[b] : 0));
  }
}

// ------------------------------------------------------------------------------ state I/O
template <template <typename> class PT, typename R>
__global__ void prim2cons_kernel(R* __restrict__ U, const double* __restrict__ prim,
                                 const int* __restrict__ blocks, double gamma) {
  using P = PT<double>;
  constexpr int NV = P::NV, NA = P::NA, NT = NV + NA;
  const int i = blockIdx.x;
  const int b = blocks[i];
  PhysParamsT<double> pp;
  pp.set(gamma, 0.0);
  for (int c = threadIdx.x; c < NCELL; c += blockDim.x) {
    double p[NV], u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) p[v] = prim[((size_t)i * NV + v) * NCELL + c];
    P::prim2cons(p, u, pp);
    R* o = U + (size_t)b * NT * NCELL + c;
#pragma unroll
    for (int v = 0; v < NV; ++v) o[(size_t)v * NCELL] = R(u[v]);
    if constexpr (NA > 0) {
      // xi = Gamma^2 rho h and Gamma from the primitives (Eq. 20)
      const double lor = sqrt(1.0 + p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
      const double h = P::enthalpy(p[0], p[4], pp);
      o[(size_t)NV * NCELL] = R(lor * lor * p[0] * h);
      o[(size_t)(NV + 1) * NCELL] = R(lor);
    }
  }
}

template <typename R>
__global__ void unpack_kernel(R* __restrict__ U, const double* __restrict__ cons, int nv, int na) {
  const int b = blockIdx.x;
  const int nt = nv + na;
  for (int i = threadIdx.x; i < nt * NCELL; i += blockDim.x) {
    const int v = i / NCELL;
    U[(size_t)b * nt * NCELL + i] = v < nv ? R(cons[(size_t)b * nv * NCELL + i]) : R(0);
  }
}

template <typename R>
__global__ void pack_kernel(const R* __restrict__ U, double* __restrict__ cons, double* __restrict__ aux,
                            int nv, int na) {
  const int b = blockIdx.x;
  const int nt = nv + na;
  for (int i = threadIdx.x; i < nt * NCELL; i += blockDim.x) {
    const int v = i / NCELL;
    const double val = (double)U[(size_t)b * nt * NCELL + i];
    if (v < nv) {
      if (cons) cons[(size_t)b * nv * NCELL + i] = val;
    } else if (aux) {
      aux[(size_t)b * na * NCELL + (i - nv * NCELL)] = val;
    }
  }
}

// Per-block volume integrals of the conserved variables, all variables in one pass. FP64
// pools add in FP64. FP32 pools add each thread's 16 values in FP32 with the exact error of
// every addition kept (Knuth's TwoSum: s = a + b, e = (a - (s - (s - a))) + (b - (s - a)),
// so s + e = a + b exactly), an FP32 pair whose sum carries about 48 significant bits, then
// in FP64: the FP64 units of the GPU add 64 times slower than its FP32 units.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

template <typename R>
__global__ void __launch_bounds__(256) sums_kernel(const R* __restrict__ U, const BlockDesc* __restrict__ bd,
                                                    double* __restrict__ part, int nv, int na) {
  const int b = blockIdx.x;
  const int nt = nv + na;
  const double dv = bd[b].dx[0] * bd[b].dx[1] * bd[b].dx[2];
  __shared__ double red[8][16];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int v = 0; v < nv; ++v) {
    const R* p = U + ((size_t)b * nt + v) * NCELL;
    double s;
    if constexpr (sizeof(R) == 4) {
      const float4* q = reinterpret_cast<const float4*>(p);
      float hi = 0.0f, lo = 0.0f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 x = q[threadIdx.x + 256 * i];
        two_sum_acc(hi, lo, x.x);
        two_sum_acc(hi, lo, x.y);
        two_sum_acc(hi, lo, x.z);
        two_sum_acc(hi, lo, x.w);
      }
      s = (double)hi + (double)lo;
    } else {
      s = 0.0;
      for (int c = threadIdx.x; c < NCELL; c += 256) s += (double)p[c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[w][v] = s;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
    part[(size_t)b * nv + threadIdx.x] = t * dv;
  }
}

template <template <typename> class PT, typename R>
__global__ void halo_kernel(const R* __restrict__ U, const R* __restrict__ G,
                            const BlockDesc* __restrict__ bd, int b, double* __restrict__ out) {
  using P = PT<R>;
  constexpr int NT = P::NV + P::NA;
  int src[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) src[i] = bd[b].src[i];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 8000; c += gridDim.x * blockDim.x) {
    const int x = c % 20 - 2, y = (c / 20) % 20 - 2, z = c / 400 - 2;
    const int outside = (x < 0 || x > 15) + (y < 0 || y > 15) + (z < 0 || z > 15);
    if (outside > 1) {
      for (int v = 0; v < NT; ++v) out[(size_t)v * 8000 + c] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    R u[NT];
    load_cell<P, R>(U, G, src, b, x, y, z, u);
    for (int v = 0; v < NT; ++v) out[(size_t)v * 8000 + c] = (double)u[v];
  }
}

// ------------------------------------------------------------------------------ dispatch
#define AGILE_DISPATCH(phys, rb, CALL)                         \
  do {                                                         \
    if ((phys) == PH_HD) {                                     \
      if ((rb) == 8) { using R = double; CALL(HdPhys); }       \
      else { using R = float; CALL(HdPhys); }                  \
    } else if ((phys) == PH_MHD) {                             \
      if ((rb) == 8) { using R = double; CALL(MhdPhys); }      \
      else { using R = float; CALL(MhdPhys); }                 \
    } else if ((phys) == PH_SRHD) {                            \
      if ((rb) == 8) { using R = double; CALL(SrhdPhys); }     \
      else { using R = float; CALL(SrhdPhys); }                \
    } else if ((phys) == PH_FFHD) {                            \
      if ((rb) == 8) { using R = double; CALL(FfhdPhys); }     \
      else { using R = float; CALL(FfhdPhys); }                \
    } else if ((phys) == PH_FFHD_HTC) {                        \
      if ((rb) == 8) { using R = double; CALL(FfhdHtcPhys); }  \
      else { using R = float; CALL(FfhdHtcPhys); }             \
    } else {                                                   \
      if ((rb) == 8) { using R = double; CALL(SrhdSyngePhys); }\
      else { using R = float; CALL(SrhdSyngePhys); }           \
    }                                                          \
  } while (0)

cudaError_t launch_ghosts(const AuxArgs& a, const GhostTask* tasks, int ntasks, cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
#define CALL(PT) ghost_kernel<PT, R><<<ntasks, 256, 0, s>>>((const R*)a.U, (R*)a.Gw, a.bd, tasks)
  AGILE_DISPATCH(a.phys, a.real_bytes, CALL);
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_fixup(const AuxArgs& a, const FixupTask* tasks, int ntasks, double b,
                         const double* dtch, cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  const int nv = phys_nvar(a.phys), nt = nv + phys_naux(a.phys);
  if (nv == 6) return cudaErrorInvalidValue;   // ffhd runs on uniform meshes only
  if (a.real_bytes == 8) {
    if (nv == 9) fixup_kernel<double, 9, 9><<<ntasks, 256, 0, s>>>((double*)a.Uw, (const double*)a.FR, a.bd, tasks, b, dtch, a.solve_of);
    else if (nt == 5) fixup_kernel<double, 5, 5><<<ntasks, 256, 0, s>>>((double*)a.Uw, (const double*)a.FR, a.bd, tasks, b, dtch, a.solve_of);
    else fixup_kernel<double, 5, 7><<<ntasks, 256, 0, s>>>((double*)a.Uw, (const double*)a.FR, a.bd, tasks, b, dtch, a.solve_of);
  } else {
    if (nv == 9) fixup_kernel<float, 9, 9><<<ntasks, 256, 0, s>>>((float*)a.Uw, (const float*)a.FR, a.bd, tasks, b, dtch, a.solve_of);
    else if (nt == 5) fixup_kernel<float, 5, 5><<<ntasks, 256, 0, s>>>((float*)a.Uw, (const float*)a.FR, a.bd, tasks, b, dtch, a.solve_of);
    else fixup_kernel<float, 5, 7><<<ntasks, 256, 0, s>>>((float*)a.Uw, (const float*)a.FR, a.bd, tasks, b, dtch, a.solve_of);
  }
  return cudaGetLastError();
}

cudaError_t launch_speeds(const AuxArgs& a, unsigned long long* speeds, cudaStream_t s) {
  if (a.nblk == 0) return cudaSuccess;
#define CALL(PT)                                                                                  \
  do {                                                                                            \
    PhysParamsT<R> pp;                                                                            \
    pp.set(a.gamma, 0.0);                                                                         \
    speeds_kernel<PT, R><<<a.nblk, 256, 0, s>>>((const R*)a.U, a.bd, pp, speeds, a.status, a.solve_of, a.wl); \
  } while (0)
  AGILE_DISPATCH(a.phys, a.real_bytes, CALL);
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_set_dt(const unsigned long long* speeds, double* dtch, double dt_host,
                          double cfl, cudaStream_t s, int nsolve, double rate_floor) {
  set_dt_kernel<<<(nsolve + 127) / 128, 128, 0, s>>>(speeds, dtch, dt_host, cfl, nsolve, rate_floor);
  return cudaGetLastError();
}

cudaError_t launch_glm_decay(const AuxArgs& a, const double* dtch, cudaStream_t s) {
  if (a.nblk == 0) return cudaSuccess;
  if (a.real_bytes == 8)
    glm_decay_kernel<double><<<a.nblk, 256, 0, s>>>((double*)a.Uw, a.bd, dtch, a.glm_alpha, a.solve_of, a.wl);
  else glm_decay_kernel<float><<<a.nblk, 256, 0, s>>>((float*)a.Uw, a.bd, dtch, a.glm_alpha, a.solve_of, a.wl);
  return cudaGetLastError();
}

cudaError_t launch_estimate(const AuxArgs& a, const int* vars, const double* weights, int nvars,
                            double eps, double* emax, cudaStream_t s, const double* tols, double margin) {
  if (a.nblk == 0) return cudaSuccess;
#define CALL(PT)                                                                                          \
  estimate_kernel<PT, R><<<a.nblk, 256, 0, s>>>((const R*)a.U, (const R*)a.G, a.bd, vars, weights, nvars, eps, \
                                                emax, a.wl, tols, a.solve_of, margin)
  AGILE_DISPATCH(a.phys, a.real_bytes, CALL);
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_regrid(const AuxArgs& a, void* Unew, const RegridSrc* src, int nnew, cudaStream_t s) {
  if (nnew == 0) return cudaSuccess;
#define CALL(PT) regrid_kernel<PT, R><<<nnew, 256, 0, s>>>((const R*)a.U, (const R*)a.G, a.bd, (R*)Unew, src)
  AGILE_DISPATCH(a.phys, a.real_bytes, CALL);
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_prim_pass(const AuxArgs& a, void* W, void* WG, int nslots, unsigned long long* speeds,
                             cudaStream_t s) {
  const long long grid = 16LL * a.nblk + 2LL * nslots;
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (a.phys != PH_SRHD && a.phys != PH_SRHD_SYNGE) return cudaErrorInvalidValue;
#define CALL(PT)                                                                               \
  do {                                                                                         \
    PhysParamsT<R> pp;                                                                         \
    pp.set(a.gamma, 0.0);                                                                      \
    prim_pass_kernel<PT, R><<<(unsigned)grid, 256, 0, s>>>((const R*)a.U, (R*)W, (const R*)a.G, \
                                                           (R*)WG, a.wl, a.nblk, pp, a.status,   \
                                                           a.bd, a.solve_of, speeds);            \
  } while (0)
  if (a.phys == PH_SRHD) {
    if (a.real_bytes == 8) { using R = double; CALL(SrhdPhys); }
    else { using R = float; CALL(SrhdPhys); }
  } else {
    if (a.real_bytes == 8) { using R = double; CALL(SrhdSyngePhys); }
    else { using R = float; CALL(SrhdSyngePhys); }
  }
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_prim2cons(const AuxArgs& a, const double* prim, const int* blocks, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
#define CALL(PT) prim2cons_kernel<PT, R><<<n, 256, 0, s>>>((R*)a.Uw, prim, blocks, a.gamma)
  AGILE_DISPATCH(a.phys, a.real_bytes, CALL);
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_unpack(const AuxArgs& a, const double* cons, cudaStream_t s) {
  if (a.nblk == 0) return cudaSuccess;
  const int nv = phys_nvar(a.phys), na = phys_naux(a.phys);
  if (a.real_bytes == 8) unpack_kernel<double><<<a.nblk, 256, 0, s>>>((double*)a.Uw, cons, nv, na);
  else unpack_kernel<float><<<a.nblk, 256, 0, s>>>((float*)a.Uw, cons, nv, na);
  return cudaGetLastError();
}

cudaError_t launch_pack(const AuxArgs& a, double* cons, double* aux, cudaStream_t s) {
  if (a.nblk == 0) return cudaSuccess;
  const int nv = phys_nvar(a.phys), na = phys_naux(a.phys);
  if (a.real_bytes == 8) pack_kernel<double><<<a.nblk, 256, 0, s>>>((const double*)a.U, cons, aux, nv, na);
  else pack_kernel<float><<<a.nblk, 256, 0, s>>>((const float*)a.U, cons, aux, nv, na);
  return cudaGetLastError();
}

cudaError_t launch_sums(const AuxArgs& a, double* part, cudaStream_t s) {
  if (a.nblk == 0) return cudaSuccess;
  const int nv = phys_nvar(a.phys), na = phys_naux(a.phys);
  if (a.real_bytes == 8) sums_kernel<double><<<a.nblk, 256, 0, s>>>((const double*)a.U, a.bd, part, nv, na);
  else sums_kernel<float><<<a.nblk, 256, 0, s>>>((const float*)a.U, a.bd, part, nv, na);
  return cudaGetLastError();
}

cudaError_t launch_halo(const AuxArgs& a, int block, double* out, cudaStream_t s) {
#define CALL(PT) halo_kernel<PT, R><<<32, 256, 0, s>>>((const R*)a.U, (const R*)a.G, a.bd, block, out)
  AGILE_DISPATCH(a.phys, a.real_bytes, CALL);
#undef CALL
  return cudaGetLastError();
}

}  // namespace agile
