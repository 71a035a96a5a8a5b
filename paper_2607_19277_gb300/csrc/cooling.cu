// Optically thin radiative losses (paper Section 2.3.1, energy sink of Eq. 4) integrated
// exactly per cell (Townsend 2009): in code units de/dt = -rho^2 Lambda(T), T = p / rho, at
// fixed rho and momentum, i.e. dT/dt = -(gamma - 1) rho Lambda(T), so a step of dt moves T
// down to the T_new with  int_{T_new}^{T} dT'/Lambda = r = (gamma - 1) rho dt.
//
// Lambda is a caller's table (T_k, Lambda_k), a power law between nodes (the last segment
// continues above the table; no losses at or below T_0, which is the floor). On segment k,
// with e = 1 - alpha_k, the integral of 1/Lambda from T_k up to t is
//   (T_k / Lambda_k) expm1(e ln(t/T_k)) / e,
// and a remainder r' consumed below the upper end t of a (partial) segment lands on
//   T_new = t exp(log1p(-e q) / e),   q = r' Lambda(t) / t
// (limits ln(t/T_k) T_k/Lambda_k and t exp(-q) at e = 0). r is consumed segment by segment
// downward from T: Townsend's exact integration with the evolution function referred to
// each segment's upper end, so every quantity stays on the scale of the local cooling time.
// The table is built here on the host in FP64 and evaluated in the stencil precision. The
// losses are Strang split around each step: half of dt before, half after.
#include <math.h>

#include <vector>

#include "kernels.cuh"
#include "launch.h"

namespace agile {

namespace {
double em1_over(double e, double x) { return e != 0.0 ? std::expm1(e * x) / e : x; }
}  // namespace

int build_cool_table(const double* T, const double* L, int n, double gamma, int real_bytes, CoolHost* out) {
  if (n < 2 || n > COOL_MAX_NODES || !T || !L || !out) return 1;
  for (int k = 0; k < n; ++k) {
    if (!(T[k] > 0.0) || !(L[k] > 0.0) || !std::isfinite(T[k]) || !std::isfinite(L[k])) return 1;
    if (k > 0 && !(T[k] > T[k - 1])) return 1;
  }
  const int ns = n - 1;
  out->segd.assign((size_t)ns * COOL_SEG, 0.0);
  for (int k = 0; k < ns; ++k) {
    const double lt0 = std::log(T[k]), lt1 = std::log(T[k + 1]);
    const double alpha = std::log(L[k + 1] / L[k]) / std::log(T[k + 1] / T[k]);
    const double e = 1.0 - alpha;
    double* s = &out->segd[(size_t)k * COOL_SEG];
    s[0] = lt0;
    s[1] = T[k] / L[k];
    s[2] = e;
    s[3] = T[k] / L[k] * em1_over(e, std::log(T[k + 1] / T[k]));   // whole-segment integral
    s[4] = T[k + 1];
    s[5] = L[k + 1] / T[k + 1];
    s[6] = L[k] / T[k];
    s[7] = lt1;
  }
  out->segf.resize(out->segd.size());
  for (size_t i = 0; i < out->segd.size(); ++i) {
    if (!std::isfinite(out->segd[i])) return 1;
    out->segf[i] = (float)out->segd[i];
  }
  // nodes uniform in ln T allow an O(1) segment lookup
  const double l0 = std::log(T[0]), dl = (std::log(T[n - 1]) - l0) / ns;
  bool uni = dl > 0.0;
  for (int k = 1; k < n && uni; ++k)
    uni = std::fabs(std::log(T[k]) - (l0 + k * dl)) <= 1e-9 * dl;
  if (real_bytes == 4) {   // the FP32 stencil evaluates the table in float: it must fit
    for (float v : out->segf)
      if (!std::isfinite(v)) return 1;
  }
  out->nseg = ns;
  out->uniform = uni ? 1 : 0;
  out->lnT0 = l0;
  out->idln = uni ? 1.0 / dl : 0.0;
  out->T0 = T[0];
  out->g1 = gamma - 1.0;
  out->lnT0f = (float)out->lnT0;
  out->idlnf = (float)out->idln;
  out->T0f = (float)out->T0;
  out->g1f = (float)out->g1;
  return 0;
}

template <typename R> __device__ __forceinline__ R c_log(R x);
template <> __device__ __forceinline__ float c_log<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double c_log<double>(double x) { return log(x); }
template <typename R> __device__ __forceinline__ R c_exp(R x);
template <> __device__ __forceinline__ float c_exp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double c_exp<double>(double x) { return exp(x); }
template <typename R> __device__ __forceinline__ R c_expm1(R x);
template <> __device__ __forceinline__ float c_expm1<float>(float x) { return expm1f(x); }
template <> __device__ __forceinline__ double c_expm1<double>(double x) { return expm1(x); }
template <typename R> __device__ __forceinline__ R c_log1p(R x);
template <> __device__ __forceinline__ float c_log1p<float>(float x) { return log1pf(x); }
template <> __device__ __forceinline__ double c_log1p<double>(double x) { return log1p(x); }

// Temperature after dt of losses at density rho (unchanged at or below the floor, or when
// T is not a number).
template <typename R>
__device__ __forceinline__ R cool_temperature(R rho, R T, R dt, const CoolDev& c, const R* seg) {
  const R t0 = sizeof(R) == 4 ? R(c.T0f) : R(c.T0);
  if (!(T > t0)) return T;
  const R lt = c_log<R>(T);
  const int last = c.nseg - 1;
  int k;
  if (c.uniform) {
    k = sizeof(R) == 4 ? (int)((lt - R(c.lnT0f)) * R(c.idlnf)) : (int)((lt - R(c.lnT0)) * R(c.idln));
    k = k < 0 ? 0 : (k > last ? last : k);
    // rounding of the index near a node: step to the segment that holds lt
    if (k > 0 && lt < seg[k * COOL_SEG + 0]) --k;
    else if (k < last && lt >= seg[k * COOL_SEG + 7]) ++k;
  } else {
    int lo = 0, hi = last;      // largest k with ln T_k <= lt
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg[mid * COOL_SEG + 0] <= lt) lo = mid;
      else hi = mid - 1;
    }
    k = lo;
  }
  const R* s = seg + k * COOL_SEG;
  R e = s[2];
  const R x = lt - s[0];                                            // ln(T / T_k)
  R avail = s[1] * (e != R(0) ? c_expm1<R>(e * x) / e : x);         // int_{T_k}^{T} dT/Lambda
  R lam_t = s[6] * c_exp<R>(-e * x);                                // Lambda(T) / T
  R top = T;
  R r = (sizeof(R) == 4 ? R(c.g1f) : R(c.g1)) * rho * dt;
  for (int it = 0; it <= last; ++it) {     // at most one pass per segment below T
    if (r < avail) {
      const R q = r * lam_t;
      const R tn = top * c_exp<R>(e != R(0) ? c_log1p<R>(-e * q) / e : -q);
      return tn > t0 ? tn : t0;
    }
    if (k == 0) break;
    r -= avail;
    --k;
    s = seg + k * COOL_SEG;
    e = s[2];
    avail = s[3];
    top = s[4];
    lam_t = s[5];
  }
  return t0;
}

// One pass over the state: losses over frac * dt of each block's solve, then (optionally)
// the CFL signal speeds of the result.
template <template <typename> class PT, typename R>
__global__ void __launch_bounds__(256) cooling_kernel(R* __restrict__ U, const BlockDesc* __restrict__ bd,
                                                       CoolDev c, const R* __restrict__ seg,
                                                       const double* __restrict__ dtch, double frac,
                                                       const PhysParamsT<R> pp,   // formed on the host
                                                       unsigned long long* speeds,
                                                       int* status, const int* __restrict__ solve_of) {
  using P = PT<R>;
  constexpr int NV = P::NV;
  const int b = blockIdx.x;
  const int sv = solve_of ? solve_of[b] : 0;
  const R dt = R(frac * dtch[2 * sv]);
  const R ig1 = pp.ig1;
  const R dxr[3] = {R(bd[b].dx[0]), R(bd[b].dx[1]), R(bd[b].dx[2])};
  R ssum = R(0), smax = R(0);
  int st = 0;
  R* base = U + (size_t)b * NV * NCELL;
  for (int i = threadIdx.x; i < NCELL; i += 256) {
    R u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = base[(size_t)v * NCELL + i];
    R p[NV], aux[1] = {R(0)};
    P::cons2prim(u, p, aux, pp, st);
    constexpr int IE = P::IE;   // energy in U, pressure in P
    const R rho = p[0];
    const R T = p[IE] / rho;
    const R tn = cool_temperature<R>(rho, T, dt, c, seg);
    u[IE] = u[IE] - rho * (T - tn) * ig1;
    base[(size_t)IE * NCELL + i] = u[IE];
    if (speeds) cell_speeds<PT, R>(u, aux, pp, dxr, ssum, smax, st);
  }
  if (speeds) block_max2<256>(ssum, smax, speeds + 2 * sv);
  if (st) atomicOr(status, st);
}

cudaError_t launch_cooling(const AuxArgs& a, const CoolDev& c, const void* seg, const double* dtch,
                           double frac, unsigned long long* speeds, cudaStream_t s) {
  if (a.nblk == 0 || c.nseg <= 0) return cudaSuccess;
#define CALL(PT)                                                                                   \
  do {                                                                                             \
    PhysParamsT<R> pp;                                                                             \
    pp.set(a.gamma, 0.0);                                                                          \
    cooling_kernel<PT, R><<<a.nblk, 256, 0, s>>>((R*)a.Uw, a.bd, c, (const R*)seg, dtch, frac, pp, speeds, \
                                                 a.status, a.solve_of);                            \
  } while (0)
  if (a.phys == PH_HD) {
    if (a.real_bytes == 8) { using R = double; CALL(HdPhys); }
    else { using R = float; CALL(HdPhys); }
  } else if (a.phys == PH_MHD) {
    if (a.real_bytes == 8) { using R = double; CALL(MhdPhys); }
    else { using R = float; CALL(MhdPhys); }
  } else if (a.phys == PH_FFHD) {
    if (a.real_bytes == 8) { using R = double; CALL(FfhdPhys); }
    else { using R = float; CALL(FfhdPhys); }
  } else if (a.phys == PH_FFHD_HTC) {
    if (a.real_bytes == 8) { using R = double; CALL(FfhdHtcPhys); }
    else { using R = float; CALL(FfhdHtcPhys); }
  } else {
    return cudaErrorInvalidValue;
  }
#undef CALL
  return cudaGetLastError();
}

}  // namespace agile
