// Device physics traits for the finite-volume stage kernel (sm_103a).
//
// Each trait gives the conserved <-> primitive maps, the physical flux along one axis and
// the approximate Riemann flux at a face, evaluated per cell in registers (the paper's
// cell-local physics routines, Section 2.3):
//   HdPhys   : Eqs. 2-4 with e = p/(gamma-1) + rho v^2/2 (Eq. 6; Section 2.3.1; HD flux listing)
//   MhdPhys  : Eqs. 11-13 with GLM (Eq. 14), e = p/(gamma-1) + rho v^2/2 + B^2/2 (Section 2.3.3)
//   SrhdPhys : Eqs. 15-20 with the ideal-gas enthalpy of Eq. 21 (Section 2.3.4), and
//   SrhdSyngePhys with the approximate Synge-gas enthalpy (Eq. 22, Mathews' form); the
//              conserved-to-primitive recovery is a Newton root find in xi = Gamma^2 rho h,
//              always in FP64.
// Riemann fluxes: HLL with Davis wave-speed estimates, or TVDLF (Rusanov) with the larger
// of the two sides' fastest speeds (paper Table 1 lists the solvers per module).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace agile {

enum : int { LIM_MINMOD = 0, LIM_VANLEER = 1 };
enum : int { FLUX_TVDLF = 0, FLUX_HLL = 1, FLUX_HLLC = 2 };
enum : int { ST_ENOCONV = 1, ST_EUNPHYS = 2 };

// Equation parameters in the stencil precision R, derived once per CTA (the FP64 copy of
// gamma serves the SRHD primitive recovery, which always runs in FP64).
template <typename R>
struct PhysParamsT {
  double gamma_d, gm_d;    // gamma and (gamma - 1) / gamma in FP64 (SRHD primitive recovery)
  R gamma, g1, ig1, gg1;   // gamma, gamma - 1, 1 / (gamma - 1), gamma / (gamma - 1)
  R gmr;                   // (gamma - 1) / gamma in the stencil precision
  R ch, ich, ch2;          // GLM cleaning speed c_h = c_max of U^n (MHD), 1 / c_h, c_h^2
  __host__ __device__ void set(double gamma_, double ch_) {
    gamma_d = gamma_;
    gm_d = (gamma_ - 1.0) / gamma_;
    gamma = R(gamma_);
    g1 = R(gamma_ - 1.0);
    ig1 = R(1.0 / (gamma_ - 1.0));
    gg1 = R(gamma_ / (gamma_ - 1.0));
    gmr = R(gm_d);
    set_ch(ch_);
  }
  __host__ __device__ void set_ch(double ch_) {
    ch = R(ch_);
    ich = ch_ > 0.0 ? R(1.0 / ch_) : R(0);
    ch2 = R(ch_ * ch_);
  }
};

__device__ __forceinline__ float rabs(float a) { return fabsf(a); }
__device__ __forceinline__ double rabs(double a) { return fabs(a); }
__device__ __forceinline__ float rmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double rmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float rsqrt_(float a) { return sqrtf(a); }
__device__ __forceinline__ double rsqrt_(double a) { return sqrt(a); }
__device__ __forceinline__ float rsign(float a) { return copysignf(1.0f, a); }
__device__ __forceinline__ double rsign(double a) { return copysign(1.0, a); }
// Reciprocal and quotient in the stencil precision. FP32: the build's fast single-precision
// divide. FP64: the hardware reciprocal estimate (PTX rcp.approx.ftz.f64) refined by one
// third-order Newton-Raphson step: with e = 1 - s r0, r1 = r0 (1 + e + e^2) is the series of
// r0 / (s r0) = r0 / (1 - e) truncated after e^2, so its relative error is e^3, far below
// 2^-53 for the estimate's error. The product a r1 lies within 1 ulp of the rounded quotient
// a / s (4 FP64 operations against about twice as many for the IEEE divide, which the FP64
// units of this GPU make the costly part of the stencil). Valid for normal, finite s with
// |s| < 2^1022; every divisor below is a density, a sum of two same-sign slopes, a signal-
// speed interval or a Newton derivative (a zero or non-finite one yields NaN, as the IEEE
// quotient's use would).
__device__ __forceinline__ double rcp64(double s) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(s));
  const double e = fma(-s, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ float rrcp(float s) { return 1.0f / s; }
__device__ __forceinline__ double rrcp(double s) { return rcp64(s); }
__device__ __forceinline__ float rdiv(float a, float s) { return a / s; }
__device__ __forceinline__ double rdiv(double a, double s) { return a * rcp64(s); }
template <typename R> __device__ __forceinline__ R rtiny();
template <> __device__ __forceinline__ float rtiny<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double rtiny<double>() { return 1e-300; }

// Half of the limited slope, sigma / 2, from the two one-sided differences a and b, written
// without branches (the final choice is a select):
//   minmod: sigma = (sgn a + sgn b)/2 min(|a|, |b|)  (0 unless a and b share a sign);
//   van Leer (1974): sigma = 2ab / (a + b) when ab > 0, else 0. The quotient is formed for
//   every input and discarded when ab <= 0, where a + b may vanish.
// Halving is exact, so sigma / 2 equals half the limiter value bit for bit.
template <typename R, int LIM>
__device__ __forceinline__ R half_slope(R a, R b) {
  if (LIM == LIM_MINMOD) {
    return (R(0.25) * (rsign(a) + rsign(b))) * rmin(rabs(a), rabs(b));
  } else {
    const R ab = a * b;
    const R q = rdiv(ab, a + b);
    return ab > R(0) ? q : R(0);
  }
}

// ------------------------------------------------------------------------------ hydro
template <typename R>
struct HdPhys {
  static constexpr int NV = 5;   // rho, m, e
  static constexpr int NA = 0;
  static constexpr int BOFF = -1;  // no magnetic field
  static constexpr int IV = 1;     // first velocity / momentum component
  static constexpr int NREC = NV;  // reconstructed variables
  static constexpr int FROZEN = NV;  // variables from this index on are never updated
  static constexpr int QV = -1;      // a variable with no face flux (source-only), or -1
  static constexpr int IE = 4;     // energy in U, pressure in P
  static constexpr bool SOURCE = false;
  static constexpr bool GLM = false;

  __device__ static __forceinline__ void cons2prim(const R* u, R* p, R*, const PhysParamsT<R>& pp,
                                                   int& st) {
    const R g1 = pp.g1;
    const R rho = u[0];
    const R ir = rrcp(rho);
    const R vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
    p[0] = rho;
    p[1] = vx;
    p[2] = vy;
    p[3] = vz;
    p[4] = g1 * (u[4] - R(0.5) * rho * (vx * vx + vy * vy + vz * vz));
    st |= (!(rho > R(0)) | !(p[4] > R(0))) ? ST_EUNPHYS : 0;
  }

  __device__ static __forceinline__ void prim2cons(const R* p, R* u, const PhysParamsT<R>& pp) {
    const R ig1 = pp.ig1;
    u[0] = p[0];
    u[1] = p[0] * p[1];
    u[2] = p[0] * p[2];
    u[3] = p[0] * p[3];
    u[4] = p[4] * ig1 + R(0.5) * p[0] * (p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  }

  template <int D>
  __device__ static __forceinline__ void flux(const R* p, const R* u, R* f, const PhysParamsT<R>&) {
    const R vd = p[1 + D];
    f[0] = u[0] * vd;
    f[1] = u[1] * vd;
    f[2] = u[2] * vd;
    f[3] = u[3] * vd;
    f[1 + D] += p[4];
    f[4] = vd * (u[4] + p[4]);
  }

  template <int D>
  __device__ static __forceinline__ void lambdas(const R* p, R& lm, R& lp, const PhysParamsT<R>& pp) {
    const R c = rsqrt_(rdiv(pp.gamma * p[4], p[0]));
    lm = p[1 + D] - c;
    lp = p[1 + D] + c;
  }

  template <int D>
  __device__ static __forceinline__ void interface(R*, R*, const PhysParamsT<R>&) {}
};

// ------------------------------------------------------------------------------ MHD + GLM
template <typename R>
struct MhdPhys {
  static constexpr int NV = 9;   // rho, m, e, B, psi
  static constexpr int NA = 0;
  static constexpr int BOFF = 5;   // B_x is variable 5
  static constexpr int IV = 1;
  static constexpr int NREC = NV;
  static constexpr int FROZEN = NV;
  static constexpr int QV = -1;
  static constexpr int IE = 4;
  static constexpr bool SOURCE = false;
  static constexpr bool GLM = true;

  __device__ static __forceinline__ void cons2prim(const R* u, R* p, R*, const PhysParamsT<R>& pp,
                                                   int& st) {
    const R g1 = pp.g1;
    const R rho = u[0];
    const R ir = rrcp(rho);
    const R vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
    const R b2 = u[5] * u[5] + u[6] * u[6] + u[7] * u[7];
    p[0] = rho;
    p[1] = vx;
    p[2] = vy;
    p[3] = vz;
    p[4] = g1 * (u[4] - R(0.5) * rho * (vx * vx + vy * vy + vz * vz) - R(0.5) * b2);
    p[5] = u[5];
    p[6] = u[6];
    p[7] = u[7];
    p[8] = u[8];
    st |= (!(rho > R(0)) | !(p[4] > R(0))) ? ST_EUNPHYS : 0;
  }

  __device__ static __forceinline__ void prim2cons(const R* p, R* u, const PhysParamsT<R>& pp) {
    const R ig1 = pp.ig1;
    u[0] = p[0];
    u[1] = p[0] * p[1];
    u[2] = p[0] * p[2];
    u[3] = p[0] * p[3];
    u[4] = p[4] * ig1 + R(0.5) * p[0] * (p[1] * p[1] + p[2] * p[2] + p[3] * p[3]) +
           R(0.5) * (p[5] * p[5] + p[6] * p[6] + p[7] * p[7]);
    u[5] = p[5];
    u[6] = p[6];
    u[7] = p[7];
    u[8] = p[8];
  }

  template <int D>
  __device__ static __forceinline__ void flux(const R* p, const R* u, R* f, const PhysParamsT<R>& pp) {
    const R vd = p[1 + D], bd = p[5 + D];
    const R ptot = p[4] + R(0.5) * (p[5] * p[5] + p[6] * p[6] + p[7] * p[7]);
    const R vb = p[1] * p[5] + p[2] * p[6] + p[3] * p[7];
    f[0] = u[0] * vd;
    f[1] = u[1] * vd - p[5] * bd;
    f[2] = u[2] * vd - p[6] * bd;
    f[3] = u[3] * vd - p[7] * bd;
    f[1 + D] += ptot;
    f[4] = vd * (u[4] + ptot) - bd * vb;
    f[5] = vd * p[5] - bd * p[1];
    f[6] = vd * p[6] - bd * p[2];
    f[7] = vd * p[7] - bd * p[3];
    f[5 + D] = p[8];
    f[8] = pp.ch2 * bd;
  }

  template <int D>
  __device__ static __forceinline__ void lambdas(const R* p, R& lm, R& lp, const PhysParamsT<R>& pp) {
    const R ir = rrcp(p[0]);
    const R a2 = pp.gamma * p[4] * ir;
    const R b2 = (p[5] * p[5] + p[6] * p[6] + p[7] * p[7]) * ir;
    const R bd2 = p[5 + D] * p[5 + D] * ir;
    const R s = a2 + b2;
    const R disc = rmax(s * s - R(4) * a2 * bd2, R(0));
    const R cf = rsqrt_(R(0.5) * (s + rsqrt_(disc)));
    lm = p[1 + D] - cf;
    lp = p[1 + D] + cf;
  }

  // Exact solution of the linear (B_d, psi) subsystem at the face (Dedner et al. 2002):
  // both face states carry B_d* and psi*, so the face flux of B_d is psi* and of psi is
  // c_h^2 B_d*.
  template <int D>
  __device__ static __forceinline__ void interface(R* pl, R* pr, const PhysParamsT<R>& pp) {
    const R ch = pp.ch;
    const R bl = pl[5 + D], br = pr[5 + D], sl = pl[8], sr = pr[8];
    const R bs = R(0.5) * (bl + br) - R(0.5) * (sr - sl) * pp.ich;
    const R ss = R(0.5) * (sl + sr) - R(0.5) * ch * (br - bl);
    pl[5 + D] = bs;
    pr[5 + D] = bs;
    pl[8] = ss;
    pr[8] = ss;
  }
};

// Ideal MHD with uniform resistivity eta (Section 2.3.3: -curl(eta J) in the induction
// equation, div(B x eta J) in the energy equation): the MHD trait with the RES flag, for
// which the stage kernel adds eta lap B to the induction equation and eta (J.J + B.lap B)
// to the energy equation, from the stage state with the compact stencil over the six face
// neighbours (central differences for J = curl B, the 7-point Laplacian).
template <typename R>
struct MhdResPhys : MhdPhys<R> {
  static constexpr bool RES = true;
};

// Whether a trait carries the resistive terms.
template <class P, class = void>
struct res_of {
  static constexpr bool value = false;
};
template <class P>
struct res_of<P, std::void_t<decltype(P::RES)>> {
  static constexpr bool value = P::RES;
};

// Whether a trait's primitive recovery is costly enough (an iteration) to be done once per
// cell in a pass of its own before the stage kernel, which then reads primitives: the stage
// kernel would otherwise recover each stored cell 1.75 times (own z-halo planes, x/y halo
// cells of the neighbours).
template <class P, class = void>
struct prim_pass_of {
  static constexpr bool value = false;
};
template <class P>
struct prim_pass_of<P, std::void_t<decltype(P::PRIM_PASS)>> {
  static constexpr bool value = P::PRIM_PASS;
};

// ------------------------------------------------------------------------------ SRHD
enum : int { EOS_IDEAL = 0, EOS_SYNGE = 1 };

// Closure h(rho, p) of Section 2.3.4: the ideal gas h = 1 + gamma/(gamma-1) theta (Eq. 21)
// or the Synge gas (Eq. 22) in Mathews' approximation h = 5/2 theta + sqrt(9/4 theta^2 + 1),
// theta = p / rho, which tends to the ideal gas with gamma = 5/3 (cold) and 4/3 (hot).
template <typename R, int EOS>
struct SrhdEos {
  __device__ static __forceinline__ R enthalpy(R theta, const PhysParamsT<R>& pp) {
    if constexpr (EOS == EOS_SYNGE) return R(2.5) * theta + rsqrt_(R(2.25) * theta * theta + R(1));
    else return R(1) + pp.gg1 * theta;
  }
  // squared sound speed: gamma theta / h, or theta (5h - 8 theta) / (3h (h - theta)) for the
  // approximate Synge gas (the isentropic derivative of its enthalpy)
  __device__ static __forceinline__ R sound_speed2(R theta, R h, const PhysParamsT<R>& pp) {
    if constexpr (EOS == EOS_SYNGE) return rdiv(theta * (R(5) * h - R(8) * theta), R(3) * h * (h - theta));
    else return rdiv(pp.gamma * theta, h);
  }
};

template <typename R, int EOS>
struct SrhdPhysE {
  static constexpr int NV = 5;   // D, m, tau ; primitives rho, u = Gamma v, p
  static constexpr int NA = 2;   // xi = Gamma^2 rho h, Gamma
  static constexpr bool PRIM_PASS = true;   // the Newton recovery runs once per cell
  static constexpr int BOFF = -1;
  static constexpr int IV = 1;
  static constexpr int NREC = NV;
  static constexpr int FROZEN = NV;
  static constexpr int QV = -1;
  static constexpr int IE = 4;
  static constexpr bool SOURCE = false;
  static constexpr bool GLM = false;
  using Eos = SrhdEos<R, EOS>;

  // The same Newton iteration in FP32, to |dxi| <= 1e-6 xi (at most 12 steps): in the FP32
  // stencil it moves the starting point of the FP64 iteration close to the root, so that the
  // FP64 iteration (which alone decides convergence and the result) needs about one step.
  // Returns the start unchanged when it does not converge (the caller checks the bracket).
  __device__ static __forceinline__ double seed_f32(float x, float df_, float s2f, float ef, float l, float h,
                                                    const PhysParamsT<R>& pp) {
    const float gmf = (float)pp.gmr;
    const float idf = EOS == EOS_SYNGE ? 1.0f / df_ : 0.0f;
    const float x0 = x;
    for (int it = 0; it < 12; ++it) {
      const float ixi = 1.0f / x;
      const float w = s2f * ixi * ixi;
      const float ig2 = 1.0f - w;
      const float lor = rsqrtf(ig2);
      const float rho = df_ * (ig2 * lor);
      const float drho = df_ * lor * w * ixi;
      float pr, dp;
      if constexpr (EOS == EOS_SYNGE) {
        const float hh = x * (ig2 * lor) * idf;
        const float q = 9.0f * hh * hh + 16.0f;
        const float iq = rsqrtf(q);
        const float th = 0.125f * (5.0f * hh - q * iq);
        pr = rho * th;
        dp = th * drho + 0.125f * (5.0f - 9.0f * hh * iq);
      } else {
        pr = gmf * (x * ig2 - rho);
        dp = gmf * (1.0f + w - drho);
      }
      const float f = x - pr - ef;
      if (f < 0.0f) l = x; else h = x;
      float xn = x - f / (1.0f - dp);
      if (!(xn >= l && xn <= h)) xn = 0.5f * (l + h);
      const bool conv = fabsf(xn - x) <= 1e-6f * xn;
      x = xn;
      if (conv) return (double)x;
    }
    return (double)x0;
  }

  // Newton root find for f(xi) = xi - p(xi) - (tau + D) = 0 inside the bracket [E, k E]
  // (k = gamma for the ideal gas, whose p <= (gamma-1)/gamma xi; k = 4/3 for the approximate
  // Synge gas, whose h >= 4 theta gives p <= xi/4); starts from the stored xi when it lies
  // strictly inside the bracket, else from the midpoint (in the FP32 stencil first refined by
  // seed_f32); a step leaving the closed bracket is replaced by bisection; stops when
  // |dxi| <= tol xi (below); at most 50 iterations. FP64.
  __device__ static __forceinline__ void cons2prim(const R* u, R* p, R* aux, const PhysParamsT<R>& pp,
                                                   int& st) {
    const double g = pp.gamma_d;
    const double gm = pp.gm_d;
    const double D = (double)u[0];
    const double mx = (double)u[1], my = (double)u[2], mz = (double)u[3];
    const double s2 = mx * mx + my * my + mz * mz;
    const double E = (double)u[4] + D;
    double lo = E, hi = (EOS == EOS_SYNGE ? 4.0 / 3.0 : g) * E;
    const double iD = EOS == EOS_SYNGE ? rcp64(D) : 0.0;
    double xi;
    if constexpr (sizeof(R) == 4) {
      // the FP32 start from the FP32 inputs (no FP64 -> FP32 conversions), in the bracket
      // [E, k E] formed in FP32; the result lands in the FP64 bracket or the FP64 midpoint
      // is taken
      const float ef = u[4] + u[0];
      const float lof = ef, hif = (EOS == EOS_SYNGE ? 4.0f / 3.0f : (float)pp.gamma) * ef;
      float x0 = aux[0];
      if (!(x0 > lof && x0 < hif)) x0 = 0.5f * (lof + hif);
      const float s2f = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
      xi = seed_f32(x0, u[0], s2f, ef, lof, hif, pp);
    } else {
      xi = (double)aux[0];
    }
    if (!(xi > lo && xi < hi)) xi = 0.5 * (lo + hi);
    // FP64 stencil: |dxi| <= 1e-14 xi. FP32 stencil: |dxi| <= 1e-6 xi; Newton converges
    // quadratically, so the iterate after such a step is within about (1e-6)^2 relative
    // (times a factor that grows like Gamma^3), far below the FP32 rounding of the output.
    constexpr double tol = sizeof(R) == 4 ? 1e-6 : 1e-14;
    bool ok = false;
    // quantities of the last iteration, evaluated at its starting point xs
    double xs = xi, ixi = 1.0, w = 0.0, lor = 1.0, rho = 0.0, drho = 0.0, pr = 0.0, dp = 0.0;
    for (int it = 0; it < 50; ++it) {
      xs = xi;
      ixi = rcp64(xi);
      w = s2 * ixi * ixi;                       // v^2
      const double ig2 = 1.0 - w;               // 1 / Gamma^2
      lor = rsqrt(ig2);                         // Gamma
      rho = D * (ig2 * lor);                    // D / Gamma
      drho = D * lor * w * ixi;                 // d rho / d xi
      if constexpr (EOS == EOS_SYNGE) {
        // h = xi / (D Gamma), theta(h) = (5h - sqrt(9h^2 + 16)) / 8, dh/dxi = Gamma / D
        const double h = xi * (ig2 * lor) * iD;
        const double q = 9.0 * h * h + 16.0;
        const double iq = rsqrt(q);
        const double th = 0.125 * (5.0 * h - q * iq);
        pr = rho * th;
        dp = th * drho + 0.125 * (5.0 - 9.0 * h * iq);
      } else {
        pr = gm * (xi * ig2 - rho);
        dp = gm * (1.0 + w - drho);
      }
      const double f = xi - pr - E;
      const double df = 1.0 - dp;
      if (f < 0.0) lo = xi; else hi = xi;
      double xn = xi - f * rcp64(df);
      if (!(xn >= lo && xn <= hi)) xn = 0.5 * (lo + hi);
      const bool conv = fabs(xn - xi) <= tol * xn;
      xi = xn;
      if (conv) { ok = true; break; }
    }
    if (!ok) st |= ST_ENOCONV;
    // The primitives at the converged xi from those of the last iterate xs by first-order
    // Taylor steps (the derivatives are the iteration's own): |xi - xs| <= tol xi, so the
    // neglected second-order terms are of relative size tol^2 (1e-28 in the FP64 stencil,
    // 1e-12 in the FP32 one), far below the rounding of the result.
    const double dx = xi - xs;
    const double ixn = fma(-ixi * ixi, dx, ixi);                    // d(1/xi) = -dx / xi^2
    const double lorn = fma(-(lor * lor * lor) * (w * ixi), dx, lor);   // dGamma/dxi = -Gamma^3 v^2 / xi
    const double rhon = fma(drho, dx, rho);
    const double prn = fma(dp, dx, pr);
    const double sc = lorn * ixn;
    p[0] = (R)rhon;
    if constexpr (sizeof(R) == 4) {   // u = Gamma v = m Gamma / xi: one conversion of the factor
      const R scr = (R)sc;
      p[1] = u[1] * scr;
      p[2] = u[2] * scr;
      p[3] = u[3] * scr;
    } else {
      p[1] = (R)(mx * sc);
      p[2] = (R)(my * sc);
      p[3] = (R)(mz * sc);
    }
    pr = prn;
    rho = rhon;
    lor = lorn;
    p[4] = (R)pr;
    aux[0] = (R)xi;
    aux[1] = (R)lor;
    if (!(rho > 0.0) || !(pr > 0.0)) st |= ST_EUNPHYS;
  }

  __device__ static __forceinline__ R enthalpy(R rho, R pres, const PhysParamsT<R>& pp) {
    return Eos::enthalpy(rdiv(pres, rho), pp);
  }

  __device__ static __forceinline__ void prim2cons(const R* p, R* u, const PhysParamsT<R>& pp) {
    const R lor = rsqrt_(R(1) + p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    R h;
    if constexpr (EOS == EOS_SYNGE) h = Eos::enthalpy(rdiv(p[4], p[0]), pp);
    else h = R(1) + rdiv(pp.gg1 * p[4], p[0]);
    const R lr = lor * p[0];
    const R lrh = lr * h;
    u[0] = lr;
    u[1] = lrh * p[1];
    u[2] = lrh * p[2];
    u[3] = lrh * p[3];
    u[4] = lor * lrh - p[4] - lr;
  }

  template <int D>
  __device__ static __forceinline__ void flux(const R* p, const R* u, R* f, const PhysParamsT<R>&) {
    const R lor = rsqrt_(R(1) + p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    const R vd = rdiv(p[1 + D], lor);
    f[0] = u[0] * vd;
    f[1] = u[1] * vd;
    f[2] = u[2] * vd;
    f[3] = u[3] * vd;
    f[1 + D] += p[4];
    f[4] = u[1 + D] - u[0] * vd;
  }

  template <int D>
  __device__ static __forceinline__ void lambdas(const R* p, R& lm, R& lp, const PhysParamsT<R>& pp) {
    const R lor2 = R(1) + p[1] * p[1] + p[2] * p[2] + p[3] * p[3];
    const R v2 = R(1) - rrcp(lor2);
    const R vd = rdiv(p[1 + D], rsqrt_(lor2));
    R cs2;
    if constexpr (EOS == EOS_SYNGE) {
      const R th = rdiv(p[4], p[0]);
      cs2 = Eos::sound_speed2(th, Eos::enthalpy(th, pp), pp);
    } else {
      const R h = R(1) + rdiv(pp.gg1 * p[4], p[0]);
      cs2 = rdiv(pp.gamma * p[4], p[0] * h);
    }
    const R cs = rsqrt_(cs2);
    const R den = R(1) - v2 * cs2;
    const R root = cs * rsqrt_(rmax((R(1) - v2) * (R(1) - v2 * cs2 - vd * vd * (R(1) - cs2)), R(0)));
    const R iden = rrcp(den);
    lm = (vd * (R(1) - cs2) - root) * iden;
    lp = (vd * (R(1) - cs2) + root) * iden;
  }

  template <int D>
  __device__ static __forceinline__ void interface(R*, R*, const PhysParamsT<R>&) {}
};

template <typename R> using SrhdPhys = SrhdPhysE<R, EOS_IDEAL>;
template <typename R> using SrhdSyngePhys = SrhdPhysE<R, EOS_SYNGE>;

// ------------------------------------------------------------------------------ FFHD
// Frozen-field hydrodynamics (Section 2.3.2, Eqs. 7-9): U = (rho, m_par, e, b), P = (rho,
// v_par, p, b) with b the frozen unit field, never updated and not reconstructed (cell
// values; the face value of b_d is the mean of the two cells'). The flux along d is
// b_d (rho v, rho v^2 + p, (e + p) v) and b_d for the variable b_d (0 for the other two), so
// the flux divergence of the b variables is -div b of the same face values; the source
// p div b of the m_par equation is added from it. TVDLF only (paper Table 1).
// With hyperbolic thermal conduction (HTC, Eqs. 9-10): U = (rho, m_par, e, q_par, b); q_par
// is reconstructed, has no face flux of its own (no dissipation either) and enters the
// energy flux as -q_par b_d; its relaxation towards kappa0 T^(5/2) b.grad T over tau = 4 dt
// is the stage kernel's source term for it.
template <typename R, bool HTC>
struct FfhdPhysT {
  static constexpr int NV = HTC ? 7 : 6;
  static constexpr int NA = 0;
  static constexpr int BOFF = HTC ? 4 : 3;   // b: swapped with the x/y trick, b_n negated at walls
  static constexpr int IV = -1;              // no vector velocity
  static constexpr int NREC = HTC ? 4 : 3;
  static constexpr int FROZEN = BOFF;
  static constexpr int QV = HTC ? 3 : -1;
  static constexpr int IE = 2;
  static constexpr bool SOURCE = true;
  static constexpr bool GLM = false;

  __device__ static __forceinline__ void cons2prim(const R* u, R* p, R*, const PhysParamsT<R>& pp,
                                                   int& st) {
    const R rho = u[0];
    const R v = u[1] * rrcp(rho);
    p[0] = rho;
    p[1] = v;
    p[2] = pp.g1 * (u[2] - R(0.5) * rho * v * v);
#pragma unroll
    for (int i = 3; i < NV; ++i) p[i] = u[i];
    st |= (!(rho > R(0)) | !(p[2] > R(0))) ? ST_EUNPHYS : 0;
  }

  __device__ static __forceinline__ void prim2cons(const R* p, R* u, const PhysParamsT<R>& pp) {
    u[0] = p[0];
    u[1] = p[0] * p[1];
    u[2] = p[2] * pp.ig1 + R(0.5) * p[0] * p[1] * p[1];
#pragma unroll
    for (int i = 3; i < NV; ++i) u[i] = p[i];
  }

  template <int D>
  __device__ static __forceinline__ void flux(const R* p, const R* u, R* f, const PhysParamsT<R>&) {
    const R b = p[BOFF + D];
    const R vb = p[1] * b;
    f[0] = u[0] * vb;
    f[1] = u[1] * vb + p[2] * b;
    if constexpr (HTC) f[2] = (u[2] + p[2]) * vb - p[3] * b;
    else f[2] = (u[2] + p[2]) * vb;
#pragma unroll
    for (int i = 3; i < NV; ++i) f[i] = R(0);
    f[BOFF + D] = b;
  }

  template <int D>
  __device__ static __forceinline__ void lambdas(const R* p, R& lm, R& lp, const PhysParamsT<R>& pp) {
    const R c = rsqrt_(rdiv(pp.gamma * p[2], p[0]));
    const R b = p[BOFF + D];
    const R a = p[1] * b;
    const R w = c * rabs(b);
    lm = a - w;
    lp = a + w;
  }

  template <int D>
  __device__ static __forceinline__ void interface(R* pl, R* pr, const PhysParamsT<R>&) {
    const R bf = R(0.5) * (pl[BOFF + D] + pr[BOFF + D]);
    pl[BOFF + D] = bf;
    pr[BOFF + D] = bf;
  }

  // L holds -div F of every variable: L[BOFF..BOFF+2] sum to -div b; adds p div b to m_par.
  __device__ static __forceinline__ void source(R* L, const R* pcell) {
    L[1] = L[1] - pcell[2] * ((L[BOFF] + L[BOFF + 1]) + L[BOFF + 2]);
  }
};
template <typename R> using FfhdPhys = FfhdPhysT<R, false>;
template <typename R> using FfhdHtcPhys = FfhdPhysT<R, true>;

// Riemann flux at a face from reconstructed primitive states (modified in place).
template <class P, typename R, int D, int FLUX>
__device__ __forceinline__ void riemann(R* pl, R* pr, R* f, const PhysParamsT<R>& pp) {
  constexpr int NV = P::NV;
  P::template interface<D>(pl, pr, pp);
  R ul[NV], ur[NV], fl[NV], fr[NV];
  P::prim2cons(pl, ul, pp);
  P::prim2cons(pr, ur, pp);
  P::template flux<D>(pl, ul, fl, pp);
  P::template flux<D>(pr, ur, fr, pp);
  R lml, lpl, lmr, lpr;
  P::template lambdas<D>(pl, lml, lpl, pp);
  P::template lambdas<D>(pr, lmr, lpr, pp);
  if constexpr (FLUX == FLUX_HLLC) {
    // HLLC (Toro, Spruce & Speares 1994) for hydrodynamics: the HLL fan with the contact
    // restored; star states U*_K = rho_K (S_K - u_K)/(S_K - S*) [1, S* e_d + v_t,
    // E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))], flux F_K + S_K (U*_K - U_K).
    const R sl = rmin(lml, lmr), sr = rmax(lpl, lpr);
    const R rl = pl[0], rr = pr[0], vl = pl[1 + D], vr = pr[1 + D];
    const R ml = rl * (sl - vl), mr = rr * (sr - vr);
    const R ss = rdiv(pr[4] - pl[4] + ml * vl - mr * vr, ml - mr);
    const R fl_ = rdiv(ml, sl - ss), fr_ = rdiv(mr, sr - ss);
    R usl[NV], usr[NV];
    usl[0] = fl_;
    usr[0] = fr_;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      usl[1 + i] = fl_ * pl[1 + i];
      usr[1 + i] = fr_ * pr[1 + i];
    }
    usl[1 + D] = fl_ * ss;
    usr[1 + D] = fr_ * ss;
    usl[4] = fl_ * (rdiv(ul[4], rl) + (ss - vl) * (ss + rdiv(pl[4], ml)));
    usr[4] = fr_ * (rdiv(ur[4], rr) + (ss - vr) * (ss + rdiv(pr[4], mr)));
    const bool left = sl >= R(0), star_l = ss >= R(0), star_r = sr > R(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R fsl = fl[v] + sl * (usl[v] - ul[v]);
      const R fsr = fr[v] + sr * (usr[v] - ur[v]);
      f[v] = left ? fl[v] : (star_l ? fsl : (star_r ? fsr : fr[v]));
    }
  } else if (FLUX == FLUX_TVDLF) {
    const R c = rmax(rmax(rabs(lml), rabs(lpl)), rmax(rabs(lmr), rabs(lpr)));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (v >= P::FROZEN) f[v] = fl[v];   // frozen variables: exact flux, no dissipation
      else if (v == P::QV) f[v] = R(0);   // no flux term at all
      else f[v] = R(0.5) * (fl[v] + fr[v]) - R(0.5) * c * (ur[v] - ul[v]);
    }
  } else {
    const R sl = rmin(rmin(lml, lmr), R(0));
    const R sr = rmax(rmax(lpl, lpr), R(0));
    const R inv = rrcp(sr - sl);
    const R wl = sr * inv, wr = sl * inv, wd = sl * sr * inv;
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = wl * fl[v] - wr * fr[v] + wd * (ur[v] - ul[v]);
  }
}

// PLM face states: pl = P_i + phi_i / 2, pr = P_{i+1} - phi_{i+1} / 2 from the four cells
// i-1, i, i+1, i+2 around face i+1/2.
template <int NV, typename R, int LIM, int NREC = NV>
__device__ __forceinline__ void plm(const R* a, const R* b, const R* c, const R* d, R* pl, R* pr) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v < NREC) {
      const R d0 = b[v] - a[v], d1 = c[v] - b[v], d2 = d[v] - c[v];
      pl[v] = b[v] + half_slope<R, LIM>(d0, d1);
      pr[v] = c[v] - half_slope<R, LIM>(d1, d2);
    } else {                 // not reconstructed: the cell values
      pl[v] = b[v];
      pr[v] = c[v];
    }
  }
}

}  // namespace agile
