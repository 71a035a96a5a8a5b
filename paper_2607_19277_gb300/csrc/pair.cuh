// Packed FP32 pairs for the x/y-face pass of the FP32 stage kernel.
//
// A thread of the stage kernel owns one x-face and one y-face of the current plane. With the
// x and y vector components of the y-face states exchanged, both are Riemann problems of the
// same form (the x-face solver), so their arithmetic runs as one stream of the packed FP32
// instructions of the sm_100 family (add / sub / mul / fma .f32x2: one issue, two results).
// Reciprocals, square roots, minima, maxima and selects act on each half. The pair forms
// below restate, for the x direction, the face states (PLM, Section 2.1.1), the primitive-to-
// conserved map, physical fluxes and signal speeds of HD (Section 2.3.1, Eqs. 2-6) and MHD
// with GLM (Section 2.3.3, Eqs. 11-14) and the HLL / TVDLF fluxes of the scalar solver; their
// products and sums are contracted into fused multiply-adds in places where the scalar code
// rounds separately, so a face flux agrees with the scalar solver's to a few FP32 ulps.
#pragma once
#include "physics.cuh"

namespace agile {

struct f2 {
  unsigned long long v;
};

__device__ __forceinline__ f2 f2_of(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_split(f2 a, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
}
__device__ __forceinline__ f2 bc2(float a) { return f2_of(a, a); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
  f2 r;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
// a * b + c, one rounding per half
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f2 rcp2(f2 a) {
  float x, y;
  f2_split(a, x, y);
  return f2_of(1.0f / x, 1.0f / y);
}
__device__ __forceinline__ f2 div2(f2 a, f2 b) {
  float ax, ay, bx, by;
  f2_split(a, ax, ay);
  f2_split(b, bx, by);
  return f2_of(ax / bx, ay / by);
}
__device__ __forceinline__ f2 sqrt2(f2 a) {
  float x, y;
  f2_split(a, x, y);
  return f2_of(sqrtf(x), sqrtf(y));
}
__device__ __forceinline__ f2 max2(f2 a, f2 b) {
  float ax, ay, bx, by;
  f2_split(a, ax, ay);
  f2_split(b, bx, by);
  return f2_of(fmaxf(ax, bx), fmaxf(ay, by));
}
__device__ __forceinline__ f2 min2(f2 a, f2 b) {
  float ax, ay, bx, by;
  f2_split(a, ax, ay);
  f2_split(b, bx, by);
  return f2_of(fminf(ax, bx), fminf(ay, by));
}
__device__ __forceinline__ f2 abs2(f2 a) {
  float x, y;
  f2_split(a, x, y);
  return f2_of(fabsf(x), fabsf(y));
}

// Half limited slope of each half (the scalar half_slope's limiters).
template <int LIM>
__device__ __forceinline__ f2 half_slope2(f2 a, f2 b) {
  if (LIM == LIM_MINMOD) {
    float ax, ay, bx, by;
    f2_split(a, ax, ay);
    f2_split(b, bx, by);
    return f2_of(half_slope<float, LIM>(ax, bx), half_slope<float, LIM>(ay, by));
  } else {
    const f2 ab = a * b;
    const f2 q = ab * rcp2(a + b);
    float abx, aby, qx, qy;
    f2_split(ab, abx, aby);
    f2_split(q, qx, qy);
    return f2_of(abx > 0.0f ? qx : 0.0f, aby > 0.0f ? qy : 0.0f);
  }
}

// PLM face states from the four cells around each face of the pair; variables from NREC on
// are not reconstructed (the cell values).
template <int NV, int LIM, int NREC = NV>
__device__ __forceinline__ void plm2(const f2* a, const f2* b, const f2* c, const f2* d, f2* pl, f2* pr) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v < NREC) {
      const f2 d1 = c[v] - b[v];
      pl[v] = b[v] + half_slope2<LIM>(b[v] - a[v], d1);
      pr[v] = c[v] - half_slope2<LIM>(d1, d[v] - c[v]);
    } else {
      pl[v] = b[v];
      pr[v] = c[v];
    }
  }
}

// Constants of the pair solvers, broadcast to both halves.
struct PairK {
  f2 zero, half, gamma, g1, ig1, m4, ch2, nhich, nhch;
  __device__ __forceinline__ explicit PairK(const PhysParamsT<float>& pp)
      : zero(bc2(0.0f)), half(bc2(0.5f)), gamma(bc2(pp.gamma)), g1(bc2(pp.g1)), ig1(bc2(pp.ig1)),
        m4(bc2(-4.0f)), ch2(bc2(pp.ch2)), nhich(bc2(-0.5f * pp.ich)), nhch(bc2(-0.5f * pp.ch)) {}
};

// x-direction pair forms of a physics module (none: the scalar solver serves both faces).
template <class P>
struct PairPhys {
  static constexpr bool OK = false;
};

template <>
struct PairPhys<HdPhys<float>> {
  static constexpr bool OK = true;
  static constexpr int NV = 5;
  // variable in slot v when the z axis takes the place of the x axis
  __host__ __device__ static constexpr int zrot(int v) { return v == 1 ? 3 : v == 3 ? 1 : v; }
  __device__ static __forceinline__ void interface(f2*, f2*, const PairK&) {}
  __device__ static __forceinline__ void prim2cons(const f2* p, f2* u, const PairK& k) {
    const f2 v2 = fma2(p[3], p[3], fma2(p[2], p[2], p[1] * p[1]));
    u[0] = p[0];
    u[1] = p[0] * p[1];
    u[2] = p[0] * p[2];
    u[3] = p[0] * p[3];
    u[4] = fma2(k.half * p[0], v2, p[4] * k.ig1);
  }
  __device__ static __forceinline__ void flux(const f2* p, const f2* u, f2* f, const PairK&) {
    const f2 vd = p[1];
    f[0] = u[0] * vd;
    f[1] = fma2(u[1], vd, p[4]);
    f[2] = u[2] * vd;
    f[3] = u[3] * vd;
    f[4] = vd * (u[4] + p[4]);
  }
  __device__ static __forceinline__ void lambdas(const f2* p, f2& lm, f2& lp, const PairK& k) {
    const f2 c = sqrt2(div2(k.gamma * p[4], p[0]));
    lm = p[1] - c;
    lp = p[1] + c;
  }
};

template <>
struct PairPhys<MhdPhys<float>> {
  static constexpr bool OK = true;
  static constexpr int NV = 9;
  __host__ __device__ static constexpr int zrot(int v) {
    return v == 1 ? 3 : v == 3 ? 1 : v == 5 ? 7 : v == 7 ? 5 : v;
  }
  // GLM face values B_x* and psi* (the scalar interface<0>)
  __device__ static __forceinline__ void interface(f2* pl, f2* pr, const PairK& k) {
    const f2 bl = pl[5], br = pr[5], sl = pl[8], sr = pr[8];
    const f2 bs = fma2(sr - sl, k.nhich, k.half * (bl + br));
    const f2 ss = fma2(br - bl, k.nhch, k.half * (sl + sr));
    pl[5] = bs;
    pr[5] = bs;
    pl[8] = ss;
    pr[8] = ss;
  }
  __device__ static __forceinline__ f2 b2(const f2* p) {
    return fma2(p[7], p[7], fma2(p[6], p[6], p[5] * p[5]));
  }
  __device__ static __forceinline__ void prim2cons(const f2* p, f2* u, const PairK& k) {
    const f2 v2 = fma2(p[3], p[3], fma2(p[2], p[2], p[1] * p[1]));
    u[0] = p[0];
    u[1] = p[0] * p[1];
    u[2] = p[0] * p[2];
    u[3] = p[0] * p[3];
    u[4] = fma2(k.half, fma2(p[0], v2, b2(p)), p[4] * k.ig1);
    u[5] = p[5];
    u[6] = p[6];
    u[7] = p[7];
    u[8] = p[8];
  }
  __device__ static __forceinline__ void flux(const f2* p, const f2* u, f2* f, const PairK& k) {
    const f2 vd = p[1], nbd = k.zero - p[5];
    const f2 ptot = fma2(b2(p), k.half, p[4]);
    const f2 vb = fma2(p[3], p[7], fma2(p[2], p[6], p[1] * p[5]));
    f[0] = u[0] * vd;
    f[1] = fma2(u[1], vd, fma2(p[5], nbd, ptot));
    f[2] = fma2(u[2], vd, p[6] * nbd);
    f[3] = fma2(u[3], vd, p[7] * nbd);
    f[4] = fma2(vd, u[4] + ptot, vb * nbd);
    f[5] = p[8];
    f[6] = fma2(vd, p[6], p[2] * nbd);
    f[7] = fma2(vd, p[7], p[3] * nbd);
    f[8] = k.ch2 * p[5];
  }
  __device__ static __forceinline__ void lambdas(const f2* p, f2& lm, f2& lp, const PairK& k) {
    const f2 ir = rcp2(p[0]);
    const f2 a2 = k.gamma * p[4] * ir;
    const f2 s = fma2(b2(p), ir, a2);
    const f2 bd2 = p[5] * p[5] * ir;
    const f2 disc = max2(fma2(s, s, k.m4 * a2 * bd2), k.zero);
    const f2 cf = sqrt2(k.half * (s + sqrt2(disc)));
    lm = p[1] - cf;
    lp = p[1] + cf;
  }
};

// The resistive MHD trait solves its faces like ideal MHD (the resistive terms are sources).
template <>
struct PairPhys<MhdResPhys<float>> : PairPhys<MhdPhys<float>> {};

// Frozen-field hydrodynamics (with or without conduction): the flux along the field b_x,
// whose face value is the mean of the two cells' b_x; b and q_par carry no dissipation
// (FROZEN, QV of the scalar trait, applied in the combinations below).
template <bool HTC>
struct PairPhys<FfhdPhysT<float, HTC>> {
  using S = FfhdPhysT<float, HTC>;
  static constexpr bool OK = true;
  static constexpr int NV = S::NV;
  static constexpr int B = S::BOFF;
  __host__ __device__ static constexpr int zrot(int v) { return v == B ? B + 2 : v == B + 2 ? B : v; }
  __device__ static __forceinline__ void interface(f2* pl, f2* pr, const PairK& k) {
    const f2 bf = k.half * (pl[B] + pr[B]);
    pl[B] = bf;
    pr[B] = bf;
  }
  __device__ static __forceinline__ void prim2cons(const f2* p, f2* u, const PairK& k) {
    u[0] = p[0];
    u[1] = p[0] * p[1];
    u[2] = fma2(k.half * p[0] * p[1], p[1], p[2] * k.ig1);
#pragma unroll
    for (int i = 3; i < NV; ++i) u[i] = p[i];
  }
  __device__ static __forceinline__ void flux(const f2* p, const f2* u, f2* f, const PairK& k) {
    const f2 b = p[B];
    const f2 vb = p[1] * b;
    f[0] = u[0] * vb;
    f[1] = fma2(u[1], vb, p[2] * b);
    if constexpr (HTC) f[2] = fma2(k.zero - p[3], b, (u[2] + p[2]) * vb);
    else f[2] = (u[2] + p[2]) * vb;
#pragma unroll
    for (int i = 3; i < NV; ++i) f[i] = k.zero;
    f[B] = b;
  }
  __device__ static __forceinline__ void lambdas(const f2* p, f2& lm, f2& lp, const PairK& k) {
    const f2 c = sqrt2(div2(k.gamma * p[2], p[0]));
    const f2 a = p[1] * p[B];
    const f2 w = c * abs2(p[B]);
    lm = a - w;
    lp = a + w;
  }
};

// HLL or TVDLF flux of the pair from reconstructed primitive states (modified in place).
template <class P, int FLUX>
__device__ __forceinline__ void riemann2(f2* pl, f2* pr, f2* f, const PairK& k) {
  using Q = PairPhys<P>;
  constexpr int NV = Q::NV;
  Q::interface(pl, pr, k);
  f2 ul[NV], ur[NV], fl[NV], fr[NV];
  Q::prim2cons(pl, ul, k);
  Q::prim2cons(pr, ur, k);
  Q::flux(pl, ul, fl, k);
  Q::flux(pr, ur, fr, k);
  f2 lml, lpl, lmr, lpr;
  Q::lambdas(pl, lml, lpl, k);
  Q::lambdas(pr, lmr, lpr, k);
  if constexpr (FLUX == FLUX_TVDLF) {
    const f2 c = max2(max2(abs2(lml), abs2(lpl)), max2(abs2(lmr), abs2(lpr)));
    const f2 nhc = k.zero - k.half * c;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (v >= P::FROZEN) f[v] = fl[v];   // frozen variables: exact flux, no dissipation
      else if (v == P::QV) f[v] = k.zero; // no flux term at all
      else f[v] = fma2(nhc, ur[v] - ul[v], k.half * (fl[v] + fr[v]));
    }
  } else {
    const f2 sl = min2(min2(lml, lmr), k.zero);
    const f2 sr = max2(max2(lpl, lpr), k.zero);
    const f2 inv = rcp2(sr - sl);
    const f2 wl = sr * inv, nwr = (k.zero - sl) * inv, wd = sl * sr * inv;
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = fma2(wd, ur[v] - ul[v], fma2(wl, fl[v], nwr * fr[v]));
  }
}

// z-face flux of one face with its left and right states as the pair: the states rotated so
// that z takes the place of x, the primitive-to-conserved map, physical fluxes and signal
// speeds of both sides in packed instructions, the HLL / TVDLF combination of the two halves
// at the end. pl and pr are the scalar face states (modified by the GLM face values).
template <class P, int FLUX>
__device__ __forceinline__ void riemann_z_lr(float* pl, float* pr, float* f, const PhysParamsT<float>& pp) {
  using Q = PairPhys<P>;
  constexpr int NV = Q::NV;
  P::template interface<2>(pl, pr, pp);
  const PairK k(pp);
  f2 q[NV], u[NV], fq[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) q[v] = f2_of(pl[Q::zrot(v)], pr[Q::zrot(v)]);
  Q::prim2cons(q, u, k);
  Q::flux(q, u, fq, k);
  f2 lm, lp;
  Q::lambdas(q, lm, lp, k);
  float lml, lmr, lpl, lpr;
  f2_split(lm, lml, lmr);
  f2_split(lp, lpl, lpr);
  f2 w, dw;   // F = w.x fl + w.y fr + dw.x ul + dw.y ur
  if constexpr (FLUX == FLUX_TVDLF) {
    const float c = fmaxf(fmaxf(fabsf(lml), fabsf(lpl)), fmaxf(fabsf(lmr), fabsf(lpr)));
    w = k.half;
    dw = f2_of(0.5f * c, -0.5f * c);
  } else {
    const float sl = fminf(fminf(lml, lmr), 0.0f);
    const float sr = fmaxf(fmaxf(lpl, lpr), 0.0f);
    const float inv = 1.0f / (sr - sl);
    const float wd = sl * sr * inv;
    w = f2_of(sr * inv, -(sl * inv));
    dw = f2_of(-wd, wd);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float a, b;
    if (FLUX == FLUX_TVDLF && v >= P::FROZEN) {          // frozen: the left flux exactly
      f2_split(fq[v], a, b);
      f[Q::zrot(v)] = a;
    } else if (FLUX == FLUX_TVDLF && v == P::QV) {       // no flux term
      f[Q::zrot(v)] = 0.0f;
    } else {
      f2_split(fma2(w, fq[v], dw * u[v]), a, b);
      f[Q::zrot(v)] = a + b;
    }
  }
}

}  // namespace agile
