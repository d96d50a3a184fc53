// mg_vertices.cuh -- device library of helicity wavefunctions and vertices.
//
// Helicity amplitudes in the spirit of HELAS (Murayama, Watanabe, Hagiwara
// 1992; cited by the paper in Sect. 1 for its Feynman-diagram method), written
// here from the Feynman rules in the Weyl (chiral) representation:
//   gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]],  psi = (psi_L, psi_R),
//   sigma^mu = (1, sigma^i), sigmabar^mu = (1, -sigma^i),  metric (+,-,-,-).
// A vector J gives Jslash = [[0, X], [Y, 0]] with
//   X = sigma.J    = [[J0-J3, -J1+iJ2], [-J1-iJ2, J0+J3]]
//   Y = sigmabar.J = [[J0+J3,  J1-iJ2], [ J1+iJ2, J0-J3]].
// Row spinors (ubar-like, 4 components) multiply from the left, column
// spinors (u/v-like) from the right.  Everything is templated on the real
// type R (double for the FP64 path, float for the mixed path).
#pragma once

#ifdef __CUDACC__
#include <cuda_runtime.h>
#endif
#include <math.h>
#include <stdint.h>

#include <type_traits>

// MG_VERTEX: inlining of the vertex routines (ffv_*, vvv_*, vvvv_*).  Inlined
// by default; a translation unit may define it as __noinline__, which turns a
// large process's straight-line helicity program into a sequence of calls to
// a few small routines that stay in the instruction cache (the inlined
// program is hundreds of KB of machine code, fetched again for every
// helicity).  Arguments are passed by value so that calls keep them in
// registers.
#ifndef MG_VERTEX
#define MG_VERTEX __forceinline__
#endif
// MG_VERTEX_AMP: the same for the amplitude routines (ffv_amp, vvv_amp, vvvv_amp)
#ifndef MG_VERTEX_AMP
#define MG_VERTEX_AMP MG_VERTEX
#endif
// MG_VERTEX_SMALL: the same for the shortest routines (vvvv_cur, vvvv_amp,
// ffv_vcur), whose call overhead is a larger share of their work
#ifndef MG_VERTEX_SMALL
#define MG_VERTEX_SMALL MG_VERTEX
#endif

namespace mg {

template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> C(R a, R b) {
  return cx<R>{a, b};
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) {
  return {-a.re, -a.im};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) {
  return {s * a.re, s * a.im};
}
template <typename R>
__device__ __forceinline__ cx<R> conj(cx<R> a) {
  return {a.re, -a.im};
}
// i * a
template <typename R>
__device__ __forceinline__ cx<R> mul_i(cx<R> a) {
  return {-a.im, a.re};
}
// a + b*c (complex)
template <typename R>
__device__ __forceinline__ cx<R> fma(cx<R> b, cx<R> c, cx<R> a) {
  return {a.re + b.re * c.re - b.im * c.im, a.im + b.re * c.im + b.im * c.re};
}
// a + s*b (real s)
template <typename R>
__device__ __forceinline__ cx<R> fma(R s, cx<R> b, cx<R> a) {
  return {a.re + s * b.re, a.im + s * b.im};
}

// MG_F32X2 (default 1): on sm_100 and later, the FP32 complex additions,
// subtractions and real-scalar products use the paired FP32 instructions
// (two lanes of FP32 in one instruction: the real and imaginary parts),
// halving their instruction count.  Same IEEE rounding per lane as the scalar
// forms.  Measured on gg -> t t~ g g mixed, 524288 events: 1.472e7 ->
// 1.527e7 MEs/s, the same error distribution.  MG_F32X2_MUL=1 also pairs the
// complex products, (ar, ar)(br, bi) + (-ai, ai)(bi, br), whose operands need
// their lanes swapped or duplicated.
#ifndef MG_F32X2
#define MG_F32X2 1
#endif
#ifndef MG_F32X2_MUL
#define MG_F32X2_MUL 0
#endif
#if MG_F32X2 && defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ float2 f2_of(cx<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ cx<float> cx_of(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ cx<float> operator+(cx<float> a, cx<float> b) {
  return cx_of(__fadd2_rn(f2_of(a), f2_of(b)));
}
__device__ __forceinline__ cx<float> operator-(cx<float> a, cx<float> b) {
  return cx_of(__fadd2_rn(f2_of(a), make_float2(-b.re, -b.im)));
}
__device__ __forceinline__ cx<float> operator*(float s, cx<float> a) {
  return cx_of(__fmul2_rn(make_float2(s, s), f2_of(a)));
}
__device__ __forceinline__ cx<float> fma(float s, cx<float> b, cx<float> a) {
  return cx_of(__ffma2_rn(make_float2(s, s), f2_of(b), f2_of(a)));
}
#if MG_F32X2_MUL
__device__ __forceinline__ cx<float> operator*(cx<float> a, cx<float> b) {
  const float2 t = __fmul2_rn(make_float2(a.re, a.re), f2_of(b));
  return cx_of(__ffma2_rn(make_float2(-a.im, a.im), make_float2(b.im, b.re), t));
}
__device__ __forceinline__ cx<float> fma(cx<float> b, cx<float> c, cx<float> a) {
  const float2 t = __ffma2_rn(make_float2(b.re, b.re), f2_of(c), f2_of(a));
  return cx_of(__ffma2_rn(make_float2(-b.im, b.im), make_float2(c.im, c.re), t));
}
#endif
#endif

template <typename R>
__device__ __forceinline__ R fmaf_t(R a, R b, R c) {
  return a * b + c;
}

template <typename R>
struct V4 {  // contravariant vector current
  cx<R> c[4];
};
template <typename R>
struct Sp {  // Weyl-basis 4-spinor (row or column)
  cx<R> c[4];
};
// a current kept in a V4-typed store slot and read back as a spinor (and back)
template <typename R>
__device__ __forceinline__ Sp<R> as_sp(const V4<R>& w) {
  Sp<R> s;
  for (int i = 0; i < 4; i++) s.c[i] = w.c[i];
  return s;
}
template <typename R>
__device__ __forceinline__ V4<R> as_v4(const Sp<R>& s) {
  V4<R> w;
  for (int i = 0; i < 4; i++) w.c[i] = s.c[i];
  return w;
}
template <typename R>
struct M4 {  // real 4-vector (a momentum), passed by value like V4 and Sp
  R v[4];
  __host__ __device__ constexpr R operator[](int i) const { return v[i]; }
};

// Minkowski products
template <typename R>
__device__ __forceinline__ cx<R> dot(const V4<R>& a, const V4<R>& b) {
  cx<R> s = a.c[0] * b.c[0];
  s = s - a.c[1] * b.c[1];
  s = s - a.c[2] * b.c[2];
  s = s - a.c[3] * b.c[3];
  return s;
}
template <typename R>
__device__ __forceinline__ cx<R> dot(const M4<R> k, const V4<R>& b) {
  return {k[0] * b.c[0].re - k[1] * b.c[1].re - k[2] * b.c[2].re - k[3] * b.c[3].re,
          k[0] * b.c[0].im - k[1] * b.c[1].im - k[2] * b.c[2].im - k[3] * b.c[3].im};
}

// ---------------------------------------------------------------------------
// external wavefunctions (per helicity, from per-event ingredients)
// ---------------------------------------------------------------------------

// Massless vector of helicity lam = +-1; e1s, e2s = e1/sqrt2, e2/sqrt2 with
// e1 = (cos th cos ph, cos th sin ph, -sin th), e2 = (-sin ph, cos ph, 0):
//   incoming eps = -lam e1s - i e2s,  outgoing eps* = -lam e1s + i e2s.
template <typename R>
__device__ __forceinline__ V4<R> ext_vector(const R e1s[3], const R e2s[3], R lam, bool outgoing) {
  V4<R> w;
  const R s = outgoing ? R(1) : R(-1);
  w.c[0] = {R(0), R(0)};
  for (int i = 0; i < 3; i++) w.c[i + 1] = {-lam * e1s[i], s * e2s[i]};
  return w;
}

// Two-component helicity eigenstates along phat: chi+ = (a, b), chi- = (-b*, a).
// Fermion ingredients per event: a (real), b (complex), om_m = sqrt(E-|p|),
// om_p = sqrt(E+|p|).
template <typename R>
struct FermIngr {
  R a, bre, bim, om_m, om_p;
};

template <typename R>
__device__ __forceinline__ void chi(const FermIngr<R>& f, int lam, cx<R>& c0, cx<R>& c1) {
  if (lam > 0) {
    c0 = {f.a, R(0)};
    c1 = {f.bre, f.bim};
  } else {
    c0 = {-f.bre, f.bim};
    c1 = {f.a, R(0)};
  }
}

// outgoing fermion: ubar(lam) = ( om_lam chi_lam^*, om_{-lam} chi_lam^* )
template <typename R>
__device__ __forceinline__ Sp<R> ext_ubar(const FermIngr<R>& f, int lam) {
  cx<R> c0, c1;
  chi(f, lam, c0, c1);
  const R wl = lam > 0 ? f.om_p : f.om_m;
  const R wm = lam > 0 ? f.om_m : f.om_p;
  Sp<R> s;
  s.c[0] = wl * conj(c0);
  s.c[1] = wl * conj(c1);
  s.c[2] = wm * conj(c0);
  s.c[3] = wm * conj(c1);
  return s;
}
// outgoing antifermion: v(lam) = ( om_lam chi_{-lam} ; -om_{-lam} chi_{-lam} )
template <typename R>
__device__ __forceinline__ Sp<R> ext_v(const FermIngr<R>& f, int lam) {
  cx<R> c0, c1;
  chi(f, -lam, c0, c1);
  const R wl = lam > 0 ? f.om_p : f.om_m;
  const R wm = lam > 0 ? f.om_m : f.om_p;
  Sp<R> s;
  s.c[0] = wl * c0;
  s.c[1] = wl * c1;
  s.c[2] = -wm * c0;
  s.c[3] = -wm * c1;
  return s;
}
// incoming fermion: u(lam) = ( om_{-lam} chi_lam ; om_lam chi_lam )
template <typename R>
__device__ __forceinline__ Sp<R> ext_u(const FermIngr<R>& f, int lam) {
  cx<R> c0, c1;
  chi(f, lam, c0, c1);
  const R wl = lam > 0 ? f.om_p : f.om_m;
  const R wm = lam > 0 ? f.om_m : f.om_p;
  Sp<R> s;
  s.c[0] = wm * c0;
  s.c[1] = wm * c1;
  s.c[2] = wl * c0;
  s.c[3] = wl * c1;
  return s;
}
// incoming antifermion: vbar(lam) = ( -om_{-lam} chi_{-lam}^*, om_lam chi_{-lam}^* )
template <typename R>
__device__ __forceinline__ Sp<R> ext_vbar(const FermIngr<R>& f, int lam) {
  cx<R> c0, c1;
  chi(f, -lam, c0, c1);
  const R wl = lam > 0 ? f.om_p : f.om_m;
  const R wm = lam > 0 ? f.om_m : f.om_p;
  Sp<R> s;
  s.c[0] = -wm * conj(c0);
  s.c[1] = -wm * conj(c1);
  s.c[2] = wl * conj(c0);
  s.c[3] = wl * conj(c1);
  return s;
}

// Per-event fermion ingredients in the set-up precision D (FP64, or FP32 in
// the all-float mode); stable forms: E - |p| = m^2/(E+|p|),
// |p| + pz = pT^2/(|p| - pz) for pz < 0.
template <typename D>
__device__ __forceinline__ void fermion_ingredients(const D p[4], D m, D out[5]) {
  const D pt2 = p[1] * p[1] + p[2] * p[2];
  const D P = sqrt(pt2 + p[3] * p[3]);
  const D E = p[0];
  const D om_p = sqrt(E + P);
  const D om_m = (m == D(0.0)) ? D(0.0) : sqrt(m * m / (E + P));
  const D s = (p[3] >= D(0.0)) ? (P + p[3]) : (pt2 / (P - p[3]));
  D a, bre, bim;
  if (s > D(0.0)) {
    a = sqrt(s / (D(2.0) * P));
    const D r = D(1.0) / sqrt(D(2.0) * P * s);
    bre = p[1] * r;
    bim = p[2] * r;
  } else {
    a = D(0.0);
    bre = D(1.0);
    bim = D(0.0);
  }
  out[0] = a;
  out[1] = bre;
  out[2] = bim;
  out[3] = om_m;
  out[4] = om_p;
}

// Per-event transverse basis e1/sqrt2, e2/sqrt2 of a massless vector (set-up
// precision D).
template <typename D>
__device__ __forceinline__ void vector_basis(const D k[4], D out[6]) {
  const D pt2 = k[1] * k[1] + k[2] * k[2];
  const D P = sqrt(pt2 + k[3] * k[3]);
  D cph, sph, cth, sth;
  if (pt2 > D(0.0)) {
    const D pt = sqrt(pt2);
    cph = k[1] / pt;
    sph = k[2] / pt;
    cth = k[3] / P;
    sth = pt / P;
  } else {
    cph = D(1.0);
    sph = D(0.0);
    cth = (k[3] >= D(0.0)) ? D(1.0) : -D(1.0);
    sth = D(0.0);
  }
  const D r = D(0.70710678118654752440);
  out[0] = r * cth * cph;
  out[1] = r * cth * sph;
  out[2] = -r * sth;
  out[3] = -r * sph;
  out[4] = r * cph;
  out[5] = D(0.0);
}

// Minkowski square of a signed sum of four-vectors minus m2,
//   (sum_n s_n v_n)^2 - m2,   s_n = +-1.
// In the FP64 path (R and D double) every component sum and square is carried
// as an unevaluated sum of two doubles (Knuth's error-free two-sum, and the
// product error from an FMA): the invariant of nearly collinear momenta, or of
// a nearly on-shell top, then keeps full relative precision instead of losing
// the digits of its cancellation.  Elsewhere it is the plain formula in D.
template <typename D>
__host__ __device__ __forceinline__ void two_sum(D a, D b, D& s, D& e) {
  s = a + b;
  const D bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
template <typename R, typename D, int N>
__device__ __forceinline__ D inv_mass2(const D* const (&v)[N], const D (&s)[N], D m2) {
  if constexpr (sizeof(R) == 8 && sizeof(D) == 8) {
    D hi = -m2, lo = D(0);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      D ch = s[0] * v[0][mu], cl = D(0);
#pragma unroll
      for (int k = 1; k < N; k++) {
        D e;
        two_sum(ch, s[k] * v[k][mu], ch, e);
        cl += e;
      }
      const D sq = ch * ch;
      const D sq_lo = ::fma(ch, ch, -sq) + D(2) * ch * cl;
      D e;
      if (mu == 0) {
        two_sum(hi, sq, hi, e);
        lo += e + sq_lo;
      } else {
        two_sum(hi, -sq, hi, e);
        lo += e - sq_lo;
      }
    }
    return hi + lo;
  } else {
    D c[4];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      c[mu] = s[0] * v[0][mu];
#pragma unroll
      for (int k = 1; k < N; k++) c[mu] = c[mu] + s[k] * v[k][mu];
    }
    return c[0] * c[0] - c[1] * c[1] - c[2] * c[2] - c[3] * c[3] - m2;
  }
}

// Same ingredients in the compute precision R, from a momentum in R: used by
// the FP32 path, which recomputes them per helicity instead of keeping them in
// shared memory (a few flops against tens of thousands per helicity).
template <typename R>
__device__ __forceinline__ FermIngr<R> fermion_ingredients_r(const R p[4], R m) {
  const R pt2 = p[1] * p[1] + p[2] * p[2];
  const R P = sqrt(pt2 + p[3] * p[3]);
  const R E = p[0];
  FermIngr<R> f;
  f.om_p = sqrt(E + P);
  f.om_m = (m == R(0)) ? R(0) : sqrt(m * m / (E + P));
  const R s = (p[3] >= R(0)) ? (P + p[3]) : (pt2 / (P - p[3]));
  if (s > R(0)) {
    f.a = sqrt(s / (R(2) * P));
    const R r = R(1) / sqrt(R(2) * P * s);
    f.bre = p[1] * r;
    f.bim = p[2] * r;
  } else {
    f.a = R(0);
    f.bre = R(1);
    f.bim = R(0);
  }
  return f;
}
template <typename R>
__device__ __forceinline__ void vector_basis_r(const R k[4], R e1[3], R e2[3]) {
  const R pt2 = k[1] * k[1] + k[2] * k[2];
  const R P = sqrt(pt2 + k[3] * k[3]);
  R cph, sph, cth, sth;
  if (pt2 > R(0)) {
    const R pt = sqrt(pt2);
    cph = k[1] / pt;
    sph = k[2] / pt;
    cth = k[3] / P;
    sth = pt / P;
  } else {
    cph = R(1);
    sph = R(0);
    cth = (k[3] >= R(0)) ? R(1) : R(-1);
    sth = R(0);
  }
  const R r = R(0.70710678118654752440);
  e1[0] = r * cth * cph;
  e1[1] = r * cth * sph;
  e1[2] = -r * sth;
  e2[0] = -r * sph;
  e2[1] = r * cph;
  e2[2] = R(0);
}

// ---------------------------------------------------------------------------
// vertices
// ---------------------------------------------------------------------------

// X = sigma.J, Y = sigmabar.J for a complex vector J (2x2 each, row-major)
template <typename R>
__device__ __forceinline__ void sigma_blocks(const V4<R>& J, cx<R> X[4], cx<R> Y[4]) {
  const cx<R> iJ2 = mul_i(J.c[2]);
  X[0] = J.c[0] - J.c[3];
  X[1] = iJ2 - J.c[1];
  X[2] = -(J.c[1] + iJ2);
  X[3] = J.c[0] + J.c[3];
  Y[0] = X[3];
  Y[1] = J.c[1] - iJ2;
  Y[2] = J.c[1] + iJ2;
  Y[3] = X[0];
}
// same for a real momentum Q
template <typename R>
__device__ __forceinline__ void sigma_blocks(const M4<R> Q, cx<R> X[4], cx<R> Y[4]) {
  X[0] = {Q[0] - Q[3], R(0)};
  X[1] = {-Q[1], Q[2]};
  X[2] = {-Q[1], -Q[2]};
  X[3] = {Q[0] + Q[3], R(0)};
  Y[0] = X[3];
  Y[1] = {Q[1], -Q[2]};
  Y[2] = {Q[1], Q[2]};
  Y[3] = X[0];
}
// row (r0, r1) times 2x2 M
template <typename R>
__device__ __forceinline__ void rowmul(cx<R> r0, cx<R> r1, const cx<R> M[4], cx<R>& o0, cx<R>& o1) {
  o0 = r0 * M[0] + r1 * M[2];
  o1 = r0 * M[1] + r1 * M[3];
}
// 2x2 M times column (c0, c1)
template <typename R>
__device__ __forceinline__ void mulcol(const cx<R> M[4], cx<R> c0, cx<R> c1, cx<R>& o0, cx<R>& o1) {
  o0 = M[0] * c0 + M[1] * c1;
  o1 = M[2] * c0 + M[3] * c1;
}

// Fbar Jslash F
template <typename R>
__device__ MG_VERTEX_AMP cx<R> ffv_amp(const Sp<R> a, const V4<R> J, const Sp<R> b) {
  cx<R> X[4], Y[4];
  sigma_blocks(J, X, Y);
  cx<R> t0, t1, u0, u1;
  mulcol(X, b.c[2], b.c[3], t0, t1);
  mulcol(Y, b.c[0], b.c[1], u0, u1);
  return a.c[0] * t0 + a.c[1] * t1 + a.c[2] * u0 + a.c[3] * u1;
}

// row current: coef * Fbar Jslash (Qslash + m)
template <typename R>
__device__ MG_VERTEX Sp<R> ffv_row(const Sp<R> a, const V4<R> J, const M4<R> Q, R m, cx<R> coef) {
  cx<R> X[4], Y[4], XQ[4], YQ[4];
  sigma_blocks(J, X, Y);
  sigma_blocks(Q, XQ, YQ);
  cx<R> rL0, rL1, rR0, rR1;
  rowmul(a.c[2], a.c[3], Y, rL0, rL1);  // (a_R Y, a_L X)
  rowmul(a.c[0], a.c[1], X, rR0, rR1);
  cx<R> s0, s1, t0, t1;
  rowmul(rR0, rR1, YQ, s0, s1);  // m rL + rR YQ
  rowmul(rL0, rL1, XQ, t0, t1);  // rL XQ + m rR
  Sp<R> o;
  o.c[0] = coef * fma(m, rL0, s0);
  o.c[1] = coef * fma(m, rL1, s1);
  o.c[2] = coef * fma(m, rR0, t0);
  o.c[3] = coef * fma(m, rR1, t1);
  return o;
}

// column current: coef * (qslash + m) Jslash F
template <typename R>
__device__ MG_VERTEX Sp<R> ffv_col(const V4<R> J, const Sp<R> b, const M4<R> q, R m, cx<R> coef) {
  cx<R> X[4], Y[4], XQ[4], YQ[4];
  sigma_blocks(J, X, Y);
  sigma_blocks(q, XQ, YQ);
  cx<R> cL0, cL1, cR0, cR1;
  mulcol(X, b.c[2], b.c[3], cL0, cL1);  // Jslash F = (X F_R, Y F_L)
  mulcol(Y, b.c[0], b.c[1], cR0, cR1);
  cx<R> s0, s1, t0, t1;
  mulcol(XQ, cR0, cR1, s0, s1);  // m cL + XQ cR
  mulcol(YQ, cL0, cL1, t0, t1);  // YQ cL + m cR
  Sp<R> o;
  o.c[0] = coef * fma(m, cL0, s0);
  o.c[1] = coef * fma(m, cL1, s1);
  o.c[2] = coef * fma(m, cR0, t0);
  o.c[3] = coef * fma(m, cR1, t1);
  return o;
}

// vector current coef * Fbar gamma^mu (cL PL + cR PR) F
template <typename R>
__device__ MG_VERTEX_SMALL V4<R> ffv_vcur(const Sp<R> a, const Sp<R> b, cx<R> coef, R cL = R(1), R cR = R(1)) {
  // upper: (a0,a1) sigma^mu (b2,b3) [right-handed F], lower: (a2,a3) sigmabar^mu (b0,b1)
  const cx<R> u02 = a.c[0] * b.c[2], u13 = a.c[1] * b.c[3], u03 = a.c[0] * b.c[3], u12 = a.c[1] * b.c[2];
  const cx<R> l20 = a.c[2] * b.c[0], l31 = a.c[3] * b.c[1], l21 = a.c[2] * b.c[1], l30 = a.c[3] * b.c[0];
  V4<R> g;
  g.c[0] = cR * (u02 + u13) + cL * (l20 + l31);
  g.c[1] = cR * (u03 + u12) - cL * (l21 + l30);
  g.c[2] = cR * mul_i(u12 - u03) + cL * mul_i(l21 - l30);
  g.c[3] = cR * (u02 - u13) - cL * (l20 - l31);
  for (int mu = 0; mu < 4; mu++) g.c[mu] = coef * g.c[mu];
  return g;
}

// three-gluon current: c * V3(kx, Jx, ky, Jy),
//   V3 = (Jx.Jy)(kx-ky) + Jy (2ky+kx).Jx - Jx (2kx+ky).Jy
template <typename R>
__device__ MG_VERTEX V4<R> vvv_cur(const M4<R> kx, const V4<R> Jx, const M4<R> ky, const V4<R> Jy, R c) {
  M4<R> a, b;
  for (int mu = 0; mu < 4; mu++) {
    a.v[mu] = R(2) * ky[mu] + kx[mu];
    b.v[mu] = R(2) * kx[mu] + ky[mu];
  }
  const cx<R> xy = dot(Jx, Jy);
  const cx<R> ax = dot(a, Jx);
  const cx<R> by = dot(b, Jy);
  V4<R> o;
  for (int mu = 0; mu < 4; mu++) {
    cx<R> t = (kx[mu] - ky[mu]) * xy;
    t = t + Jy.c[mu] * ax;
    t = t - Jx.c[mu] * by;
    o.c[mu] = c * t;
  }
  return o;
}
// amplitude: c * V3(kx, Jx, ky, Jy) . G
template <typename R>
__device__ MG_VERTEX_AMP cx<R> vvv_amp(const M4<R> kx, const V4<R> Jx, const M4<R> ky, const V4<R> Jy,
                                         const V4<R> G, R c) {
  M4<R> a, b, d;
  for (int mu = 0; mu < 4; mu++) {
    a.v[mu] = R(2) * ky[mu] + kx[mu];
    b.v[mu] = R(2) * kx[mu] + ky[mu];
    d.v[mu] = kx[mu] - ky[mu];
  }
  const cx<R> xy = dot(Jx, Jy);
  const cx<R> t = xy * dot(d, G) + dot(Jy, G) * dot(a, Jx) - dot(Jx, G) * dot(b, Jy);
  return c * t;
}

// four-gluon Lorentz structures for the three colour branches
//   br 0: (X.Z) Y - (Y.Z) X     br 1: (X.Y) Z - (Y.Z) X     br 2: (X.Y) Z - (X.Z) Y
template <int BR, typename R>
__device__ MG_VERTEX_SMALL V4<R> vvvv_cur(const V4<R> X, const V4<R> Y, const V4<R> Z, R c) {
  V4<R> o;
  if (BR == 0) {
    const cx<R> xz = dot(X, Z), yz = dot(Y, Z);
    for (int mu = 0; mu < 4; mu++) o.c[mu] = c * (xz * Y.c[mu] - yz * X.c[mu]);
  } else if (BR == 1) {
    const cx<R> xy = dot(X, Y), yz = dot(Y, Z);
    for (int mu = 0; mu < 4; mu++) o.c[mu] = c * (xy * Z.c[mu] - yz * X.c[mu]);
  } else {
    const cx<R> xy = dot(X, Y), xz = dot(X, Z);
    for (int mu = 0; mu < 4; mu++) o.c[mu] = c * (xy * Z.c[mu] - xz * Y.c[mu]);
  }
  return o;
}
template <int BR, typename R>
__device__ MG_VERTEX_SMALL cx<R> vvvv_amp(const V4<R> X, const V4<R> Y, const V4<R> Z, const V4<R> G, R c) {
  cx<R> t;
  if (BR == 0) t = dot(X, Z) * dot(Y, G) - dot(Y, Z) * dot(X, G);
  else if (BR == 1) t = dot(X, Y) * dot(Z, G) - dot(Y, Z) * dot(X, G);
  else t = dot(X, Y) * dot(Z, G) - dot(X, Z) * dot(Y, G);
  return c * t;
}

}  // namespace mg
