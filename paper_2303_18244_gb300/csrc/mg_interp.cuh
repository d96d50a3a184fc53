// mg_interp.cuh -- table-driven evaluation of the per-helicity diagram program.
//
// For the largest process (1240 diagrams, 1890 amplitude terms per helicity)
// straight-line code does not compile in reasonable time, so the generator
// emits the same evaluation plan -- the same currents, amplitudes, colour
// coefficients and emission order -- as a table of op records, and this
// interpreter runs it with warp-uniform control flow (every thread of the CTA
// executes the same op sequence on its own event).  Off-shell currents live in
// a per-thread store W whose slots the generator assigns by liveness.
//
// Op record f[0..7] (int32), f[0] = type:
//   OP_VVV   out=f1 a=f2 b=f3 maskA=f4 maskB=f5 cg=f6    three-gluon current
//   OP_VVVV  out=f1 a=f2 b=f3 c=f4 br=f5 cg=f6           four-gluon current (colour branch br)
//   OP_ROW   out=f1 prev=f2 g=f3 mask=f4 cf=f5           top current, t side (Q = p_t - K_mask)
//   OP_COL   out=f1 g=f2 next=f3 mask=f4 cf=f5           top current, t~ side (q = K_mask - p_tbar)
//   OP_GTT   out=f1 ubar=f2 v=f3 cgtt=f4                 G = (i g / P^2) ubar gamma v
//   OP_AF    row=f1 g=f2 col=f3 jl=f6 njl=f7             amplitude (i g) Fbar Jslash F
//   OP_A3    a=f1 b=f2 maskA=f3 maskB=f4 gtt=f5 jl=f6 njl=f7   amplitude -g V3(a,b).G
//   OP_A4    a=f1 b=f2 c=f3 br=f4 gtt=f5 jl=f6 njl=f7          amplitude +-g^2 L_br(a,b,c).G
// cg, cf, cgtt: slab offsets of the per-event propagator coefficients
// (cf: complex, two slots).  Amplitudes come grouped by colour pattern (the
// same flows with the same coefficients up to one overall sign): bit 8 of the
// type word gives the amplitude's sign relative to its pattern (set: +1), the
// amplitudes are summed in a register, and the last one of a group carries the
// pattern's colour list jl/njl (njl = 0 on the others), whose entries are
// (flow << 1) | (coefficient is -1).  P provides NG, koff(i) (slab offset of
// gluon i's incoming momentum), PT and PTB (slab offsets of p_t and p_tbar).
#pragma once

#include "mg_vertices.cuh"

namespace mg {

enum : int { OP_VVV = 1, OP_VVVV = 2, OP_ROW = 3, OP_COL = 4, OP_GTT = 5, OP_AF = 6, OP_A3 = 7, OP_A4 = 8 };

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

// K = sum of the incoming gluon momenta in mask: precomputed per event in the
// FP32 slab (P::KBASE + 4 (mask - 1)), summed from gluon i's momentum at slab
// offset P::koff(i) in FP64
template <class P, typename R>
__device__ __forceinline__ void ksum(const R* __restrict__ ev, int es, int mask, R K[4]) {
  if constexpr (sizeof(R) == 4 && P::KBASE > 0) {
    if (mask == 0) {
      K[0] = K[1] = K[2] = K[3] = R(0);
      return;
    }
    const int o = P::KBASE + 4 * (mask - 1);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) K[mu] = ev[(o + mu) * es];
  } else {
    K[0] = K[1] = K[2] = K[3] = R(0);
#pragma unroll
    for (int i = 0; i < P::NG; i++)
      if (mask & (1 << i))
#pragma unroll
        for (int mu = 0; mu < 4; mu++) K[mu] = K[mu] + ev[(P::koff(i) + mu) * es];
  }
}

template <typename R>
__device__ __forceinline__ void add_colour(const short* __restrict__ jl, int j0, int n, cx<R> a,
                                           cx<R>* __restrict__ jamp, int js) {
#pragma unroll 1
  for (int j = j0; j < j0 + n; j++) {
    const int e = __ldg(jl + j);
    cx<R>& t = jamp[(e >> 1) * js];
    t = (e & 1) ? t - a : t + a;
  }
}

// Run the op table for one helicity.  W holds the external wavefunctions in
// their slots on entry; jamp (stride js) must be zero.
template <class P, typename R>
__device__ __forceinline__ void run_program(const int4* __restrict__ ops, int nops, const short* __restrict__ jl,
                                            const R* __restrict__ ev, int es, R g, R mt, V4<R>* W,
                                            cx<R>* __restrict__ jamp, int js) {
#define EV(k) ev[(k) * es]
  cx<R> pacc = {R(0), R(0)};  // running sum of the current colour pattern's amplitudes
#pragma unroll 1
  for (int i = 0; i < nops; i++) {
    const int4 a = __ldg(ops + 2 * i);
    const int4 b = __ldg(ops + 2 * i + 1);
    // a = (type | sign << 8, f1, f2, f3), b = (f4, f5, f6, f7)
    const int type = a.x & 0xff;
    const bool plus = (a.x >> 8) & 1;
    cx<R> amp = {R(0), R(0)};
    bool is_amp = false;
    switch (type) {
      case OP_VVV: {
        R kx[4], ky[4];
        ksum<P, R>(ev, es, b.x, kx);
        ksum<P, R>(ev, es, b.y, ky);
        W[a.y] = vvv_cur<R>(kx, W[a.z], ky, W[a.w], EV(b.z));
        break;
      }
      case OP_VVVV: {
        const R c = EV(b.z);
        if (b.y == 0) W[a.y] = vvvv_cur<0, R>(W[a.z], W[a.w], W[b.x], -g * c);
        else if (b.y == 1) W[a.y] = vvvv_cur<1, R>(W[a.z], W[a.w], W[b.x], -g * c);
        else W[a.y] = vvvv_cur<2, R>(W[a.z], W[a.w], W[b.x], g * c);
        break;
      }
      case OP_ROW: {
        R K[4], Q[4];
        ksum<P, R>(ev, es, b.x, K);
        for (int mu = 0; mu < 4; mu++) Q[mu] = EV(P::PT + mu) - K[mu];
        W[a.y] = as_v4(ffv_row<R>(as_sp(W[a.z]), W[a.w], Q, mt, cx<R>{EV(b.y), EV(b.y + 1)}));
        break;
      }
      case OP_COL: {
        R K[4], q[4];
        ksum<P, R>(ev, es, b.x, K);
        for (int mu = 0; mu < 4; mu++) q[mu] = K[mu] - EV(P::PTB + mu);
        W[a.y] = as_v4(ffv_col<R>(W[a.z], as_sp(W[a.w]), q, mt, cx<R>{EV(b.y), EV(b.y + 1)}));
        break;
      }
      case OP_GTT:
        W[a.y] = ffv_vcur<R>(as_sp(W[a.z]), as_sp(W[a.w]), cx<R>{R(0), EV(b.x)});
        break;
      case OP_AF:
        amp = mul_i(g * ffv_amp<R>(as_sp(W[a.y]), W[a.z], as_sp(W[a.w])));
        is_amp = true;
        break;
      case OP_A3: {
        R kx[4], ky[4];
        ksum<P, R>(ev, es, a.w, kx);
        ksum<P, R>(ev, es, b.x, ky);
        amp = vvv_amp<R>(kx, W[a.y], ky, W[a.z], W[b.y], -g);
        is_amp = true;
        break;
      }
      case OP_A4:
        if (b.x == 0) amp = vvvv_amp<0, R>(W[a.y], W[a.z], W[a.w], W[b.y], g * g);
        else if (b.x == 1) amp = vvvv_amp<1, R>(W[a.y], W[a.z], W[a.w], W[b.y], g * g);
        else amp = vvvv_amp<2, R>(W[a.y], W[a.z], W[a.w], W[b.y], -g * g);
        is_amp = true;
        break;
      default:
        break;
    }
    if (is_amp) {
      pacc = plus ? pacc + amp : pacc - amp;
      if (b.w > 0) {
        add_colour<R>(jl, b.z, b.w, pacc, jamp, js);
        pacc = cx<R>{R(0), R(0)};
      }
    }
  }
#undef EV
}

}  // namespace mg
