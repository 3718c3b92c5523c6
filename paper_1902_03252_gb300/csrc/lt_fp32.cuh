// FP32 per-potential deflections with their running error-bound terms, shared
// by the deflection kernel and the allocation-free deflection entry point.
#pragma once

#include "lt_internal.cuh"

namespace lt {

// The node set of one thread: NPT nodes of one grid column, at X and at the
// rows Y[0..NPT-1].  The translation dx = X - c_x and its products with the
// rotation coefficients are formed once per potential and shared by the NPT
// nodes; each node then needs dy = Y - c_y and one fma per rotated component.
// Which of the two products of a rotated component is rounded separately
// (dx c or dy s) does not change its error bound: both are at most the
// distance times the coefficient.

// Blocked summation over the potentials (Higham, "Accuracy and Stability of
// Numerical Algorithms", ch. 4): the potentials' terms are summed into a
// partial sum per group of kSumGroup potentials, and each group's partial sum
// is added to the node's total.  A term's rounding is then bounded by the
// partial sum it joins (per potential, in the functions below) and a group's
// by the total once per group, instead of every term by the running total:
// with n potentials the running-sum part of the bound shrinks from about
// n |alpha| to about (kSumGroup + n / kSumGroup) |alpha|, and so does the
// error itself.  (kSumGroup and the staging chunk kChunk32 are defined with
// the records in lt_internal.cuh: k_prep derives the coarse bound from them.)

// The bound's terms are non-negative and are accumulated with round-to-
// nearest FMAs (directed rounding measured slower on the FMA pipes): a float
// sum of non-negative terms through k roundings is at least the exact sum
// times 1 - gamma(k), which node_bound covers with its factor
// 1 + (6 n_pot + 64) u (at most five roundings per potential, two per
// group); the terms themselves are derived in k_prep.
//
// Two forms of the bound (template flag TIGHT):
//  * tight: per node and potential the term P / d, the evaluation terms
//    Gx |gx| + Gy |gy| of the PIEMD and the accumulation terms 2 (|PX| + |PY|)
//    per step and 2 (|AX| + |AY|) per group;
//  * coarse: only P / d per node and potential; the evaluation and
//    accumulation terms are replaced by their largest values over the plane,
//    summed once per sample in k_prep (Seg32::c_tot).  Valid everywhere and
//    about twice the tight bound on cluster lenses; four instructions per
//    node and potential cheaper.  The triangle search certifies what it can
//    with the coarse bound, and the resolution re-evaluates the few
//    undecided nodes with the tight one (k_res_tight32).

// Coefficient P of the per-node term P / d of one potential (units of u) on a
// grid whose largest |node coordinate| is theta1: errP0 W, W = theta1 + |cx| +
// |cy|, and for the PIEMD the factor of the segment between the exact and the
// rounded node: 1 / (1 - x) for x = 14.18 (1 + 3u) u W / (q a) <= 1/2, else
// 10.03 max(1, x) (see k_prep).  Rounded up throughout; strictly positive, so
// that P times an infinite 1/d (a node on an SIS/SIE centre) is +inf, never
// NaN, even for a zero-mass potential.
__device__ __forceinline__ float stage_p32(const Pot32& r, bool piemd, float theta1) {
  const float W = __fadd_ru(__fadd_ru(theta1, fabsf(r.f[0].x)), fabsf(r.f[0].y));
  float P = __fmul_ru(r.f[4].x, W);
  if (piemd) {
    const float qa = __fsqrt_rd(__fmul_rd(r.f[2].x, r.f[2].z));  // q a, rounded down
    const float xk = __fdiv_ru(__fmul_ru(8.4521e-7f, W), qa);   // 14.18 (1 + 3u) u, rounded up
    P = xk <= 0.5f ? __fdiv_ru(P, __fsub_rd(1.0f, xk)) : __fmul_ru(P, __fmul_ru(10.03f, fmaxf(1.0f, xk)));
  }
  return __fadd_ru(P, 1e-30f);
}

// ------------------------------------------------ explicit FP32 operations
// The per-node arithmetic below is written once for a node lane type V:
// float (one node) or F2 (two nodes of one thread, in the paired FP32
// instructions add/sub/mul/fma .f32x2 of sm_100 and later, which do two
// lanes' operations in one issue slot at the FP32 pipe's lane rate).  Every
// operation is explicit (inline PTX, round to nearest, flush to zero), so a
// node gets the same operations, roundings and results whether it sits in
// a pair or alone: a thread's nodes are paired as far as they go, and an odd
// last node runs the same code with V = float.  No operation is contracted
// or reassociated by the compiler.  (Per-thread, per-potential scalars such
// as the column's translation are ordinary float expressions; they do not
// depend on the pairing.)
struct F2 {
  unsigned long long v;
};
__device__ __forceinline__ F2 f2_pack(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(F2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}

__device__ __forceinline__ float xfma(float a, float b, float c) {
  float d;
  asm("fma.rn.ftz.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float xmul(float a, float b) {
  float d;
  asm("mul.rn.ftz.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float xadd(float a, float b) {
  float d;
  asm("add.rn.ftz.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float xsub(float a, float b) {
  float d;
  asm("sub.rn.ftz.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ F2 xfma(F2 a, F2 b, F2 c) {
  F2 d;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
__device__ __forceinline__ F2 xmul(F2 a, F2 b) {
  F2 d;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ F2 xadd(F2 a, F2 b) {
  F2 d;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ F2 xsub(F2 a, F2 b) {
  F2 d;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}

// lane access, broadcast and lane-wise maps (the MUFU approximations, the
// rare range-reduced special functions, absolute values, selects)
template <class V> struct Lanes;
template <> struct Lanes<float> {
  static constexpr int n = 1;
  __device__ __forceinline__ static float bc(float a) { return a; }
  __device__ __forceinline__ static float get(float a, int) { return a; }
};
template <> struct Lanes<F2> {
  static constexpr int n = 2;
  __device__ __forceinline__ static F2 bc(float a) { return f2_pack(a, a); }
  __device__ __forceinline__ static float get(F2 a, int l) {
    float lo, hi;
    f2_unpack(a, lo, hi);
    return l ? hi : lo;
  }
};
template <class V, class Fn>
__device__ __forceinline__ V lanewise(V a, Fn fn) {
  if constexpr (Lanes<V>::n == 1) {
    return fn(a);
  } else {
    float a0, a1;
    f2_unpack(a, a0, a1);
    return f2_pack(fn(a0), fn(a1));
  }
}
template <class V> __device__ __forceinline__ V xrsqrt(V a) { return lanewise(a, rsqrt_approx32); }
template <class V> __device__ __forceinline__ V xsqrt(V a) { return lanewise(a, sqrt_approx32); }
template <class V> __device__ __forceinline__ V xrcp(V a) { return lanewise(a, rcp_approx32); }
template <class V> __device__ __forceinline__ V xabs(V a) {
  return lanewise(a, [](float x) { return fabsf(x); });
}
// per lane: a where x > thr, else b
template <class V> __device__ __forceinline__ V xselect_gt(V x, float thr, V a, V b) {
  if constexpr (Lanes<V>::n == 1) {
    return x > thr ? a : b;
  } else {
    float x0, x1, a0, a1, b0, b1;
    f2_unpack(x, x0, x1);
    f2_unpack(a, a0, a1);
    f2_unpack(b, b0, b1);
    return f2_pack(x0 > thr ? a0 : b0, x1 > thr ? a1 : b1);
  }
}

// r on lanes where R2 > 0, else 0 (the deflection is zero at an SIS/SIE centre)
template <class V> __device__ __forceinline__ V xpos_or_zero(V R2, V r) {
  return xselect_gt(R2, 0.0f, r, Lanes<V>::bc(0.0f));
}

// The polynomials of atanc_poly32 / atanhc_poly32 (the same coefficients, by
// Horner's rule), on node lanes.
template <class V> __device__ __forceinline__ V atanc_poly(V u) {
  typedef Lanes<V> L;
  V p = L::bc(7.685306482e-03f);
  p = xfma(p, u, L::bc(-3.647336364e-02f));
  p = xfma(p, u, L::bc(8.325644583e-02f));
  p = xfma(p, u, L::bc(-1.345480382e-01f));
  p = xfma(p, u, L::bc(1.987373084e-01f));
  p = xfma(p, u, L::bc(-3.332583010e-01f));
  return xfma(p, u, L::bc(9.999992251e-01f));
}
template <class V> __device__ __forceinline__ V atanhc_poly(V u) {
  typedef Lanes<V> L;
  V p = L::bc(1.953562647e-01f);
  p = xfma(p, u, L::bc(1.221839786e-01f));
  p = xfma(p, u, L::bc(2.019458860e-01f));
  p = xfma(p, u, L::bc(3.332709372e-01f));
  return xfma(p, u, L::bc(1.000000358e+00f));
}

// The range-reduced forms of atanc_reduced32 / atanhc_reduced32 on node
// lanes, with the same operations in the same order (so every node gets the
// values of the scalar functions): atan(t)/t for t2 > 1 and atanh(t)/t for
// t2 > 1/4.
template <class V> __device__ __forceinline__ V atanc_reduced(V t2) {
  typedef Lanes<V> L;
  const V r = xrsqrt(t2);
  const V inv = xmul(r, r);
  const V pinv = xmul(atanc_poly(inv), inv);
  return xfma(L::bc(1.57079633f), r, xmul(L::bc(-1.0f), pinv));  // pi/2 r - p inv
}
template <class V> __device__ __forceinline__ V atanhc_reduced(V t2) {
  typedef Lanes<V> L;
  const V tc = lanewise(t2, [](float x) { return fminf(x, 0.99999988f); });
  const V r = xrsqrt(tc);
  const V num = xfma(tc, r, L::bc(1.0f));
  const V den = xfma(xmul(L::bc(-1.0f), tc), r, L::bc(1.0f));
  const V ratio = xmul(num, xrcp(den));
  return xmul(xmul(lanewise(ratio, lg2_approx32), L::bc(0.5f * 0.693147181f)), r);
}

// The largest of the NV node lanes' values (three-input max of sm_100 and
// later).  Used only to test whether any lane exceeds a threshold; a NaN lane
// never counts as exceeding it, as with x > thr.
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
template <class V, int NV> __device__ __forceinline__ float lanes_max(const V* v) {
  if constexpr (Lanes<V>::n == 1) {
    float m = v[0];
#pragma unroll
    for (int i = 1; i < NV; ++i) m = fmaxf(m, v[i]);
    return m;
  } else {
    float m, a, b;
    f2_unpack(v[0], m, a);
    m = fmaxf(m, a);
#pragma unroll
    for (int i = 1; i < NV; ++i) {
      f2_unpack(v[i], a, b);
      m = max3f(m, a, b);
    }
    return m;
  }
}

// Add a group's partial sums to the totals (one rounding per component,
// bounded by the new total) and clear them.
template <class V, int NV, bool TIGHT>
__device__ __forceinline__ void flush_group(V* AX, V* AY, V* PX, V* PY, V* ER) {
  typedef Lanes<V> L;
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    AX[m] = xadd(AX[m], PX[m]);
    AY[m] = xadd(AY[m], PY[m]);
    if (TIGHT) ER[m] = xfma(L::bc(2.0f), xadd(xabs(AX[m]), xabs(AY[m])), ER[m]);
    PX[m] = L::bc(0.0f);
    PY[m] = L::bc(0.0f);
  }
}

// One SIS: alpha += b0 (theta - c)/R (zero at the centre).  err accumulates in
// units of the FP32 unit roundoff.  In this and the two functions below, AX
// and AY are a group's partial sums (flush_group), NV node lanes of type V
// at the column X and the rows Y[].
template <class V, int NV, bool TIGHT>
__device__ __forceinline__ void sis32_nodes(const float4* f, float P, float X, const V* Y,
                                            V* AX, V* AY, V* ER) {
  typedef Lanes<V> L;
  const float dx = X - f[0].x;
  const float dx2 = dx * dx;
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    const V dy = xsub(Y[m], L::bc(f[0].y));
    const V R2 = xfma(dy, dy, L::bc(dx2));
    // rr is +inf on the centre: there the direction of alpha is undefined and
    // the bound term P rr makes the node's bound infinite (never certified)
    const V rr = xrsqrt(R2);
    const V ri = xpos_or_zero(R2, rr);
    const V g = xmul(L::bc(f[0].z), ri);
    AX[m] = xfma(g, L::bc(dx), AX[m]);
    AY[m] = xfma(g, dy, AY[m]);
    ER[m] = xfma(L::bc(P), rr, ER[m]);
    if (TIGHT) ER[m] = xfma(L::bc(2.0f), xadd(xabs(AX[m]), xabs(AY[m])), ER[m]);
  }
}

// One SIE (Algorithm 1), with the axis weights folded into the rotation:
// u = sqrt(1-eps) x', v = sqrt(1+eps) y' (so R^2 = u^2 + v^2), and the
// rotation back applied to (b0 sqrt(1-eps) u, b0 sqrt(1+eps) v) before the
// division by R:
//   alpha_x += (b0 sqrt(1-eps) c u - b0 sqrt(1+eps) s v) / R,
//   alpha_y += (b0 sqrt(1+eps) c v + b0 sqrt(1-eps) s u) / R,
// which is Algorithm 1's (1 -+ eps) b0 x'/R rotated by -phi.  Record:
// f[0] = {cx, cy, sqrt(1-eps) c, sqrt(1-eps) s},
// f[1] = {sqrt(1+eps) c, sqrt(1+eps) s, b0 sqrt(1-eps) c, b0 sqrt(1+eps) s},
// f[2] = {b0 sqrt(1+eps) c, b0 sqrt(1-eps) s, 0, 0}.
template <class V, int NV, bool TIGHT>
__device__ __forceinline__ void sie32_nodes(const float4* f, float P, float X, const V* Y,
                                            V* AX, V* AY, V* ER) {
  typedef Lanes<V> L;
  const float dx = X - f[0].x;
  const float dxu = dx * f[0].z, ndxv = -dx * f[1].y;
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    const V dy = xsub(Y[m], L::bc(f[0].y));
    const V u = xfma(dy, L::bc(f[0].w), L::bc(dxu));
    const V v = xfma(dy, L::bc(f[1].x), L::bc(ndxv));
    const V R2 = xfma(u, u, xmul(v, v));
    const V rr = xrsqrt(R2);  // +inf on the centre: an infinite bound there
    const V ri = xpos_or_zero(R2, rr);
    const V t1 = xfma(L::bc(f[1].z), u, xmul(L::bc(-f[1].w), v));
    const V t2 = xfma(L::bc(f[2].x), v, xmul(L::bc(f[2].y), u));
    AX[m] = xfma(ri, t1, AX[m]);
    AY[m] = xfma(ri, t2, AY[m]);
    ER[m] = xfma(L::bc(P), rr, ER[m]);
    if (TIGHT) ER[m] = xfma(L::bc(2.0f), xadd(xabs(AX[m]), xabs(AY[m])), ER[m]);
  }
}

// One PIEMD (dPIE) in difference form.  With psi_w = sqrt(q^2(w^2+x'^2)+y'^2),
// F(a) - F(s) is evaluated as one atan / atanh of
//   tx = x' ds_x / ((psi_a+a)(psi_s+s) + k^2 x'^2),
//   ty = y' ds_y / ((psi_a+q^2 a)(psi_s+q^2 s) - k^2 y'^2),
// ds_x = (s-a)(1 + q^2 (s+a)/(psi_a+psi_s)), ds_y = q^2 (s-a)(1 + (s+a)/(psi_a+psi_s))
// (atan u - atan v = atan((u-v)/(1+uv)), atanh likewise, and
// psi_s - psi_a = q^2 (s^2-a^2)/(psi_a+psi_s)), which avoids the cancellation
// of the two cored terms and halves the transcendental work.  psi_a enters
// the sums as the fused psi_a^2 rsqrt(psi_a^2) + z (one rounding each).
//
// The range tests of the two special functions are one branch per thread,
// potential and function: both polynomials are evaluated on the unreduced
// arguments for every node (out of range the value may overflow; it is
// replaced), and where any of the thread's nodes is outside a range (atan:
// t2 > 1, about 1 % of a warp's potentials on cluster lenses; atanh:
// t2 > 0.25, about 15 %) the reduced form is evaluated for all its nodes and
// selected per node.  Every node gets exactly the values and roundings of
// atanc_sq32 / atanhc_sq32; the per-thread tests keep the branches out of
// most of the issue stream.
template <class V, int NV, bool TIGHT>
__device__ __forceinline__ void piemd32_nodes(const float4* f, float P, float X, const V* Y,
                                              V* AX, V* AY, V* ER) {
  typedef Lanes<V> L;
  const float dx = X - f[0].x;
  const float dxc = dx * f[0].z, ndxs = -dx * f[0].w;
  V tx[NV], ty[NV], ux[NV], uy[NV], ra[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    const V dy = xsub(Y[m], L::bc(f[0].y));
    const V xp = xfma(dy, L::bc(f[0].w), L::bc(dxc));
    const V yp = xfma(dy, L::bc(f[0].z), L::bc(ndxs));
    const V x2 = xmul(xp, xp), y2 = xmul(yp, yp);
    const V t = xfma(L::bc(f[1].x), x2, y2);
    const V pa2 = xadd(t, L::bc(f[1].y)), ps2 = xadd(t, L::bc(f[1].z));
    ra[m] = xrsqrt(pa2);
    // psi_s in one MUFU operation.  Over every float mantissa (four binades
    // checked exhaustively on GB300) sqrt.approx.ftz errs by at most 1.68 u
    // against the rounded sqrt, below the 2.71 u of ps2 * rsqrt(ps2) that the
    // error bound was derived for; psi_a keeps that form, as 1/psi_a is needed.
    const V ps = xsqrt(ps2);
    const V iD = xrcp(xfma(pa2, ra[m], ps));
    const V dsx = xfma(L::bc(f[3].y), iD, L::bc(f[3].x));
    const V dsy = xfma(L::bc(f[3].y), iD, L::bc(f[3].z));
    const V px = xmul(xfma(pa2, ra[m], L::bc(f[2].x)), xadd(ps, L::bc(f[2].y)));
    const V py = xmul(xfma(pa2, ra[m], L::bc(f[2].z)), xadd(ps, L::bc(f[2].w)));
    const V denx = xfma(L::bc(f[1].w), x2, px);
    const V deny = xfma(L::bc(-f[1].w), y2, py);
    // the ds coefficients carry sig = sqrt(k2): these are sig tx, sig ty
    tx[m] = xmul(xmul(xp, dsx), xrcp(denx));
    ty[m] = xmul(xmul(yp, dsy), xrcp(deny));
    ux[m] = xmul(tx[m], tx[m]);
    uy[m] = xmul(ty[m], ty[m]);
    ER[m] = xfma(L::bc(P), ra[m], ER[m]);
  }
  V px_[NV], py_[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    // the polynomials of atanc_sq32 / atanhc_sq32 on the unreduced arguments
    px_[m] = atanc_poly(ux[m]);
    py_[m] = atanhc_poly(uy[m]);
  }
  // every node's reduced form, kept where its argument is out of range: one
  // select per node, each pair rebuilt whole (no register of a pair is
  // written under a branch)
  if (lanes_max<V, NV>(ux) > 1.0f) {
#pragma unroll
    for (int m = 0; m < NV; ++m) px_[m] = xselect_gt(ux[m], 1.0f, atanc_reduced(ux[m]), px_[m]);
  }
  if (lanes_max<V, NV>(uy) > 0.25f) {
#pragma unroll
    for (int m = 0; m < NV; ++m)
      py_[m] = xselect_gt(uy[m], 0.25f, atanhc_reduced(uy[m]), py_[m]);
  }
  const V Bc = L::bc(f[3].w), Bs = L::bc(f[4].w), nBs = L::bc(-f[4].w);
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    // the rotated-frame components are (B/sig) gx, (B/sig) gy
    const V gx = xmul(tx[m], px_[m]);
    const V gy = xmul(ty[m], py_[m]);
    AX[m] = xfma(gx, Bc, xfma(gy, nBs, AX[m]));
    AY[m] = xfma(gy, Bc, xfma(gx, Bs, AY[m]));
    if (TIGHT) {
      ER[m] = xfma(L::bc(f[4].y), xabs(gx), xfma(L::bc(f[4].z), xabs(gy), ER[m]));
      ER[m] = xfma(L::bc(2.0f), xadd(xabs(AX[m]), xabs(AY[m])), ER[m]);
    }
  }
}

// Stage potentials [c0, c0 + cn) of a sample's records into shared memory,
// f[4].x replaced by the grid's coefficient P (stage_p32).  Called by all NT
// threads of the block.
template <int NT>
__device__ __forceinline__ void stage_chunk32(float4* sp, const Pot32* __restrict__ pb, int c0,
                                              int cn, const Seg32& sg, float theta1) {
  for (int v = threadIdx.x; v < cn * 5; v += NT) {
    const int k = v / 5, w = v - k * 5;
    float4 val = pb[c0 + k].f[w];
    if (w == 4) {
      const int kk = c0 + k;
      val.x = stage_p32(pb[kk], kk >= sg.n_sis && kk < sg.n_sis + sg.n_piemd, theta1);
    }
    sp[v] = val;
  }
}

// The node lanes of one thread: its NPT nodes as NPT / 2 pairs (F2) and, for
// odd NPT, one single node (float).
template <int NPT>
struct NodeLanes {
  static constexpr int NP = NPT / 2;
  static constexpr bool ODD = (NPT % 2) != 0;
  F2 p[NP > 0 ? NP : 1];
  float s[1];
};

// Apply one kind's per-potential function KF to a thread's node lanes.
#define LT_NODES_APPLY(KF, TIGHT, f, P, X, Y, AX, AY, ER)                              \
  do {                                                                                \
    if constexpr (decltype(Y)::NP > 0)                                                \
      KF<F2, decltype(Y)::NP, TIGHT>(f, P, X, Y.p, AX.p, AY.p, ER.p);                  \
    if constexpr (decltype(Y)::ODD) KF<float, 1, TIGHT>(f, P, X, Y.s, AX.s, AY.s, ER.s); \
  } while (0)

template <int NPT, bool TIGHT>
__device__ __forceinline__ void flush_lanes(NodeLanes<NPT>& AX, NodeLanes<NPT>& AY,
                                            NodeLanes<NPT>& PX, NodeLanes<NPT>& PY,
                                            NodeLanes<NPT>& ER) {
  constexpr int NP = NodeLanes<NPT>::NP;
  if constexpr (NP > 0) flush_group<F2, NP, TIGHT>(AX.p, AY.p, PX.p, PY.p, ER.p);
  if constexpr (NodeLanes<NPT>::ODD) flush_group<float, 1, TIGHT>(AX.s, AY.s, PX.s, PY.s, ER.s);
}

// The per-item body of both FP32 deflection kernels: the deflection (AX, AY)
// and the running-bound terms ER (tight or coarse) of one thread's NPT nodes (column X, rows
// Y[]) over all n_pot potentials of one sample, kind segment by kind segment
// ([0, n_sis) SIS, then PIEMD, then SIE), in groups of at most kSumGroup
// potentials whose partial sums join the totals once per group.  The order of
// every operation of a node depends only on the potentials, not on NT, NPT or
// the pairing of the thread's nodes.
// sp: shared memory of kChunk32 * 5 float4; called by all NT threads.
//
// restage: false when sp already holds this sample's records (the block's
// previous item was of the same sample and all its potentials fit one
// chunk); the caller decides block-uniformly.
template <int NT, int NPT, bool TIGHT>
__device__ __forceinline__ void deflect32_nodes(const Pot32* __restrict__ pb, int n_pot,
                                                const Seg32& sg, float theta1, float X,
                                                const float* Y, float4* sp, float* AX,
                                                float* AY, float* ER, bool restage = true) {
  typedef NodeLanes<NPT> NL;
  NL y, ax, ay, px, py, er;
#pragma unroll
  for (int m = 0; m < NL::NP; ++m) {
    y.p[m] = f2_pack(Y[2 * m], Y[2 * m + 1]);
    ax.p[m] = ay.p[m] = px.p[m] = py.p[m] = er.p[m] = f2_pack(0.0f, 0.0f);
  }
  if constexpr (NL::ODD) {
    y.s[0] = Y[NPT - 1];
    ax.s[0] = ay.s[0] = px.s[0] = py.s[0] = er.s[0] = 0.0f;
  }
  for (int c0 = 0; c0 < n_pot; c0 += kChunk32) {
    const int cn = min(kChunk32, n_pot - c0);
    if (restage || n_pot > kChunk32) {
      __syncthreads();  // the previous chunk's (or item's) readers of sp are done
      stage_chunk32<NT>(sp, pb, c0, cn, sg, theta1);
      __syncthreads();
    }
    const int e_sis = min(max(sg.n_sis - c0, 0), cn);
    const int e_pie = min(max(sg.n_sis + sg.n_piemd - c0, 0), cn);
    for (int k0 = 0; k0 < e_sis; k0 += kSumGroup) {
      for (int k = k0; k < min(k0 + kSumGroup, e_sis); ++k)
        LT_NODES_APPLY(sis32_nodes, TIGHT, &sp[k * 5], sp[k * 5 + 4].x, X, y, px, py, er);
      flush_lanes<NPT, TIGHT>(ax, ay, px, py, er);
    }
    for (int k0 = e_sis; k0 < e_pie; k0 += kSumGroup) {
      for (int k = k0; k < min(k0 + kSumGroup, e_pie); ++k)
        LT_NODES_APPLY(piemd32_nodes, TIGHT, &sp[k * 5], sp[k * 5 + 4].x, X, y, px, py, er);
      flush_lanes<NPT, TIGHT>(ax, ay, px, py, er);
    }
    for (int k0 = e_pie; k0 < cn; k0 += kSumGroup) {
      for (int k = k0; k < min(k0 + kSumGroup, cn); ++k)
        LT_NODES_APPLY(sie32_nodes, TIGHT, &sp[k * 5], sp[k * 5 + 4].x, X, y, px, py, er);
      flush_lanes<NPT, TIGHT>(ax, ay, px, py, er);
    }
  }
#pragma unroll
  for (int m = 0; m < NL::NP; ++m) {
    f2_unpack(ax.p[m], AX[2 * m], AX[2 * m + 1]);
    f2_unpack(ay.p[m], AY[2 * m], AY[2 * m + 1]);
    f2_unpack(er.p[m], ER[2 * m], ER[2 * m + 1]);
  }
  if constexpr (NL::ODD) {
    AX[NPT - 1] = ax.s[0];
    AY[NPT - 1] = ay.s[0];
    ER[NPT - 1] = er.s[0];
  }
}
#undef LT_NODES_APPLY

}  // namespace lt
