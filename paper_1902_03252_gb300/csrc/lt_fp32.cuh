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

// Add a group's partial sums to the totals (one rounding per component,
// bounded by the new total) and clear them.
template <int NPT, bool TIGHT>
__device__ __forceinline__ void flush_group(float* AX, float* AY, float* PX, float* PY,
                                            float* ER) {
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    AX[m] += PX[m];
    AY[m] += PY[m];
    if (TIGHT) ER[m] = fmaf(2.0f, fabsf(AX[m]) + fabsf(AY[m]), ER[m]);
    PX[m] = 0.0f;
    PY[m] = 0.0f;
  }
}

// One SIS: alpha += b0 (theta - c)/R (zero at the centre).  err accumulates in
// units of the FP32 unit roundoff.  In this and the two functions below, AX
// and AY are a group's partial sums (flush_group).
template <int NPT, bool TIGHT>
__device__ __forceinline__ void sis32_nodes(const float4* f, float P, float X, const float* Y,
                                            float* AX, float* AY, float* ER) {
  const float dx = X - f[0].x;
  const float dx2 = dx * dx;
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const float dy = Y[m] - f[0].y;
    const float R2 = fmaf(dy, dy, dx2);
    // rr is +inf on the centre: there the direction of alpha is undefined and
    // the bound term P rr makes the node's bound infinite (never certified)
    const float rr = rsqrt_approx32(R2);
    const float ri = R2 > 0.0f ? rr : 0.0f;
    const float g = f[0].z * ri;
    AX[m] = fmaf(g, dx, AX[m]);
    AY[m] = fmaf(g, dy, AY[m]);
    ER[m] = fmaf(P, rr, ER[m]);
    if (TIGHT) ER[m] = fmaf(2.0f, fabsf(AX[m]) + fabsf(AY[m]), ER[m]);
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
template <int NPT, bool TIGHT>
__device__ __forceinline__ void sie32_nodes(const float4* f, float P, float X, const float* Y,
                                            float* AX, float* AY, float* ER) {
  const float dx = X - f[0].x;
  const float dxu = dx * f[0].z, dxv = dx * f[1].y;
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const float dy = Y[m] - f[0].y;
    const float u = fmaf(dy, f[0].w, dxu);
    const float v = fmaf(dy, f[1].x, -dxv);
    const float R2 = fmaf(u, u, v * v);
    const float rr = rsqrt_approx32(R2);  // +inf on the centre: an infinite bound there
    const float ri = R2 > 0.0f ? rr : 0.0f;
    const float t1 = fmaf(f[1].z, u, -(f[1].w * v));
    const float t2 = fmaf(f[2].x, v, f[2].y * u);
    AX[m] = fmaf(ri, t1, AX[m]);
    AY[m] = fmaf(ri, t2, AY[m]);
    ER[m] = fmaf(P, rr, ER[m]);
    if (TIGHT) ER[m] = fmaf(2.0f, fabsf(AX[m]) + fabsf(AY[m]), ER[m]);
  }
}

// One PIEMD (dPIE) in difference form.  With psi_w = sqrt(q^2(w^2+x'^2)+y'^2),
// F(a) - F(s) is evaluated as one atan / atanh of
//   tx = x' ds_x / ((psi_a+a)(psi_s+s) + k^2 x'^2),
//   ty = y' ds_y / ((psi_a+q^2 a)(psi_s+q^2 s) - k^2 y'^2),
// ds_x = (s-a)(1 + q^2 (s+a)/(psi_a+psi_s)), ds_y = q^2 (s-a)(1 + (s+a)/(psi_a+psi_s))
// (atan u - atan v = atan((u-v)/(1+uv)), atanh likewise, and
// psi_s - psi_a = q^2 (s^2-a^2)/(psi_a+psi_s)), which avoids the cancellation
// of the two cored terms and halves the transcendental work.
//
// One PIEMD on the NPT nodes of a thread (one column).  The range tests of
// the two special functions are merged into one branch per thread and
// potential: both polynomials of atanc_sq32 / atanhc_sq32 are evaluated on
// the unreduced arguments for every node (out of range the value may
// overflow; it is replaced), and the nodes outside their ranges (atan:
// t2 > 1, atanh: t2 > 0.25; about 14 % of node-potential pairs on cluster
// lenses) are then recomputed by those functions.  Every node gets exactly
// the values and roundings of the per-node evaluation; the merged test
// removes most of the branch instructions from the issue stream.
template <int NPT, bool TIGHT>
__device__ __forceinline__ void piemd32_nodes(const float4* f, float P, float X, const float* Y,
                                              float* AX, float* AY, float* ER) {
  const float cy = f[0].y, c = f[0].z, s = f[0].w;
  const float k2 = f[1].w, Bc = f[3].w, Bs = f[4].w;
  const float dx = X - f[0].x;
  const float dxc = dx * c, dxs = dx * s;
  float tx[NPT], ty[NPT], ux[NPT], uy[NPT], ra[NPT], px_[NPT], py_[NPT];
  bool any = false;
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const float dy = Y[m] - cy;
    const float xp = fmaf(dy, s, dxc);
    const float yp = fmaf(dy, c, -dxs);
    const float x2 = xp * xp, y2 = yp * yp;
    const float t = fmaf(f[1].x, x2, y2);
    const float pa2 = t + f[1].y, ps2 = t + f[1].z;
    ra[m] = rsqrt_approx32(pa2);
    // psi_s in one MUFU operation.  Over every float mantissa (four binades
    // checked exhaustively on GB300) sqrt.approx.ftz errs by at most 1.68 u
    // against the rounded sqrt, below the 2.71 u of ps2 * rsqrt(ps2) that the
    // error bound was derived for; psi_a keeps that form, as 1/psi_a is needed.
    const float ps = sqrt_approx32(ps2);
    const float pa = pa2 * ra[m];
    const float iD = rcp_approx32(pa + ps);
    const float dsx = fmaf(f[3].y, iD, f[3].x);
    const float dsy = fmaf(f[3].y, iD, f[3].z);
    const float px = (pa + f[2].x) * (ps + f[2].y);
    const float py = (pa + f[2].z) * (ps + f[2].w);
    const float denx = fmaf(k2, x2, px);
    const float deny = fmaf(-k2, y2, py);
    // the ds coefficients carry sig = sqrt(k2): these are sig tx, sig ty
    tx[m] = (xp * dsx) * rcp_approx32(denx);
    ty[m] = (yp * dsy) * rcp_approx32(deny);
    ux[m] = tx[m] * tx[m];
    uy[m] = ty[m] * ty[m];
    any |= (ux[m] > 1.0f) | (uy[m] > 0.25f);
  }
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    // the polynomials of atanc_sq32 / atanhc_sq32 on the unreduced arguments
    const float p = atanc_poly32(ux[m]);
    const float h = atanhc_poly32(uy[m]);
    px_[m] = p;
    py_[m] = h;
  }
  if (any) {
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      if (ux[m] > 1.0f) px_[m] = atanc_sq32(ux[m]);
      if (uy[m] > 0.25f) py_[m] = atanhc_sq32(uy[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    // the rotated-frame components are (B/sig) gx, (B/sig) gy
    const float gx = tx[m] * px_[m];
    const float gy = ty[m] * py_[m];
    AX[m] = fmaf(gx, Bc, fmaf(-gy, Bs, AX[m]));
    AY[m] = fmaf(gy, Bc, fmaf(gx, Bs, AY[m]));
    ER[m] = fmaf(P, ra[m], ER[m]);
    if (TIGHT) {
      ER[m] = fmaf(f[4].y, fabsf(gx), fmaf(f[4].z, fabsf(gy), ER[m]));
      ER[m] = fmaf(2.0f, fabsf(AX[m]) + fabsf(AY[m]), ER[m]);
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

// The per-item body of both FP32 deflection kernels: the deflection (AX, AY)
// and the running-bound terms ER (tight or coarse) of one thread's NPT nodes (column X, rows
// Y[]) over all n_pot potentials of one sample, kind segment by kind segment
// ([0, n_sis) SIS, then PIEMD, then SIE), in groups of at most kSumGroup
// potentials whose partial sums join the totals once per group.  The order of
// every operation of a node depends only on the potentials, not on NT or NPT.
// sp: shared memory of kChunk32 * 5 float4; called by all NT threads.
template <int NT, int NPT, bool TIGHT>
__device__ __forceinline__ void deflect32_nodes(const Pot32* __restrict__ pb, int n_pot,
                                                const Seg32& sg, float theta1, float X,
                                                const float* Y, float4* sp, float* AX,
                                                float* AY, float* ER) {
  float PX[NPT], PY[NPT];
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    PX[m] = 0.0f;
    PY[m] = 0.0f;
    AX[m] = 0.0f;
    AY[m] = 0.0f;
    ER[m] = 0.0f;
  }
  for (int c0 = 0; c0 < n_pot; c0 += kChunk32) {
    const int cn = min(kChunk32, n_pot - c0);
    __syncthreads();  // the previous chunk's (or item's) readers of sp are done
    stage_chunk32<NT>(sp, pb, c0, cn, sg, theta1);
    __syncthreads();
    const int e_sis = min(max(sg.n_sis - c0, 0), cn);
    const int e_pie = min(max(sg.n_sis + sg.n_piemd - c0, 0), cn);
    for (int k0 = 0; k0 < e_sis; k0 += kSumGroup) {
      for (int k = k0; k < min(k0 + kSumGroup, e_sis); ++k)
        sis32_nodes<NPT, TIGHT>(&sp[k * 5], sp[k * 5 + 4].x, X, Y, PX, PY, ER);
      flush_group<NPT, TIGHT>(AX, AY, PX, PY, ER);
    }
    for (int k0 = e_sis; k0 < e_pie; k0 += kSumGroup) {
      for (int k = k0; k < min(k0 + kSumGroup, e_pie); ++k)
        piemd32_nodes<NPT, TIGHT>(&sp[k * 5], sp[k * 5 + 4].x, X, Y, PX, PY, ER);
      flush_group<NPT, TIGHT>(AX, AY, PX, PY, ER);
    }
    for (int k0 = e_pie; k0 < cn; k0 += kSumGroup) {
      for (int k = k0; k < min(k0 + kSumGroup, cn); ++k)
        sie32_nodes<NPT, TIGHT>(&sp[k * 5], sp[k * 5 + 4].x, X, Y, PX, PY, ER);
      flush_group<NPT, TIGHT>(AX, AY, PX, PY, ER);
    }
  }
}

}  // namespace lt
