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
// error itself.
constexpr int kSumGroup = 32;

// Add a group's partial sums to the totals (one rounding per component,
// bounded by the new total) and clear them.
template <int NPT>
__device__ __forceinline__ void flush_group(float* AX, float* AY, float* PX, float* PY,
                                            float* ER) {
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    AX[m] += PX[m];
    AY[m] += PY[m];
    ER[m] = fmaf(2.0f, fabsf(AX[m]) + fabsf(AY[m]), ER[m]);
    PX[m] = 0.0f;
    PY[m] = 0.0f;
  }
}

// One SIS: alpha += b0 (theta - c)/R (zero at the centre).  err accumulates in
// units of the FP32 unit roundoff.  In this and the two functions below, AX
// and AY are a group's partial sums (flush_group).
template <int NPT>
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
    ER[m] = fmaf(2.0f, fabsf(AX[m]) + fabsf(AY[m]), ER[m]);
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
template <int NPT>
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
    ER[m] = fmaf(2.0f, fabsf(AX[m]) + fabsf(AY[m]), ER[m]);
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
template <int NPT>
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
    ER[m] = fmaf(f[4].y, fabsf(gx), fmaf(f[4].z, fabsf(gy), ER[m]));
    ER[m] = fmaf(2.0f, fabsf(AX[m]) + fabsf(AY[m]), ER[m]);
  }
}

}  // namespace lt
