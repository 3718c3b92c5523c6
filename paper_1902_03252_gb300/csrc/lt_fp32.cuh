// FP32 per-potential deflections shared by the deflection kernel and the
// adjoint (which recomputes vertex deflections with the same arithmetic).
#pragma once

#include "lt_internal.cuh"

namespace lt {

// One SIS: alpha += b0 (theta - c)/R (zero at the centre).  err accumulates in
// units of the FP32 unit roundoff.
__device__ __forceinline__ void sis32(const float4* f, float P, float x, float y, float& ax,
                                      float& ay, float& err) {
  float dx = x - f[0].x, dy = y - f[0].y;
  float R2 = fmaf(dx, dx, dy * dy);
  float ri = R2 > 0.0f ? rsqrtf(R2) : 0.0f;
  float g = f[0].z * ri;
  ax = fmaf(g, dx, ax);
  ay = fmaf(g, dy, ay);
  err = fmaf(P, ri, err);
  err = fmaf(2.0f, fabsf(ax) + fabsf(ay), err);
}

// One SIE (Algorithm 1).
__device__ __forceinline__ void sie32(const float4* f, float P, float x, float y, float& ax,
                                      float& ay, float& err) {
  float dx = x - f[0].x, dy = y - f[0].y;
  float c = f[0].z, s = f[0].w;
  float xp = fmaf(dx, c, dy * s);
  float yp = fmaf(dy, c, -(dx * s));
  float R2 = fmaf(xp * xp, f[1].x, yp * yp * f[1].y);
  float ri = R2 > 0.0f ? rsqrtf(R2) : 0.0f;
  float gx = f[1].z * xp * ri;
  float gy = f[1].w * yp * ri;
  ax = fmaf(gx, c, fmaf(-gy, s, ax));
  ay = fmaf(gy, c, fmaf(gx, s, ay));
  err = fmaf(P, ri, err);
  err = fmaf(2.0f, fabsf(ax) + fabsf(ay), err);
}

// One PIEMD (dPIE) in difference form.  With psi_w = sqrt(q^2(w^2+x'^2)+y'^2),
// F(a) - F(s) is evaluated as one atan / atanh of
//   tx = x' ds_x / ((psi_a+a)(psi_s+s) + k^2 x'^2),
//   ty = y' ds_y / ((psi_a+q^2 a)(psi_s+q^2 s) - k^2 y'^2),
// ds_x = (s-a)(1 + q^2 (s+a)/(psi_a+psi_s)), ds_y = q^2 (s-a)(1 + (s+a)/(psi_a+psi_s))
// (atan u - atan v = atan((u-v)/(1+uv)), atanh likewise, and
// psi_s - psi_a = q^2 (s^2-a^2)/(psi_a+psi_s)), which avoids the cancellation
// of the two cored terms and halves the transcendental work.
__device__ __forceinline__ void piemd32(const float4* f, float P, float x, float y, float& ax,
                                        float& ay, float& err) {
  float dx = x - f[0].x, dy = y - f[0].y;
  float c = f[0].z, s = f[0].w;
  float xp = fmaf(dx, c, dy * s);
  float yp = fmaf(dy, c, -(dx * s));
  float x2 = xp * xp, y2 = yp * yp;
  float t = fmaf(f[1].x, x2, y2);
  float pa2 = t + f[1].y, ps2 = t + f[1].z;
  float ra = rsqrtf(pa2), rs = rsqrtf(ps2);
  float pa = pa2 * ra, ps = ps2 * rs;
  float iD = __fdividef(1.0f, pa + ps);
  float dsx = fmaf(f[3].y, iD, f[3].x);
  float dsy = fmaf(f[3].y, iD, f[3].z);
  float px = (pa + f[2].x) * (ps + f[2].y);
  float py = (pa + f[2].z) * (ps + f[2].w);
  float k2 = f[1].w;
  float denx = fmaf(k2, x2, px);
  float deny = fmaf(-k2, y2, py);
  float tx = __fdividef(xp * dsx, denx);
  float ty = __fdividef(yp * dsy, deny);
  float B = f[3].w;
  float gx = B * tx * atanc_sq32(k2 * tx * tx);
  float gy = B * ty * atanhc_sq32(k2 * ty * ty);
  ax = fmaf(gx, c, fmaf(-gy, s, ax));
  ay = fmaf(gy, c, fmaf(gx, s, ay));
  err = fmaf(P, ra, err);
  err = fmaf(f[4].y, fabsf(gx), fmaf(f[4].z, fabsf(gy), err));
  err = fmaf(2.0f, fabsf(ax) + fabsf(ay), err);
}

}  // namespace lt
