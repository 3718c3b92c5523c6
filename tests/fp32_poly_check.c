/*
 * Exhaustive check of an FP32 Horner polynomial against a function, over
 * every float in [lo, hi] (test helper, built by tests/test_fp32_poly.py).
 *
 * The polynomial is evaluated exactly as the CUDA kernel does: p = c[0];
 * p = fmaf(p, u, c[k]) for k = 1..n-1, each fused multiply-add rounded once
 * to float (C99 fmaf), with subnormal inputs flushed to zero as the kernel's
 * flush-to-zero mode does.  The reference is the function in double
 * precision (errors near 1e-16, far below the FP32 unit roundoff 2^-24).
 * Returns the largest |p(u) - f(u)| / |f(u)| and the u where it occurs.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

static double atanc(double u) {
  if (u == 0.0) return 1.0;
  double t = sqrt(u);
  return atan(t) / t;
}
static double atanhc(double u) {
  if (u == 0.0) return 1.0;
  double t = sqrt(u);
  return atanh(t) / t;
}

static float bits_to_float(uint32_t b) {
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
}
static uint32_t float_to_bits(float f) {
  uint32_t b;
  memcpy(&b, &f, sizeof b);
  return b;
}

/* which: 0 = atan(t)/t, 1 = atanh(t)/t, both as functions of u = t*t. */
double poly_max_rel_err(int which, const float* c, int n, float lo, float hi, int n_threads,
                        float* worst_u) {
  const uint32_t b0 = float_to_bits(lo), b1 = float_to_bits(hi);
  double best = 0.0;
  float wu = lo;
#pragma omp parallel num_threads(n_threads > 0 ? n_threads : 1)
  {
    double tb = 0.0;
    float tu = lo;
#pragma omp for schedule(static)
    for (int64_t b = (int64_t)b0; b <= (int64_t)b1; ++b) {
      float u = bits_to_float((uint32_t)b);
      float uf = (u < FLT_MIN) ? 0.0f : u; /* flush-to-zero input */
      float p = c[0];
      for (int k = 1; k < n; ++k) p = fmaf(p, uf, c[k]);
      double f = which == 0 ? atanc((double)u) : atanhc((double)u);
      double e = fabs((double)p - f) / fabs(f);
      if (e > tb) {
        tb = e;
        tu = u;
      }
    }
#pragma omp critical
    {
      if (tb > best) {
        best = tb;
        wu = tu;
      }
    }
  }
  if (worst_u) *worst_u = wu;
  return best;
}
