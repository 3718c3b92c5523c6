// D_ls/D_s from redshifts in a Friedmann-Lemaitre cosmology with matter and a
// cosmological constant (the paper's benchmark uses z_l = 0.3, z_s = 2.0 in
// flat LambdaCDM with Omega_m = 0.3, Omega_Lambda = 0.7, Sect. 4).  Host code:
// an input of the lens equation (Eq. 13), computed once per source.
//
// With E(z) = sqrt(Om (1+z)^3 + Ok (1+z)^2 + OL), Ok = 1 - Om - OL, the
// line-of-sight comoving distance in units of c/H0 is D_C(z) = int_0^z dz'/E,
// the transverse one D_M = D_C (Ok = 0) or sinh(sqrt(Ok) D_C)/sqrt(Ok)
// (Ok > 0), and the angular-diameter distance between z1 < z2 is
// D_M12/(1+z2) with D_M12 = D_M2 sqrt(1 + Ok D_M1^2) - D_M1 sqrt(1 + Ok D_M2^2)
// (valid for Ok >= 0).  So D_ls/D_s = D_M12 / D_M2 (H0 cancels).
#include <cmath>

#include "lt_internal.cuh"

namespace {

constexpr int kGL = 48;  // Gauss-Legendre points per integral

// Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1]: roots of
// P_n by Newton's method from cos(pi (k - 1/4)/(n + 1/2)), P_n and P_n' from
// the three-term recurrence, weights 2 / ((1 - x^2) P_n'(x)^2).
struct GaussLegendre {
  double x[kGL], w[kGL];
  GaussLegendre() {
    const int n = kGL;
    for (int k = 0; k < n; ++k) {
      double z = std::cos(M_PI * (k + 0.75) / (n + 0.5));
      double dp = 0.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int m = 2; m <= n; ++m) {
          const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[k] = z;
      w[k] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

double comoving(double z, double om, double ol, double ok) {
  static const GaussLegendre gl;
  // split [0, z] into pieces of width <= 0.5 for a smooth integrand per piece
  const int pieces = 1 + (int)(z / 0.5);
  const double h = z / pieces;
  double sum = 0.0;
  for (int p = 0; p < pieces; ++p) {
    const double a = p * h, mid = a + 0.5 * h;
    for (int k = 0; k < kGL; ++k) {
      const double zz = mid + 0.5 * h * gl.x[k];
      const double zp = 1.0 + zz;
      const double E = std::sqrt(om * zp * zp * zp + ok * zp * zp + ol);
      sum += 0.5 * h * gl.w[k] / E;
    }
  }
  return sum;
}

double transverse(double dc, double ok) {
  if (ok > 1e-12) {
    const double s = std::sqrt(ok);
    return std::sinh(s * dc) / s;
  }
  return dc;
}

}  // namespace

extern "C" lt_status lt_dls_ds(double z_l, double z_s, double omega_m, double omega_l,
                               double* dls_ds) {
  if (!dls_ds || !std::isfinite(z_l) || !std::isfinite(z_s) || !std::isfinite(omega_m) ||
      !std::isfinite(omega_l) || !(z_l >= 0.0) || !(z_s > z_l) || omega_m < 0.0)
    return LT_ERR_INVALID_ARG;
  const double ok = 1.0 - omega_m - omega_l;
  if (ok < -1e-12) return LT_ERR_INVALID_ARG;  // closed universes are not supported
  // E(z)^2 must stay positive on [0, z_s]
  for (int k = 0; k <= 64; ++k) {
    const double zp = 1.0 + z_s * k / 64.0;
    if (!(omega_m * zp * zp * zp + ok * zp * zp + omega_l > 0.0)) return LT_ERR_INVALID_ARG;
  }
  const double okc = ok > 0.0 ? ok : 0.0;
  const double m1 = transverse(comoving(z_l, omega_m, omega_l, ok), okc);
  const double m2 = transverse(comoving(z_s, omega_m, omega_l, ok), okc);
  const double m12 = m2 * std::sqrt(1.0 + okc * m1 * m1) - m1 * std::sqrt(1.0 + okc * m2 * m2);
  *dls_ds = m12 / m2;
  return LT_OK;
}
