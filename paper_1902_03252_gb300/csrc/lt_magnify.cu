// Magnifications and the source-plane chi^2, FP64 throughout (compiled
// without FMA contraction, like the other FP64 stages).
//
// The relensing pipeline (Fig. 1) maps observed images to the source plane
// and lenses grid triangles there; both give magnifications for free:
//   * point magnification at an observed image: mu = 1/det(I - r J), with
//     J = d alpha/d theta summed over the potentials from closed forms;
//   * triangle magnification of a predicted image: the image-plane area of
//     its triangle over the signed area of the lensed triangle (Eq. 13).
// The source-plane chi^2 (the LENSTOOL source-plane fit of Jullo et al. 2007)
// weights the scatter of each system's sources about their barycentre by the
// squared magnification: sum_m |beta_m - beta_bar|^2 mu_m^2 / sigma_m^2.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lt_internal.cuh"

namespace lt {

constexpr int kMagThreads = 128;

// d alpha/d theta of one potential (symmetric: jxy = jyx).
//   SIS : b0/R^3 (dy^2, -dx dy, dx^2).
//   SIE : in the rotated frame b0 a1 a2/R^3 (y'^2, -x'y', x'^2) with
//         R^2 = a1 x'^2 + a2 y'^2, a1,2 = 1 -+ eps (second derivatives of
//         the pseudo-elliptical potential b0 R).
//   PIEMD: per cored term w, with psi = sqrt(q^2 (w^2 + x'^2) + y'^2) and
//         den = psi ((psi + w)^2 + k^2 x'^2):
//         (q^2 w^2 + y'^2 + w psi, -x'y', w^2 + x'^2 + w psi) / den;
//         scaled by b0 s/(s-a) and differenced (core minus cut).
// The rotated-frame matrix H is taken back by J = R(phi)^T H R(phi).
// Zero where the profile is singular (SIS/SIE centre), like the deflection.
__device__ __forceinline__ void jac64_one(const Pot64& p, double x, double y, double& jxx,
                                          double& jxy, double& jyy) {
  const double dx = x - p.cx;
  const double dy = y - p.cy;
  const int kind = (int)p.kind;
  if (kind == LT_SIS) {
    const double R2 = dx * dx + dy * dy;
    if (R2 == 0.0) { jxx = 0.0; jxy = 0.0; jyy = 0.0; return; }
    const double f = p.b0 / (R2 * sqrt(R2));
    jxx = f * (dy * dy);
    jxy = -f * (dx * dy);
    jyy = f * (dx * dx);
    return;
  }
  const double xp = dx * p.c + dy * p.s;
  const double yp = dy * p.c - dx * p.s;
  double hxx, hxy, hyy;
  if (kind == LT_SIE) {
    const double a1 = 1.0 - p.e, a2 = 1.0 + p.e;
    const double R2 = a1 * (xp * xp) + a2 * (yp * yp);
    if (R2 == 0.0) { jxx = 0.0; jxy = 0.0; jyy = 0.0; return; }
    const double f = p.b0 * a1 * a2 / (R2 * sqrt(R2));
    hxx = f * (yp * yp);
    hxy = -f * (xp * yp);
    hyy = f * (xp * xp);
  } else {
    double h[2][3];
    for (int t = 0; t < 2; ++t) {
      const double w = t == 0 ? p.a : p.sc;
      const double psi = sqrt(p.q2 * (w * w + xp * xp) + yp * yp);
      const double pw = psi + w;
      const double den = psi * (pw * pw + p.k2 * (xp * xp));
      h[t][0] = (p.q2 * (w * w) + yp * yp + w * psi) / den;
      h[t][1] = -(xp * yp) / den;
      h[t][2] = (w * w + xp * xp + w * psi) / den;
    }
    hxx = p.scale * (h[0][0] - h[1][0]);
    hxy = p.scale * (h[0][1] - h[1][1]);
    hyy = p.scale * (h[0][2] - h[1][2]);
  }
  const double c = p.c, s = p.s;
  const double cc = c * c, ss = s * s, cs = c * s;
  jxx = cc * hxx - 2.0 * cs * hxy + ss * hyy;
  jxy = cs * (hxx - hyy) + (cc - ss) * hxy;
  jyy = ss * hxx + 2.0 * cs * hxy + cc * hyy;
}

// Sum over a block of NT threads of three doubles; the result is valid in
// thread 0.  Fixed order: warp butterflies, then the warps in index order.
template <int NT>
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sm /*[3][NT/32]*/) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  if (l == 0) { sm[w] = a; sm[NW + w] = b; sm[2 * NW + w] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = sm[0]; b = sm[NW]; c = sm[2 * NW];
    for (int k = 1; k < NW; ++k) { a += sm[k]; b += sm[NW + k]; c += sm[2 * NW + k]; }
  }
  __syncthreads();
}

// One block per (sample, observed image): beta = theta - r alpha (the
// deflection summed in potential index order, as for the barycentres of the
// image-plane chi^2) and the point magnification.
__global__ void __launch_bounds__(kMagThreads)
    k_src_obs(const Pot64* __restrict__ pot64, int n_pot, int batch, lt_obs obs,
              double2* __restrict__ beta, double* __restrict__ mu) {
  __shared__ double2 buf[kMagThreads];
  __shared__ double res[2];
  __shared__ double red[3 * (kMagThreads / 32)];
  for (int64_t f = blockIdx.x; f < (int64_t)batch * obs.n_obs; f += gridDim.x) {
    const int b = (int)(f / obs.n_obs);
    const int m = (int)(f - (int64_t)b * obs.n_obs);
    const Pot64* pb = pot64 + (int64_t)b * n_pot;
    const double x = obs.x[m], y = obs.y[m];
    block_alpha64<kMagThreads>(pb, n_pot, 1, &x, &y, &res[0], &res[1], buf);
    double jxx = 0.0, jxy = 0.0, jyy = 0.0;
    for (int k = threadIdx.x; k < n_pot; k += kMagThreads) {
      double a, bb, c;
      jac64_one(pb[k], x, y, a, bb, c);
      jxx += a;
      jxy += bb;
      jyy += c;
    }
    block_sum3<kMagThreads>(jxx, jxy, jyy, red);
    if (threadIdx.x == 0) {
      const double r = obs.dls_ds[obs.sys[m]];
      beta[f] = make_double2(x - r * res[0], y - r * res[1]);
      const double det = (1.0 - r * jxx) * (1.0 - r * jyy) - (r * jxy) * (r * jxy);
      mu[f] = 1.0 / det;
    }
    __syncthreads();
  }
}

// One block per sample: barycentres (each system's sources summed in
// observation order) and the magnification-weighted scatter.
__global__ void __launch_bounds__(kMagThreads)
    k_src_chi2(int batch, lt_obs obs, const double2* __restrict__ beta,
               const double* __restrict__ mu, double2* __restrict__ bary,
               double* __restrict__ chi2) {
  __shared__ double red[3 * (kMagThreads / 32)];
  for (int b = blockIdx.x; b < batch; b += gridDim.x) {
    const double2* bb = beta + (int64_t)b * obs.n_obs;
    double2* br = bary + (int64_t)b * obs.n_sys;
    for (int i = threadIdx.x; i < obs.n_sys; i += kMagThreads) {
      double sx = 0.0, sy = 0.0;
      int n = 0;
      for (int m = 0; m < obs.n_obs; ++m)
        if (obs.sys[m] == i) {
          sx = sx + bb[m].x;
          sy = sy + bb[m].y;
          ++n;
        }
      br[i] = n ? make_double2(sx / n, sy / n) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    double acc = 0.0, d1 = 0.0, d2 = 0.0;
    for (int m = threadIdx.x; m < obs.n_obs; m += kMagThreads) {
      const double2 c = br[obs.sys[m]];
      const double ex = bb[m].x - c.x, ey = bb[m].y - c.y;
      const double u = mu[(int64_t)b * obs.n_obs + m];
      const double sg = obs.sigma[m];
      acc += (ex * ex + ey * ey) * (u * u) / (sg * sg);
    }
    block_sum3<kMagThreads>(acc, d1, d2, red);
    if (threadIdx.x == 0) chi2[b] = acc;
  }
}

// One block per (sample, observed image): the signed triangle magnification of
// its matched predicted image (NaN without a match), from FP64 deflections of
// the triangle's three nodes.
__global__ void __launch_bounds__(kMagThreads)
    k_mag_pred(const Pot64* __restrict__ pot64, int n_pot, int batch,
               const SampleGrid* __restrict__ grids, const Hit* __restrict__ hits,
               int64_t hit_cap, lt_obs obs, const int32_t* __restrict__ match_hit,
               double* __restrict__ mu) {
  __shared__ double2 buf[3 * kMagThreads];
  __shared__ double res[6];
  for (int64_t f = blockIdx.x; f < (int64_t)batch * obs.n_obs; f += gridDim.x) {
    const int b = (int)(f / obs.n_obs);
    const int m = (int)(f - (int64_t)b * obs.n_obs);
    const int h = match_hit[f];
    if (h < 0) {  // block-uniform
      if (threadIdx.x == 0) mu[f] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    const SampleGrid g = grids[b];
    const Hit H = hits[(int64_t)b * hit_cap + h];
    const int64_t cell = H.tri / 2;
    const int t = (int)(H.tri % 2);
    const int i = (int)(cell % (g.nx - 1)), j = (int)(cell / (g.nx - 1));
    const int di[3] = {0, 1, t == 0 ? 1 : 0};
    const int dj[3] = {0, t == 0 ? 0 : 1, 1};
    double TX[3], TY[3];
    for (int v = 0; v < 3; ++v) {
      TX[v] = g.x0 + (double)(i + di[v]) * g.dx;
      TY[v] = g.y0 + (double)(j + dj[v]) * g.dy;
    }
    block_alpha64<kMagThreads>(pot64 + (int64_t)b * n_pot, n_pot, 3, TX, TY, &res[0], &res[3],
                               buf);
    if (threadIdx.x == 0) {
      const double r = obs.dls_ds[obs.sys[m]];
      double BX[3], BY[3];
      for (int v = 0; v < 3; ++v) {
        BX[v] = TX[v] - r * res[v];
        BY[v] = TY[v] - r * res[3 + v];
      }
      const double a_img = (TX[1] - TX[0]) * (TY[2] - TY[0]) - (TY[1] - TY[0]) * (TX[2] - TX[0]);
      const double a_src = (BX[1] - BX[0]) * (BY[2] - BY[0]) - (BY[1] - BY[0]) * (BX[2] - BX[0]);
      mu[f] = a_img / a_src;
    }
    __syncthreads();
  }
}

static int grid_blocks(int64_t items, int sm_count) {
  const int64_t cap = (int64_t)sm_count * 16;
  return (int)(items < cap ? (items > 0 ? items : 1) : cap);
}

cudaError_t launch_chi2_source(const Pot64* pot64, int n_pot, int batch, const lt_obs& obs,
                               double2* beta, double* mu, double2* bary, double* chi2,
                               int sm_count, cudaStream_t st) {
  k_src_obs<<<grid_blocks((int64_t)batch * obs.n_obs, sm_count), kMagThreads, 0, st>>>(
      pot64, n_pot, batch, obs, beta, mu);
  k_src_chi2<<<grid_blocks(batch, sm_count), kMagThreads, 0, st>>>(batch, obs, beta, mu, bary,
                                                                  chi2);
  return cudaGetLastError();
}

cudaError_t launch_mag_pred(const Pot64* pot64, int n_pot, int batch, const SampleGrid* grids,
                            const Hit* hits, int64_t hit_cap, const lt_obs& obs,
                            const int32_t* match_hit, double* mu, int sm_count,
                            cudaStream_t st) {
  k_mag_pred<<<grid_blocks((int64_t)batch * obs.n_obs, sm_count), kMagThreads, 0, st>>>(
      pot64, n_pot, batch, grids, hits, hit_cap, obs, match_hit, mu);
  return cudaGetLastError();
}

}  // namespace lt
