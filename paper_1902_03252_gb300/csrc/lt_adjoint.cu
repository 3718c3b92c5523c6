// Hand-written adjoint of the chi^2 path with the triangle assignment and the
// image matching of the forward evaluation held fixed.
//
// chi^2 = sum_m |x_obs,m - x_m|^2 / sigma_m^2 (Eq. 11) with
//   x_m = theta_A + w_B (theta_B - theta_A) + w_C (theta_C - theta_A) inside the
//   matched triangle, where (w_B, w_C) solve
//   [beta_B - beta_A, beta_C - beta_A] (w_B, w_C)^T = beta_bar - beta_A,
//   beta_v = theta_v - r alpha(theta_v) (Eq. 13) and beta_bar the system's
//   barycentre of theta_obs - r alpha(theta_obs).
// With G = dchi^2/dx of a predicted image and lambda = M^-T (G.(theta_B -
// theta_A), G.(theta_C - theta_A)), dchi^2 = lambda . (dbeta_bar - sum_v w_v
// dbeta_v), so every parameter derivative is a sum over "adjoint points"
// (the three vertices of each matched triangle, coefficient r w_v lambda, and
// every observed image of the system, coefficient -(r/n) sum lambda) of
// coefficient . d alpha_k(point) / d p_k.
//
//   k_adj_vtx / k_adj_lam  build those points and coefficients (vertex
//                deflections of matched triangles recomputed in FP64, one
//                block per vertex; then one block per sample for the
//                coefficients);
//   k_adj_grad   one block per potential: the 2x6 Jacobian of its deflection
//                w.r.t. (x, y, e, phi, r_core, sigma_v) at every point, in
//                FP32, contracted with the coefficients (one point per lane,
//                the warps over the point chunks); FP32 warp sums of 32
//                points are accumulated in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lt_internal.cuh"

namespace lt {

constexpr int kAdjThreads = 128;

// ------------------------------------------------------------ coefficients
// Pass 1a, one block per (sample, observed image m, vertex v): if m is the
// first observed image matched to its predicted image h, the FP64
// deflection of vertex v of h's triangle (threads split the potentials, sums
// in index order), parked in the point's coefficient fields for pass 1b.
// The vertex deflections are recomputed in FP64: M = [beta_B - beta_A,
// beta_C - beta_A] is a difference of large deflections and its FP32 rounding
// would be amplified by M's conditioning in magnified triangles.  One block
// per vertex spreads a model's matched triangles over three times as many
// SMs as one block per triangle.
constexpr int kAdjVtxThreads = 128;

// h's owner: the first observed image of the sample matched to it
__device__ __forceinline__ bool adj_owner(const int32_t* mh, int m, int h) {
  bool owner = h >= 0;
  for (int k = 0; k < m && owner; ++k) owner = mh[k] != h;
  return owner;
}

// triangle vertices of hit H: T0 = (00, 10, 11), T1 = (00, 11, 01)
__device__ __forceinline__ void adj_vertex(const SampleGrid& g, int64_t tri, int v, double& X,
                                           double& Y) {
  const int64_t cell = tri / 2;
  const int t = (int)(tri % 2);
  const int i = (int)(cell % (g.nx - 1)), j = (int)(cell / (g.nx - 1));
  const int di = v == 0 ? 0 : (v == 1 ? 1 : (t == 0 ? 1 : 0));
  const int dj = v == 0 ? 0 : (v == 1 ? (t == 0 ? 0 : 1) : 1);
  X = g.x0 + (double)(i + di) * g.dx;
  Y = g.y0 + (double)(j + dj) * g.dy;
}

__global__ void __launch_bounds__(kAdjVtxThreads)
    k_adj_vtx(const Pot64* __restrict__ pot64, int n_pot, int batch,
              const SampleGrid* __restrict__ grids, const Hit* __restrict__ hits,
              int64_t hit_cap, lt_obs obs, const int32_t* __restrict__ match_hit,
              AdjPt* __restrict__ pts, int P) {
  __shared__ double2 buf[kAdjVtxThreads];
  __shared__ double res[2];
  for (int64_t f3 = blockIdx.x; f3 < (int64_t)batch * obs.n_obs * 3; f3 += gridDim.x) {
    const int64_t f = f3 / 3;
    const int v = (int)(f3 - f * 3);
    const int b = (int)(f / obs.n_obs);
    const int m = (int)(f - (int64_t)b * obs.n_obs);
    const int32_t* mh = match_hit + (int64_t)b * obs.n_obs;
    const int h = mh[m];
    if (!adj_owner(mh, m, h)) continue;  // block-uniform
    const SampleGrid g = grids[b];
    const Hit H = hits[(int64_t)b * hit_cap + h];
    double TX, TY;
    adj_vertex(g, H.tri, v, TX, TY);
    block_alpha64<kAdjVtxThreads>(pot64 + (int64_t)b * n_pot, n_pot, 1, &TX, &TY, &res[0],
                                  &res[1], buf);
    if (threadIdx.x == 0) pts[(int64_t)b * P + 3 * m + v] = AdjPt{TX, TY, res[0], res[1]};
    __syncthreads();  // res is read before the next vertex overwrites it
  }
}

// Pass 1b, one block per sample, threads over its observed images m: for
// h's owner, the coefficients of its three vertex points from the parked
// deflections: lambda = M^-T (dB, dC) with (dB, dC) the chi^2 gradient of
// h's position along the triangle's image-plane edges; other images get zero
// points.  Pass 2, after a block barrier: every observed image of system i is
// a barycentre point with coefficient -(r_i / n_i) sum over the system's
// predicted images of lambda.  The matched-hit and system arrays are first
// staged in shared memory (the loops over them would otherwise wait on one
// global load per observed image), with per-system lists of the observed
// images in index order, so the system sums issue one FP64 add per image of
// the longest system rather than one per observed image (GB300's FP64 unit
// takes ~80 cycles per warp instruction, whatever the active lanes).  Beyond
// kAdjLamSmemInts the kernel reads the arrays from global memory and scans;
// both sum in the same order.
constexpr int kAdjLamThreads = 256;
constexpr int kAdjLamSmemInts = 12000;  // 3 n_obs + n_sys + 1 ints (48 000 bytes)

__global__ void __launch_bounds__(kAdjLamThreads)
    k_adj_lam(int batch, const Hit* __restrict__ hits, int64_t hit_cap, lt_obs obs,
              const int32_t* __restrict__ match_hit, double2* __restrict__ lam,
              AdjPt* __restrict__ pts, int P) {
  const int b = blockIdx.x;
  if (b >= batch) return;  // block-uniform
  const int n_obs = obs.n_obs, n_sys = obs.n_sys;
  const int32_t* mh = match_hit + (int64_t)b * n_obs;
  const int32_t* sy = obs.sys;
  AdjPt* pp = pts + (int64_t)b * P;
  double2* lb = lam + (int64_t)b * n_obs;
  extern __shared__ int s_obs[];  // [n_obs] hits, [n_obs] systems, [n_sys + 1] starts, [n_obs] list
  const bool staged = 3 * n_obs + n_sys + 1 <= kAdjLamSmemInts;
  int* first = s_obs + 2 * n_obs;
  int* idx = first + n_sys + 1;
  if (staged) {
    int* smh = s_obs;
    int* ssy = s_obs + n_obs;
    for (int k = threadIdx.x; k < n_obs; k += kAdjLamThreads) {
      smh[k] = mh[k];
      ssy[k] = sy[k];
    }
    for (int i = threadIdx.x; i <= n_sys; i += kAdjLamThreads) first[i] = 0;
    __syncthreads();
    mh = smh;
    sy = ssy;
    // (indices outside [0, n_sys) break the lt_obs contract; they are left
    // out of the lists so that no shared-memory write leaves them)
    for (int k = threadIdx.x; k < n_obs; k += kAdjLamThreads) {
      const int i = sy[k];
      if ((unsigned)i < (unsigned)n_sys) atomicAdd(&first[i + 1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < n_sys; ++i) first[i + 1] += first[i];
    __syncthreads();
    // image k's place in its system's list: the images of the system before it
    for (int k = threadIdx.x; k < n_obs; k += kAdjLamThreads) {
      const int i = sy[k];
      if ((unsigned)i >= (unsigned)n_sys) continue;
      int rank = 0;
      for (int k2 = 0; k2 < k; ++k2) rank += sy[k2] == i;
      idx[first[i] + rank] = k;
    }
  }
  for (int m = threadIdx.x; m < n_obs; m += kAdjLamThreads) {
    const int h = mh[m];
    if (!adj_owner(mh, m, h)) {
      for (int v = 0; v < 3; ++v) pp[3 * m + v] = AdjPt{0.0, 0.0, 0.0, 0.0};
      lb[m] = make_double2(0.0, 0.0);
      continue;
    }
    const Hit H = hits[(int64_t)b * hit_cap + h];
    // dchi^2/dx of this predicted image, over every observed image matched to it
    double Gx = 0.0, Gy = 0.0;
    for (int k = m; k < n_obs; ++k) {
      if (mh[k] != h) continue;
      const double s2 = obs.sigma[k] * obs.sigma[k];
      Gx += -2.0 * (obs.x[k] - H.x) / s2;
      Gy += -2.0 * (obs.y[k] - H.y) / s2;
    }
    const double r = obs.dls_ds[sy[m]];
    double TX[3], TY[3], BX[3], BY[3];
    for (int v = 0; v < 3; ++v) {
      const AdjPt q = pp[3 * m + v];
      TX[v] = q.x;
      TY[v] = q.y;
      BX[v] = TX[v] - r * q.cx;
      BY[v] = TY[v] - r * q.cy;
    }
    const double M00 = BX[1] - BX[0], M01 = BX[2] - BX[0];
    const double M10 = BY[1] - BY[0], M11 = BY[2] - BY[0];
    const double det = M00 * M11 - M01 * M10;
    const double dB = Gx * (TX[1] - TX[0]) + Gy * (TY[1] - TY[0]);
    const double dC = Gx * (TX[2] - TX[0]) + Gy * (TY[2] - TY[0]);
    const double lx = (M11 * dB - M10 * dC) / det;
    const double ly = (-M01 * dB + M00 * dC) / det;
    lb[m] = make_double2(lx, ly);
    for (int v = 0; v < 3; ++v)
      pp[3 * m + v] = AdjPt{TX[v], TY[v], r * H.w[v] * lx, r * H.w[v] * ly};
  }
  __syncthreads();  // every lambda of the sample is written
  for (int m = threadIdx.x; m < n_obs; m += kAdjLamThreads) {
    const int i = sy[m];
    double Lx = 0.0, Ly = 0.0;
    int n = 0;
    if (staged && (unsigned)i < (unsigned)n_sys) {
      for (int j = first[i]; j < first[i + 1]; ++j) {
        const double2 v = lb[idx[j]];
        ++n;
        Lx += v.x;
        Ly += v.y;
      }
    } else {
      for (int k = 0; k < n_obs; ++k) {
        if (sy[k] != i) continue;
        ++n;
        Lx += lb[k].x;
        Ly += lb[k].y;
      }
    }
    const double fct = -obs.dls_ds[i] / n;
    pp[3 * n_obs + m] = AdjPt{obs.x[m], obs.y[m], fct * Lx, fct * Ly};
  }
}

// --------------------------------------------------------------- Jacobians
// atan(sqrt t)/sqrt t, atanh(sqrt t)/sqrt t and their t-derivatives.
__device__ __forceinline__ void atanc_d(float t, float& A, float& dA) {
  if (t < 0.05f) {
    A = 1.f - t * (1.f / 3 - t * (1.f / 5 - t * (1.f / 7 - t * (1.f / 9))));
    dA = -1.f / 3 + t * (2.f / 5 - t * (3.f / 7 - t * (4.f / 9 - t * (5.f / 11))));
  } else {
    const float s = sqrtf(t);
    A = atanf(s) / s;
    dA = (1.f / (1.f + t) - A) / (2.f * t);
  }
}
__device__ __forceinline__ void atanhc_d(float t, float& H, float& dH) {
  if (t < 0.05f) {
    H = 1.f + t * (1.f / 3 + t * (1.f / 5 + t * (1.f / 7 + t * (1.f / 9))));
    dH = 1.f / 3 + t * (2.f / 5 + t * (3.f / 7 + t * (4.f / 9 + t * (5.f / 11))));
  } else {
    const float s = sqrtf(t);
    H = 0.5f * log1pf(2.f * s / (1.f - s)) / s;
    dH = (1.f / (1.f - t) - H) / (2.f * t);
  }
}

// One cored isothermal term F(w) = (atan(k zx)/k, atanh(k zy)/k) of the
// PIEMD in its own frame and its derivatives w.r.t. x', y', q and w.
struct CoredD {
  float Fx, Fy, Fx_x, Fx_y, Fy_x, Fy_y, Fx_q, Fy_q, Fx_w, Fy_w;
};
__device__ __forceinline__ CoredD cored_d(float xp, float yp, float q, float w) {
  const float q2 = q * q, T = (1.f - q) * (1.f + q);
  const float psi = sqrtf(q2 * (w * w + xp * xp) + yp * yp);
  const float Dx = psi + w, Dy = psi + q2 * w;
  const float zx = xp / Dx, zy = yp / Dy;
  float A, dA, H, dH;
  atanc_d(T * zx * zx, A, dA);
  atanhc_d(T * zy * zy, H, dH);
  const float fzx = 1.f / (1.f + T * zx * zx), fzy = 1.f / (1.f - T * zy * zy);
  const float ipsi = 1.f / psi;
  const float px = q2 * xp * ipsi, py = yp * ipsi, pq = q * (w * w + xp * xp) * ipsi,
              pw = q2 * w * ipsi;
  const float zx_x = (1.f - zx * px) / Dx, zx_y = -zx * py / Dx, zx_q = -zx * pq / Dx,
              zx_w = -zx * (pw + 1.f) / Dx;
  const float zy_x = -zy * px / Dy, zy_y = (1.f - zy * py) / Dy,
              zy_q = -zy * (pq + 2.f * q * w) / Dy, zy_w = -zy * (pw + q2) / Dy;
  CoredD d;
  d.Fx = zx * A;
  d.Fy = zy * H;
  d.Fx_x = fzx * zx_x;
  d.Fx_y = fzx * zx_y;
  d.Fy_x = fzy * zy_x;
  d.Fy_y = fzy * zy_y;
  d.Fx_q = fzx * zx_q - 2.f * q * zx * zx * zx * dA;
  d.Fy_q = fzy * zy_q - 2.f * q * zy * zy * zy * dH;
  d.Fx_w = fzx * zx_w;
  d.Fy_w = fzy * zy_w;
  return d;
}

// Contract c . d alpha / d (x_c, y_c, e, phi, r_core, sigma_v) for one
// potential at (x, y) (FP32).  P: FP64 record (index order).
__device__ __forceinline__ void contract(const Pot64& P, float x, float y, float cx, float cy,
                                         float out[6]) {
  const int kind = (int)P.kind;
  const float dx = x - (float)P.cx, dy = y - (float)P.cy;
  const float b0 = (float)P.b0;
  for (int k = 0; k < 6; ++k) out[k] = 0.f;
  if (kind == LT_SIS) {
    const float R2 = dx * dx + dy * dy;
    if (!(R2 > 0.f)) return;
    const float iR = rsqrtf(R2), ux = dx * iR, uy = dy * iR;
    const float s = b0 * iR;  // d alpha / d theta = s (I - u u^T)
    const float cu = cx * ux + cy * uy;
    // d alpha / d c = -(d alpha / d theta)
    out[0] = -s * (cx - cu * ux);
    out[1] = -s * (cy - cu * uy);
    const float sv = (float)P.sv;
    if (sv > 0.f) out[5] = 2.f / sv * b0 * cu;
    return;
  }
  const float c = (float)P.c, sn = (float)P.s;
  const float xp = dx * c + dy * sn, yp = dy * c - dx * sn;
  // coefficient in the lens frame: c' = R(phi) c
  const float cpx = c * cx + sn * cy, cpy = -sn * cx + c * cy;
  float gx, gy, J00, J01, J10, J11, ge_x, ge_y, ga_x = 0.f, ga_y = 0.f;
  if (kind == LT_SIE) {
    const float e = (float)P.e;
    const float R2 = (1.f - e) * xp * xp + (1.f + e) * yp * yp;
    if (!(R2 > 0.f)) return;
    const float iR = rsqrtf(R2), iR3 = iR * iR * iR;
    const float ax = b0 * (1.f - e), ay = b0 * (1.f + e);
    gx = ax * xp * iR;
    gy = ay * yp * iR;
    J00 = ax * (iR - (1.f - e) * xp * xp * iR3);
    J01 = -ax * (1.f + e) * xp * yp * iR3;
    J10 = -ay * (1.f - e) * xp * yp * iR3;
    J11 = ay * (iR - (1.f + e) * yp * yp * iR3);
    const float dR = 0.5f * (yp * yp - xp * xp) * iR;  // dR/deps
    ge_x = b0 * (-xp * iR - (1.f - e) * xp * dR * iR * iR);
    ge_y = b0 * (yp * iR - (1.f + e) * yp * dR * iR * iR);
  } else {
    const float q = (float)P.q, a = (float)P.a, s = (float)P.sc;
    const float Bu = s / (s - a);  // unit-b0 scale
    const CoredD A = cored_d(xp, yp, q, a), S = cored_d(xp, yp, q, s);
    const float B = b0 * Bu;
    gx = B * (A.Fx - S.Fx);
    gy = B * (A.Fy - S.Fy);
    J00 = B * (A.Fx_x - S.Fx_x);
    J01 = B * (A.Fx_y - S.Fx_y);
    J10 = B * (A.Fy_x - S.Fy_x);
    J11 = B * (A.Fy_y - S.Fy_y);
    // parameter e: q = 1 - e
    ge_x = -B * (A.Fx_q - S.Fx_q);
    ge_y = -B * (A.Fy_q - S.Fy_q);
    const float dBu = s / ((s - a) * (s - a));
    ga_x = b0 * (dBu * (A.Fx - S.Fx) + Bu * A.Fx_w);
    ga_y = b0 * (dBu * (A.Fy - S.Fy) + Bu * A.Fy_w);
  }
  // d alpha / d theta = R(-phi) J R(phi); c . that = (c'^T J) R(phi)
  const float r0 = cpx * J00 + cpy * J10, r1 = cpx * J01 + cpy * J11;
  out[0] = -(r0 * c - r1 * sn);
  out[1] = -(r0 * sn + r1 * c);
  out[2] = cpx * ge_x + cpy * ge_y;
  // d alpha / d phi = R(-phi) [(-gy, gx) + J (y', -x')]
  out[3] = cpx * (-gy + J00 * yp - J01 * xp) + cpy * (gx + J10 * yp - J11 * xp);
  out[4] = cpx * ga_x + cpy * ga_y;
  // alpha is proportional to sigma_v^2
  const float sv = (float)P.sv;
  if (sv > 0.f) out[5] = 2.f / sv * (cpx * gx + cpy * gy);
}

// One warp per (sample, potential): lane l takes adjoint points l, l + 32, ...;
// each round of 32 points is reduced across the warp in FP32 (a fixed
// butterfly, so the result is deterministic) and accumulated in FP64.
// One block per (sample, potential): warp w takes the point chunks
// 32 w, 32 w + kAdjThreads, ...; each chunk's FP32 warp sum is accumulated
// in FP64 per warp, and the warps' sums are added in warp order (a fixed
// order: the gradient is deterministic).
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_grad(const Pot64* __restrict__ pot64, int n_pot, int batch,
               const AdjPt* __restrict__ pts, int P, double* __restrict__ grad) {
  constexpr int NW = kAdjThreads / 32;
  __shared__ double part[NW][6];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t pid = blockIdx.x;  // sample * n_pot + potential
  if (pid >= (int64_t)batch * n_pot) return;  // block-uniform
  const int b = (int)(pid / n_pot);
  const Pot64 p = pot64[pid];
  const AdjPt* pb = pts + (int64_t)b * P;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int c0 = 32 * w; c0 < P; c0 += kAdjThreads) {
    float o[6] = {0, 0, 0, 0, 0, 0};
    const int v = c0 + lane;
    if (v < P) {
      const AdjPt q = pb[v];
      if (q.cx != 0.0 || q.cy != 0.0)
        contract(p, (float)q.x, (float)q.y, (float)q.cx, (float)q.cy, o);
    }
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      float t = o[m];
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      acc[m] += t;
    }
  }
  if (lane == 0)
    for (int m = 0; m < 6; ++m) part[w][m] = acc[m];
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int k = 0; k < NW; ++k) s += part[k][threadIdx.x];
    grad[pid * 6 + threadIdx.x] = s;
  }
}

cudaError_t launch_adjoint(const Pot64* pot64, int n_pot, int batch, const SampleGrid* grids,
                           const Hit* hits, int64_t hit_cap, const lt_obs& obs,
                           const int32_t* match_hit, double2* lam, AdjPt* pts, double* grad,
                           int sm_count, cudaStream_t st) {
  const int P = 4 * obs.n_obs;
  const int64_t warps = (int64_t)batch * obs.n_obs;
  int64_t vblocks = warps * 3;
  if (vblocks > (int64_t)sm_count * 16) vblocks = (int64_t)sm_count * 16;
  k_adj_vtx<<<(unsigned)vblocks, kAdjVtxThreads, 0, st>>>(pot64, n_pot, batch, grids, hits,
                                                          hit_cap, obs, match_hit, pts, P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nl = 3 * obs.n_obs + obs.n_sys + 1;
  const size_t lam_smem = nl <= kAdjLamSmemInts ? sizeof(int) * (size_t)nl : 0;
  k_adj_lam<<<(unsigned)batch, kAdjLamThreads, lam_smem, st>>>(batch, hits, hit_cap, obs,
                                                               match_hit, lam, pts, P);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t gblocks = (int64_t)batch * n_pot;
  k_adj_grad<<<(unsigned)gblocks, kAdjThreads, 0, st>>>(pot64, n_pot, batch, pts, P, grad);
  return cudaGetLastError();
}

}  // namespace lt
