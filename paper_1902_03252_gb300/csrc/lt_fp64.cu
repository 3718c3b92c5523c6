// FP64 kernels.  This translation unit is compiled with -fmad=false: every
// double operation is rounded separately, in the order written, so the FP64
// path evaluates the stated formulas exactly as an FP64 reference that follows
// the same statement (up to the ulps of atan/atanh/sin/cos).
//   k_prep        parameter preparation (a1): b0 = 4 pi (sigma_v/c)^2,
//                 rotations, axis ratios; FP64 records in index order and
//                 FP32 records grouped by kind with error-bound coefficients.
//   k_deflect64   FP64 deflection of every node (Sect. 2.2.2, Algorithm 1).
//   k_search64    FP64 lens mapping (Eq. 13) and exact triangle predicate.
//   k_resolve64   FP64 re-evaluation of the pairs the FP32 filter could not
//                 certify and of FP32 hits whose position bound is too large.
//   k_bary_obs / k_bary_sys   barycentres of the observed systems.
//   k_sort_hits   images of each sample in (source, triangle) order.
//   k_chi2_match / k_chi2_sum   nearest-image matching and the chi^2 of Eq. 11.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lt_internal.cuh"
#include "lt_source.cuh"

namespace lt {

__device__ __forceinline__ int find_sample64(const int64_t* off, int n, int64_t item) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------- preparation
constexpr int kPrepThreads = 256;

// The error-bound coefficients are formed in FP32 with directed rounding
// (GB300 issues an FP64 warp instruction only every ~80 cycles per SM
// sub-partition, and this kernel is one chain of them per potential): every
// quantity that enlarges a bound is rounded up, every divisor down, so each
// result is an upper bound of its formula's exact value.  Constants are
// evaluated in FP64 at compile time and rounded up to float (cup: a relative
// 2^-22 above the value, more than the 2^-24 of the rounding to float).
constexpr double cU = kU32d;
constexpr float cup(double x) { return (float)(x * (1.0 + 0x1p-22)); }
constexpr double gamc(double n) { return n / (1.0 - n * cU); }  // gamma(n) for n u << 1
// gamma(n) = n / (1 - n u) of a runtime n >= 0, rounded up; 1e30 once n u >= 1/4
__device__ __forceinline__ float gam_up(float n) {
  const float nu = __fmul_ru(n, kU32);
  return nu >= 0.25f ? 1e30f : __fdiv_ru(n, __fsub_rd(1.0f, nu));
}
constexpr double cM7 = 4.0 + (kEpsRsqrt > kEpsSqrt - 1.0 ? kEpsRsqrt : kEpsSqrt - 1.0) + kEpsRcp;
constexpr double cNtx = cM7 + 13.0 + kEpsRsqrt + kEpsSqrt + kEpsRcp;
// SIS: P, Q, Q2 and T per unit b0
constexpr float kP0Sis = cup(8.0 * (1.0 + cU) / ((1.0 - 3.1 * cU) * (1.0 - (1.01 + kEpsRsqrt) * cU)));
constexpr float kQSis = cup(gamc(3.0 + kEpsRsqrt) + 3.0 * (1.0 + 3.0 * cU));
constexpr float kQ2Sis = cup(gamc(3.0 + kEpsRsqrt) + 1.01);
constexpr float kTSis = cup(1.41421357 * (1.0 + gamc(5.0 + kEpsRsqrt) * cU));
// SIE: per unit b0 r2 (and 1/r1 terms)
constexpr float kP0Sie = cup(11.32 * (1.0 + 3.0 * cU) / (1.0 - (1.01 + kEpsRsqrt) * cU));
constexpr float kP0SieR1 = cup(16.1 * cU);
constexpr float kGSie = cup(gamc(5.25 + kEpsRsqrt));
constexpr float kQSieR1 = cup(16.04 * (1.0 + 3.0 * cU));
constexpr float kQ2SieR1 = cup(10.1 * (1.0 + 3.0 * cU));
constexpr float kTSie = cup(1.41421357 * (1.0 + gamc(6.25 + kEpsRsqrt) * cU));
// PIEMD
constexpr float kC8 = cup(8.0 + kEpsRsqrt + kEpsSqrt);
constexpr float kNty0 = cup(cM7 + 4.0 + kEpsRcp);
constexpr float kGx = cup(gamc(cNtx + kEpsAtanc + 3.5));
constexpr float kEpsAtanhcF = cup(kEpsAtanhc), kEpsAtanhcLogF = cup(kEpsAtanhcLog);
constexpr float kP0Piemd = cup(2.8285 * (1.0 + 3.0 * cU) / (1.0 - (2.0 + kEpsRsqrt) * cU));
constexpr float kQPiemd = cup(16.04 * (1.0 + 3.0 * cU));
constexpr float kQ2Piemd = cup(10.1 * (1.0 + 3.0 * cU));
constexpr float kAtanF = cup(1.0 + (kEpsAtanc + 0.1) * cU);
constexpr float kT2u = cup(1.0 + 2.0 * cU);

__device__ __forceinline__ bool valid_params(const double* v, int* kind_out) {
  bool ok = true;
  for (int r = 0; r < LT_N_ROWS; ++r) ok = ok && isfinite(v[r]);
  int kind = ok ? (int)v[LT_ROW_KIND] : -1;
  ok = ok && (double)kind == v[LT_ROW_KIND] && kind >= 0 && kind <= 2 && v[LT_ROW_SIGMA] >= 0.0;
  if (ok && kind != LT_SIS) ok = v[LT_ROW_E] >= 0.0 && v[LT_ROW_E] < 1.0;
  if (ok && kind == LT_PIEMD) ok = v[LT_ROW_RCORE] > 0.0 && v[LT_ROW_RCUT] > v[LT_ROW_RCORE];
  *kind_out = ok ? kind : LT_SIS;
  return ok;
}

// Summation weights of the potential at kind-sorted position r, for the
// chunk / kind-segment / group order of the FP32 deflection: *w_partial the
// accumulation steps whose partial sum contains its term (its own and the
// later steps of its group), *w_flush the group flushes whose total contains
// it (its group's and every later one).
__device__ void sum_weights(int r, int n_pot, int n_sis, int n_piemd, int* w_partial,
                            int* w_flush) {
  int groups = 0, mine = 0;
  *w_partial = 1;
  for (int c0 = 0; c0 < n_pot; c0 += kChunk32) {
    const int cn = min(kChunk32, n_pot - c0);
    const int seg[4] = {0, min(max(n_sis - c0, 0), cn), min(max(n_sis + n_piemd - c0, 0), cn),
                        cn};
    for (int t = 0; t < 3; ++t)
      for (int k0 = seg[t]; k0 < seg[t + 1]; k0 += kSumGroup) {
        const int k1 = min(k0 + kSumGroup, seg[t + 1]);
        if (r >= c0 + k0 && r < c0 + k1) {
          mine = groups;
          *w_partial = c0 + k1 - r;
        }
        ++groups;
      }
  }
  *w_flush = groups - mine;
}

// One block per sample.  Pass 1 validates every potential and writes its
// FP64 record (invalid ones are latched and neutralised to a zero-mass SIS);
// pass 2 ranks potentials kind-major in index order (block-wide ballot
// prefix counts) and writes the FP32 record at that rank, so the FP32 kernel
// loops over kind segments.
__global__ void __launch_bounds__(kPrepThreads)
    k_prep(const double* __restrict__ params, int n_pot, Pot64* __restrict__ pot64,
           Pot32* __restrict__ pot32, Seg32* __restrict__ seg, uint32_t* status) {
  constexpr int NW = kPrepThreads / 32;
  const int b = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double* P = params + (int64_t)b * LT_N_ROWS * n_pot;
  Pot64* p64 = pot64 + (int64_t)b * n_pot;
  __shared__ int cnt[3];
  __shared__ int wcnt[3][NW];
  __shared__ float qpart[NW], cpart[NW], tpart[NW];
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < n_pot; k += kPrepThreads) {
    double v[LT_N_ROWS];
    for (int r = 0; r < LT_N_ROWS; ++r) v[r] = P[(int64_t)r * n_pot + k];
    int kind;
    if (!valid_params(v, &kind)) {
      atomicOr(status, ST_NONFINITE);
      for (int r = 0; r < LT_N_ROWS; ++r) v[r] = 0.0;
    }
    Pot64 p;
    p.kind = (double)kind;
    p.cx = v[LT_ROW_X];
    p.cy = v[LT_ROW_Y];
    sincos(v[LT_ROW_PHI], &p.s, &p.c);
    double t = v[LT_ROW_SIGMA] / kC;
    p.b0 = 4.0 * kPi * t * t * kArcsec;
    p.e = v[LT_ROW_E];
    p.q = 1.0 - p.e;
    p.k2 = (1.0 - p.q) * (1.0 + p.q);
    p.q2 = p.q * p.q;
    p.a = v[LT_ROW_RCORE];
    p.sc = v[LT_ROW_RCUT];
    p.scale = kind == LT_PIEMD ? p.b0 * (p.sc / (p.sc - p.a)) : 0.0;
    p.sv = v[LT_ROW_SIGMA];
    p.k = sqrt(p.k2);
    p.ik = p.k > 0.0 ? 1.0 / p.k : 0.0;
    p64[k] = p;
    atomicAdd(&cnt[kind], 1);
  }
  __syncthreads();
  float qsum = 0.0f, csum = 0.0f, tsum = 0.0f;
  int base[3] = {0, 0, 0};  // potentials of each kind in earlier chunks
  for (int k0 = 0; k0 < n_pot; k0 += kPrepThreads) {
    const int k = k0 + threadIdx.x;
    const bool act = k < n_pot;
    Pot64 p;
    int kind = -1;
    if (act) {
      p = p64[k];
      kind = (int)p.kind;
    }
    // rank = potentials of a lower kind + potentials of this kind before k
    int before = 0;
    for (int j = 0; j < 3; ++j) {
      const unsigned m = __ballot_sync(0xffffffffu, kind == j);
      if (lane == 0) wcnt[j][wid] = __popc(m);
      if (kind == j) before = __popc(m & ((1u << lane) - 1u));
    }
    __syncthreads();
    int rank = 0;
    if (act) {
      for (int j = 0; j < kind; ++j) rank += cnt[j];
      rank += base[kind] + before;
      for (int w = 0; w < wid; ++w) rank += wcnt[kind][w];
    }
    for (int j = 0; j < 3; ++j)
      for (int w = 0; w < NW; ++w) base[j] += wcnt[j][w];
    __syncthreads();
    if (!act) continue;
    Pot32 f;
    for (int w = 0; w < 5; ++w) f.f[w] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float cx = (float)p.cx, cy = (float)p.cy, c = (float)p.c, s = (float)p.s;
    // Coefficients of the FP32 running error bound, in units of u = 2^-24
    // (every constant below is rounded up to float).  The bound of a node is
    //   E = (1 + 2^-16) u [ sum_k P_k / d_k + sum_k (Gx_k |gx_k| + Gy_k |gy_k|)
    //                       + sum_k Q_k + summation terms ],
    // d_k the node's FP32 distance measure to potential k (|theta - c| for the
    // SIS, R for the SIE, psi_a for the PIEMD).  It bounds both components
    // of |alpha_FP32 - alpha|, alpha the exact deflection at the FP64 node
    // position with the FP64 parameters.  Derivation, term by term:
    //  * input errors: the node coordinate (rounded once from FP64), the
    //    centre and the translation err by at most 2u(1+u)(Theta + |c_x|) per
    //    coordinate, W = Theta + |c_x| + |c_y|; the rotation (two rounded
    //    coefficients, one product, one FMA) adds 4.01 u |Delta|_1, Delta the
    //    translated node.  They move the deflection by at most
    //    |J|_2 |e|_2, J its Jacobian along the segment between the exact and
    //    the rounded rotated node: P / d carries the W part, Q the |Delta| part;
    //  * evaluation errors: relative errors of the rotated-frame components,
    //    counted operation by operation (each rounding one u, the hardware
    //    approximations and special functions their measured maxima kEps*),
    //    as coefficients G of |g| (PIEMD) or, when |alpha_k| is bounded by a
    //    constant, folded into Q (SIS, SIE);
    //  * accumulation: every fused step errs by at most u (2 + u) max|partial|,
    //    charged per node by the 2 (|PX| + |PY|) and 2 (|AX| + |AY|) terms of
    //    the kernel;
    //  * second order: counted units n enter as gamma(n) = n / (1 - n u)
    //    (Higham, Accuracy and Stability of Numerical Algorithms, Lemma 3.1).
    float Q, T, Q2, Gmax = 0.0f;
    if (kind == LT_SIS) {
      // Jacobian of b0 n(Delta): b0/|Delta| (2-norm).  Where |D| >= 2|e|:
      // error <= 2 b0 |e| / |D| with |e| <= u(1+u)(W2 + |Delta|), W2 =
      // 2 Theta + |c_x| + |c_y| <= 2 W: P = 4 b0 W, and the |Delta| part
      // (|Delta| <= 1.5 |D|) gives 3 b0 in Q.  Where |D| < 2|e| the error is
      // at most 2 b0 (two vectors of length b0), which P / |D| covers with
      // P >= 4 b0 |e| / u: P = 8 b0 W.  rr = rsqrt(R2) errs by (1.01 + eps_r) u.
      // Evaluation: b0 (1 u), R2 (2 u, halved by the root), rsqrt, b0 * rr
      // (1 u): 3 + eps_r relative, |alpha_k| <= b0, into Q.
      const float b0u = __double2float_ru(p.b0);
      f.f[0] = make_float4(cx, cy, (float)p.b0, 0.f);
      f.f[4] = make_float4(__fmul_ru(kP0Sis, b0u), 0.f, 0.f, 0.f);
      Q = __fmul_ru(kQSis, b0u);
      // tight re-evaluation (node translated in FP64, rounded once: error
      // u (1 + 2^-28) |Delta| per coordinate, so |e| <= 1.0001 u |Delta|):
      // the Jacobian b0/|Delta| gives 1.01 u b0, with the evaluation terms
      Q2 = __fmul_ru(kQ2Sis, b0u);
      // |t_x| + |t_y| = g (|dx| + |dy|) <= sqrt(2) b0 (1 + (3 + eps_r) u)
      T = __fmul_ru(kTSis, b0u);
    } else if (kind == LT_SIE) {
      const double r1 = sqrt(1.0 - p.e), r2 = sqrt(1.0 + p.e);
      // z = (r1 x', r2 y'), g = b0 diag(r1, r2) z / |z|: Jacobian in z at most
      // b0 r2 / |z|; the input error in z is at most sqrt(2) u (1+3u)
      // (W2 + 4.01 |Delta|_1) (r1^2 + r2^2 = 2).  Where |z| >= 2|e_z|: the W
      // part gives P = 2 sqrt(2) b0 r2 W2 <= 5.66 b0 r2 W and the |Delta| part
      // (|Delta|_1 <= sqrt(2) |z| / r1 (1 + ...)) Q = 16.04 b0 r2 / r1; where
      // |z| < 2 |e_z| (then |Delta|_1 < 2 sqrt(2) |e_z| / r1) the error is at
      // most 2 b0 r2, covered by P = 4 sqrt(2) b0 r2 W2 / (1 - 16.04 u / r1)
      // <= 11.32 b0 r2 W / (...).  Evaluation of t = b0 R(-phi) (r1 u, r2 v):
      // three roundings on each product term, |t| <= b0 r2 R, so
      // |t_FP32 - t| <= 3 sqrt(2) u b0 r2 R; times rr ((1.01 + eps_r) u):
      // (5.25 + eps_r) b0 r2 into Q.
      const float r1d = __double2float_rd(r1);
      const float b0r2 = __fmul_ru(__double2float_ru(p.b0), __double2float_ru(r2));
      const float den1 = __fsub_rd(1.0f, __fdiv_ru(kP0SieR1, r1d));
      const float p0 = den1 > 0.0f ? __fdiv_ru(__fmul_ru(kP0Sie, b0r2), den1) : 1e30f;
      f.f[0] = make_float4(cx, cy, (float)(r1 * p.c), (float)(r1 * p.s));
      f.f[1] = make_float4((float)(r2 * p.c), (float)(r2 * p.s), (float)(p.b0 * r1 * p.c),
                           (float)(p.b0 * r2 * p.s));
      f.f[2] = make_float4((float)(p.b0 * r2 * p.c), (float)(p.b0 * r1 * p.s), 0.f, 0.f);
      f.f[4] = make_float4(p0, 0.f, 0.f, 0.f);
      Q = __fmul_ru(b0r2, __fadd_ru(kGSie, __fdiv_ru(kQSieR1, r1d)));
      // tight re-evaluation: translation error 1.0001 u |Delta|_1 and the
      // rotation's 4.01 u |Delta|_1, so |e_z| <= sqrt(2) 5.02 u (1+3u) |Delta|_1
      // <= 10.04 u (1+3u) |z| / r1, far below |z| / 2: 10.1 b0 r2 / r1 with
      // the evaluation terms (r1 < 1e-3 is not bounded)
      Q2 = r1 < 1e-3 ? 1e30f : __fmul_ru(b0r2, __fadd_ru(kGSie, __fdiv_ru(kQ2SieR1, r1d)));
      // |t_x| + |t_y| <= sqrt(2) |rr (t1, t2)| <= sqrt(2) b0 r2 (1 + (6.25 + eps_r) u)
      T = __fmul_ru(kTSie, b0r2);
    } else {
      const double a = p.a, sc = p.sc, q2 = p.q2, q = p.q;
      const double B = p.scale;
      // sig = sqrt(k2) is folded into the ds coefficients, so the kernel forms
      // sig*t directly and (sig t)^2 = k2 t^2 in one product; B/sig and the
      // rotation back are folded into (Bc, Bs).  For a circular PIEMD (k2 = 0)
      // sig is 1e-8: then (sig t)^2 < 1e-16 (|t| < 1 there) instead of 0, a
      // relative change of atan(sig t)/(sig t) far below the FP32 roundoff.
      const double sig = sqrt(fmax(p.k2, 1e-16)), Bs = B / sig;
      f.f[0] = make_float4(cx, cy, c, s);
      f.f[1] = make_float4((float)q2, (float)(q2 * a * a), (float)(q2 * sc * sc), (float)p.k2);
      f.f[2] = make_float4((float)a, (float)sc, (float)(q2 * a), (float)(q2 * sc));
      f.f[3] = make_float4((float)(sig * (sc - a)), (float)(sig * q2 * (sc + a) * (sc - a)),
                           (float)(sig * q2 * (sc - a)), (float)(Bs * p.c));
      // Evaluation at the rounded rotated node (x, y), relative errors in u
      // (each record constant, product, sum and FMA one u; sums of positive
      // terms keep the larger relative error):
      //   psi_a^2, psi_s^2: 4; pa = psi_a: 3 + eps_r (rsqrt, times psi_a^2);
      //   ps: 2 + eps_s; 1/(pa + ps): m7 = 4 + max(eps_r, eps_s - 1) + eps_rcp;
      //   ds_x, ds_y: m7 + 2; (pa + a)(ps + s), (pa + q2 a)(ps + q2 s):
      //   8 + eps_r + eps_s; den_x (a sum of positive terms): 9 + eps_r + eps_s;
      //   den_y = p_y - k2 y^2 >= q^2 p_y (y^2 <= psi_a psi_s <= p_y), so
      //   (8 + eps_r + eps_s + 2 k2)/q^2 + 1; t_x = x ds_x rcp(den_x):
      //   n_tx = m7 + 13 + eps_r + eps_s + eps_rcp; t_y: n_ty = m7 + 4 +
      //   eps_rcp + that of den_y.
      //   g_x = atan(t_x): elasticity of atan <= 1, the rounded square 1 u at
      //   elasticity <= 1/2, the special function eps_atanc, the product 1 u;
      //   g_y = atanh(t_y): elasticity <= 1/(1 - t_y^2) <= 1/q^2 (|t_y| < k),
      //   the square at k2/(2 q^2), eps_atanhc, 1 u.  Two more units for the
      //   rounded (Bc, Bs) and the inner FMA of the accumulation.
      // (m7 = 4 + max(eps_r, eps_s - 1) + eps_rcp, n_tx = m7 + 13 + eps_r +
      // eps_s + eps_rcp: constants, folded into kNty0 and kGx.)
      const float qd = __double2float_rd(q), q2d = __double2float_rd(q2);
      const float k2u = __double2float_ru(p.k2), Bu = __double2float_ru(B);
      const float sgu = __double2float_ru(sig), Bsu = __fdiv_ru(Bu, __double2float_rd(sig));
      const float c_dy = __fadd_ru(__fdiv_ru(__fmaf_ru(2.0f, k2u, kC8), q2d), 1.0f);
      const float n_ty = __fadd_ru(kNty0, c_dy);
      // q < 0.01 (e > 0.99): the atan argument (below 1/q) leaves the range
      // over which kEpsAtanc is measured, and the bound is not finite
      const bool flat = q < 0.01;
      const float Gx = flat ? 1e30f : kGx;
      // 1/(q^2 - 3 n_ty u): the elasticity along the perturbed path
      const float eld = __fsub_rd(q2d, __fmul_ru(3.0f * kU32, n_ty));
      const float el = eld > 0.0f ? __frcp_ru(eld) : 1e30f;
      // atanh(t)/t: the polynomial's error, or the logarithm's divided by
      // 1 - t_y^2 >= q^2 - 3 n_ty u
      const float eps_h = fmaxf(kEpsAtanhcF, __fmul_ru(kEpsAtanhcLogF, el));
      const float Gy = flat || !(eld > 0.0f)
                           ? 1e30f
                           : gam_up(__fadd_ru(__fadd_ru(__fmaf_ru(n_ty, el, __fmul_ru(__fmul_ru(0.5f, k2u), el)),
                                                        eps_h),
                                              3.0f));
      // Input errors (rotated frame, 2-norm): |e'| <= sqrt(2) u (1+3u)
      // (W2 + 4.01 |Delta|_1), W2 <= 2 W.  The Jacobian of the dPIE in the
      // rotated frame, per unit B, is H_a - H_s with H_w positive
      // semidefinite of trace 1/psi_w, so |H|_2 <= 1/psi_a, and psi_a has
      // gradient norm <= 1 and psi_a >= q a, psi_a >= q |Delta|.  With
      // x_k = 14.18 (1+3u) u W / (q a) (>= |e'| / psi_a): if x_k <= 1/2 the W
      // part gives P = 2 sqrt(2) B W / (1 - x_k) (staging applies the
      // factor; errP0 = 2 sqrt(2) B (1+3u) / (1 - (2 + eps_r) u), ra errs by
      // (2 + eps_r) u) and the |Delta| part Q = 16.04 B / q; otherwise P =
      // 28.36 B W max(1, x_k) covers all input errors (stage_p32).
      f.f[4] = make_float4(__fmul_ru(kP0Piemd, Bu), __fmul_ru(Gx, Bsu), __fmul_ru(Gy, Bsu),
                           (float)(Bs * p.s));
      Q = __fdiv_ru(__fmul_ru(kQPiemd, Bu), qd);
      // tight re-evaluation: the input errors are relative to the distance,
      // |e'| <= sqrt(2) 5.02 u (1+3u) |Delta|_1 <= 10.04 u (1+3u) |Delta|, and
      // psi_a >= q |Delta| along the segment (|e'| / psi_a <= 10.04 u / q is
      // negligible for q >= 0.01), so B |H|_2 |e'| <= 10.1 (1+3u) u B / q; the
      // evaluation terms stay per node (G)
      Q2 = flat ? 1e30f : __fdiv_ru(__fmul_ru(kQ2Piemd, Bu), qd);
      // coarse bound: the largest |gx|, |gy| over the plane.  |g_x| =
      // |atan(A) - atan(B)| <= atan(sig/q) (0 <= B <= A < sig/q) and |g_y| <=
      // atanh(sig) (the two atanh arguments lie in (-sig, sig) with one sign),
      // each times its evaluation factor 1 + G u.  Both from the FP32
      // functions whose errors are measured over every float argument:
      // atan(x) = x atanc(x^2) <= x_up atanc_sq32(x_dn^2) (1 + (eps_atanc + 0.1) u)
      // (atan(t)/t decreases in t^2), and atanh(s) = s atanhc(s^2) <= s_up
      // atanhc_sq32(s_up^2) (1 + (eps + 0.1) u), eps the polynomial's error or the
      // logarithm's divided by 1 - s^2 (atanh(t)/t increases in t^2).
      const float xu = __fdiv_ru(sgu, qd);
      const float xd = __fdiv_rd(__double2float_rd(sig), __double2float_ru(q));
      const float atn = __fmul_ru(__fmul_ru(xu, atanc_sq32(fminf(__fmul_rd(xd, xd), 16384.0f))),
                                  kAtanF);
      const float s2 = fminf(__fmul_ru(sgu, sgu), 0.99999988f);
      const float eh = s2 <= 0.25f ? kEpsAtanhcF : __fdiv_ru(kEpsAtanhcLogF, __fsub_rd(1.0f, s2));
      const float atnh = __fmul_ru(__fmul_ru(fminf(sgu, 0.99999994f), atanhc_sq32(s2)),
                                   __fmaf_ru(__fadd_ru(eh, 0.1f), kU32, 1.0f));
      const float mgx = __fmul_ru(atn, __fmaf_ru(Gx, kU32, 1.0f));
      const float mgy = __fmul_ru(atnh, __fmaf_ru(Gy, kU32, 1.0f));
      Gmax = __fmul_ru(Bsu, __fmaf_ru(Gx, mgx, __fmul_ru(Gy, mgy)));
      // |t_x| + |t_y| <= (B/sig)(|c| + |s|)(|gx| + |gy|)(1 + u)
      T = __fmul_ru(__fmul_ru(__fmul_ru(Bsu, __double2float_ru(fabs(p.c) + fabs(p.s))),
                              __fadd_ru(mgx, mgy)),
                    kT2u);
    }
    qsum = __fadd_ru(qsum, Q);
    tsum = __fadd_ru(tsum, Q2);
    // coarse bound: Q, the largest evaluation terms, and every accumulation
    // step's 2 (|PX| + |PY|) and flush's 2 (|AX| + |AY|) bounded by the
    // largest terms they can contain
    int w_partial, w_flush;
    sum_weights(rank, n_pot, cnt[LT_SIS], cnt[LT_PIEMD], &w_partial, &w_flush);
    csum = __fadd_ru(csum, __fadd_ru(__fadd_ru(Q, Gmax),
                                     __fmul_ru(__fmul_ru(2.0f, T), (float)(w_partial + w_flush))));
    f.c64 = make_double2(p.cx, p.cy);
    pot32[(int64_t)b * n_pot + rank] = f;
  }
  // sum of the static bound terms (rounded up): fixed order (warp
  // butterflies, then warps)
  for (int o = 16; o > 0; o >>= 1) {
    qsum = __fadd_ru(qsum, __shfl_xor_sync(0xffffffffu, qsum, o));
    tsum = __fadd_ru(tsum, __shfl_xor_sync(0xffffffffu, tsum, o));
    csum = __fadd_ru(csum, __shfl_xor_sync(0xffffffffu, csum, o));
  }
  if (lane == 0) {
    qpart[wid] = qsum;
    tpart[wid] = tsum;
    cpart[wid] = csum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.0f, ctot = 0.0f, ttot = 0.0f;
    for (int w = 0; w < NW; ++w) {
      tot = __fadd_ru(tot, qpart[w]);
      ttot = __fadd_ru(ttot, tpart[w]);
      ctot = __fadd_ru(ctot, cpart[w]);
    }
    seg[b] = Seg32{cnt[LT_SIS], cnt[LT_PIEMD], cnt[LT_SIE], tot, ctot, ttot};
  }
}

__global__ void k_zero64(unsigned long long* a, int64_t na, unsigned long long* b, int64_t nb,
                         unsigned long long* c, int64_t nc, unsigned long long* d, int64_t nd) {
  const int64_t n = na + nb + nc + nd;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = i;
    if (k < na) { a[k] = 0ull; continue; }
    k -= na;
    if (k < nb) { b[k] = 0ull; continue; }
    k -= nb;
    if (k < nc) { c[k] = 0ull; continue; }
    k -= nc;
    d[k] = 0ull;
  }
}

cudaError_t launch_zero64(unsigned long long* a, int64_t na, unsigned long long* b, int64_t nb,
                          unsigned long long* c, int64_t nc, unsigned long long* d, int64_t nd,
                          cudaStream_t st) {
  if (!a) na = 0;
  if (!b) nb = 0;
  if (!c) nc = 0;
  if (!d) nd = 0;
  const int64_t n = na + nb + nc + nd;
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_zero64<<<(unsigned)blocks, 256, 0, st>>>(a, na, b, nb, c, nc, d, nd);
  return cudaGetLastError();
}

cudaError_t launch_prep(const double* params, int batch, int n_pot, Pot64* pot64, Pot32* pot32,
                        Seg32* seg, uint32_t* status, cudaStream_t st) {
  k_prep<<<batch, kPrepThreads, 0, st>>>(params, n_pot, pot64, pot32, seg, status);
  return cudaGetLastError();
}

// ----------------------------------------------------------- FP64 deflection
constexpr int kDefl64Threads = 128;
constexpr int kChunk64 = 64;

__global__ void __launch_bounds__(kDefl64Threads)
    k_deflect64(const Pot64* __restrict__ pot64, int n_pot, const SampleGrid* __restrict__ grids,
                const int64_t* __restrict__ item_off, int n_samples, int64_t n_items,
                double2* __restrict__ node_out) {
  __shared__ Pot64 sp[kChunk64];
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int b = find_sample64(item_off, n_samples, item);
    const SampleGrid g = grids[b];
    const int64_t nodes = (int64_t)g.nx * g.ny;
    int64_t n = (item - item_off[b]) * kDefl64Threads + threadIdx.x;
    const bool valid = n < nodes;
    if (!valid) n = nodes - 1;
    const int j = (int)(n / g.nx);
    const int i = (int)(n - (int64_t)j * g.nx);
    const double x = g.x0 + (double)i * g.dx;
    const double y = g.y0 + (double)j * g.dy;
    double ax = 0.0, ay = 0.0;
    const Pot64* pb = pot64 + (int64_t)b * n_pot;
    for (int c0 = 0; c0 < n_pot; c0 += kChunk64) {
      const int cn = min(kChunk64, n_pot - c0);
      __syncthreads();
      for (int k = threadIdx.x; k < cn; k += kDefl64Threads) sp[k] = pb[c0 + k];
      __syncthreads();
      for (int k = 0; k < cn; ++k) {
        double kx, ky;
        alpha64_one(sp[k], x, y, kx, ky);
        ax = ax + kx;
        ay = ay + ky;
      }
    }
    if (valid) node_out[g.node_off + n] = make_double2(ax, ay);
  }
}

cudaError_t launch_deflect64(const Pot64* pot64, int n_pot, const SampleGrid* grids,
                             const int64_t* item_off, int n_samples, int64_t n_items,
                             double2* node_out, int sm_count, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deflect64, kDefl64Threads, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)sm_count * per_sm;
  if (blocks > n_items) blocks = n_items;
  k_deflect64<<<(unsigned)blocks, kDefl64Threads, 0, st>>>(pot64, n_pot, grids, item_off,
                                                           n_samples, n_items, node_out);
  return cudaGetLastError();
}

// ------------------------------------------------------ exact FP64 predicate
// Edge function e(a, b, p) = (b - a) x (p - a), each operation rounded.
__device__ __forceinline__ double edge64(double ax, double ay, double bx, double by, double px,
                                         double py) {
  double t1 = (bx - ax) * (py - ay);
  double t2 = (by - ay) * (px - ax);
  return t1 - t2;
}
__device__ __forceinline__ bool owned64(double dx, double dy) {
  return dy > 0.0 || (dy == 0.0 && dx < 0.0);
}

// Containment of P in the mapped triangle (A, B, C): parity follows the sign
// of the determinant, zero determinant is skipped, points on an edge belong
// to the counter-clockwise edge with dy > 0 (or dy == 0, dx < 0).
__device__ __forceinline__ bool in_tri64(double Ax, double Ay, double Bx, double By, double Cx,
                                         double Cy, double Px, double Py, double w[3]) {
  double det = edge64(Ax, Ay, Bx, By, Cx, Cy);
  if (det == 0.0) return false;
  double e[3] = {edge64(Ax, Ay, Bx, By, Px, Py), edge64(Bx, By, Cx, Cy, Px, Py),
                 edge64(Cx, Cy, Ax, Ay, Px, Py)};
  double fx[3] = {Ax, Bx, Cx}, fy[3] = {Ay, By, Cy};
  double s = det > 0.0 ? 1.0 : -1.0;
  for (int k = 0; k < 3; ++k) {
    double se = s * e[k];
    if (se > 0.0) continue;
    if (se < 0.0) return false;
    int k1 = k == 2 ? 0 : k + 1;
    double dx = s > 0.0 ? fx[k1] - fx[k] : fx[k] - fx[k1];
    double dy = s > 0.0 ? fy[k1] - fy[k] : fy[k] - fy[k1];
    if (!owned64(dx, dy)) return false;
  }
  w[0] = e[1] / det;
  w[1] = e[2] / det;
  w[2] = e[0] / det;
  return true;
}

__device__ __forceinline__ void append_hit(const Hit& h, Hit* hits, int64_t cap,
                                           unsigned long long* count, uint32_t* status) {
  unsigned long long idx = atomicAdd(count, 1ull);
  if (idx < (unsigned long long)cap) hits[idx] = h;
  else atomicOr(status, ST_OVERFLOW_HITS);
}

__device__ __forceinline__ void warp_append_hit64(bool flag, const Hit& h, Hit* hits,
                                                  int64_t cap, unsigned long long* count,
                                                  uint32_t* status) {
  unsigned mask = __ballot_sync(0xffffffffu, flag);
  if (!mask) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (flag) {
    unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
    if (idx < (unsigned long long)cap) hits[idx] = h;
    else atomicOr(status, ST_OVERFLOW_HITS);
  }
}

// ------------------------------------------------------------ FP64 search
constexpr int kSearch64Threads = 128;

__global__ void __launch_bounds__(kSearch64Threads)
    k_search64(const double2* __restrict__ nodes, const SampleGrid* __restrict__ grids,
               const int64_t* __restrict__ item_off, int n_samples, int64_t n_items, Sources src,
               Hit* __restrict__ hits, int64_t hit_cap, unsigned long long* hit_count,
               long long* counters, uint32_t* status) {
  long long n_hit = 0;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int b = find_sample64(item_off, n_samples, item);
    const SampleGrid g = grids[b];
    const int sample = src.sample_base + b;
    const int64_t cells = (int64_t)(g.nx - 1) * (g.ny - 1);
    const int64_t cell = (item - item_off[b]) * kSearch64Threads + threadIdx.x;
    const bool valid = cell < cells;
    const int64_t cl = valid ? cell : 0;
    const int j = (int)(cl / (g.nx - 1));
    const int i = (int)(cl - (int64_t)j * (g.nx - 1));
    const int64_t n00 = g.node_off + (int64_t)j * g.nx + i;
    const double2 a00 = nodes[n00], a10 = nodes[n00 + 1], a01 = nodes[n00 + g.nx],
                  a11 = nodes[n00 + g.nx + 1];
    const double X0 = g.x0 + (double)i * g.dx, X1 = g.x0 + (double)(i + 1) * g.dx;
    const double Y0 = g.y0 + (double)j * g.dy, Y1 = g.y0 + (double)(j + 1) * g.dy;
    const double* sxy = src.xy + (int64_t)sample * src.n_src * 2;
    const double* sr = src.r + (int64_t)sample * src.n_src * (src.stride_r ? 1 : 0);
    for (int k = 0; k < src.n_src; ++k) {
      const double Px = sxy[2 * k], Py = sxy[2 * k + 1], r = sr[k];
      // the mixed path's input domain: a finite position and 0 <= r < 1e30;
      // anything else is latched and the source has no images
      if (!source_ok(Px, Py, r)) {
        if (threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
        continue;
      }
      // mapped vertices beta = theta - r alpha (Eq. 13)
      const double b00x = X0 - r * a00.x, b00y = Y0 - r * a00.y;
      const double b10x = X1 - r * a10.x, b10y = Y0 - r * a10.y;
      const double b01x = X0 - r * a01.x, b01y = Y1 - r * a01.y;
      const double b11x = X1 - r * a11.x, b11y = Y1 - r * a11.y;
      // exact bounding-box rejection: a point strictly outside cannot be inside
      const double minx = fmin(fmin(b00x, b10x), fmin(b01x, b11x));
      const double maxx = fmax(fmax(b00x, b10x), fmax(b01x, b11x));
      const double miny = fmin(fmin(b00y, b10y), fmin(b01y, b11y));
      const double maxy = fmax(fmax(b00y, b10y), fmax(b01y, b11y));
      bool cand = valid && !(Px < minx || Px > maxx || Py < miny || Py > maxy);
      bool in0 = false, in1 = false;
      double w0[3] = {0, 0, 0}, w1[3] = {0, 0, 0};
      if (cand) {
        in0 = in_tri64(b00x, b00y, b10x, b10y, b11x, b11y, Px, Py, w0);
        in1 = in_tri64(b00x, b00y, b11x, b11y, b01x, b01y, Px, Py, w1);
      }
      if (__any_sync(0xffffffffu, in0 || in1)) {
        Hit h;
        h.src = k;
        h.fp64 = 1;
        h.tri = 2 * cl;
        h.w[0] = w0[0]; h.w[1] = w0[1]; h.w[2] = w0[2];
        h.x = w0[0] * X0 + w0[1] * X1 + w0[2] * X1;
        h.y = w0[0] * Y0 + w0[1] * Y0 + w0[2] * Y1;
        Hit* hb = hits + (int64_t)b * hit_cap;
        warp_append_hit64(in0, h, hb, hit_cap, hit_count + b, status);
        h.tri = 2 * cl + 1;
        h.w[0] = w1[0]; h.w[1] = w1[1]; h.w[2] = w1[2];
        h.x = w1[0] * X0 + w1[1] * X1 + w1[2] * X0;
        h.y = w1[0] * Y0 + w1[1] * Y1 + w1[2] * Y1;
        warp_append_hit64(in1, h, hb, hit_cap, hit_count + b, status);
        n_hit += (int)in0 + (int)in1;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) n_hit += __shfl_xor_sync(0xffffffffu, n_hit, o);
  if ((threadIdx.x & 31) == 0 && n_hit)
    atomicAdd((unsigned long long*)&counters[CNT_HITS], (unsigned long long)n_hit);
}

cudaError_t launch_search64(const double2* nodes, const SampleGrid* grids, const int64_t* item_off,
                            int n_samples, int64_t n_items, Sources src, Hit* hits,
                            int64_t hit_cap, unsigned long long* hit_count, long long* counters,
                            uint32_t* status, int sm_count, cudaStream_t st) {
  if (n_items <= 0 || src.n_src <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search64, kSearch64Threads, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)sm_count * per_sm;
  if (blocks > n_items) blocks = n_items;
  k_search64<<<(unsigned)blocks, kSearch64Threads, 0, st>>>(nodes, grids, item_off, n_samples,
                                                            n_items, src, hits, hit_cap,
                                                            hit_count, counters, status);
  return cudaGetLastError();
}


// ------------------------------------------------------------ FP64 resolution
// The FP64 work items of a chunk (ambiguous (triangle, source) pairs and hits
// to refine) share many triangle nodes: the two triangles of a cell, and the
// cells around a source that several systems' barycentres sit near.  Each
// distinct node is evaluated in FP64 once:
//   k_res_insert  one thread per (item, vertex): key (chunk-local sample,
//                 node index) into an open-addressing table (linear probing,
//                 capacity >= twice the number of vertices, so it cannot
//                 fill); the thread that inserts a key appends its slot to
//                 the list of distinct nodes;
//   (the tight FP32 stage, launch_tight32: each distinct node re-evaluated
//                 with its tight bound and every item classified again; the
//                 items it decides are done)
//   k_res_nodes   one block per node of an item still undecided: FP64
//                 deflection summed in potential index order (block_alpha64);
//   k_res_tri     one thread per item still undecided: exact FP64 predicates
//                 with the tie rule and the FP64 barycentric position.
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kResNodeThreads = 128;

__device__ __forceinline__ unsigned long long res_hash(unsigned long long k) {
  // splitmix64 finaliser
  k ^= k >> 30;
  k *= 0xbf58476d1ce4e5b9ull;
  k ^= k >> 27;
  k *= 0x94d049bb133111ebull;
  k ^= k >> 31;
  return k;
}

__device__ __forceinline__ void tri_vertex(const SampleGrid& g, int64_t tri, int v, int& i, int& j) {
  const int64_t cell = tri / 2;
  const int t = (int)(tri % 2);
  i = (int)(cell % (g.nx - 1)) + (v == 0 ? 0 : (v == 1 ? 1 : (t == 0 ? 1 : 0)));
  j = (int)(cell / (g.nx - 1)) + (v == 0 ? 0 : (v == 1 ? (t == 0 ? 0 : 1) : 1));
}

__global__ void k_res_insert(const Work64* __restrict__ work,
                             const unsigned long long* __restrict__ work_count, int n_samples,
                             int64_t work_cap, const SampleGrid* __restrict__ grids,
                             unsigned long long* __restrict__ keys, unsigned long long mask,
                             int32_t* __restrict__ vslot, int32_t* __restrict__ ulist,
                             unsigned int* __restrict__ n_unique) {
  grid_dependency_wait();
  const int64_t total = (int64_t)n_samples * work_cap * 3;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(f / (work_cap * 3));
    const int64_t rem = f - (int64_t)b * work_cap * 3;
    const int64_t idx = rem / 3;
    const int v = (int)(rem - idx * 3);
    const unsigned long long cnt = work_count[b];
    if ((unsigned long long)idx >= (cnt < (unsigned long long)work_cap ? cnt : work_cap)) continue;
    const Work64 wk = work[(int64_t)b * work_cap + idx];
    const SampleGrid g = grids[b];
    int i, j;
    tri_vertex(g, wk.tri, v, i, j);
    const unsigned long long key =
        ((unsigned long long)b << 40) | (unsigned long long)((int64_t)j * g.nx + i);
    unsigned long long h = res_hash(key) & mask;
    int32_t slot = -1;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
      const unsigned long long prev = atomicCAS(&keys[h], kEmptyKey, key);
      if (prev == kEmptyKey) {
        ulist[atomicAdd(n_unique, 1u)] = (int32_t)h;
        slot = (int32_t)h;
        break;
      }
      if (prev == key) {
        slot = (int32_t)h;
        break;
      }
      h = (h + 1) & mask;
    }
    vslot[((int64_t)b * work_cap + idx) * 3 + v] = slot;
  }
}

__global__ void __launch_bounds__(kResNodeThreads)
    k_res_nodes(const Pot64* __restrict__ pot64, int n_pot, int sample_base,
                const SampleGrid* __restrict__ grids, const unsigned long long* __restrict__ keys,
                const int32_t* __restrict__ ulist, const unsigned int* __restrict__ n_unique,
                double2* __restrict__ hval, long long* counters) {
  // ulist / n_unique: the FP64 stage's list (nodes of the items the tight
  // FP32 stage left undecided)
  grid_dependency_wait();
  __shared__ double2 buf[kResNodeThreads];
  __shared__ double res[2];
  const unsigned int nu = *n_unique;
  if (blockIdx.x == 0 && threadIdx.x == 0 && nu)
    atomicAdd((unsigned long long*)&counters[CNT_FP64_NODES], (unsigned long long)nu);
  for (unsigned int u = blockIdx.x; u < nu; u += gridDim.x) {
    const int32_t slot = ulist[u];
    const unsigned long long key = keys[slot];
    const int b = (int)(key >> 40);
    const int64_t node = (int64_t)(key & ((1ull << 40) - 1));
    const SampleGrid g = grids[b];
    const int j = (int)(node / g.nx), i = (int)(node - (int64_t)j * g.nx);
    const double X = g.x0 + (double)i * g.dx;
    const double Y = g.y0 + (double)j * g.dy;
    block_alpha64<kResNodeThreads>(pot64 + (int64_t)(sample_base + b) * n_pot, n_pot, 1, &X, &Y,
                                   &res[0], &res[1], buf);
    if (threadIdx.x == 0) hval[slot] = make_double2(res[0], res[1]);
  }
}

__global__ void k_res_tri(const SampleGrid* __restrict__ grids, Sources src,
                          const Work64* __restrict__ work,
                          const unsigned long long* __restrict__ work_count, int n_samples,
                          int64_t work_cap, const int32_t* __restrict__ vslot,
                          const double2* __restrict__ hval, Hit* __restrict__ hits,
                          int64_t hit_cap, unsigned long long* hit_count, long long* counters,
                          uint32_t* status, unsigned long long* __restrict__ keys,
                          unsigned int* __restrict__ n_unique, uint32_t* __restrict__ flag64,
                          unsigned int* __restrict__ n64) {
  grid_dependency_wait();
  // this kernel is the table's last reader: it leaves the table empty for the
  // next call (the list counts here, every used slot and its flag below)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *n_unique = 0u;
    *n64 = 0u;
  }
  long long n_hit = 0;
  const int64_t total = (int64_t)n_samples * work_cap;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(f / work_cap);
    const int64_t idx = f - (int64_t)b * work_cap;
    const unsigned long long cnt = work_count[b];
    if ((unsigned long long)idx >= (cnt < (unsigned long long)work_cap ? cnt : work_cap)) continue;
    const Work64 wk = work[f];
    // several items may share a slot: they all write the same value
    for (int v = 0; v < 3; ++v) {
      const int32_t slot = vslot[f * 3 + v];
      if (slot >= 0) {
        keys[slot] = kEmptyKey;
        flag64[slot] = 0u;
      }
    }
    if (wk.resolved) continue;  // decided by the tight FP32 stage
    const SampleGrid g = grids[b];
    const double* sxy = src.xy + (int64_t)wk.sample * src.n_src * 2;
    const double r = src.r[(int64_t)wk.sample * src.n_src * (src.stride_r ? 1 : 0) + wk.src];
    const double Px = sxy[2 * wk.src], Py = sxy[2 * wk.src + 1];
    double X[3], Y[3], Bx[3], By[3];
    bool ok = true;
    for (int v = 0; v < 3; ++v) {
      int i, j;
      tri_vertex(g, wk.tri, v, i, j);
      X[v] = g.x0 + (double)i * g.dx;
      Y[v] = g.y0 + (double)j * g.dy;
      const int32_t slot = vslot[f * 3 + v];
      if (slot < 0) { ok = false; break; }
      const double2 a = hval[slot];
      Bx[v] = X[v] - r * a.x;
      By[v] = Y[v] - r * a.y;
    }
    if (!ok) {  // cannot happen with the table sized as it is; recorded, never silent
      atomicOr(status, ST_OVERFLOW_WORK);
      continue;
    }
    double w[3];
    if (in_tri64(Bx[0], By[0], Bx[1], By[1], Bx[2], By[2], Px, Py, w)) {
      Hit h;
      h.src = wk.src;
      h.fp64 = 1;
      h.tri = wk.tri;
      h.w[0] = w[0]; h.w[1] = w[1]; h.w[2] = w[2];
      h.x = w[0] * X[0] + w[1] * X[1] + w[2] * X[2];
      h.y = w[0] * Y[0] + w[1] * Y[1] + w[2] * Y[2];
      append_hit(h, hits + (int64_t)b * hit_cap, hit_cap, hit_count + b, status);
      ++n_hit;
    }
  }
  for (int o = 16; o > 0; o >>= 1) n_hit += __shfl_xor_sync(0xffffffffu, n_hit, o);
  if ((threadIdx.x & 31) == 0 && n_hit)
    atomicAdd((unsigned long long*)&counters[CNT_HITS], (unsigned long long)n_hit);
}

cudaError_t launch_resolve64(const Pot64* pot64, const Pot32* pot32, const Seg32* seg, int n_pot,
                             const SampleGrid* grids, Sources src, Work64* work,
                             const unsigned long long* work_count, int n_samples,
                             int64_t work_cap, Hit* hits, int64_t hit_cap,
                             unsigned long long* hit_count, long long* counters,
                             uint32_t* status, ResolveScratch rs, int sm_count,
                             cudaStream_t st) {
  // table capacity: the smallest power of two >= 2 x the vertex slots
  unsigned long long cap = 1024;
  while (cap < 6ull * (unsigned long long)n_samples * (unsigned long long)work_cap) cap <<= 1;
  if (cap > rs.cap) return cudaErrorInvalidValue;  // sized by the caller from the same formula
  // the table (all keys empty, no distinct nodes) is cleared once at
  // allocation and left empty again by k_res_tri
  const int64_t slots3 = (int64_t)n_samples * work_cap * 3;
  int64_t b1 = (slots3 + 255) / 256;
  if (b1 > (int64_t)sm_count * 16) b1 = (int64_t)sm_count * 16;
  cudaError_t e = launch_pdl(k_res_insert, dim3((unsigned)b1), dim3(256), st, work, work_count,
                             n_samples, work_cap, grids, rs.keys, cap - 1, rs.vslot, rs.ulist,
                             rs.n_unique);
  if (e != cudaSuccess) return e;
  e = launch_tight32(pot32, seg, n_pot, grids, src, work, work_count, n_samples, work_cap, hits,
                     hit_cap, hit_count, counters, status, rs, sm_count, st);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_res_nodes, dim3(sm_count * 8), dim3(kResNodeThreads), st, pot64, n_pot,
                 src.sample_base, grids, rs.keys, rs.ulist64, rs.n64, rs.hval, counters);
  if (e != cudaSuccess) return e;
  int64_t b3 = ((int64_t)n_samples * work_cap + 127) / 128;
  if (b3 > (int64_t)sm_count * 16) b3 = (int64_t)sm_count * 16;
  return launch_pdl(k_res_tri, dim3((unsigned)b3), dim3(128), st, grids, src,
                    (const Work64*)work, work_count, n_samples, work_cap, rs.vslot, rs.hval, hits,
                    hit_cap, hit_count, counters, status, rs.keys, rs.n_unique, rs.flag64, rs.n64);
}

// -------------------------------------------------------------- barycentres
// beta_m = theta_obs,m - r_i alpha(theta_obs,m) for every (sample, observed
// image); then each system's unweighted mean in observation order.
constexpr int kBaryThreads = 128;

__global__ void __launch_bounds__(kBaryThreads)
    k_bary_obs(const Pot64* __restrict__ pot64, int n_pot, int batch, lt_obs obs,
               double* __restrict__ beta_obs) {
  __shared__ double2 buf[3 * kBaryThreads];
  __shared__ double res[6];
  for (int64_t f = blockIdx.x; f < (int64_t)batch * obs.n_obs; f += gridDim.x) {
    const int b = (int)(f / obs.n_obs);
    const int m = (int)(f - (int64_t)b * obs.n_obs);
    double X = obs.x[m], Y = obs.y[m];
    block_alpha64<kBaryThreads>(pot64 + (int64_t)b * n_pot, n_pot, 1, &X, &Y, &res[0], &res[3],
                                buf);
    if (threadIdx.x == 0) {
      const double r = obs.dls_ds[obs.sys[m]];
      beta_obs[2 * f] = X - r * res[0];
      beta_obs[2 * f + 1] = Y - r * res[3];
    }
    __syncthreads();
  }
}

__global__ void k_bary_sys(int batch, lt_obs obs, const double* __restrict__ beta_obs,
                           double* __restrict__ bary) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= (int64_t)batch * obs.n_sys) return;
  const int b = (int)(f / obs.n_sys);
  const int i = (int)(f - (int64_t)b * obs.n_sys);
  double sx = 0.0, sy = 0.0;
  int cnt = 0;
  for (int m = 0; m < obs.n_obs; ++m) {
    if (obs.sys[m] != i) continue;
    sx = sx + beta_obs[2 * ((int64_t)b * obs.n_obs + m)];
    sy = sy + beta_obs[2 * ((int64_t)b * obs.n_obs + m) + 1];
    ++cnt;
  }
  bary[2 * f] = cnt ? sx / cnt : 0.0;
  bary[2 * f + 1] = cnt ? sy / cnt : 0.0;
}

cudaError_t launch_barycentres(const Pot64* pot64, int n_pot, int batch, const lt_obs& obs,
                               double* beta_obs, double* bary, cudaStream_t st) {
  int64_t blocks = (int64_t)batch * obs.n_obs;
  if (blocks > 8192) blocks = 8192;
  k_bary_obs<<<(unsigned)blocks, kBaryThreads, 0, st>>>(pot64, n_pot, batch, obs, beta_obs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t n = (int64_t)batch * obs.n_sys;
  k_bary_sys<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(batch, obs, beta_obs, bary);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ sorting
// Write each sample's hits to lt_image records in (src, tri) order: the rank
// of a hit is the number of hits with a smaller key (keys are unique).
constexpr int kSortThreads = 256;

__global__ void __launch_bounds__(kSortThreads)
    k_sort_hits(const Hit* __restrict__ hits, const unsigned long long* __restrict__ hit_count,
                int64_t hit_cap, int sample_base, lt_image* __restrict__ out, int64_t out_cap,
                int64_t* __restrict__ n_out, uint32_t* status) {
  const int b = blockIdx.x;
  const unsigned long long total = hit_count[b];
  const int64_t n = (int64_t)min((unsigned long long)hit_cap, total);
  const Hit* hb = hits + (int64_t)b * hit_cap;
  const int sample = sample_base + b;
  if (threadIdx.x == 0) {
    n_out[sample] = (int64_t)total;
    if (total > (unsigned long long)out_cap) atomicOr(status, ST_OVERFLOW_HITS);
  }
  for (int64_t h = threadIdx.x; h < n; h += kSortThreads) {
    const Hit me = hb[h];
    int64_t rank = 0;
    for (int64_t o = 0; o < n; ++o) {
      const Hit& ot = hb[o];
      if (ot.src < me.src || (ot.src == me.src && ot.tri < me.tri)) ++rank;
    }
    if (rank < out_cap) {
      lt_image im;
      im.sample = sample;
      im.src = me.src;
      im.tri = me.tri;
      im.x = me.x;
      im.y = me.y;
      im.w[0] = me.w[0];
      im.w[1] = me.w[1];
      im.w[2] = me.w[2];
      im.fp64 = me.fp64;
      im.reserved = 0;
      out[(int64_t)sample * out_cap + rank] = im;
    }
  }
}

cudaError_t launch_sort_hits(const Hit* hits, const unsigned long long* hit_count, int n_samples,
                             int64_t hit_cap, int sample_base, lt_image* out, int64_t out_cap,
                             int64_t* n_out, uint32_t* status, cudaStream_t st) {
  if (n_samples <= 0) return cudaSuccess;
  k_sort_hits<<<n_samples, kSortThreads, 0, st>>>(hits, hit_count, hit_cap, sample_base, out,
                                                  out_cap, n_out, status);
  return cudaGetLastError();
}

// -------------------------------------------------------------------- chi^2
// Each observed image is matched to the nearest predicted image of its
// system (ties to the lower triangle id) and adds |x_obs - x|^2/sigma^2, or
// the penalty (L_diag/sigma)^2 when the system has no image.
constexpr int kChi2Threads = 128;

// Matching: one warp per (sample, observed image).  The lanes scan the hits
// of the sample (lane l takes hits l, l + 32, ...), each keeping the nearest
// predicted image of the observed image's system, ties to the lower triangle
// id; the warp then reduces the lanes' candidates by the same rule, which
// orders (distance^2, triangle) totally, so the result does not depend on the
// reduction order.  The term of Eq. 11 (or the no-image penalty) goes to
// terms[]; k_chi2_sum adds a sample's terms in a fixed order.
constexpr int kMatchThreads = 128;

__device__ __forceinline__ bool better(double d2, int64_t tri, double bd, int64_t btri) {
  return bd < 0.0 || d2 < bd || (d2 == bd && tri < btri);
}

__global__ void __launch_bounds__(kMatchThreads)
    k_chi2_match(const Hit* __restrict__ hits, const unsigned long long* __restrict__ hit_count,
                 int64_t hit_cap, int n_samples, int sample_base,
                 const SampleGrid* __restrict__ grids, lt_obs obs, double* __restrict__ terms,
                 int64_t* __restrict__ match_tri, int32_t* __restrict__ match_hit,
                 double* __restrict__ match_xy) {
  grid_dependency_wait();
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * kMatchThreads + threadIdx.x) >> 5;
  if (wid >= (int64_t)n_samples * obs.n_obs) return;  // warp-uniform
  const int b = (int)(wid / obs.n_obs);
  const int m = (int)(wid - (int64_t)b * obs.n_obs);
  const int sample = sample_base + b;
  const int64_t n = (int64_t)min((unsigned long long)hit_cap, hit_count[b]);
  const Hit* hb = hits + (int64_t)b * hit_cap;
  const int i = obs.sys[m];
  const double ox = obs.x[m], oy = obs.y[m];
  double bd = -1.0;  // -1: none yet
  int64_t btri = 0, bh = -1;
  for (int64_t h = lane; h < n; h += 32) {
    if (hb[h].src != i) continue;
    const double ex = ox - hb[h].x, ey = oy - hb[h].y;
    const double d2 = ex * ex + ey * ey;
    const int64_t tri = hb[h].tri;
    if (better(d2, tri, bd, btri)) {
      bd = d2;
      btri = tri;
      bh = h;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double od = __shfl_xor_sync(0xffffffffu, bd, off);
    const long long ot = __shfl_xor_sync(0xffffffffu, (long long)btri, off);
    const long long oh = __shfl_xor_sync(0xffffffffu, (long long)bh, off);
    if (od >= 0.0 && better(od, ot, bd, btri)) {
      bd = od;
      btri = ot;
      bh = oh;
    }
  }
  if (lane == 0) {
    const double sg = obs.sigma[m];
    const int64_t o = (int64_t)sample * obs.n_obs + m;
    double term;
    if (bh < 0) {
      const SampleGrid g = grids[b];
      const double Lx = (g.nx - 1) * g.dx, Ly = (g.ny - 1) * g.dy;
      const double t = sqrt(Lx * Lx + Ly * Ly) / sg;
      term = t * t;
      if (match_tri) match_tri[o] = -1;
      if (match_hit) match_hit[o] = -1;
      if (match_xy) { match_xy[2 * o] = 0.0; match_xy[2 * o + 1] = 0.0; }
    } else {
      term = bd / (sg * sg);
      if (match_tri) match_tri[o] = hb[bh].tri;
      if (match_hit) match_hit[o] = (int32_t)bh;
      if (match_xy) { match_xy[2 * o] = hb[bh].x; match_xy[2 * o + 1] = hb[bh].y; }
    }
    terms[o] = term;
  }
}

// chi^2 of each sample: thread t adds terms t, t + 128, ..., then warp
// shuffles and the warps in order (a fixed order).
__global__ void __launch_bounds__(kChi2Threads)
    k_chi2_sum(int sample_base, int n_obs, const double* __restrict__ terms,
               double* __restrict__ chi2) {
  grid_dependency_wait();
  __shared__ double wsum[kChi2Threads / 32];
  const int sample = sample_base + blockIdx.x;
  const double* tb = terms + (int64_t)sample * n_obs;
  double acc = 0.0;
  for (int m = threadIdx.x; m < n_obs; m += kChi2Threads) acc = acc + tb[m];
  for (int off = 16; off > 0; off >>= 1) acc = acc + __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kChi2Threads / 32; ++w) tot = tot + wsum[w];
    chi2[sample] = tot;
  }
}

cudaError_t launch_chi2(const Hit* hits, const unsigned long long* hit_count, int n_samples,
                        int64_t hit_cap, int sample_base, const SampleGrid* grids,
                        const lt_obs& obs, double* chi2, double* terms, int64_t* match_tri,
                        int32_t* match_hit, double* match_xy, cudaStream_t st) {
  if (n_samples <= 0) return cudaSuccess;
  const int64_t warps = (int64_t)n_samples * obs.n_obs;
  const int64_t blocks = (warps * 32 + kMatchThreads - 1) / kMatchThreads;
  cudaError_t e = launch_pdl(k_chi2_match, dim3((unsigned)blocks), dim3(kMatchThreads), st, hits,
                             hit_count, hit_cap, n_samples, sample_base, grids, obs, terms,
                             match_tri, match_hit, match_xy);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_chi2_sum, dim3(n_samples), dim3(kChi2Threads), st, sample_base, obs.n_obs,
                    terms, chi2);
}

}  // namespace lt

namespace lt {

// FP64 recomputation of the listed nodes (the paper's mixed rule): one node
// per thread, potentials staged in shared memory and summed in index order,
// exactly as the FP64 deflection kernel does.
__global__ void __launch_bounds__(kDefl64Threads)
    k_paper_fp64(const Pot64* __restrict__ pot64, int n_pot, double x0, double y0, double dx,
                 double dy, int nx, const int32_t* __restrict__ list,
                 const unsigned long long* __restrict__ count, double2* __restrict__ out) {
  __shared__ Pot64 sp[kChunk64];
  const int64_t n_list = (int64_t)*count;
  for (int64_t base = (int64_t)blockIdx.x * kDefl64Threads; base < n_list;
       base += (int64_t)gridDim.x * kDefl64Threads) {
    const int64_t idx = base + threadIdx.x;
    const bool valid = idx < n_list;
    const int64_t n = valid ? list[idx] : list[base];
    const int j = (int)(n / nx), i = (int)(n - (int64_t)j * nx);
    const double x = x0 + (double)i * dx;
    const double y = y0 + (double)j * dy;
    double ax = 0.0, ay = 0.0;
    for (int c0 = 0; c0 < n_pot; c0 += kChunk64) {
      const int cn = min(kChunk64, n_pot - c0);
      __syncthreads();
      for (int k = threadIdx.x; k < cn; k += kDefl64Threads) sp[k] = pot64[c0 + k];
      __syncthreads();
      for (int k = 0; k < cn; ++k) {
        double kx, ky;
        alpha64_one(sp[k], x, y, kx, ky);
        ax = ax + kx;
        ay = ay + ky;
      }
    }
    if (valid) out[n] = make_double2(ax, ay);
  }
}

cudaError_t launch_paper_fp64(const Pot64* pot64, int n_pot, const lt_grid& g, const int32_t* list,
                              const unsigned long long* count, double2* out, int sm_count,
                              cudaStream_t st) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_paper_fp64, kDefl64Threads, 0);
  if (per_sm < 1) per_sm = 1;
  k_paper_fp64<<<sm_count * per_sm, kDefl64Threads, 0, st>>>(pot64, n_pot, g.x0, g.y0, g.dx, g.dy,
                                                             g.nx, list, count, out);
  return cudaGetLastError();
}

}  // namespace lt
