// Internal declarations of the GB300 chi^2 library: prepared potential
// records, the FP64 and FP32 per-potential deflections, error-bound
// constants, device status bits and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lt.h"

namespace lt {

// ------------------------------------------------------------------ status
// Device-side status word (latched, OR-ed): reported by lt_model_sync.
enum : uint32_t {
  ST_OVERFLOW_HITS = 1u << 0,
  ST_OVERFLOW_WORK = 1u << 1,
  ST_NONFINITE = 1u << 2,
};

// Counters written by kernels (int64, device), one set per model.
enum {
  CNT_HITS = 0,
  CNT_AMBIG,        // (triangle, source) pairs the coarse FP32 bound left undecided
  CNT_REFINE,       // coarse-certain hits whose position bound was too large
  CNT_FP64_NODES,   // distinct nodes evaluated in FP64
  CNT_DROPPED,
  CNT_TIGHT_NODES,  // distinct nodes re-evaluated with the tight FP32 bound
  CNT_FP64_ITEMS,   // work items the tight bound left to FP64
  CNT_N
};

constexpr double kC = 299792.458;         // km/s
constexpr double kArcsec = 206264.80625;  // arcsec per radian
constexpr double kPi = 3.14159265358979323846;
constexpr float kU32 = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of FP32

// --------------------------------------------------------- prepared records
// FP64 record of one potential, in parameter index order (16 doubles).  The
// FP64 path sums potentials in index order with the formulas of alpha64_one:
// the SIS and SIE as stated there (an FP64 reference that follows the same
// statement is reproduced to the ulps of sin and cos), the PIEMD in the
// difference form (a few ulps of the deflection).  k = sqrt(k2), ik = 1/k (0
// for k = 0).
struct Pot64 {
  double kind, cx, cy, c, s, b0, e, q, k2, q2, a, sc, scale, sv, k, ik;
};
static_assert(sizeof(Pot64) == 128, "Pot64 layout");

// FP32 record of one potential (5 float4 and an FP64 centre = 96 bytes),
// grouped by kind.
//   SIS   : f[0] = {cx, cy, b0, 0}
//   SIE   : f[0] = {cx, cy, r1 c, r1 s}; f[1] = {r2 c, r2 s, b0 r1 c, b0 r2 s};
//           f[2] = {b0 r2 c, b0 r1 s, 0, 0} with r1,2 = sqrt(1 -+ eps)
//   PIEMD : f[0] = {cx, cy, c, s}; f[1] = {q2, q2*a*a, q2*s*s, k2};
//           f[2] = {a, s, q2*a, q2*s};
//           f[3] = {sig(s-a), sig q2(s+a)(s-a), sig q2(s-a), (B/sig) c};
//           f[4] = {errP0, errGx B/sig, errGy B/sig, (B/sig) s}, sig = sqrt(k2)
//   SIS/SIE: f[4] = {errP0, 0, 0, 0}
// (error-bound coefficients errP0, errGx, errGy, in units of u; the static
// terms errQ are summed into Seg32::q_tot).  At staging, errP0 times
// W = Theta + |cx| + |cy| (Theta = largest |node coordinate| of the grid; node
// coordinates are rounded once from FP64) becomes the coefficient P of the
// per-node term P / distance (stage_p32); see k_prep for the derivation of
// every coefficient.
//   c64   : the centre in FP64 (cx, cy), read only by the tight FP32
//           re-evaluation, which translates nodes in FP64; the deflection
//           kernels stage f[0..4] alone.
struct Pot32 {
  float4 f[5];
  double2 c64;
};
static_assert(sizeof(Pot32) == 96, "Pot32 layout");

// ------------------------------------------------ FP32 error-bound constants
// Largest relative errors, in units of the FP32 unit roundoff u = 2^-24, of
// the FP32 primitives of the deflection: the hardware approximations and the
// library's atan(t)/t and atanh(t)/t (polynomials with range reduction), each
// measured at every float argument the kernels can give it
// (tests/test_gpu_special.py; tests/test_fp32_poly.py for the polynomials
// alone).  Those tests fail if a measurement exceeds the value here, so the
// bound's coefficients, derived from these values in k_prep, stay valid.
// For atanh(t)/t above u = 1/4 the relative error grows like 1/(1 - u) (the
// logarithm's argument (1 + t)/(1 - t) inherits the rounding of t): the
// constant is the largest (1 - u) times the relative error, and the bound
// divides it by its own lower bound on 1 - u (1 - t^2 > q^2).
constexpr double kEpsRsqrt = 2.1;       // rsqrt.approx.ftz.f32 (measured 2.092)
constexpr double kEpsSqrt = 1.7;        // sqrt.approx.ftz.f32 (1.678)
constexpr double kEpsRcp = 1.7;         // rcp.approx.ftz.f32 (1.649)
constexpr double kEpsAtanc = 13.6;      // atanc_sq32 on [0, 2^14] (13.500)
constexpr double kEpsAtanhc = 7.7;      // atanhc_sq32 on [0, 1/4] (7.574)
constexpr double kEpsAtanhcLog = 5.0;   // (1 - u) x atanhc_sq32 on [1/4, 0.99999988] (4.917)
constexpr double kU32d = 5.9604644775390625e-8;  // u as a double

// A node's bound from its accumulated terms (units of u) for a sample of
// n_pot potentials.  The factor 1 + (6 n_pot + 64) u + 2^-16 covers the
// round-to-nearest accumulation of the non-negative terms (at most five
// roundings per potential and two per group, so a relative shortfall below
// gamma(6 n_pot + 64)) and the terms of second order in u that the
// coefficients leave out (the FP64 rounding of the record constants, the
// 2 + u of a fused accumulation step).  Capped at 1e30: a node on an SIS/SIE
// centre has an infinite term, and a finite cap keeps every later product
// (r E with r = 0 included) a number.
__device__ __forceinline__ float node_bound(float terms, int n_pot) {
  const float f = __fmaf_ru((float)(6 * n_pot + 64), kU32, 1.0000152587890625f);
  return fminf(__fmul_ru(__fmul_ru(kU32, f), terms), 1e30f);
}

// Per-sample kind segments of the FP32 records (n_sis, n_piemd, n_sie), the
// static part of the tight error bound, sum_k errQ_k, the static part of
// the coarse one, which adds every potential's largest evaluation and
// accumulation terms, and that of the tight re-evaluation with FP64
// translation (units of u, rounded up).
struct Seg32 {
  int n_sis, n_piemd, n_sie;
  float q_tot, c_tot;
  float q_tight;  // static terms of the tight re-evaluation's bound (k_res_tight32)
};

// Summation structure of the FP32 deflection: potentials are staged kChunk32
// at a time (kind-sorted order), and within a chunk each kind segment is
// summed in groups of at most kSumGroup potentials whose partial sums join
// the node's total once per group.
constexpr int kChunk32 = 256;
constexpr int kSumGroup = 32;

// ---------------------------------------------------- FP64 deflection (one)
// atan(k T)/k and atanh(k T)/k of a record's k = sqrt(k2) and ik = 1/k: the
// short Taylor series in u = k2 T^2 below 1e-6 (which also covers k = 0 and
// keeps the q -> 1 limit exact), else the library function times 1/k.
__device__ __forceinline__ double atan_k64(double T, double k, double ik, double k2) {
  const double u = k2 * T * T;
  if (u < 1e-6) return T * (1.0 - u * (1.0 / 3.0 - u * (1.0 / 5.0 - u * (1.0 / 7.0))));
  return atan(k * T) * ik;
}
__device__ __forceinline__ double atanh_k64(double T, double k, double ik, double k2) {
  const double u = k2 * T * T;
  if (u < 1e-6) return T * (1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0))));
  return atanh(k * T) * ik;
}

// Scaled deflection of one potential at (x, y) in FP64.  Must be compiled
// without FMA contraction (-fmad=false): every operation is rounded in the
// order written.
//   SIS  (Sect. 2.1): b0 (theta - c)/|theta - c|, zero at the centre.
//   SIE  (Algorithm 1): translate, rotate by phi, R = sqrt(x'^2 (1-eps) +
//        y'^2 (1+eps)), ((1-eps) b0 x'/R, (1+eps) b0 y'/R), rotate by -phi.
//   PIEMD (dPIE core a, cut s, q = 1 - e): alpha' = b0 s/(s-a) [F(a) - F(s)]
//        rotated by -phi, with per cored term w in (a, s) psi_w = sqrt(q^2
//        (w^2 + x'^2) + y'^2) and F(w) = (atan(k x'/(psi_w + w)),
//        atanh(k y'/(psi_w + q^2 w)))/k, evaluated in difference form: with
//        atan u - atan v = atan((u - v)/(1 + uv)), the atanh analogue and
//        psi_s - psi_a = q^2 (s^2 - a^2)/(psi_a + psi_s),
//          F_x(a) - F_x(s) = atan(k Tx)/k, Tx = x' (s-a)(1 + q^2 (s+a)/(psi_a
//            + psi_s)) / ((psi_a + a)(psi_s + s) + k^2 x'^2),
//          F_y(a) - F_y(s) = atanh(k Ty)/k, Ty = y' q^2 (s-a)(1 + (s+a)/(psi_a
//            + psi_s)) / ((psi_a + q^2 a)(psi_s + q^2 s) - k^2 y'^2),
//        one atan and one atanh instead of two each (the FP32 path's form).
__device__ __forceinline__ void alpha64_one(const Pot64& p, double x, double y, double& ax,
                                            double& ay) {
  double dx = x - p.cx;
  double dy = y - p.cy;
  int kind = (int)p.kind;
  if (kind == LT_SIS) {
    double R = sqrt(dx * dx + dy * dy);
    if (R == 0.0) { ax = 0.0; ay = 0.0; return; }
    ax = p.b0 * dx / R;
    ay = p.b0 * dy / R;
    return;
  }
  double xp = dx * p.c + dy * p.s;
  double yp = dy * p.c - dx * p.s;
  double gx, gy;
  if (kind == LT_SIE) {
    double R = sqrt(xp * xp * (1.0 - p.e) + yp * yp * (1.0 + p.e));
    if (R == 0.0) { ax = 0.0; ay = 0.0; return; }
    gx = (1.0 - p.e) * p.b0 * xp / R;
    gy = (1.0 + p.e) * p.b0 * yp / R;
  } else {
    const double x2 = xp * xp, y2 = yp * yp;
    const double t = p.q2 * x2 + y2;
    const double pa = sqrt(t + p.q2 * (p.a * p.a));
    const double ps = sqrt(t + p.q2 * (p.sc * p.sc));
    const double iD = 1.0 / (pa + ps);
    const double sa = p.sc - p.a;
    const double Tx = xp * (sa * (1.0 + p.q2 * (p.sc + p.a) * iD)) /
                      ((pa + p.a) * (ps + p.sc) + p.k2 * x2);
    const double Ty = yp * (p.q2 * sa * (1.0 + (p.sc + p.a) * iD)) /
                      ((pa + p.q2 * p.a) * (ps + p.q2 * p.sc) - p.k2 * y2);
    gx = p.scale * atan_k64(Tx, p.k, p.ik, p.k2);
    gy = p.scale * atanh_k64(Ty, p.k, p.ik, p.k2);
  }
  ax = gx * p.c - gy * p.s;
  ay = gy * p.c + gx * p.s;
}

// ------------------------------------------------- FP64 point deflections
// Deflection at up to 3 points by a whole block of NT threads.  The threads
// form one group of NT/npts per point; in each chunk of NT/npts potentials,
// thread k of group q evaluates (point q, potential c0 + k), and then lanes
// 2q and 2q + 1 of the first warp sum point q's x and y components over the
// chunk in potential index order, so each result is the oracle's
// left-to-right sum exactly.  GB300's FP64 unit issues a warp instruction
// only every few dozen cycles per SM sub-partition, so giving each thread a
// single evaluation (NT >= npts * n_pot) keeps the serial FP64 depth of a
// block at one potential, and summing every component in one chain of warp
// instructions keeps the sum's depth at one add per potential.  Must be
// called by every thread of the block; results in ax[q], ay[q] (shared); buf
// holds NT double2.
template <int NT>
__device__ inline void block_alpha64(const Pot64* __restrict__ pb, int n_pot, int npts,
                                     const double* px, const double* py, double* ax, double* ay,
                                     double2* buf /*[NT]*/) {
  const int t = threadIdx.x;
  const int G = NT / npts;
  const int q = t / G, k = t - q * G;
  double sum = 0.0;  // summing lanes: component t & 1 of point t >> 1
  for (int c0 = 0; c0 < n_pot; c0 += G) {
    if (q < npts && c0 + k < n_pot) {
      const Pot64 p = pb[c0 + k];
      double kx, ky;
      alpha64_one(p, px[q], py[q], kx, ky);
      buf[q * G + k] = make_double2(kx, ky);
    }
    __syncthreads();
    if (t < 2 * npts) {
      const int cn = min(G, n_pot - c0);
      const double* col = reinterpret_cast<const double*>(buf + (t >> 1) * G) + (t & 1);
      for (int m = 0; m < cn; ++m) sum = sum + col[2 * m];
    }
    __syncthreads();
  }
  if (t < 2 * npts) (t & 1 ? ay : ax)[t >> 1] = sum;
  __syncthreads();
}

// ---------------------------------------------------- FP32 special functions
// The hardware approximations the FP32 path uses, named by their PTX
// instructions (flush-to-zero forms).  Their largest relative errors are
// measured exhaustively on the GPU over every input the path can give them
// (tests/test_gpu_special.py) and enter the error bound through those
// measured maxima.
__device__ __forceinline__ float rsqrt_approx32(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx32(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_approx32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx32(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Polynomials in u = t*t, evaluated by Horner's rule with fused
// multiply-adds: atan(t)/t on 0 <= u <= 1 (degree 6) and atanh(t)/t on
// 0 <= u <= 1/4 (degree 4).  Least-squares fits in the relative sense at
// Chebyshev nodes (csrc/fit_poly.py).  The relative errors of these FP32
// evaluations against the exact functions, taken over every float u of the
// two intervals (tests/test_fp32_poly.py), are 13.5 and 7.7 ulp.  These
// literals are the single copy of the coefficients.
__device__ __forceinline__ float atanc_poly32(float u) {
  float p = 7.685306482e-03f;
  p = fmaf(p, u, -3.647336364e-02f);
  p = fmaf(p, u, 8.325644583e-02f);
  p = fmaf(p, u, -1.345480382e-01f);
  p = fmaf(p, u, 1.987373084e-01f);
  p = fmaf(p, u, -3.332583010e-01f);
  p = fmaf(p, u, 9.999992251e-01f);
  return p;
}
__device__ __forceinline__ float atanhc_poly32(float u) {
  float p = 1.953562647e-01f;
  p = fmaf(p, u, 1.221839786e-01f);
  p = fmaf(p, u, 2.019458860e-01f);
  p = fmaf(p, u, 3.332709372e-01f);
  p = fmaf(p, u, 1.000000358e+00f);
  return p;
}

// atan(t)/t of t2 = t*t >= 0: the polynomial for t2 <= 1; for t2 > 1,
// atan(t) = pi/2 - atan(1/t) gives (pi/2)/t - P(1/t2)/t2 with one rsqrt.
// The range test is a real branch: the 32 nodes of a warp see one potential
// from nearly the same direction, so it is almost always uniform.
//
// atanh(t)/t of t2 = t*t in [0, 1): the polynomial for t2 <= 1/4; above,
// atanh(t) = ln((1+t)/(1-t))/2 with rsqrt, rcp and lg2 (the ratio is >= 3
// there, away from lg2's absolute-error range around 1).
// The largest relative errors of both functions over all their float
// arguments are measured on the GPU (tests/test_gpu_special.py).
// The range-reduced forms alone (no test; valid for t2 > 1 and t2 > 1/4
// respectively, finite or not elsewhere): the deflection kernels evaluate
// them for all of a thread's nodes and select per node, so no register of a
// node pair is updated under a branch.  Every operation is written out
// (__fmaf_rn / __fmul_rn are never contracted or split), so the deflection
// kernels' lane forms (lt_fp32.cuh) repeat them exactly.
__device__ __forceinline__ float atanc_reduced32(float t2) {
  const float r = rsqrt_approx32(t2);
  const float inv = __fmul_rn(r, r);
  const float p = atanc_poly32(inv);
  return __fmaf_rn(1.57079633f, r, -__fmul_rn(p, inv));
}
__device__ __forceinline__ float atanhc_reduced32(float t2) {
  t2 = fminf(t2, 0.99999988f);
  const float r = rsqrt_approx32(t2);
  // 1 + t and 1 - t with t = t2 r, each one fused multiply-add
  const float num = __fmaf_rn(t2, r, 1.0f), den = __fmaf_rn(-t2, r, 1.0f);
  return __fmul_rn(__fmul_rn(lg2_approx32(__fmul_rn(num, rcp_approx32(den))),
                             0.5f * 0.693147181f),
                   r);
}
__device__ __forceinline__ float atanc_sq32(float t2) {
  return t2 > 1.0f ? atanc_reduced32(t2) : atanc_poly32(t2);
}
__device__ __forceinline__ float atanhc_sq32(float t2) {
  return t2 > 0.25f ? atanhc_reduced32(t2) : atanhc_poly32(t2);
}

// Launch-shape variants of the FP32 deflection kernel (autotuned).
struct DeflectShape {
  int threads;     // threads per block
  int npt;         // nodes per thread (rows of one column)
  int min_blocks;  // resident blocks per SM the register budget must allow
};
constexpr int kNumShapes = 8;
__host__ __device__ constexpr DeflectShape deflect_shape(int v) {
  const DeflectShape tab[kNumShapes] = {{256, 4, 3}, {256, 2, 5}, {256, 3, 4}, {128, 8, 3},
                                        {128, 8, 4}, {128, 4, 7}, {128, 4, 4}, {256, 4, 2}};
  return tab[v < 0 || v >= kNumShapes ? 0 : v];
}

// Work items of the FP32 triangle search.  A thread takes kSearch32Rows cells
// of one cell column (a band); a sample's (band, cell column) positions,
// band-major, are cut into items of kSearch32Threads positions.
constexpr int kSearch32Threads = 32, kSearch32Rows = 2;
__host__ __device__ inline int64_t search32_items(int nx, int ny) {
  const int64_t cw = (int64_t)nx - 1, ch = (int64_t)ny - 1;
  if (cw <= 0 || ch <= 0) return 0;
  const int64_t bands = (ch + kSearch32Rows - 1) / kSearch32Rows;
  return (bands * cw + kSearch32Threads - 1) / kSearch32Threads;
}

// Work items of the FP32 deflection.  A thread takes npt nodes of one grid
// column: rows [band*npt, band*npt + npt) of band `band`.  A sample's
// (band, column) positions, band-major, are cut into items of `threads`
// consecutive positions; only the last band of a sample can be partly empty.
__host__ __device__ inline int64_t defl32_items(int nx, int ny, int threads, int npt) {
  const int64_t bands = ((int64_t)ny + npt - 1) / npt;
  return (bands * nx + threads - 1) / threads;
}

// ----------------------------------------------------------- batch layout
// One sample's grid and where its node / cell data live in a workspace.
struct SampleGrid {
  double x0, y0, dx, dy;
  int nx, ny;
  int64_t node_off;  // offset of node (0,0) in the node workspace
  float theta_max;   // largest |coordinate| of any node
  float pad;
  float x0f, y0f, dxf, dyf;  // x0, y0, dx, dy rounded to FP32 (once, on the host)
  // offset of this grid's node coordinates in the FP32 coordinate table:
  // nx values x0 + i dx, then ny values y0 + j dy, each evaluated in FP64 as
  // written (no fused multiply-add) and rounded once to FP32, on the host
  int64_t coord_off;
};

// Work item of the FP64 stage: an ambiguous (triangle, source) pair or an
// FP32 hit to re-interpolate.
struct Work64 {
  int32_t sample, src;
  int64_t tri;
  int32_t type;      // 0 = ambiguous pair, 1 = refine a certain hit
  int32_t resolved;  // set by the tight FP32 stage when it decided the item
};

// Adjoint point: position and the 2-vector coefficient of d alpha there.
struct AdjPt {
  double x, y, cx, cy;
};

// Hit record kept between the search and the chi^2 kernels.
struct Hit {
  int32_t src, fp64;
  int64_t tri;
  double x, y;
  double w[3];
};

// Sample of a work item: off[] holds each sample's first item, off[n] the total.
__device__ __forceinline__ int find_sample(const int64_t* off, int n, int64_t item) {
  int lo = 0, hi = n;  // off[lo] <= item < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------ programmatic dependent launch
// Kernels of the chi^2 chain are launched with programmatic stream
// serialization: the next kernel's grid may be scheduled while the previous
// kernel of the stream drains, which hides its launch latency.  Every such
// kernel calls grid_dependency_wait() before it touches any memory, which
// returns once the previous kernel has completed and its writes are visible
// (a no-op when the kernel was launched without the attribute).  Not under
// stream capture: a CUDA graph already launches its kernels back to back, and
// measured slower (about 8 us per c2 evaluation) with programmatic edges.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusActive;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = cs == cudaStreamCaptureStatusNone ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return the cudaGetLastError() value.
// Zero up to four arrays of 64-bit counters in one launch (the per-call
// counter resets of a chi^2 evaluation: one kernel instead of four memsets).
cudaError_t launch_zero64(unsigned long long* a, int64_t na, unsigned long long* b, int64_t nb,
                          unsigned long long* c, int64_t nc, unsigned long long* d, int64_t nd,
                          cudaStream_t st);
cudaError_t launch_prep(const double* params, int batch, int n_pot, Pot64* pot64, Pot32* pot32,
                        Seg32* seg, uint32_t* status, cudaStream_t st);
// next_item: a zeroed device counter, taken by atomicAdd (dynamic items);
// tight: the node bound in its tight form (else the coarse one)
cudaError_t launch_deflect32(const Pot32* pot32, const Seg32* seg, int n_pot,
                             const SampleGrid* grids, const float* coords,
                             const int64_t* item_off, int n_samples, int64_t n_items, int shape,
                             bool tight, float4* node_out, unsigned long long* next_item,
                             int sm_count, cudaStream_t st);
cudaError_t launch_deflect64(const Pot64* pot64, int n_pot, const SampleGrid* grids,
                             const int64_t* item_off, int n_samples, int64_t n_items,
                             double2* node_out, int sm_count, cudaStream_t st);
// Copy one sample's node workspace into a caller layout.
cudaError_t launch_unpack32(const float4* nodes, int64_t n, float2* alpha, float* err,
                            cudaStream_t st);

// Sources of the triangle search: positions (FP64), ratios D_ls/D_s.
struct Sources {
  const double* xy;   // [batch][n_src][2]
  const double* r;    // [batch][n_src] (stride_r = n_src) or [n_src] (stride_r = 0)
  int n_src;
  int stride_r;
  int sample_base;    // sample index of the first sample in this chunk
};

cudaError_t launch_search32(const float4* nodes, const SampleGrid* grids, const int64_t* item_off,
                            int n_samples, int64_t n_items, Sources src, Hit* hits,
                            int64_t hit_cap, Work64* work, int64_t work_cap,
                            unsigned long long* hit_count, unsigned long long* work_count,
                            long long* counters, uint32_t* status,
                            unsigned long long* next_item, int sm_count, cudaStream_t st);
cudaError_t launch_search64(const double2* nodes, const SampleGrid* grids, const int64_t* item_off,
                            int n_samples, int64_t n_items, Sources src, Hit* hits,
                            int64_t hit_cap, unsigned long long* hit_count, long long* counters,
                            uint32_t* status, int sm_count, cudaStream_t st);
// Scratch of the resolution of undecided work items: node table (keys, FP64
// values, tight FP32 values), per-vertex slots, list of distinct nodes and
// its length, and the FP64 stage's node flags and list.  cap: table entries
// (power of two) allocated, at least the smallest power of two >= 6 x
// samples x work_cap of any chunk.  Every resolution leaves keys, flag64,
// n_unique and n64 as it found them (all empty).
// A node's deflection from the tight re-evaluation: the FP64 sum of its
// potentials' FP32 deflections and a bound on both components' error.
struct TightVal {
  double ax, ay;
  float e, pad;
};
static_assert(sizeof(TightVal) == 24, "TightVal layout");

struct ResolveScratch {
  unsigned long long* keys;
  double2* hval;
  int32_t* vslot;  // [samples][work_cap][3]
  int32_t* ulist;  // [cap]
  unsigned int* n_unique;
  unsigned long long cap;
  TightVal* tval;    // [cap] tight re-evaluation (alpha, bound) per slot
  uint32_t* flag64;  // [cap] 1 once a slot is listed for FP64
  int32_t* ulist64;  // [cap] slots to evaluate in FP64
  unsigned int* n64;
};
// Resolution of a chunk's undecided work items: distinct nodes keyed
// (k_res_insert), re-evaluated in FP32 with the tight bound and the items
// re-classified (launch_tight32), the nodes of the items still undecided
// evaluated in FP64 and those items decided exactly (k_res_nodes, k_res_tri).
// pot32 / seg: the chunk's FP32 records; pot64: all samples' FP64 records.
cudaError_t launch_resolve64(const Pot64* pot64, const Pot32* pot32, const Seg32* seg, int n_pot,
                             const SampleGrid* grids, Sources src, Work64* work,
                             const unsigned long long* work_count, int n_samples,
                             int64_t work_cap, Hit* hits, int64_t hit_cap,
                             unsigned long long* hit_count, long long* counters,
                             uint32_t* status, ResolveScratch rs, int sm_count,
                             cudaStream_t st);
// The tight FP32 stage of the resolution (k_res_tight32, k_res_tri32).
cudaError_t launch_tight32(const Pot32* pot32, const Seg32* seg, int n_pot,
                           const SampleGrid* grids, Sources src, Work64* work,
                           const unsigned long long* work_count, int n_samples, int64_t work_cap,
                           Hit* hits, int64_t hit_cap, unsigned long long* hit_count,
                           long long* counters, uint32_t* status, ResolveScratch rs,
                           int sm_count, cudaStream_t st);
cudaError_t launch_sort_hits(const Hit* hits, const unsigned long long* hit_count, int n_samples,
                             int64_t hit_cap, int sample_base, lt_image* out, int64_t out_cap,
                             int64_t* n_out, uint32_t* status, cudaStream_t st);
cudaError_t launch_barycentres(const Pot64* pot64, int n_pot, int batch, const lt_obs& obs,
                               double* beta_obs, double* bary, cudaStream_t st);
cudaError_t launch_adjoint(const Pot64* pot64, int n_pot, int batch, const SampleGrid* grids,
                           const Hit* hits, int64_t hit_cap, const lt_obs& obs,
                           const int32_t* match_hit, double2* lam, AdjPt* pts, double* grad,
                           int sm_count, cudaStream_t st);
// Source-plane chi^2: beta and point magnification per (sample, observed
// image), then barycentres and chi^2 per sample.  beta, mu: [batch][n_obs];
// bary: [batch][n_sys]; chi2: [batch].
cudaError_t launch_chi2_source(const Pot64* pot64, int n_pot, int batch, const lt_obs& obs,
                               double2* beta, double* mu, double2* bary, double* chi2,
                               int sm_count, cudaStream_t st);
// Triangle magnification of each observed image's matched predicted image.
cudaError_t launch_mag_pred(const Pot64* pot64, int n_pot, int batch, const SampleGrid* grids,
                            const Hit* hits, int64_t hit_cap, const lt_obs& obs,
                            const int32_t* match_hit, double* mu, int sm_count,
                            cudaStream_t st);
// The paper's mixed rule for a deflection grid (LT_PREC_PAPER).
cudaError_t launch_paper_flags(const float4* nodes, const Pot64* pot64, int n_pot,
                               const lt_grid& g, double2* out, unsigned char* flags,
                               int32_t* list, unsigned long long* count, float* map,
                               int sm_count, cudaStream_t st);
cudaError_t launch_paper_fp64(const Pot64* pot64, int n_pot, const lt_grid& g, const int32_t* list,
                              const unsigned long long* count, double2* out, int sm_count,
                              cudaStream_t st);
cudaError_t launch_chi2(const Hit* hits, const unsigned long long* hit_count, int n_samples,
                        int64_t hit_cap, int sample_base, const SampleGrid* grids,
                        const lt_obs& obs, double* chi2, double* terms, int64_t* match_tri,
                        int32_t* match_hit, double* match_xy, cudaStream_t st);

}  // namespace lt
