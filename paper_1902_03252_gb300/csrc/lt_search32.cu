// FP32 triangle search of the mixed-precision path: k_search32, the fused lens
// mapping (Eq. 13) and triangle test (Fig. 1) with a certified FP32
// orientation filter; certain hits and the pairs that need FP64 are compacted
// by warp ballots.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lt_internal.cuh"
#include "lt_fp32.cuh"
#include "lt_source.cuh"

namespace lt {

// ---------------------------------------------------------- triangle search
constexpr int kSearchThreads = kSearch32Threads;  // positions per work item
constexpr int kSearchBlocksPerSM = 16;
constexpr int kMaxSrcSmem = 256;     // sources staged in shared memory at a time

// Source data staged per sample: position relative coordinates use FP32.
struct SrcSmem {
  float px, py, r, mu0;  // mu0 = u (4 Theta + |px| + |py|) (input rounding)
};

// 2u(1 + u) rounded up: the FP32 rounding of an edge function a x b =
// fma(ax, by, -(ay bx)) is at most u |ay bx| + u |result| <= 2u(1 + u)
// (|ax by| + |ay bx|).
__device__ __forceinline__ float u2_up() { return __int_as_float(0x34000001); }

// Bound on |a x b - a* x b*| for vertices a, b (relative to the source, FP32)
// whose coordinates are within ma, mb of the exact a*, b*: the input part
// ma |b|_1 + mb |a|_1 + 2 ma mb and the rounding of the FP32 edge function.
// Rounded up throughout.
__device__ __forceinline__ float edge_bound(float ax, float ay, float bx, float by, float ma,
                                            float mb) {
  const float la = __fadd_ru(fabsf(ax), fabsf(ay)), lb = __fadd_ru(fabsf(bx), fabsf(by));
  const float rnd = __fmul_ru(u2_up(), __fadd_ru(__fmul_ru(fabsf(ax), fabsf(by)),
                                                 __fmul_ru(fabsf(ay), fabsf(bx))));
  return __fmaf_ru(ma, lb, __fmaf_ru(mb, la, __fmaf_ru(__fmul_ru(2.0f, ma), mb, rnd)));
}

// Classify one triangle with relative vertices a, b, c (vertex - source,
// FP32) and per-vertex error bounds m[3].  Returns 0 = certainly outside,
// 1 = certainly inside, 2 = undecided.  An edge function whose magnitude
// exceeds its bound has the sign of the exact one; the triangle is certainly
// outside if two edge functions certainly differ in sign, certainly inside if
// all three certainly agree (then no tie rule applies).  On 1, w[] receives
// the weights and *pos_err a bound on the interpolated image's position
// error in units of the cell size: the weights w_v = e_v / det err by at most
// (E_v + w_v sE') / (|det| - sE'), sE' the edge bounds plus the rounding of
// det = e0 + e1 + e2, and by 2u in their own rounding; the image position
// A + w_B (B - A) + w_C (C - A), |B - A|, |C - A| <= h per coordinate, then
// errs by at most h (|dw_B| + |dw_C|) <= h (2 sE' / (|det| - sE') + 4u).
__device__ __forceinline__ int classify32(float ax, float ay, float bx, float by, float cx,
                                          float cy, float ma, float mb, float mc, float w[3],
                                          float* pos_err) {
  // edge functions of the origin: e_AB = a x b, e_BC = b x c, e_CA = c x a
  float e0 = fmaf(ax, by, -(ay * bx));
  float e1 = fmaf(bx, cy, -(by * cx));
  float e2 = fmaf(cx, ay, -(cy * ax));
  const float E0 = edge_bound(ax, ay, bx, by, ma, mb);
  const float E1 = edge_bound(bx, by, cx, cy, mb, mc);
  const float E2 = edge_bound(cx, cy, ax, ay, mc, ma);
  bool p0 = e0 > E0, p1 = e1 > E1, p2 = e2 > E2;
  bool n0 = e0 < -E0, n1 = e1 < -E1, n2 = e2 < -E2;
  if ((p0 || p1 || p2) && (n0 || n1 || n2)) return 0;
  if ((p0 && p1 && p2) || (n0 && n1 && n2)) {
    float det = e0 + e1 + e2;
    float inv = 1.0f / det;
    w[0] = e1 * inv;
    w[1] = e2 * inv;
    w[2] = e0 * inv;
    const float sE = __fadd_ru(__fadd_ru(__fadd_ru(E0, E1), E2),
                               __fmul_ru(u2_up(), __fadd_ru(__fadd_ru(fabsf(e0), fabsf(e1)),
                                                            fabsf(e2))));
    const float den = __fsub_rd(fabsf(det), sE);
    *pos_err = den > 0.0f ? __fadd_ru(__fdiv_ru(__fmul_ru(2.0f, sE), den), 4.8e-7f)
                          : __int_as_float(0x7f800000);
    return 1;
  }
  return 2;
}

__device__ __forceinline__ void warp_append_hit(bool flag, const Hit& h, Hit* hits,
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

__device__ __forceinline__ void warp_append_work(bool flag, const Work64& wk, Work64* work,
                                                 int64_t cap, unsigned long long* count,
                                                 uint32_t* status, long long* counters) {
  unsigned mask = __ballot_sync(0xffffffffu, flag);
  if (!mask) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (flag) {
    unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
    if (idx < (unsigned long long)cap) {
      work[idx] = wk;
    } else {  // dropped: latched and counted
      atomicOr(status, ST_OVERFLOW_WORK);
      atomicAdd((unsigned long long*)&counters[CNT_DROPPED], 1ull);
    }
  }
}

// Warp-wide float minimum / maximum in one instruction (sm_100 and later);
// exact, like the butterfly of shuffles it replaces.
__device__ __forceinline__ float warp_min(float v) {
  float r;
  asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float warp_max(float v) {
  float r;
  asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}

// A vertex bound with its second-order terms: the first-order sum times
// (1 + 8u), rounded up.
__device__ __forceinline__ float mu_up(float m) { return __fmul_ru(m, 1.00000048f); }

struct StripBox {
  float tx0, tx1, ty0, ty1, ax0, ax1, ay0, ay1, e, l;
};

// Image position of an FP32-certified hit, interpolated in FP64 from the
// triangle's node coordinates: T0 = (X0,Y0), (X1,Y0), (X1,Y1); T1 = (X0,Y0),
// (X1,Y1), (X0,Y1); w1, w2 the barycentric weights of the 2nd and 3rd
// vertex.  Out of line so that the compiler does not hoist this rare FP64
// work (GB300's FP64 pipe runs at 1/64 of the FP32 rate) into the per-cell
// path.
__device__ __noinline__ double2 hit_xy(double x0, double y0, double dx, double dy, int i, int j,
                                       int t, float w1, float w2) {
  const double X0 = x0 + (double)i * dx, X1 = x0 + (double)(i + 1) * dx;
  const double Y0 = y0 + (double)j * dy, Y1 = y0 + (double)(j + 1) * dy;
  if (t == 0)
    return make_double2(X0 + (double)w1 * (X1 - X0) + (double)w2 * (X1 - X0),
                        Y0 + (double)w2 * (Y1 - Y0));
  return make_double2(X0 + (double)w1 * (X1 - X0),
                      Y0 + (double)w1 * (Y1 - Y0) + (double)w2 * (Y1 - Y0));
}

// Emit the outcome of one cell's two triangles for the whole warp: certain
// hits (interpolated in FP64 from the node coordinates) and the pairs that go
// to the FP64 work list.  Every lane calls it (warp ballots inside).
__device__ __forceinline__ void emit_cell(const SampleGrid& g, int sample, int b, int src_k,
                                          int64_t cell, int i, int j, int r0, int r1,
                                          const float* w0, const float* w1, bool ok0, bool ok1,
                                          Hit* hits, int64_t hit_cap, Work64* work,
                                          int64_t work_cap, unsigned long long* hit_count,
                                          unsigned long long* work_count, uint32_t* status,
                                          long long* counters) {
  const bool wk0 = r0 == 2 || (r0 == 1 && !ok0);
  const bool wk1 = r1 == 2 || (r1 == 1 && !ok1);
  if (!__any_sync(0xffffffffu, ok0 || ok1 || wk0 || wk1)) return;
  const int64_t tri0 = 2 * cell, tri1 = 2 * cell + 1;
  Hit h;
  h.src = src_k;
  h.fp64 = 0;
  h.tri = tri0;
  h.w[0] = w0[0]; h.w[1] = w0[1]; h.w[2] = w0[2];
  double2 xy = hit_xy(g.x0, g.y0, g.dx, g.dy, i, j, 0, w0[1], w0[2]);
  h.x = xy.x;
  h.y = xy.y;
  Hit* hb = hits + (int64_t)b * hit_cap;
  warp_append_hit(ok0, h, hb, hit_cap, hit_count + b, status);
  h.tri = tri1;
  h.w[0] = w1[0]; h.w[1] = w1[1]; h.w[2] = w1[2];
  xy = hit_xy(g.x0, g.y0, g.dx, g.dy, i, j, 1, w1[1], w1[2]);
  h.x = xy.x;
  h.y = xy.y;
  warp_append_hit(ok1, h, hb, hit_cap, hit_count + b, status);
  Work64* wb = work + (int64_t)b * work_cap;
  warp_append_work(wk0, Work64{sample, src_k, tri0, r0 == 2 ? 0 : 1, 0}, wb, work_cap,
                   work_count + b, status, counters);
  warp_append_work(wk1, Work64{sample, src_k, tri1, r1 == 2 ? 0 : 1, 0}, wb, work_cap,
                   work_count + b, status, counters);
}

// One work item = 32 positions ("a strip"), one warp, one block; a position
// is two vertically adjacent cells of one cell column (rows j and j + 1),
// which share a row of nodes.  For each chunk of up to 32 sources: (1) lane k
// tests source k against a conservative source-plane box of the strip,
//   beta_x in [min theta_x - r max alpha_x, max theta_x - r min alpha_x]
// (the same in y) widened by the strip's largest vertex uncertainty, whose
// extremes every lane receives from the warp reductions; (2) the warp walks
// the surviving sources (a ballot mask) and runs the per-cell test for each.
// Most pairs never reach the per-cell arithmetic.  No barrier and no shared
// memory besides the staged sources.
//
// The kernel is latency-bound (the per-item chain of node loads and warp
// reductions; its time barely changes between 1 and 20 sources): two cells
// per thread halve the number of item iterations.  Sixteen one-warp blocks
// per SM (128 registers) measure faster than more blocks with spills.
__global__ void __launch_bounds__(kSearchThreads, kSearchBlocksPerSM)
    k_search32(const float4* __restrict__ nodes, const SampleGrid* __restrict__ grids,
               const int64_t* __restrict__ item_off, int n_samples, int64_t n_items, Sources src,
               Hit* __restrict__ hits, int64_t hit_cap, Work64* __restrict__ work,
               int64_t work_cap, unsigned long long* hit_count, unsigned long long* work_count,
               long long* counters, uint32_t* status,
               unsigned long long* __restrict__ /*next_item: unused, static items*/) {
  static_assert(kSearch32Rows == 2, "the kernel handles two cell rows per thread");
  static_assert(kSearchThreads == 32, "one warp per block and per work item");
  __shared__ SrcSmem ss[kMaxSrcSmem];
  const float u = kU32;
  const int lane = threadIdx.x;
  long long n_hit = 0, n_amb = 0, n_ref = 0;
  int staged = -1;  // sample whose whole source list is in ss (block-uniform)
  // static distribution of the items, a contiguous range per block: the
  // search follows the deflection on the same stream, so every block starts
  // together, and the fetch latency of a shared counter would sit on each
  // item's critical path; consecutive items mostly share a sample (its
  // sources stay staged)
  const int64_t per_block = (n_items + gridDim.x - 1) / gridDim.x;
  const int64_t it0 = (int64_t)blockIdx.x * per_block;
  const int64_t it1 = min(n_items, it0 + per_block);
  int b = it0 < n_items ? find_sample(item_off, n_samples, it0) : 0;
  for (int64_t item = it0; item < it1; ++item) {
    while (item >= item_off[b + 1]) ++b;
    const SampleGrid g = grids[b];
    const int sample = src.sample_base + b;
    // this thread's cell column i and cell rows j, j + 1 (see search32_items)
    const int cw = g.nx - 1, ch = g.ny - 1;
    const int64_t npos = ((int64_t)ch + 1) / 2 * cw;
    const int64_t p = (item - item_off[b]) * kSearchThreads + threadIdx.x;
    const bool validA = p < npos;
    const int64_t pc = validA ? p : 0;
    int i, band;
    if (npos < ((int64_t)1 << 31)) {  // 32-bit index arithmetic
      const unsigned c32 = (unsigned)pc, w32 = (unsigned)cw;
      band = (int)(c32 / w32);
      i = (int)(c32 - (unsigned)band * w32);
    } else {
      band = (int)(pc / cw);
      i = (int)(pc - (int64_t)band * cw);
    }
    const int j = 2 * band;
    const bool validB = validA && j + 1 < ch;
    const int64_t n00 = g.node_off + (int64_t)j * g.nx + i;
    // rows j, j + 1 and j + 2 (a copy of row j + 1 when there is no second cell)
    const int64_t n02 = validB ? n00 + 2 * (int64_t)g.nx : n00 + g.nx;
    const float4 v00 = nodes[n00], v10 = nodes[n00 + 1], v01 = nodes[n00 + g.nx],
                 v11 = nodes[n00 + g.nx + 1], v02 = nodes[n02], v12 = nodes[n02 + 1];
    const float hx = g.dxf, hy = g.dyf, gx0 = g.x0f, gy0 = g.y0f;
    const float hmax = fmaxf(fabsf(hx), fabsf(hy));
    const float xl = fmaf((float)i, hx, gx0);
    const float xr = fmaf((float)(i + 1), hx, gx0);
    const float yb = fmaf((float)j, hy, gy0);
    const float ym = fmaf((float)(j + 1), hy, gy0);
    const float yt = fmaf((float)(j + 2), hy, gy0);
    // largest vertex bound and |alpha|_1 over both cells (the culling tests
    // use these; the triangle tests use each vertex's own)
    const float emax = fmaxf(fmaxf(fmaxf(v00.z, v10.z), fmaxf(v01.z, v11.z)),
                             fmaxf(v02.z, v12.z));
    const float lmax =
        fmaxf(fmaxf(fmaxf(fabsf(v00.x) + fabsf(v00.y), fabsf(v10.x) + fabsf(v10.y)),
                    fmaxf(fabsf(v01.x) + fabsf(v01.y), fabsf(v11.x) + fabsf(v11.y))),
              fmaxf(fabsf(v02.x) + fabsf(v02.y), fabsf(v12.x) + fabsf(v12.y)));
    // the strip's box (every lane receives the warp-wide minima and maxima)
    const float inf = __int_as_float(0x7f800000);
    StripBox B;
    B.tx0 = warp_min(validA ? xl : inf);
    B.tx1 = warp_max(validA ? xr : -inf);
    B.ty0 = warp_min(validA ? yb : inf);
    B.ty1 = warp_max(validA ? (validB ? yt : ym) : -inf);
    B.ax0 = warp_min(validA ? fminf(fminf(fminf(v00.x, v10.x), fminf(v01.x, v11.x)),
                                    fminf(v02.x, v12.x))
                            : inf);
    B.ax1 = warp_max(validA ? fmaxf(fmaxf(fmaxf(v00.x, v10.x), fmaxf(v01.x, v11.x)),
                                    fmaxf(v02.x, v12.x))
                            : -inf);
    B.ay0 = warp_min(validA ? fminf(fminf(fminf(v00.y, v10.y), fminf(v01.y, v11.y)),
                                    fminf(v02.y, v12.y))
                            : inf);
    B.ay1 = warp_max(validA ? fmaxf(fmaxf(fmaxf(v00.y, v10.y), fmaxf(v01.y, v11.y)),
                                    fmaxf(v02.y, v12.y))
                            : -inf);
    B.e = warp_max(validA ? emax : 0.0f);
    B.l = warp_max(validA ? lmax : 0.0f);
    const bool any_valid = __any_sync(0xffffffffu, validA);
    // |box corners|_1, the same for every source of the strip
    const float box1 = __fadd_ru(__fadd_ru(fabsf(B.tx0), fabsf(B.tx1)),
                                 __fadd_ru(fabsf(B.ty0), fabsf(B.ty1)));
    const double* sxy = src.xy + (int64_t)sample * src.n_src * 2;
    const double* sr = src.r + (int64_t)sample * src.n_src * (src.stride_r ? 1 : 0);
    for (int s0 = 0; s0 < src.n_src; s0 += kMaxSrcSmem) {
      const int sn = min(kMaxSrcSmem, src.n_src - s0);
      const bool whole = sn == src.n_src;
      if (!whole || staged != sample) {
        __syncwarp();  // earlier readers of ss are done
        for (int v = lane; v < sn; v += kSearchThreads) {
          const double pxd = sxy[2 * (s0 + v)], pyd = sxy[2 * (s0 + v) + 1], rd = sr[s0 + v];
          // searched only with a finite position and a ratio 0 <= r < 1e30
          // (Eq. 13); otherwise latched, and the NaN ratio fails every
          // comparison of the cull, so the source has no images.  Tested on
          // the bits (lt_source.cuh: every warp stages at once, and FP64
          // compares would queue on the FP64 unit).
          const bool ok = source_ok(pxd, pyd, rd);
          if (!ok) atomicOr(status, ST_NONFINITE);
          const float px = (float)pxd, py = (float)pyd;
          ss[v] = SrcSmem{px, py, ok ? (float)rd : __int_as_float(0x7fffffff),
                          __fmul_ru(u, __fmaf_ru(4.0f, g.theta_max,
                                                 __fadd_ru(fabsf(px), fabsf(py))))};
        }
        __syncwarp();
      }
      staged = whole ? sample : -1;
      for (int c0 = 0; c0 < sn; c0 += 32) {
        // (1) lane k tests source c0 + k against the strip's box; the warp
        // then walks the surviving sources (a ballot mask), one at a time
        unsigned keep_mask = 0u;
        if (any_valid) {
          bool keep = false;
          if (c0 + lane < sn) {
            const SrcSmem S = ss[c0 + lane];
            const float wmu = mu_up(__fmaf_ru(
                S.r, B.e,
                __fmaf_ru(u, __fmaf_ru(2.0f, __fadd_ru(box1, __fadd_ru(fabsf(S.px), fabsf(S.py))),
                                       __fmul_ru(__fmul_ru(4.0f, S.r), B.l)),
                          S.mu0)));
            const float bx0 = fmaf(-S.r, B.ax1, B.tx0), bx1 = fmaf(-S.r, B.ax0, B.tx1);
            const float by0 = fmaf(-S.r, B.ay1, B.ty0), by1 = fmaf(-S.r, B.ay0, B.ty1);
            keep = S.px >= bx0 - wmu && S.px <= bx1 + wmu && S.py >= by0 - wmu &&
                   S.py <= by1 + wmu;
          }
          keep_mask = __ballot_sync(0xffffffffu, keep);
        }
      // (2) the surviving sources, one per iteration
      while (keep_mask) {
        const int k = c0 + __ffs(keep_mask) - 1;
        keep_mask &= keep_mask - 1u;
        const SrcSmem S = ss[k];
        const float dl = xl - S.px, dr = xr - S.px;
        const float db = yb - S.py, dm = ym - S.py, dt = yt - S.py;
        // relative mapped vertices beta_v - P = (theta_v - P) - r alpha_v
        const float a00x = fmaf(-S.r, v00.x, dl), a00y = fmaf(-S.r, v00.y, db);
        const float a10x = fmaf(-S.r, v10.x, dr), a10y = fmaf(-S.r, v10.y, db);
        const float a01x = fmaf(-S.r, v01.x, dl), a01y = fmaf(-S.r, v01.y, dm);
        const float a11x = fmaf(-S.r, v11.x, dr), a11y = fmaf(-S.r, v11.y, dm);
        const float a02x = fmaf(-S.r, v02.x, dl), a02y = fmaf(-S.r, v02.y, dt);
        const float a12x = fmaf(-S.r, v12.x, dr), a12y = fmaf(-S.r, v12.y, dt);
        const float dxm = fmaxf(fabsf(dl), fabsf(dr));
        const float base = __fmaf_ru(__fmul_ru(u * 2.0f, S.r), lmax, S.mu0);
        const float muA = mu_up(__fmaf_ru(
            S.r, emax, __fmaf_ru(u * 2.0f, __fadd_ru(dxm, fmaxf(fabsf(db), fabsf(dm))), base)));
        const float muB = mu_up(__fmaf_ru(
            S.r, emax, __fmaf_ru(u * 2.0f, __fadd_ru(dxm, fmaxf(fabsf(dm), fabsf(dt))), base)));
        const bool candA = validA && fminf(fminf(a00x, a10x), fminf(a01x, a11x)) <= muA &&
                           fmaxf(fmaxf(a00x, a10x), fmaxf(a01x, a11x)) >= -muA &&
                           fminf(fminf(a00y, a10y), fminf(a01y, a11y)) <= muA &&
                           fmaxf(fmaxf(a00y, a10y), fmaxf(a01y, a11y)) >= -muA;
        const bool candB = validB && fminf(fminf(a01x, a11x), fminf(a02x, a12x)) <= muB &&
                           fmaxf(fmaxf(a01x, a11x), fmaxf(a02x, a12x)) >= -muB &&
                           fminf(fminf(a01y, a11y), fminf(a02y, a12y)) <= muB &&
                           fmaxf(fmaxf(a01y, a11y), fmaxf(a02y, a12y)) >= -muB;
        if (!__any_sync(0xffffffffu, candA || candB)) continue;
        // per-vertex bounds
        auto muv = [&](const float4& v, float d) {
          return mu_up(__fmaf_ru(
              S.r, v.z,
              __fmaf_ru(u * 2.0f, __fmaf_ru(S.r, __fadd_ru(fabsf(v.x), fabsf(v.y)), d), S.mu0)));
        };
        int r0 = 0, r1 = 0;
        float w0[3], w1[3], pe0 = 0.0f, pe1 = 0.0f;
        const float m01 = muv(v01, __fadd_ru(fabsf(dl), fabsf(dm)));
        const float m11 = muv(v11, __fadd_ru(fabsf(dr), fabsf(dm)));
        if (candA) {
          const float m00 = muv(v00, __fadd_ru(fabsf(dl), fabsf(db)));
          const float m10 = muv(v10, __fadd_ru(fabsf(dr), fabsf(db)));
          // T0 = (v00, v10, v11), T1 = (v00, v11, v01)
          r0 = classify32(a00x, a00y, a10x, a10y, a11x, a11y, m00, m10, m11, w0, &pe0);
          r1 = classify32(a00x, a00y, a11x, a11y, a01x, a01y, m00, m11, m01, w1, &pe1);
        }
        bool ok0 = r0 == 1 && pe0 * hmax <= (float)LT_POS_TOL;
        bool ok1 = r1 == 1 && pe1 * hmax <= (float)LT_POS_TOL;
        emit_cell(g, sample, b, s0 + k, (int64_t)j * cw + i, i, j, r0, r1, w0, w1, ok0, ok1,
                  hits, hit_cap, work, work_cap, hit_count, work_count, status, counters);
        n_hit += (int)ok0 + (int)ok1;
        n_amb += (int)(r0 == 2) + (int)(r1 == 2);
        n_ref += (int)(r0 == 1 && !ok0) + (int)(r1 == 1 && !ok1);
        r0 = 0;
        r1 = 0;
        pe0 = 0.0f;
        pe1 = 0.0f;
        if (candB) {
          const float m02 = muv(v02, __fadd_ru(fabsf(dl), fabsf(dt)));
          const float m12 = muv(v12, __fadd_ru(fabsf(dr), fabsf(dt)));
          // the cell above: T0 = (v01, v11, v12), T1 = (v01, v12, v02)
          r0 = classify32(a01x, a01y, a11x, a11y, a12x, a12y, m01, m11, m12, w0, &pe0);
          r1 = classify32(a01x, a01y, a12x, a12y, a02x, a02y, m01, m12, m02, w1, &pe1);
        }
        ok0 = r0 == 1 && pe0 * hmax <= (float)LT_POS_TOL;
        ok1 = r1 == 1 && pe1 * hmax <= (float)LT_POS_TOL;
        emit_cell(g, sample, b, s0 + k, (int64_t)(j + 1) * cw + i, i, j + 1, r0, r1, w0, w1,
                  ok0, ok1, hits, hit_cap, work, work_cap, hit_count, work_count, status,
                  counters);
        n_hit += (int)ok0 + (int)ok1;
        n_amb += (int)(r0 == 2) + (int)(r1 == 2);
        n_ref += (int)(r0 == 1 && !ok0) + (int)(r1 == 1 && !ok1);
      }
      }
    }
  }
  // block-level counter update (one atomic per counter per warp)
  for (int o = 16; o > 0; o >>= 1) {
    n_hit += __shfl_xor_sync(0xffffffffu, n_hit, o);
    n_amb += __shfl_xor_sync(0xffffffffu, n_amb, o);
    n_ref += __shfl_xor_sync(0xffffffffu, n_ref, o);
  }
  if (lane == 0 && (n_hit | n_amb | n_ref)) {
    atomicAdd((unsigned long long*)&counters[CNT_HITS], (unsigned long long)n_hit);
    atomicAdd((unsigned long long*)&counters[CNT_AMBIG], (unsigned long long)n_amb);
    atomicAdd((unsigned long long*)&counters[CNT_REFINE], (unsigned long long)n_ref);
  }
}

cudaError_t launch_search32(const float4* nodes, const SampleGrid* grids, const int64_t* item_off,
                            int n_samples, int64_t n_items, Sources src, Hit* hits,
                            int64_t hit_cap, Work64* work, int64_t work_cap,
                            unsigned long long* hit_count, unsigned long long* work_count,
                            long long* counters, uint32_t* status,
                            unsigned long long* next_item, int sm_count, cudaStream_t st) {
  if (n_items <= 0 || src.n_src <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search32, kSearchThreads, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)sm_count * per_sm;
  if (blocks > n_items) blocks = n_items;
  k_search32<<<(unsigned)blocks, kSearchThreads, 0, st>>>(nodes, grids, item_off, n_samples,
                                                          n_items, src, hits, hit_cap, work,
                                                          work_cap, hit_count, work_count,
                                                          counters, status, next_item);
  return cudaGetLastError();
}

// ------------------------------------------------- tight FP32 resolution
// The search certifies with the coarse node bound.  The work items it leaves
// undecided (and its certain hits whose position bound is too large) are
// re-evaluated here before any FP64 work: every distinct node of those items
// gets a tighter FP32 deflection (k_res_tight32), and every item is
// classified again (k_res_tri32).  Items decided there are done; the others
// list their nodes for the FP64 stage.
//
// k_res_tight32: one block per node.  The node is translated to each
// potential's centre in FP64 and rounded once (error u |Delta|, relative to
// the distance, instead of the u (Theta + |c|) of an FP32 translation), the
// potential's FP32 deflection is evaluated from there by the deflection
// kernels' per-potential functions, and the potentials' deflections are
// summed in FP64 (thread l takes potentials l, l + 128, ... of the
// kind-sorted records; the threads' sums are combined by a butterfly of
// shuffles per warp and then across the warps).  The
// bound is then each potential's evaluation terms (G |g| per node for the
// PIEMD, 2 |alpha_k|_1 for the rounding of the product that forms alpha_k)
// plus the static input and evaluation terms Seg32::q_tight derived in
// k_prep, plus the FP64 summation: at most n + 8 roundings of 2^-53 on
// sum_k |alpha_k|_1 (summed in FP32, rounded up).
constexpr int kTightThreads = 128;

__global__ void __launch_bounds__(kTightThreads)
    k_res_tight32(const Pot32* __restrict__ pot32, const Seg32* __restrict__ seg, int n_pot,
                  const SampleGrid* __restrict__ grids, const unsigned long long* __restrict__ keys,
                  const int32_t* __restrict__ ulist, const unsigned int* __restrict__ n_unique,
                  TightVal* __restrict__ tval, long long* counters) {
  constexpr int NW = kTightThreads / 32;
  __shared__ double s_x[NW], s_y[NW];
  __shared__ float s_a[NW], s_e[NW];
  grid_dependency_wait();
  const unsigned int nu = *n_unique;
  if (blockIdx.x == 0 && threadIdx.x == 0 && nu)
    atomicAdd((unsigned long long*)&counters[CNT_TIGHT_NODES], (unsigned long long)nu);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // one block per node: thread l takes potentials l, l + 128, ...
  for (unsigned int t = blockIdx.x; t < nu; t += gridDim.x) {
    const int32_t slot = ulist[t];
    const unsigned long long key = keys[slot];
    const int b = (int)(key >> 40);
    const int64_t node = (int64_t)(key & ((1ull << 40) - 1));
    const SampleGrid g = grids[b];
    const Seg32 sg = seg[b];
    const int j = (int)(node / g.nx), i = (int)(node - (int64_t)j * g.nx);
    // the node's FP64 position, formed as the FP64 stages and the reference
    // form it (product and sum rounded separately, never contracted)
    const double X = __dadd_rn(g.x0, __dmul_rn((double)i, g.dx));
    const double Y = __dadd_rn(g.y0, __dmul_rn((double)j, g.dy));
    const Pot32* pb = pot32 + (int64_t)b * n_pot;
    double sx = 0.0, sy = 0.0;
    float er = 0.0f, sa = 0.0f;
    for (int k = threadIdx.x; k < n_pot; k += kTightThreads) {
      Pot32 r = pb[k];
      // translated in FP64, rounded once; the record's centre set to 0 so
      // that the function's own translation is exact
      const float dx = (float)(X - r.c64.x);
      const float dy[1] = {(float)(Y - r.c64.y)};
      r.f[0].x = 0.0f;
      r.f[0].y = 0.0f;
      // the input errors are in q_tight; 1e-30 keeps an SIS/SIE node whose
      // translation rounds to zero distance unbounded (+inf)
      float px[1] = {0.0f}, py[1] = {0.0f}, ek[1] = {0.0f};
      if (k < sg.n_sis)
        sis32_nodes<float, 1, true>(r.f, 1e-30f, dx, dy, px, py, ek);
      else if (k < sg.n_sis + sg.n_piemd)
        piemd32_nodes<float, 1, true>(r.f, 1e-30f, dx, dy, px, py, ek);
      else
        sie32_nodes<float, 1, true>(r.f, 1e-30f, dx, dy, px, py, ek);
      sx += (double)px[0];
      sy += (double)py[0];
      sa = __fadd_ru(sa, __fadd_ru(fabsf(px[0]), fabsf(py[0])));
      er += ek[0];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sa = __fadd_ru(sa, __shfl_xor_sync(0xffffffffu, sa, o));
      er += __shfl_xor_sync(0xffffffffu, er, o);
    }
    if (lane == 0) {
      s_x[wid] = sx;
      s_y[wid] = sy;
      s_a[wid] = sa;
      s_e[wid] = er;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < NW; ++w) {
        sx += s_x[w];
        sy += s_y[w];
        sa = __fadd_ru(sa, s_a[w]);
        er += s_e[w];
      }
      // FP64 summation of n terms (sequential per thread, 5 butterfly
      // levels, NW - 1 additions across warps): at most n + 8 roundings of
      // 2^-53 each on sum |alpha_k|, in units of u: (n + 8) 2^-29 sa
      const float fp64sum = __fmul_ru(sa, __fmul_ru((float)(n_pot + 8), 1.8626451e-09f));
      const float e = node_bound(__fadd_ru(__fadd_ru(er, sg.q_tight), fp64sum), n_pot);
      tval[slot] = TightVal{sx, sy, e, 0.0f};
    }
    __syncthreads();  // the block's partial sums are read before the next node
  }
}

// Vertex v (0, 1, 2) of triangle tri: cell (i, j) = (tri/2 mod (nx-1),
// tri/2 div (nx-1)); T0 = (v00, v10, v11), T1 = (v00, v11, v01).
__device__ __forceinline__ void tri_vertex32(int nx, int64_t tri, int v, int& i, int& j) {
  const int64_t cell = tri / 2;
  const int t = (int)(tri % 2);
  i = (int)(cell % (nx - 1)) + (v == 0 ? 0 : (v == 1 ? 1 : (t == 0 ? 1 : 0)));
  j = (int)(cell / (nx - 1)) + (v == 0 ? 0 : (v == 1 ? (t == 0 ? 0 : 1) : 1));
}

__global__ void k_res_tri32(const SampleGrid* __restrict__ grids, Sources src,
                            Work64* __restrict__ work, const unsigned long long* __restrict__ work_count,
                            int n_samples, int64_t work_cap, const int32_t* __restrict__ vslot,
                            const TightVal* __restrict__ tval, Hit* __restrict__ hits,
                            int64_t hit_cap, unsigned long long* hit_count, long long* counters,
                            uint32_t* status, uint32_t* __restrict__ flag64,
                            int32_t* __restrict__ ulist64, unsigned int* __restrict__ n64) {
  grid_dependency_wait();
  const float u = kU32;
  long long n_hit = 0, n_left = 0;
  const int64_t total = (int64_t)n_samples * work_cap;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(f / work_cap);
    const int64_t idx = f - (int64_t)b * work_cap;
    const unsigned long long cnt = work_count[b];
    if ((unsigned long long)idx >= (cnt < (unsigned long long)work_cap ? cnt : work_cap)) continue;
    const Work64 wk = work[f];
    const SampleGrid g = grids[b];
    // the mapped vertex relative to the source, beta_v - P = (theta_v - P)
    // - r alpha_v, formed in FP64 from the node's FP64 position, the FP64
    // source and ratio and the re-evaluated deflection (every FP64 operation
    // rounded separately), then rounded once to FP32 for the orientation
    // test.  Its bound: r E (the deflection's) + the rounding to FP32,
    // u |.|_1, + the three FP64 roundings of each coordinate (2^-50 on the
    // magnitudes involved, a margin over 3 x 2^-53), and the second-order
    // terms (mu_up).
    const double* sxy = src.xy + (int64_t)wk.sample * src.n_src * 2;
    const double px = sxy[2 * wk.src], py = sxy[2 * wk.src + 1];
    const double r = src.r[(int64_t)wk.sample * src.n_src * (src.stride_r ? 1 : 0) + wk.src];
    const float rf = __double2float_ru(fabs(r));
    float ax[3], ay[3], mv[3];
    bool ok = true;
    for (int v = 0; v < 3; ++v) {
      const int32_t slot = vslot[f * 3 + v];
      if (slot < 0) { ok = false; break; }
      int i, j;
      tri_vertex32(g.nx, wk.tri, v, i, j);
      const TightVal a = tval[slot];
      const double dx = __dsub_rn(__dadd_rn(g.x0, __dmul_rn((double)i, g.dx)), px);
      const double dy = __dsub_rn(__dadd_rn(g.y0, __dmul_rn((double)j, g.dy)), py);
      const double bx = __dsub_rn(dx, __dmul_rn(r, a.ax)), by = __dsub_rn(dy, __dmul_rn(r, a.ay));
      ax[v] = (float)bx;
      ay[v] = (float)by;
      const float mag = __double2float_ru(fabs(dx) + fabs(dy) + fabs(r) * (fabs(a.ax) + fabs(a.ay)));
      mv[v] = mu_up(__fmaf_ru(
          rf, a.e,
          __fmaf_ru(u, __fadd_ru(fabsf(ax[v]), fabsf(ay[v])), __fmul_ru(8.8817842e-16f, mag))));
    }
    if (!ok) {  // cannot happen with the table sized as it is; recorded, never silent
      atomicOr(status, ST_OVERFLOW_WORK);
      continue;
    }
    float w[3], pe = 0.0f;
    const int cls = classify32(ax[0], ay[0], ax[1], ay[1], ax[2], ay[2], mv[0], mv[1], mv[2], w,
                               &pe);
    const float hmax = fmaxf(fabsf(g.dxf), fabsf(g.dyf));
    bool done = cls == 0;
    if (cls == 1 && pe * hmax <= (float)LT_POS_TOL) {
      const int64_t cell = wk.tri / 2;
      const int t = (int)(wk.tri % 2);
      const int ci = (int)(cell % (g.nx - 1)), cj = (int)(cell / (g.nx - 1));
      Hit h;
      h.src = wk.src;
      h.fp64 = 0;
      h.tri = wk.tri;
      h.w[0] = w[0]; h.w[1] = w[1]; h.w[2] = w[2];
      const double2 xy = hit_xy(g.x0, g.y0, g.dx, g.dy, ci, cj, t, w[1], w[2]);
      h.x = xy.x;
      h.y = xy.y;
      const unsigned long long k = atomicAdd(hit_count + b, 1ull);
      if (k < (unsigned long long)hit_cap) hits[(int64_t)b * hit_cap + k] = h;
      else atomicOr(status, ST_OVERFLOW_HITS);
      ++n_hit;
      done = true;
    }
    work[f].resolved = done ? 1 : 0;
    if (!done) {
      ++n_left;
      for (int v = 0; v < 3; ++v) {
        const int32_t slot = vslot[f * 3 + v];
        if (atomicExch(&flag64[slot], 1u) == 0u) ulist64[atomicAdd(n64, 1u)] = slot;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    n_hit += __shfl_xor_sync(0xffffffffu, n_hit, o);
    n_left += __shfl_xor_sync(0xffffffffu, n_left, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (n_hit) atomicAdd((unsigned long long*)&counters[CNT_HITS], (unsigned long long)n_hit);
    if (n_left)
      atomicAdd((unsigned long long*)&counters[CNT_FP64_ITEMS], (unsigned long long)n_left);
  }
}

cudaError_t launch_tight32(const Pot32* pot32, const Seg32* seg, int n_pot,
                           const SampleGrid* grids, Sources src, Work64* work,
                           const unsigned long long* work_count, int n_samples, int64_t work_cap,
                           Hit* hits, int64_t hit_cap, unsigned long long* hit_count,
                           long long* counters, uint32_t* status, ResolveScratch rs,
                           int sm_count, cudaStream_t st) {
  // one block per distinct node (at most three per item)
  int64_t b1 = (int64_t)n_samples * work_cap * 3;
  if (b1 > (int64_t)sm_count * 8) b1 = (int64_t)sm_count * 8;
  cudaError_t e = launch_pdl(k_res_tight32, dim3((unsigned)b1), dim3(kTightThreads), st, pot32,
                             seg, n_pot, grids, rs.keys, rs.ulist, rs.n_unique, rs.tval, counters);
  if (e != cudaSuccess) return e;
  int64_t b2 = ((int64_t)n_samples * work_cap + 127) / 128;
  if (b2 > (int64_t)sm_count * 16) b2 = (int64_t)sm_count * 16;
  return launch_pdl(k_res_tri32, dim3((unsigned)b2), dim3(128), st, grids, src, work, work_count,
                    n_samples, work_cap, rs.vslot, rs.tval, hits, hit_cap, hit_count, counters,
                    status, rs.flag64, rs.ulist64, rs.n64);
}

}  // namespace lt
