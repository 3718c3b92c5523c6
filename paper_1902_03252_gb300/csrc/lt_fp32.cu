// FP32 kernels of the mixed-precision path:
//   k_deflect32  potential-tiled deflection of every node, with a running
//                first-order error bound per node (Sect. 2.2.2 / Algorithm 1
//                superposition; error propagation in the style of App. A);
//   k_search32   fused lens mapping (Eq. 11) and triangle test (Fig. 1) with
//                a certified FP32 orientation filter; certain hits and the
//                pairs that need FP64 are compacted by warp ballots.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lt_internal.cuh"
#include "lt_fp32.cuh"

namespace lt {

// Safety factor applied to the first-order error bound of every node.
constexpr float kBoundSafety = 2.0f;
constexpr int kChunk32 = 256;  // potentials staged in shared memory at a time

__device__ __forceinline__ int find_sample(const int64_t* off, int n, int64_t item) {
  int lo = 0, hi = n;  // off[lo] <= item < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// --------------------------------------------------------------- deflection
template <int NT, int NPT>
__global__ void __launch_bounds__(NT) k_deflect32(const Pot32* __restrict__ pot32,
                                                  const Seg32* __restrict__ seg, int n_pot,
                                                  const SampleGrid* __restrict__ grids,
                                                  const int64_t* __restrict__ item_off,
                                                  int n_samples, int64_t n_items,
                                                  float4* __restrict__ node_out) {
  __shared__ float4 sp[kChunk32 * 5];
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    int b = find_sample(item_off, n_samples, item);
    const SampleGrid g = grids[b];
    const Seg32 sg = seg[b];
    const int64_t nodes = (int64_t)g.nx * g.ny;
    const int64_t base = (item - item_off[b]) * (int64_t)(NT * NPT);
    const float x0 = (float)g.x0, y0 = (float)g.y0, hx = (float)g.dx, hy = (float)g.dy;
    float X[NPT], Y[NPT], AX[NPT], AY[NPT], ER[NPT];
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      int64_t n = base + m * NT + threadIdx.x;
      if (n >= nodes) n = nodes - 1;
      int j = (int)(n / g.nx);
      int i = (int)(n - (int64_t)j * g.nx);
      X[m] = fmaf((float)i, hx, x0);
      Y[m] = fmaf((float)j, hy, y0);
      AX[m] = 0.0f;
      AY[m] = 0.0f;
      ER[m] = 0.0f;
    }
    const float theta4 = 4.0f * g.theta_max;
    const Pot32* pb = pot32 + (int64_t)b * n_pot;
    for (int c0 = 0; c0 < n_pot; c0 += kChunk32) {
      const int cn = min(kChunk32, n_pot - c0);
      __syncthreads();
      for (int v = threadIdx.x; v < cn * 5; v += NT) {
        int k = v / 5, w = v - k * 5;
        float4 val = pb[c0 + k].f[w];
        if (w == 4) {  // translation-error coefficient for this grid
          float4 h = pb[c0 + k].f[0];
          val.x = val.x * (theta4 + fabsf(h.x) + fabsf(h.y));
        }
        sp[v] = val;
      }
      __syncthreads();
      // kind segments [0, n_sis) SIS, [n_sis, n_sis + n_piemd) PIEMD, rest SIE
      const int e_sis = min(max(sg.n_sis - c0, 0), cn);
      const int e_pie = min(max(sg.n_sis + sg.n_piemd - c0, 0), cn);
      for (int k = 0; k < e_sis; ++k) {
        const float4* f = &sp[k * 5];
        const float P = f[4].x;
#pragma unroll
        for (int m = 0; m < NPT; ++m) sis32(f, P, X[m], Y[m], AX[m], AY[m], ER[m]);
      }
      for (int k = e_sis; k < e_pie; ++k) {
        const float4* f = &sp[k * 5];
        const float P = f[4].x;
#pragma unroll
        for (int m = 0; m < NPT; ++m) piemd32(f, P, X[m], Y[m], AX[m], AY[m], ER[m]);
      }
      for (int k = e_pie; k < cn; ++k) {
        const float4* f = &sp[k * 5];
        const float P = f[4].x;
#pragma unroll
        for (int m = 0; m < NPT; ++m) sie32(f, P, X[m], Y[m], AX[m], AY[m], ER[m]);
      }
    }
    const float qs = sg.q_tot;
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      int64_t n = base + m * NT + threadIdx.x;
      if (n < nodes)
        node_out[g.node_off + n] =
            make_float4(AX[m], AY[m], kBoundSafety * kU32 * (ER[m] + qs), 0.0f);
    }
  }
}

template <int NT, int NPT>
static cudaError_t launch_deflect32_t(const Pot32* pot32, const Seg32* seg, int n_pot,
                                      const SampleGrid* grids, const int64_t* item_off,
                                      int n_samples, int64_t n_items, float4* node_out,
                                      int sm_count, cudaStream_t st) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deflect32<NT, NPT>, NT, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)sm_count * per_sm;
  if (blocks > n_items) blocks = n_items;
  if (blocks < 1) return cudaSuccess;
  k_deflect32<NT, NPT><<<(unsigned)blocks, NT, 0, st>>>(pot32, seg, n_pot, grids, item_off,
                                                          n_samples, n_items, node_out);
  return cudaGetLastError();
}

cudaError_t launch_deflect32(const Pot32* pot32, const Seg32* seg, int n_pot,
                             const SampleGrid* grids, const int64_t* item_off, int n_samples,
                             int64_t n_items, int shape, float4* node_out, int sm_count,
                             cudaStream_t st) {
  switch (shape) {
    case 0: return launch_deflect32_t<256, 2>(pot32, seg, n_pot, grids, item_off, n_samples,
                                              n_items, node_out, sm_count, st);
    case 2: return launch_deflect32_t<128, 4>(pot32, seg, n_pot, grids, item_off, n_samples,
                                              n_items, node_out, sm_count, st);
    case 3: return launch_deflect32_t<128, 8>(pot32, seg, n_pot, grids, item_off, n_samples,
                                              n_items, node_out, sm_count, st);
    default: return launch_deflect32_t<256, 4>(pot32, seg, n_pot, grids, item_off, n_samples,
                                               n_items, node_out, sm_count, st);
  }
}

__global__ void k_unpack32(const float4* __restrict__ nodes, int64_t n, float2* __restrict__ alpha,
                           float* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 v = nodes[i];
    alpha[i] = make_float2(v.x, v.y);
    if (err) err[i] = v.z;
  }
}

cudaError_t launch_unpack32(const float4* nodes, int64_t n, float2* alpha, float* err,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  k_unpack32<<<(unsigned)blocks, 256, 0, st>>>(nodes, n, alpha, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------- triangle search
constexpr int kSearchThreads = 256;  // cells per work item (one per thread)
constexpr int kMaxSrcSmem = 1024;    // sources staged in shared memory at a time

// Source data staged per sample: position relative coordinates use FP32.
struct SrcSmem {
  float px, py, r, mu0;  // mu0 = u (4 Theta + |px| + |py|) (input rounding)
};

// Classify one triangle with relative vertices a, b, c (vertex - source,
// FP32) and per-vertex error bounds m[3].  Returns 0 = certainly outside,
// 1 = certainly inside, 2 = undecided.  On 1, w[] receives the weights and
// *pos_err a bound on the position error of the interpolated image
// (in units of the cell size).
__device__ __forceinline__ int classify32(float ax, float ay, float bx, float by, float cx,
                                          float cy, float ma, float mb, float mc, float w[3],
                                          float* pos_err) {
  // edge functions of the origin: e_AB = a x b, e_BC = b x c, e_CA = c x a
  float e0 = fmaf(ax, by, -(ay * bx));
  float e1 = fmaf(bx, cy, -(by * cx));
  float e2 = fmaf(cx, ay, -(cy * ax));
  const float u2 = 2.0f * kU32;
  float la = fabsf(ax) + fabsf(ay), lb = fabsf(bx) + fabsf(by), lc = fabsf(cx) + fabsf(cy);
  float E0 = 1.25f * (ma * lb + mb * la + 2.0f * ma * mb + u2 * (fabsf(ax * by) + fabsf(ay * bx)));
  float E1 = 1.25f * (mb * lc + mc * lb + 2.0f * mb * mc + u2 * (fabsf(bx * cy) + fabsf(by * cx)));
  float E2 = 1.25f * (mc * la + ma * lc + 2.0f * mc * ma + u2 * (fabsf(cx * ay) + fabsf(cy * ax)));
  bool p0 = e0 > E0, p1 = e1 > E1, p2 = e2 > E2;
  bool n0 = e0 < -E0, n1 = e1 < -E1, n2 = e2 < -E2;
  if ((p0 || p1 || p2) && (n0 || n1 || n2)) return 0;
  if ((p0 && p1 && p2) || (n0 && n1 && n2)) {
    float det = e0 + e1 + e2;
    float inv = 1.0f / det;
    w[0] = e1 * inv;
    w[1] = e2 * inv;
    w[2] = e0 * inv;
    float sE = E0 + E1 + E2;
    // |dw_v| <= (E_v + w_v sE)/(|det| - sE); x = A + w_B (B-A) + w_C (C-A)
    *pos_err = 1.1f * 2.0f * sE / (fabsf(det) - sE);
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
    if (idx < (unsigned long long)cap) work[idx] = wk;
    else atomicOr(status, ST_OVERFLOW_WORK);
  }
}

__device__ __forceinline__ float warp_min(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(kSearchThreads)
    k_search32(const float4* __restrict__ nodes, const SampleGrid* __restrict__ grids,
               const int64_t* __restrict__ item_off, int n_samples, int64_t n_items, Sources src,
               Hit* __restrict__ hits, int64_t hit_cap, Work64* __restrict__ work,
               int64_t work_cap, unsigned long long* hit_count, unsigned long long* work_count,
               long long* counters, uint32_t* status) {
  __shared__ SrcSmem ss[kMaxSrcSmem];
  const float u = kU32;
  long long n_hit = 0, n_amb = 0, n_ref = 0;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int b = find_sample(item_off, n_samples, item);
    const SampleGrid g = grids[b];
    const int sample = src.sample_base + b;
    const int64_t cells = (int64_t)(g.nx - 1) * (g.ny - 1);
    const int64_t cell = (item - item_off[b]) * kSearchThreads + threadIdx.x;
    const bool valid = cell < cells;
    const int64_t cl = valid ? cell : 0;
    const int j = (int)(cl / (g.nx - 1));
    const int i = (int)(cl - (int64_t)j * (g.nx - 1));
    const int64_t n00 = g.node_off + (int64_t)j * g.nx + i;
    const float4 v00 = nodes[n00], v10 = nodes[n00 + 1], v01 = nodes[n00 + g.nx],
                 v11 = nodes[n00 + g.nx + 1];
    const float xl = fmaf((float)i, (float)g.dx, (float)g.x0);
    const float xr = fmaf((float)(i + 1), (float)g.dx, (float)g.x0);
    const float yb = fmaf((float)j, (float)g.dy, (float)g.y0);
    const float yt = fmaf((float)(j + 1), (float)g.dy, (float)g.y0);
    const float emax = fmaxf(fmaxf(v00.z, v10.z), fmaxf(v01.z, v11.z));
    const float l00 = fabsf(v00.x) + fabsf(v00.y), l10 = fabsf(v10.x) + fabsf(v10.y);
    const float l01 = fabsf(v01.x) + fabsf(v01.y), l11 = fabsf(v11.x) + fabsf(v11.y);
    const float lmax = fmaxf(fmaxf(l00, l10), fmaxf(l01, l11));
    // Conservative source-plane box of the warp's 32 cells for any r > 0:
    // beta_x in [min theta_x - r max alpha_x, max theta_x - r min alpha_x].
    const float inf = __int_as_float(0x7f800000);
    const float W_tx0 = warp_min(valid ? xl : inf), W_tx1 = warp_max(valid ? xr : -inf);
    const float W_ty0 = warp_min(valid ? yb : inf), W_ty1 = warp_max(valid ? yt : -inf);
    const float W_ax0 = warp_min(valid ? fminf(fminf(v00.x, v10.x), fminf(v01.x, v11.x)) : inf);
    const float W_ax1 = warp_max(valid ? fmaxf(fmaxf(v00.x, v10.x), fmaxf(v01.x, v11.x)) : -inf);
    const float W_ay0 = warp_min(valid ? fminf(fminf(v00.y, v10.y), fminf(v01.y, v11.y)) : inf);
    const float W_ay1 = warp_max(valid ? fmaxf(fmaxf(v00.y, v10.y), fmaxf(v01.y, v11.y)) : -inf);
    const float W_e = warp_max(valid ? emax : 0.0f);
    const float W_l = warp_max(valid ? lmax : 0.0f);
    const bool W_any = __any_sync(0xffffffffu, valid);
    const double* sxy = src.xy + (int64_t)sample * src.n_src * 2;
    const double* sr = src.r + (int64_t)sample * src.n_src * (src.stride_r ? 1 : 0);
    for (int s0 = 0; s0 < src.n_src; s0 += kMaxSrcSmem) {
      const int sn = min(kMaxSrcSmem, src.n_src - s0);
      __syncthreads();
      for (int v = threadIdx.x; v < sn; v += kSearchThreads) {
        float px = (float)sxy[2 * (s0 + v)], py = (float)sxy[2 * (s0 + v) + 1];
        ss[v] = SrcSmem{px, py, (float)sr[s0 + v],
                        u * (4.0f * g.theta_max + fabsf(px) + fabsf(py))};
      }
      __syncthreads();
      for (int k = 0; k < sn; ++k) {
        const SrcSmem S = ss[k];
        {
          // warp-uniform rejection of the whole strip (interval bound widened
          // by the strip's largest vertex uncertainty and a relative margin)
          const float wmu = fmaf(S.r, W_e, S.mu0 + u * (2.0f * (fabsf(W_tx0) + fabsf(W_tx1) +
                                                                fabsf(W_ty0) + fabsf(W_ty1) +
                                                                fabsf(S.px) + fabsf(S.py)) +
                                                         4.0f * S.r * W_l));
          const float bx0 = fmaf(-S.r, W_ax1, W_tx0), bx1 = fmaf(-S.r, W_ax0, W_tx1);
          const float by0 = fmaf(-S.r, W_ay1, W_ty0), by1 = fmaf(-S.r, W_ay0, W_ty1);
          if (!W_any || S.px < bx0 - wmu || S.px > bx1 + wmu || S.py < by0 - wmu ||
              S.py > by1 + wmu)
            continue;
        }
        const float dl = xl - S.px, dr = xr - S.px, db = yb - S.py, dt = yt - S.py;
        // relative mapped vertices beta_v - P = (theta_v - P) - r alpha_v
        const float a00x = fmaf(-S.r, v00.x, dl), a00y = fmaf(-S.r, v00.y, db);
        const float a10x = fmaf(-S.r, v10.x, dr), a10y = fmaf(-S.r, v10.y, db);
        const float a01x = fmaf(-S.r, v01.x, dl), a01y = fmaf(-S.r, v01.y, dt);
        const float a11x = fmaf(-S.r, v11.x, dr), a11y = fmaf(-S.r, v11.y, dt);
        const float dmax = fmaxf(fabsf(dl), fabsf(dr)) + fmaxf(fabsf(db), fabsf(dt));
        const float mu = fmaf(S.r, emax, S.mu0 + u * (2.0f * dmax + 2.0f * S.r * lmax));
        const float minx = fminf(fminf(a00x, a10x), fminf(a01x, a11x));
        const float maxx = fmaxf(fmaxf(a00x, a10x), fmaxf(a01x, a11x));
        const float miny = fminf(fminf(a00y, a10y), fminf(a01y, a11y));
        const float maxy = fmaxf(fmaxf(a00y, a10y), fmaxf(a01y, a11y));
        bool cand = valid && minx <= mu && maxx >= -mu && miny <= mu && maxy >= -mu;
        int r0 = 0, r1 = 0;
        float w0[3], w1[3], pe0 = 0.0f, pe1 = 0.0f;
        if (cand) {
          // per-vertex bounds
          auto muv = [&](float e, float l, float d) {
            return fmaf(S.r, e, S.mu0 + u * (2.0f * d + 2.0f * S.r * l));
          };
          const float m00 = muv(v00.z, l00, fabsf(dl) + fabsf(db));
          const float m10 = muv(v10.z, l10, fabsf(dr) + fabsf(db));
          const float m01 = muv(v01.z, l01, fabsf(dl) + fabsf(dt));
          const float m11 = muv(v11.z, l11, fabsf(dr) + fabsf(dt));
          // T0 = (v00, v10, v11), T1 = (v00, v11, v01)
          r0 = classify32(a00x, a00y, a10x, a10y, a11x, a11y, m00, m10, m11, w0, &pe0);
          r1 = classify32(a00x, a00y, a11x, a11y, a01x, a01y, m00, m11, m01, w1, &pe1);
        }
        const float hmax = fmaxf((float)fabs(g.dx), (float)fabs(g.dy));
        const bool ok0 = r0 == 1 && pe0 * hmax <= (float)LT_POS_TOL;
        const bool ok1 = r1 == 1 && pe1 * hmax <= (float)LT_POS_TOL;
        const bool wk0 = r0 == 2 || (r0 == 1 && !ok0);
        const bool wk1 = r1 == 2 || (r1 == 1 && !ok1);
        if (__any_sync(0xffffffffu, ok0 || ok1 || wk0 || wk1)) {
          const int64_t tri0 = 2 * cl, tri1 = 2 * cl + 1;
          const double X0 = g.x0 + (double)i * g.dx, X1 = g.x0 + (double)(i + 1) * g.dx;
          const double Y0 = g.y0 + (double)j * g.dy, Y1 = g.y0 + (double)(j + 1) * g.dy;
          Hit h;
          h.src = s0 + k;
          h.fp64 = 0;
          // T0 vertices: (X0,Y0), (X1,Y0), (X1,Y1)
          h.tri = tri0;
          h.w[0] = w0[0]; h.w[1] = w0[1]; h.w[2] = w0[2];
          h.x = X0 + (double)w0[1] * (X1 - X0) + (double)w0[2] * (X1 - X0);
          h.y = Y0 + (double)w0[2] * (Y1 - Y0);
          Hit* hb = hits + (int64_t)b * hit_cap;
          warp_append_hit(ok0, h, hb, hit_cap, hit_count + b, status);
          // T1 vertices: (X0,Y0), (X1,Y1), (X0,Y1)
          h.tri = tri1;
          h.w[0] = w1[0]; h.w[1] = w1[1]; h.w[2] = w1[2];
          h.x = X0 + (double)w1[1] * (X1 - X0);
          h.y = Y0 + (double)w1[1] * (Y1 - Y0) + (double)w1[2] * (Y1 - Y0);
          warp_append_hit(ok1, h, hb, hit_cap, hit_count + b, status);
          Work64* wb = work + (int64_t)b * work_cap;
          warp_append_work(wk0, Work64{sample, s0 + k, tri0, r0 == 2 ? 0 : 1, 0}, wb, work_cap,
                           work_count + b, status);
          warp_append_work(wk1, Work64{sample, s0 + k, tri1, r1 == 2 ? 0 : 1, 0}, wb, work_cap,
                           work_count + b, status);
          n_hit += (int)ok0 + (int)ok1;
          n_amb += (int)(r0 == 2) + (int)(r1 == 2);
          n_ref += (int)(r0 == 1 && !ok0) + (int)(r1 == 1 && !ok1);
        }
      }
    }
  }
  // block-level counter update (one atomic per counter per block)
  for (int o = 16; o > 0; o >>= 1) {
    n_hit += __shfl_xor_sync(0xffffffffu, n_hit, o);
    n_amb += __shfl_xor_sync(0xffffffffu, n_amb, o);
    n_ref += __shfl_xor_sync(0xffffffffu, n_ref, o);
  }
  if ((threadIdx.x & 31) == 0 && (n_hit | n_amb | n_ref)) {
    atomicAdd((unsigned long long*)&counters[CNT_HITS], (unsigned long long)n_hit);
    atomicAdd((unsigned long long*)&counters[CNT_AMBIG], (unsigned long long)n_amb);
    atomicAdd((unsigned long long*)&counters[CNT_REFINE], (unsigned long long)n_ref);
  }
}

cudaError_t launch_search32(const float4* nodes, const SampleGrid* grids, const int64_t* item_off,
                            int n_samples, int64_t n_items, Sources src, Hit* hits,
                            int64_t hit_cap, Work64* work, int64_t work_cap,
                            unsigned long long* hit_count, unsigned long long* work_count,
                            long long* counters, uint32_t* status, int sm_count,
                            cudaStream_t st) {
  if (n_items <= 0 || src.n_src <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search32, kSearchThreads, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)sm_count * per_sm;
  if (blocks > n_items) blocks = n_items;
  k_search32<<<(unsigned)blocks, kSearchThreads, 0, st>>>(nodes, grids, item_off, n_samples,
                                                          n_items, src, hits, hit_cap, work,
                                                          work_cap, hit_count, work_count,
                                                          counters, status);
  return cudaGetLastError();
}

}  // namespace lt
