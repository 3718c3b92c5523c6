// FP32 deflection of the mixed-precision path: k_deflect32, a potential-tiled
// deflection of every node (Sect. 2.2.2 / Algorithm 1 superposition) with a
// running first-order error bound per node (error propagation in the style of
// App. A).
#include <cuda_runtime.h>
#include <stdint.h>

#include "lt_internal.cuh"
#include "lt_fp32.cuh"

namespace lt {

constexpr int kChunk32 = 256;  // potentials staged in shared memory at a time

// --------------------------------------------------------------- deflection
template <int NT, int NPT>
__global__ void __launch_bounds__(NT) k_deflect32(const Pot32* __restrict__ pot32,
                                                  const Seg32* __restrict__ seg, int n_pot,
                                                  const SampleGrid* __restrict__ grids,
                                                  const int64_t* __restrict__ item_off,
                                                  int n_samples, int64_t n_items,
                                                  float4* __restrict__ node_out,
                                                  unsigned long long* __restrict__ next_item) {
  __shared__ float4 sp[kChunk32 * 5];
  __shared__ long long s_item;
  for (;;) {
    // dynamic distribution of the equal-size work items: blocks that start
    // late (another kernel still resident on their SM) simply take fewer
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(next_item, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= n_items) break;
    int b = find_sample(item_off, n_samples, item);
    const SampleGrid g = grids[b];
    const Seg32 sg = seg[b];
    const int64_t nodes = (int64_t)g.nx * g.ny;
    const int64_t base = (item - item_off[b]) * (int64_t)(NT * NPT);
        float X[NPT], Y[NPT], AX[NPT], AY[NPT], ER[NPT];
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      int64_t n = base + m * NT + threadIdx.x;
      if (n >= nodes) n = nodes - 1;
      int j = (int)(n / g.nx);
      int i = (int)(n - (int64_t)j * g.nx);
      // node coordinates rounded once from FP64: error u|theta| (App. A's
      // stored-value model), not u|x0| as an FP32 x0 + i*dx would give
      X[m] = (float)(g.x0 + (double)i * g.dx);
      Y[m] = (float)(g.y0 + (double)j * g.dy);
      AX[m] = 0.0f;
      AY[m] = 0.0f;
      ER[m] = 0.0f;
    }
    const float theta1 = g.theta_max;
    const Pot32* pb = pot32 + (int64_t)b * n_pot;
    for (int c0 = 0; c0 < n_pot; c0 += kChunk32) {
      const int cn = min(kChunk32, n_pot - c0);
      __syncthreads();
      for (int v = threadIdx.x; v < cn * 5; v += NT) {
        int k = v / 5, w = v - k * 5;
        float4 val = pb[c0 + k].f[w];
        if (w == 4) {  // translation-error coefficient for this grid
          float4 h = pb[c0 + k].f[0];
          // strictly positive, so that P times an infinite 1/R (a node on an
          // SIS/SIE centre) is +inf, never NaN, even for a zero-mass potential
          val.x = fmaf(val.x, theta1 + fabsf(h.x) + fabsf(h.y), 1e-30f);
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
        piemd32_nodes<NPT>(f, f[4].x, X, Y, AX, AY, ER);
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
            make_float4(AX[m], AY[m], node_bound(ER[m] + qs), 0.0f);
    }
  }
}

template <int NT, int NPT>
static cudaError_t launch_deflect32_t(const Pot32* pot32, const Seg32* seg, int n_pot,
                                      const SampleGrid* grids, const int64_t* item_off,
                                      int n_samples, int64_t n_items, float4* node_out,
                                      unsigned long long* next_item, int sm_count,
                                      cudaStream_t st) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deflect32<NT, NPT>, NT, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)sm_count * per_sm;
  if (blocks > n_items) blocks = n_items;
  if (blocks < 1) return cudaSuccess;
  k_deflect32<NT, NPT><<<(unsigned)blocks, NT, 0, st>>>(pot32, seg, n_pot, grids, item_off,
                                                          n_samples, n_items, node_out,
                                                          next_item);
  return cudaGetLastError();
}

cudaError_t launch_deflect32(const Pot32* pot32, const Seg32* seg, int n_pot,
                             const SampleGrid* grids, const int64_t* item_off, int n_samples,
                             int64_t n_items, int shape, float4* node_out,
                             unsigned long long* next_item, int sm_count, cudaStream_t st) {
  switch (shape) {
    case 1: return launch_deflect32_t<256, 2>(pot32, seg, n_pot, grids, item_off, n_samples,
                                              n_items, node_out, next_item, sm_count, st);
    case 2: return launch_deflect32_t<512, 2>(pot32, seg, n_pot, grids, item_off, n_samples,
                                              n_items, node_out, next_item, sm_count, st);
    case 3: return launch_deflect32_t<128, 4>(pot32, seg, n_pot, grids, item_off, n_samples,
                                              n_items, node_out, next_item, sm_count, st);
    case 4: return launch_deflect32_t<128, 8>(pot32, seg, n_pot, grids, item_off, n_samples,
                                              n_items, node_out, next_item, sm_count, st);
    default: return launch_deflect32_t<256, 4>(pot32, seg, n_pot, grids, item_off, n_samples,
                                               n_items, node_out, next_item, sm_count, st);
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

}  // namespace lt
