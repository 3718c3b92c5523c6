// FP32 deflection of the mixed-precision path: k_deflect32, a potential-tiled
// deflection of every node (Sect. 2.2.2 / Algorithm 1 superposition) with a
// running first-order error bound per node (error propagation in the style of
// App. A).
#include <cuda_runtime.h>
#include <stdint.h>

#include "lt_internal.cuh"
#include "lt_fp32.cuh"

namespace lt {

// --------------------------------------------------------------- deflection
// MINB: the resident blocks per SM the register allocation must allow (left
// to the compiler, the (256, 4) shape is squeezed into 64 registers and spills)
// TIGHT: the node's tight running bound (deflection grids with a bound) or
// the coarse one (the chi^2 path, whose undecided triangles are re-evaluated
// with the tight bound); see lt_fp32.cuh.
template <int NT, int NPT, int MINB, bool TIGHT>
__global__ void __launch_bounds__(NT, MINB) k_deflect32(const Pot32* __restrict__ pot32,
                                                  const Seg32* __restrict__ seg, int n_pot,
                                                  const SampleGrid* __restrict__ grids,
                                                  const float* __restrict__ coords,
                                                  const int64_t* __restrict__ item_off,
                                                  int n_samples, int64_t n_items,
                                                  float4* __restrict__ node_out,
                                                  unsigned long long* __restrict__ next_item) {
  __shared__ float4 sp[kChunk32 * 5];
  __shared__ long long s_item;
  grid_dependency_wait();
  int staged = -1;  // sample whose records sp holds (block-uniform)
  int b = 0;        // sample of the previous item: items arrive in increasing order
  for (;;) {
    // dynamic distribution of the equal-size work items: blocks that start
    // late (another kernel still resident on their SM) simply take fewer
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(next_item, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= n_items) break;
    if (item >= item_off[b + 1])  // a later sample: search from the previous one on
      b += find_sample(item_off + b, n_samples - b, item);
    const SampleGrid g = grids[b];
    const Seg32 sg = seg[b];
    // this thread's column i and rows j0 .. j0 + NPT - 1 (see defl32_items)
    const int64_t bands = ((int64_t)g.ny + NPT - 1) / NPT;
    const int64_t p = (item - item_off[b]) * NT + threadIdx.x;
    const bool live = p < bands * g.nx;
    const int64_t pc = live ? p : 0;
    const int band = (int)(pc / g.nx);
    const int i = (int)(pc - (int64_t)band * g.nx);
    const int j0 = band * NPT;
    // node coordinates rounded once from FP64 (the grid's coordinate table):
    // error u|theta| (App. A's stored-value model), not u|x0| as an FP32
    // x0 + i*dx would give, and no FP64 instruction in the kernel
    const float* cx = coords + g.coord_off;
    const float X = cx[i];
    float Y[NPT], AX[NPT], AY[NPT], ER[NPT];
#pragma unroll
    for (int m = 0; m < NPT; ++m) Y[m] = cx[g.nx + min(j0 + m, g.ny - 1)];
    deflect32_nodes<NT, NPT, TIGHT>(pot32 + (int64_t)b * n_pot, n_pot, sg, g.theta_max, X, Y,
                                    sp, AX, AY, ER, staged != b);
    staged = b;
    const float qs = TIGHT ? sg.q_tot : sg.c_tot;
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      if (live && j0 + m < g.ny)
        node_out[g.node_off + (int64_t)(j0 + m) * g.nx + i] =
            make_float4(AX[m], AY[m], node_bound(__fadd_ru(ER[m], qs), n_pot), 0.0f);
    }
  }
}

template <int NT, int NPT, int MINB, bool TIGHT>
static cudaError_t launch_deflect32_t(const Pot32* pot32, const Seg32* seg, int n_pot,
                                      const SampleGrid* grids, const float* coords,
                                      const int64_t* item_off,
                                      int n_samples, int64_t n_items, float4* node_out,
                                      unsigned long long* next_item, int sm_count,
                                      cudaStream_t st) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deflect32<NT, NPT, MINB, TIGHT>, NT,
                                                0);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)sm_count * per_sm;
  if (blocks > n_items) blocks = n_items;
  if (blocks < 1) return cudaSuccess;
  return launch_pdl(k_deflect32<NT, NPT, MINB, TIGHT>, dim3((unsigned)blocks), dim3(NT), st,
                    pot32, seg, n_pot, grids, coords, item_off, n_samples, n_items, node_out,
                    next_item);
}

template <int V>
static cudaError_t launch_shape(const Pot32* pot32, const Seg32* seg, int n_pot,
                               const SampleGrid* grids, const float* coords,
                               const int64_t* item_off, int n_samples,
                               int64_t n_items, bool tight, float4* node_out,
                               unsigned long long* next_item, int sm_count, cudaStream_t st) {
  constexpr DeflectShape sh = deflect_shape(V);
  if (tight)
    return launch_deflect32_t<sh.threads, sh.npt, sh.min_blocks, true>(
        pot32, seg, n_pot, grids, coords, item_off, n_samples, n_items, node_out, next_item,
        sm_count, st);
  return launch_deflect32_t<sh.threads, sh.npt, sh.min_blocks, false>(
      pot32, seg, n_pot, grids, coords, item_off, n_samples, n_items, node_out, next_item,
      sm_count, st);
}

cudaError_t launch_deflect32(const Pot32* pot32, const Seg32* seg, int n_pot,
                             const SampleGrid* grids, const float* coords,
                             const int64_t* item_off, int n_samples, int64_t n_items, int shape,
                             bool tight, float4* node_out, unsigned long long* next_item,
                             int sm_count, cudaStream_t st) {
  static_assert(kNumShapes == 8, "one case per launch shape");
  switch (shape) {
    case 1: return launch_shape<1>(pot32, seg, n_pot, grids, coords, item_off, n_samples,
                                   n_items, tight, node_out, next_item, sm_count, st);
    case 2: return launch_shape<2>(pot32, seg, n_pot, grids, coords, item_off, n_samples,
                                   n_items, tight, node_out, next_item, sm_count, st);
    case 3: return launch_shape<3>(pot32, seg, n_pot, grids, coords, item_off, n_samples,
                                   n_items, tight, node_out, next_item, sm_count, st);
    case 4: return launch_shape<4>(pot32, seg, n_pot, grids, coords, item_off, n_samples,
                                   n_items, tight, node_out, next_item, sm_count, st);
    case 5: return launch_shape<5>(pot32, seg, n_pot, grids, coords, item_off, n_samples,
                                   n_items, tight, node_out, next_item, sm_count, st);
    case 6: return launch_shape<6>(pot32, seg, n_pot, grids, coords, item_off, n_samples,
                                   n_items, tight, node_out, next_item, sm_count, st);
    case 7: return launch_shape<7>(pot32, seg, n_pot, grids, coords, item_off, n_samples,
                                   n_items, tight, node_out, next_item, sm_count, st);
    default: return launch_shape<0>(pot32, seg, n_pot, grids, coords, item_off, n_samples,
                                    n_items, tight, node_out, next_item, sm_count, st);
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
