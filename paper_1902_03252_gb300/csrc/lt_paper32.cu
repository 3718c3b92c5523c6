// FP32 side of the paper's mixed-precision rule for a deflection grid (Sect.
// 3.3, App. A.3): widening, distortion criteria, halo patches, compaction.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lt_internal.cuh"
#include "lt_fp32.cuh"

namespace lt {

// ------------------------------------------------- the paper's mixed rule
// Widen the FP32 deflections into the FP64 output and flag the nodes where
// the distortion criteria fire (Eqs. 23-28): with d1 = a1(i,j) - a1(i-1,j),
// d2 = a2(i,j) - a2(i,j-1), d3 = a1(i,j) - a1(i,j-1), d4 = a2(i,j) - a2(i-1,j),
// recompute in FP64 if |h_x - d1| or |h_y - d2| < 0.0092" (h/0.03") or
// |d3| or |d4| > 0.0104" (h/0.03"), h the node spacing along the difference.
__global__ void k_paper_init(const float4* __restrict__ nodes, int nx, int ny, float hx, float hy,
                             double2* __restrict__ out, unsigned char* __restrict__ flags) {
  const int64_t n_all = (int64_t)nx * ny;
  const float t12x = 0.0092f * hx / 0.03f, t12y = 0.0092f * hy / 0.03f;
  const float t34x = 0.0104f * hx / 0.03f, t34y = 0.0104f * hy / 0.03f;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n_all;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(n / nx), i = (int)(n - (int64_t)j * nx);
    const float4 v = nodes[n];
    out[n] = make_double2((double)v.x, (double)v.y);
    bool crit = false;
    if (i >= 1 && j >= 1) {
      const float4 l = nodes[n - 1], b = nodes[n - nx];
      const float d1 = v.x - l.x, d2 = v.y - b.y, d3 = v.x - b.x, d4 = v.y - l.y;
      crit = fabsf(hx - d1) < t12x || fabsf(hy - d2) < t12y || fabsf(d3) > t34y ||
             fabsf(d4) > t34x;
    }
    flags[n] = crit ? 1 : 0;
  }
}

// Square patches centred on every halo: 2*half nodes on a side, half = 200
// for cluster-scale halos (b0 >= LT_PAPER_CLUSTER_B0), 10 for the others
// (App. A.3.2: 400 x 400 and 20 x 20 pixels).  One block per potential.
__global__ void k_paper_patches(const Pot64* __restrict__ pot64, int n_pot, double x0, double y0,
                                double dx, double dy, int nx, int ny,
                                unsigned char* __restrict__ flags) {
  const Pot64 p = pot64[blockIdx.x];
  if (p.b0 <= 0.0) return;  // zero-mass or neutralised potential
  const int half = p.b0 >= LT_PAPER_CLUSTER_B0 ? 200 : 10;
  const long long ic = llround((p.cx - x0) / dx), jc = llround((p.cy - y0) / dy);
  const int side = 2 * half;
  for (int idx = threadIdx.x; idx < side * side; idx += blockDim.x) {
    const long long i = ic - half + idx % side, j = jc - half + idx / side;
    if (i >= 0 && i < nx && j >= 0 && j < ny) flags[j * (long long)nx + i] = 2;
  }
}

// Compact the flagged nodes into a list (warp ballots, one atomic per warp).
__global__ void k_paper_compact(const unsigned char* __restrict__ flags, int64_t n_all,
                                int32_t* __restrict__ list, unsigned long long* count,
                                float* __restrict__ map) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n_all; base += stride) {
    const int64_t n = base + threadIdx.x;
    const bool f = n < n_all && flags[n] != 0;
    if (map && n < n_all) map[n] = f ? 1.0f : 0.0f;
    const unsigned mask = __ballot_sync(0xffffffffu, f);
    if (!mask) continue;
    const int leader = __ffs(mask) - 1;
    unsigned long long b = 0;
    if (lane == leader) b = atomicAdd(count, (unsigned long long)__popc(mask));
    b = __shfl_sync(0xffffffffu, b, leader);
    if (f) list[b + __popc(mask & ((1u << lane) - 1u))] = (int32_t)n;
  }
}

cudaError_t launch_paper_flags(const float4* nodes, const Pot64* pot64, int n_pot,
                               const lt_grid& g, double2* out, unsigned char* flags,
                               int32_t* list, unsigned long long* count, float* map,
                               int sm_count, cudaStream_t st) {
  const int64_t n_all = (int64_t)g.nx * g.ny;
  int64_t blocks = (n_all + 255) / 256;
  if (blocks > (int64_t)sm_count * 32) blocks = (int64_t)sm_count * 32;
  k_paper_init<<<(unsigned)blocks, 256, 0, st>>>(nodes, g.nx, g.ny, (float)g.dx, (float)g.dy,
                                                 out, flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_paper_patches<<<n_pot, 256, 0, st>>>(pot64, n_pot, g.x0, g.y0, g.dx, g.dy, g.nx, g.ny,
                                         flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  k_paper_compact<<<(unsigned)blocks, 256, 0, st>>>(flags, n_all, list, count, map);
  return cudaGetLastError();
}

}  // namespace lt
