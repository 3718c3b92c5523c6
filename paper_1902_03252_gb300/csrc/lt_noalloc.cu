// lt_deflect_grid_noalloc: the mixed-precision deflection grid of one lens
// model for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a host
// allocator hook or a memory-pool callback, plugins of applications that own
// every allocation on the device, and processes that pre-reserve all device
// memory at start-up.  This entry point serves them: it needs no model and no
// workspace.  Its scratch -- the prepared potential records, the kind
// segments and a status word -- lives in one file-scope device array of fixed
// size (kNoallocBytes, about 0.8 MiB), which every GPU that loads the library
// holds until the process exits.  The caller still passes the parameters and
// the output buffers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "lt_fp32.cuh"
#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int kNoallocMaxPot = 4096;  // largest model this entry point accepts
constexpr size_t kOffPot64 = 0;
constexpr size_t kOffPot32 = kOffPot64 + sizeof(Pot64) * kNoallocMaxPot;
constexpr size_t kOffSeg = kOffPot32 + sizeof(Pot32) * kNoallocMaxPot;
constexpr size_t kOffStatus = kOffSeg + 256;
constexpr size_t kNoallocBytes = kOffStatus + 256;

// The scratch.  In host code this name is only a stand-in for the symbol: the
// device address must be obtained with cudaGetSymbolAddress on each device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Resolve the scratch address and SM count once per device (the device must
// be current).  Neither call allocates.
lt_status device_setup(int dev, unsigned char** base, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return LT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LT_ERR_CUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return LT_ERR_CUDA;
    g_scratch_ptr[dev] = p;
    g_sm_count[dev] = n;
  }
  *base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  *sms = g_sm_count[dev];
  return LT_OK;
}

// the default launch shape of the batched kernel: 256 threads, 4 rows each,
// registers for 3 resident blocks per SM
constexpr int kNT = 256, kNPT = 4, kMinBlocks = 3;

// The batched deflection kernel's per-item body (deflect32_nodes) for one
// sample, writing alpha and the running error bound straight into the
// caller's buffers.
__global__ void __launch_bounds__(kNT, kMinBlocks)
    k_deflect32_noalloc(const Pot32* __restrict__ pot32, const Seg32* __restrict__ seg, int n_pot,
                        SampleGrid g, int64_t n_items, float2* __restrict__ alpha,
                        float* __restrict__ err) {
  __shared__ float4 sp[kChunk32 * 5];
  const Seg32 sg = *seg;
  const int64_t bands = ((int64_t)g.ny + kNPT - 1) / kNPT;
  const float theta1 = g.theta_max;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    // this thread's column i and rows j0 .. j0 + kNPT - 1 (see defl32_items)
    const int64_t p = item * kNT + threadIdx.x;
    const bool live = p < bands * g.nx;
    const int64_t pc = live ? p : 0;
    const int band = (int)(pc / g.nx);
    const int i = (int)(pc - (int64_t)band * g.nx);
    const int j0 = band * kNPT;
    // node coordinates rounded once from FP64 x0 + i dx, the product and the
    // sum rounded separately (the batched path's coordinate table holds the
    // same values): error u|theta| (App. A's stored-value model), not u|x0|
    // as an FP32 x0 + i*dx would give
    const float X = (float)__dadd_rn(g.x0, __dmul_rn((double)i, g.dx));
    float Y[kNPT], AX[kNPT], AY[kNPT], ER[kNPT];
#pragma unroll
    for (int m = 0; m < kNPT; ++m)
      Y[m] = (float)__dadd_rn(g.y0, __dmul_rn((double)min(j0 + m, g.ny - 1), g.dy));
    // the batched kernel's body: the same operations in the same order
    deflect32_nodes<kNT, kNPT, true>(pot32, n_pot, sg, theta1, X, Y, sp, AX, AY, ER,
                                     item == blockIdx.x);
#pragma unroll
    for (int m = 0; m < kNPT; ++m) {
      if (live && j0 + m < g.ny) {
        const int64_t n = (int64_t)(j0 + m) * g.nx + i;
        alpha[n] = make_float2(AX[m], AY[m]);
        if (err) err[n] = node_bound(__fadd_ru(ER[m], sg.q_tot), n_pot);
      }
    }
  }
}

__global__ void k_noalloc_status(const uint32_t* st, int32_t* out) {
  *out = (*st & ST_NONFINITE) ? (int32_t)LT_ERR_NONFINITE : (int32_t)LT_OK;
}

}  // namespace
}  // namespace lt

using namespace lt;

extern "C" lt_status lt_deflect_grid_noalloc(const double* params, int32_t n_pot,
                                             const lt_grid* grid, float* alpha_out,
                                             float* err_out, int32_t* status_out,
                                             uintptr_t stream) {
  if (!params || !grid || !alpha_out) return LT_ERR_INVALID_ARG;
  if (n_pot < 1 || n_pot > kNoallocMaxPot) return LT_ERR_INVALID_ARG;
  const lt_grid& gr = *grid;
  if (gr.nx < 1 || gr.ny < 1 || !std::isfinite(gr.x0) || !std::isfinite(gr.y0) ||
      !std::isfinite(gr.dx) || !std::isfinite(gr.dy) || !(gr.dx > 0) || !(gr.dy > 0))
    return LT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LT_ERR_CUDA;
  unsigned char* base = nullptr;
  int sms = 1;
  lt_status s = device_setup(dev, &base, &sms);
  if (s != LT_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Pot64* p64 = reinterpret_cast<Pot64*>(base + kOffPot64);
  Pot32* p32 = reinterpret_cast<Pot32*>(base + kOffPot32);
  Seg32* seg = reinterpret_cast<Seg32*>(base + kOffSeg);
  uint32_t* status = reinterpret_cast<uint32_t*>(base + kOffStatus);
  // the status word keeps the previous call's value: clear it first
  if (cudaMemsetAsync(status, 0, sizeof(uint32_t), st) != cudaSuccess) return LT_ERR_CUDA;
  if (launch_prep(params, 1, n_pot, p64, p32, seg, status, st) != cudaSuccess) return LT_ERR_CUDA;
  SampleGrid g;
  g.x0 = gr.x0; g.y0 = gr.y0; g.dx = gr.dx; g.dy = gr.dy; g.nx = gr.nx; g.ny = gr.ny;
  g.node_off = 0;
  const double tm = std::fmax(std::fmax(std::fabs(gr.x0), std::fabs(gr.x0 + (gr.nx - 1) * gr.dx)),
                              std::fmax(std::fabs(gr.y0), std::fabs(gr.y0 + (gr.ny - 1) * gr.dy)));
  g.theta_max = (float)(tm * (1.0 + 1e-6));
  g.pad = 0.f;
  g.x0f = (float)gr.x0; g.y0f = (float)gr.y0; g.dxf = (float)gr.dx; g.dyf = (float)gr.dy;
  g.coord_off = 0;  // unused: this kernel forms its coordinates itself
  const int64_t n_items = defl32_items(gr.nx, gr.ny, kNT, kNPT);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deflect32_noalloc, kNT, 0) !=
      cudaSuccess)
    return LT_ERR_CUDA;
  int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (blocks > n_items) blocks = n_items;
  k_deflect32_noalloc<<<(unsigned)blocks, kNT, 0, st>>>(p32, seg, n_pot, g, n_items,
                                                        reinterpret_cast<float2*>(alpha_out),
                                                        err_out);
  if (cudaGetLastError() != cudaSuccess) return LT_ERR_CUDA;
  if (status_out) {
    k_noalloc_status<<<1, 1, 0, st>>>(status, status_out);
    if (cudaGetLastError() != cudaSuccess) return LT_ERR_CUDA;
  }
  return LT_OK;
}
