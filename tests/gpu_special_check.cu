// Exhaustive checks of the FP32 special functions of the deflection kernel on
// the GPU (test helper, built by tests/test_gpu_special.py with nvcc).
//
// For every float x in [lo, hi] (by bit pattern), one function of the
// library's FP32 path is evaluated exactly as the kernels evaluate it and
// compared with a double-precision reference; the largest relative error
// |f32(x) - f(x)| / |f(x)| is returned.  The functions: the hardware
// approximations rsqrt, sqrt, rcp and lg2 (flush-to-zero forms), and the
// library's atan(t)/t and atanh(t)/t of u = t^2 (polynomials plus range
// reduction).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../paper_1902_03252_gb300/csrc/lt_internal.cuh"

using namespace lt;

namespace {

__device__ double reference(int which, double x) {
  switch (which) {
    case 0: return 1.0 / sqrt(x);
    case 1: return sqrt(x);
    case 2: return 1.0 / x;
    case 3: return log2(x);
    case 4: {
      if (x == 0.0) return 1.0;
      const double t = sqrt(x);
      return atan(t) / t;
    }
    default: {
      if (x == 0.0) return 1.0;
      const double t = sqrt(x);
      return atanh(t) / t;
    }
  }
}

__device__ double weight(int which, float x) { return which == 6 ? 1.0 - (double)x : 1.0; }

__device__ float approx(int which, float x) {
  switch (which) {
    case 0: return rsqrt_approx32(x);
    case 1: return sqrt_approx32(x);
    case 2: return rcp_approx32(x);
    case 3: return lg2_approx32(x);
    case 4: return atanc_sq32(x);
    default: return atanhc_sq32(x);  // 5 and 6
  }
}

// Largest relative error over the bit patterns [b0, b1]; errors are
// non-negative doubles, whose bit patterns order like their values.
__global__ void k_max_err(int which, uint32_t b0, uint32_t b1, unsigned long long* out) {
  double best = 0.0;
  const uint64_t n = (uint64_t)b1 - b0 + 1;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((uint32_t)(b0 + k));
    const double r = reference(which, (double)x);
    const double e = fabs((double)approx(which, x) - r) / fabs(r) * weight(which, x);
    best = e > best ? e : best;  // a NaN error (never expected) is caught below
    if (e != e) best = 1e300;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double v = __shfl_xor_sync(0xffffffffu, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0)
    atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

// The first x (by bit pattern, among those found) whose error equals `err`.
__global__ void k_where(int which, uint32_t b0, uint32_t b1, double err, unsigned int* out) {
  const uint64_t n = (uint64_t)b1 - b0 + 1;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((uint32_t)(b0 + k));
    const double r = reference(which, (double)x);
    const double e = fabs((double)approx(which, x) - r) / fabs(r) * weight(which, x);
    if (e == err) atomicMin(out, (unsigned int)(b0 + k));
  }
}

}  // namespace

// Returns 0 on success, else a CUDA error code; *max_err receives the largest
// relative error, *worst the smallest argument found reaching it.
extern "C" int special_max_err(int which, float lo, float hi, double* max_err, float* worst) {
  if (!(lo <= hi) || !(lo >= 0.0f) || which < 0 || which > 6) return -1;
  uint32_t b0, b1;
  memcpy(&b0, &lo, 4);
  memcpy(&b1, &hi, 4);
  unsigned long long* d_err = nullptr;
  unsigned int* d_where = nullptr;
  cudaError_t e = cudaMalloc(&d_err, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&d_where, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d_where, 0xff, sizeof(unsigned int));
  int sms = 1;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const unsigned blocks = (unsigned)sms * 8;
  unsigned long long bits = 0;
  unsigned int wb = 0xffffffffu;
  if (e == cudaSuccess) {
    k_max_err<<<blocks, 256>>>(which, b0, b1, d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&bits, d_err, sizeof bits, cudaMemcpyDeviceToHost);
  double err = 0.0;
  memcpy(&err, &bits, sizeof err);
  if (e == cudaSuccess) {
    k_where<<<blocks, 256>>>(which, b0, b1, err, d_where);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&wb, d_where, sizeof wb, cudaMemcpyDeviceToHost);
  if (d_err) cudaFree(d_err);
  if (d_where) cudaFree(d_where);
  if (e != cudaSuccess) return (int)e;
  *max_err = err;
  memcpy(worst, &wb, sizeof wb);
  return 0;
}
