// Input domain of a source (Eq. 13): a finite position and a ratio
// 0 <= D_ls/D_s < 1e30.  The tests are exact integer forms of isfinite(x)
// and of the FP64 comparison 0 <= r < 1e30 on the bits of the doubles (-0 is
// accepted, NaN and infinities are not): an FP64 compare holds a GB300
// sub-partition's FP64 unit for ~80 cycles.
#pragma once

namespace lt {

__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) !=
         0x7ff0000000000000ull;
}
__device__ __forceinline__ bool ratio_ok_bits(double r) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(r);
  return b == 0x8000000000000000ull || b < (unsigned long long)__double_as_longlong(1e30);
}
__device__ __forceinline__ bool source_ok(double px, double py, double r) {
  return finite_bits(px) && finite_bits(py) && ratio_ok_bits(r);
}

}  // namespace lt
