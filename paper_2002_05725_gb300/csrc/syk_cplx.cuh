// Complex helpers on CUDA vector types (float2 / double2 hold (re, im)).
#pragma once
#include <cuda_runtime.h>

namespace syk {

template <typename R>
struct CT;
template <>
struct CT<float> {
  using T = float2;
};
template <>
struct CT<double> {
  using T = double2;
};

template <typename R>
__host__ __device__ inline typename CT<R>::T make_c(R re, R im) {
  typename CT<R>::T v;
  v.x = re;
  v.y = im;
  return v;
}

// acc += (cr + i ci) * v
template <typename C, typename R>
__device__ __forceinline__ void cmac(C& acc, R cr, R ci, const C v) {
  acc.x = fma(cr, v.x, fma(-ci, v.y, acc.x));
  acc.y = fma(cr, v.y, fma(ci, v.x, acc.y));
}

}  // namespace syk
