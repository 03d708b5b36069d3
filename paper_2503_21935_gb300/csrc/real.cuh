// Real types of the amplitude arithmetic: double (the float64 path) and float (single
// precision, the paper's float build), behind one set of helpers so that the amplitude code
// is written once.
#pragma once
#include <cstdint>

namespace mgx {

// ---- uniform helpers over double / float
template <class R> struct Real;

template <> struct Real<double> {
  __device__ __forceinline__ static double from(double x) { return x; }
  __device__ __forceinline__ static double to_double(double x) { return x; }
  __device__ __forceinline__ static double rcp(double x) { return 1.0 / x; }
  __device__ __forceinline__ static double sqrt_(double x) { return ::sqrt(x); }
  __device__ __forceinline__ static double max0(double x) { return x > 0.0 ? x : 0.0; }
  __device__ __forceinline__ static bool positive(double x) { return x > 0.0; }
  // exact +0.0 / 1.0 and sign flips as bit operations on the integer pipe (the float64 pipe is
  // the bottleneck of the amplitude code)
  __device__ __forceinline__ static bool is_zero(double x) { return __double_as_longlong(x) == 0ll; }
  __device__ __forceinline__ static bool is_one(double x) { return __double_as_longlong(x) == 0x3FF0000000000000ll; }
  __device__ __forceinline__ static double neg(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
  }
};

template <> struct Real<float> {
  __device__ __forceinline__ static float from(double x) { return (float)x; }
  __device__ __forceinline__ static double to_double(float x) { return (double)x; }
  __device__ __forceinline__ static float rcp(float x) { return 1.0f / x; }
  __device__ __forceinline__ static float sqrt_(float x) { return sqrtf(x); }
  __device__ __forceinline__ static float max0(float x) { return x > 0.0f ? x : 0.0f; }
  __device__ __forceinline__ static bool positive(float x) { return x > 0.0f; }
  __device__ __forceinline__ static bool is_zero(float x) { return __float_as_int(x) == 0; }
  __device__ __forceinline__ static bool is_one(float x) { return __float_as_int(x) == 0x3F800000; }
  __device__ __forceinline__ static float neg(float x) { return __int_as_float(__float_as_int(x) ^ (int)0x80000000u); }
};

}  // namespace mgx
