// Arithmetic shared by the step kernels of kernels.cu and stream.cu
// (internal): value types, the FP32-to-FP64 widening of option values32, and
// the reflected Halpern combination.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace pdhg {

template <class T>
struct Pair;
template <>
struct Pair<double> {
  using type = double2;
};
template <>
struct Pair<float> {
  using type = float2;
};

// A value of type V as the arithmetic type T. FP32 to FP64 moves the bit
// fields with integer operations (the sign, the exponent rebiased by
// 1023 - 127 = 896, the 23 mantissa bits at the top of the 52), exact for
// zeros and normal numbers, the only FP32 values option values32 admits: a
// conversion instruction would run on the FP64 pipe, which the FP64 steps'
// multiply-adds already keep busy.
template <class T, class V>
struct AsAcc {
  static __device__ __forceinline__ T get(V v) { return v; }
};
template <>
struct AsAcc<double, float> {
  static __device__ __forceinline__ double get(float v) {
    const unsigned f = __float_as_uint(v);
    const unsigned mag = f & 0x7fffffffu;
    const unsigned hi = (f & 0x80000000u) | (mag ? (mag >> 3) + 0x38000000u : 0u);
    return __hiloint2double((int)hi, (int)(f << 29));
  }
};
template <class T, class V>
__device__ __forceinline__ T as_acc(V v) {
  return AsAcc<T, V>::get(v);
}

// weight w = (t + 1) / (t + 2) of the reflected Halpern step that runs as step
// `it` after st->t was last updated (t = iterations since the last restart)
__device__ __forceinline__ double halpern_weight(const DevState* st, int it) {
  const double t = (double)(st->t + it);
  return (t + 1.0) / (t + 2.0);
}

// The Halpern combination w ((1 + rho) t - rho z) + (1 - w) r, written as
// w (t + rho (t - z)) + (1 - w) r; for the default rho = 1 (R1, chosen once per
// kernel, so that no entry computes both forms) the reflection t + (t - z) =
// 2t - z is the extrapolated point the step computes anyway, and the update
// costs one multiply and one multiply-add more
template <bool R1, class T>
__device__ __forceinline__ T halpern_mix_r(T t, T z, T refl, T r, T w, T omw, T rho) {
  const T u = R1 ? refl : t + rho * (t - z);
  return w * u + omw * r;
}

}  // namespace pdhg
