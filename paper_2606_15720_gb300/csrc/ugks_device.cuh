// Device helpers shared by the two velocity-block sweeps (ugks_sweep.cu and
// ugks_blocked.cu): fast exponential / division in the sweep precision, the
// Maxwellian prefactor, and warp reductions over the 32 velocity lanes.
#pragma once
#include <cmath>
#include <cstdint>

#include "ugks_internal.cuh"

namespace ugks {
namespace {

template <typename T>
__device__ __forceinline__ T t_exp(T x);
template <>
__device__ __forceinline__ float t_exp<float>(float x) {
  return __expf(x);
}
template <>
__device__ __forceinline__ double t_exp<double>(double x) {
  return exp(x);
}

// (lambda/pi)^(D/2)
template <int D, typename T>
__device__ __forceinline__ T maxwell_pref(T lam) {
  T s = lam * T(0.31830988618379067154);
  if (D == 1) return sqrt(s);
  if (D == 2) return s;
  return s * sqrt(s);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ size_t frow(int r, int64_t m, int64_t c, int64_t M, int64_t Nc) {
  return ((size_t(r) * size_t(M) + size_t(m)) * size_t(Nc) + size_t(c)) * BV;
}

// Selects component t (0..4) of five warp-uniform values without local memory.
template <typename T>
__device__ __forceinline__ T pick5(int t, T a0, T a1, T a2, T a3, T a4) {
  return t == 0 ? a0 : t == 1 ? a1 : t == 2 ? a2 : t == 3 ? a3 : a4;
}

// Sums eight per-lane values over the warp with a transposed butterfly (9
// shuffles instead of 5 per value): afterwards lane L holds the total of value
// number ((L >> 4) & 1) * 4 + ((L >> 3) & 1) * 2 + ((L >> 2) & 1).
template <typename T>
__device__ __forceinline__ T warp_sum8(T v0, T v1, T v2, T v3, T v4, T v5, T v6, T v7, int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  T a0 = (b4 ? v4 : v0) + __shfl_xor_sync(0xffffffffu, b4 ? v0 : v4, 16);
  T a1 = (b4 ? v5 : v1) + __shfl_xor_sync(0xffffffffu, b4 ? v1 : v5, 16);
  T a2 = (b4 ? v6 : v2) + __shfl_xor_sync(0xffffffffu, b4 ? v2 : v6, 16);
  T a3 = (b4 ? v7 : v3) + __shfl_xor_sync(0xffffffffu, b4 ? v3 : v7, 16);
  T c0 = (b3 ? a2 : a0) + __shfl_xor_sync(0xffffffffu, b3 ? a0 : a2, 8);
  T c1 = (b3 ? a3 : a1) + __shfl_xor_sync(0xffffffffu, b3 ? a1 : a3, 8);
  T d0 = (b2 ? c1 : c0) + __shfl_xor_sync(0xffffffffu, b2 ? c0 : c1, 4);
  d0 += __shfl_xor_sync(0xffffffffu, d0, 2);
  d0 += __shfl_xor_sync(0xffffffffu, d0, 1);
  return d0;
}

template <typename T>
__device__ __forceinline__ T energy_in(int, T wi, T u2, T phi_h, T phi_b) {
  return T(0.5) * wi * (u2 * phi_h + phi_b);
}

__device__ __forceinline__ int sum8_index(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

template <typename T>
__device__ __forceinline__ T fast_div(T a, T b);
template <>
__device__ __forceinline__ float fast_div<float>(float a, float b) {
  return __fdividef(a, b);
}
template <>
__device__ __forceinline__ double fast_div<double>(double a, double b) {
  return a / b;
}

// Unevaluated float pairs hi + lo (Knuth's two-sum, then a fast
// renormalisation): sums of many FP32 terms to ~2^-44 relative without FP64
// instructions, which GB300 executes at a small fraction of its FP32 rate.
// (hi, lo) + v:
__device__ __forceinline__ float2 pair_add(float2 p, float v) {
  const float s = p.x + v;
  const float bp = s - p.x;
  const float e = (p.x - (s - bp)) + (v - bp);
  const float lo = p.y + e;
  const float hi = s + lo;
  return make_float2(hi, lo - (hi - s));
}
// (hi, lo) + (hi, lo):
__device__ __forceinline__ float2 pair_add(float2 p, float2 q) {
  const float s = p.x + q.x;
  const float bp = s - p.x;
  const float e = (p.x - (s - bp)) + (q.x - bp) + (p.y + q.y);
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

}  // namespace
}  // namespace ugks
