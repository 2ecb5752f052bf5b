// Storage of the distribution: plain FP64 / FP32 values, or FP16 / BF16
// deviations from a per-cell reference Maxwellian, scaled per row.
//
// Scaled form: a row of 32 velocities of one (reduced distribution, velocity
// block, cell) holds delta_k = (f_k - g_ref,k) / s in the storage type, with
// s = max_k |f_k - g_ref,k| over the row (FP32, stored beside the row) and
// g_ref the cell's reference Maxwellian (RefMaxwell, FP32).  Decoding is
// f = g_ref + s delta: the rounding error of each value is about 2^-11
// (FP16) or 2^-8 (BF16) of its own deviation |f - g_ref|, so regions near
// equilibrium are stored almost exactly.  Padded velocities keep f = 0.
#pragma once
#include <cmath>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ugks_internal.cuh"

namespace ugks {

template <typename S>
struct StoreTraits {
  static constexpr bool scaled = false;
};
template <>
struct StoreTraits<__half> {
  static constexpr bool scaled = true;
  static __device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
  static __device__ __forceinline__ __half from_f(float v) { return __float2half_rn(v); }
};
template <>
struct StoreTraits<__nv_bfloat16> {
  static constexpr bool scaled = true;
  static __device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
};

// Reference value g_ref of reduced distribution r at velocity u (0 on padding).
template <int D>
__device__ __forceinline__ float ref_value(const RefMaxwell& R, int r, const float (&u)[3], bool real) {
  float c2 = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) c2 += (u[d] - R.U[d]) * (u[d] - R.U[d]);
  const float g = real ? R.pref * __expf(-R.lam * c2) : 0.f;
  return r == 0 ? g : R.kap * g;
}

__device__ __forceinline__ float warp_max_abs(float v) {
  v = fabsf(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Encodes one row (all 32 lanes call it with their value f and reference g):
// returns the stored deviation and sets scale (the same on every lane).
// Rows whose largest deviation is below kScaleFloor are stored as exactly
// their reference (scale 0): the floor keeps 1/scale finite (an FP32
// subnormal scale would overflow it), and deviations that small are far below
// any value of f that matters.  A NaN deviation still propagates.
constexpr float kScaleFloor = 1e-30f;

template <typename S>
__device__ __forceinline__ S encode_value(float f, float g, float& scale) {
  const float dev = f - g;
  scale = warp_max_abs(dev);
  if (scale < kScaleFloor) scale = 0.f;
  const float inv = scale > 0.f ? 1.f / scale : 0.f;
  return StoreTraits<S>::from_f(dev * inv);
}

template <typename S>
__device__ __forceinline__ float decode_value(S d, float scale, float g) {
  return fmaf(scale, StoreTraits<S>::to_f(d), g);
}

// Reference Maxwellian of a cell from its FP64 primitive record.
template <int D>
__device__ __forceinline__ RefMaxwell make_ref(const CellPrim& p, int Kxi) {
  RefMaxwell R;
  R.pref = float(p.rho * pow(p.lam / M_PI, 0.5 * D));
  R.lam = float(p.lam);
#pragma unroll
  for (int d = 0; d < 3; ++d) R.U[d] = float(p.U[d]);
  R.kap = float(Kxi / (2.0 * p.lam));
  R.pad[0] = R.pad[1] = 0.f;
  return R;
}

}  // namespace ugks
