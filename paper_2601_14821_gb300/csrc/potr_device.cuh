// potr_device.cuh -- device helpers shared by the sm_103a kernels of libpotr.
//
// Binary32 arithmetic on every path that decides an integer (tile rectangle, depth key,
// the per-pixel alpha test and the transmittance stop) is written with the _rn intrinsics
// so that nvcc cannot contract or reorder it: the same inputs give the same bits in every
// kernel that re-evaluates them (forward pass, removal pass, backward pass).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/potr.h"

namespace potr {

constexpr int kTilePixels = 256;  // tile_w * tile_h
constexpr int kRecFloats = 12;    // raster record: 3 x float4
constexpr float kLog2e = 1.44269504088896340736f;

// ---------------------------------------------------------------------------------------
// Reproducible exp2: Cody & Waite reduction y = n + f with n = nearest integer (ties to
// even) and |f| <= 1/2, then the Taylor series of 2^f = e^{f ln 2} to degree 6 by Horner's
// rule, then an exact scaling by 2^n through the exponent field.  Coefficients are
// (ln 2)^k / k!, evaluated in binary64 by the recurrence c_k = (c_{k-1} * ln 2) / k and
// rounded to binary32.  Inputs are clamped to [-125, 125] (NaN goes to -125), so every
// result is a normal number and the exponent-field scaling is exact.
// ---------------------------------------------------------------------------------------
constexpr double kLn2d = 0.6931471805599453;
__host__ __device__ constexpr float exp2_coef(int k) {
  double c = 1.0;
  for (int i = 1; i <= k; ++i) {
    c = c * kLn2d;
    c = c / (double)i;
  }
  return (float)c;
}

__device__ __forceinline__ float exp2r(float y) {
  constexpr float c0 = exp2_coef(0), c1 = exp2_coef(1), c2 = exp2_coef(2), c3 = exp2_coef(3);
  constexpr float c4 = exp2_coef(4), c5 = exp2_coef(5), c6 = exp2_coef(6);
  y = (y >= -125.0f) ? y : -125.0f;
  y = (y > 125.0f) ? 125.0f : y;
  // y + 1.5 * 2^23 rounds y to the nearest integer (ties to even: 1.5 * 2^23 is even);
  // the low mantissa bits of t then hold that integer in two's complement.
  const float t = __fadd_rn(y, 12582912.0f);
  const float n = __fsub_rn(t, 12582912.0f);
  const float f = __fsub_rn(y, n);
  float p = __fmaf_rn(c6, f, c5);
  p = __fmaf_rn(p, f, c4);
  p = __fmaf_rn(p, f, c3);
  p = __fmaf_rn(p, f, c2);
  p = __fmaf_rn(p, f, c1);
  p = __fmaf_rn(p, f, c0);
  // (bits(t) << 23) == n << 23 modulo 2^32 because the low 9 bits of bits(1.5 * 2^23) are 0.
  return __int_as_float(__float_as_int(p) + (__float_as_int(t) << 23));
}

// Per-pair opacity exponent: log2 G = A dx^2 + B dx dy + C dy^2, evaluated as
// fma(fma(A, dx, B dy), dx, (C dy) dy).
__device__ __forceinline__ float pair_exponent(float A, float B, float C, float dx, float dy) {
  const float u = __fmaf_rn(A, dx, __fmul_rn(B, dy));
  const float v = __fmul_rn(C, dy);
  return __fmaf_rn(u, dx, __fmul_rn(v, dy));
}

// alpha = min(alpha_max, o * exp2r(p)); the caller compares it with alpha_min.
__device__ __forceinline__ float pair_alpha(float o, float p, float alpha_max) {
  return fminf(alpha_max, __fmul_rn(o, exp2r(p)));
}

// Transmittance after compositing a splat of opacity a: T (1 - a) as fma(-a, T, T).
__device__ __forceinline__ float trans_next(float a, float T) { return __fmaf_rn(-a, T, T); }

// Rectangle packing of the raster record word 11: x0 (11 bits) | y0 (11 bits) | w (10 bits).
__device__ __forceinline__ uint32_t pack_rect_word(uint32_t x0, uint32_t y0, uint32_t w) {
  return x0 | (y0 << 11) | (w << 22);
}

// Index of the view owning global tile t (binary search over tile bases; n_views >= 1).
__device__ __forceinline__ int view_of_tile(const potr_view_info* info, int n_views, int64_t t) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (info[mid].tile_base <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void set_status(potr_device_status* st, int32_t code, int64_t required) {
  if (st) {
    atomicCAS(&st->code, 0, code);
    if (required > 0) atomicMax(reinterpret_cast<unsigned long long*>(&st->required_instances),
                                (unsigned long long)required);
  }
}

// Host-side count of kernel launches issued by the library (potr_launch_count).
void note_launches(int n);

}  // namespace potr

#define POTR_CHECK_LAUNCH()                                   \
  do {                                                        \
    potr::note_launches(1);                                   \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) return POTR_ERR_CUDA;              \
  } while (0)
