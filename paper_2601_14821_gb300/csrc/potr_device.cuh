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
constexpr int kRec = 3;           // raster record: 3 x float4 (48 bytes) per (view, splat)
constexpr int kCullMaxTiles = 64;  // rectangles with more tiles keep every tile
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

// ---------------------------------------------------------------------------------------
// packed binary32 pairs: one f32x2 instruction rounds each half as its scalar form would
// ---------------------------------------------------------------------------------------
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2(float lo, float hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2_t f2s(float x) { return f2(x, x); }
__device__ __forceinline__ void f2split(f2_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ float f2lo(f2_t v) {
  float lo, hi;
  f2split(v, lo, hi);
  (void)hi;
  return lo;
}
__device__ __forceinline__ float f2hi(f2_t v) {
  float lo, hi;
  f2split(v, lo, hi);
  (void)lo;
  return hi;
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
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

// Binning tile test: can some pixel centre of tile (tx, ty) reach alpha >= alpha_min?  The
// exponent log2 G = A u^2 + B u v + C v^2 (u = x - mx, v = y - my) is maximised over the
// rectangle of the tile's pixel centres: on each edge it is a concave parabola, largest at
// its vertex clamped to the edge, and the splat centre counts when it lies inside.  The tile
// is kept when o * exp2r(max + margin) >= alpha_min, the margin 1e-5 |terms| + 1e-4 covering
// the binary32 rounding of this maximum and of any pixel's own exponent and the error of
// exp2r, so every pixel that takes the splat lies in a kept tile.  Fixed operation order: the
// exponent at an edge point (u, v) is ((A u + B v) u) + (C v) v, every product and sum rounded
// on its own.

// The per-splat part: the parabola vertices along the two edge directions, u = ku v and
// v = kv u (only meaningful when A < 0 and C < 0; otherwise every tile is kept).
__device__ __forceinline__ float tile_ku(float A, float B) { return __fdiv_rn(-B, __fmul_rn(2.0f, A)); }

// The per-tile part, for a splat with A < 0 and C < 0 and its ku = tile_ku(A, B), kv = tile_ku(C, B).
// pthr is the record's prefilter log2(alpha_min / o) - 0.01 (log2f, error a few units in the
// last place): with y the margin-raised maximum, y < pthr means o 2^y < alpha_min 2^-0.0099
// and y >= pthr + 0.02 means o 2^y >= alpha_min 2^0.0099, so in both cases the decision of
// o * exp2r(y) >= alpha_min is known (exp2r is within 4e-7 of 2^y) without evaluating it;
// only the band between takes exp2r.  The result is the same as evaluating it always.
__device__ __forceinline__ bool tile_hit_concave(float mx, float my, float A, float B, float C, float o, float ku,
                                                 float kv, float pthr, int tx, int ty, int tile_w, int tile_h,
                                                 float alpha_min) {
  const float X0 = __fadd_rn((float)(tx * tile_w), 0.5f), X1 = __fadd_rn(X0, (float)(tile_w - 1));
  const float Y0 = __fadd_rn((float)(ty * tile_h), 0.5f), Y1 = __fadd_rn(Y0, (float)(tile_h - 1));
  // the two edges of each direction as one pair: (ux0, ux1) and (vy0, vy1)
  const f2_t ux = sub2(f2(X0, X1), f2s(mx)), vy = sub2(f2(Y0, Y1), f2s(my));
  float ux0, ux1, vy0, vy1, kuv0, kuv1, kvu0, kvu1;
  f2split(ux, ux0, ux1);
  f2split(vy, vy0, vy1);
  f2split(mul2(f2s(ku), vy), kuv0, kuv1);
  f2split(mul2(f2s(kv), ux), kvu0, kvu1);
  // vertices on the edges v = vy0, vy1 (u clamped to [ux0, ux1]) and on u = ux0, ux1
  const f2_t uh = f2(fminf(fmaxf(kuv0, ux0), ux1), fminf(fmaxf(kuv1, ux0), ux1));
  const f2_t vv = f2(fminf(fmaxf(kvu0, vy0), vy1), fminf(fmaxf(kvu1, vy0), vy1));
  // the edge exponents ((A u + B v) u) + (C v) v, two edges per instruction
  const f2_t A2 = f2s(A), B2 = f2s(B), C2 = f2s(C);
  const f2_t eh = add2(mul2(add2(mul2(A2, uh), mul2(B2, vy)), uh), mul2(mul2(C2, vy), vy));
  const f2_t ev = add2(mul2(add2(mul2(A2, ux), mul2(B2, vv)), ux), mul2(mul2(C2, vv), vv));
  float p0, p1, p2, p3;
  f2split(eh, p0, p1);
  f2split(ev, p2, p3);
  float pmax = fmaxf(fmaxf(p0, p1), fmaxf(p2, p3));
  if (ux0 <= 0.0f && ux1 >= 0.0f && vy0 <= 0.0f && vy1 >= 0.0f) pmax = fmaxf(pmax, 0.0f);
  const float um = fmaxf(fabsf(ux0), fabsf(ux1)), vm = fmaxf(fabsf(vy0), fabsf(vy1));
  const float mag = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(fabsf(A), um), um), __fmul_rn(__fmul_rn(fabsf(B), um), vm)),
                              __fmul_rn(__fmul_rn(fabsf(C), vm), vm));
  const float margin = __fadd_rn(__fmul_rn(1e-5f, mag), 1e-4f);
  const float y = __fadd_rn(pmax, margin);
  if (y < pthr) return false;
  if (y >= pthr + 0.02f) return true;
  return __fmul_rn(o, exp2r(y)) >= alpha_min;
}

// q = li / w for li < 2^12 and 1 <= w < 2^12: (li + 1/2) / w lies at least 1/(2w) away from
// an integer, far more than the few units in the last place of the approximate division, so
// truncating it gives the exact quotient.
__device__ __forceinline__ uint32_t small_div(uint32_t li, uint32_t w) {
  return (uint32_t)__fdividef((float)li + 0.5f, (float)w);
}

// Position of the r-th set bit (r counted from 0) of a 64-bit word that has more than r.
__device__ __forceinline__ uint32_t select_bit64(uint64_t m, uint32_t r) {
  uint32_t pos = 0;
  uint32_t w = (uint32_t)m;
  uint32_t c = (uint32_t)__popc(w);
  if (r >= c) {
    r -= c;
    w = (uint32_t)(m >> 32);
    pos = 32;
  }
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    c = (uint32_t)__popc(w & ((1u << half) - 1u));
    if (r >= c) {
      r -= c;
      w >>= half;
      pos += half;
    }
  }
  return pos;
}

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

// Lanes whose values d agree in their low NBITS bits (every lane of the warp takes part): one
// ballot per bit, the lane keeping the lanes that agree with it on that bit.
template <int NBITS>
__device__ __forceinline__ uint32_t match_low_bits(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < NBITS; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
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

// Measurement hook (potr_time_next_tile_kernel): the events armed by this host thread, recorded
// on the launching stream around the next tile-pass kernel and then disarmed.
void tile_timing_begin(cudaStream_t s);
void tile_timing_end(cudaStream_t s);

}  // namespace potr

#define POTR_CHECK_LAUNCH()                                   \
  do {                                                        \
    potr::note_launches(1);                                   \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) return POTR_ERR_CUDA;              \
  } while (0)
