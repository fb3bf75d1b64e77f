// tile_pass.cuh -- building blocks of the tile kernels that give each lane two pixels.
//
// A tile (256 pixels) is one CTA of four warps; warp w covers an 8 x 8 block of the tile and
// lane l the two vertically adjacent pixels (l mod 8, 2 (l div 8)) and (l mod 8, 2 (l div 8) + 1)
// of it.  The per-pixel binary32 arithmetic of the two pixels runs as packed pairs (the f32x2
// add / sub / mul / fma of the sm_100 family: one instruction, two IEEE round-to-nearest
// results, bit-identical to the scalar operations), so a splat record read once from shared
// memory, one loop step and one warp vote serve two pixels, and the two pixels' exponent,
// exp2 and compositing updates issue as one instruction each.
//
// Which splats a warp visits: per group of 32 list positions, lane j tests position j against
// the warp's 8 x 8 block (the exponent's maximum over the block's pixel-centre rectangle, on
// its edges or at the splat centre, raised by a rounding margin, against the record's
// prefilter); a position whose bit is clear has alpha < alpha_min at all 64 pixels, so
// skipping it changes no decision.
#pragma once

#include "raster_common.cuh"

namespace potr {
namespace {

constexpr int kT2 = 128;           // threads per CTA: four warps, two pixels per lane
constexpr int kW2 = kT2 / 32;      // warps per CTA
constexpr int kSRec2 = 3;          // float4 per staged record

// exp2r (potr_device.cuh) on a pair: the same clamps, operations and order, so the same bits.
__device__ __forceinline__ f2_t exp2r2(f2_t yy) {
  constexpr float c0 = exp2_coef(0), c1 = exp2_coef(1), c2 = exp2_coef(2), c3 = exp2_coef(3);
  constexpr float c4 = exp2_coef(4), c5 = exp2_coef(5), c6 = exp2_coef(6);
  float y0, y1;
  f2split(yy, y0, y1);
  y0 = (y0 >= -125.0f) ? y0 : -125.0f;
  y0 = (y0 > 125.0f) ? 125.0f : y0;
  y1 = (y1 >= -125.0f) ? y1 : -125.0f;
  y1 = (y1 > 125.0f) ? 125.0f : y1;
  const f2_t y = f2(y0, y1);
  const f2_t magic = f2s(12582912.0f);
  const f2_t t = add2(y, magic);
  const f2_t n = sub2(t, magic);
  const f2_t f = sub2(y, n);
  f2_t p = fma2(f2s(c6), f, f2s(c5));
  p = fma2(p, f, f2s(c4));
  p = fma2(p, f, f2s(c3));
  p = fma2(p, f, f2s(c2));
  p = fma2(p, f, f2s(c1));
  p = fma2(p, f, f2s(c0));
  float p0, p1, t0, t1;
  f2split(p, p0, p1);
  f2split(t, t0, t1);
  return f2(__int_as_float(__float_as_int(p0) + (__float_as_int(t0) << 23)),
            __int_as_float(__float_as_int(p1) + (__float_as_int(t1) << 23)));
}

// pair_exponent (potr_device.cuh) for the two pixels of a lane: dx shared, dy per pixel.
//   u = fma(A, dx, B dy), v = C dy, p = fma(u, dx, v dy)
__device__ __forceinline__ f2_t pair_exponent2(float A, float B, float C, f2_t dx2, f2_t dy2) {
  const f2_t u = fma2(f2s(A), dx2, mul2(f2s(B), dy2));
  const f2_t v = mul2(f2s(C), dy2);
  return fma2(u, dx2, mul2(v, dy2));
}

// ---------------------------------------------------------------------------------------
// cp.async staging of list batches (128 threads)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16_2(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
template <int N>
__device__ __forceinline__ void cp_async_wait2() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Double-buffered batch staging: the gathers of one batch are in flight (cp.async, one commit
// group per batch) while the CTA works on the other buffer; every thread holds the list values
// (vk) of the batch after that in registers, so issuing never waits on a load.
template <int BATCH>
struct Stager2 {
  static constexpr int kPer = (BATCH + kT2 - 1) / kT2;
  uint32_t vk[kPer];
  int loaded;
  __device__ __forceinline__ void load(const uint32_t* __restrict__ vals, uint32_t first, int cnt) {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int j = threadIdx.x + r * kT2;
      vk[r] = j < cnt ? vals[first + j] : 0u;
    }
    loaded = cnt;
  }
  __device__ __forceinline__ void issue(float4* buf, const float4* __restrict__ raster) const {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int j = threadIdx.x + r * kT2;
      if (j < loaded) {
        const float4* src = raster + (size_t)vk[r] * kRec;
        cp_async16_2(buf + kSRec2 * j + 0, src + 0);
        cp_async16_2(buf + kSRec2 * j + 1, src + 1);
        cp_async16_2(buf + kSRec2 * j + 2, src + 2);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  }
};

// ---------------------------------------------------------------------------------------
// per-tile context
// ---------------------------------------------------------------------------------------
struct Tile2 {
  int64_t tile;
  int view;
  potr_view_info vi;
  int tx, ty;
  int px, py;          // the lane's first pixel; the second is (px, py + 1)
  bool in0, in1;       // inside the image
  float fx, fy0, fy1;  // pixel centres
  float bx0, by0;      // the warp block's first pixel centre (its rectangle: + [0, 7] in x and y)
  uint32_t s, e;       // the tile's list
};

__device__ __forceinline__ Tile2 tile2_ctx(const potr_view_info* __restrict__ info, int n_views,
                                           const uint32_t* __restrict__ ranges, const potr_raster_config& cfg,
                                           int64_t tile) {
  Tile2 c;
  c.tile = tile;
  c.view = view_of_tile(info, n_views, tile);
  c.vi = info[c.view];
  const int64_t local = tile - c.vi.tile_base;
  c.ty = (int)(local / c.vi.tiles_x);
  c.tx = (int)(local - (int64_t)c.ty * c.vi.tiles_x);
  const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5), bx_n = cfg.tile_w / 8;
  const int bx = c.tx * cfg.tile_w + (warp % bx_n) * 8, by = c.ty * cfg.tile_h + (warp / bx_n) * 8;
  c.px = bx + (lane & 7);
  c.py = by + 2 * (lane >> 3);
  c.in0 = c.px < c.vi.width && c.py < c.vi.height;
  c.in1 = c.px < c.vi.width && c.py + 1 < c.vi.height;
  c.fx = (float)c.px + 0.5f;
  c.fy0 = (float)c.py + 0.5f;
  c.fy1 = (float)(c.py + 1) + 0.5f;
  c.bx0 = (float)bx + 0.5f;
  c.by0 = (float)by + 0.5f;
  c.s = ranges[2 * tile];
  c.e = ranges[2 * tile + 1];
  return c;
}

// May the splat of record (r0, r1) pass the prefilter (log2 G >= r1.z) at some pixel centre of
// the warp's 8 x 8 block?  The exponent A u^2 + B u v + C v^2 (u = x - mx, v = y - my) is
// maximised over the block's pixel-centre rectangle: on each edge a concave parabola, largest
// at its vertex clamped to the edge, and 0 at the splat centre when it lies inside.  The
// maximum is raised by 1e-4 x the largest term magnitude + 1e-3, which covers the binary32
// rounding of this maximum and of any pixel's own exponent many times over, so a false answer
// means alpha < alpha_min at all 64 pixels.
__device__ __forceinline__ bool block_may_pass(const float4& r0, const float4& r1, float bx0, float by0) {
  const float A = r0.z, B = r0.w, C = r1.x, thr = r1.z;
  if (!(thr < INFINITY)) return false;                              // o = 0: never passes
  if (!(thr > -INFINITY) || !(A < 0.0f) || !(C < 0.0f)) return true;  // no bound: keep
  const float ux0 = bx0 - r0.x, ux1 = ux0 + 7.0f, vy0 = by0 - r0.y, vy1 = vy0 + 7.0f;
  const float ku = -B / (2.0f * A), kv = -B / (2.0f * C);
  const float u0 = fminf(fmaxf(ku * vy0, ux0), ux1), u1 = fminf(fmaxf(ku * vy1, ux0), ux1);
  const float v0 = fminf(fmaxf(kv * ux0, vy0), vy1), v1 = fminf(fmaxf(kv * ux1, vy0), vy1);
  float pmax = fmaxf(fmaxf((A * u0 + B * vy0) * u0 + C * vy0 * vy0, (A * u1 + B * vy1) * u1 + C * vy1 * vy1),
                     fmaxf((A * ux0 + B * v0) * ux0 + C * v0 * v0, (A * ux1 + B * v1) * ux1 + C * v1 * v1));
  if (ux0 <= 0.0f && ux1 >= 0.0f && vy0 <= 0.0f && vy1 >= 0.0f) pmax = fmaxf(pmax, 0.0f);
  const float um = fmaxf(fabsf(ux0), fabsf(ux1)), vm = fmaxf(fabsf(vy0), fabsf(vy1));
  const float mag = fabsf(A) * um * um + fabsf(B) * um * vm + fabsf(C) * vm * vm;
  return pmax + (1e-4f * mag + 1e-3f) >= thr;
}

// exp2r (potr_device.cuh) on a pair whose arguments are known to lie in [-125, 125], where its
// clamps do nothing: the same operations in the same order, so the same bits.  The tile walks
// take it for a record whose exponent is negative definite (record word 7 = 0): a pixel past the
// prefilter then has log2(alpha_min / o) - 0.01 <= y (> -9, o <= 1) and y at most a few
// rounding errors above 0, over any tile of its rectangle.  (The half of a pair that did not pass
// may hold any value; its result is not used.)
__device__ __forceinline__ f2_t exp2r2_nc(f2_t y) {
  constexpr float c0 = exp2_coef(0), c1 = exp2_coef(1), c2 = exp2_coef(2), c3 = exp2_coef(3);
  constexpr float c4 = exp2_coef(4), c5 = exp2_coef(5), c6 = exp2_coef(6);
  const f2_t magic = f2s(12582912.0f);
  const f2_t t = add2(y, magic);
  const f2_t n = sub2(t, magic);
  const f2_t f = sub2(y, n);
  f2_t p = fma2(f2s(c6), f, f2s(c5));
  p = fma2(p, f, f2s(c4));
  p = fma2(p, f, f2s(c3));
  p = fma2(p, f, f2s(c2));
  p = fma2(p, f, f2s(c1));
  p = fma2(p, f, f2s(c0));
  float p0, p1, t0, t1;
  f2split(p, p0, p1);
  f2split(t, t0, t1);
  return f2(__int_as_float(__float_as_int(p0) + (__float_as_int(t0) << 23)),
            __int_as_float(__float_as_int(p1) + (__float_as_int(t1) << 23)));
}

// ---------------------------------------------------------------------------------------
// expanded records: once staged, each 48-byte record is rewritten in shared memory as five
// float4 holding every operand the two pixels share as a packed pair, so one 128-bit shared
// load gives two packed operands and no register moves build them:
//   [0] (A, A, B, B)  [1] (C, C, mx, mx)  [2] (my, my, o, o)  [3] (prefilter, indefinite, r, r)
//   [4] (g, g, b, b)
// ---------------------------------------------------------------------------------------
constexpr int kERec = 5;

__device__ __forceinline__ void expand_record(const float4* raw, float4* dst) {
  const float4 r0 = raw[0], r1 = raw[1], r2 = raw[2];
  dst[0] = make_float4(r0.z, r0.z, r0.w, r0.w);
  dst[1] = make_float4(r1.x, r1.x, r0.x, r0.x);
  dst[2] = make_float4(r0.y, r0.y, r1.y, r1.y);
  dst[3] = make_float4(r1.z, r1.w, r2.x, r2.x);
  dst[4] = make_float4(r2.y, r2.y, r2.z, r2.z);
}

// The block test (block_may_pass) on an expanded record.
__device__ __forceinline__ bool block_may_pass_e(const float4* e, float bx0, float by0) {
  const float4 q0 = e[0], q1 = e[1], q2 = e[2], q3 = e[3];
  return block_may_pass(make_float4(q1.z, q2.x, q0.x, q0.z), make_float4(q1.x, q2.z, q3.x, 0.0f), bx0, by0);
}

// exp2r on the pair of an expanded record's exponents: without the clamps for a definite form.
__device__ __forceinline__ f2_t exp2r2_rec(f2_t y, float indefinite) {
  return indefinite == 0.0f ? exp2r2_nc(y) : exp2r2(y);
}

// The two pixels' exponents of an expanded record (pair_exponent on each).
__device__ __forceinline__ f2_t exponent_e(const float4* e, f2_t fx2, f2_t fy2, f2_t& o2, float& thr,
                                           float& indefinite) {
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(e);
  const ulonglong2 q0 = q[0], q1 = q[1], q2 = q[2];
  o2 = q2.y;
  const float2 t = reinterpret_cast<const float2*>(e + 3)[0];
  thr = t.x;
  indefinite = t.y;
  const f2_t dx = sub2(fx2, q1.y), dy = sub2(fy2, q2.x);
  const f2_t u = fma2(q0.x, dx, mul2(q0.y, dy));
  const f2_t v = mul2(q1.x, dy);
  return fma2(u, dx, mul2(v, dy));
}

// One splat of the forward walk at the lane's two pixels (expanded record e, list position pos):
// the decisions in binary32 exactly as the oracle takes them.  Branch-free once some pixel of
// the warp passes the prefilter: a pixel that does not take the splat gets alpha 0 in the
// packed updates (T (1 - 0) = T and c + 0 r = c exactly), so its T and colour do not change.
__device__ __forceinline__ void forward_visit_e(const float4* e, uint32_t pos, f2_t fx2, f2_t fy2,
                                                const potr_raster_config& cfg, f2_t (&C)[3], f2_t& T,
                                                uint32_t& last0, uint32_t& last1, bool& done0, bool& done1) {
  f2_t o2;
  float thr, indef;
  const f2_t p2 = exponent_e(e, fx2, fy2, o2, thr, indef);
  float p0, p1;
  f2split(p2, p0, p1);
  const bool pass0 = !done0 && p0 >= thr, pass1 = !done1 && p1 >= thr;
  if (!__any_sync(0xffffffffu, pass0 || pass1)) return;  // alpha < alpha_min at every pixel of the warp
  float a0, a1;
  f2split(mul2(o2, exp2r2_rec(p2, indef)), a0, a1);
  a0 = fminf(cfg.alpha_max, a0);
  a1 = fminf(cfg.alpha_max, a1);
  const bool ok0 = pass0 && a0 >= cfg.alpha_min, ok1 = pass1 && a1 >= cfg.alpha_min;
  const f2_t zero2 = f2s(0.0f);
  const f2_t aa = f2(ok0 ? a0 : 0.0f, ok1 ? a1 : 0.0f);
  float Tn0, Tn1;
  f2split(fma2(sub2(zero2, aa), T, T), Tn0, Tn1);  // T (1 - alpha) as fma(-alpha, T, T)
  const bool stop0 = ok0 && Tn0 < cfg.t_min, stop1 = ok1 && Tn1 < cfg.t_min;  // not composited: the pixel ends
  const bool take0 = ok0 && !stop0, take1 = ok1 && !stop1;
  done0 = done0 || stop0;
  done1 = done1 || stop1;
  const f2_t ae = f2(take0 ? a0 : 0.0f, take1 ? a1 : 0.0f);
  const f2_t w2 = mul2(ae, T);  // T alpha where taken, 0 elsewhere
  const ulonglong2 q3 = reinterpret_cast<const ulonglong2*>(e)[3], q4 = reinterpret_cast<const ulonglong2*>(e)[4];
  C[0] = fma2(w2, q3.y, C[0]);
  C[1] = fma2(w2, q4.x, C[1]);
  C[2] = fma2(w2, q4.y, C[2]);
  T = fma2(sub2(zero2, ae), T, T);  // T (1 - alpha) where taken, T elsewhere
  last0 = take0 ? pos + 1 : last0;
  last1 = take1 ? pos + 1 : last1;
}

// Forward walk (Section 3, Eqs. 2-4) of the tile list for the lane's two pixels: colour,
// final transmittance and n_last (one past the last composited list position) of each.
// smem holds two batches of records ([2][BATCH][kSRec2]); the gathers of batch k + 1 are in
// flight while the CTA composites batch k.
template <int BATCH>
__device__ __forceinline__ void expand_own(const float4* raw, float4* ex, int cnt) {
#pragma unroll
  for (int r = 0; r < Stager2<BATCH>::kPer; ++r) {
    const int j = threadIdx.x + r * kT2;
    if (j < cnt) expand_record(raw + kSRec2 * j, ex + kERec * j);  // this thread's own copies
  }
}

template <int BATCH>
__device__ __forceinline__ void forward_walk2(float4* smem, float4* ex, const float4* __restrict__ raster,
                                              const uint32_t* __restrict__ vals, const Tile2& c,
                                              const potr_raster_config& cfg, f2_t (&C)[3], f2_t& T,
                                              uint32_t& last0, uint32_t& last1) {
  C[0] = C[1] = C[2] = f2s(0.0f);
  T = f2s(1.0f);
  last0 = last1 = 0;
  bool done0 = !c.in0, done1 = !c.in1;
  const int lane = threadIdx.x & 31;
  const f2_t fx2 = f2s(c.fx), fy2 = f2(c.fy0, c.fy1);
  const uint32_t len = c.e - c.s;
  const uint32_t nb = (len + BATCH - 1) / BATCH;
  Stager2<BATCH> st;
  if (nb > 0) {
    st.load(vals, c.s, (int)min((uint32_t)BATCH, len));
    st.issue(smem, raster);
  }
  if (nb > 1) st.load(vals, c.s + BATCH, (int)min((uint32_t)BATCH, len - BATCH));
  for (uint32_t k = 0; k < nb; ++k) {
    if (__syncthreads_and(done0 && done1)) break;  // also: batch k - 1 (and its buffer) fully consumed
    const uint32_t pos0 = k * BATCH;
    const int cnt = (int)min((uint32_t)BATCH, len - pos0);
    const float4* buf = smem + kSRec2 * BATCH * (k & 1);
    if (k + 1 < nb) {
      st.issue(smem + kSRec2 * BATCH * ((k + 1) & 1), raster);
      cp_async_wait2<1>();
      if (k + 2 < nb) st.load(vals, c.s + pos0 + 2 * BATCH, (int)min((uint32_t)BATCH, len - pos0 - 2 * BATCH));
    } else {
      cp_async_wait2<0>();
    }
    expand_own<BATCH>(buf, ex, cnt);
    __syncthreads();  // every thread's expanded records of batch k are visible
    for (int g = 0; g < cnt; g += 32) {
      if (__all_sync(0xffffffffu, done0 && done1)) break;
      const int jl = g + lane;
      const bool cand = jl < cnt && block_may_pass_e(ex + kERec * jl, c.bx0, c.by0);
      uint32_t m = __ballot_sync(0xffffffffu, cand);
      while (m) {
        const int j = g + __ffs(m) - 1;
        m &= m - 1;
        forward_visit_e(ex + kERec * j, pos0 + (uint32_t)j, fx2, fy2, cfg, C, T, last0, last1, done0, done1);
      }
    }
  }
  cp_async_wait2<0>();  // after an early exit the next batch may still be landing
}

// ---------------------------------------------------------------------------------------
// warp-independent walks: each warp takes (tile, 8 x 8 block) items of its own and stages the
// tile's records itself, 32 list positions at a time, in a two-slot ring of its own; no
// barrier couples the warps of a CTA.
// ---------------------------------------------------------------------------------------
constexpr int kWRing = 2;                                 // staged groups per warp
constexpr int kWSlot = 32 * kSRec2;                       // float4 per staged group
constexpr int kWarpSmemF4 = kWRing * kWSlot + 32 * kERec;  // float4 of shared memory per warp

// The next (tile, block) item of this warp: items i = 4 t' + b over the tile order (longest
// lists first; t' = t without an order), taken from the order's counter, or strided over the
// grid's warps without one.  Returns false when none is left.
__device__ __forceinline__ bool next_block_item(const TileQueue& q, int64_t total_tiles, int64_t& stride_next,
                                                int64_t& tile, int& block) {
  const int lane = threadIdx.x & 31;
  int64_t item;
  if (q.order) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(q.counter, 1u);
    item = (int64_t)__shfl_sync(0xffffffffu, it, 0);
    if (item >= 4 * (int64_t)q.total) return false;
    tile = q.order[item >> 2];
  } else {
    item = stride_next;
    stride_next += (int64_t)gridDim.x * (blockDim.x >> 5);
    if (item >= 4 * total_tiles) return false;
    tile = item >> 2;
  }
  block = (int)(item & 3);
  return true;
}

__device__ __forceinline__ Tile2 tile2_block_ctx(const potr_view_info* __restrict__ info, int n_views,
                                                 const uint32_t* __restrict__ ranges,
                                                 const potr_raster_config& cfg, int64_t tile, int blk) {
  Tile2 c;
  c.tile = tile;
  c.view = view_of_tile(info, n_views, tile);
  c.vi = info[c.view];
  const int64_t local = tile - c.vi.tile_base;
  c.ty = (int)(local / c.vi.tiles_x);
  c.tx = (int)(local - (int64_t)c.ty * c.vi.tiles_x);
  const int lane = (int)(threadIdx.x & 31), bx_n = cfg.tile_w / 8;
  const int bx = c.tx * cfg.tile_w + (blk % bx_n) * 8, by = c.ty * cfg.tile_h + (blk / bx_n) * 8;
  c.px = bx + (lane & 7);
  c.py = by + 2 * (lane >> 3);
  c.in0 = c.px < c.vi.width && c.py < c.vi.height;
  c.in1 = c.px < c.vi.width && c.py + 1 < c.vi.height;
  c.fx = (float)c.px + 0.5f;
  c.fy0 = (float)c.py + 0.5f;
  c.fy1 = (float)(c.py + 1) + 0.5f;
  c.bx0 = (float)bx + 0.5f;
  c.by0 = (float)by + 0.5f;
  c.s = ranges[2 * tile];
  c.e = ranges[2 * tile + 1];
  return c;
}

// Lane j gathers the record of list entry first + j (if j < cnt) into slot[j] (cp.async, one
// commit group per call).
__device__ __forceinline__ void warp_stage(float4* slot, const float4* __restrict__ raster,
                                           const uint32_t* __restrict__ vals, uint32_t first, int cnt) {
  const int lane = threadIdx.x & 31;
  if (lane < cnt) {
    const float4* src = raster + (size_t)vals[first + lane] * kRec;
    cp_async16_2(slot + kSRec2 * lane + 0, src + 0);
    cp_async16_2(slot + kSRec2 * lane + 1, src + 1);
    cp_async16_2(slot + kSRec2 * lane + 2, src + 2);
  }
  asm volatile("cp.async.commit_group;\n" ::);
}

// Forward walk (Section 3, Eqs. 2-4) of the tile list at the lane's two pixels, by one warp on
// its own: colour, final transmittance and n_last of each pixel.  ring: the warp's kWRing
// slots of kWSlot float4.
__device__ __forceinline__ void forward_walk_w(float4* ring, const float4* __restrict__ raster,
                                               const uint32_t* __restrict__ vals, const Tile2& c,
                                               const potr_raster_config& cfg, f2_t (&C)[3], f2_t& T,
                                               uint32_t& last0, uint32_t& last1) {
  C[0] = C[1] = C[2] = f2s(0.0f);
  T = f2s(1.0f);
  last0 = last1 = 0;
  bool done0 = !c.in0, done1 = !c.in1;
  const int lane = threadIdx.x & 31;
  const f2_t fx2 = f2s(c.fx), fy2 = f2(c.fy0, c.fy1);
  const uint32_t len = c.e - c.s;
  const uint32_t ng = (len + 31) / 32;
  if (ng > 0) warp_stage(ring, raster, vals, c.s, (int)min(32u, len));
  for (uint32_t gi = 0; gi < ng; ++gi) {
    if (__all_sync(0xffffffffu, done0 && done1)) break;
    const uint32_t g = gi * 32;
    const int cnt = (int)min(32u, len - g);
    if (gi + 1 < ng) {
      warp_stage(ring + kWSlot * ((gi + 1) % kWRing), raster, vals, c.s + g + 32, (int)min(32u, len - g - 32));
      cp_async_wait2<1>();
    } else {
      cp_async_wait2<0>();
    }
    float4* ex = ring + kWRing * kWSlot;
    if (lane < cnt) expand_record(ring + kWSlot * (gi % kWRing) + kSRec2 * lane, ex + kERec * lane);  // own copy
    __syncwarp();  // every lane's expanded record of this group is visible
    const bool cand = lane < cnt && block_may_pass_e(ex + kERec * lane, c.bx0, c.by0);
    uint32_t m = __ballot_sync(0xffffffffu, cand);
    while (m) {
      const int j = __ffs(m) - 1;
      m &= m - 1;
      forward_visit_e(ex + kERec * j, g + (uint32_t)j, fx2, fy2, cfg, C, T, last0, last1, done0, done1);
    }
    __syncwarp();  // the expanded records and this slot are rewritten later
  }
  cp_async_wait2<0>();  // after an early exit the next group may still be landing
  __syncwarp();
}

}  // namespace
}  // namespace potr
