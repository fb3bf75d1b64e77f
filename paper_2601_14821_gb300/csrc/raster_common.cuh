// raster_common.cuh -- tile-kernel building blocks shared by the forward, removal and
// backward passes (one CTA of 256 threads per (view, tile), one pixel per thread).
#pragma once

#include "potr_device.cuh"

namespace potr {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSRec = 3;  // float4 per record in shared memory: the whole record
constexpr int kWarpW = 8, kWarpH = 4;  // pixel block of one warp

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit_wait() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

// Gather the raster records (three float4 each) of list entries [first, first + cnt) into smem
// (record stride kSRec) and wait for them; the culling words are read from global memory only
// where an emission slot is needed.
template <int BATCH>
__device__ __forceinline__ void stage_batch(float4* smem, const float4* __restrict__ raster,
                                            const uint32_t* __restrict__ vals, uint32_t first, int cnt) {
  for (int j = threadIdx.x; j < cnt; j += kThreads) {
    const uint32_t vk = vals[first + j];
    const float4* src = raster + (size_t)vk * kRec;
    cp_async16(smem + kSRec * j + 0, src + 0);
    cp_async16(smem + kSRec * j + 1, src + 1);
    cp_async16(smem + kSRec * j + 2, src + 2);
  }
  cp_async_commit_wait();
}

// Double-buffered batch staging: the gathers of one batch are in flight (cp.async, one commit
// group per batch) while the CTA works on the other buffer, and every thread already holds the
// list values (vk) of the batch after that in registers, so issuing never waits on a load.
template <int BATCH>
struct BatchStager {
  static constexpr int kPer = (BATCH + kThreads - 1) / kThreads;
  uint32_t vk[kPer];
  int loaded;
  __device__ __forceinline__ void load(const uint32_t* __restrict__ vals, uint32_t first, int cnt) {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int j = threadIdx.x + r * kThreads;
      vk[r] = j < cnt ? vals[first + j] : 0u;
    }
    loaded = cnt;
  }
  // With stored warp masks: their bytes for the same entries (gmask: the list's, from first).
  __device__ __forceinline__ void load_masks(const uint8_t* __restrict__ gmask, uint32_t first, int cnt,
                                             uint32_t (&mk)[kPer]) const {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int j = threadIdx.x + r * kThreads;
      mk[r] = j < cnt ? gmask[first + j] : 0u;
    }
  }
  __device__ __forceinline__ void issue(float4* buf, const float4* __restrict__ raster) const {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int j = threadIdx.x + r * kThreads;
      if (j < loaded) {
        const float4* src = raster + (size_t)vk[r] * kRec;
        cp_async16(buf + kSRec * j + 0, src + 0);
        cp_async16(buf + kSRec * j + 1, src + 1);
        cp_async16(buf + kSRec * j + 2, src + 2);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  }
};

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

struct TileCtx {
  int64_t tile;
  int view;
  potr_view_info vi;
  int px, py;
  bool inside;
  float fx, fy;
  uint32_t s, e;
  int tx, ty;
};

__device__ __forceinline__ TileCtx tile_ctx(const potr_view_info* __restrict__ info, int n_views,
                                            const uint32_t* __restrict__ ranges, const potr_raster_config& cfg,
                                            int64_t tile) {
  TileCtx c;
  c.tile = tile;
  c.view = view_of_tile(info, n_views, c.tile);
  c.vi = info[c.view];
  const int64_t local = c.tile - c.vi.tile_base;
  c.ty = (int)(local / c.vi.tiles_x);
  c.tx = (int)(local - (int64_t)c.ty * c.vi.tiles_x);
  // warp w covers the 8 x 4 pixel block (w mod (tile_w / 8), w div (tile_w / 8)) of the tile,
  // lane l its pixel (l mod 8, l div 8): compact blocks meet fewer splats only in part than
  // rows of the tile would
  const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5), bx_n = cfg.tile_w / kWarpW;
  c.px = c.tx * cfg.tile_w + (warp % bx_n) * kWarpW + (lane % kWarpW);
  c.py = c.ty * cfg.tile_h + (warp / bx_n) * kWarpH + (lane / kWarpW);
  c.inside = c.px < c.vi.width && c.py < c.vi.height;
  c.fx = (float)c.px + 0.5f;
  c.fy = (float)c.py + 0.5f;
  c.s = ranges[2 * c.tile];
  c.e = ranges[2 * c.tile + 1];
  return c;
}

// Bit w of the result is set when the splat of record (r0, r1) may pass the opacity
// prefilter (log2 G >= r1.z) at some pixel centre of warp w's 8 x 4 block of this tile.  For
// each pixel row y the exponent A u^2 + B u v + C v^2 (v = y - my fixed) is a concave parabola
// in u = x - mx, maximised over each block's 8-pixel span of the row; a pair whose warp bit is
// clear therefore has alpha < alpha_min at every pixel of that warp and is skipped without
// changing any decision.  The margin covers binary32 rounding of both evaluations.
__device__ __forceinline__ uint32_t warp_mask(const float4& r0, const float4& r1, const TileCtx& c,
                                              const potr_raster_config& cfg) {
  const float A = r0.z, B = r0.w, C = r1.x, thr = r1.z;
  if (!(thr < INFINITY)) return 0u;                             // o = 0: never passes
  if (!(thr > -INFINITY) || !(A < 0.0f) || !(C < 0.0f)) return 0xffu;  // no bound: keep all
  const float ux0 = ((float)(c.tx * cfg.tile_w) + 0.5f) - r0.x;
  const float k1 = -B / (2.0f * A);
  const int bx_n = cfg.tile_w / kWarpW;
  const float vy0 = ((float)(c.ty * cfg.tile_h) + 0.5f) - r0.y;
  uint32_t m = 0;
  for (int r = 0; r < cfg.tile_h; ++r) {
    const float v = vy0 + (float)r;
    const float us = k1 * v, bv = B * v, t3 = C * v * v;
    for (int xb = 0; xb < bx_n; ++xb) {
      const float lo = ux0 + (float)(kWarpW * xb);
      const float u = fminf(fmaxf(us, lo), lo + (float)(kWarpW - 1));
      const float t1 = A * u * u, t2 = bv * u;
      const float pmax = t1 + t2 + t3;
      const float margin = 1e-4f * (fabsf(t1) + fabsf(t2) + fabsf(t3)) + 1e-3f;
      if (pmax + margin >= thr) m |= 1u << ((r / kWarpH) * bx_n + xb);
    }
  }
  return m;
}

// Warp masks of the entries this thread gathered (its own cp.async copies are complete), also
// written to gout[j] when gout is not null.
template <int BATCH>
__device__ __forceinline__ void compute_masks(const float4* buf, uint8_t* wmask, int cnt, const TileCtx& c,
                                              const potr_raster_config& cfg, uint8_t* gout = nullptr) {
#pragma unroll
  for (int r = 0; r < BatchStager<BATCH>::kPer; ++r) {
    const int j = threadIdx.x + r * kThreads;
    if (j < cnt) {
      const uint8_t mk = (uint8_t)warp_mask(buf[kSRec * j], buf[kSRec * j + 1], c, cfg);
      wmask[j] = mk;
      if (gout) gout[j] = mk;
    }
  }
}

// Forward walk of the tile list (Section 3, Eqs. 2-4).  Returns colour, final T and n_last.
// smem holds two batches of records ([2][BATCH][kSRec]): the gathers of batch k + 1 are in
// flight while the CTA composites batch k.  Warp masks go to wmask, or, for list positions below
// mcap (a multiple of BATCH), to mcache[position], where a later back-to-front walk of the same
// list finds them instead of recomputing them (mcache may be null with mcap = 0); with gmask not
// null they are also written to gmask[position] (device memory, this tile's list).
template <int BATCH>
__device__ __forceinline__ void forward_walk(float4* smem, uint8_t* wmask, uint8_t* mcache, uint32_t mcap,
                                             const float4* __restrict__ raster, const uint32_t* __restrict__ vals,
                                             const TileCtx& c, const potr_raster_config& cfg, float (&C)[3], float& T,
                                             uint32_t& last, uint8_t* gmask = nullptr) {
  C[0] = C[1] = C[2] = 0.0f;
  T = 1.0f;
  last = 0;
  bool done = !c.inside;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t len = c.e - c.s;
  const uint32_t nb = (len + BATCH - 1) / BATCH;
  BatchStager<BATCH> st;
  if (nb > 0) {
    st.load(vals, c.s, (int)min((uint32_t)BATCH, len));
    st.issue(smem, raster);
  }
  if (nb > 1) st.load(vals, c.s + BATCH, (int)min((uint32_t)BATCH, len - BATCH));
  for (uint32_t k = 0; k < nb; ++k) {
    if (__syncthreads_and(done)) break;  // also: batch k - 1 (and its buffer) fully consumed
    const uint32_t pos0 = k * BATCH;
    const int cnt = (int)min((uint32_t)BATCH, len - pos0);
    const float4* buf = smem + kSRec * BATCH * (k & 1);
    if (k + 1 < nb) {
      st.issue(smem + kSRec * BATCH * ((k + 1) & 1), raster);
      cp_async_wait<1>();
      if (k + 2 < nb) st.load(vals, c.s + pos0 + 2 * BATCH, (int)min((uint32_t)BATCH, len - pos0 - 2 * BATCH));
    } else {
      cp_async_wait<0>();
    }
    uint8_t* bm = pos0 + BATCH <= mcap ? mcache + pos0 : wmask;
    compute_masks<BATCH>(buf, bm, cnt, c, cfg, gmask ? gmask + pos0 : nullptr);
    __syncthreads();
    for (int g = 0; g < cnt; g += 32) {
      if (__all_sync(0xffffffffu, done)) break;
      const int jl = g + lane;
      uint32_t m = __ballot_sync(0xffffffffu, jl < cnt && ((bm[jl] >> warp) & 1u));
      while (m) {
        const int j = g + __ffs(m) - 1;
        m &= m - 1;
        if (done) continue;
        const float4 r0 = buf[kSRec * j];
        const float4 r1 = buf[kSRec * j + 1];
        const float p = pair_exponent(r0.z, r0.w, r1.x, __fsub_rn(c.fx, r0.x), __fsub_rn(c.fy, r0.y));
        if (p < r1.z) continue;  // alpha < alpha_min certainly (prefilter with margin)
        const float a = pair_alpha(r1.y, p, cfg.alpha_max);
        if (a < cfg.alpha_min) continue;
        const float Tn = trans_next(a, T);
        if (Tn < cfg.t_min) {
          done = true;
          continue;
        }
        const float4 r2 = buf[kSRec * j + 2];
        const float w = a * T;
        C[0] = fmaf(w, r2.x, C[0]);
        C[1] = fmaf(w, r2.y, C[1]);
        C[2] = fmaf(w, r2.z, C[2]);
        T = Tn;
        last = pos0 + (uint32_t)j + 1;
      }
    }
  }
  cp_async_wait<0>();  // after an early exit the next batch may still be landing
}

// Emission slot of the instance in tile (tx, ty) of the splat whose first emission slot is off
// and whose culling word is m (kept-tile mask low / high, rectangle word, kept count | all-kept
// << 31): the first slot plus the number of its kept tiles before (tx, ty) in row-major order
// of its rectangle.
__device__ __forceinline__ uint32_t emission_slot(uint32_t off, const uint4& m, int tx, int ty) {
  const uint32_t rw = m.z;
  const uint32_t x0 = rw & 0x7ffu, y0 = (rw >> 11) & 0x7ffu, w = rw >> 22;
  const uint32_t pos = ((uint32_t)ty - y0) * w + ((uint32_t)tx - x0);
  if (m.w >> 31) return off + pos;
  const uint64_t mask = ((uint64_t)m.y << 32) | m.x;
  return off + (uint32_t)__popcll(mask & ((1ull << pos) - 1ull));
}

// Compensated (Kahan) binary32 summation: s + (-c) carries the sum to about binary64 accuracy
// for the handful of tile partials one (view, splat) has; plain adds, so nothing is contracted.
struct KahanSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Tile scheduling.  Without an order every CTA renders the tile of its block index.  With an
// order (a permutation of the frame's tiles, longest lists first, plus one work-counter word
// after it) a persistent grid of CTAs takes the next entry from the counter until the order
// is exhausted; only the processing order changes, never a result.
struct TileQueue {
  const uint32_t* order;  // nullable
  uint32_t* counter;
  uint32_t total;
};

__device__ __forceinline__ bool next_tile(const TileQueue& q, uint32_t* s_slot, bool first, int64_t& tile) {
  if (!q.order) {
    tile = blockIdx.x;
    return first;
  }
  __syncthreads();  // the previous tile's reads of s_slot and shared memory are done
  if (threadIdx.x == 0) *s_slot = atomicAdd(q.counter, 1u);
  __syncthreads();
  const uint32_t item = *s_slot;
  if (item >= q.total) return false;
  tile = q.order[item];
  return true;
}

// Grid for a tile kernel: one CTA per tile, or as many CTAs as fit on the device at once.
template <typename K>
inline unsigned tile_grid(K kernel, size_t smem, const TileQueue& q, int64_t total_tiles, int block = kTilePixels) {
  if (!q.order) return (unsigned)total_tiles;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  int64_t g = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  if (g > total_tiles) g = total_tiles;
  return (unsigned)(g > 0 ? g : 1);
}

inline bool valid_cfg(const potr_raster_config* cfg) {
  if (!cfg) return false;
  if (cfg->tile_w * cfg->tile_h != kTilePixels) return false;
  if (!((cfg->tile_w == 16 && cfg->tile_h == 16) || (cfg->tile_w == 8 && cfg->tile_h == 32) ||
        (cfg->tile_w == 32 && cfg->tile_h == 8)))
    return false;
  return cfg->batch == 128 || cfg->batch == 256 || cfg->batch == 512;
}

}  // namespace
}  // namespace potr
