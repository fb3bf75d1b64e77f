// raster_common.cuh -- building blocks shared by the tile kernels: the record gather of the
// pair-count kernel (one CTA of 256 threads per tile, one pixel per thread), emission slots,
// compensated sums and the tile queue.
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
  __device__ __forceinline__ float sum() const { return __fsub_rn(s, c); }  // rounded to binary32
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
