// schedule.cu -- longest-list-first order of a frame's tiles for the persistent tile kernels.
//
// A tile's cost grows with its list length, and the lengths are very uneven (a few hundred
// tiles over a dense region hold most instances).  Tiles are bucketed by bit length of their
// list length (bucket 0 = empty); the order lists buckets from the longest down, so the
// heaviest tiles start first and the short ones fill the tail.  Order inside a bucket is the
// order of atomic increments: it affects only which CTA renders a tile, never a result.
#include "potr_device.cuh"

namespace potr {
namespace {

constexpr int kBuckets = 33;

__device__ __forceinline__ int bucket_of(uint32_t len) { return len == 0 ? 0 : 32 - __clz(len); }

__global__ void __launch_bounds__(256) bucket_count_kernel(const uint32_t* __restrict__ ranges, int64_t total,
                                                           uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[kBuckets];
  if (threadIdx.x < kBuckets) h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[bucket_of(ranges[2 * t + 1] - ranges[2 * t])], 1u);
  __syncthreads();
  if (threadIdx.x < kBuckets && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

// start[b] = number of tiles in buckets above b (longest first); cursors start there.
__global__ void bucket_start_kernel(const uint32_t* __restrict__ counts, uint32_t* __restrict__ cursor) {
  uint32_t run = 0;
  for (int b = kBuckets - 1; b >= 0; --b) {
    cursor[b] = run;
    run += counts[b];
  }
}

__global__ void __launch_bounds__(256) bucket_scatter_kernel(const uint32_t* __restrict__ ranges, int64_t total,
                                                             uint32_t* __restrict__ cursor, uint32_t* __restrict__ order) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int b = bucket_of(ranges[2 * t + 1] - ranges[2 * t]);
    order[atomicAdd(&cursor[b], 1u)] = (uint32_t)t;
  }
}

}  // namespace
}  // namespace potr

extern "C" size_t potr_tile_schedule_workspace_size(void) { return sizeof(uint32_t) * 2 * potr::kBuckets; }

extern "C" potr_status potr_tile_schedule(const potr_frame* frame, const uint32_t* d_tile_ranges,
                                          uint32_t* d_tile_order, void* d_ws, size_t ws_bytes, potr_stream_t stream) {
  using namespace potr;
  if (!frame || !d_tile_ranges || !d_tile_order || !d_ws) return POTR_ERR_INVALID_ARGUMENT;
  if (frame->total_tiles <= 0 || frame->total_tiles > 0x7fffffffll) return POTR_ERR_INVALID_ARGUMENT;
  if (ws_bytes < potr_tile_schedule_workspace_size()) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* counts = static_cast<uint32_t*>(d_ws);
  uint32_t* cursor = counts + kBuckets;
  if (cudaMemsetAsync(counts, 0, sizeof(uint32_t) * kBuckets, s) != cudaSuccess) return POTR_ERR_CUDA;
  int64_t g = (frame->total_tiles + 255) / 256;
  if (g > 152 * 4) g = 152 * 4;
  bucket_count_kernel<<<(unsigned)g, 256, 0, s>>>(d_tile_ranges, frame->total_tiles, counts);
  POTR_CHECK_LAUNCH();
  bucket_start_kernel<<<1, 1, 0, s>>>(counts, cursor);
  POTR_CHECK_LAUNCH();
  bucket_scatter_kernel<<<(unsigned)g, 256, 0, s>>>(d_tile_ranges, frame->total_tiles, cursor, d_tile_order);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
