// codec_common.cuh -- pieces the codec's encoder and decoder (Section IV-E) share: the octree's
// depth limit, the root cube, and an exclusive running maximum down the columns of a table
// (the per-block "last position" tables that both sides' backward searches fall back to).
#pragma once

#include "potr_device.cuh"

namespace potr {
namespace {

constexpr int kDepth = 21;          // octree depth limit: 63-bit cell codes
constexpr int kLevels = kDepth + 1;
constexpr int kChunkCodec = 1024;   // positions per block of a backward search

struct Cube {
  double corner[3];
  double S;
};

// Centre coordinate of the cell with integer coordinate X at depth d along one axis:
// corner + (X + 1/2) S / 2^d, binary64 in that order.
__device__ __forceinline__ double cell_centre(double corner, double S, uint32_t X, int d) {
  const double w = __ddiv_rn(S, (double)(1u << d));
  return __dadd_rn(corner, __dmul_rn(__dadd_rn((double)X, 0.5), w));
}

// a[r][c] <- max(-1, a[0][c], ..., a[r-1][c]) for every column c (one block per column).
__global__ void __launch_bounds__(256) prefix_max_columns_kernel(int64_t rows, int cols, int* __restrict__ a) {
  __shared__ int warp_max[8];
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int carry = -1;
  for (int64_t r0 = 0; r0 < rows; r0 += 256) {
    const int64_t r = r0 + threadIdx.x;
    const int x = r < rows ? a[r * cols + c] : -1;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl = max(incl, y);
    }
    if (lane == 31) warp_max[warp] = incl;
    __syncthreads();
    int before = carry;
    for (int w = 0; w < warp; ++w) before = max(before, warp_max[w]);
    const int prev = __shfl_up_sync(0xffffffffu, incl, 1);  // every lane takes part
    if (r < rows) a[r * cols + c] = lane > 0 ? max(before, prev) : before;
    int tile = carry;
    for (int w = 0; w < 8; ++w) tile = max(tile, warp_max[w]);
    carry = tile;
    __syncthreads();
  }
}

}  // namespace
}  // namespace potr
