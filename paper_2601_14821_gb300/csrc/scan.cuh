// scan.cuh -- exclusive prefix sums on the device: a two-level reduce-then-scan (no waiting
// between blocks).  Shared by the binning and the codec.
#pragma once

#include "potr_device.cuh"

namespace potr {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;  // items per block

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// -----------------------------------------------------------------------------------------
// Block-wide exclusive scan of kScanChunk items.  Warp w owns items [w*256, w*256+256) with
// lane l holding items l + 32 j (j = 0..7): loads and stores are coalesced.
// -----------------------------------------------------------------------------------------
template <typename Tin, typename Tacc, typename Tout>
__global__ void __launch_bounds__(kScanThreads) scan_chunks_kernel(const Tin* in, Tout* out, int64_t n,
                                                                   Tacc* __restrict__ chunk_sums) {
  __shared__ Tacc warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)warp * 256;
  Tacc v[kScanItems];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = base + lane + 32 * j;
    v[j] = (i < n) ? (Tacc)in[i] : (Tacc)0;
  }
  Tacc carry = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    Tacc x = v[j];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Tacc y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const Tacc row_total = __shfl_sync(0xffffffffu, x, 31);
    v[j] = carry + x - v[j];  // exclusive within the warp's 256 items
    carry += row_total;
  }
  if (lane == 0) warp_tot[warp] = carry;
  __syncthreads();
  Tacc wbase = 0, btot = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    const Tacc t = warp_tot[w];
    if (w < warp) wbase += t;
    btot += t;
  }
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = base + lane + 32 * j;
    if (i < n) out[i] = (Tout)(v[j] + wbase);
  }
  if (threadIdx.x == 0) chunk_sums[blockIdx.x] = btot;
}

template <typename Tout>
__global__ void __launch_bounds__(256) add_chunk_base_kernel(Tout* out, int64_t n,
                                                             const uint64_t* __restrict__ chunk_base) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (Tout)((uint64_t)out[i] + chunk_base[i / kScanChunk]);
}

__global__ void store_total_kernel(const uint64_t* __restrict__ chunk_sums, uint64_t* __restrict__ total) {
  *total = chunk_sums[0];
}

// Workspace for an exclusive scan of n items: one u64 per chunk at each level.
int64_t scan_ws_words(int64_t n) {
  int64_t w = 0;
  int64_t m = n;
  do {
    m = ceil_div(m, kScanChunk);
    w += m;
  } while (m > 1);
  return w + 1;
}

// Exclusive scan of x_i = in[i] for i in [0, n) -> out, total (u64) -> *total.  ws:
// scan_ws_words(n) u64 words.
template <typename Tin, typename Tout>
cudaError_t scan_exclusive(const Tin* in, Tout* out, int64_t n, uint64_t* total, uint64_t* ws, cudaStream_t s) {
  const int64_t nb = ceil_div(n, kScanChunk);
  uint64_t* sums = ws;
  scan_chunks_kernel<Tin, uint64_t, Tout><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  note_launches(2);  // this level's scan plus the store or the add below
  if (nb == 1) {
    store_total_kernel<<<1, 1, 0, s>>>(sums, total);
  } else {
    cudaError_t e = scan_exclusive<uint64_t, uint64_t>(sums, sums, nb, total, ws + nb, s);
    if (e != cudaSuccess) return e;
    add_chunk_base_kernel<Tout><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(out, n, sums);
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace potr
