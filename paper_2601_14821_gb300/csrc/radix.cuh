// radix.cuh -- stable LSD radix sort passes of 32-bit keys with 32-bit values, one kernel per
// 8-bit pass ("onesweep": Adinets & Merrill, 2022), shared by the tile binning and the codec.
#pragma once

#include "potr_device.cuh"

namespace potr {
namespace {

constexpr int kOsThreads = 256;
constexpr int kOsItems = 16;
constexpr int kOsTile = kOsThreads * kOsItems;  // items per block and pass
constexpr int kMaxPasses = 8;
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62, kCountMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;

// -----------------------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits, one kernel per pass ("onesweep": Adinets & Merrill,
// 2022).  One read of the keys builds the digit histograms of every pass; then each pass
// ranks 4096 items per block stably (per-warp equal-digit masks built by shared-memory ORs,
// warps in order), publishes its per-digit counts, finds the counts of all earlier blocks by decoupled
// look-back over the published words, and writes its items grouped by digit through shared
// memory so that the global stores are contiguous runs.  Blocks take their item range from an
// atomic counter, so every block a look-back waits on is already running; the wait is bounded
// and reports POTR_ERR_TIMEOUT instead of hanging.
// -----------------------------------------------------------------------------------------
size_t onesweep_smem_bytes() { return sizeof(uint32_t) * 2 * kOsTile + sizeof(uint32_t) * (8 * 257 + 2 * 256); }

// Exclusive scan of one value per thread over a 256-thread block (returns this thread's prefix).
__device__ __forceinline__ uint32_t block_exclusive_scan256(uint32_t x, uint32_t* tmp8) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) tmp8[warp] = incl;
  __syncthreads();
  uint32_t wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += tmp8[w];
  __syncthreads();
  return wbase + incl - x;
}

// Decoupled look-back for digit t of block `tile`: the sum of the counts published by blocks
// 0 .. tile-1 (walking back until an inclusive prefix).  Four predecessors' words are loaded
// at once (independent loads) and consumed nearest first; a word that is not yet published
// restarts the window there.  After spin_limit such restarts the wait ends: *err is set and the
// partial sum returned.
__device__ __forceinline__ uint64_t lookback_prefix(volatile unsigned long long* vst, int64_t tile, uint32_t t,
                                                    int spin_limit, int* err) {
  constexpr int kWin = 4;
  uint64_t excl = 0;
  int64_t p = tile - 1;
  int spins = 0;
  while (p >= 0) {
    unsigned long long x[kWin];
#pragma unroll
    for (int i = 0; i < kWin; ++i) x[i] = (p - i >= 0) ? vst[(p - i) * 256 + t] : (kFlagInc | 0ull);
    int used = 0;
    bool done = false, stalled = false;
#pragma unroll
    for (int i = 0; i < kWin; ++i) {
      if (done || stalled) continue;
      const unsigned long long flag = x[i] >> 62;
      if (flag == 0) {
        stalled = true;
        continue;
      }
      excl += x[i] & kCountMask;
      ++used;
      if (flag == 2) done = true;
    }
    if (done) break;
    p -= used;
    if (stalled) {
      if (++spins > spin_limit) {
        *err = 1;
        break;
      }
      __nanosleep(64);  // leave the issue slots to the blocks that do work meanwhile
    }
  }
  return excl;
}

__global__ void __launch_bounds__(256) digit_base_kernel(const uint32_t* __restrict__ ghist, int passes,
                                                         uint32_t* __restrict__ gbase) {
  __shared__ uint32_t tmp8[8];
  for (int p = 0; p < passes; ++p) gbase[p * 256 + threadIdx.x] = block_exclusive_scan256(ghist[p * 256 + threadIdx.x], tmp8);
}

// vals_in == nullptr: the value of item i is i itself.  The item count is *m_dev, or m_host
// when m_dev is null.
__global__ void __launch_bounds__(kOsThreads, 5) onesweep_kernel(const uint32_t* __restrict__ keys_in,
                                                              const uint32_t* __restrict__ vals_in,
                                                              const uint64_t* __restrict__ m_dev, int64_t m_host,
                                                              int shift,
                                                              const uint32_t* __restrict__ gbase,
                                                              uint32_t* __restrict__ tile_counter,
                                                              unsigned long long* status,
                                                              uint32_t* __restrict__ keys_out,
                                                              uint32_t* __restrict__ vals_out,
                                                              potr_device_status* __restrict__ st) {
  extern __shared__ uint32_t os_smem[];
  uint32_t* s_keys = os_smem;                                          // [kOsTile]
  uint32_t* s_vals = s_keys + kOsTile;                                 // [kOsTile]
  uint32_t* warp_cnt = s_vals + kOsTile;                               // [8][257]
  uint32_t* dig_glob = warp_cnt + 8 * 257;                             // [256]
  uint32_t* tmp8 = dig_glob + 256;                                     // [8]
  __shared__ uint32_t s_tile;
  __shared__ int s_err;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(tile_counter, 1u);
    s_err = 0;
  }
  for (int w = 0; w < 8; ++w) warp_cnt[w * 257 + threadIdx.x] = s_vals[w * 257 + threadIdx.x] = 0;
  if (threadIdx.x < 8) warp_cnt[threadIdx.x * 257 + 256] = s_vals[threadIdx.x * 257 + 256] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t m = m_dev ? (int64_t)*m_dev : m_host;
  const int64_t base = (int64_t)tile * kOsTile;
  if (base >= m) return;  // uniform per block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  // Keys (and ranks) stay in registers; values are loaded only when they are scattered, and
  // digits are recomputed from the keys, so that five blocks fit on an SM.
  const int64_t ibase = base + warp * (kOsItems * 32) + lane;  // item r is ibase + 32 r
  const int nv = (int)min((int64_t)kOsItems, (m - ibase + 31) / 32);  // items r < nv are valid
  uint32_t k[kOsItems], lr[kOsItems];
#pragma unroll
  for (int r = 0; r < kOsItems; ++r) k[r] = r < nv ? keys_in[ibase + 32 * r] : 0u;
  // stable rank inside the warp: rounds in order, lanes in order.  The lanes holding the same
  // digit find each other through a per-warp mask word per digit (each lane ORs in its bit; the
  // result does not depend on the order of the ORs), kept in the value staging area, which is
  // unused until the scatter; the round's lowest such lane adds the count and clears the word.
  uint32_t* wc = warp_cnt + warp * 257;
  uint32_t* wm = s_vals + warp * 257;
#pragma unroll
  for (int r = 0; r < kOsItems; ++r) {
    const uint32_t d = r < nv ? (k[r] >> shift) & 0xffu : 256u;
    atomicOr(&wm[d], 1u << lane);
    __syncwarp();
    const uint32_t peers = wm[d];
    const uint32_t rank = __popc(peers & lt);
    const uint32_t c0 = wc[d];
    __syncwarp();
    if (rank == 0) {
      wc[d] = c0 + __popc(peers);
      wm[d] = 0u;
    }
    __syncwarp();
    lr[r] = c0 + rank;
  }
  __syncthreads();
  // per digit (one per thread): exclusive prefix over warps, block count
  const uint32_t t = threadIdx.x;
  uint32_t run = 0;
  for (int w = 0; w < 8; ++w) {
    const uint32_t c = warp_cnt[w * 257 + t];
    warp_cnt[w * 257 + t] = run;
    run += c;
  }
  volatile unsigned long long* vst = status;
  const int64_t si = (int64_t)tile * 256 + t;
  uint64_t excl = 0;
  if (tile == 0) {
    vst[si] = kFlagInc | run;
  } else {
    vst[si] = kFlagAgg | run;
    excl = lookback_prefix(vst, tile, t, kSpinLimit, &s_err);
    vst[si] = kFlagInc | (excl + run);
  }
  // the block's digit-t items start at bo in the block's digit order: item i of that order (a
  // digit-t item) goes to dig_glob[t] + i, and an item of warp w goes to warp_cnt[w][t] + rank
  const uint32_t bo = block_exclusive_scan256(run, tmp8);
  dig_glob[t] = gbase[t] + (uint32_t)excl - bo;
  for (int w = 0; w < 8; ++w) warp_cnt[w * 257 + t] += bo;
  __syncthreads();
  // items grouped by digit in shared memory: keys, then the values (loaded now)
#pragma unroll
  for (int r = 0; r < kOsItems; ++r) {
    if (r < nv) {
      const uint32_t d = (k[r] >> shift) & 0xffu;
      const uint32_t pos = warp_cnt[warp * 257 + d] + lr[r];
      s_keys[pos] = k[r];
      lr[r] = pos;
    }
  }
#pragma unroll
  for (int r = 0; r < kOsItems; ++r)
    if (r < nv) s_vals[lr[r]] = vals_in ? vals_in[ibase + 32 * r] : (uint32_t)(ibase + 32 * r);
  __syncthreads();
  const int nvalid = (int)min((int64_t)kOsTile, m - base);
  for (int i = threadIdx.x; i < nvalid; i += kOsThreads) {
    const uint32_t key = s_keys[i];
    const uint32_t d = (key >> shift) & 0xffu;
    const uint32_t o = dig_glob[d] + (uint32_t)i;
    keys_out[o] = key;
    vals_out[o] = s_vals[i];
  }
  if (threadIdx.x == 0 && s_err) set_status(st, POTR_ERR_TIMEOUT, 0);
}

// One onesweep pass over m items (count in device memory at m_dev, or m_host).
cudaError_t onesweep_pass(const uint32_t* k_in, const uint32_t* v_in, const uint64_t* m_dev, int64_t m_host,
                          int64_t blocks, int shift, const uint32_t* gbase, uint32_t* counter,
                          unsigned long long* status, uint32_t* k_out, uint32_t* v_out, potr_device_status* st,
                          cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned long long) * 256 * (size_t)blocks, s);
  if (e != cudaSuccess) return e;
  onesweep_kernel<<<(unsigned)blocks, kOsThreads, onesweep_smem_bytes(), s>>>(k_in, v_in, m_dev, m_host, shift, gbase,
                                                                            counter, status, k_out, v_out, st);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace
}  // namespace potr
