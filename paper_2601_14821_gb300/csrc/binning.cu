// binning.cu -- tile binning of the projected splats (paper Section 3: splats are
// alpha-composited as layers ordered by approximate depth): exclusive scan of the per-(view,
// splat) kept-tile counts, a stable radix sort of the (view, splat) pairs by depth, emission of
// one (global tile, vk) instance per kept tile in that depth order, a stable radix partition of
// the instances by tile, and per-tile [start, end) ranges.
//
// Everything is integer work and bit-exact: the scan is a two-level reduce-then-scan (no
// inter-block waiting), the sort ranks items stably inside a block with per-warp equal-digit
// masks, so its result equals std::stable_sort of the keys.  The kernels read the instance
// count from device memory so that a whole frame can be captured in a CUDA graph.
#include "radix.cuh"
#include "scan.cuh"

namespace potr {
namespace {

// -----------------------------------------------------------------------------------------
// Instance count check, depth keys and emission.
// -----------------------------------------------------------------------------------------
__global__ void count_check_kernel(const uint64_t* __restrict__ total, int64_t capacity, uint32_t* __restrict__ n_inst,
                                   uint64_t* __restrict__ m_eff, potr_device_status* __restrict__ st) {
  const uint64_t t = *total;
  const bool ok = t <= (uint64_t)capacity;
  *n_inst = t > 0xffffffffull ? 0xffffffffu : (uint32_t)t;
  *m_eff = ok ? t : 0;
  if (!ok) set_status(st, POTR_ERR_CAPACITY, (int64_t)t);
}

// Depth sort keys of every vk (bits of the camera-space depth, which order like the positive
// floats they are; 0xffffffff for a vk without kept tiles, so it sorts last) and the digit
// histograms of the four depth passes.
__global__ void __launch_bounds__(256) depth_key_kernel(const uint32_t* __restrict__ touched,
                                                        const float* __restrict__ depth, int64_t n_vk,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[4][256];
  for (int p = 0; p < 4; ++p) h[p][threadIdx.x] = 0;
  __syncthreads();
  for (int64_t vk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; vk < n_vk; vk += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = touched[vk] ? __float_as_uint(depth[vk]) : 0xffffffffu;
    keys[vk] = key;
#pragma unroll
    for (int p = 0; p < 4; ++p) atomicAdd(&h[p][(key >> (8 * p)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int p = 0; p < 4; ++p)
    if (h[p][threadIdx.x]) atomicAdd(&ghist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

// Kept-tile count of every group of 32 consecutive entries of the depth-sorted vk order (one
// warp per group: the counts gathered from touched and added by a warp reduction).
__global__ void __launch_bounds__(256) group_count_kernel(const uint32_t* __restrict__ order,
                                                          const uint32_t* __restrict__ touched, int64_t n_vk,
                                                          uint32_t* __restrict__ gcount) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wv = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wv * 32 < n_vk; wv += warps_total) {
    const int64_t i = wv * 32 + lane;
    const uint32_t c = i < n_vk ? touched[order[i]] : 0u;
    const uint32_t sum = __reduce_add_sync(0xffffffffu, c);  // a count is below 2^21
    if (lane == 0) gcount[wv] = sum;
  }
}

// Emission in depth order.  One warp per 32 consecutive entries of the depth-sorted vk order;
// their emission slots form one contiguous run, which starts at gbase[group] (the exclusive
// prefix of the groups' kept-tile counts), so lane l takes slots l, l + 32, ... of the run, finds the owning
// entry by a 5-step shuffle search over the warp's exclusive counts, and derives the tile
// from the slot's rank among that vk's kept tiles (row-major in its rectangle, through the
// kept-tile mask).  Stores are coalesced whatever the rectangle sizes.  Each instance gets key
// = global tile and value = vk; a stable partition by tile then yields per-tile lists in
// (depth, vk) order.  An entry's fields travel packed: its first tile (the rectangle's corner),
// and rectangle width | all-kept flag << 11 | view tiles_x << 12.  The tile digits of every
// partition pass are counted here in shared memory: one add per warp when the warp's 32 keys
// share the digit (the usual case above the lowest byte), else one add per lane.
__global__ void __launch_bounds__(256) emit_kernel(const uint32_t* __restrict__ order, const uint32_t* __restrict__ gbase,
                                                   const potr_view_info* __restrict__ info, int64_t n, int64_t n_vk,
                                                   const uint64_t* __restrict__ m_eff,
                                                   const uint4* __restrict__ cull, uint32_t* __restrict__ keys,
                                                   uint32_t* __restrict__ vals, int passes, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[kMaxPasses][256];
  for (int p = 0; p < passes; ++p) h[p][threadIdx.x] = 0;
  __syncthreads();
  if (*m_eff == 0) return;  // uniform: nothing emitted, nothing counted
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wv = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wv * 32 < n_vk; wv += warps_total) {
    const int64_t i = wv * 32 + lane;
    uint32_t vk = 0, cnt = 0, corner = 0, pk = 1u, m_lo = 0, m_hi = 0;
    if (i < n_vk) {
      vk = order[i];
      // culling word: kept-tile mask, rectangle word, kept count | all-kept << 31
      const uint4 m = cull[vk];
      cnt = m.w & 0x7fffffffu;
      if (cnt) {
        const potr_view_info& vi = info[(int)(vk / (uint32_t)n)];  // n * n_views < 2^32
        const uint32_t rw = m.z;
        const uint32_t tiles_x = (uint32_t)vi.tiles_x;
        corner = (uint32_t)vi.tile_base + ((rw >> 11) & 0x7ffu) * tiles_x + (rw & 0x7ffu);
        pk = (rw >> 22) | ((m.w >> 31) << 11) | (tiles_x << 12);
        m_lo = m.x;
        m_hi = m.y;
      }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;
    const uint32_t run0 = gbase[wv];  // below the capacity when m_eff is not 0
    for (uint32_t e0 = 0; e0 < total; e0 += 32) {
      const uint32_t e = e0 + lane;
      // owner: the last lane whose exclusive count is <= e (lanes with cnt = 0 never win ties
      // because the owner of e must have excl <= e < excl + cnt)
      uint32_t owner = 0;
#pragma unroll
      for (int b = 16; b >= 1; b >>= 1) {
        const uint32_t cand = owner + b;
        const uint32_t ce = __shfl_sync(0xffffffffu, excl, cand & 31);
        if (cand < 32 && ce <= e) owner = cand;
      }
      const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, owner);
      const uint32_t o_vk = __shfl_sync(0xffffffffu, vk, owner);
      const uint32_t o_corner = __shfl_sync(0xffffffffu, corner, owner);
      const uint32_t o_pk = __shfl_sync(0xffffffffu, pk, owner);
      const uint32_t o_mlo = __shfl_sync(0xffffffffu, m_lo, owner);
      const uint32_t o_mhi = __shfl_sync(0xffffffffu, m_hi, owner);
      uint32_t tile = 0;
      if (e < total) {
        // the li-th kept tile of the owner's rectangle, row-major
        const uint32_t w = o_pk & 0x7ffu, all = (o_pk >> 11) & 1u, tiles_x = o_pk >> 12;
        const uint32_t li = all ? e - o_excl : select_bit64(((uint64_t)o_mhi << 32) | o_mlo, e - o_excl);
        const uint32_t dy = all ? li / w : small_div(li, w), dx = li - dy * w;  // masked: li < 64
        tile = o_corner + dy * tiles_x + dx;
        keys[run0 + e] = tile;
        vals[run0 + e] = o_vk;
      }
      const uint32_t n_valid = min(32u, total - e0);  // lanes 0 .. n_valid - 1 hold keys
      for (int p = 0; p < passes; ++p) {
        const uint32_t d = (tile >> (8 * p)) & 0xffu;
        const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
        if (__all_sync(0xffffffffu, e >= total || d == d0)) {
          if (lane == 0) atomicAdd(&h[p][d0], n_valid);
        } else if (e < total) {
          atomicAdd(&h[p][d], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p)
    if (h[p][threadIdx.x]) atomicAdd(&ghist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

// Self-test of the bounded wait: block 1 looks back at block 0, whose words nobody publishes.
__global__ void lookback_timeout_probe_kernel(unsigned long long* status, int spin_limit,
                                              potr_device_status* __restrict__ st) {
  __shared__ int s_err;
  if (threadIdx.x == 0) s_err = 0;
  __syncthreads();
  volatile unsigned long long* vst = status;
  const uint64_t got = lookback_prefix(vst, 1, threadIdx.x, spin_limit, &s_err);
  __syncthreads();
  if (threadIdx.x == 0 && s_err && got == 0) set_status(st, POTR_ERR_TIMEOUT, 0);
}

// Per tile [first, end) of its instances in the sorted keys.  Each thread takes four consecutive
// keys (one 16-byte load when the array is 16-byte aligned) and the key after them.
__global__ void __launch_bounds__(256) tile_ranges_kernel(const uint32_t* __restrict__ tiles, const uint64_t* __restrict__ m_eff,
                                                          int64_t total_tiles, uint32_t* __restrict__ ranges) {
  const int64_t m = (int64_t)*m_eff;
  const bool vec = (reinterpret_cast<uintptr_t>(tiles) & 15u) == 0;
  for (int64_t i0 = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); i0 < m;
       i0 += 4 * (int64_t)gridDim.x * blockDim.x) {
    uint32_t t[5];
    if (vec && i0 + 4 <= m) {
      const uint4 q = *reinterpret_cast<const uint4*>(tiles + i0);
      t[0] = q.x; t[1] = q.y; t[2] = q.z; t[3] = q.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) t[j] = i0 + j < m ? tiles[i0 + j] : 0xffffffffu;
    }
    t[4] = i0 + 4 < m ? tiles[i0 + 4] : 0xffffffffu;
    uint32_t prev = i0 > 0 ? tiles[i0 - 1] : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t i = i0 + j;
      if (i < m && t[j] < (uint64_t)total_tiles) {
        if (i == 0 || prev != t[j]) ranges[2 * t[j]] = (uint32_t)i;
        if (i == m - 1 || t[j + 1] != t[j]) ranges[2 * t[j] + 1] = (uint32_t)(i + 1);
      }
      prev = t[j];
    }
  }
}

int bits_for(int64_t x) {  // bits needed to represent values in [0, x)
  int b = 1;
  while (b < 63 && (int64_t(1) << b) < x) ++b;
  return b;
}

struct SortLayout {
  int64_t n_vk, scan_words, blocks_vk, blocks_inst, blocks_max;
  size_t off_scan, off_total, off_meff, off_dk0, off_dv0, off_dk1, off_dv1, off_keys_alt, off_vals_alt, off_status,
      off_ghist, off_gbase, off_counter, bytes;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

SortLayout sort_layout(int64_t n, int32_t n_views, int64_t capacity) {
  SortLayout L{};
  L.n_vk = n * (int64_t)n_views;
  L.scan_words = scan_ws_words(L.n_vk > 0 ? L.n_vk : 1);
  L.blocks_vk = ceil_div(L.n_vk > 0 ? L.n_vk : 1, kOsTile);
  L.blocks_inst = ceil_div(capacity > 0 ? capacity : 1, kOsTile);
  L.blocks_max = L.blocks_vk > L.blocks_inst ? L.blocks_vk : L.blocks_inst;
  const size_t vk_words = sizeof(uint32_t) * (size_t)L.n_vk;
  size_t o = 0;
  L.off_scan = o; o = align_up(o + sizeof(uint64_t) * L.scan_words);
  L.off_total = o; o = align_up(o + 2 * sizeof(uint64_t));
  L.off_meff = o; o = align_up(o + sizeof(uint64_t));
  L.off_dk0 = o; o = align_up(o + vk_words);
  L.off_dv0 = o; o = align_up(o + vk_words);
  L.off_dk1 = o; o = align_up(o + vk_words);
  L.off_dv1 = o; o = align_up(o + vk_words);
  L.off_keys_alt = o; o = align_up(o + sizeof(uint32_t) * (size_t)capacity);
  L.off_vals_alt = o; o = align_up(o + sizeof(uint32_t) * (size_t)capacity);
  L.off_status = o; o = align_up(o + sizeof(unsigned long long) * 256 * (size_t)L.blocks_max);
  L.off_ghist = o; o = align_up(o + sizeof(uint32_t) * 256 * kMaxPasses);
  L.off_gbase = o; o = align_up(o + sizeof(uint32_t) * 256 * kMaxPasses);
  L.off_counter = o; o = align_up(o + sizeof(uint32_t) * kMaxPasses);
  L.bytes = o;
  return L;
}

}  // namespace
}  // namespace potr

extern "C" size_t potr_bin_sort_workspace_size(int64_t n, int32_t n_views, int64_t total_tiles,
                                               int64_t instance_capacity) {
  (void)total_tiles;
  if (n <= 0 || n_views <= 0 || instance_capacity <= 0) return 0;
  return potr::sort_layout(n, n_views, instance_capacity).bytes;
}

// Binning in four steps, every one integer work and bit-exact:
//   1. exclusive scan of the kept-tile counts in vk order -> offsets (emission slots of the
//      vk-order definition, in views->offsets) and the instance total;
//   2. a stable LSD radix sort (4 x 8-bit passes) of the vk by depth bits: ties keep vk order;
//   3. emission in that depth order (slots from a scan of the counts of its groups of 32 entries),
//      key = global tile, value = vk;
//   4. a stable LSD radix sort of the instances by tile (8-bit passes over its significant
//      bits).  Per tile the instances keep step 3's order, (depth bits, vk), which is the
//      order of a stable sort of (tile, depth) keys emitted in vk order.
extern "C" potr_status potr_bin_sort(const potr_views* views, const potr_frame* frame, const potr_raster_config* cfg,
                                     int64_t n, int64_t instance_capacity, uint32_t* d_tiles, uint32_t* d_vals,
                                     uint32_t* d_tile_ranges, potr_device_status* d_status, void* d_ws, size_t ws_bytes,
                                     potr_stream_t stream) {
  using namespace potr;
  if (!views || !frame || !cfg || !d_tiles || !d_vals || !d_tile_ranges || !d_ws) return POTR_ERR_INVALID_ARGUMENT;
  if (n <= 0 || frame->n_views < 1 || frame->total_tiles <= 0 || !frame->info) return POTR_ERR_INVALID_ARGUMENT;
  if (instance_capacity <= 0 || instance_capacity > (int64_t)0xffffffffll) return POTR_ERR_INVALID_ARGUMENT;
  if (!views->touched || !views->offsets || !views->rect || !views->depth || !views->raster || !views->n_instances ||
      !views->cull)
    return POTR_ERR_INVALID_ARGUMENT;
  if (frame->total_tiles > (int64_t)0xffffffffll || n * (int64_t)frame->n_views >= (int64_t)0xffffffffll)
    return POTR_ERR_UNSUPPORTED;
  const SortLayout L = sort_layout(n, frame->n_views, instance_capacity);
  if (ws_bytes < L.bytes) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  uint64_t* scan_ws = reinterpret_cast<uint64_t*>(ws + L.off_scan);
  uint64_t* total = reinterpret_cast<uint64_t*>(ws + L.off_total);
  uint64_t* m_eff = reinterpret_cast<uint64_t*>(ws + L.off_meff);
  uint32_t* dk0 = reinterpret_cast<uint32_t*>(ws + L.off_dk0);
  uint32_t* dv0 = reinterpret_cast<uint32_t*>(ws + L.off_dv0);
  uint32_t* dk1 = reinterpret_cast<uint32_t*>(ws + L.off_dk1);
  uint32_t* dv1 = reinterpret_cast<uint32_t*>(ws + L.off_dv1);
  uint32_t* keys_alt = reinterpret_cast<uint32_t*>(ws + L.off_keys_alt);
  uint32_t* vals_alt = reinterpret_cast<uint32_t*>(ws + L.off_vals_alt);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(ws + L.off_status);
  uint32_t* ghist = reinterpret_cast<uint32_t*>(ws + L.off_ghist);
  uint32_t* gbase = reinterpret_cast<uint32_t*>(ws + L.off_gbase);
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws + L.off_counter);
  const int tile_passes = (bits_for(frame->total_tiles) + 7) / 8;
  if (4 + tile_passes > kMaxPasses) return POTR_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem_bytes()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return POTR_ERR_CUDA;

  // 1. slots in vk order, instance total, capacity check
  if (scan_exclusive<uint32_t, uint32_t>(views->touched, views->offsets, L.n_vk, total, scan_ws, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  count_check_kernel<<<1, 1, 0, s>>>(total, instance_capacity, views->n_instances, m_eff, d_status);
  POTR_CHECK_LAUNCH();
  if (cudaMemsetAsync(ghist, 0, sizeof(uint32_t) * 256 * kMaxPasses, s) != cudaSuccess) return POTR_ERR_CUDA;
  if (cudaMemsetAsync(counter, 0, sizeof(uint32_t) * kMaxPasses, s) != cudaSuccess) return POTR_ERR_CUDA;

  // 2. vk by depth: keys dk0 (values implicit) -> dk1/dv1 -> dk0/dv0 -> dk1/dv1 -> dk0/dv0
  {
    const int64_t g = ceil_div(L.n_vk, 256);
    depth_key_kernel<<<(unsigned)(g < 152 * 8 ? g : 152 * 8), 256, 0, s>>>(
        views->touched, views->depth, L.n_vk, dk0, ghist);
    POTR_CHECK_LAUNCH();
    digit_base_kernel<<<1, 256, 0, s>>>(ghist, 4, gbase);
    POTR_CHECK_LAUNCH();
  }
  uint32_t *ka = dk0, *va = nullptr, *kb = dk1, *vb = dv1;
  for (int p = 0; p < 4; ++p) {
    if (onesweep_pass(ka, va, nullptr, L.n_vk, L.blocks_vk, 8 * p, gbase + 256 * p, counter + p, status, kb, vb,
                      d_status, s) != cudaSuccess)
      return POTR_ERR_CUDA;
    uint32_t* t = ka; ka = kb; kb = t;
    va = vb;
    vb = (vb == dv1) ? dv0 : dv1;
  }
  const uint32_t* order = va;  // dv0: vk in (depth bits, vk) order

  // 3. slots in depth order: counts of the groups of 32 entries, their exclusive scan (dv1 is free
  // now: the counts in its first half, the scan in its second), then the emission
  const int64_t n_groups = ceil_div(L.n_vk, 32);
  uint32_t* gcount = dv1;
  uint32_t* group_base = dv1 + n_groups;
  {
    const int64_t g = ceil_div(L.n_vk, 256);
    group_count_kernel<<<(unsigned)(g < 152 * 16 ? g : 152 * 16), 256, 0, s>>>(order, views->touched, L.n_vk, gcount);
    POTR_CHECK_LAUNCH();
  }
  if (scan_exclusive<uint32_t, uint32_t>(gcount, group_base, n_groups, total + 1, scan_ws, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  // emit where the last tile pass lands in d_tiles / d_vals
  uint32_t* k_src = (tile_passes & 1) ? keys_alt : d_tiles;
  uint32_t* v_src = (tile_passes & 1) ? vals_alt : d_vals;
  uint32_t* k_dst = (tile_passes & 1) ? d_tiles : keys_alt;
  uint32_t* v_dst = (tile_passes & 1) ? d_vals : vals_alt;
  {
    const int64_t g = ceil_div(L.n_vk, 256);
    emit_kernel<<<(unsigned)(g < 152 * 32 ? g : 152 * 32), 256, 0, s>>>(
        order, group_base, frame->info, n, L.n_vk, m_eff, reinterpret_cast<const uint4*>(views->cull), k_src, v_src,
        tile_passes, ghist + 256 * 4);
    POTR_CHECK_LAUNCH();
    digit_base_kernel<<<1, 256, 0, s>>>(ghist + 256 * 4, tile_passes, gbase + 256 * 4);
    POTR_CHECK_LAUNCH();
  }

  // 4. instances by tile
  for (int p = 0; p < tile_passes; ++p) {
    if (onesweep_pass(k_src, v_src, m_eff, 0, L.blocks_inst, 8 * p, gbase + 256 * (4 + p), counter + 4 + p, status,
                      k_dst, v_dst, d_status, s) != cudaSuccess)
      return POTR_ERR_CUDA;
    uint32_t* tk = k_src; k_src = k_dst; k_dst = tk;
    uint32_t* tv = v_src; v_src = v_dst; v_dst = tv;
  }
  if (cudaMemsetAsync(d_tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)frame->total_tiles, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  {
    const int64_t g = ceil_div(instance_capacity, 4 * 256);
    tile_ranges_kernel<<<(unsigned)(g < 152 * 64 ? g : 152 * 64), 256, 0, s>>>(d_tiles, m_eff, frame->total_tiles,
                                                                               d_tile_ranges);
    POTR_CHECK_LAUNCH();
  }
  return POTR_OK;
}

extern "C" potr_status potr_selftest_wait_timeout(void* d_ws, size_t ws_bytes, int32_t spin_limit,
                                                  potr_device_status* d_status, potr_stream_t stream) {
  using namespace potr;
  if (!d_ws || !d_status || spin_limit < 1 || ws_bytes < 2 * 256 * sizeof(unsigned long long))
    return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* status = static_cast<unsigned long long*>(d_ws);
  if (cudaMemsetAsync(status, 0, 2 * 256 * sizeof(unsigned long long), s) != cudaSuccess) return POTR_ERR_CUDA;
  lookback_timeout_probe_kernel<<<1, 256, 0, s>>>(status, spin_limit, d_status);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
