// binning.cu -- tile binning of the projected splats: exclusive scan of per-(view, splat)
// tile counts, emission of one (global tile, depth) key per touched tile, a stable LSD radix
// sort of the 64-bit keys, and per-tile [start, end) ranges (paper Section 3: splats are
// alpha-composited as layers ordered by approximate depth).
//
// Everything is integer work and bit-exact: the scan is a two-level reduce-then-scan (no
// inter-block waiting), the sort ranks items stably inside a block with warp match masks, so
// its result equals std::stable_sort of the keys.  All kernels are HBM-bound; they read the
// instance count from device memory so that a whole frame can be captured in a CUDA graph.
#include "potr_device.cuh"

namespace potr {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;  // items per block
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // items per block

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// -----------------------------------------------------------------------------------------
// Block-wide exclusive scan of kScanChunk items.  Warp w owns items [w*256, w*256+256) with
// lane l holding items l + 32 j (j = 0..7): loads and stores are coalesced.
// -----------------------------------------------------------------------------------------
template <typename Tin, typename Tacc, typename Tout>
__global__ void __launch_bounds__(kScanThreads) scan_chunks_kernel(const Tin* in, Tout* out,
                                                                   int64_t n, Tacc* __restrict__ chunk_sums) {
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

// Exclusive scan in[0..n) -> out, total (u64) -> *total.  ws: scan_ws_words(n) u64 words.
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

// -----------------------------------------------------------------------------------------
// Instance count check and emission.
// -----------------------------------------------------------------------------------------
__global__ void count_check_kernel(const uint64_t* __restrict__ total, int64_t capacity, uint32_t* __restrict__ n_inst,
                                   uint64_t* __restrict__ m_eff, potr_device_status* __restrict__ st) {
  const uint64_t t = *total;
  const bool ok = t <= (uint64_t)capacity;
  *n_inst = t > 0xffffffffull ? 0xffffffffu : (uint32_t)t;
  *m_eff = ok ? t : 0;
  if (!ok) set_status(st, POTR_ERR_CAPACITY, (int64_t)t);
}

__global__ void __launch_bounds__(256) emit_kernel(const uint32_t* __restrict__ touched, const uint32_t* __restrict__ offsets,
                                                   const uint2* __restrict__ rect, const float* __restrict__ depth,
                                                   const potr_view_info* __restrict__ info, int64_t n, int64_t n_vk,
                                                   const uint64_t* __restrict__ m_eff, float4* __restrict__ raster,
                                                   uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  if (*m_eff == 0) return;
  for (int64_t vk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; vk < n_vk; vk += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t cnt = touched[vk];
    if (cnt == 0) continue;
    const uint32_t off = offsets[vk];
    reinterpret_cast<float*>(raster + vk * 3 + 1)[3] = __uint_as_float(off);
    const int v = (int)(vk / n);
    const potr_view_info vi = info[v];
    const uint2 r = rect[vk];
    const uint32_t x0 = r.x & 0xffffu, y0 = r.x >> 16, x1 = r.y & 0xffffu, y1 = r.y >> 16;
    const uint64_t lo = (uint64_t)__float_as_uint(depth[vk]);
    uint32_t e = off;
    for (uint32_t ty = y0; ty < y1; ++ty) {
      const uint64_t row = (uint64_t)vi.tile_base + (uint64_t)ty * (uint64_t)vi.tiles_x;
      for (uint32_t tx = x0; tx < x1; ++tx, ++e) {
        keys[e] = ((row + tx) << 32) | lo;
        vals[e] = (uint32_t)vk;
      }
    }
  }
}

// -----------------------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.
// -----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t* __restrict__ keys,
                                                                  const uint64_t* __restrict__ m_eff, int shift,
                                                                  int64_t n_tiles, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t m = (int64_t)*m_eff;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < m) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];  // digit-major
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint64_t* __restrict__ keys_in,
                                                                     const uint32_t* __restrict__ vals_in,
                                                                     const uint64_t* __restrict__ m_eff, int shift,
                                                                     int64_t n_tiles, const uint32_t* __restrict__ hist_scan,
                                                                     uint64_t* __restrict__ keys_out,
                                                                     uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t dig_base[256];
  __shared__ uint32_t warp_cnt[kSortThreads / 32][257];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t m = (int64_t)*m_eff;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= m) return;  // uniform per block
  dig_base[threadIdx.x] = hist_scan[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) warp_cnt[w][threadIdx.x] = 0;
  if (threadIdx.x < kSortThreads / 32) warp_cnt[threadIdx.x][256] = 0;
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * kSortThreads + threadIdx.x;
    const bool valid = i < m;
    uint64_t key = 0;
    uint32_t val = 0, d = 256;
    if (valid) {
      key = keys_in[i];
      val = vals_in[i];
      d = (uint32_t)(key >> shift) & 0xffu;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt);
    if (rank == 0) warp_cnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = dig_base[d] + rank;
      for (int w = 0; w < warp; ++w) pos += warp_cnt[w][d];
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
    {
      uint32_t tot = 0;
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; ++w) {
        tot += warp_cnt[w][threadIdx.x];
        warp_cnt[w][threadIdx.x] = 0;
      }
      dig_base[threadIdx.x] += tot;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) tile_ranges_kernel(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ m_eff,
                                                          int64_t total_tiles, uint32_t* __restrict__ ranges) {
  const int64_t m = (int64_t)*m_eff;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t t = keys[i] >> 32;
    if (t >= (uint64_t)total_tiles) continue;
    if (i == 0 || (keys[i - 1] >> 32) != t) ranges[2 * t] = (uint32_t)i;
    if (i == m - 1 || (keys[i + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(i + 1);
  }
}

int bits_for(int64_t x) {  // bits needed to represent values in [0, x)
  int b = 1;
  while (b < 63 && (int64_t(1) << b) < x) ++b;
  return b;
}

struct SortLayout {
  int64_t n_vk, scan_words, tiles_cap, hist_n, hist_scan_words;
  size_t off_scan, off_total, off_meff, off_keys_alt, off_vals_alt, off_hist, off_hist_scan, bytes;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

SortLayout sort_layout(int64_t n, int32_t n_views, int64_t capacity) {
  SortLayout L{};
  L.n_vk = n * (int64_t)n_views;
  L.scan_words = scan_ws_words(L.n_vk > 0 ? L.n_vk : 1);
  L.tiles_cap = ceil_div(capacity > 0 ? capacity : 1, kSortTile);
  L.hist_n = 256 * L.tiles_cap;
  L.hist_scan_words = scan_ws_words(L.hist_n);
  size_t o = 0;
  L.off_scan = o; o = align_up(o + sizeof(uint64_t) * L.scan_words);
  L.off_total = o; o = align_up(o + 2 * sizeof(uint64_t));
  L.off_meff = o; o = align_up(o + sizeof(uint64_t));
  L.off_keys_alt = o; o = align_up(o + sizeof(uint64_t) * (size_t)capacity);
  L.off_vals_alt = o; o = align_up(o + sizeof(uint32_t) * (size_t)capacity);
  L.off_hist = o; o = align_up(o + sizeof(uint32_t) * (size_t)L.hist_n);
  L.off_hist_scan = o; o = align_up(o + sizeof(uint64_t) * (size_t)L.hist_scan_words);
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

extern "C" potr_status potr_bin_sort(const potr_views* views, const potr_frame* frame, const potr_raster_config* cfg,
                                     int64_t n, int64_t instance_capacity, uint64_t* d_keys, uint32_t* d_vals,
                                     uint32_t* d_tile_ranges, potr_device_status* d_status, void* d_ws, size_t ws_bytes,
                                     potr_stream_t stream) {
  using namespace potr;
  if (!views || !frame || !cfg || !d_keys || !d_vals || !d_tile_ranges || !d_ws) return POTR_ERR_INVALID_ARGUMENT;
  if (n <= 0 || frame->n_views < 1 || frame->total_tiles <= 0 || !frame->info) return POTR_ERR_INVALID_ARGUMENT;
  if (instance_capacity <= 0 || instance_capacity > (int64_t)0xffffffffll) return POTR_ERR_INVALID_ARGUMENT;
  if (!views->touched || !views->offsets || !views->rect || !views->depth || !views->raster || !views->n_instances)
    return POTR_ERR_INVALID_ARGUMENT;
  const SortLayout L = sort_layout(n, frame->n_views, instance_capacity);
  if (ws_bytes < L.bytes) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  uint64_t* scan_ws = reinterpret_cast<uint64_t*>(ws + L.off_scan);
  uint64_t* total = reinterpret_cast<uint64_t*>(ws + L.off_total);
  uint64_t* m_eff = reinterpret_cast<uint64_t*>(ws + L.off_meff);
  uint64_t* keys_alt = reinterpret_cast<uint64_t*>(ws + L.off_keys_alt);
  uint32_t* vals_alt = reinterpret_cast<uint32_t*>(ws + L.off_vals_alt);
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.off_hist);
  uint64_t* hist_scan_ws = reinterpret_cast<uint64_t*>(ws + L.off_hist_scan);

  if (scan_exclusive<uint32_t, uint32_t>(views->touched, views->offsets, L.n_vk, total, scan_ws, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  count_check_kernel<<<1, 1, 0, s>>>(total, instance_capacity, views->n_instances, m_eff, d_status);
  POTR_CHECK_LAUNCH();

  const int key_bits = 32 + bits_for(frame->total_tiles);
  const int passes = (key_bits + 7) / 8;
  // emit into the buffer that makes the last pass land in d_keys / d_vals
  uint64_t* k_src = (passes & 1) ? keys_alt : d_keys;
  uint32_t* v_src = (passes & 1) ? vals_alt : d_vals;
  uint64_t* k_dst = (passes & 1) ? d_keys : keys_alt;
  uint32_t* v_dst = (passes & 1) ? d_vals : vals_alt;
  {
    const int64_t g = ceil_div(L.n_vk, 256);
    emit_kernel<<<(unsigned)(g < 152 * 64 ? g : 152 * 64), 256, 0, s>>>(
        views->touched, views->offsets, reinterpret_cast<const uint2*>(views->rect), views->depth, frame->info, n, L.n_vk,
        m_eff, reinterpret_cast<float4*>(views->raster), k_src, v_src);
    POTR_CHECK_LAUNCH();
  }
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    radix_hist_kernel<<<(unsigned)L.tiles_cap, kSortThreads, 0, s>>>(k_src, m_eff, shift, L.tiles_cap, hist);
    POTR_CHECK_LAUNCH();
    if (scan_exclusive<uint32_t, uint32_t>(hist, hist, L.hist_n, total + 1, hist_scan_ws, s) != cudaSuccess)
      return POTR_ERR_CUDA;
    radix_scatter_kernel<<<(unsigned)L.tiles_cap, kSortThreads, 0, s>>>(k_src, v_src, m_eff, shift, L.tiles_cap, hist,
                                                                        k_dst, v_dst);
    POTR_CHECK_LAUNCH();
    uint64_t* tk = k_src; k_src = k_dst; k_dst = tk;
    uint32_t* tv = v_src; v_src = v_dst; v_dst = tv;
  }
  if (cudaMemsetAsync(d_tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)frame->total_tiles, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  {
    const int64_t g = ceil_div(instance_capacity, 256);
    tile_ranges_kernel<<<(unsigned)(g < 152 * 64 ? g : 152 * 64), 256, 0, s>>>(d_keys, m_eff, frame->total_tiles,
                                                                               d_tile_ranges);
    POTR_CHECK_LAUNCH();
  }
  return POTR_OK;
}
