// codec_decode.cu -- the POTR decoder's device part (Section IV-E, inverted): splat positions
// from the depth-first node bytes and the shared-leaf table, attributes dequantised.
//
// Parallel parse of a pre-order tree.  With c_j the number of set bits of node j's byte (its
// children), e_i = sum_{j<i} (c_j - 1) counts the subtrees still pending, besides node i's own,
// when node i is met; a well-formed stream has 0 <= e_i <= 7 D for every node and ends with
// e_m = -1.  Node i's parent is the last j < i with e_j <= e_i (found by a backward search
// inside blocks of 1024 nodes, else from a per-level table of the last such position before the
// block), and node i is child number e_j + c_j - 1 - e_i of it, i.e. the octant of that set bit
// of the parent's byte.  A leaf (byte 0) walks up to the root (at most D steps) to get its cell
// and depth; its splats start at its leaf ordinal plus the extra splats of the table entries
// before it.  Malformed input is reported through the status word (POTR_ERR_CORRUPT) and never
// indexes outside the buffers.
#include "codec_common.cuh"
#include "scan.cuh"

namespace potr {
namespace {

constexpr int kMaxPending = 7 * kDepth;  // e_i <= 7 D: at most 7 pending siblings per level
constexpr int kELevels = kMaxPending + 1;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// Packed per node: its child count (low word) and whether it is a leaf (high word).
__global__ void __launch_bounds__(256) dec_flags_kernel(int64_t m, const uint8_t* __restrict__ nodes,
                                                        uint64_t* __restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = nodes[i];
    flags[i] = (uint64_t)__popc(b) | ((uint64_t)(b == 0) << 32);
  }
}

// e_i = (children before i) - i, checked; the block's last position with e == v for every v,
// turned into the last position with e <= t for every threshold t.
__global__ void __launch_bounds__(256) dec_pending_kernel(int64_t m, const uint64_t* __restrict__ excl,
                                                          const uint64_t* __restrict__ total, uint8_t* __restrict__ e,
                                                          int* __restrict__ last, potr_device_status* st) {
  __shared__ int s[kELevels];
  for (int v = threadIdx.x; v < kELevels; v += blockDim.x) s[v] = -1;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kChunkCodec;
  for (int j = threadIdx.x; j < kChunkCodec; j += blockDim.x) {
    const int64_t i = base + j;
    if (i >= m) break;
    const int64_t ei = (int64_t)(uint32_t)excl[i] - i;
    if (ei < 0 || ei > kMaxPending) {
      set_status(st, POTR_ERR_CORRUPT, 0);
      e[i] = 0xff;
      continue;
    }
    e[i] = (uint8_t)ei;
    atomicMax(&s[ei], (int)i);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (uint32_t)*total != (uint32_t)(m - 1))
    set_status(st, POTR_ERR_CORRUPT, 0);  // the children must number m - 1 (every node but the root)
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = -1;
    for (int t = 0; t < kELevels; ++t) {
      run = max(run, s[t]);
      last[blockIdx.x * kELevels + t] = run;
    }
  }
}

__device__ __forceinline__ int nth_set_bit(uint32_t b, int r) {  // position of the r-th set bit (r >= 0)
  for (int k = 0; k < r; ++k) b &= b - 1;
  return b ? __ffs(b) - 1 : -1;
}

// Parent and octant of every node but the root; one block per 1024 nodes, e staged in shared
// memory for the backward search.
__global__ void __launch_bounds__(256) dec_parent_kernel(int64_t m, const uint8_t* __restrict__ nodes,
                                                         const uint8_t* __restrict__ e,
                                                         const int* __restrict__ prefix_last,
                                                         uint32_t* __restrict__ parent, uint8_t* __restrict__ octant,
                                                         potr_device_status* st) {
  __shared__ uint8_t se[kChunkCodec];
  const int64_t base = (int64_t)blockIdx.x * kChunkCodec;
  for (int j = threadIdx.x; j < kChunkCodec; j += blockDim.x) se[j] = base + j < m ? e[base + j] : 0xff;
  __syncthreads();
  for (int j = threadIdx.x; j < kChunkCodec; j += blockDim.x) {
    const int64_t i = base + j;
    if (i >= m) break;
    if (i == 0) {
      parent[0] = 0;
      octant[0] = 0;
      continue;
    }
    const int ei = se[j];
    if (ei > kMaxPending) {  // reported by dec_pending_kernel
      parent[i] = 0;
      octant[i] = 0xff;
      continue;
    }
    int k = j - 1;
    while (k >= 0 && se[k] > ei) --k;
    const int64_t p = k >= 0 ? base + k : (int64_t)prefix_last[blockIdx.x * (int64_t)kELevels + ei];
    const uint32_t bp = p >= 0 ? nodes[p] : 0u;
    const int r = p >= 0 ? (int)e[p] + __popc(bp) - 1 - ei : -1;
    const int oct = (r >= 0 && r < __popc(bp)) ? nth_set_bit(bp, r) : -1;
    if (oct < 0) {
      set_status(st, POTR_ERR_CORRUPT, 0);
      parent[i] = 0;
      octant[i] = 0xff;
      continue;
    }
    parent[i] = (uint32_t)p;
    octant[i] = (uint8_t)oct;
  }
}

// The table's extra splats as an array of counts (for the scan), its ordinals checked.
__global__ void __launch_bounds__(256) dec_dup_counts_kernel(int64_t n_dups, const uint32_t* __restrict__ dups,
                                                             const uint64_t* __restrict__ leaf_total,
                                                             uint32_t* __restrict__ extra, potr_device_status* st) {
  const uint32_t n_leaves = (uint32_t)(*leaf_total >> 32);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_dups; t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t ord = dups[2 * t], cnt = dups[2 * t + 1];
    if (ord >= n_leaves || cnt == 0 || (t > 0 && dups[2 * (t - 1)] >= ord)) set_status(st, POTR_ERR_CORRUPT, 0);
    extra[t] = cnt;
  }
}

// Every leaf: its cell and depth (walking up), then the centre written for each of its splats.
__global__ void __launch_bounds__(256) dec_leaf_kernel(int64_t m, int64_t n, const uint64_t* __restrict__ excl,
                                                       const uint8_t* __restrict__ nodes,
                                                       const uint32_t* __restrict__ parent,
                                                       const uint8_t* __restrict__ octant,
                                                       const uint32_t* __restrict__ dups, int64_t n_dups,
                                                       const uint32_t* __restrict__ extra_excl, Cube cube,
                                                       float* __restrict__ means, potr_device_status* st) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (nodes[i] != 0) continue;
    const uint32_t ord = (uint32_t)(excl[i] >> 32);
    // table entries with a smaller ordinal (binary search over the sorted ordinals)
    int64_t lo = 0, hi = n_dups;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (dups[2 * mid] < ord) lo = mid + 1;
      else hi = mid;
    }
    const int64_t first = (int64_t)ord + (lo > 0 ? (int64_t)extra_excl[lo - 1] + dups[2 * (lo - 1) + 1] : 0);
    const int64_t mult = 1 + (lo < n_dups && dups[2 * lo] == ord ? (int64_t)dups[2 * lo + 1] : 0);
    uint32_t X = 0, Y = 0, Z = 0;
    int d = 0;
    int64_t k = i;
    bool ok = true;
    while (k != 0) {
      const uint32_t oc = octant[k];
      if (oc > 7 || d >= kDepth) {
        ok = false;
        break;
      }
      X |= ((oc >> 2) & 1u) << d;
      Y |= ((oc >> 1) & 1u) << d;
      Z |= (oc & 1u) << d;
      ++d;
      k = parent[k];
    }
    if (!ok || first + mult > n) {
      set_status(st, POTR_ERR_CORRUPT, 0);
      continue;
    }
    const float x = (float)cell_centre(cube.corner[0], cube.S, X, d);
    const float y = (float)cell_centre(cube.corner[1], cube.S, Y, d);
    const float z = (float)cell_centre(cube.corner[2], cube.S, Z, d);
    for (int64_t s = first; s < first + mult; ++s) {
      means[s] = x;
      means[n + s] = y;
      means[2 * n + s] = z;
    }
  }
}

// Leaves plus the table's extra splats must number n.
__global__ void dec_count_check_kernel(const uint64_t* __restrict__ leaf_total, const uint64_t* __restrict__ extra_total,
                                       int64_t n_dups, int64_t n, potr_device_status* st) {
  const uint64_t leaves = *leaf_total >> 32;
  const uint64_t extra = n_dups > 0 ? *extra_total : 0;
  if (leaves + extra != (uint64_t)n) set_status(st, POTR_ERR_CORRUPT, 0);
}

// Attributes in stream order: x~ = x^ / SF (opacity (x^ + 1/4) / SF, clamped to [1e-6, 1 - 1e-6]
// and stored as its logit), the quaternion's w = sqrt(max(0, 1 - x^2 - y^2 - z^2)), the DC
// coefficients from the running sums of their differences (dc_excl: exclusive sums over the three
// DC planes laid end to end).
__global__ void __launch_bounds__(256) dec_attr_kernel(int64_t n, const int32_t* __restrict__ attrs,
                                                       const int32_t* __restrict__ dc_excl, double sf_scale,
                                                       double sf_rot, double sf_op, double sf_sh,
                                                       float* __restrict__ log_scales, float* __restrict__ quats,
                                                       float* __restrict__ logits, float* __restrict__ sh) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; ++a) log_scales[a * n + i] = (float)__ddiv_rn((double)attrs[a * n + i], sf_scale);
    const double x = __ddiv_rn((double)attrs[3 * n + i], sf_rot);
    const double y = __ddiv_rn((double)attrs[4 * n + i], sf_rot);
    const double z = __ddiv_rn((double)attrs[5 * n + i], sf_rot);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
    quats[i] = (float)__dsqrt_rn(fmax(0.0, __dsub_rn(1.0, r2)));
    quats[n + i] = (float)x;
    quats[2 * n + i] = (float)y;
    quats[3 * n + i] = (float)z;
    double o = __ddiv_rn(__dadd_rn((double)attrs[6 * n + i], 0.25), sf_op);
    o = fmin(fmax(o, 1e-6), 1.0 - 1e-6);
    logits[i] = (float)log(__ddiv_rn(o, __dsub_rn(1.0, o)));
    for (int c = 0; c < 48; ++c) {
      int32_t q = attrs[(7 + c) * n + i];
      if (c < 3) q = (int32_t)((uint32_t)dc_excl[c * n + i] + (uint32_t)q - (uint32_t)dc_excl[c * n]);
      sh[c * n + i] = (float)__ddiv_rn((double)q, sf_sh);
    }
  }
}

struct DecodeLayout {
  size_t flags, excl, e, parent, octant, chunk, extra, extra_excl, dc_excl, scan, totals, bytes;
  int64_t n_chunks;
};

DecodeLayout decode_layout(int64_t m, int64_t n) {
  DecodeLayout L{};
  L.n_chunks = cdiv(m, kChunkCodec);
  const int64_t big = m > 3 * n ? m : 3 * n;
  size_t o = 0;
  L.flags = o; o = al(o + 8 * (size_t)m);
  L.excl = o; o = al(o + 8 * (size_t)m);
  L.e = o; o = al(o + (size_t)m);
  L.parent = o; o = al(o + 4 * (size_t)m);
  L.octant = o; o = al(o + (size_t)m);
  L.chunk = o; o = al(o + 4 * (size_t)L.n_chunks * kELevels);
  L.extra = o; o = al(o + 4 * (size_t)(n / 2 + 1));
  L.extra_excl = o; o = al(o + 4 * (size_t)(n / 2 + 1));
  L.dc_excl = o; o = al(o + 4 * 3 * (size_t)n);
  L.scan = o; o = al(o + 8 * (size_t)scan_ws_words(big));
  L.totals = o; o = al(o + 8 * 4);
  L.bytes = o;
  return L;
}

}  // namespace
}  // namespace potr

extern "C" size_t potr_codec_decode_workspace_size(int64_t n_nodes, int64_t n) {
  if (n_nodes <= 0 || n <= 0) return 0;
  return potr::decode_layout(n_nodes, n).bytes;
}

extern "C" potr_status potr_codec_decode(const uint8_t* d_nodes, int64_t n_nodes, const uint32_t* d_dups,
                                         int64_t n_dups, const int32_t* d_attrs, int64_t n, const double* cube,
                                         const potr_codec_params* params, const potr_scene_grads* out,
                                         potr_device_status* d_status, void* d_ws, size_t ws_bytes,
                                         potr_stream_t stream) {
  using namespace potr;
  if (!d_nodes || !d_attrs || !cube || !params || !out || !d_ws || (n_dups > 0 && !d_dups))
    return POTR_ERR_INVALID_ARGUMENT;
  if (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh)
    return POTR_ERR_INVALID_ARGUMENT;
  if (n_nodes <= 0 || n <= 0 || n_dups < 0 || n_dups > n / 2) return POTR_ERR_INVALID_ARGUMENT;
  if (n_nodes > (int64_t)0x7fffffff || n > (int64_t)0x7fffffff / 55) return POTR_ERR_UNSUPPORTED;
  if (!(params->sf_scale > 0.0 && params->sf_rotation > 0.0 && params->sf_opacity > 0.0 && params->sf_sh > 0.0) ||
      !(cube[3] > 0.0))
    return POTR_ERR_INVALID_ARGUMENT;
  const DecodeLayout L = decode_layout(n_nodes, n);
  if (ws_bytes < L.bytes) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  uint64_t *flags = reinterpret_cast<uint64_t*>(ws + L.flags), *excl = reinterpret_cast<uint64_t*>(ws + L.excl);
  uint8_t* e = reinterpret_cast<uint8_t*>(ws + L.e);
  uint32_t* parent = reinterpret_cast<uint32_t*>(ws + L.parent);
  uint8_t* octant = reinterpret_cast<uint8_t*>(ws + L.octant);
  int* chunk = reinterpret_cast<int*>(ws + L.chunk);
  uint32_t *extra = reinterpret_cast<uint32_t*>(ws + L.extra), *extra_excl = reinterpret_cast<uint32_t*>(ws + L.extra_excl);
  int32_t* dc_excl = reinterpret_cast<int32_t*>(ws + L.dc_excl);
  uint64_t* scan_ws = reinterpret_cast<uint64_t*>(ws + L.scan);
  uint64_t* totals = reinterpret_cast<uint64_t*>(ws + L.totals);
  const Cube cb{{cube[0], cube[1], cube[2]}, cube[3]};
  auto grid = [](int64_t k) { return (unsigned)(cdiv(k, 256) < 152 * 16 ? cdiv(k, 256) : 152 * 16); };

  // tree structure
  dec_flags_kernel<<<grid(n_nodes), 256, 0, s>>>(n_nodes, d_nodes, flags);
  POTR_CHECK_LAUNCH();
  if (scan_exclusive<uint64_t, uint64_t>(flags, excl, n_nodes, totals, scan_ws, s) != cudaSuccess) return POTR_ERR_CUDA;
  dec_pending_kernel<<<(unsigned)L.n_chunks, 256, 0, s>>>(n_nodes, excl, totals, e, chunk, d_status);
  POTR_CHECK_LAUNCH();
  prefix_max_columns_kernel<<<kELevels, 256, 0, s>>>(L.n_chunks, kELevels, chunk);
  POTR_CHECK_LAUNCH();
  dec_parent_kernel<<<(unsigned)L.n_chunks, 256, 0, s>>>(n_nodes, d_nodes, e, chunk, parent, octant, d_status);
  POTR_CHECK_LAUNCH();
  // shared leaves, then every leaf's position
  if (n_dups > 0) {
    dec_dup_counts_kernel<<<grid(n_dups), 256, 0, s>>>(n_dups, d_dups, totals, extra, d_status);
    POTR_CHECK_LAUNCH();
    if (scan_exclusive<uint32_t, uint32_t>(extra, extra_excl, n_dups, totals + 1, scan_ws, s) != cudaSuccess)
      return POTR_ERR_CUDA;
  }
  dec_count_check_kernel<<<1, 1, 0, s>>>(totals, totals + 1, n_dups, n, d_status);
  POTR_CHECK_LAUNCH();
  dec_leaf_kernel<<<grid(n_nodes), 256, 0, s>>>(n_nodes, n, excl, d_nodes, parent, octant, d_dups, n_dups, extra_excl,
                                                cb, out->means, d_status);
  POTR_CHECK_LAUNCH();
  // attributes
  if (scan_exclusive<int32_t, int32_t>(d_attrs + 7 * n, dc_excl, 3 * n, totals + 2, scan_ws, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  dec_attr_kernel<<<grid(n), 256, 0, s>>>(n, d_attrs, dc_excl, params->sf_scale, params->sf_rotation,
                                          params->sf_opacity, params->sf_sh, out->log_scales, out->quats,
                                          out->opacity_logits, out->sh);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
