// codec.cu -- the POTR encoder's device part (Section IV-E): the octree of the splat positions
// under the precision criterion, its depth-first node bytes, and the uniformly quantised
// attributes in the order of that traversal.
//
// Octree without recursion.  Positions map to integer cells at the depth limit D = 21 and to
// their 63-bit cell codes (3 bits per level, x bit high); the splats are radix-sorted by code
// (stable: ties keep index order), which is the depth-first leaf order.  With L_i the number
// of leading levels splat i shares with splat i - 1 (-1 for the first), a splat's cell holds
// no other splat from depth max(L_i, L_{i+1}) + 1 on, so its leaf is the first depth from
// there whose cell centre passes the precision test (depth D at most).  Splat i then
// introduces the nodes of its path below depth L_i -- internal nodes at depths L_i + 1 ..
// D_i - 1 and its leaf -- in exactly the order a depth-first traversal meets them, so a scan
// of those counts gives every node's byte offset.  An internal node's byte is the OR of its
// children's octants: each splat sets its own nodes' bits, and the one bit it adds to the node
// at depth L_i it shares with earlier splats goes to the node created by the last splat j < i
// with L_j < L_i (found by a backward search inside blocks of 1024 splats and a per-level
// running maximum over blocks).  Every leaf writes 0; a depth-D leaf that holds several
// (coincident) splats goes into a table of (leaf ordinal, count - 1) pairs, compacted with one
// scan of packed (leaf, shared-leaf) flags.
#include "codec_common.cuh"
#include "radix.cuh"
#include "scan.cuh"

namespace potr {
namespace {

__device__ __forceinline__ double atomic_min_d(double* a, double v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
  unsigned long long old = *p;
  while (v < __longlong_as_double((long long)old)) {
    const unsigned long long prev = atomicCAS(p, old, (unsigned long long)__double_as_longlong(v));
    if (prev == old) break;
    old = prev;
  }
  return __longlong_as_double((long long)old);
}

__device__ __forceinline__ double atomic_max_d(double* a, double v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
  unsigned long long old = *p;
  while (v > __longlong_as_double((long long)old)) {
    const unsigned long long prev = atomicCAS(p, old, (unsigned long long)__double_as_longlong(v));
    if (prev == old) break;
    old = prev;
  }
  return __longlong_as_double((long long)old);
}

// Per-axis min and max of the positions (mm[0..2] min, mm[3..5] max; binary64 of the floats).
__global__ void __launch_bounds__(256) codec_bounds_kernel(int64_t n, const float* __restrict__ means,
                                                           double* __restrict__ mm) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double x = means[a * n + k];
      lo[a] = fmin(lo[a], x);
      hi[a] = fmax(hi[a], x);
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
    for (int o = 16; o >= 1; o >>= 1) {
      lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; ++a) {
      atomic_min_d(&mm[a], lo[a]);
      atomic_max_d(&mm[3 + a], hi[a]);
    }
}

__global__ void codec_cube_kernel(const double* __restrict__ mm, Cube* cube) {
  double S = 0.0;
  for (int a = 0; a < 3; ++a) {
    cube->corner[a] = mm[a];
    S = fmax(S, __dsub_rn(mm[3 + a], mm[a]));
  }
  cube->S = S > 0.0 ? S : 1.0;
}

__device__ __forceinline__ uint32_t cell_of(double x, double corner, double S) {
  // floor((x - corner) / S * 2^D), clamped to [0, 2^D - 1]
  const double f = floor(__dmul_rn(__ddiv_rn(__dsub_rn(x, corner), S), (double)(1 << kDepth)));
  return f < 0.0 ? 0u : (f > (double)((1 << kDepth) - 1) ? (uint32_t)((1 << kDepth) - 1) : (uint32_t)f);
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {  // bit b of v -> bit 3b
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// Cell codes (split into 32-bit halves for the sort) and the precision tolerance of every splat.
__global__ void __launch_bounds__(256) codec_codes_kernel(int64_t n, const float* __restrict__ means,
                                                          const Cube* __restrict__ cube,
                                                          const double* __restrict__ eyes, int n_eyes, double beta,
                                                          double gamma, uint32_t* __restrict__ code_lo,
                                                          uint32_t* __restrict__ code_hi,
                                                          double* __restrict__ tol) {
  const Cube c = *cube;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double x = means[k], y = means[n + k], z = means[2 * n + k];
    const uint64_t code = (spread3(cell_of(x, c.corner[0], c.S)) << 2) | (spread3(cell_of(y, c.corner[1], c.S)) << 1) |
                          spread3(cell_of(z, c.corner[2], c.S));
    code_lo[k] = (uint32_t)code;
    code_hi[k] = (uint32_t)(code >> 32);
    double dmin = INFINITY;
    for (int e = 0; e < n_eyes; ++e) {
      const double dx = __dsub_rn(x, eyes[3 * e]), dy = __dsub_rn(y, eyes[3 * e + 1]), dz = __dsub_rn(z, eyes[3 * e + 2]);
      const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
      dmin = fmin(dmin, d);
    }
    tol[k] = fmax(gamma, __dmul_rn(beta, dmin));
  }
}

__device__ __forceinline__ uint32_t compact3(uint64_t x) {  // bit 3b of x -> bit b (21 bits)
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x | (x >> 4)) & 0x100f00f00f00f00full;
  x = (x | (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x | (x >> 16)) & 0x1f00000000ffffull;
  x = (x | (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

__global__ void __launch_bounds__(256) gather_u32_kernel(int64_t n, const uint32_t* __restrict__ src,
                                                         const uint32_t* __restrict__ idx, uint32_t* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

__global__ void __launch_bounds__(256) radix_hist_kernel(int64_t n, const uint32_t* __restrict__ keys,
                                                         uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[4][256];
  for (int p = 0; p < 4; ++p) h[p][threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
#pragma unroll
    for (int p = 0; p < 4; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int p = 0; p < 4; ++p)
    if (h[p][threadIdx.x]) atomicAdd(&ghist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

__device__ __forceinline__ int lcp_levels(uint64_t a, uint64_t b) {
  const uint64_t x = a ^ b;
  if (x == 0) return kDepth;
  return (__clzll((long long)x) - 1) / 3;  // codes use the low 63 bits
}

__device__ __forceinline__ uint64_t code_at(const uint32_t* lo, const uint32_t* hi, int64_t i) {
  return ((uint64_t)hi[i] << 32) | lo[i];
}

__device__ __forceinline__ uint32_t digit_at(uint64_t code, int d) {  // octant of level d (0 = top)
  return (uint32_t)(code >> (3 * (kDepth - 1 - d))) & 7u;
}

// Per sorted position: L (shared levels with the predecessor), leaf depth, new node count.
__global__ void __launch_bounds__(256) codec_depth_kernel(int64_t n, const uint32_t* __restrict__ lo,
                                                          const uint32_t* __restrict__ hi,
                                                          const uint32_t* __restrict__ order,
                                                          const float* __restrict__ means,
                                                          const Cube* __restrict__ cube,
                                                          const double* __restrict__ tol, int8_t* __restrict__ Lout,
                                                          int8_t* __restrict__ Dout, uint32_t* __restrict__ cnt) {
  const Cube c = *cube;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t code = code_at(lo, hi, i);
    const int L = i > 0 ? lcp_levels(code_at(lo, hi, i - 1), code) : -1;
    const int R = i + 1 < n ? lcp_levels(code_at(lo, hi, i + 1), code) : -1;
    const int k = (int)order[i];
    const double mx = means[k], my = means[n + k], mz = means[2 * n + k];
    const double t = tol[k];
    int d = min(max(L, R) + 1, kDepth);
    const uint32_t X = compact3(code >> 2), Y = compact3(code >> 1), Z = compact3(code);
    for (; d < kDepth; ++d) {
      const int sh = kDepth - d;  // cell at depth d = full-depth cell >> (D - d)
      const double px = cell_centre(c.corner[0], c.S, X >> sh, d);
      const double py = cell_centre(c.corner[1], c.S, Y >> sh, d);
      const double pz = cell_centre(c.corner[2], c.S, Z >> sh, d);
      const double ddx = __dsub_rn(mx, px), ddy = __dsub_rn(my, py), ddz = __dsub_rn(mz, pz);
      const double dist = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz)));
      if (dist < t) break;
    }
    Lout[i] = (int8_t)L;
    Dout[i] = (int8_t)d;
    cnt[i] = L == kDepth ? 0u : (uint32_t)(d - 1 - L + 1);  // internal nodes L+1 .. d-1, then the leaf
  }
}

// Per block of kChunkCodec sorted positions: the last position with L < t, for every level t.
__global__ void __launch_bounds__(256) codec_chunk_last_kernel(int64_t n, const int8_t* __restrict__ L,
                                                               int* __restrict__ last) {
  __shared__ int s[kLevels + 1];  // s[l + 1]: last position with L == l (l = -1 .. D)
  if (threadIdx.x <= kLevels) s[threadIdx.x] = -1;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kChunkCodec;
  for (int j = threadIdx.x; j < kChunkCodec; j += blockDim.x) {
    const int64_t i = base + j;
    if (i < n) atomicMax(&s[L[i] + 1], (int)i);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = -1;
    for (int t = 0; t < kLevels; ++t) {  // L < t  <=>  L in -1 .. t - 1
      run = max(run, s[t]);
      last[blockIdx.x * kLevels + t] = run;
    }
  }
}

// Node bytes: every splat sets the octant bits of its own internal nodes (its leaf stays 0) and
// the bit it adds to the node at depth L_i created by an earlier splat.
__global__ void __launch_bounds__(256) codec_nodes_kernel(int64_t n, const uint32_t* __restrict__ lo,
                                                          const uint32_t* __restrict__ hi, const int8_t* __restrict__ L,
                                                          const int8_t* __restrict__ D, const uint32_t* __restrict__ off,
                                                          const int* __restrict__ prefix_last,
                                                          uint32_t* __restrict__ node) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int li = L[i];
    if (li == kDepth) continue;  // shares a depth-limit leaf with its predecessor
    const int di = D[i];
    const uint64_t code = code_at(lo, hi, i);
    const uint32_t o = off[i];
    for (int d = li + 1; d < di; ++d) atomicOr(&node[o + (d - li - 1)], 1u << digit_at(code, d));
    if (li >= 0) {
      // the node at depth li on this path: created by the last j < i with L_j < li
      int64_t j = i - 1;
      const int64_t start = (i / kChunkCodec) * kChunkCodec;
      while (j >= start && L[j] >= li) --j;
      if (j < start) j = prefix_last[(i / kChunkCodec) * kLevels + li];
      const uint32_t id = off[j] + (uint32_t)(li - L[j] - 1);
      atomicOr(&node[id], 1u << digit_at(code, li));
    }
  }
}

// Per sorted position: bit 0 -- it opens a leaf (it shares no depth-limit cell with its
// predecessor); bit 32 -- that leaf is at the depth limit and the next splat shares it.
__global__ void __launch_bounds__(256) codec_leaf_flags_kernel(int64_t n, const int8_t* __restrict__ L,
                                                               const int8_t* __restrict__ D,
                                                               uint64_t* __restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool opens = L[i] != kDepth;
    const bool shared = opens && D[i] == kDepth && i + 1 < n && L[i + 1] == kDepth;
    flags[i] = (uint64_t)opens | ((uint64_t)shared << 32);
  }
}

// The shared-leaf table: (leaf ordinal, splat count - 1) at the slot the packed scan gives.
__global__ void __launch_bounds__(256) codec_dups_kernel(int64_t n, const int8_t* __restrict__ L,
                                                         const uint64_t* __restrict__ flags,
                                                         const uint64_t* __restrict__ excl,
                                                         uint32_t* __restrict__ dups) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!(flags[i] >> 32)) continue;
    int64_t j = i + 1;
    while (j < n && L[j] == kDepth) ++j;
    const uint64_t e = excl[i];
    const uint32_t slot = (uint32_t)(e >> 32);
    dups[2 * (size_t)slot] = (uint32_t)e;
    dups[2 * (size_t)slot + 1] = (uint32_t)(j - i - 1);
  }
}

__global__ void store_high_word_kernel(const uint64_t* __restrict__ total, uint32_t* __restrict__ out) {
  *out = (uint32_t)(*total >> 32);
}

__global__ void __launch_bounds__(256) pack_bytes_kernel(const uint32_t* __restrict__ total, const uint32_t* __restrict__ node,
                                                         uint8_t* __restrict__ out) {
  const uint32_t m = *total;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) out[i] = (uint8_t)node[i];
}

__device__ __forceinline__ int32_t quant(double x, double sf) { return (int32_t)floor(__dadd_rn(0.5, __dmul_rn(x, sf))); }

// Attributes in stream order, property after property: 3 log-scales, 3 rotation (x, y, z of the
// normalised quaternion with w >= 0), opacity (sigmoid of the logit), 48 SH values (DC as
// differences from the previous splat in stream order).
__global__ void __launch_bounds__(256) codec_attr_kernel(int64_t n, const uint32_t* __restrict__ order,
                                                         const float* __restrict__ log_scales,
                                                         const float* __restrict__ quats,
                                                         const float* __restrict__ logits, const float* __restrict__ sh,
                                                         double sf_scale, double sf_rot, double sf_op, double sf_sh,
                                                         int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = order[i];
    for (int a = 0; a < 3; ++a) out[a * n + i] = quant((double)log_scales[a * n + k], sf_scale);
    const double qw = quats[k], qx = quats[n + k], qy = quats[2 * n + k], qz = quats[3 * n + k];
    const double nrm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(qw, qw), __dmul_rn(qx, qx)), __dmul_rn(qy, qy)),
                                            __dmul_rn(qz, qz)));
    const double sgn = __ddiv_rn(qw, nrm) < 0.0 ? -1.0 : 1.0;
    out[(3 + 0) * n + i] = quant(sgn * __ddiv_rn(qx, nrm), sf_rot);
    out[(3 + 1) * n + i] = quant(sgn * __ddiv_rn(qy, nrm), sf_rot);
    out[(3 + 2) * n + i] = quant(sgn * __ddiv_rn(qz, nrm), sf_rot);
    const double op = __ddiv_rn(1.0, __dadd_rn(1.0, exp(-(double)logits[k])));
    out[6 * n + i] = quant(op, sf_op);
    for (int c = 0; c < 48; ++c) {
      int32_t v = quant((double)sh[c * n + k], sf_sh);
      if (c < 3) v -= i > 0 ? quant((double)sh[c * n + order[i - 1]], sf_sh) : 0;
      out[(7 + c) * n + i] = v;
    }
  }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t al(size_t x) { return (x + 255) & ~size_t(255); }

struct CodecLayout {
  size_t mm, cube, lo, hi, lo2, hi2, v, v2, tol, L, D, cnt, off, scan, total, chunk, node, status, ghist, gbase,
      counter, flags, fscan, bytes;
  int64_t blocks, n_chunks;
};

int64_t scan_words_for(int64_t n) {  // the scan's partial sums: one u64 per chunk of 2048 at each level
  int64_t w = 0, m = n;
  do {
    m = cdiv(m, 2048);
    w += m;
  } while (m > 1);
  return w + 1;
}

CodecLayout codec_layout(int64_t n) {
  CodecLayout L{};
  L.blocks = cdiv(n, kOsTile);
  L.n_chunks = cdiv(n, kChunkCodec);
  size_t o = 0;
  L.mm = o; o = al(o + 6 * sizeof(double));
  L.cube = o; o = al(o + sizeof(Cube));
  L.lo = o; o = al(o + 4 * (size_t)n);
  L.hi = o; o = al(o + 4 * (size_t)n);
  L.lo2 = o; o = al(o + 4 * (size_t)n);
  L.hi2 = o; o = al(o + 4 * (size_t)n);
  L.v = o; o = al(o + 4 * (size_t)n);
  L.v2 = o; o = al(o + 4 * (size_t)n);
  L.tol = o; o = al(o + 8 * (size_t)n);
  L.L = o; o = al(o + (size_t)n);
  L.D = o; o = al(o + (size_t)n);
  L.cnt = o; o = al(o + 4 * (size_t)n);
  L.off = o; o = al(o + 4 * (size_t)n);
  L.scan = o; o = al(o + 8 * (size_t)scan_words_for(n));
  L.total = o; o = al(o + 16);
  L.chunk = o; o = al(o + 4 * (size_t)L.n_chunks * kLevels);
  L.node = o; o = al(o + 4 * (size_t)n * (kDepth + 1));
  L.status = o; o = al(o + 8 * 256 * (size_t)L.blocks);
  L.ghist = o; o = al(o + 4 * 256 * 8);
  L.gbase = o; o = al(o + 4 * 256 * 8);
  L.counter = o; o = al(o + 4 * 8);
  L.flags = o; o = al(o + 8 * (size_t)n);
  L.fscan = o; o = al(o + 8 * (size_t)n);
  L.bytes = o;
  return L;
}

}  // namespace
}  // namespace potr

extern "C" size_t potr_codec_workspace_size(int64_t n) {
  if (n <= 0) return 0;
  return potr::codec_layout(n).bytes;
}

extern "C" potr_status potr_codec_encode(const potr_scene* scene, const double* d_eyes, int32_t n_eyes,
                                         const potr_codec_params* params, uint8_t* d_nodes, uint32_t* d_n_nodes,
                                         uint32_t* d_dups, uint32_t* d_n_dups, uint32_t* d_order, int32_t* d_attrs, double* d_cube,
                                         potr_device_status* d_status, void* d_ws, size_t ws_bytes,
                                         potr_stream_t stream) {
  using namespace potr;
  if (!scene || !d_eyes || n_eyes < 1 || !params || !d_nodes || !d_n_nodes || !d_dups || !d_n_dups || !d_order ||
      !d_attrs || !d_ws)
    return POTR_ERR_INVALID_ARGUMENT;
  if (!scene->means || !scene->log_scales || !scene->quats || !scene->opacity_logits || !scene->sh)
    return POTR_ERR_INVALID_ARGUMENT;
  const int64_t n = scene->n;
  if (n <= 0 || n > (int64_t)(0x7fffffff / (kDepth + 1))) return POTR_ERR_UNSUPPORTED;
  const CodecLayout L = codec_layout(n);
  if (ws_bytes < L.bytes) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  double* mm = reinterpret_cast<double*>(ws + L.mm);
  Cube* cube = reinterpret_cast<Cube*>(ws + L.cube);
  uint32_t *lo = reinterpret_cast<uint32_t*>(ws + L.lo), *hi = reinterpret_cast<uint32_t*>(ws + L.hi);
  uint32_t *lo2 = reinterpret_cast<uint32_t*>(ws + L.lo2), *hi2 = reinterpret_cast<uint32_t*>(ws + L.hi2);
  uint32_t *v = reinterpret_cast<uint32_t*>(ws + L.v), *v2 = reinterpret_cast<uint32_t*>(ws + L.v2);
  double* tol = reinterpret_cast<double*>(ws + L.tol);
  int8_t *Ls = reinterpret_cast<int8_t*>(ws + L.L), *Ds = reinterpret_cast<int8_t*>(ws + L.D);
  uint32_t *cnt = reinterpret_cast<uint32_t*>(ws + L.cnt), *off = reinterpret_cast<uint32_t*>(ws + L.off);
  uint64_t* scan_ws = reinterpret_cast<uint64_t*>(ws + L.scan);
  uint64_t* total = reinterpret_cast<uint64_t*>(ws + L.total);
  int* chunk = reinterpret_cast<int*>(ws + L.chunk);
  uint32_t* node = reinterpret_cast<uint32_t*>(ws + L.node);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(ws + L.status);
  uint32_t* ghist = reinterpret_cast<uint32_t*>(ws + L.ghist);
  uint32_t* gbase = reinterpret_cast<uint32_t*>(ws + L.gbase);
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws + L.counter);
  uint64_t *flags = reinterpret_cast<uint64_t*>(ws + L.flags), *fscan = reinterpret_cast<uint64_t*>(ws + L.fscan);
  const int g = (int)(cdiv(n, 256) < 152 * 16 ? cdiv(n, 256) : 152 * 16);
  if (cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem_bytes()) !=
      cudaSuccess)
    return POTR_ERR_CUDA;

  // root cube, cell codes, tolerances
  const double init[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  if (cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess) return POTR_ERR_CUDA;
  codec_bounds_kernel<<<g, 256, 0, s>>>(n, scene->means, mm);
  POTR_CHECK_LAUNCH();
  codec_cube_kernel<<<1, 1, 0, s>>>(mm, cube);
  POTR_CHECK_LAUNCH();
  codec_codes_kernel<<<g, 256, 0, s>>>(n, scene->means, cube, d_eyes, n_eyes, params->beta, params->gamma, lo, hi,
                                       tol);
  POTR_CHECK_LAUNCH();

  // stable sort by the 63-bit code: low word (values = index), then high word
  if (cudaMemsetAsync(ghist, 0, 4 * 256 * 8, s) != cudaSuccess) return POTR_ERR_CUDA;
  if (cudaMemsetAsync(counter, 0, 4 * 8, s) != cudaSuccess) return POTR_ERR_CUDA;
  radix_hist_kernel<<<g, 256, 0, s>>>(n, lo, ghist);
  POTR_CHECK_LAUNCH();
  digit_base_kernel<<<1, 256, 0, s>>>(ghist, 4, gbase);
  POTR_CHECK_LAUNCH();
  {
    // low words: lo -> A -> B -> A -> B (values: index -> v -> v2 -> v -> v2)
    uint32_t *A = lo2, *Bk = hi2;
    uint32_t* kin[4] = {lo, A, Bk, A};
    uint32_t* kout[4] = {A, Bk, A, Bk};
    uint32_t* vin[4] = {nullptr, v, v2, v};
    uint32_t* vout[4] = {v, v2, v, v2};
    for (int p = 0; p < 4; ++p)
      if (onesweep_pass(kin[p], vin[p], nullptr, n, L.blocks, 8 * p, gbase + 256 * p, counter + p, status, kout[p],
                        vout[p], d_status, s) != cudaSuccess)
        return POTR_ERR_CUDA;
    // high words in that order: A; then A -> B -> A -> B -> A (values: v2 -> v -> v2 -> v -> v2)
    gather_u32_kernel<<<g, 256, 0, s>>>(n, hi, v2, A);
    POTR_CHECK_LAUNCH();
    if (cudaMemsetAsync(ghist + 256 * 4, 0, 4 * 256 * 4, s) != cudaSuccess) return POTR_ERR_CUDA;
    radix_hist_kernel<<<g, 256, 0, s>>>(n, A, ghist + 256 * 4);
    POTR_CHECK_LAUNCH();
    digit_base_kernel<<<1, 256, 0, s>>>(ghist + 256 * 4, 4, gbase + 256 * 4);
    POTR_CHECK_LAUNCH();
    uint32_t* kin2[4] = {A, Bk, A, Bk};
    uint32_t* kout2[4] = {Bk, A, Bk, A};
    uint32_t* vin2[4] = {v2, v, v2, v};
    uint32_t* vout2[4] = {v, v2, v, v2};
    for (int p = 0; p < 4; ++p)
      if (onesweep_pass(kin2[p], vin2[p], nullptr, n, L.blocks, 8 * p, gbase + 256 * (4 + p), counter + 4 + p, status,
                        kout2[p], vout2[p], d_status, s) != cudaSuccess)
        return POTR_ERR_CUDA;
    // the leaf order (v2), sorted high words (A), sorted low words gathered (into Bk)
    if (cudaMemcpyAsync(d_order, v2, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return POTR_ERR_CUDA;
    uint32_t* hs = A;
    uint32_t* ls = Bk;
    gather_u32_kernel<<<g, 256, 0, s>>>(n, lo, d_order, ls);
    POTR_CHECK_LAUNCH();
    // leaf depths, node counts, node offsets
    codec_depth_kernel<<<g, 256, 0, s>>>(n, ls, hs, d_order, scene->means, cube, tol, Ls, Ds, cnt);
    POTR_CHECK_LAUNCH();
    if (scan_exclusive<uint32_t, uint32_t>(cnt, off, n, total, scan_ws, s) != cudaSuccess) return POTR_ERR_CUDA;
    codec_chunk_last_kernel<<<(unsigned)L.n_chunks, 256, 0, s>>>(n, Ls, chunk);
    POTR_CHECK_LAUNCH();
    prefix_max_columns_kernel<<<kLevels, 256, 0, s>>>(L.n_chunks, kLevels, chunk);
    POTR_CHECK_LAUNCH();
    if (cudaMemsetAsync(node, 0, 4 * (size_t)n * (kDepth + 1), s) != cudaSuccess) return POTR_ERR_CUDA;
    codec_nodes_kernel<<<g, 256, 0, s>>>(n, ls, hs, Ls, Ds, off, chunk, node);
    POTR_CHECK_LAUNCH();
    // the shared-leaf table
    codec_leaf_flags_kernel<<<g, 256, 0, s>>>(n, Ls, Ds, flags);
    POTR_CHECK_LAUNCH();
    if (scan_exclusive<uint64_t, uint64_t>(flags, fscan, n, total + 1, scan_ws, s) != cudaSuccess) return POTR_ERR_CUDA;
    codec_dups_kernel<<<g, 256, 0, s>>>(n, Ls, flags, fscan, d_dups);
    POTR_CHECK_LAUNCH();
    store_high_word_kernel<<<1, 1, 0, s>>>(total + 1, d_n_dups);
    POTR_CHECK_LAUNCH();
  }
  if (cudaMemcpyAsync(d_n_nodes, total, 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return POTR_ERR_CUDA;
  pack_bytes_kernel<<<g, 256, 0, s>>>(d_n_nodes, node, d_nodes);
  POTR_CHECK_LAUNCH();
  codec_attr_kernel<<<g, 256, 0, s>>>(n, d_order, scene->log_scales, scene->quats, scene->opacity_logits, scene->sh,
                                      params->sf_scale, params->sf_rotation, params->sf_opacity, params->sf_sh,
                                      d_attrs);
  POTR_CHECK_LAUNCH();
  if (d_cube && cudaMemcpyAsync(d_cube, cube, sizeof(Cube), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  return POTR_OK;
}
