// prune.cu -- one iteration of POTR's pruning controller (Section IV-C) on the device.
//
// Candidates are the live splats with dMSE_k < dMSE_MAX.  The budget is B = (sum of the
// candidates' importance) / (remaining iterations), and the removal set S is the shortest
// prefix of the candidates in ascending (m(dMSE_k / dMSE_MAX), k) order whose importance
// reaches B.  Importance is counted in integer units of 2^-40 (q_k = floor(I_k 2^40)), so every
// sum and the "budget reached" test are exact and independent of summation order.
//
// S is found without sorting: a weighted radix select over the 96-bit composite key
// (bits of m, which order like the non-negative doubles they are, then k) finds the element
// e* at which the running q-sum first reaches B, one 8-bit digit per level (12 levels); each
// level is a q-weighted digit histogram of the elements that share the digits chosen so far,
// followed by one block that picks the digit.  S is then every candidate whose key is <= e*'s.
// Everything runs on the stream, with no host synchronisation.
#include "potr_device.cuh"

namespace potr {
namespace {

constexpr int kPruneThreads = 256;
constexpr int kPruneLevels = 12;  // 8 digits of the m bits, 4 of the splat index
constexpr unsigned long long kNotCandidate = ~0ull;

struct PruneState {
  unsigned long long total;    // sum of q over the candidates
  unsigned long long budget;   // B
  unsigned long long below;    // q-sum of the elements ordered before the chosen prefix
  unsigned long long pkey;     // chosen digits of the m bits (left-aligned)
  unsigned long long removed;  // |S|
  uint32_t pidx;               // chosen digits of the index (left-aligned)
  uint32_t pad;
};

// m(x) = x (x >= 0, -0 -> +0), (sqrt(1 - 2 a x) - 1) / a (x < 0); IEEE operations in that order.
__device__ __forceinline__ double m_map(double x, double a) {
  if (x >= 0.0) return __dadd_rn(x, 0.0);
  return __ddiv_rn(__dsub_rn(__dsqrt_rn(__dsub_rn(1.0, __dmul_rn(2.0 * a, x))), 1.0), a);
}

__global__ void __launch_bounds__(kPruneThreads) prune_prep_kernel(int64_t n, const double* __restrict__ dmse,
                                                                  const double* __restrict__ imp,
                                                                  const uint8_t* __restrict__ alive, double dmax,
                                                                  double a, unsigned long long* __restrict__ key,
                                                                  unsigned long long* __restrict__ q,
                                                                  PruneState* st) {
  unsigned long long part = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double d = dmse[k];
    const bool cand = alive[k] != 0 && d < dmax;
    unsigned long long kk = kNotCandidate, qq = 0;
    if (cand) {
      kk = (unsigned long long)__double_as_longlong(m_map(__ddiv_rn(d, dmax), a));
      const double i = imp[k];
      qq = i >= 0.0 ? (unsigned long long)floor(__dmul_rn(i, 1099511627776.0)) : 0ull;  // 2^40
    }
    key[k] = kk;
    q[k] = qq;
    part += qq;
  }
  // integer sums: any order gives the same total
  for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0 && part) atomicAdd(&st->total, part);
}

__global__ void prune_budget_kernel(int32_t remaining, PruneState* st) {
  st->budget = st->total / (unsigned long long)remaining;
  st->below = 0;
  st->pkey = 0;
  st->pidx = 0;
  st->removed = 0;
}

// Digit `level` of element k's composite key, or 256 when k is no candidate or differs from the
// chosen prefix in an earlier digit.
__device__ __forceinline__ uint32_t prune_digit(unsigned long long key, uint32_t k, int level,
                                                unsigned long long pkey, uint32_t pidx) {
  if (key == kNotCandidate) return 256u;
  if (level < 8) {
    if (level > 0 && (key >> (64 - 8 * level)) != (pkey >> (64 - 8 * level))) return 256u;
    return (uint32_t)(key >> (56 - 8 * level)) & 0xffu;
  }
  if (key != pkey) return 256u;
  const int l = level - 8;
  if (l > 0 && (k >> (32 - 8 * l)) != (pidx >> (32 - 8 * l))) return 256u;
  return (k >> (24 - 8 * l)) & 0xffu;
}

__global__ void __launch_bounds__(kPruneThreads) prune_hist_kernel(int64_t n, const unsigned long long* __restrict__ key,
                                                                  const unsigned long long* __restrict__ q, int level,
                                                                  const PruneState* __restrict__ st,
                                                                  unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const unsigned long long pkey = st->pkey;
  const uint32_t pidx = st->pidx;
  if (st->budget > 0) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
      const uint32_t d = prune_digit(key[k], (uint32_t)k, level, pkey, pidx);
      if (d < 256u && q[k]) atomicAdd(&h[d], q[k]);
    }
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// Smallest digit d with below + sum_{d' <= d} hist[d'] >= B; below grows by the sum over d' < d.
__global__ void __launch_bounds__(256) prune_pick_kernel(int level, const unsigned long long* __restrict__ hist,
                                                         PruneState* st) {
  __shared__ unsigned long long tot[8];
  __shared__ int s_pick;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned long long budget = st->budget, below = st->below;
  if (t == 0) s_pick = 256;
  unsigned long long x = hist[t], incl = x;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) tot[warp] = incl;
  __syncthreads();
  unsigned long long wb = 0;
  for (int w = 0; w < warp; ++w) wb += tot[w];
  incl += wb;
  const unsigned long long excl = incl - x;
  if (budget > 0 && below + excl < budget && below + incl >= budget) s_pick = t;  // exactly one t
  __syncthreads();
  if (t == s_pick) {
    st->below = below + excl;
    if (level < 8) st->pkey |= (unsigned long long)t << (56 - 8 * level);
    else st->pidx |= (uint32_t)t << (24 - 8 * (level - 8));
  }
}

__global__ void __launch_bounds__(kPruneThreads) prune_mark_kernel(int64_t n, const unsigned long long* __restrict__ key,
                                                                  PruneState* st, uint8_t* __restrict__ alive) {
  const unsigned long long pkey = st->pkey;
  const uint32_t pidx = st->pidx;
  const bool any = st->budget > 0;
  unsigned long long cnt = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long kk = key[k];
    if (any && kk != kNotCandidate && (kk < pkey || (kk == pkey && (uint32_t)k <= pidx))) {
      alive[k] = 0;
      ++cnt;
    }
  }
  for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&st->removed, cnt);
}

__global__ void prune_apply_kernel(int64_t n, const uint8_t* __restrict__ alive, float* __restrict__ logits) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if (!alive[k]) logits[k] = -INFINITY;
}

size_t prune_align(size_t x) { return (x + 255) & ~size_t(255); }

struct PruneLayout {
  size_t off_key, off_q, off_hist, off_state, bytes;
};

PruneLayout prune_layout(int64_t n) {
  PruneLayout L{};
  size_t o = 0;
  L.off_key = o; o = prune_align(o + sizeof(unsigned long long) * (size_t)n);
  L.off_q = o; o = prune_align(o + sizeof(unsigned long long) * (size_t)n);
  L.off_hist = o; o = prune_align(o + sizeof(unsigned long long) * 256 * kPruneLevels);
  L.off_state = o; o = prune_align(o + sizeof(PruneState));
  L.bytes = o;
  return L;
}

int prune_grid(int64_t n) {
  const int64_t g = (n + kPruneThreads - 1) / kPruneThreads;
  return (int)(g < 152 * 8 ? (g < 1 ? 1 : g) : 152 * 8);
}

}  // namespace
}  // namespace potr

extern "C" size_t potr_prune_workspace_size(int64_t n) {
  if (n <= 0) return 0;
  return potr::prune_layout(n).bytes;
}

extern "C" potr_status potr_prune_select(int64_t n, const double* d_dmse, const double* d_importance,
                                         uint8_t* d_alive, double dmse_max, double a, int32_t remaining_iterations,
                                         unsigned long long* d_removed, void* d_ws, size_t ws_bytes,
                                         potr_stream_t stream) {
  using namespace potr;
  if (n <= 0 || n > (int64_t)0xffffffffll || !d_dmse || !d_importance || !d_alive || !d_ws)
    return POTR_ERR_INVALID_ARGUMENT;
  if (remaining_iterations < 1 || !(dmse_max > 0.0) || !(a > 0.0)) return POTR_ERR_INVALID_ARGUMENT;
  const PruneLayout L = prune_layout(n);
  if (ws_bytes < L.bytes) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(ws + L.off_key);
  unsigned long long* q = reinterpret_cast<unsigned long long*>(ws + L.off_q);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(ws + L.off_hist);
  PruneState* st = reinterpret_cast<PruneState*>(ws + L.off_state);
  if (cudaMemsetAsync(st, 0, sizeof(PruneState), s) != cudaSuccess) return POTR_ERR_CUDA;
  if (cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 256 * kPruneLevels, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  const int g = prune_grid(n);
  prune_prep_kernel<<<g, kPruneThreads, 0, s>>>(n, d_dmse, d_importance, d_alive, dmse_max, a, key, q, st);
  POTR_CHECK_LAUNCH();
  prune_budget_kernel<<<1, 1, 0, s>>>(remaining_iterations, st);
  POTR_CHECK_LAUNCH();
  for (int level = 0; level < kPruneLevels; ++level) {
    prune_hist_kernel<<<g, kPruneThreads, 0, s>>>(n, key, q, level, st, hist + 256 * level);
    POTR_CHECK_LAUNCH();
    prune_pick_kernel<<<1, 256, 0, s>>>(level, hist + 256 * level, st);
    POTR_CHECK_LAUNCH();
  }
  prune_mark_kernel<<<g, kPruneThreads, 0, s>>>(n, key, st, d_alive);
  POTR_CHECK_LAUNCH();
  if (d_removed && cudaMemcpyAsync(d_removed, &st->removed, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                   s) != cudaSuccess)
    return POTR_ERR_CUDA;
  return POTR_OK;
}

extern "C" potr_status potr_prune_apply(int64_t n, const uint8_t* d_alive, float* d_opacity_logits,
                                        potr_stream_t stream) {
  using namespace potr;
  if (n <= 0 || !d_alive || !d_opacity_logits) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  prune_apply_kernel<<<prune_grid(n), kPruneThreads, 0, s>>>(n, d_alive, d_opacity_logits);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
