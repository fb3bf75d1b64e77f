// raster.cu -- per-tile compositing (paper Section 3, Eqs. 2-4) and the removal-effect pass
// (Section IV-B), plus the per-splat reduction into dMSE_k and I_k (Section IV-B last
// equation, Section IV-A).
//
// Warps work on their own: each takes (tile, 8 x 8 block) items from a queue (longest tile
// lists first), two vertically adjacent pixels per lane, their binary32 arithmetic in packed
// pairs (tile_pass.cuh).  A warp gathers the 48-byte raster records of its tile's depth-sorted
// list into a ring of its own in shared memory with cp.async (16-byte copies), 32 list
// positions at a time, so its 64 pixels read them as shared-memory broadcasts.  The per-pair
// work is plain FP32 ALU: these kernels are bound by instruction issue, not by HBM.
//
// Removal effect: after the forward walk (c, T_final, n_last per pixel) the same list is
// walked back to front, recovering T_i = T_{i+1} / (1 - alpha_i) and accumulating the
// suffix S_{>i} = sum_{j>i} T_j alpha_j c_j, so that
//     PD_i = alpha_i / (1 - alpha_i) S_{>i} - T_i alpha_i c_i
// which equals the paper's P_i - P_{i+1} / (1 - alpha_i) + alpha_i / (1 - alpha_i) P_K because
// P_K - P_{i+1} = S_{>i}; every term is a sum of non-negative numbers, so no prefix sums are
// subtracted.  dSE_i = sum_ch PD_i (PD_i + 2 (c - c_t)).  Per (tile, splat) the 256 pixel
// values are summed without atomics: each lane adds its two pixels, then 8 splats at a time a
// warp transpose-sum leaves a lane with its block's total for one splat, and the last of the
// tile's four blocks to finish adds the four block totals in block order.  The order is fixed,
// so the result does not depend on scheduling.
#include <atomic>

#include "raster_common.cuh"
#include "tile_pass.cuh"

namespace potr {
namespace {

// Compositing by independent warps: each takes (tile, 8 x 8 block) items and walks the tile's
// list on its own (no barrier between the warps of a CTA).
__global__ void __launch_bounds__(kT2, 8) render_kernel(const float4* __restrict__ raster,
                                                     const uint32_t* __restrict__ vals,
                                                     const uint32_t* __restrict__ ranges,
                                                     const potr_view_info* __restrict__ info, int n_views,
                                                     int64_t total_tiles, potr_raster_config cfg,
                                                     float* __restrict__ images, float* __restrict__ t_final,
                                                     uint32_t* __restrict__ n_last, TileQueue queue) {
  extern __shared__ float4 smem[];
  float4* ring = smem + (threadIdx.x >> 5) * kWarpSmemF4;
  int64_t stride_next = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int64_t tile;
  int blk;
  while (next_block_item(queue, total_tiles, stride_next, tile, blk)) {
    const Tile2 c = tile2_block_ctx(info, n_views, ranges, cfg, tile, blk);
    f2_t C[3], T;
    uint32_t last0, last1;
    forward_walk_w(ring, raster, vals, c, cfg, C, T, last0, last1);
    const int64_t plane = (int64_t)c.vi.width * c.vi.height;
    const int64_t pix = c.vi.pixel_base + (int64_t)c.py * c.vi.width + c.px;
    float* im = images ? images + 3 * c.vi.pixel_base + (int64_t)c.py * c.vi.width + c.px : nullptr;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!(h ? c.in1 : c.in0)) continue;
      const int64_t row = h ? c.vi.width : 0;
      float lo0, hi0;
      if (im) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          f2split(C[ch], lo0, hi0);
          im[row + ch * plane] = h ? hi0 : lo0;
        }
      }
      f2split(T, lo0, hi0);
      if (t_final) t_final[pix + row] = h ? hi0 : lo0;
      if (n_last) n_last[pix + row] = h ? last1 : last0;
    }
  }
}

// Lanes l, l^8, l^16, l^24 receive the sum over all 32 lanes of v[l & 7] (fixed order): a
// transpose-sum inside each 8-lane group, then exchanges between the groups.
__device__ __forceinline__ float warp_transpose_sum8(float (&v)[8]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 4; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = upper ? v[i] : v[i + off];
      const float keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  float r = v[0];
  r += __shfl_xor_sync(0xffffffffu, r, 8);
  r += __shfl_xor_sync(0xffffffffu, r, 16);
  return r;
}

constexpr int kChunk = 8;  // splats per warp transpose-sum

// Removal pass with independent warps.  Each warp takes (tile, 8 x 8 block) items of its own
// (longest lists first), walks the tile's list forward at its 64 pixels, then back to front
// over positions [0, top) of its block (top = the block's largest n_last), staging the records
// itself, 32 positions at a time, in its own ring: no barrier couples the warps.  Per position,
// the block's sums over its pixels (warp transpose-sums) go to part[position][block] in global
// memory; the last of a tile's four blocks to finish (an arrival counter per tile) adds the four
// blocks in block order -- a block contributes 0 at positions it never reached -- and writes each
// (tile, splat) sum to the instance's emission slot.  The sums and their order are those of a
// tile-wide walk whose warps meet at every batch; only the waiting is gone.
struct RemovalScratch {
  float4* part_d;        // [instances] block sums of dSE, blocks 0..3 in x..w
  float4* part_i;        // [instances] block sums of T alpha (importance), or null
  uint4* tile_top;       // [tiles] the four blocks' top positions
  uint32_t* tile_arrive;  // [tiles] blocks finished (zero before the launch)
};

constexpr size_t kRemovalWarpF4 = kWarpSmemF4 + 16;  // + 64 floats of group sums per warp

template <bool IMP>
__global__ void __launch_bounds__(kT2, 8) removal_kernel(const float4* __restrict__ raster,
                                                       const uint32_t* __restrict__ vals,
                                                       const uint32_t* __restrict__ ranges,
                                                       const potr_view_info* __restrict__ info, int n_views,
                                                       int64_t total_tiles, potr_raster_config cfg,
                                                       const float* __restrict__ targets, float* __restrict__ images,
                                                       float* __restrict__ inst_dse, float* __restrict__ inst_imp,
                                                       const uint4* __restrict__ cull,
                                                       const uint32_t* __restrict__ offsets, TileQueue queue,
                                                       RemovalScratch scr) {
  extern __shared__ float4 dyn[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* ring = dyn + warp * kRemovalWarpF4;                               // kWRing staged groups
  float4* ex = ring + kWRing * kWSlot;                                      // [32][kERec] expanded
  float* gsum_d = reinterpret_cast<float*>(ring + kWarpSmemF4);             // [32] this group's sums
  float* gsum_i = gsum_d + 32;                                              // [32]
  float* part_d = reinterpret_cast<float*>(scr.part_d);
  float* part_i = reinterpret_cast<float*>(scr.part_i);
  int64_t stride_next = (int64_t)blockIdx.x * kW2 + warp;
  int64_t tile;
  int blk;
  while (next_block_item(queue, total_tiles, stride_next, tile, blk)) {
    const Tile2 c = tile2_block_ctx(info, n_views, ranges, cfg, tile, blk);
    f2_t C[3], T;
    uint32_t last0, last1;
    forward_walk_w(ring, raster, vals, c, cfg, C, T, last0, last1);

    // 2 (c - c_t) per channel and pixel (0 outside the image)
    f2_t e2[3];
    {
      const int64_t plane = (int64_t)c.vi.width * c.vi.height;
      const int64_t o = 3 * c.vi.pixel_base + (int64_t)c.py * c.vi.width + c.px;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float v0 = 0.0f, v1 = 0.0f;
        if (c.in0) v0 = 2.0f * (f2lo(C[ch]) - targets[o + ch * plane]);
        if (c.in1) v1 = 2.0f * (f2hi(C[ch]) - targets[o + c.vi.width + ch * plane]);
        e2[ch] = f2(v0, v1);
        if (images) {
          if (c.in0) images[o + ch * plane] = f2lo(C[ch]);
          if (c.in1) images[o + c.vi.width + ch * plane] = f2hi(C[ch]);
        }
      }
    }
    const uint32_t top = __reduce_max_sync(0xffffffffu, max(last0, last1));
    const f2_t fx2 = f2s(c.fx), fy2 = f2(c.fy0, c.fy1);

    // Back to front over positions [0, top): T_i = T_{i+1} / (1 - alpha_i), S = sum of
    // T_j alpha_j c_j over the composited j > i.  The splats the block test keeps are visited
    // 8 at a time, highest position first.
    f2_t S[3] = {f2s(0.0f), f2s(0.0f), f2s(0.0f)};
    const uint32_t ng = (top + 31) / 32;
    if (ng > 0) {
      const uint32_t g0 = 32 * (ng - 1);
      warp_stage(ring + kWSlot * ((ng - 1) % kWRing), raster, vals, c.s + g0, (int)(top - g0));
    }
    for (uint32_t gg = ng; gg-- > 0;) {
      const uint32_t g0 = 32 * gg;
      const int cnt = (int)min(32u, top - g0);
      if (gg > 0) {
        warp_stage(ring + kWSlot * ((gg - 1) % kWRing), raster, vals, c.s + g0 - 32, 32);
        cp_async_wait2<1>();
      } else {
        cp_async_wait2<0>();
      }
      if (lane < cnt) expand_record(ring + kWSlot * (gg % kWRing) + kSRec2 * lane, ex + kERec * lane);
      gsum_d[lane] = 0.0f;
      if (IMP) gsum_i[lane] = 0.0f;
      __syncwarp();  // the group's expanded records and zeroed sums are visible
      const bool cand = lane < cnt && block_may_pass_e(ex + kERec * lane, c.bx0, c.by0);
      uint32_t m = __ballot_sync(0xffffffffu, cand);
      while (m) {
        float d[kChunk], im[kChunk];
        int mypos = -1;
        bool any = false;
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          d[u] = 0.0f;
          if (IMP) im[u] = 0.0f;
          if (m) {
            const int j = 31 - __clz(m);
            m &= ~(1u << j);
            if (lane == u) mypos = j;
            const uint32_t pos = g0 + (uint32_t)j;
            const float4* e = ex + kERec * j;
            f2_t o2;
            float thr, indef;
            const f2_t p2 = exponent_e(e, fx2, fy2, o2, thr, indef);
            float p0, p1;
            f2split(p2, p0, p1);
            const bool pass0 = pos < last0 && p0 >= thr, pass1 = pos < last1 && p1 >= thr;
            if (__any_sync(0xffffffffu, pass0 || pass1)) {  // warp-uniform: branch-free below
              float a0, a1;
              f2split(mul2(o2, exp2r2_rec(p2, indef)), a0, a1);
              a0 = fminf(cfg.alpha_max, a0);
              a1 = fminf(cfg.alpha_max, a1);
              const bool ok0 = pass0 && a0 >= cfg.alpha_min, ok1 = pass1 && a1 >= cfg.alpha_min;
              // a pixel that does not take the splat: alpha 0 and 1 / (1 - alpha) = 1, so its
              // T, S and dSE do not change (every update adds or scales by exact zeros and ones)
              const float q0 = __fdividef(1.0f, 1.0f - a0), q1 = __fdividef(1.0f, 1.0f - a1);
              const f2_t ae = f2(ok0 ? a0 : 0.0f, ok1 ? a1 : 0.0f);
              const f2_t rcp = f2(ok0 ? q0 : 1.0f, ok1 ? q1 : 1.0f);
              T = mul2(T, rcp);                      // T_i = T_{i+1} / (1 - alpha_i)
              const f2_t w = mul2(ae, T);            // T_i alpha_i
              const f2_t ratio = mul2(ae, rcp);      // alpha_i / (1 - alpha_i)
              const f2_t nw = sub2(f2s(0.0f), w);    // -T_i alpha_i (exact)
              const ulonglong2 q3 = reinterpret_cast<const ulonglong2*>(e)[3];
              const ulonglong2 q4 = reinterpret_cast<const ulonglong2*>(e)[4];
              const f2_t nwc0 = mul2(nw, q3.y), nwc1 = mul2(nw, q4.x), nwc2 = mul2(nw, q4.y);
              // PD = alpha / (1 - alpha) S - T alpha c, one rounding per channel
              const f2_t pd0 = fma2(ratio, S[0], nwc0);
              const f2_t pd1 = fma2(ratio, S[1], nwc1);
              const f2_t pd2 = fma2(ratio, S[2], nwc2);
              f2_t dse = mul2(pd0, add2(pd0, e2[0]));  // sum_ch PD (PD + 2 (c - c_t))
              dse = fma2(pd1, add2(pd1, e2[1]), dse);
              dse = fma2(pd2, add2(pd2, e2[2]), dse);
              S[0] = sub2(S[0], nwc0);  // S + T alpha c
              S[1] = sub2(S[1], nwc1);
              S[2] = sub2(S[2], nwc2);
              float x0, x1;
              f2split(dse, x0, x1);
              d[u] = x0 + x1;
              if (IMP) {
                f2split(w, x0, x1);
                im[u] = x0 + x1;
              }
              any = true;
            }
          }
        }
        float sd = 0.0f, si = 0.0f;
        if (__any_sync(0xffffffffu, any)) {
          sd = warp_transpose_sum8(d);
          if (IMP) si = warp_transpose_sum8(im);
        }
        if (lane < kChunk && mypos >= 0) {
          gsum_d[mypos] = sd;
          if (IMP) gsum_i[mypos] = si;
        }
      }
      __syncwarp();  // the group's sums are complete
      if (lane < cnt) {
        part_d[(int64_t)(c.s + g0 + lane) * 4 + blk] = gsum_d[lane];
        if (IMP) part_i[(int64_t)(c.s + g0 + lane) * 4 + blk] = gsum_i[lane];
      }
      __syncwarp();  // this slot, the expanded records and the sums are rewritten next
    }

    // arrival: the tile's last block to finish adds the four blocks' sums in block order
    uint32_t arrived = 0;
    if (lane == 0) reinterpret_cast<uint32_t*>(scr.tile_top)[tile * 4 + blk] = top;
    __threadfence();  // every lane's sums, and the top, are visible device-wide before the count
    __syncwarp();
    if (lane == 0) arrived = atomicAdd(scr.tile_arrive + tile, 1u);
    arrived = __shfl_sync(0xffffffffu, arrived, 0);
    if (arrived == 3u) {
      __threadfence();
      const uint4 tops = __ldcg(scr.tile_top + tile);
      const uint32_t mt = max(max(tops.x, tops.y), max(tops.z, tops.w));
      for (uint32_t p0 = 0; p0 < mt; p0 += 32) {
        const uint32_t pos = p0 + (uint32_t)lane;
        if (pos >= mt) break;
        const float4 bd = __ldcg(scr.part_d + c.s + pos);
        float sd = 0.0f, si = 0.0f;
        sd += pos < tops.x ? bd.x : 0.0f;
        sd += pos < tops.y ? bd.y : 0.0f;
        sd += pos < tops.z ? bd.z : 0.0f;
        sd += pos < tops.w ? bd.w : 0.0f;
        if (IMP) {
          const float4 bi = __ldcg(scr.part_i + c.s + pos);
          si += pos < tops.x ? bi.x : 0.0f;
          si += pos < tops.y ? bi.y : 0.0f;
          si += pos < tops.z ? bi.z : 0.0f;
          si += pos < tops.w ? bi.w : 0.0f;
        }
        if (sd != 0.0f || (IMP && si != 0.0f)) {
          const uint32_t vk = vals[c.s + pos];
          const uint32_t slot = emission_slot(offsets[vk], cull[vk], c.tx, c.ty);  // L2
          inst_dse[slot] = sd;
          if (IMP) inst_imp[slot] = si;
        }
      }
    }
  }  // items
}

template <bool IMP>
constexpr size_t removal_smem_bytes() {
  return sizeof(float4) * kW2 * kRemovalWarpF4;
}

// Per splat k: dSSE_k(v) = sum over its emission slots (emission order, compensated binary32),
// then dmse[k] += dSSE_k(v) * scale_d[v] in binary64, views in order, with the term
// dSSE_k(v) * scale_d[v] rounded to binary32 and scale_d[v] the binary32 rounding of
// 1 / (3 P_v N); the importance likewise with scale_i[v] = 1 / (P_v N).  The scales are
// computed once per view, so the loop has no division; a call over one view chunk adds the
// same binary64 terms in the same order as a call over the whole frame.  The binary64 pipe
// runs 2 lane operations per SM and cycle, so a view costs it one addition per output: the
// terms are widened to binary64 by moving their bits (widen_f32).
constexpr int kReduceChunk = 256;  // partials staged per warp, view and array

// The binary64 value of a binary32 x, by moving its bits: the exponent rebiased by 1023 - 127
// and the 23 mantissa bits placed at the top of the 52 (exact for zeros and normal numbers,
// IEEE 754 formats); subnormals, infinities and NaN take the conversion instruction.
__device__ __forceinline__ double widen_f32(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0xffu || (e == 0u && (b << 1) != 0u)) return (double)x;
  const uint32_t hi = (b & 0x80000000u) | (e ? (e + 896u) << 20 : 0u) | ((b >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(b << 29));
}

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}

// The warp's slots [c0, c0 + m) of both partial arrays into one staging buffer, as one group.
__device__ __forceinline__ void stage_partials(float* wd, float* wi, const float* __restrict__ inst_dse,
                                               const float* __restrict__ inst_imp, uint32_t c0, uint32_t m, int lane) {
  for (uint32_t i = (uint32_t)lane; i < m; i += 32) {
    cp_async4(wd + i, inst_dse + c0 + i);
    if (inst_imp) cp_async4(wi + i, inst_imp + c0 + i);
  }
  asm volatile("cp.async.commit_group;\n" ::);
}

// Per-view scales of the reduce, one 16-byte word per view: the binary32 roundings of
// 1 / (3 P_v N) and 1 / (P_v N), and 1 / P_v in binary64 (computed once here, so the reduce
// has no division).
__global__ void view_scale_kernel(const potr_view_info* __restrict__ info, int n_views, double n_total,
                                  uint4* __restrict__ scales) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  const double P = (double)info[v].width * (double)info[v].height;
  const double ip = 1.0 / P;
  scales[v] = make_uint4(__float_as_uint((float)(1.0 / (3.0 * P * n_total))), __float_as_uint((float)(1.0 / (P * n_total))),
                         (uint32_t)__double2loint(ip), (uint32_t)__double2hiint(ip));
}

__global__ void __launch_bounds__(256, 5) splat_reduce_kernel(const uint32_t* __restrict__ touched,
                                                              const uint32_t* __restrict__ offsets,
                                                              const uint32_t* __restrict__ n_inst, int64_t capacity,
                                                              const float* __restrict__ inst_dse,
                                                              const float* __restrict__ inst_imp, int64_t n, int n_views,
                                                              const uint4* __restrict__ scales,
                                                              double* __restrict__ dmse, double* __restrict__ importance,
                                                              double* __restrict__ dsse_view,
                                                              double* __restrict__ imp_view) {
  // One warp per 32 consecutive splats.  For one view their emission slots form one contiguous
  // range (offsets are the exclusive prefix in vk order), which the warp stages through its own
  // shared memory with coalesced copies; each lane then adds its own slots, in slot order, from
  // there.  The views are pipelined: while a view is summed, the next view's slots are in
  // flight to the other buffer and the counts and offsets of the one after are being loaded.
  // Warps synchronise only among their own lanes.
  __shared__ float s_d[kWarps][2][kReduceChunk], s_i[kWarps][2][kReduceChunk];
  if ((int64_t)*n_inst > capacity) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t k0 = ((int64_t)blockIdx.x * kWarps + warp) * 32;
  const int64_t k = k0 + lane;
  if (k0 >= n) return;  // warp-uniform
  const int last_lane = (int)(min(k0 + 32, n) - 1 - k0);
  double acc_d = (dmse && k < n) ? dmse[k] : 0.0;
  double acc_i = (importance && k < n) ? importance[k] : 0.0;
  // count and offset of this lane's splat in the next view (a) and the one after (b)
  uint32_t cnt_a = 0, off_a = 0, cnt_b = 0, off_b = 0;
  if (k < n) {
    cnt_a = touched[k];
    off_a = offsets[k];
    if (n_views > 1) {
      cnt_b = touched[n + k];
      off_b = offsets[n + k];
    }
  }
  uint32_t lo = __shfl_sync(0xffffffffu, off_a, 0);
  uint32_t hi = __shfl_sync(0xffffffffu, off_a + cnt_a, last_lane);
  stage_partials(s_d[warp][0], s_i[warp][0], inst_dse, inst_imp, lo, min((uint32_t)kReduceChunk, hi - lo), lane);
  for (int v = 0; v < n_views; ++v) {
    const int64_t row = (int64_t)v * n;
    const uint32_t cnt = cnt_a, off = off_a, vlo = lo, vhi = hi;
    float* wd = s_d[warp][v & 1];
    float* wi = s_i[warp][v & 1];
    const uint4 sc = scales[v];  // the same word for every lane
    cnt_a = cnt_b;
    off_a = off_b;
    if (k < n && v + 2 < n_views) {
      cnt_b = touched[row + 2 * n + k];
      off_b = offsets[row + 2 * n + k];
    }
    if (v + 1 < n_views) {  // the next view's first chunk, into the other buffer
      lo = __shfl_sync(0xffffffffu, off_a, 0);
      hi = __shfl_sync(0xffffffffu, off_a + cnt_a, last_lane);
      stage_partials(s_d[warp][(v + 1) & 1], s_i[warp][(v + 1) & 1], inst_dse, inst_imp, lo,
                     min((uint32_t)kReduceChunk, hi - lo), lane);
      asm volatile("cp.async.wait_group 1;\n" ::);
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::);
    }
    __syncwarp();  // this view's first chunk is visible to every lane
    KahanSum kd, ki;
    for (uint32_t c0 = vlo; c0 < vhi; c0 += kReduceChunk) {
      const uint32_t m = min((uint32_t)kReduceChunk, vhi - c0);
      if (c0 != vlo) {  // a range longer than one chunk: the rest is staged here and waited for
        __syncwarp();   // every lane is done with the previous chunk
        stage_partials(wd, wi, inst_dse, inst_imp, c0, m, lane);
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncwarp();
      }
      const uint32_t a = max(off, c0), b = min(off + cnt, c0 + m);
      for (uint32_t i = a; i < b; ++i) {
        kd.add(wd[i - c0]);
        if (inst_imp) ki.add(wi[i - c0]);
      }
    }
    __syncwarp();  // every lane is done with this buffer, which the next iteration restages
    const float sd = kd.sum(), si = ki.sum();  // 0 for a splat without slots in the view
    acc_d = __dadd_rn(acc_d, widen_f32(__fmul_rn(sd, __uint_as_float(sc.x))));
    if (importance) acc_i = __dadd_rn(acc_i, widen_f32(__fmul_rn(si, __uint_as_float(sc.y))));
    if (dsse_view && k < n) dsse_view[row + k] = (double)sd;
    if (imp_view && k < n) imp_view[row + k] = (double)si * __hiloint2double((int)sc.w, (int)sc.z);
  }
  if (k < n) {
    if (dmse) dmse[k] = acc_d;
    if (importance) importance[k] = acc_i;
  }
}

template <int BATCH>
cudaError_t launch_render(const potr_views* views, const potr_frame* frame, const potr_raster_config& cfg,
                          const uint32_t* vals, const uint32_t* ranges, float* images, float* t_final,
                          uint32_t* n_last, const TileQueue& q, cudaStream_t s) {
  const size_t smem = sizeof(float4) * kW2 * kWarpSmemF4;
  // a persistent grid: every CTA that fits on the device at once
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_kernel, kT2, smem);
  int64_t g = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (4 * frame->total_tiles + kW2 - 1) / kW2;
  if (g > need) g = need;
  tile_timing_begin(s);
  render_kernel<<<(unsigned)(g > 0 ? g : 1), kT2, smem, s>>>(reinterpret_cast<const float4*>(views->raster), vals,
                                                           ranges, frame->info, frame->n_views, frame->total_tiles, cfg,
                                                           images, t_final, n_last, q);
  tile_timing_end(s);
  note_launches(1);
  return cudaGetLastError();
}


template <bool IMP>
cudaError_t launch_removal(const potr_views* views, const potr_frame* frame, const potr_raster_config& cfg,
                           const uint32_t* vals, const uint32_t* ranges, const float* targets, float* images,
                           float* inst_dse, float* inst_imp, const TileQueue& q, const RemovalScratch& scr,
                           cudaStream_t s) {
  constexpr size_t smem = removal_smem_bytes<IMP>();
  cudaError_t e = cudaFuncSetAttribute(removal_kernel<IMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // several CTAs per SM only fit with the largest shared-memory carveout
  e = cudaFuncSetAttribute(removal_kernel<IMP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(scr.tile_arrive, 0, sizeof(uint32_t) * (size_t)frame->total_tiles, s);
  if (e != cudaSuccess) return e;
  // a persistent grid: every CTA that fits on the device at once, at most one warp per item
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, removal_kernel<IMP>, kT2, smem);
  int64_t g = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (4 * frame->total_tiles + kW2 - 1) / kW2;
  if (g > need) g = need;
  tile_timing_begin(s);
  removal_kernel<IMP><<<(unsigned)(g > 0 ? g : 1), kT2, smem, s>>>(
      reinterpret_cast<const float4*>(views->raster), vals, ranges, frame->info, frame->n_views, frame->total_tiles,
      cfg, targets, images, inst_dse, inst_imp, reinterpret_cast<const uint4*>(views->cull), views->offsets, q, scr);
  tile_timing_end(s);
  note_launches(1);
  return cudaGetLastError();
}

// The work counter word after the order is reset before each persistent launch.
cudaError_t make_queue(uint32_t* d_tile_order, int64_t total_tiles, TileQueue& q, cudaStream_t s) {
  q.order = d_tile_order;
  q.counter = d_tile_order ? d_tile_order + total_tiles : nullptr;
  q.total = (uint32_t)total_tiles;
  if (d_tile_order) return cudaMemsetAsync(q.counter, 0, sizeof(uint32_t), s);
  return cudaSuccess;
}

}  // namespace
}  // namespace potr

extern "C" potr_status potr_render(const potr_views* views, const potr_frame* frame, const potr_raster_config* cfg,
                                   int64_t n, const uint32_t* d_vals, const uint32_t* d_tile_ranges,
                                   uint32_t* d_tile_order, float* d_images, float* d_t_final, uint32_t* d_n_last,
                                   potr_stream_t stream) {
  using namespace potr;
  if (!views || !frame || !valid_cfg(cfg) || !d_vals || !d_tile_ranges || !views->raster || !frame->info)
    return POTR_ERR_INVALID_ARGUMENT;
  if (n <= 0 || frame->n_views < 1 || frame->total_tiles <= 0 || frame->total_tiles > 0x7fffffffll)
    return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TileQueue q;
  if (make_queue(d_tile_order, frame->total_tiles, q, s) != cudaSuccess) return POTR_ERR_CUDA;
  cudaError_t e;
  switch (cfg->batch) {
    case 128: e = launch_render<128>(views, frame, *cfg, d_vals, d_tile_ranges, d_images, d_t_final, d_n_last, q, s); break;
    case 256: e = launch_render<256>(views, frame, *cfg, d_vals, d_tile_ranges, d_images, d_t_final, d_n_last, q, s); break;
    default: e = launch_render<512>(views, frame, *cfg, d_vals, d_tile_ranges, d_images, d_t_final, d_n_last, q, s); break;
  }
  return e == cudaSuccess ? POTR_OK : POTR_ERR_CUDA;
}

namespace potr {
namespace {
struct RemovalLayout {
  size_t off_part_d, off_part_i, off_top, off_arrive, bytes;
};
RemovalLayout removal_layout(int64_t capacity, int64_t total_tiles, bool imp) {
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  RemovalLayout L{};
  size_t o = 0;
  L.off_part_d = o; o = up(o + sizeof(float4) * (size_t)capacity);
  L.off_part_i = o; if (imp) o = up(o + sizeof(float4) * (size_t)capacity);
  L.off_top = o; o = up(o + sizeof(uint4) * (size_t)total_tiles);
  L.off_arrive = o; o = up(o + sizeof(uint32_t) * (size_t)total_tiles);
  L.bytes = o;
  return L;
}
}  // namespace
}  // namespace potr

extern "C" size_t potr_removal_workspace_size(int64_t instance_capacity, int64_t total_tiles,
                                              int32_t with_importance) {
  if (instance_capacity <= 0 || total_tiles <= 0) return 0;
  return potr::removal_layout(instance_capacity, total_tiles, with_importance != 0).bytes;
}

extern "C" potr_status potr_removal_effect(const potr_views* views, const potr_frame* frame,
                                           const potr_raster_config* cfg, int64_t n, const uint32_t* d_vals,
                                           const uint32_t* d_tile_ranges, uint32_t* d_tile_order,
                                           const float* d_targets, int32_t n_views_total,
                                           int64_t instance_capacity, float* d_inst_dse, float* d_inst_imp,
                                           double* d_dmse, double* d_importance, double* d_dsse_view,
                                           double* d_imp_view, float* d_images, void* d_ws, size_t ws_bytes,
                                           potr_stream_t stream) {
  using namespace potr;
  if (!views || !frame || !valid_cfg(cfg) || !d_vals || !d_tile_ranges || !d_targets || !d_inst_dse || !d_ws)
    return POTR_ERR_INVALID_ARGUMENT;
  if (!views->raster || !views->touched || !views->offsets || !views->n_instances || !views->cull || !frame->info)
    return POTR_ERR_INVALID_ARGUMENT;
  if (n <= 0 || frame->n_views < 1 || n_views_total < 1 || instance_capacity <= 0) return POTR_ERR_INVALID_ARGUMENT;
  if (frame->total_tiles <= 0 || frame->total_tiles > 0x7fffffffll) return POTR_ERR_INVALID_ARGUMENT;
  if ((d_importance || d_imp_view) && !d_inst_imp) return POTR_ERR_INVALID_ARGUMENT;
  const bool imp = d_inst_imp != nullptr;
  if (ws_bytes < potr_removal_workspace_size(instance_capacity, frame->total_tiles, imp ? 1 : 0))
    return POTR_ERR_INVALID_ARGUMENT;
  const RemovalLayout L = removal_layout(instance_capacity, frame->total_tiles, imp);
  char* ws = static_cast<char*>(d_ws);
  RemovalScratch scr;
  scr.part_d = reinterpret_cast<float4*>(ws + L.off_part_d);
  scr.part_i = imp ? reinterpret_cast<float4*>(ws + L.off_part_i) : nullptr;
  scr.tile_top = reinterpret_cast<uint4*>(ws + L.off_top);
  scr.tile_arrive = reinterpret_cast<uint32_t*>(ws + L.off_arrive);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_inst_dse, 0, sizeof(float) * (size_t)instance_capacity, s) != cudaSuccess) return POTR_ERR_CUDA;
  if (d_inst_imp && cudaMemsetAsync(d_inst_imp, 0, sizeof(float) * (size_t)instance_capacity, s) != cudaSuccess)
    return POTR_ERR_CUDA;
  TileQueue q;
  if (make_queue(d_tile_order, frame->total_tiles, q, s) != cudaSuccess) return POTR_ERR_CUDA;
  const cudaError_t e = imp ? launch_removal<true>(views, frame, *cfg, d_vals, d_tile_ranges, d_targets, d_images,
                                                   d_inst_dse, d_inst_imp, q, scr, s)
                            : launch_removal<false>(views, frame, *cfg, d_vals, d_tile_ranges, d_targets, d_images,
                                                    d_inst_dse, d_inst_imp, q, scr, s);
  if (e != cudaSuccess) return POTR_ERR_CUDA;
  if (d_dmse || d_importance || d_dsse_view || d_imp_view) {
    // the per-view scales in the tile tops' words, free once the removal kernel has finished
    // (a frame has at least one tile per view)
    view_scale_kernel<<<(unsigned)((frame->n_views + 127) / 128), 128, 0, s>>>(frame->info, frame->n_views,
                                                                             (double)n_views_total, scr.tile_top);
    const int64_t g = (n + 255) / 256;  // one block per 256 splats (a warp per 32)
    splat_reduce_kernel<<<(unsigned)g, 256, 0, s>>>(views->touched, views->offsets, views->n_instances,
                                                     instance_capacity, d_inst_dse, d_inst_imp, n, frame->n_views,
                                                     scr.tile_top, d_dmse, d_importance, d_dsse_view, d_imp_view);
    note_launches(2);
    if (cudaGetLastError() != cudaSuccess) return POTR_ERR_CUDA;
  }
  return POTR_OK;
}

namespace potr {
namespace {

// Exact pair counts of the forward walk and of the back-to-front walk of the removal pass:
// c[0] pairs examined forward, c[1] of those passing the prefilter, c[2] composited,
// c[3] positions walked back to front (sum of n_last), c[4] of those passing the prefilter.
template <int BATCH>
__global__ void __launch_bounds__(kThreads) pair_stats_kernel(const float4* __restrict__ raster,
                                                              const uint32_t* __restrict__ vals,
                                                              const uint32_t* __restrict__ ranges,
                                                              const potr_view_info* __restrict__ info, int n_views,
                                                              potr_raster_config cfg,
                                                              unsigned long long* __restrict__ counts) {
  extern __shared__ float4 smem[];
  __shared__ unsigned long long red[5][kWarps];
  const TileCtx c = tile_ctx(info, n_views, ranges, cfg, blockIdx.x);
  float T = 1.0f;
  uint32_t n_ex = 0, n_pass = 0, n_comp = 0, last = 0, pass_at_last = 0;
  bool done = !c.inside;
  for (uint32_t base = c.s; base < c.e; base += BATCH) {
    if (__syncthreads_and(done)) break;
    const int cnt = (int)min((uint32_t)BATCH, c.e - base);
    stage_batch<BATCH>(smem, raster, vals, base, cnt);
    __syncthreads();
    if (done) continue;
    for (int j = 0; j < cnt; ++j) {
      const float4 r0 = smem[kSRec * j];
      const float4 r1 = smem[kSRec * j + 1];
      ++n_ex;
      const float p = pair_exponent(r0.z, r0.w, r1.x, __fsub_rn(c.fx, r0.x), __fsub_rn(c.fy, r0.y));
      if (p < r1.z) continue;
      ++n_pass;
      const float a = pair_alpha(r1.y, p, cfg.alpha_max);
      if (a < cfg.alpha_min) continue;
      const float Tn = trans_next(a, T);
      if (Tn < cfg.t_min) {
        done = true;
        break;
      }
      T = Tn;
      ++n_comp;
      last = base - c.s + (uint32_t)j + 1;
      pass_at_last = n_pass;
    }
  }
  const uint32_t v[5] = {n_ex, n_pass, n_comp, last, pass_at_last};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    unsigned long long x = v[q];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[q][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    unsigned long long x = 0;
    for (int w = 0; w < kWarps; ++w) x += red[threadIdx.x][w];
    atomicAdd(counts + threadIdx.x, x);
  }
}

std::atomic<unsigned long long> g_launches{0};

struct TileTiming {
  cudaEvent_t start = nullptr, stop = nullptr;
  bool armed = false, open = false;
};
thread_local TileTiming g_tile_timing;

}  // namespace

void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

void tile_timing_begin(cudaStream_t s) {
  TileTiming& t = g_tile_timing;
  if (!t.armed) return;
  t.open = cudaEventRecord(t.start, s) == cudaSuccess;
}

void tile_timing_end(cudaStream_t s) {
  TileTiming& t = g_tile_timing;
  if (!t.armed || !t.open) return;
  cudaEventRecord(t.stop, s);
  t.armed = t.open = false;
}

}  // namespace potr

extern "C" potr_status potr_pair_stats(const potr_views* views, const potr_frame* frame, const potr_raster_config* cfg,
                                       int64_t n, const uint32_t* d_vals, const uint32_t* d_tile_ranges,
                                       uint64_t* d_counts, potr_stream_t stream) {
  using namespace potr;
  if (!views || !frame || !valid_cfg(cfg) || !d_vals || !d_tile_ranges || !d_counts || !views->raster || !frame->info)
    return POTR_ERR_INVALID_ARGUMENT;
  if (n <= 0 || frame->total_tiles <= 0 || frame->total_tiles > 0x7fffffffll) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_counts, 0, 5 * sizeof(uint64_t), s) != cudaSuccess) return POTR_ERR_CUDA;
  pair_stats_kernel<256><<<(unsigned)frame->total_tiles, kThreads, sizeof(float4) * kSRec * 256, s>>>(
      reinterpret_cast<const float4*>(views->raster), d_vals, d_tile_ranges, frame->info, frame->n_views, *cfg,
      reinterpret_cast<unsigned long long*>(d_counts));
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}

extern "C" uint64_t potr_launch_count(void) { return potr::g_launches.load(); }

extern "C" potr_status potr_time_next_tile_kernel(void* start_event, void* stop_event) {
  potr::TileTiming& t = potr::g_tile_timing;
  if ((start_event == nullptr) != (stop_event == nullptr)) return POTR_ERR_INVALID_ARGUMENT;
  t.start = static_cast<cudaEvent_t>(start_event);
  t.stop = static_cast<cudaEvent_t>(stop_event);
  t.armed = start_event != nullptr;
  t.open = false;
  return POTR_OK;
}

extern "C" const char* potr_status_string(potr_status status) {
  switch (status) {
    case POTR_OK: return "ok";
    case POTR_ERR_INVALID_ARGUMENT: return "invalid argument";
    case POTR_ERR_CUDA: return "CUDA launch or runtime error";
    case POTR_ERR_CAPACITY: return "tile-instance capacity exceeded";
    case POTR_ERR_TIMEOUT: return "bounded device wait ran out";
    case POTR_ERR_NUMERIC: return "non-finite input";
    case POTR_ERR_UNSUPPORTED: return "unsupported configuration";
    case POTR_ERR_TOO_LARGE: return "size exceeds the fixed scratch of potr_bin_sort_static";
    case POTR_ERR_CORRUPT: return "malformed codec stream";
    default: return "unknown status";
  }
}

extern "C" int32_t potr_version(void) { return 100; }
