// backward.cu -- the adjoint of the forward rasterizer for fine-tuning (the paper notes its
// CUDA pass is meant to interoperate with the standard forward-backward render pass,
// Section IV-B; POTR-FT fine-tunes with the original 3DGS training routine, Section IV-F).
//
//   loss_grad_kernel      L = (1 - l) mean|c - c_t| + l mean (c - c_t)^2 and dL/dc per channel.
//   render_bwd_kernel     per tile, back to front over each pixel's composited splats: with
//                         S_{>i} = sum_{j>i} T_j alpha_j c_j (the same suffix as the removal
//                         pass), dc/dalpha_i = T_i c_i - S_{>i} / (1 - alpha_i) and dc/dc_i =
//                         T_i alpha_i; through alpha = o 2^p (unclamped) to the opacity, the
//                         exponent coefficients A, B, C and the pixel-space centre.  Four warps
//                         per tile, each on an 8 x 8 block, two pixels per lane in packed f32x2
//                         arithmetic over expanded records (tile_pass.cuh).  The nine per-pair
//                         gradients are summed per (tile, splat) without atomics (each lane's two
//                         pixels, then warp transpose-sums in a fixed order, then warps in
//                         order) into per-instance slots.  T_i comes either from the stored
//                         final transmittance of the forward render or, with none stored, from
//                         re-running the forward walk.
//   vk_bwd_kernel         per (view, splat): its instance slots summed (fixed tree), then the
//                         adjoint of the projection (conic inverse, Sigma2D = T Sigma T^T,
//                         clamped Jacobian, pinhole centre).
//   splat_bwd_kernel      per splat: the views' results summed in view order, the SH colour
//                         adjoint (clamp mask, coefficients, direction) and the adjoint of the
//                         activation (Sigma = M M^T, M = R diag(exp(log_scale)), quaternion
//                         normalisation, sigmoid).
// All sums have a fixed order, so the gradients are bit-identical from run to run.
#include "tile_pass.cuh"

namespace potr {
namespace {

constexpr int kGradQ = 9;     // per-pair gradients: mx, my, A, B, C, opacity, r, g, b
constexpr int kBwdChunk = 4;  // splats per warp transpose-sum
constexpr int kBwdBatch = 64;
constexpr float kLn2 = 0.69314718055994531f;

size_t bwd_smem_bytes() {
  return sizeof(float4) * (2 * kSRec2 + kERec) * kBwdBatch + sizeof(float) * kGradQ * kW2 * kBwdBatch;
}

// Lanes l, l^4, l^8, ... receive the sum over all 32 lanes of v[l & 3] (fixed order): a
// transpose-sum inside each 4-lane group, then exchanges between the groups.
__device__ __forceinline__ float warp_transpose_sum4(float (&v)[kBwdChunk]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 2; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = upper ? v[i] : v[i + off];
      const float keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  float r = v[0];
  r += __shfl_xor_sync(0xffffffffu, r, 4);
  r += __shfl_xor_sync(0xffffffffu, r, 8);
  r += __shfl_xor_sync(0xffffffffu, r, 16);
  return r;
}

// ---------------------------------------------------------------------------------------
// K11: loss and dL/dc
// ---------------------------------------------------------------------------------------
constexpr int kLossBlocks = 1024;

__global__ void __launch_bounds__(256) loss_grad_kernel(const float* __restrict__ img, const float* __restrict__ tgt,
                                                        int64_t n_elems, float lam, float* __restrict__ grad,
                                                        double* __restrict__ block_sums) {
  __shared__ double warp_sums[8];
  const float inv_n = (float)(1.0 / (double)n_elems);
  // per thread a compensated binary32 sum (error about 2 ulps of the sum, independent of the
  // term count; binary64 adds per element would make this kernel FP64-bound), then binary64
  KahanSum part;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_elems; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = img[i] - tgt[i];
    const float sg = (r > 0.0f) ? 1.0f : ((r < 0.0f) ? -1.0f : 0.0f);
    grad[i] = ((1.0f - lam) * sg + 2.0f * lam * r) * inv_n;
    part.add((1.0f - lam) * fabsf(r) + lam * r * r);
  }
  double acc = part.value();
  if (block_sums) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += warp_sums[w];
      block_sums[blockIdx.x] = s;
    }
  }
}

// Sum of the block sums in a fixed order: thread t adds blocks t, t + 256, ..., then a fixed
// tree over the threads (one thread adding all of them serially takes ~1000 dependent binary64
// adds).
__global__ void __launch_bounds__(256) loss_finish_kernel(const double* __restrict__ block_sums, int nb,
                                                          int64_t n_elems, double* __restrict__ loss) {
  __shared__ double part[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) s += block_sums[b];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = part[0] / (double)n_elems;
}

// ---------------------------------------------------------------------------------------
// K9: back-to-front adjoint of the compositing
// ---------------------------------------------------------------------------------------
template <bool RECOMPUTE>
__global__ void __launch_bounds__(kT2, 6) render_bwd_kernel(const float4* __restrict__ raster,
                                                         const uint32_t* __restrict__ vals,
                                                         const uint32_t* __restrict__ ranges,
                                                         const potr_view_info* __restrict__ info, int n_views,
                                                         potr_raster_config cfg, const float* __restrict__ t_final,
                                                         const uint32_t* __restrict__ n_last,
                                                         const float* __restrict__ dL_dimg, int64_t capacity,
                                                         float* __restrict__ inst_grad,
                                                         const uint4* __restrict__ cull,
                                                         const uint32_t* __restrict__ offsets, TileQueue queue) {
  extern __shared__ float4 dyn[];
  constexpr uint32_t B = kBwdBatch;
  float4* smem = dyn;                                            // [2][B][kSRec2] raster records
  float4* ex = dyn + 2 * kSRec2 * B;                             // [B][kERec] expanded records
  float* red = reinterpret_cast<float*>(ex + kERec * B);         // [kGradQ][kW2][B]
  __shared__ uint32_t max_last_w[kW2];
  __shared__ uint32_t s_slot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t tile;
  for (bool first = true; next_tile(queue, &s_slot, first, tile); first = false) {
    const Tile2 c = tile2_ctx(info, n_views, ranges, cfg, tile);
    f2_t T = f2s(1.0f);
    uint32_t last0 = 0, last1 = 0;
    const int64_t pix = c.vi.pixel_base + (int64_t)c.py * c.vi.width + c.px;
    if (RECOMPUTE) {
      f2_t Cc[3];
      forward_walk2<B>(smem, ex, raster, vals, c, cfg, Cc, T, last0, last1);
    } else {
      const float T0 = c.in0 ? t_final[pix] : 1.0f, T1 = c.in1 ? t_final[pix + c.vi.width] : 1.0f;
      T = f2(T0, T1);
      last0 = c.in0 ? n_last[pix] : 0u;
      last1 = c.in1 ? n_last[pix + c.vi.width] : 0u;
    }
    // dL/dc of the two pixels per channel (0 outside the image)
    f2_t gq[3];
    {
      const int64_t plane = (int64_t)c.vi.width * c.vi.height;
      const int64_t o = 3 * c.vi.pixel_base + (int64_t)c.py * c.vi.width + c.px;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch)
        gq[ch] = f2(c.in0 ? dL_dimg[o + ch * plane] : 0.0f, c.in1 ? dL_dimg[o + c.vi.width + ch * plane] : 0.0f);
    }
    const uint32_t warp_last = __reduce_max_sync(0xffffffffu, max(last0, last1));
    if (lane == 0) max_last_w[warp] = warp_last;
    __syncthreads();
    uint32_t max_last = 0;
#pragma unroll
    for (int w = 0; w < kW2; ++w) max_last = max(max_last, max_last_w[w]);
    const f2_t fx2 = f2s(c.fx), fy2 = f2(c.fy0, c.fy1);

    f2_t S[3] = {f2s(0.0f), f2s(0.0f), f2s(0.0f)};
    const uint32_t nb = (max_last + B - 1) / B;
    Stager2<B> st;
    if (nb > 0) {
      const uint32_t lo0 = max_last > B ? max_last - B : 0u;
      st.load(vals, c.s + lo0, (int)(max_last - lo0));
      st.issue(smem, raster);  // the forward walk's reads of smem ended at the barrier above
    }
    if (nb > 1) {
      const uint32_t hi1 = max_last - B, lo1 = hi1 > B ? hi1 - B : 0u;
      st.load(vals, c.s + lo1, (int)(hi1 - lo1));
    }
    for (uint32_t k = 0; k < nb; ++k) {
      const uint32_t top = max_last - k * B;
      const uint32_t lo = top > B ? top - B : 0u;
      const int cnt = (int)(top - lo);
      const float4* buf = smem + kSRec2 * B * (k & 1);
      if (k > 0) __syncthreads();  // batch k-1 (records, warp sums) fully consumed
      if (k + 1 < nb) {
        st.issue(smem + kSRec2 * B * ((k + 1) & 1), raster);
        cp_async_wait2<1>();
        if (k + 2 < nb) {
          const uint32_t hi2 = lo - B, lo2 = hi2 > B ? hi2 - B : 0u;
          st.load(vals, c.s + lo2, (int)(hi2 - lo2));
        }
      } else {
        cp_async_wait2<0>();
      }
      for (int q = 0; q < kGradQ; ++q)
        for (int j = lane; j < cnt; j += 32) red[(q * kW2 + warp) * B + j] = 0.0f;
      expand_own<B>(buf, ex, cnt);
      __syncthreads();  // every thread's expanded records of batch k are visible
      for (int ghi = cnt; ghi > 0; ghi -= 32) {
        const int glo = ghi > 32 ? ghi - 32 : 0;
        if (lo + (uint32_t)glo >= warp_last) continue;  // warp-uniform: nothing composited here
        const int jl = glo + lane;
        const bool cand = jl < ghi && lo + (uint32_t)jl < warp_last && block_may_pass_e(ex + kERec * jl, c.bx0, c.by0);
        uint32_t m = __ballot_sync(0xffffffffu, cand);
        while (m) {
          float v[kGradQ][kBwdChunk];
          int mypos = -1;
          bool any = false;
#pragma unroll
          for (int u = 0; u < kBwdChunk; ++u) {
#pragma unroll
            for (int q = 0; q < kGradQ; ++q) v[q][u] = 0.0f;
            if (m) {
              const int b = 31 - __clz(m);
              m &= ~(1u << b);
              const int j = glo + b;
              if (lane == u) mypos = j;
              const uint32_t pos = lo + (uint32_t)j;
              const float4* e = ex + kERec * j;
              f2_t o2;
              float thr, indef;
              const ulonglong2* qq = reinterpret_cast<const ulonglong2*>(e);
              const ulonglong2 q0 = qq[0], q1 = qq[1], q2 = qq[2];
              const f2_t dx = sub2(fx2, q1.y), dy = sub2(fy2, q2.x);
              const f2_t p2 = exponent_e(e, fx2, fy2, o2, thr, indef);
              float p0, p1;
              f2split(p2, p0, p1);
              const bool pass0 = pos < last0 && p0 >= thr, pass1 = pos < last1 && p1 >= thr;
              if (__any_sync(0xffffffffu, pass0 || pass1)) {  // warp-uniform: branch-free below
                const f2_t G2 = exp2r2_rec(p2, indef);
                const f2_t ao2 = mul2(o2, G2);
                float ao0, ao1;
                f2split(ao2, ao0, ao1);
                const float a0 = fminf(cfg.alpha_max, ao0), a1 = fminf(cfg.alpha_max, ao1);
                const bool ok0 = pass0 && a0 >= cfg.alpha_min, ok1 = pass1 && a1 >= cfg.alpha_min;
                // a pixel that does not take the splat: alpha 0 and 1 / (1 - alpha) = 1, so its
                // T and S do not change and its gradient terms are 0
                const float r0 = __fdividef(1.0f, 1.0f - a0), r1 = __fdividef(1.0f, 1.0f - a1);
                const f2_t ae = f2(ok0 ? a0 : 0.0f, ok1 ? a1 : 0.0f);
                const f2_t rcp = f2(ok0 ? r0 : 1.0f, ok1 ? r1 : 1.0f);
                T = mul2(T, rcp);          // T_i
                const f2_t w = mul2(ae, T);  // T_i alpha_i
                const ulonglong2 q3 = qq[3], q4 = qq[4];
                const f2_t cr = q3.y, cg = q4.x, cb = q4.y;
                const f2_t dot_c = fma2(cr, gq[0], fma2(cg, gq[1], mul2(cb, gq[2])));
                const f2_t dot_s = fma2(S[0], gq[0], fma2(S[1], gq[1], mul2(S[2], gq[2])));
                const f2_t dLda = sub2(mul2(T, dot_c), mul2(dot_s, rcp));
                S[0] = fma2(w, cr, S[0]);
                S[1] = fma2(w, cg, S[1]);
                S[2] = fma2(w, cb, S[2]);
                float x0, x1;
                f2split(mul2(w, gq[0]), x0, x1);
                v[6][u] = x0 + x1;
                f2split(mul2(w, gq[1]), x0, x1);
                v[7][u] = x0 + x1;
                f2split(mul2(w, gq[2]), x0, x1);
                v[8][u] = x0 + x1;
                // through alpha = o 2^p where the pixel takes the splat and the clamp is inactive;
                // elsewhere 2^p and o 2^p are replaced by 0 (a pixel that did not pass may hold
                // any value there)
                float G0, G1;
                f2split(G2, G0, G1);
                const bool f0 = ok0 && ao0 <= cfg.alpha_max, f1 = ok1 && ao1 <= cfg.alpha_max;
                const f2_t Gm = f2(f0 ? G0 : 0.0f, f1 ? G1 : 0.0f), aom = f2(f0 ? ao0 : 0.0f, f1 ? ao1 : 0.0f);
                f2split(mul2(dLda, Gm), x0, x1);
                v[5][u] = x0 + x1;
                const f2_t dLdp = mul2(mul2(dLda, aom), f2s(kLn2));
                const f2_t dxx = mul2(dx, dx), dxy = mul2(dx, dy), dyy = mul2(dy, dy);
                f2split(mul2(dLdp, dxx), x0, x1);
                v[2][u] = x0 + x1;
                f2split(mul2(dLdp, dxy), x0, x1);
                v[3][u] = x0 + x1;
                f2split(mul2(dLdp, dyy), x0, x1);
                v[4][u] = x0 + x1;
                const f2_t A2 = q0.x, B2 = q0.y, C2 = q1.x;
                const f2_t gx = fma2(add2(A2, A2), dx, mul2(B2, dy));  // 2 A dx + B dy
                const f2_t gy = fma2(B2, dx, mul2(add2(C2, C2), dy));  // B dx + 2 C dy
                f2split(mul2(dLdp, gx), x0, x1);
                v[0][u] = -(x0 + x1);
                f2split(mul2(dLdp, gy), x0, x1);
                v[1][u] = -(x0 + x1);
                any = true;
              }
            }
          }
          if (__any_sync(0xffffffffu, any)) {
#pragma unroll
            for (int q = 0; q < kGradQ; ++q) {
              const float sq = warp_transpose_sum4(v[q]);
              if (lane < kBwdChunk && mypos >= 0) red[(q * kW2 + warp) * B + mypos] = sq;
            }
          }
        }
      }
      __syncthreads();
      for (int j = threadIdx.x; j < cnt; j += kT2) {
        float sq[kGradQ];
        bool nz = false;
#pragma unroll
        for (int q = 0; q < kGradQ; ++q) {
          float t = 0.0f;
#pragma unroll
          for (int w = 0; w < kW2; ++w) t += red[(q * kW2 + w) * B + j];
          sq[q] = t;
          nz |= t != 0.0f;
        }
        if (nz) {
          const uint32_t vk = vals[c.s + lo + j];
          const uint32_t slot = emission_slot(offsets[vk], cull[vk], c.tx, c.ty);  // L2
          float* dst = inst_grad + (int64_t)slot * kGradQ;  // the slot's nine partials, contiguous
#pragma unroll
          for (int q = 0; q < kGradQ; ++q) dst[q] = sq[q];
        }
      }
    }
  }  // tiles
}

// ---------------------------------------------------------------------------------------
// K10: per-splat adjoint of projection, colour and activation
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void sh_basis16(float x, float y, float z, float* Y) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = 0.28209479177387814f;
  Y[1] = -0.4886025119029199f * y;
  Y[2] = 0.4886025119029199f * z;
  Y[3] = -0.4886025119029199f * x;
  Y[4] = 1.0925484305920792f * x * y;
  Y[5] = -1.0925484305920792f * y * z;
  Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
  Y[7] = -1.0925484305920792f * x * z;
  Y[8] = 0.5462742152960396f * (xx - yy);
  Y[9] = -0.5900435899266435f * y * (3.0f * xx - yy);
  Y[10] = 2.890611442640554f * x * y * z;
  Y[11] = -0.4570457994644658f * y * (4.0f * zz - xx - yy);
  Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
  Y[13] = -0.4570457994644658f * x * (4.0f * zz - xx - yy);
  Y[14] = 1.445305721320277f * z * (xx - yy);
  Y[15] = -0.5900435899266435f * x * (xx - 3.0f * yy);
}

// sum_i w_i grad Y_i(x, y, z) with the basis polynomials differentiated term by term.
__device__ __forceinline__ void sh_weighted_grad(float x, float y, float z, const float* w, float& gx, float& gy,
                                                 float& gz) {
  const float c1 = 0.4886025119029199f, c2a = 1.0925484305920792f, c2b = 0.31539156525252005f;
  const float c2c = 0.5462742152960396f, c3a = 0.5900435899266435f, c3b = 2.890611442640554f;
  const float c3c = 0.4570457994644658f, c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
  const float xx = x * x, yy = y * y, zz = z * z;
  gx = 0.0f; gy = 0.0f; gz = 0.0f;
  gy += w[1] * -c1;
  gz += w[2] * c1;
  gx += w[3] * -c1;
  gx += w[4] * c2a * y;            gy += w[4] * c2a * x;
  gy += w[5] * -c2a * z;           gz += w[5] * -c2a * y;
  gx += w[6] * -2.0f * c2b * x;    gy += w[6] * -2.0f * c2b * y;    gz += w[6] * 4.0f * c2b * z;
  gx += w[7] * -c2a * z;           gz += w[7] * -c2a * x;
  gx += w[8] * 2.0f * c2c * x;     gy += w[8] * -2.0f * c2c * y;
  gx += w[9] * -6.0f * c3a * x * y;                gy += w[9] * -3.0f * c3a * (xx - yy);
  gx += w[10] * c3b * y * z;       gy += w[10] * c3b * x * z;       gz += w[10] * c3b * x * y;
  gx += w[11] * 2.0f * c3c * x * y;                gy += w[11] * -c3c * (4.0f * zz - xx - 3.0f * yy);
  gz += w[11] * -8.0f * c3c * y * z;
  gx += w[12] * -6.0f * c3d * x * z;               gy += w[12] * -6.0f * c3d * y * z;
  gz += w[12] * c3d * (6.0f * zz - 3.0f * xx - 3.0f * yy);
  gx += w[13] * -c3c * (4.0f * zz - 3.0f * xx - yy);                gy += w[13] * 2.0f * c3c * x * y;
  gz += w[13] * -8.0f * c3c * x * z;
  gx += w[14] * 2.0f * c3e * x * z;                gy += w[14] * -2.0f * c3e * y * z;
  gz += w[14] * c3e * (xx - yy);
  gx += w[15] * -3.0f * c3a * (xx - yy);           gy += w[15] * 6.0f * c3a * x * y;
}

// Per (view, splat): the nine instance partials summed over the vk's emission slots, then the
// view-dependent part of the adjoint.  One warp per 32 consecutive vk, whose slots form one
// contiguous run (vk order): the run is read 32 slots at a time, one slot (nine contiguous
// floats) per lane, and summed per vk by a segmented scan across the lanes (a fixed tree per
// chunk, chunks in order).  Each lane then takes its vk through the adjoint of the conic
// inverse, of Sigma2D = T Sigma T^T (T = J W, J with the clamped x/z, y/z) and of the pinhole
// centre.  out[vk][0..12] receives d/dmean (3), d/dSigma (6: 00 01 02 11 12 22), d/do (1) and
// d/dcolour (3); all zero where no pixel of the view took the splat.
constexpr int kVkOut = 13;
constexpr int kVkThreads = 256;

__global__ void __launch_bounds__(kVkThreads) vk_bwd_kernel(const uint32_t* __restrict__ touched,
                                                     const uint32_t* __restrict__ offsets,
                                                     const uint32_t* __restrict__ n_inst, int64_t capacity, int64_t n,
                                                     int n_views, const float* __restrict__ inst_grad,
                                                     const float* __restrict__ means, const float* __restrict__ cov3d,
                                                     const potr_camera* __restrict__ cams, potr_raster_config cfg,
                                                     float* __restrict__ out) {
  const bool ok = (int64_t)*n_inst <= capacity;
  const int lane = threadIdx.x & 31;
  const int64_t n_vk = (int64_t)n_views * n;
  const int64_t warps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float kA = -0.5f * kLog2e;
  for (int64_t wv = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wv * 32 < n_vk; wv += warps_total) {
    const int64_t vk = wv * 32 + lane;
    uint32_t cnt = 0, off = 0;
    if (ok && vk < n_vk) {  // independent loads: the run starts at lane 0's offset whatever its count
      cnt = touched[vk];
      off = offsets[vk];
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t seg0 = incl - cnt, seg1 = incl;  // my segment inside the warp's run
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t run0 = __shfl_sync(0xffffffffu, off, 0);  // offsets are the exclusive prefix in vk order
    float gq[kGradQ];
#pragma unroll
    for (int q = 0; q < kGradQ; ++q) gq[q] = 0.0f;
    // the chunk's partials, loaded one chunk ahead of its scan
    float nx[kGradQ];
#pragma unroll
    for (int q = 0; q < kGradQ; ++q) nx[q] = lane < total ? inst_grad[(int64_t)(run0 + lane) * kGradQ + q] : 0.0f;
    for (uint32_t c0 = 0; c0 < total; c0 += 32) {
      const uint32_t e = c0 + lane;
      float x[kGradQ];
#pragma unroll
      for (int q = 0; q < kGradQ; ++q) x[q] = nx[q];
      if (c0 + 32 < total) {
        const uint32_t en = e + 32;
#pragma unroll
        for (int q = 0; q < kGradQ; ++q) nx[q] = en < total ? inst_grad[(int64_t)(run0 + en) * kGradQ + q] : 0.0f;
      }
      // the owner of slot e is the last lane whose segment starts at or before e; its segment
      // starts at lane `head` of this chunk
      uint32_t owner = 0;
#pragma unroll
      for (int b = 16; b >= 1; b >>= 1) {
        const uint32_t cand = owner + b;
        const uint32_t cs = __shfl_sync(0xffffffffu, seg0, cand & 31);
        if (cand < 32 && cs <= e) owner = cand;
      }
      const uint32_t os = __shfl_sync(0xffffffffu, seg0, owner);
      const int head = os > c0 ? (int)(os - c0) : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const bool take = lane - d >= head;
#pragma unroll
        for (int q = 0; q < kGradQ; ++q) {
          const float y = __shfl_up_sync(0xffffffffu, x[q], d);
          if (take) x[q] += y;
        }
      }
      // my segment's slots in this chunk end at lane hi - 1 - c0, which now holds their sum
      const uint32_t lo = max(seg0, c0), hi = min(seg1, c0 + 32u);
      const int src_lane = lo < hi ? (int)(hi - 1u - c0) : lane;
#pragma unroll
      for (int q = 0; q < kGradQ; ++q) {
        const float y = __shfl_sync(0xffffffffu, x[q], src_lane);
        if (lo < hi) gq[q] += y;
      }
    }
    float res[kVkOut];
#pragma unroll
    for (int q = 0; q < kVkOut; ++q) res[q] = 0.0f;
    bool nz = false;
#pragma unroll
    for (int q = 0; q < kGradQ; ++q) nz |= gq[q] != 0.0f;
    if (vk < n_vk && cnt && nz) {
      const int v = (int)((uint32_t)vk / (uint32_t)n);  // n_views * n < 2^32
      const int64_t k = vk - (int64_t)v * n;
      const float mu[3] = {means[k], means[n + k], means[2 * n + k]};
      const float Sg[3][3] = {{cov3d[k], cov3d[n + k], cov3d[2 * n + k]},
                              {cov3d[n + k], cov3d[3 * n + k], cov3d[4 * n + k]},
                              {cov3d[2 * n + k], cov3d[4 * n + k], cov3d[5 * n + k]}};
      const potr_camera& cam = cams[v];
      const float* W = cam.w2c;
      // forward recomputation (values only)
      float t[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) t[i] = W[i * 4] * mu[0] + W[i * 4 + 1] * mu[1] + W[i * 4 + 2] * mu[2] + W[i * 4 + 3];
      const float lim_x = 1.3f * (0.5f * (float)cam.width / cam.fx);
      const float lim_y = 1.3f * (0.5f * (float)cam.height / cam.fy);
      const float iz = 1.0f / t[2], iz2 = iz * iz, iz3 = iz2 * iz;
      const float txz = t[0] * iz, tyz = t[1] * iz;
      const bool inx = txz >= -lim_x && txz <= lim_x;
      const bool iny = tyz >= -lim_y && tyz <= lim_y;
      const float xc = fminf(lim_x, fmaxf(-lim_x, txz)) * t[2];
      const float yc = fminf(lim_y, fmaxf(-lim_y, tyz)) * t[2];
      const float j00 = cam.fx * iz, j02 = -cam.fx * xc * iz2, j11 = cam.fy * iz, j12 = -cam.fy * yc * iz2;
      float Tm[2][3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Tm[0][j] = j00 * W[j] + j02 * W[8 + j];
        Tm[1][j] = j11 * W[4 + j] + j12 * W[8 + j];
      }
      float TS[2][3];  // T Sigma
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) TS[i][j] = Tm[i][0] * Sg[0][j] + Tm[i][1] * Sg[1][j] + Tm[i][2] * Sg[2][j];
      const float a = TS[0][0] * Tm[0][0] + TS[0][1] * Tm[0][1] + TS[0][2] * Tm[0][2] + cfg.lowpass;
      const float b = TS[0][0] * Tm[1][0] + TS[0][1] * Tm[1][1] + TS[0][2] * Tm[1][2];
      const float cc2 = TS[1][0] * Tm[1][0] + TS[1][1] * Tm[1][1] + TS[1][2] * Tm[1][2] + cfg.lowpass;
      const float idet = 1.0f / (a * cc2 - b * b);
      const float ca = cc2 * idet, cb = -b * idet, cc = a * idet;
      // conic and Sigma2D adjoint
      const float gca = kA * gq[2], gcb = -kLog2e * gq[3], gcc = kA * gq[4];
      const float ga = -(gca * ca * ca + gcb * ca * cb + gcc * cb * cb);
      const float gc = -(gca * cb * cb + gcb * cb * cc + gcc * cc * cc);
      const float gb = -(2.0f * gca * ca * cb + gcb * (ca * cc + cb * cb) + 2.0f * gcc * cb * cc);
      const float G2[2][2] = {{ga, 0.5f * gb}, {0.5f * gb, gc}};
      // Sigma gradient T^T G2 T (symmetric: the six entries on and above the diagonal)
      float G2T[2][3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        G2T[0][j] = G2[0][0] * Tm[0][j] + G2[0][1] * Tm[1][j];
        G2T[1][j] = G2[1][0] * Tm[0][j] + G2[1][1] * Tm[1][j];
      }
      const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int e6 = 0; e6 < 6; ++e6)
        res[3 + e6] = Tm[0][ii[e6]] * G2T[0][jj[e6]] + Tm[1][ii[e6]] * G2T[1][jj[e6]];
      // T gradient 2 G2 T Sigma, then J gradient (dL/dT) W_rot^T
      float gT[2][3];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) gT[i][j] = 2.0f * (G2[i][0] * TS[0][j] + G2[i][1] * TS[1][j]);
      const float gj00 = gT[0][0] * W[0] + gT[0][1] * W[1] + gT[0][2] * W[2];
      const float gj02 = gT[0][0] * W[8] + gT[0][1] * W[9] + gT[0][2] * W[10];
      const float gj11 = gT[1][0] * W[4] + gT[1][1] * W[5] + gT[1][2] * W[6];
      const float gj12 = gT[1][0] * W[8] + gT[1][1] * W[9] + gT[1][2] * W[10];
      float gt[3] = {0.0f, 0.0f, 0.0f};
      gt[2] += -gj00 * cam.fx * iz2 - gj11 * cam.fy * iz2;
      if (inx) {
        gt[0] += -gj02 * cam.fx * iz2;
        gt[2] += gj02 * 2.0f * cam.fx * xc * iz3;
      } else {
        gt[2] += gj02 * cam.fx * xc * iz3;
      }
      if (iny) {
        gt[1] += -gj12 * cam.fy * iz2;
        gt[2] += gj12 * 2.0f * cam.fy * yc * iz3;
      } else {
        gt[2] += gj12 * cam.fy * yc * iz3;
      }
      // pixel-space centre
      gt[0] += gq[0] * cam.fx * iz;
      gt[1] += gq[1] * cam.fy * iz;
      gt[2] += -gq[0] * cam.fx * t[0] * iz2 - gq[1] * cam.fy * t[1] * iz2;
#pragma unroll
      for (int j = 0; j < 3; ++j) res[j] = W[j] * gt[0] + W[4 + j] * gt[1] + W[8 + j] * gt[2];
      res[9] = gq[5];
      res[10] = gq[6];
      res[11] = gq[7];
      res[12] = gq[8];
    }
    if (vk < n_vk) {
#pragma unroll
      for (int q = 0; q < kVkOut; ++q) out[vk * kVkOut + q] = res[q];
    }
  }
}

// Per splat: the per-view results summed in view order, the SH colour adjoint (clamp mask,
// coefficients and the direction from the camera), then the activation adjoint (Sigma = M M^T,
// M = R diag(exp(log_scale)), quaternion normalisation, sigmoid).  A block takes 32 splats with
// one warp per colour channel: warp c holds the 16 coefficients of channel c and their 16
// gradients, and its share of the direction gradient (linear in the weighted coefficients);
// warp 0 adds the three shares in channel order and finishes the splat.
constexpr int kSplatBwdThreads = 96;

__global__ void __launch_bounds__(kSplatBwdThreads, 6) splat_bwd_kernel(
    const float* __restrict__ means, const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ sh, const float* __restrict__ opacity, int64_t n, const potr_camera* __restrict__ cams,
    int n_views, const float* __restrict__ vk_res, float* __restrict__ g_means, float* __restrict__ g_log_scales,
    float* __restrict__ g_quats, float* __restrict__ g_logits, float* __restrict__ g_sh) {
  __shared__ float s_gdir[2][3][32];  // channels 1 and 2: their direction gradients
  const int lane = threadIdx.x & 31, ch = threadIdx.x >> 5;
  for (int64_t k0 = (int64_t)blockIdx.x * 32; k0 < n; k0 += (int64_t)gridDim.x * 32) {
    const int64_t k = k0 + lane;
    const bool live = k < n;
    float gp[3] = {0.0f, 0.0f, 0.0f}, gd[3] = {0.0f, 0.0f, 0.0f};
    float G6[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float go = 0.0f;
    float gsh[16], shc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) gsh[i] = 0.0f;
    bool used = false;
    float mu[3] = {0.0f, 0.0f, 0.0f};
    if (live) {
#pragma unroll
      for (int i = 0; i < 16; ++i) shc[i] = __ldg(sh + (int64_t)(i * 3 + ch) * n + k);
      mu[0] = means[k];
      mu[1] = means[n + k];
      mu[2] = means[2 * n + k];
    }
    float rn[kVkOut];  // the next view's values, loaded one view ahead
    if (live) {
#pragma unroll
      for (int q = 0; q < kVkOut; ++q) rn[q] = vk_res[k * kVkOut + q];
    }
#pragma unroll 1
    for (int v = 0; live && v < n_views; ++v) {
      float r[kVkOut];
      bool nz = false;
#pragma unroll
      for (int q = 0; q < kVkOut; ++q) {
        r[q] = rn[q];
        nz |= r[q] != 0.0f;
      }
      if (v + 1 < n_views) {
        const int64_t vk1 = (int64_t)(v + 1) * n + k;
#pragma unroll
        for (int q = 0; q < kVkOut; ++q) rn[q] = vk_res[vk1 * kVkOut + q];
      }
      if (!nz) continue;
      used = true;
      if (ch == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) gp[j] += r[j];
#pragma unroll
        for (int e6 = 0; e6 < 6; ++e6) G6[e6] += r[3 + e6];
        go += r[9];
      }
      // colour of this channel: clamp mask, coefficients, direction
      const float* W = cams[v].w2c;
      float cpos[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) cpos[j] = -(W[j] * W[3] + W[4 + j] * W[7] + W[8 + j] * W[11]);
      const float u0 = mu[0] - cpos[0], u1 = mu[1] - cpos[1], u2 = mu[2] - cpos[2];
      const float inv_len = rsqrtf(u0 * u0 + u1 * u1 + u2 * u2);
      const float dx = u0 * inv_len, dy = u1 * inv_len, dz = u2 * inv_len;
      float Y[16];
      sh_basis16(dx, dy, dz, Y);
      float acc = 0.0f;
#pragma unroll
      for (int i = 0; i < 16; ++i) acc = fmaf(shc[i], Y[i], acc);
      const float gcol = ch == 0 ? r[10] : (ch == 1 ? r[11] : r[12]);  // (no dynamic register index)
      const float gv = (acc + 0.5f > 0.0f) ? gcol : 0.0f;
#pragma unroll
      for (int i = 0; i < 16; ++i) gsh[i] += gv * Y[i];
      if (gv != 0.0f) {  // d colour / d direction = sum_i shc_i grad Y_i, times gv
        float gdx, gdy, gdz;
        sh_weighted_grad(dx, dy, dz, shc, gdx, gdy, gdz);
        gdx *= gv;
        gdy *= gv;
        gdz *= gv;
        const float dotg = gdx * dx + gdy * dy + gdz * dz;
        gd[0] += (gdx - dx * dotg) * inv_len;
        gd[1] += (gdy - dy * dotg) * inv_len;
        gd[2] += (gdz - dz * dotg) * inv_len;
      }
    }
    if (ch > 0) {
#pragma unroll
      for (int j = 0; j < 3; ++j) s_gdir[ch - 1][j][lane] = gd[j];
    }
    __syncthreads();
    if (live) {
#pragma unroll
      for (int i = 0; i < 16; ++i) g_sh[(int64_t)(i * 3 + ch) * n + k] = used ? gsh[i] : 0.0f;
    }
    if (live && ch == 0) {
      if (!used) {  // no pixel of any view took the splat (also a splat culled for non-finite parameters)
#pragma unroll
        for (int j = 0; j < 3; ++j) g_means[j * n + k] = g_log_scales[j * n + k] = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) g_quats[j * n + k] = 0.0f;
        g_logits[k] = 0.0f;
      } else {
        float gmu[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) gmu[j] = gp[j] + ((gd[j] + s_gdir[0][j][lane]) + s_gdir[1][j][lane]);
        const float G3[3][3] = {{G6[0], G6[1], G6[2]}, {G6[1], G6[3], G6[4]}, {G6[2], G6[4], G6[5]}};
        // activation adjoint: Sigma = M M^T, M = R diag(s), s = exp(log_scale), R(q / |q|)
        float s[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) s[j] = expf(log_scales[j * n + k]);
        float qw = quats[k], qx = quats[n + k], qy = quats[2 * n + k], qz = quats[3 * n + k];
        const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float iqn = qn > 0.0f ? 1.0f / qn : 0.0f;
        qw *= iqn; qx *= iqn; qy *= iqn; qz *= iqn;
        const float R[3][3] = {{1.0f - 2.0f * (qy * qy + qz * qz), 2.0f * (qx * qy - qw * qz), 2.0f * (qx * qz + qw * qy)},
                               {2.0f * (qx * qy + qw * qz), 1.0f - 2.0f * (qx * qx + qz * qz), 2.0f * (qy * qz - qw * qx)},
                               {2.0f * (qx * qz - qw * qy), 2.0f * (qy * qz + qw * qx), 1.0f - 2.0f * (qx * qx + qy * qy)}};
        float gs[3] = {0.0f, 0.0f, 0.0f};
        float gR[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            // dL/dM_ij = 2 (G3 M)_ij with M_lj = R_lj s_j
            const float gM = 2.0f * (G3[i][0] * R[0][j] + G3[i][1] * R[1][j] + G3[i][2] * R[2][j]) * s[j];
            gs[j] += gM * R[i][j];
            gR[i][j] = gM * s[j];
          }
        const float gqw = 2.0f * (-qz * gR[0][1] + qy * gR[0][2] + qz * gR[1][0] - qx * gR[1][2] - qy * gR[2][0] + qx * gR[2][1]);
        const float gqx = 2.0f * (qy * gR[0][1] + qz * gR[0][2] + qy * gR[1][0] - 2.0f * qx * gR[1][1] - qw * gR[1][2] +
                                  qz * gR[2][0] + qw * gR[2][1] - 2.0f * qx * gR[2][2]);
        const float gqy = 2.0f * (-2.0f * qy * gR[0][0] + qx * gR[0][1] + qw * gR[0][2] + qx * gR[1][0] + qz * gR[1][2] -
                                  qw * gR[2][0] + qz * gR[2][1] - 2.0f * qy * gR[2][2]);
        const float gqz = 2.0f * (-2.0f * qz * gR[0][0] - qw * gR[0][1] + qx * gR[0][2] + qw * gR[1][0] - 2.0f * qz * gR[1][1] +
                                  qy * gR[1][2] + qx * gR[2][0] + qy * gR[2][1]);
        const float dq = gqw * qw + gqx * qx + gqy * qy + gqz * qz;
        g_quats[k] = (gqw - qw * dq) * iqn;
        g_quats[n + k] = (gqx - qx * dq) * iqn;
        g_quats[2 * n + k] = (gqy - qy * dq) * iqn;
        g_quats[3 * n + k] = (gqz - qz * dq) * iqn;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          g_log_scales[j * n + k] = gs[j] * s[j];
          g_means[j * n + k] = gmu[j];
        }
        const float o = opacity[k];
        g_logits[k] = go * o * (1.0f - o);
      }
    }
    __syncthreads();  // s_gdir is rewritten by the next group of splats
  }
}

}  // namespace
}  // namespace potr

extern "C" size_t potr_loss_workspace_size(int64_t total_pixels) {
  (void)total_pixels;
  return sizeof(double) * potr::kLossBlocks;
}

extern "C" potr_status potr_loss_grad(const potr_frame* frame, const float* d_images, const float* d_targets,
                                      float lambda, double* d_loss, float* d_dL_dimages, void* d_ws, size_t ws_bytes,
                                      potr_stream_t stream) {
  using namespace potr;
  if (!frame || !d_images || !d_targets || !d_dL_dimages || frame->total_pixels <= 0) return POTR_ERR_INVALID_ARGUMENT;
  if (!(lambda >= 0.0f && lambda <= 1.0f)) return POTR_ERR_INVALID_ARGUMENT;
  if (d_loss && (!d_ws || ws_bytes < sizeof(double) * kLossBlocks)) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n_elems = 3 * frame->total_pixels;
  double* block_sums = d_loss ? static_cast<double*>(d_ws) : nullptr;
  loss_grad_kernel<<<kLossBlocks, 256, 0, s>>>(d_images, d_targets, n_elems, lambda, d_dL_dimages, block_sums);
  POTR_CHECK_LAUNCH();
  if (d_loss) {
    loss_finish_kernel<<<1, 256, 0, s>>>(block_sums, kLossBlocks, n_elems, d_loss);
    POTR_CHECK_LAUNCH();
  }
  return POTR_OK;
}

extern "C" size_t potr_render_backward_workspace_size(int64_t instance_capacity, int64_t n_view_splats) {
  if (instance_capacity <= 0 || n_view_splats <= 0) return 0;
  return sizeof(float) * ((size_t)potr::kGradQ * (size_t)instance_capacity +
                          (size_t)potr::kVkOut * (size_t)n_view_splats);
}

extern "C" potr_status potr_render_backward(const potr_scene* scene, const potr_views* views, const potr_frame* frame,
                                            const potr_raster_config* cfg, const uint32_t* d_vals,
                                            const uint32_t* d_tile_ranges, uint32_t* d_tile_order,
                                            const float* d_t_final,
                                            const uint32_t* d_n_last, const float* d_dL_dimages,
                                            int64_t instance_capacity, const potr_scene_grads* grads, void* d_ws,
                                            size_t ws_bytes, potr_stream_t stream) {
  using namespace potr;
  if (!scene || !views || !frame || !valid_cfg(cfg) || !grads || !d_vals || !d_tile_ranges || !d_dL_dimages)
    return POTR_ERR_INVALID_ARGUMENT;
  if (!scene->means || !scene->log_scales || !scene->quats || !scene->sh || scene->n <= 0) return POTR_ERR_INVALID_ARGUMENT;
  if (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits || !grads->sh)
    return POTR_ERR_INVALID_ARGUMENT;
  if (!views->raster || !views->cov3d || !views->opacity || !views->touched || !views->offsets || !views->n_instances ||
      !views->cull)
    return POTR_ERR_INVALID_ARGUMENT;
  if ((d_t_final == nullptr) != (d_n_last == nullptr)) return POTR_ERR_INVALID_ARGUMENT;
  if (frame->total_tiles <= 0 || frame->total_tiles > 0x7fffffffll || !frame->cams || !frame->info)
    return POTR_ERR_INVALID_ARGUMENT;
  const int64_t n_vk = (int64_t)frame->n_views * scene->n;
  if (instance_capacity <= 0 || !d_ws || ws_bytes < potr_render_backward_workspace_size(instance_capacity, n_vk))
    return POTR_ERR_INVALID_ARGUMENT;
  const size_t inst_bytes = sizeof(float) * (size_t)kGradQ * (size_t)instance_capacity;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* inst_grad = static_cast<float*>(d_ws);
  if (cudaMemsetAsync(inst_grad, 0, inst_bytes, s) != cudaSuccess) return POTR_ERR_CUDA;
  const size_t smem = bwd_smem_bytes();
  const bool recompute = d_t_final == nullptr;
  TileQueue q;
  q.order = d_tile_order;
  q.counter = d_tile_order ? d_tile_order + frame->total_tiles : nullptr;
  q.total = (uint32_t)frame->total_tiles;
  if (d_tile_order && cudaMemsetAsync(q.counter, 0, sizeof(uint32_t), s) != cudaSuccess) return POTR_ERR_CUDA;
  if (recompute) {
    if (cudaFuncSetAttribute(render_bwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return POTR_ERR_CUDA;
    const unsigned grid = tile_grid(render_bwd_kernel<true>, smem, q, frame->total_tiles, kT2);
    tile_timing_begin(s);
    render_bwd_kernel<true><<<grid, kT2, smem, s>>>(
        reinterpret_cast<const float4*>(views->raster), d_vals, d_tile_ranges, frame->info, frame->n_views, *cfg,
        nullptr, nullptr, d_dL_dimages, instance_capacity, inst_grad, reinterpret_cast<const uint4*>(views->cull),
        views->offsets, q);
    tile_timing_end(s);
  } else {
    if (cudaFuncSetAttribute(render_bwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return POTR_ERR_CUDA;
    const unsigned grid = tile_grid(render_bwd_kernel<false>, smem, q, frame->total_tiles, kT2);
    tile_timing_begin(s);
    render_bwd_kernel<false><<<grid, kT2, smem, s>>>(
        reinterpret_cast<const float4*>(views->raster), d_vals, d_tile_ranges, frame->info, frame->n_views, *cfg,
        d_t_final, d_n_last, d_dL_dimages, instance_capacity, inst_grad, reinterpret_cast<const uint4*>(views->cull),
        views->offsets, q);
    tile_timing_end(s);
  }
  POTR_CHECK_LAUNCH();
  const int64_t n = scene->n;
  float* vk_res = reinterpret_cast<float*>(static_cast<char*>(d_ws) + inst_bytes);
  {
    int64_t gw = (n_vk + kVkThreads - 1) / kVkThreads;
    if (gw > 152 * 8) gw = 152 * 8;
    vk_bwd_kernel<<<(unsigned)gw, kVkThreads, 0, s>>>(views->touched, views->offsets, views->n_instances, instance_capacity,
                                               n, frame->n_views, inst_grad, scene->means, views->cov3d, frame->cams,
                                               *cfg, vk_res);
    POTR_CHECK_LAUNCH();
  }
  int64_t g = (n + 31) / 32;
  if (g > 152 * 64) g = 152 * 64;
  splat_bwd_kernel<<<(unsigned)g, kSplatBwdThreads, 0, s>>>(scene->means, scene->log_scales, scene->quats, scene->sh,
                                               views->opacity, n, frame->cams, frame->n_views, vk_res, grads->means,
                                               grads->log_scales, grads->quats, grads->opacity_logits, grads->sh);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
