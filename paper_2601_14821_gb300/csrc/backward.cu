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
//   vk_grad_sum_kernel    per (view, splat): its instance slots summed in emission order.
//   preprocess_bwd_kernel per splat: the adjoint of the projection (conic inverse, Sigma2D = T Sigma T^T,
//                         clamped Jacobian, pinhole centre, SH colour and its direction) and of
//                         the activation (Sigma = M M^T, M = R diag(exp(log_scale)), quaternion
//                         normalisation, sigmoid), accumulated over views in view order.
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
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_elems; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = img[i] - tgt[i];
    const float sg = (r > 0.0f) ? 1.0f : ((r < 0.0f) ? -1.0f : 0.0f);
    grad[i] = ((1.0f - lam) * sg + 2.0f * lam * r) * inv_n;
    acc += (double)((1.0f - lam) * fabsf(r) + lam * r * r);
  }
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

__global__ void loss_finish_kernel(const double* __restrict__ block_sums, int nb, int64_t n_elems,
                                   double* __restrict__ loss) {
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += block_sums[b];
  *loss = s / (double)n_elems;
}

// ---------------------------------------------------------------------------------------
// K9: back-to-front adjoint of the compositing
// ---------------------------------------------------------------------------------------
template <bool RECOMPUTE>
__global__ void __launch_bounds__(kT2, 5) render_bwd_kernel(const float4* __restrict__ raster,
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
#pragma unroll
          for (int q = 0; q < kGradQ; ++q) inst_grad[(int64_t)q * capacity + slot] = sq[q];
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

// Per (view, splat): the nine instance partials summed over the vk's emission slots (emission
// order, compensated).  One warp per 32 consecutive vk, whose slots form one contiguous run:
// the run is read coalesced into shared memory a chunk at a time and each lane adds the part of
// its own segment that the chunk holds.  vk_grad[q][vk] receives the sums.
constexpr int kSumChunk = 128;  // a warp's run is usually shorter (about 32 x 3.5 slots)

__global__ void __launch_bounds__(128, 8) vk_grad_sum_kernel(const uint32_t* __restrict__ touched,
                                                          const uint32_t* __restrict__ offsets,
                                                          const uint32_t* __restrict__ n_inst, int64_t capacity,
                                                          int64_t n_vk, const float* __restrict__ inst_grad,
                                                          float* __restrict__ vk_grad) {
  __shared__ float buf[4][kGradQ][kSumChunk];
  const bool ok = (int64_t)*n_inst <= capacity;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wv = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wv * 32 < n_vk; wv += warps_total) {
    const int64_t vk = wv * 32 + lane;
    uint32_t cnt = 0, off = 0;
    if (ok && vk < n_vk) {
      cnt = touched[vk];
      if (cnt) off = offsets[vk];
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t seg0 = incl - cnt, seg1 = incl;  // my segment inside the warp's run
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t first_lane = total ? __ffs(__ballot_sync(0xffffffffu, cnt != 0)) - 1 : 0;
    const uint32_t run0 = __shfl_sync(0xffffffffu, off, first_lane);
    KahanSum acc[kGradQ];
    for (uint32_t c0 = 0; c0 < total; c0 += kSumChunk) {
      const uint32_t cn = min((uint32_t)kSumChunk, total - c0);
      for (uint32_t i = lane; i < cn; i += 32)
#pragma unroll
        for (int q = 0; q < kGradQ; ++q) buf[wib][q][i] = inst_grad[(int64_t)q * capacity + run0 + c0 + i];
      __syncwarp();
      const uint32_t a = max(seg0, c0), b = min(seg1, c0 + cn);
      for (uint32_t i = a; i < b; ++i)
#pragma unroll
        for (int q = 0; q < kGradQ; ++q) acc[q].add(buf[wib][q][i - c0]);
      __syncwarp();
    }
    if (vk < n_vk) {
#pragma unroll
      for (int q = 0; q < kGradQ; ++q) vk_grad[(int64_t)q * n_vk + vk] = (float)acc[q].value();
    }
  }
}

__global__ void __launch_bounds__(128, 3) preprocess_bwd_kernel(
    const float* __restrict__ means, const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ sh, const float* __restrict__ cov3d, const float* __restrict__ opacity, int64_t n,
    const potr_camera* __restrict__ cams, int n_views, potr_raster_config cfg, const uint32_t* __restrict__ touched,
    const float* __restrict__ vk_grad, float* __restrict__ g_means, float* __restrict__ g_log_scales,
    float* __restrict__ g_quats, float* __restrict__ g_logits, float* __restrict__ g_sh) {
  const float kA = -0.5f * kLog2e;
  const int64_t n_vk = (int64_t)n_views * n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    float gmu[3] = {0.0f, 0.0f, 0.0f};
    float G3[3][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    float go = 0.0f;
    float gsh[48], shc[48];
#pragma unroll
    for (int i = 0; i < 48; ++i) gsh[i] = 0.0f;
    bool have_sh = false, used = false;
    const float mu[3] = {means[k], means[n + k], means[2 * n + k]};
    const float Sg[3][3] = {{cov3d[k], cov3d[n + k], cov3d[2 * n + k]},
                            {cov3d[n + k], cov3d[3 * n + k], cov3d[4 * n + k]},
                            {cov3d[2 * n + k], cov3d[4 * n + k], cov3d[5 * n + k]}};
    for (int v = 0; v < n_views; ++v) {
      const int64_t vk = (int64_t)v * n + k;
      if (!touched[vk]) continue;
      float gq[kGradQ];
      bool nz = false;
#pragma unroll
      for (int q = 0; q < kGradQ; ++q) {
        gq[q] = vk_grad[(int64_t)q * n_vk + vk];
        nz |= gq[q] != 0.0f;
      }
      if (!nz) continue;
      used = true;
      if (!have_sh) {
#pragma unroll
        for (int i = 0; i < 48; ++i) shc[i] = __ldg(sh + (int64_t)i * n + k);
        have_sh = true;
      }
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
      // Sigma gradient T^T G2 T
      float G2T[2][3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        G2T[0][j] = G2[0][0] * Tm[0][j] + G2[0][1] * Tm[1][j];
        G2T[1][j] = G2[1][0] * Tm[0][j] + G2[1][1] * Tm[1][j];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) G3[i][j] += Tm[0][i] * G2T[0][j] + Tm[1][i] * G2T[1][j];
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
      for (int j = 0; j < 3; ++j) gmu[j] += W[j] * gt[0] + W[4 + j] * gt[1] + W[8 + j] * gt[2];
      // colour: clamp mask, SH coefficients, direction
      float shc_w[16];
      float cpos[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) cpos[j] = -(W[j] * W[3] + W[4 + j] * W[7] + W[8 + j] * W[11]);
      const float u0 = mu[0] - cpos[0], u1 = mu[1] - cpos[1], u2 = mu[2] - cpos[2];
      const float inv_len = rsqrtf(u0 * u0 + u1 * u1 + u2 * u2);
      const float dx = u0 * inv_len, dy = u1 * inv_len, dz = u2 * inv_len;
      float Y[16];
      sh_basis16(dx, dy, dz, Y);
      float gv[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 16; ++i) acc = fmaf(shc[i * 3 + ch], Y[i], acc);
        gv[ch] = (acc + 0.5f > 0.0f) ? gq[6 + ch] : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        shc_w[i] = 0.0f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          gsh[i * 3 + ch] += gv[ch] * Y[i];
          shc_w[i] += gv[ch] * shc[i * 3 + ch];
        }
      }
      float gdx, gdy, gdz;
      sh_weighted_grad(dx, dy, dz, shc_w, gdx, gdy, gdz);
      const float dotg = gdx * dx + gdy * dy + gdz * dz;
      gmu[0] += (gdx - dx * dotg) * inv_len;
      gmu[1] += (gdy - dy * dotg) * inv_len;
      gmu[2] += (gdz - dz * dotg) * inv_len;
      go += gq[5];
    }
    if (!used) {  // no pixel of any view took the splat (also a splat culled for non-finite parameters)
#pragma unroll
      for (int j = 0; j < 3; ++j) g_means[j * n + k] = g_log_scales[j * n + k] = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) g_quats[j * n + k] = 0.0f;
      g_logits[k] = 0.0f;
#pragma unroll
      for (int i = 0; i < 48; ++i) g_sh[(int64_t)i * n + k] = 0.0f;
      continue;
    }
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
#pragma unroll
    for (int i = 0; i < 48; ++i) g_sh[(int64_t)i * n + k] = gsh[i];
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
    loss_finish_kernel<<<1, 1, 0, s>>>(block_sums, kLossBlocks, n_elems, d_loss);
    POTR_CHECK_LAUNCH();
  }
  return POTR_OK;
}

extern "C" size_t potr_render_backward_workspace_size(int64_t instance_capacity) {
  return sizeof(float) * (size_t)potr::kGradQ * (size_t)(instance_capacity > 0 ? instance_capacity : 0);
}

// Extra workspace for the per-(view, splat) sums: 9 floats per vk, after the instance partials.
static size_t vk_grad_bytes(int64_t n_vk) { return sizeof(float) * (size_t)potr::kGradQ * (size_t)n_vk; }

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
  const size_t inst_bytes = potr_render_backward_workspace_size(instance_capacity);
  if (instance_capacity <= 0 || !d_ws || ws_bytes < inst_bytes + vk_grad_bytes(n_vk)) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* inst_grad = static_cast<float*>(d_ws);
  if (cudaMemsetAsync(inst_grad, 0, potr_render_backward_workspace_size(instance_capacity), s) != cudaSuccess)
    return POTR_ERR_CUDA;
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
  float* vk_grad = reinterpret_cast<float*>(static_cast<char*>(d_ws) + inst_bytes);
  {
    int64_t gw = (n_vk + 127) / 128;
    if (gw > 152 * 32) gw = 152 * 32;
    vk_grad_sum_kernel<<<(unsigned)gw, 128, 0, s>>>(views->touched, views->offsets, views->n_instances,
                                                     instance_capacity, n_vk, inst_grad, vk_grad);
    POTR_CHECK_LAUNCH();
  }
  int64_t g = (n + 127) / 128;
  if (g > 152 * 64) g = 152 * 64;
  preprocess_bwd_kernel<<<(unsigned)g, 128, 0, s>>>(
      scene->means, scene->log_scales, scene->quats, scene->sh, views->cov3d, views->opacity, n, frame->cams,
      frame->n_views, *cfg, views->touched, vk_grad, grads->means, grads->log_scales, grads->quats,
      grads->opacity_logits, grads->sh);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
