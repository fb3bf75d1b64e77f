// preprocess.cu -- activation and EWA projection of every splat into every view of a frame
// (paper Section 3: the 3D Gaussian, its affine-approximated 2D projection, the SH colour).
//
// Two kernels:
//   activate_kernel   one thread per splat: scale = exp(log_scale), q / |q|, Sigma = (R S)(R S)^T,
//                     o = sigmoid(logit).  View independent, so it runs once per frame.
//   project_kernel    one thread per splat, looping over the frame's views: the splat's
//                     centre, covariance and opacity are read once and kept in registers, its
//                     48 SH coefficients (on first visibility) in the thread's own column of
//                     shared memory, for all views.
// Both are HBM-bound: 32 B read / 28 B written per splat for activation; 40 B read per splat
// plus 192 B of SH per splat visible in the frame, and 48 B written per visible (view, splat).
#include "potr_device.cuh"

namespace potr {
namespace {

__global__ void __launch_bounds__(256) activate_kernel(const float* __restrict__ log_scales,
                                                       const float* __restrict__ quats,
                                                       const float* __restrict__ logits, int64_t n,
                                                       float* __restrict__ cov3d, float* __restrict__ opacity) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    float qw = quats[k], qx = quats[n + k], qy = quats[2 * n + k], qz = quats[3 * n + k];
    const float ls0 = log_scales[k], ls1 = log_scales[n + k], ls2 = log_scales[2 * n + k], lg = logits[k];
    if (!(isfinite(ls0) && isfinite(ls1) && isfinite(ls2) && isfinite(qw) && isfinite(qx) && isfinite(qy) &&
          isfinite(qz) && isfinite(lg))) {
      // a non-finite parameter: the splat is marked by a NaN opacity and culled by the projection
#pragma unroll
      for (int e = 0; e < 6; ++e) cov3d[e * n + k] = 0.0f;
      opacity[k] = __int_as_float(0x7fc00000);
      continue;
    }
    float s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s[a] = exp2r(__fmul_rn(log_scales[a * n + k], kLog2e));
    const float n2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(qw, qw), __fmul_rn(qx, qx)), __fmul_rn(qy, qy)),
                               __fmul_rn(qz, qz));
    if (n2 > 0.0f) {
      const float r = __fsqrt_rn(n2);
      qw = __fdiv_rn(qw, r);
      qx = __fdiv_rn(qx, r);
      qy = __fdiv_rn(qy, r);
      qz = __fdiv_rn(qz, r);
    } else {
      qw = 1.0f; qx = 0.0f; qy = 0.0f; qz = 0.0f;
    }
    float R[3][3];
    R[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(qy, qy), __fmul_rn(qz, qz))));
    R[0][1] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(qx, qy), __fmul_rn(qw, qz)));
    R[0][2] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(qx, qz), __fmul_rn(qw, qy)));
    R[1][0] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(qx, qy), __fmul_rn(qw, qz)));
    R[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(qx, qx), __fmul_rn(qz, qz))));
    R[1][2] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(qy, qz), __fmul_rn(qw, qx)));
    R[2][0] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(qx, qz), __fmul_rn(qw, qy)));
    R[2][1] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(qy, qz), __fmul_rn(qw, qx)));
    R[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(qx, qx), __fmul_rn(qy, qy))));
    float M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) M[i][j] = __fmul_rn(R[i][j], s[j]);
    const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int i = ii[e], j = jj[e];
      cov3d[e * n + k] =
          __fadd_rn(__fadd_rn(__fmul_rn(M[i][0], M[j][0]), __fmul_rn(M[i][1], M[j][1])), __fmul_rn(M[i][2], M[j][2]));
    }
    const float ex = exp2r(__fmul_rn(-logits[k], kLog2e));
    opacity[k] = __fdiv_rn(1.0f, __fadd_rn(1.0f, ex));
  }
}

// Real SH basis of degree <= 3 (Condon-Shortley phase), index l(l+1)+m, for a unit direction.
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

constexpr int kProjectThreads = 128;

__global__ void __launch_bounds__(kProjectThreads, 8) project_kernel(const float* __restrict__ means, const float* __restrict__ cov3d,
                                                      const float* __restrict__ opacity, const float* __restrict__ sh,
                                                      int64_t n, const potr_camera* __restrict__ cams,
                                                      const potr_view_info* __restrict__ info, int n_views,
                                                      potr_raster_config cfg, float4* __restrict__ raster,
                                                      float* __restrict__ depth_out, uint2* __restrict__ rect_out,
                                                      uint32_t* __restrict__ touched_out,
                                                      potr_device_status* __restrict__ status) {
  __shared__ float s_sh[48][kProjectThreads];  // each thread's own column: no sharing, no barrier
  const float kA = -0.5f * kLog2e;  // exact: a power-of-two scaling
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float mu0 = means[k], mu1 = means[n + k], mu2 = means[2 * n + k];
    const float S00 = cov3d[k], S01 = cov3d[n + k], S02 = cov3d[2 * n + k];
    const float S11 = cov3d[3 * n + k], S12 = cov3d[4 * n + k], S22 = cov3d[5 * n + k];
    const float o = opacity[k];
    const float pthr = log2f(cfg.alpha_min / o) - 0.01f;  // conservative prefilter, see render
    bool sh_checked = false;  // the SH coefficients wait in shared memory after the first use
    // non-finite centre or activation input (NaN opacity from activate_kernel): culled in every view
    bool bad = !(isfinite(mu0) && isfinite(mu1) && isfinite(mu2) && isfinite(o));
#pragma unroll 1
    for (int v = 0; v < n_views; ++v) {
      const int64_t vk = (int64_t)v * n + k;
      if (bad) {
        touched_out[vk] = 0;
        continue;
      }
      const potr_camera& cam = cams[v];
      const float* W = cam.w2c;
      float t[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        t[i] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(W[i * 4 + 0], mu0), __fmul_rn(W[i * 4 + 1], mu1)),
                                   __fmul_rn(W[i * 4 + 2], mu2)),
                         W[i * 4 + 3]);
      if (!(t[2] > cfg.near_z)) {
        touched_out[vk] = 0;
        continue;
      }
      const float lim_x = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)cam.width), cam.fx));
      const float lim_y = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)cam.height), cam.fy));
      const float txz = __fdiv_rn(t[0], t[2]);
      const float tyz = __fdiv_rn(t[1], t[2]);
      const float xc = __fmul_rn(fminf(lim_x, fmaxf(-lim_x, txz)), t[2]);
      const float yc = __fmul_rn(fminf(lim_y, fmaxf(-lim_y, tyz)), t[2]);
      const float z2 = __fmul_rn(t[2], t[2]);
      const float j00 = __fdiv_rn(cam.fx, t[2]);
      const float j02 = __fdiv_rn(-__fmul_rn(cam.fx, xc), z2);
      const float j11 = __fdiv_rn(cam.fy, t[2]);
      const float j12 = __fdiv_rn(-__fmul_rn(cam.fy, yc), z2);
      float T0[3], T1[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T0[j] = __fadd_rn(__fmul_rn(j00, W[0 * 4 + j]), __fmul_rn(j02, W[2 * 4 + j]));
        T1[j] = __fadd_rn(__fmul_rn(j11, W[1 * 4 + j]), __fmul_rn(j12, W[2 * 4 + j]));
      }
      const float S[3][3] = {{S00, S01, S02}, {S01, S11, S12}, {S02, S12, S22}};
      float U0[3], U1[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        U0[j] = __fadd_rn(__fadd_rn(__fmul_rn(T0[0], S[0][j]), __fmul_rn(T0[1], S[1][j])), __fmul_rn(T0[2], S[2][j]));
        U1[j] = __fadd_rn(__fadd_rn(__fmul_rn(T1[0], S[0][j]), __fmul_rn(T1[1], S[1][j])), __fmul_rn(T1[2], S[2][j]));
      }
      const float a = __fadd_rn(
          __fadd_rn(__fadd_rn(__fmul_rn(U0[0], T0[0]), __fmul_rn(U0[1], T0[1])), __fmul_rn(U0[2], T0[2])), cfg.lowpass);
      const float b = __fadd_rn(__fadd_rn(__fmul_rn(U0[0], T1[0]), __fmul_rn(U0[1], T1[1])), __fmul_rn(U0[2], T1[2]));
      const float c = __fadd_rn(
          __fadd_rn(__fadd_rn(__fmul_rn(U1[0], T1[0]), __fmul_rn(U1[1], T1[1])), __fmul_rn(U1[2], T1[2])), cfg.lowpass);
      const float det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, b));
      if (!(det > 0.0f)) {
        touched_out[vk] = 0;
        continue;
      }
      const float ca = __fdiv_rn(c, det), cb = __fdiv_rn(-b, det), cc = __fdiv_rn(a, det);
      const float mid = __fmul_rn(0.5f, __fadd_rn(a, c));
      const float disc = fmaxf(0.1f, __fsub_rn(__fmul_rn(mid, mid), det));
      const float lam = __fadd_rn(mid, __fsqrt_rn(disc));
      const float r = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));
      const float mx = __fadd_rn(__fmul_rn(cam.fx, txz), cam.cx);
      const float my = __fadd_rn(__fmul_rn(cam.fy, tyz), cam.cy);
      const potr_view_info vi = info[v];
      // x / tile_w as x * (1 / tile_w): tile_w tile_h = 256 makes both powers of two, so the
      // reciprocal is exact and the product is the correctly rounded quotient
      const float itw = 1.0f / (float)cfg.tile_w, ith = 1.0f / (float)cfg.tile_h;
      const float fx0 = floorf(__fmul_rn(__fsub_rn(mx, r), itw));
      const float fx1 = __fadd_rn(floorf(__fmul_rn(__fadd_rn(mx, r), itw)), 1.0f);
      const float fy0 = floorf(__fmul_rn(__fsub_rn(my, r), ith));
      const float fy1 = __fadd_rn(floorf(__fmul_rn(__fadd_rn(my, r), ith)), 1.0f);
      const int x0 = (int)fminf(fmaxf(fx0, 0.0f), (float)vi.tiles_x);
      const int x1 = (int)fminf(fmaxf(fx1, 0.0f), (float)vi.tiles_x);
      const int y0 = (int)fminf(fmaxf(fy0, 0.0f), (float)vi.tiles_y);
      const int y1 = (int)fminf(fmaxf(fy1, 0.0f), (float)vi.tiles_y);
      if (!(x1 > x0 && y1 > y0)) {
        touched_out[vk] = 0;
        continue;
      }
      // SH colour along the camera-to-splat direction (values only: plain fp32 arithmetic)
      if (!sh_checked) {
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 48; ++i) {
          const float c = __ldg(sh + (int64_t)i * n + k);
          s_sh[i][threadIdx.x] = c;
          fin = fin && isfinite(c);
        }
        sh_checked = true;
        if (!fin) {  // a non-finite SH coefficient: culled here and in the later views (not seen before)
          bad = true;
          touched_out[vk] = 0;
          continue;
        }
      }
      const float cx0 = -(W[0] * W[3] + W[4] * W[7] + W[8] * W[11]);
      const float cy0 = -(W[1] * W[3] + W[5] * W[7] + W[9] * W[11]);
      const float cz0 = -(W[2] * W[3] + W[6] * W[7] + W[10] * W[11]);
      float dx = mu0 - cx0, dy = mu1 - cy0, dz = mu2 - cz0;
      const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
      dx *= inv; dy *= inv; dz *= inv;
      float Y[16];
      sh_basis16(dx, dy, dz, Y);
      float rgb[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 16; ++i) acc = fmaf(s_sh[i * 3 + ch][threadIdx.x], Y[i], acc);
        rgb[ch] = fmaxf(acc + 0.5f, 0.0f);
      }
      const uint32_t rw = pack_rect_word((uint32_t)x0, (uint32_t)y0, (uint32_t)(x1 - x0));
      float4* rec = raster + vk * kRec;
      rec[0] = make_float4(mx, my, __fmul_rn(ca, kA), __fmul_rn(cb, -kLog2e));
      // word 7: 0 when the exponent A u^2 + B u v + C v^2 is negative definite (A < 0, C < 0,
      // 4 A C - B^2 > 0, decided exactly: the products of binary32 values are exact in
      // binary64), so that it never exceeds a rounding error above 0; 1 otherwise
      const float qa = __fmul_rn(ca, kA), qb = __fmul_rn(cb, -kLog2e), qc = __fmul_rn(cc, kA);
      const bool definite = qa < 0.0f && qc < 0.0f && 4.0 * (double)qa * (double)qc - (double)qb * (double)qb > 0.0;
      rec[1] = make_float4(qc, o, pthr, definite ? 0.0f : 1.0f);
      rec[2] = make_float4(rgb[0], rgb[1], rgb[2], __uint_as_float(rw));
      depth_out[vk] = t[2];
      rect_out[vk] = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
      touched_out[vk] = (uint32_t)((x1 - x0) * (y1 - y0));  // candidates; tile_mask_kernel keeps some
    }
    if (bad && status) {
      atomicCAS(&status->code, 0, (int32_t)POTR_ERR_NUMERIC);
      atomicAdd(&status->n_nonfinite, 1);
    }
  }
}

// Kept tiles of every (view, splat) rectangle of at most kCullMaxTiles tiles.  One warp per 32
// consecutive vk: their candidate tiles (rectangle cells, row-major) are dealt to the lanes 32
// at a time, each lane runs the tile test for one candidate, and every owner collects its bits
// from the ballot.  Each lane's splat parameters sit in its row of the warp's shared memory; a
// candidate's owner is the lane whose candidates start at the last start position at or before
// it (a bitmap of the round's start positions, and the lane starting at each), or the owner of
// the previous round's last candidate.  Writes the culling word of every vk -- mask low, mask
// high, the rectangle word (as record word 11) and the kept count | all-kept flag << 31 (0 for
// a culled vk) -- to its own 16-byte array (coalesced whole-sector stores, not a partial
// rewrite of the record), and touched = the kept count, so that the emission reads one 16-byte
// word per vk.
__global__ void __launch_bounds__(256, 5) tile_mask_kernel(const uint2* __restrict__ rect, int64_t n_vk,
                                                           potr_raster_config cfg, const float4* __restrict__ raster,
                                                           uint4* __restrict__ cull, uint32_t* __restrict__ touched) {
  // per warp and lane: {mx, my, A, B}, {C, o, ku, kv}, {pthr, x0 | y0 << 16, w | concave << 31,
  // first candidate}; 48-byte rows, so 16-byte reads of 8 consecutive rows hit distinct banks
  __shared__ float4 s_par[8][32][3];
  __shared__ uint8_t s_start[8][32];  // lane whose candidates start at each position of the round
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t warps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wv = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wv * 32 < n_vk; wv += warps_total) {
    const int64_t vk = wv * 32 + lane;
    uint32_t area = 0, cand = 0, x0 = 0, y0 = 0, w = 1;
    float mx = 0.0f, my = 0.0f, qa = 0.0f, qb = 0.0f, qc = 0.0f, o = 0.0f, ku = 0.0f, kv = 0.0f, pthr = 0.0f;
    bool concave = false;
    if (vk < n_vk) {
      area = touched[vk];
      if (area) {
        const uint2 r = rect[vk];
        x0 = r.x & 0xffffu;
        y0 = r.x >> 16;
        w = (r.y & 0xffffu) - x0;
        if (area <= (uint32_t)kCullMaxTiles) {
          cand = area;
          const float4 r0 = raster[vk * kRec], r1 = raster[vk * kRec + 1];
          mx = r0.x; my = r0.y; qa = r0.z; qb = r0.w; qc = r1.x; o = r1.y; pthr = r1.z;
          concave = qa < 0.0f && qc < 0.0f;
          if (concave) {
            ku = tile_ku(qa, qb);
            kv = tile_ku(qc, qb);
          }
        }
      }
    }
    uint32_t incl = cand;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, s);
      if (lane >= s) incl += y;
    }
    const uint32_t excl = incl - cand;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();  // the previous item's rows are no longer read
    s_par[warp][lane][0] = make_float4(mx, my, qa, qb);
    s_par[warp][lane][1] = make_float4(qc, o, ku, kv);
    s_par[warp][lane][2] = make_float4(pthr, __uint_as_float(x0 | (y0 << 16)),
                                       __uint_as_float(w | (concave ? 0x80000000u : 0u)), __uint_as_float(excl));
    uint64_t mask = 0;
    uint32_t carry = 0;  // owner of the previous round's last position
    for (uint32_t e0 = 0; e0 < total; e0 += 32) {
      const uint32_t e = e0 + lane;
      const bool starts = cand > 0 && excl >= e0 && excl < e0 + 32u;
      if (starts) s_start[warp][excl - e0] = (uint8_t)lane;
      const uint32_t S = __reduce_or_sync(0xffffffffu, starts ? 1u << (excl - e0) : 0u);
      __syncwarp();  // the rows and the round's starts are visible
      const uint32_t below = S & (0xffffffffu >> (31 - lane));  // starts at positions e0 .. e
      const uint32_t owner = below ? (uint32_t)s_start[warp][31 - __clz(below)] : carry;
      carry = __shfl_sync(0xffffffffu, owner, 31);
      const float4 p2 = s_par[warp][owner][2];
      const uint32_t li = e - __float_as_uint(p2.w);
      const uint32_t wb = __float_as_uint(p2.z), xy = __float_as_uint(p2.y);
      const uint32_t ow = wb & 0xffffu;
      const uint32_t dy = small_div(li, ow);  // li < 96
      const int tx = (int)((xy & 0xffffu) + (li - dy * ow));
      const int ty = (int)((xy >> 16) + dy);
      bool hit = false;
      if (e < total) {
        hit = true;
        if (wb >> 31) {
          const float4 p0 = s_par[warp][owner][0], p1 = s_par[warp][owner][1];
          hit = tile_hit_concave(p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x, tx, ty, cfg.tile_w,
                                 cfg.tile_h, cfg.alpha_min);
        }
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, hit);
      // this lane's candidates [excl, excl + cand) overlapping [e0, e0 + 32)
      const uint32_t lo = max(excl, e0), hi = min(excl + cand, e0 + 32u);
      if (lo < hi) {
        const uint32_t len = hi - lo;
        const uint32_t bits = (bal >> (lo - e0)) & (len == 32u ? 0xffffffffu : ((1u << len) - 1u));
        mask |= (uint64_t)bits << (lo - excl);
      }
      __syncwarp();  // the starts are rewritten next round
    }
    if (vk < n_vk) {
      const bool all = area > (uint32_t)kCullMaxTiles;
      const uint32_t kept = all ? area : (uint32_t)__popcll(mask);
      const uint32_t rw = area ? pack_rect_word(x0, y0, w) : 0u;
      cull[vk] = make_uint4((uint32_t)mask, (uint32_t)(mask >> 32), rw, kept | (all ? 0x80000000u : 0u));
      if (area) touched[vk] = kept;
    }
  }
}

int grid_for(int64_t n, int block, int max_blocks) {
  int64_t g = (n + block - 1) / block;
  if (g > max_blocks) g = max_blocks;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace
}  // namespace potr

extern "C" potr_status potr_view_layout(const potr_camera* h_cams, int32_t n_views, const potr_raster_config* cfg,
                                        potr_view_info* h_info, int64_t* total_tiles, int64_t* total_pixels) {
  if (!h_cams || !cfg || !h_info || n_views < 1) return POTR_ERR_INVALID_ARGUMENT;
  if (cfg->tile_w <= 0 || cfg->tile_h <= 0 || cfg->tile_w * cfg->tile_h != potr::kTilePixels)
    return POTR_ERR_INVALID_ARGUMENT;
  int64_t tb = 0, pb = 0;
  for (int v = 0; v < n_views; ++v) {
    const potr_camera& c = h_cams[v];
    if (c.width <= 0 || c.height <= 0) return POTR_ERR_INVALID_ARGUMENT;
    potr_view_info& vi = h_info[v];
    vi.width = c.width;
    vi.height = c.height;
    vi.tiles_x = (c.width + cfg->tile_w - 1) / cfg->tile_w;
    vi.tiles_y = (c.height + cfg->tile_h - 1) / cfg->tile_h;
    if (vi.tiles_x > 1023 || vi.tiles_y > 2047) return POTR_ERR_UNSUPPORTED;
    vi.tile_base = tb;
    vi.pixel_base = pb;
    tb += (int64_t)vi.tiles_x * vi.tiles_y;
    pb += (int64_t)c.width * c.height;
  }
  if (total_tiles) *total_tiles = tb;
  if (total_pixels) *total_pixels = pb;
  return POTR_OK;
}

extern "C" potr_status potr_preprocess(const potr_scene* scene, const potr_frame* frame, const potr_raster_config* cfg,
                                       const potr_views* views, potr_device_status* d_status, potr_stream_t stream) {
  if (!scene || !frame || !cfg || !views) return POTR_ERR_INVALID_ARGUMENT;
  if (cfg->tile_w <= 0 || cfg->tile_h <= 0 || cfg->tile_w * cfg->tile_h != potr::kTilePixels)
    return POTR_ERR_INVALID_ARGUMENT;
  if (scene->n <= 0 || frame->n_views < 1 || !frame->cams || !frame->info) return POTR_ERR_INVALID_ARGUMENT;
  if (!scene->means || !scene->log_scales || !scene->quats || !scene->opacity_logits || !scene->sh)
    return POTR_ERR_INVALID_ARGUMENT;
  if (!views->cov3d || !views->opacity || !views->raster || !views->depth || !views->rect || !views->touched ||
      !views->cull)
    return POTR_ERR_INVALID_ARGUMENT;
  if ((reinterpret_cast<uintptr_t>(views->raster) & 15) != 0 || (reinterpret_cast<uintptr_t>(views->cull) & 15) != 0)
    return POTR_ERR_INVALID_ARGUMENT;
  if ((int64_t)frame->n_views * scene->n >= (int64_t)UINT32_MAX) return POTR_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = scene->n;
  potr::activate_kernel<<<potr::grid_for(n, 256, 152 * 16), 256, 0, s>>>(scene->log_scales, scene->quats,
                                                                          scene->opacity_logits, n, views->cov3d,
                                                                          views->opacity);
  POTR_CHECK_LAUNCH();
  potr::project_kernel<<<potr::grid_for(n, potr::kProjectThreads, 152 * 32), potr::kProjectThreads, 0, s>>>(
      scene->means, views->cov3d, views->opacity, scene->sh, n, frame->cams, frame->info, frame->n_views, *cfg,
      reinterpret_cast<float4*>(views->raster), views->depth, reinterpret_cast<uint2*>(views->rect), views->touched,
      d_status);
  POTR_CHECK_LAUNCH();
  const int64_t n_vk = n * frame->n_views;
  potr::tile_mask_kernel<<<potr::grid_for(n_vk, 256, 152 * 16), 256, 0, s>>>(
      reinterpret_cast<const uint2*>(views->rect), n_vk, *cfg, reinterpret_cast<const float4*>(views->raster),
      reinterpret_cast<uint4*>(views->cull), views->touched);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
