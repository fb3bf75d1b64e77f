// sh_compact.cu -- spherical-harmonics energy compaction of POTR (Section IV-D), one warp per
// splat, binary64.
//
// For splat k and the frame's views s with importance I_k(s) > 0, weighted relative to each
// other (w_s = I_k(s) / max_s' I_k(s')), the rows w_s Y(d_s)
// (real SH basis at the direction camera -> splat) and the colours w_s C(d_s) (its current
// linear SH colour, taken to YCoCg) give the weighted Gram matrix G = Y~^T Y~ and the right-hand
// sides b = Y~^T C~ (lanes build them 32 views at a time through shared memory).  Columns are
// kept in index order unless their cosine with a kept preceding column exceeds alpha (or their
// norm is 0); the DC column is always kept.  Pass 1 solves the ridge system (G_AA + lambda_c D)
// x = b_A per YCoCg channel (lambda_Co = lambda_Cg = 3 lambda, D = 1 except on the DC), pass 2
// re-solves each channel without the AC coefficients that pass 1 leaves quantising to zero
// (floor(1/2 + x SF) == 0).  The factorisations are Cholesky decompositions, one channel per
// group of 8 lanes (three groups in parallel; inside a group the rows below the diagonal are
// dealt to the lanes, column by column); the cosine test compares a column with every kept
// one at once, one kept column per lane.
#include "potr_device.cuh"

namespace potr {
namespace {

constexpr int kShWarps = 4;  // splats per block

struct ShWarpMem {
  union {
    double rows[32][20];  // Gram phase: per view of the chunk, w Y (0..15), w C in YCoCg (16..18)
    double M[3][16][16];  // solve phase: one Cholesky factor per channel
  };
  double G[16][16];
  double b[16][3];
  double first[3][16];
  double second[3][16];
  double Lc[3][16];  // the splat's current coefficients (RGB)
  int cols[16];
};

// Real SH basis of degree <= 3 (Condon-Shortley phase), index l(l+1)+m, unit direction, binary64.
__device__ __forceinline__ void sh_basis16_f64(double x, double y, double z, double* Y) {
  const double xx = x * x, yy = y * y, zz = z * z;
  Y[0] = 0.28209479177387814;
  Y[1] = -0.4886025119029199 * y;
  Y[2] = 0.4886025119029199 * z;
  Y[3] = -0.4886025119029199 * x;
  Y[4] = 1.0925484305920792 * x * y;
  Y[5] = -1.0925484305920792 * y * z;
  Y[6] = 0.31539156525252005 * (2.0 * zz - xx - yy);
  Y[7] = -1.0925484305920792 * x * z;
  Y[8] = 0.5462742152960396 * (xx - yy);
  Y[9] = -0.5900435899266435 * y * (3.0 * xx - yy);
  Y[10] = 2.890611442640554 * x * y * z;
  Y[11] = -0.4570457994644658 * y * (4.0 * zz - xx - yy);
  Y[12] = 0.3731763325901154 * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
  Y[13] = -0.4570457994644658 * x * (4.0 * zz - xx - yy);
  Y[14] = 1.445305721320277 * z * (xx - yy);
  Y[15] = -0.5900435899266435 * x * (xx - 3.0 * yy);
}

// Ridge solve over the kept columns `cols` (m of them, cols[0] = 0 the DC) for channel ch:
// (G_AA + lam D) x = b_A with Cholesky in L, by the 8 lanes of one group (sub-lane sl, group mask
// gmask, first lane gbase); row i of L belongs to sub-lane i mod 8.  Binary64 divisions are long
// sequences on this part, so each diagonal entry's reciprocal is formed once (kept in the
// upper triangle, L[i][i+..] is unused) and the off-diagonal entries and the substitutions
// multiply by it.  x is written for every column (0 outside).  Returns false (on every lane of
// the group) if the matrix is not numerically positive definite.
__device__ bool ridge_solve_group(const ShWarpMem& w, const int* cols, int m, int ch, double lam, double* x,
                                  double (*L)[16], int sl, int gbase, unsigned gmask) {
  for (int i = sl; i < m; i += 8)
    for (int j = 0; j <= i; ++j) L[i][j] = w.G[cols[i]][cols[j]] + ((i == j && cols[i] != 0) ? lam : 0.0);
  __syncwarp(gmask);
  for (int j = 0; j < m; ++j) {
    const int owner = j & 7;
    int okj = 1;
    if (sl == owner) {
      double s = L[j][j];
      for (int p = 0; p < j; ++p) s -= L[j][p] * L[j][p];
      okj = s > 0.0;
      if (okj) L[j][j] = sqrt(s);
    }
    okj = __shfl_sync(gmask, okj, gbase + owner);
    if (!okj) return false;
    if (sl == owner && j + 1 < 16) L[j][j + 1] = 1.0 / L[j][j];  // the reciprocal, once
    __syncwarp(gmask);
    const double inv_d = j + 1 < 16 ? L[j][j + 1] : 1.0 / L[j][j];
    for (int i = sl; i < m; i += 8) {
      if (i <= j) continue;
      double t = L[i][j];
      for (int p = 0; p < j; ++p) t -= L[i][p] * L[j][p];
      L[i][j] = t * inv_d;
    }
    __syncwarp(gmask);
  }
  if (sl == 0) {
    double y[16];
    for (int i = 0; i < m; ++i) {
      const double inv = i + 1 < 16 ? L[i][i + 1] : 1.0 / L[i][i];
      double t = w.b[cols[i]][ch];
      for (int p = 0; p < i; ++p) t -= L[i][p] * y[p];
      y[i] = t * inv;
    }
    for (int i = 0; i < 16; ++i) x[i] = 0.0;
    for (int i = m - 1; i >= 0; --i) {
      const double inv = i + 1 < 16 ? L[i][i + 1] : 1.0 / L[i][i];
      double t = y[i];
      for (int p = i + 1; p < m; ++p) t -= L[p][i] * x[cols[p]];
      x[cols[i]] = t * inv;
    }
  }
  __syncwarp(gmask);
  return true;
}

__global__ void __launch_bounds__(32 * kShWarps) sh_compact_kernel(int64_t n, const float* __restrict__ means,
                                                                   const float* __restrict__ sh,
                                                                   const potr_camera* __restrict__ cams, int n_views,
                                                                   const double* __restrict__ imp_view, double lam,
                                                                   double alpha, double sf, float* __restrict__ sh_out,
                                                                   double* __restrict__ sh_ycocg,
                                                                   uint32_t* __restrict__ kept_out) {
  __shared__ ShWarpMem mem[kShWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  ShWarpMem& w = mem[wib];
  const int64_t warps_total = (int64_t)gridDim.x * kShWarps;
  for (int64_t k = (int64_t)blockIdx.x * kShWarps + wib; k < n; k += warps_total) {
    // current coefficients (RGB, in shared memory) and position
    for (int e = lane; e < 48; e += 32) w.Lc[e % 3][e / 3] = (double)sh[(int64_t)e * n + k];
    const double mx = means[k], my = means[n + k], mz = means[2 * n + k];
    for (int e = lane; e < 256; e += 32) (&w.G[0][0])[e] = 0.0;
    for (int e = lane; e < 48; e += 32) (&w.b[0][0])[e] = 0.0;
    double wmax = 0.0;  // the views are weighted relative to the most important one
    for (int v = lane; v < n_views; v += 32) {
      const double x = imp_view[(int64_t)v * n + k];
      if (x > wmax) wmax = x;
    }
    for (int o = 16; o >= 1; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    __syncwarp();
    // an unseen splat (wmax 0) skips the Gram phase: G stays 0 and its coefficients are kept
    for (int v0 = 0; wmax > 0.0 && v0 < n_views; v0 += 32) {
      const int v = v0 + lane;
      double wt = 0.0;
      if (v < n_views) wt = imp_view[(int64_t)v * n + k];
      wt = wt > 0.0 ? wt / wmax : 0.0;
      // the rows of the views with a weight, packed in view order (zero rows add nothing)
      const uint32_t has = __ballot_sync(0xffffffffu, wt > 0.0);
      double* row = w.rows[__popc(has & ((1u << lane) - 1u))];
      if (wt > 0.0) {
        const float* W = cams[v].w2c;
        double c[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          c[j] = -((double)W[0 * 4 + j] * W[3] + (double)W[1 * 4 + j] * W[7] + (double)W[2 * 4 + j] * W[11]);
        double dx = mx - c[0], dy = my - c[1], dz = mz - c[2];
        const double inv = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        double Y[16];
        sh_basis16_f64(dx, dy, dz, Y);
        double rgb[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          rgb[0] += w.Lc[0][i] * Y[i];
          rgb[1] += w.Lc[1][i] * Y[i];
          rgb[2] += w.Lc[2][i] * Y[i];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) row[i] = wt * Y[i];
        row[16] = wt * (0.25 * rgb[0] + 0.5 * rgb[1] + 0.25 * rgb[2]);   // Y
        row[17] = wt * (0.5 * rgb[0] - 0.5 * rgb[2]);                    // Co
        row[18] = wt * (-0.25 * rgb[0] + 0.5 * rgb[1] - 0.25 * rgb[2]);  // Cg
      }
      __syncwarp();
      const int nr = __popc(has);
      // G (upper triangle incl. diagonal, 136 entries) and b (48 entries), lanes over entries
      for (int e = lane; e < 136 + 48; e += 32) {
        int i, j;
        if (e < 136) {  // e -> (i, j), i <= j, row-major over the upper triangle
          i = 0;
          int rem = e;
          while (rem >= 16 - i) {
            rem -= 16 - i;
            ++i;
          }
          j = i + rem;
        } else {
          i = (e - 136) / 3;
          j = 16 + (e - 136) % 3;
        }
        double acc = 0.0;
        for (int r = 0; r < nr; ++r) acc += w.rows[r][i] * w.rows[r][j];
        if (e < 136) w.G[i][j] += acc;
        else w.b[i][j - 16] += acc;
      }
      __syncwarp();
    }
    for (int e = lane; e < 256; e += 32) {  // G's lower triangle from the upper one
      const int i = e >> 4, j = e & 15;
      if (j < i) w.G[i][j] = w.G[j][i];
    }
    if (lane == 0) w.cols[0] = 0;
    __syncwarp();
    const bool seen = w.G[0][0] > 0.0;  // some view sees the splat
    int m = 1;
    if (seen) {
      for (int i = 1; i < 16; ++i) {  // column i against every kept column, one per lane
        const double gii = w.G[i][i];
        if (!(gii > 0.0)) continue;
        bool par = false;
        if (lane < m) {
          const int j = w.cols[lane];
          par = fabs(w.G[i][j]) / sqrt(gii * w.G[j][j]) > alpha;
        }
        if (!__any_sync(0xffffffffu, par)) {
          if (lane == 0) w.cols[m] = i;
          ++m;
          __syncwarp();
        }
      }
    }
    // pass 1 then pass 2, channel `grp` on the 8 lanes of group grp (0-2)
    const int grp = lane >> 3, sl = lane & 7, gbase = grp * 8;
    const unsigned gmask = 0xffu << gbase;
    const double lam_c = grp == 0 ? lam : 3.0 * lam;
    bool ok_g = true;
    uint32_t kbits = 0;
    if (seen && grp < 3) ok_g = ridge_solve_group(w, w.cols, m, grp, lam_c, w.first[grp], w.M[grp], sl, gbase, gmask);
    bool ok = seen && __all_sync(0xffffffffu, ok_g);
    if (ok && grp < 3) {
      int c2[16], m2 = 1;
      c2[0] = 0;
      for (int q = 1; q < m; ++q)
        if (floor(__dadd_rn(0.5, __dmul_rn(w.first[grp][w.cols[q]], sf))) != 0.0) c2[m2++] = w.cols[q];
      for (int q = 0; q < m2; ++q) kbits |= 1u << c2[q];
      ok_g = ridge_solve_group(w, c2, m2, grp, lam_c, w.second[grp], w.M[grp], sl, gbase, gmask);
    }
    ok = ok && __all_sync(0xffffffffu, ok_g);
    const uint32_t k1 = __shfl_sync(0xffffffffu, kbits, 0), k2 = __shfl_sync(0xffffffffu, kbits, 8),
                   k3 = __shfl_sync(0xffffffffu, kbits, 16);
    if (lane == 0) {
      uint32_t keep = 0;
      for (int q = 0; q < m; ++q) keep |= 1u << w.cols[q];
      if (!ok) {  // unseen (or not positive definite): keep the coefficients
        for (int i = 0; i < 16; ++i) {
          w.second[0][i] = 0.25 * w.Lc[0][i] + 0.5 * w.Lc[1][i] + 0.25 * w.Lc[2][i];
          w.second[1][i] = 0.5 * w.Lc[0][i] - 0.5 * w.Lc[2][i];
          w.second[2][i] = -0.25 * w.Lc[0][i] + 0.5 * w.Lc[1][i] - 0.25 * w.Lc[2][i];
        }
      }
      if (kept_out) {
        kept_out[k] = ok ? keep : 0u;
        kept_out[n + k] = ok ? k1 : 0u;
        kept_out[2 * n + k] = ok ? k2 : 0u;
        kept_out[3 * n + k] = ok ? k3 : 0u;
      }
    }
    __syncwarp();
    // outputs: lanes over the 16 coefficients
    if (lane < 16) {
      const int i = lane;
      const double y = w.second[0][i], co = w.second[1][i], cg = w.second[2][i];
      if (sh_ycocg) {
        sh_ycocg[(int64_t)(i * 3 + 0) * n + k] = y;
        sh_ycocg[(int64_t)(i * 3 + 1) * n + k] = co;
        sh_ycocg[(int64_t)(i * 3 + 2) * n + k] = cg;
      }
      if (sh_out) {
        sh_out[(int64_t)(i * 3 + 0) * n + k] = (float)(y + co - cg);
        sh_out[(int64_t)(i * 3 + 1) * n + k] = (float)(y + cg);
        sh_out[(int64_t)(i * 3 + 2) * n + k] = (float)(y - co - cg);
      }
    }
    __syncwarp();
  }
}

}  // namespace
}  // namespace potr

extern "C" potr_status potr_sh_compact(const potr_scene* scene, const potr_frame* frame, const double* d_imp_view,
                                       double lambda, double alpha, double sf, float* d_sh_out, double* d_sh_ycocg,
                                       uint32_t* d_kept, potr_stream_t stream) {
  using namespace potr;
  if (!scene || !frame || !d_imp_view || !scene->means || !scene->sh || scene->n <= 0) return POTR_ERR_INVALID_ARGUMENT;
  if (frame->n_views < 1 || !frame->cams) return POTR_ERR_INVALID_ARGUMENT;
  if (!(lambda > 0.0) || !(alpha > 0.0) || !(sf > 0.0)) return POTR_ERR_INVALID_ARGUMENT;
  if (d_sh_out && d_sh_out == scene->sh) return POTR_ERR_INVALID_ARGUMENT;  // no in-place update
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = scene->n;
  int64_t g = (n + kShWarps - 1) / kShWarps;
  if (g > 152 * 64) g = 152 * 64;
  sh_compact_kernel<<<(unsigned)g, 32 * kShWarps, 0, s>>>(n, scene->means, scene->sh, frame->cams, frame->n_views,
                                                          d_imp_view, lambda, alpha, sf, d_sh_out, d_sh_ycocg, d_kept);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
