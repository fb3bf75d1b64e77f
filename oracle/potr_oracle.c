/*
 * potr_oracle.c -- plain, slow CPU reference of the POTR removal-effect rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the CPU
 * baseline leg of the benchmark may load this code.  The CUDA library never links,
 * includes or calls it, and it shares no code, header or constant table with it.
 *
 * What it computes (paper: "POTR: Post-Training 3DGS Compression", arXiv 2601.14821):
 *   - Section 3 (Eqs. 1-4): 3D Gaussians projected by the affine (EWA) approximation to
 *     2D Gaussians, per-pixel opacity alpha = o * G2D(x), transmittance T_k = prod(1-alpha_j),
 *     front-to-back compositing over black, colour from real SH of degree <= 3 indexed
 *     l(l+1)+m+1, evaluated along the camera-to-splat direction.
 *   - Section IV-A: splat importance I_k(s) = (1/P) sum_x T_{i_k} alpha_{i_k}.
 *   - Section IV-B, Eq. (partial colour) and Eq. (pruning difference):
 *       P_i = sum_{k<i} T_k alpha_k c_k,
 *       PD_k = (P_i + (P_K - P_{i+1}) / (1 - alpha_i)) - P_K,
 *     Eq. (pixel squared error): dSE_k = PD^2 + 2 PD (c - c_t),
 *     and dMSE_k = (1/N) sum_s (1/P) sum_x (1/3) dSE_k . 1 (combined by the caller).
 *   - The definition itself, for pinning: re-render with one splat left out.
 *
 * Precision.  The paper fixes none.  Every quantity that decides an integer -- the tile
 * rectangle, the depth key, whether a pixel takes a splat (alpha >= alpha_min) and whether
 * compositing stops (T (1 - alpha) < T_min) -- is computed in IEEE binary32 with a fixed
 * operation order (no contraction: build with -ffp-contract=off), with exp taken by the
 * reproducible exp2r below (Cody-Waite reduction to [-1/2, 1/2] plus a degree-6 Taylor
 * polynomial of 2^f, coefficients (ln 2)^k / k!).  The per-pair opacity alpha is that
 * binary32 value.  All sums downstream of alpha (T, P_i, c, PD, dSE, importance) and the
 * SH colours are binary64.
 *
 * Readings where the paper is silent (the original 3DGS renderer's conventions, as
 * parameters): near-plane cull, 1.3 x half-fov clamp of the Jacobian, low-pass dilation of
 * the 2D covariance, eigenvalue floor 0.1, radius ceil(3 sqrt(lambda_max)), pixel centres at
 * (x + 0.5, y + 0.5), colour = max(0, SH + 0.5), alpha <= alpha_max, skip alpha < alpha_min,
 * stop before a splat that would take T below T_min, quaternions (w, x, y, z) normalised,
 * scale = exp(log-scale), opacity = sigmoid(logit), depth ties broken by splat index.
 * Binning keeps a tile of the 3-sigma rectangle only when some pixel centre of it can reach
 * alpha_min (orc_tile_hit; rectangles of more than 64 tiles keep every tile): pixels skip
 * such splats anyway, so images and removal effects are those of whole-rectangle binning.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__FAST_MATH__)
#error "the oracle must be built without fast-math"
#endif

typedef struct {
  float w2c[12]; /* rows [R | t] of the world-to-camera transform */
  float fx, fy, cx, cy;
  int32_t width, height;
} orc_camera;

typedef struct {
  int32_t tile_w, tile_h;
  float near_z;    /* cull when camera-space z <= near_z */
  float lowpass;   /* added to both diagonal entries of the 2D covariance */
  float alpha_min; /* a pixel skips a splat with alpha < alpha_min */
  float alpha_max; /* alpha is clamped to alpha_max */
  float t_min;     /* compositing stops before T would drop below t_min */
} orc_config;

/* ---------------------------------------------------------------------------------- */
/* Reproducible binary32 exp2 (Cody & Waite range reduction, Taylor series of 2^f).    */
/* ---------------------------------------------------------------------------------- */

static float g_c[7];
static pthread_once_t g_c_once = PTHREAD_ONCE_INIT;

static void exp2r_init(void) {
  /* c_k = (ln 2)^k / k!, evaluated in binary64 by the recurrence c_k = c_{k-1} * ln2 / k,
   * then rounded to binary32. */
  const double ln2 = 0.6931471805599453;
  double c = 1.0;
  g_c[0] = 1.0f;
  for (int k = 1; k <= 6; ++k) {
    c = c * ln2;
    c = c / (double)k;
    g_c[k] = (float)c;
  }
}

float orc_exp2r(float y) {
  pthread_once(&g_c_once, exp2r_init);
  if (!(y >= -125.0f)) y = -125.0f; /* also maps NaN to the lower clamp */
  if (y > 125.0f) y = 125.0f;
  float n = rintf(y); /* nearest integer, ties to even */
  float f = y - n;    /* exact: |f| <= 1/2 */
  float p = g_c[6];
  for (int k = 5; k >= 0; --k) p = fmaf(p, f, g_c[k]);
  return ldexpf(p, (int)n);
}

void orc_exp2r_array(int64_t n, const float* y, float* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_exp2r(y[i]);
}

void orc_exp2r_coeffs(float* out7) {
  pthread_once(&g_c_once, exp2r_init);
  memcpy(out7, g_c, sizeof(g_c));
}

static const float kLog2e = 1.44269504088896340736f; /* log2(e) rounded to binary32 */

/*
 * Binning reading: a tile of a splat's 3-sigma rectangle receives the splat only if some pixel
 * centre of the tile can reach alpha >= alpha_min.  With log2 G = A u^2 + B u v + C v^2
 * (u = x - mx, v = y - my), the exponent's maximum over the rectangle of the tile's pixel
 * centres is taken on its edges (on each edge a concave parabola, maximised at its clamped
 * vertex) and at the splat centre when it lies inside; the tile is kept when
 * o * exp2r(max + margin) >= alpha_min, the margin 1e-5 |terms| + 1e-4 covering, some ten
 * times over, the binary32 rounding of this maximum and of a pixel's own exponent (a few units
 * in the last place of the largest term) and the error of exp2r.  Every pixel whose alpha reaches alpha_min therefore lies in a kept tile, so no
 * compositing decision changes.  Binary32, fixed operation order, no contraction.
 */
static float edge_max(float A, float B, float C, float u, float v) { return (A * u + B * v) * u + C * v * v; }

int orc_tile_hit(float mx, float my, float A, float B, float C, float o, int tx, int ty, int tile_w, int tile_h,
                 float alpha_min) {
  if (!(A < 0.0f && C < 0.0f)) return 1;
  float X0 = (float)(tx * tile_w) + 0.5f, X1 = X0 + (float)(tile_w - 1);
  float Y0 = (float)(ty * tile_h) + 0.5f, Y1 = Y0 + (float)(tile_h - 1);
  float ux0 = X0 - mx, ux1 = X1 - mx, vy0 = Y0 - my, vy1 = Y1 - my;
  float ku = -B / (2.0f * A), kv = -B / (2.0f * C);
  float u0 = fminf(fmaxf(ku * vy0, ux0), ux1);
  float u1 = fminf(fmaxf(ku * vy1, ux0), ux1);
  float v0 = fminf(fmaxf(kv * ux0, vy0), vy1);
  float v1 = fminf(fmaxf(kv * ux1, vy0), vy1);
  float pmax = fmaxf(fmaxf(edge_max(A, B, C, u0, vy0), edge_max(A, B, C, u1, vy1)),
                     fmaxf(edge_max(A, B, C, ux0, v0), edge_max(A, B, C, ux1, v1)));
  if (ux0 <= 0.0f && ux1 >= 0.0f && vy0 <= 0.0f && vy1 >= 0.0f) pmax = fmaxf(pmax, 0.0f);
  float um = fmaxf(fabsf(ux0), fabsf(ux1)), vm = fmaxf(fabsf(vy0), fabsf(vy1));
  float mag = (fabsf(A) * um * um + fabsf(B) * um * vm) + fabsf(C) * vm * vm;
  float margin = 1e-5f * mag + 1e-4f;
  return o * orc_exp2r(pmax + margin) >= alpha_min;
}

/* A rectangle of more than 64 tiles keeps every tile (the test is applied to smaller ones). */
#define ORC_CULL_MAX_TILES 64

static int tile_kept(int64_t area, float mx, float my, float A, float B, float C, float o, int tx, int ty,
                     const orc_config* cfg) {
  if (area > ORC_CULL_MAX_TILES) return 1;
  return orc_tile_hit(mx, my, A, B, C, o, tx, ty, cfg->tile_w, cfg->tile_h, cfg->alpha_min);
}

/* ---------------------------------------------------------------------------------- */
/* Section 3: activation of one splat (view independent).                             */
/* ---------------------------------------------------------------------------------- */

/* cov3d planes: xx, xy, xz, yy, yz, zz. */
void orc_activate(int64_t n, const float* log_scales, const float* quats, const float* logits,
                  float* cov3d, float* opacity) {
  for (int64_t k = 0; k < n; ++k) {
    float s[3];
    for (int a = 0; a < 3; ++a) s[a] = orc_exp2r(log_scales[a * n + k] * kLog2e);
    float qw = quats[0 * n + k], qx = quats[1 * n + k], qy = quats[2 * n + k], qz = quats[3 * n + k];
    float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    if (n2 > 0.0f) {
      float r = sqrtf(n2);
      qw = qw / r; qx = qx / r; qy = qy / r; qz = qz / r;
    } else {
      qw = 1.0f; qx = 0.0f; qy = 0.0f; qz = 0.0f;
    }
    /* rotation matrix of the unit quaternion (w real) */
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (qy * qy + qz * qz);
    R[0][1] = 2.0f * (qx * qy - qw * qz);
    R[0][2] = 2.0f * (qx * qz + qw * qy);
    R[1][0] = 2.0f * (qx * qy + qw * qz);
    R[1][1] = 1.0f - 2.0f * (qx * qx + qz * qz);
    R[1][2] = 2.0f * (qy * qz - qw * qx);
    R[2][0] = 2.0f * (qx * qz - qw * qy);
    R[2][1] = 2.0f * (qy * qz + qw * qx);
    R[2][2] = 1.0f - 2.0f * (qx * qx + qy * qy);
    /* Sigma = (R S)(R S)^T with S = diag(s) */
    float M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
    const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
    for (int e = 0; e < 6; ++e) {
      int i = ii[e], j = jj[e];
      cov3d[e * n + k] = (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2];
    }
    float ex = orc_exp2r(-logits[k] * kLog2e);
    opacity[k] = 1.0f / (1.0f + ex);
  }
}

/* ---------------------------------------------------------------------------------- */
/* Real spherical harmonics, degree <= 3, by the associated Legendre recurrence.        */
/* Index l(l+1)+m (zero based) for the paper's l(l+1)+m+1.                              */
/* ---------------------------------------------------------------------------------- */

static double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= (double)i;
  return f;
}

/* P_l^m(z) including the Condon-Shortley phase (-1)^m, 0 <= m <= l <= 3. */
static double assoc_legendre(int l, int m, double z) {
  double pmm = 1.0;
  double s = sqrt(fmax(0.0, 1.0 - z * z));
  double fact = 1.0;
  for (int i = 1; i <= m; ++i) {
    pmm *= -fact * s;
    fact += 2.0;
  }
  if (l == m) return pmm;
  double pm1 = z * (2.0 * m + 1.0) * pmm;
  if (l == m + 1) return pm1;
  double pl = 0.0;
  for (int ll = m + 2; ll <= l; ++ll) {
    pl = ((2.0 * ll - 1.0) * z * pm1 - (ll + m - 1.0) * pmm) / (double)(ll - m);
    pmm = pm1;
    pm1 = pl;
  }
  return pl;
}

void orc_sh_basis(double x, double y, double z, double* Y /*16*/) {
  const double pi = 3.14159265358979323846;
  double phi = atan2(y, x);
  for (int l = 0; l <= 3; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * pi) * factorial(l - am) / factorial(l + am));
      double P = assoc_legendre(l, am, z);
      double v;
      if (m == 0) v = K * P;
      else if (m > 0) v = sqrt(2.0) * K * cos(am * phi) * P;
      else v = sqrt(2.0) * K * sin(am * phi) * P;
      Y[l * (l + 1) + m] = v;
    }
  }
}

/* ---------------------------------------------------------------------------------- */
/* Section 3: projection of every splat into one view (EWA), colour, tile rectangle.   */
/* ---------------------------------------------------------------------------------- */

/*
 * Outputs per splat k (arrays of length n unless noted):
 *   depth          camera-space z (binary32; the sort key's low word)
 *   mean2d[2n]     pixel-space centre (x plane then y plane)
 *   cov2d[3n]      a, b, c of the dilated 2D covariance
 *   conic[3n]      inverse of cov2d: (c, -b, a) / det
 *   qcoef[3n]      the per-pair exponent coefficients A, B, C with
 *                  log2 G = A dx^2 + B dx dy + C dy^2
 *   radius         ceil(3 sqrt(lambda_max)) in pixels
 *   rect[4n]       tile rectangle x0, y0, x1, y1 (half open)
 *   touched        (x1 - x0)(y1 - y0), 0 when culled
 *   rgb[3n]        colour (binary64)
 * A culled splat has touched = 0 and its other outputs are zero.
 */
void orc_project(int64_t n, const float* means, const float* cov3d, const float* opacity, const float* sh, const orc_camera* cam, const orc_config* cfg, float* depth,
                 float* mean2d, float* cov2d, float* conic, float* qcoef, float* radius,
                 int32_t* rect, uint32_t* touched, double* rgb) {
  const float* W = cam->w2c;
  const int tiles_x = (cam->width + cfg->tile_w - 1) / cfg->tile_w;
  const int tiles_y = (cam->height + cfg->tile_h - 1) / cfg->tile_h;
  const float lim_x = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
  const float lim_y = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
  const float kA = -0.5f * kLog2e;
  /* camera centre in world coordinates, c = -R^T t (binary64, colour only) */
  double cc[3];
  for (int j = 0; j < 3; ++j)
    cc[j] = -((double)W[0 * 4 + j] * W[3] + (double)W[1 * 4 + j] * W[7] + (double)W[2 * 4 + j] * W[11]);

  for (int64_t k = 0; k < n; ++k) {
    depth[k] = 0.0f;
    mean2d[k] = mean2d[n + k] = 0.0f;
    for (int e = 0; e < 3; ++e) {
      cov2d[e * n + k] = conic[e * n + k] = qcoef[e * n + k] = 0.0f;
      rgb[e * n + k] = 0.0;
    }
    radius[k] = 0.0f;
    for (int e = 0; e < 4; ++e) rect[e * n + k] = 0;
    touched[k] = 0;

    float mu[3] = {means[k], means[n + k], means[2 * n + k]};
    float t[3];
    for (int i = 0; i < 3; ++i) t[i] = ((W[i * 4 + 0] * mu[0] + W[i * 4 + 1] * mu[1]) + W[i * 4 + 2] * mu[2]) + W[i * 4 + 3];
    if (!(t[2] > cfg->near_z)) continue;

    float txz = t[0] / t[2];
    float tyz = t[1] / t[2];
    float xc = fminf(lim_x, fmaxf(-lim_x, txz)) * t[2];
    float yc = fminf(lim_y, fmaxf(-lim_y, tyz)) * t[2];
    float z2 = t[2] * t[2];
    float j00 = cam->fx / t[2];
    float j02 = -(cam->fx * xc) / z2;
    float j11 = cam->fy / t[2];
    float j12 = -(cam->fy * yc) / z2;
    /* T = J W_rot (2 x 3) */
    float T0[3], T1[3];
    for (int j = 0; j < 3; ++j) {
      T0[j] = j00 * W[0 * 4 + j] + j02 * W[2 * 4 + j];
      T1[j] = j11 * W[1 * 4 + j] + j12 * W[2 * 4 + j];
    }
    float S[3][3];
    S[0][0] = cov3d[0 * n + k]; S[0][1] = S[1][0] = cov3d[1 * n + k]; S[0][2] = S[2][0] = cov3d[2 * n + k];
    S[1][1] = cov3d[3 * n + k]; S[1][2] = S[2][1] = cov3d[4 * n + k]; S[2][2] = cov3d[5 * n + k];
    float U0[3], U1[3];
    for (int j = 0; j < 3; ++j) {
      U0[j] = (T0[0] * S[0][j] + T0[1] * S[1][j]) + T0[2] * S[2][j];
      U1[j] = (T1[0] * S[0][j] + T1[1] * S[1][j]) + T1[2] * S[2][j];
    }
    float a = ((U0[0] * T0[0] + U0[1] * T0[1]) + U0[2] * T0[2]) + cfg->lowpass;
    float b = (U0[0] * T1[0] + U0[1] * T1[1]) + U0[2] * T1[2];
    float c = ((U1[0] * T1[0] + U1[1] * T1[1]) + U1[2] * T1[2]) + cfg->lowpass;
    float det = a * c - b * b;
    if (!(det > 0.0f)) continue;
    float ca = c / det, cb = -b / det, cc2 = a / det;
    float mid = 0.5f * (a + c);
    float disc = fmaxf(0.1f, mid * mid - det);
    float lam = mid + sqrtf(disc);
    float r = ceilf(3.0f * sqrtf(lam));
    float mx = cam->fx * txz + cam->cx;
    float my = cam->fy * tyz + cam->cy;
    float fx0 = floorf((mx - r) / (float)cfg->tile_w);
    float fx1 = floorf((mx + r) / (float)cfg->tile_w) + 1.0f;
    float fy0 = floorf((my - r) / (float)cfg->tile_h);
    float fy1 = floorf((my + r) / (float)cfg->tile_h) + 1.0f;
    int x0 = (int)fminf(fmaxf(fx0, 0.0f), (float)tiles_x);
    int x1 = (int)fminf(fmaxf(fx1, 0.0f), (float)tiles_x);
    int y0 = (int)fminf(fmaxf(fy0, 0.0f), (float)tiles_y);
    int y1 = (int)fminf(fmaxf(fy1, 0.0f), (float)tiles_y);
    if (!(x1 > x0 && y1 > y0)) continue;

    depth[k] = t[2];
    mean2d[k] = mx;
    mean2d[n + k] = my;
    cov2d[k] = a; cov2d[n + k] = b; cov2d[2 * n + k] = c;
    conic[k] = ca; conic[n + k] = cb; conic[2 * n + k] = cc2;
    qcoef[k] = ca * kA;
    qcoef[n + k] = cb * (-kLog2e);
    qcoef[2 * n + k] = cc2 * kA;
    radius[k] = r;
    rect[k] = x0; rect[n + k] = y0; rect[2 * n + k] = x1; rect[3 * n + k] = y1;
    {
      uint32_t kept = 0;
      const int64_t area = (int64_t)(x1 - x0) * (y1 - y0);
      for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx)
          kept += (uint32_t)tile_kept(area, mx, my, qcoef[k], qcoef[n + k], qcoef[2 * n + k], opacity[k], tx, ty, cfg);
      touched[k] = kept;
    }

    /* colour along the direction camera centre -> splat centre */
    double d[3] = {(double)mu[0] - cc[0], (double)mu[1] - cc[1], (double)mu[2] - cc[2]};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double Y[16];
    orc_sh_basis(d[0] / dn, d[1] / dn, d[2] / dn, Y);
    for (int ch = 0; ch < 3; ++ch) {
      double v = 0.0;
      for (int i = 0; i < 16; ++i) v += (double)sh[(i * 3 + ch) * n + k] * Y[i];
      v += 0.5;
      rgb[ch * n + k] = v > 0.0 ? v : 0.0;
    }
  }
}

/* ---------------------------------------------------------------------------------- */
/* Binning: emit one (tile, depth) key per touched tile, stable sort, tile ranges.     */
/* ---------------------------------------------------------------------------------- */

static void merge_sort_pairs(uint64_t* key, uint32_t* val, uint32_t* idx, int64_t m) {
  /* bottom-up stable merge sort on key; val and idx travel with it */
  uint64_t* k2 = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
  uint32_t* v2 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
  uint32_t* i2 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
  uint64_t *ks = key, *kd = k2;
  uint32_t *vs = val, *vd = v2, *is = idx, *id = i2;
  for (int64_t width = 1; width < m; width *= 2) {
    for (int64_t lo = 0; lo < m; lo += 2 * width) {
      int64_t mid = lo + width < m ? lo + width : m;
      int64_t hi = lo + 2 * width < m ? lo + 2 * width : m;
      int64_t a = lo, b = mid, o = lo;
      while (a < mid && b < hi) {
        if (ks[b] < ks[a]) { kd[o] = ks[b]; vd[o] = vs[b]; id[o] = is[b]; ++b; }
        else { kd[o] = ks[a]; vd[o] = vs[a]; id[o] = is[a]; ++a; }
        ++o;
      }
      while (a < mid) { kd[o] = ks[a]; vd[o] = vs[a]; id[o] = is[a]; ++a; ++o; }
      while (b < hi) { kd[o] = ks[b]; vd[o] = vs[b]; id[o] = is[b]; ++b; ++o; }
    }
    uint64_t* tk = ks; ks = kd; kd = tk;
    uint32_t* tv = vs; vs = vd; vd = tv;
    uint32_t* ti = is; is = id; id = ti;
  }
  if (ks != key) {
    memcpy(key, ks, sizeof(uint64_t) * (size_t)m);
    memcpy(val, vs, sizeof(uint32_t) * (size_t)m);
    memcpy(idx, is, sizeof(uint32_t) * (size_t)m);
  }
  free(k2); free(v2); free(i2);
}

/*
 * Emits, for k ascending and within each rectangle row-major (y then x), one instance
 * with key (tile_base + ty * tiles_x + tx) << 32 | bits(depth_k) and value val_base + k,
 * then sorts stably by key.  emit_index[pos] is the emission index of the instance now at
 * sorted position pos.  Returns the number of instances M, or -M when M > capacity
 * (outputs untouched).  With whole_rect = 0 only the tiles passing the tile test are
 * emitted (touched[k] of them); with whole_rect != 0 every tile of the 3-sigma rectangle
 * of every projected splat is, as the paper's renderer bins a footprint (no tile test).
 */
int64_t orc_bin(int64_t n, const uint32_t* touched, const int32_t* rect, const float* depth,
                const float* mean2d, const float* qcoef, const float* opacity, const orc_config* cfg,
                int32_t tiles_x, uint64_t tile_base, uint32_t val_base, int64_t capacity,
                uint64_t* keys, uint32_t* vals, uint32_t* emit_index, int32_t whole_rect) {
  int64_t m = 0;
  for (int64_t k = 0; k < n; ++k)
    m += whole_rect ? (int64_t)(rect[2 * n + k] - rect[k]) * (rect[3 * n + k] - rect[n + k]) : (int64_t)touched[k];
  if (m > capacity) return -m;
  int64_t e = 0;
  for (int64_t k = 0; k < n; ++k) {
    if (!whole_rect && touched[k] == 0) continue;
    uint32_t dbits;
    memcpy(&dbits, &depth[k], 4);
    const int64_t area = (int64_t)(rect[2 * n + k] - rect[k]) * (rect[3 * n + k] - rect[n + k]);
    for (int32_t ty = rect[n + k]; ty < rect[3 * n + k]; ++ty)
      for (int32_t tx = rect[k]; tx < rect[2 * n + k]; ++tx) {
        if (!whole_rect &&
            !tile_kept(area, mean2d[k], mean2d[n + k], qcoef[k], qcoef[n + k], qcoef[2 * n + k], opacity[k], tx, ty, cfg))
          continue;
        uint64_t tile = tile_base + (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;
        keys[e] = (tile << 32) | (uint64_t)dbits;
        vals[e] = val_base + (uint32_t)k;
        emit_index[e] = (uint32_t)e;
        ++e;
      }
  }
  merge_sort_pairs(keys, vals, emit_index, m);
  return m;
}

/* ranges[2 t], ranges[2 t + 1] = first and one-past-last sorted position of tile t. */
void orc_tile_ranges(int64_t m, const uint64_t* keys, uint64_t tile_base, int64_t n_tiles,
                     uint32_t* ranges) {
  for (int64_t t = 0; t < n_tiles; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
  for (int64_t i = 0; i < m; ++i) {
    int64_t t = (int64_t)((keys[i] >> 32) - tile_base);
    if (t < 0 || t >= n_tiles) continue;
    if (i == 0 || (keys[i - 1] >> 32) != (keys[i] >> 32)) ranges[2 * t] = (uint32_t)i;
    ranges[2 * t + 1] = (uint32_t)(i + 1);
  }
}

/* ---------------------------------------------------------------------------------- */
/* Per-pixel compositing walk (Section 3, Eqs. 2-4).                                    */
/* ---------------------------------------------------------------------------------- */

typedef struct {
  int64_t n;
  const float* mean2d; /* [2n] */
  const float* qcoef;  /* [3n] */
  const float* opacity;
  const double* rgb;   /* [3n] */
} orc_splats;

typedef struct {
  uint32_t pos;   /* position in the tile list */
  uint32_t k;     /* splat index */
  float alpha;    /* binary32 alpha */
} orc_entry;

/*
 * Walks the tile list [s, e) for pixel centre (px, py) and records the composited splats
 * in order.  exclude >= 0 leaves that splat out (the brute-force definition).  Returns
 * the count K; *t32 receives the binary32 transmittance chain's final value and *n_last
 * one past the list position of the last composited splat (0 when none).
 */
static int64_t walk_pixel(const orc_splats* sp, const orc_config* cfg, const uint32_t* vals,
                          uint32_t s, uint32_t e, float px, float py, int64_t exclude,
                          orc_entry* out, float* t32, uint32_t* n_last) {
  float T = 1.0f;
  int64_t K = 0;
  uint32_t last = 0;
  const int64_t n = sp->n;
  for (uint32_t i = s; i < e; ++i) {
    uint32_t k = vals[i];
    if ((int64_t)k == exclude) continue;
    float dx = px - sp->mean2d[k];
    float dy = py - sp->mean2d[n + k];
    float A = sp->qcoef[k], B = sp->qcoef[n + k], C = sp->qcoef[2 * n + k];
    float u = fmaf(A, dx, B * dy);
    float v = C * dy;
    float p = fmaf(u, dx, v * dy);
    float G = orc_exp2r(p);
    float a = fminf(cfg->alpha_max, sp->opacity[k] * G);
    if (a < cfg->alpha_min) continue;
    float Tn = fmaf(-a, T, T);
    if (Tn < cfg->t_min) break;
    out[K].pos = i - s;
    out[K].k = k;
    out[K].alpha = a;
    ++K;
    last = i - s + 1;
    T = Tn;
  }
  *t32 = T;
  *n_last = last;
  return K;
}

static uint32_t max_list(const uint32_t* ranges, int64_t n_tiles) {
  uint32_t mx = 0;
  for (int64_t t = 0; t < n_tiles; ++t) {
    uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
    if (len > mx) mx = len;
  }
  return mx;
}

/* Composite the K recorded entries in binary64: c = sum_k T_k alpha_k c_k (Eq. 4). */
static void composite64(const orc_splats* sp, const orc_entry* ent, int64_t K, double* c,
                        double* T_out) {
  double T = 1.0;
  c[0] = c[1] = c[2] = 0.0;
  for (int64_t i = 0; i < K; ++i) {
    double a = (double)ent[i].alpha;
    for (int ch = 0; ch < 3; ++ch) c[ch] += T * a * sp->rgb[ch * sp->n + ent[i].k];
    T *= (1.0 - a);
  }
  *T_out = T;
}

/*
 * Tiles are independent in the render and in the removal effect (each pixel walks its own
 * tile's list), so both may run over several threads (orc_set_threads; 1 by default).  Every
 * output is written by the one tile that owns it, and the per-splat sums are formed after all
 * tiles from per-instance sums in tile order, so the results do not depend on the number of
 * threads or on which thread took which tile.
 */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

typedef struct {
  const orc_camera* cam;
  const orc_config* cfg;
  orc_splats sp;
  const uint32_t* vals;
  const uint32_t* ranges;
  const uint8_t* tile_mask;
  int64_t exclude;
  /* render outputs (nullable) */
  double* image;
  float* t_final32;
  double* t_final64;
  uint32_t* n_last;
  /* removal-effect inputs and per-instance outputs */
  const float* target;
  double* part_dse;
  double* part_imp;
  double* part_mag; /* nullable: per-instance magnitude sums (orc_removal_magnitude) */
  int tiles_x, tiles_y;
  uint32_t cap;
  int64_t next; /* next tile to take (atomic) */
  void (*tile_fn)(void* job, int64_t t, orc_entry* ent, double* P, double* Tv);
} orc_tile_job;

static void* tile_worker(void* arg) {
  orc_tile_job* job = (orc_tile_job*)arg;
  size_t cap1 = (size_t)job->cap + 1;
  orc_entry* ent = (orc_entry*)malloc(sizeof(orc_entry) * cap1);
  double* P = (double*)malloc(sizeof(double) * 3 * cap1);
  double* Tv = (double*)malloc(sizeof(double) * cap1);
  const int64_t n_tiles = (int64_t)job->tiles_x * job->tiles_y;
  for (;;) {
    int64_t t = __atomic_fetch_add(&job->next, 1, __ATOMIC_RELAXED);
    if (t >= n_tiles) break;
    if (job->tile_mask && !job->tile_mask[t]) continue;
    job->tile_fn(job, t, ent, P, Tv);
  }
  free(ent); free(P); free(Tv);
  return NULL;
}

/* Run job->tile_fn over every tile on g_threads threads (the calling thread included). */
static void run_tiles(orc_tile_job* job) {
  job->next = 0;
  int nt = g_threads;
  pthread_t* th = nt > 1 ? (pthread_t*)malloc(sizeof(pthread_t) * (size_t)(nt - 1)) : NULL;
  int started = 0;
  for (int i = 0; i < nt - 1; ++i)
    if (pthread_create(&th[i], NULL, tile_worker, job) == 0) ++started;
  tile_worker(job);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free(th);
}

static void render_tile(void* arg, int64_t t, orc_entry* ent, double* P, double* Tv) {
  (void)P; (void)Tv;
  orc_tile_job* job = (orc_tile_job*)arg;
  const orc_config* cfg = job->cfg;
  const int W = job->cam->width, H = job->cam->height;
  const int tx = (int)(t % job->tiles_x), ty = (int)(t / job->tiles_x);
  for (int y = ty * cfg->tile_h; y < (ty + 1) * cfg->tile_h && y < H; ++y)
    for (int x = tx * cfg->tile_w; x < (tx + 1) * cfg->tile_w && x < W; ++x) {
      float T32;
      uint32_t nl;
      int64_t K = walk_pixel(&job->sp, cfg, job->vals, job->ranges[2 * t], job->ranges[2 * t + 1], (float)x + 0.5f,
                             (float)y + 0.5f, job->exclude, ent, &T32, &nl);
      double c[3], T64;
      composite64(&job->sp, ent, K, c, &T64);
      int64_t pix = (int64_t)y * W + x;
      for (int ch = 0; ch < 3; ++ch) job->image[(int64_t)ch * H * W + pix] = c[ch];
      if (job->t_final32) job->t_final32[pix] = T32;
      if (job->t_final64) job->t_final64[pix] = T64;
      if (job->n_last) job->n_last[pix] = nl;
    }
}

/*
 * Render one view.  image is planar [3][H][W] binary64; t_final32 / n_last / t_final64
 * per pixel (nullable).  exclude >= 0 renders without that splat.  tile_mask (nullable)
 * restricts the work to tiles with a non-zero mask byte.
 */
void orc_render(const orc_camera* cam, const orc_config* cfg, int64_t n, const float* mean2d,
                const float* qcoef, const float* opacity, const double* rgb, const uint32_t* vals,
                const uint32_t* ranges, int64_t exclude, const uint8_t* tile_mask, double* image,
                float* t_final32, double* t_final64, uint32_t* n_last) {
  orc_tile_job job;
  memset(&job, 0, sizeof(job));
  job.cam = cam;
  job.cfg = cfg;
  job.sp = (orc_splats){n, mean2d, qcoef, opacity, rgb};
  job.vals = vals;
  job.ranges = ranges;
  job.tile_mask = tile_mask;
  job.exclude = exclude;
  job.image = image;
  job.t_final32 = t_final32;
  job.t_final64 = t_final64;
  job.n_last = n_last;
  job.tiles_x = (cam->width + cfg->tile_w - 1) / cfg->tile_w;
  job.tiles_y = (cam->height + cfg->tile_h - 1) / cfg->tile_h;
  job.cap = max_list(ranges, (int64_t)job.tiles_x * job.tiles_y);
  job.tile_fn = render_tile;
  run_tiles(&job);
}

/*
 * Removal effect of every splat on one view (Section IV-B).
 *
 * For each pixel: the composited splats i = 0..K-1 with binary32 alpha_i, binary64
 * transmittance T_i and partial colours P_i (Eq. partial colour).  For each i:
 *   PD = (P_i + (P_K - P_{i+1}) / (1 - alpha_i)) - P_K          (Eq. pruning difference)
 *   dSE = sum over channels of PD^2 + 2 PD (c - c_t)             (Eq. pixel squared error)
 * with c = P_K and c_t the target.  Per tile instance (sorted list position) the sums over the
 * tile's pixels (row-major) of dSE and of T_i alpha_i are formed; then dsse[k] and imp[k]
 * (both nullable, accumulated) receive, tile after tile, the sums of splat k's instances.
 * inst_dse / inst_imp (nullable) receive the per-instance sums.  tile_mask as in orc_render.
 */
static void removal_tile(void* arg, int64_t t, orc_entry* ent, double* P, double* Tv) {
  orc_tile_job* job = (orc_tile_job*)arg;
  const orc_config* cfg = job->cfg;
  const int W = job->cam->width, H = job->cam->height;
  const int64_t n = job->sp.n;
  const double* rgb = job->sp.rgb;
  const int tx = (int)(t % job->tiles_x), ty = (int)(t / job->tiles_x);
  uint32_t s = job->ranges[2 * t], e = job->ranges[2 * t + 1];
  for (uint32_t i = s; i < e; ++i) job->part_dse[i] = job->part_imp[i] = 0.0;
  if (job->part_mag)
    for (uint32_t i = s; i < e; ++i) job->part_mag[i] = 0.0;
  for (int y = ty * cfg->tile_h; y < (ty + 1) * cfg->tile_h && y < H; ++y)
    for (int x = tx * cfg->tile_w; x < (tx + 1) * cfg->tile_w && x < W; ++x) {
      float T32;
      uint32_t nl;
      int64_t K = walk_pixel(&job->sp, cfg, job->vals, s, e, (float)x + 0.5f, (float)y + 0.5f, -1, ent,
                             &T32, &nl);
      /* P_0 = 0, P_{i+1} = P_i + T_i alpha_i c_i, T_0 = 1, T_{i+1} = T_i (1 - alpha_i) */
      double T = 1.0;
      P[0] = P[1] = P[2] = 0.0;
      for (int64_t i = 0; i < K; ++i) {
        double a = (double)ent[i].alpha;
        Tv[i] = T;
        for (int ch = 0; ch < 3; ++ch)
          P[3 * (i + 1) + ch] = P[3 * i + ch] + T * a * rgb[ch * n + ent[i].k];
        T *= (1.0 - a);
      }
      int64_t pix = (int64_t)y * W + x;
      double diff[3];
      for (int ch = 0; ch < 3; ++ch) diff[ch] = P[3 * K + ch] - (double)job->target[(int64_t)ch * H * W + pix];
      for (int64_t i = 0; i < K; ++i) {
        double a = (double)ent[i].alpha;
        double dse = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
          double PK = P[3 * K + ch];
          double pd = (P[3 * i + ch] + (PK - P[3 * (i + 1) + ch]) / (1.0 - a)) - PK;
          dse += pd * pd + 2.0 * pd * diff[ch];
        }
        double w = Tv[i] * a;
        job->part_dse[s + ent[i].pos] += dse;
        job->part_imp[s + ent[i].pos] += w;
        if (job->part_mag) {
          /* magnitude of the terms dSE is formed from: the two parts of PD (the later splats'
           * colour behind this one, alpha / (1 - alpha) (P_K - P_{i+1}), and T alpha c) times
           * |2 PD + 2 (c - c_t)| bounded by 2 |PD| + 2 |c - c_t|, per channel */
          double mg = 0.0;
          for (int ch = 0; ch < 3; ++ch) {
            double PK = P[3 * K + ch];
            double behind = (PK - P[3 * (i + 1) + ch]) * a / (1.0 - a);
            double own = Tv[i] * a * rgb[ch * n + ent[i].k];
            double pd = (P[3 * i + ch] + (PK - P[3 * (i + 1) + ch]) / (1.0 - a)) - PK;
            mg += (fabs(behind) + fabs(own)) * (2.0 * fabs(pd) + 2.0 * fabs(diff[ch]));
          }
          job->part_mag[s + ent[i].pos] += mg;
        }
      }
    }
}

static void removal_effect_impl(const orc_camera* cam, const orc_config* cfg, int64_t n,
                                const float* mean2d, const float* qcoef, const float* opacity,
                                const double* rgb, const uint32_t* vals, const uint32_t* ranges,
                                const float* target, const uint8_t* tile_mask, double* dsse, double* imp,
                                double* inst_dse, double* inst_imp, double* mag, double* inst_mag) {
  orc_tile_job job;
  memset(&job, 0, sizeof(job));
  job.cam = cam;
  job.cfg = cfg;
  job.sp = (orc_splats){n, mean2d, qcoef, opacity, rgb};
  job.vals = vals;
  job.ranges = ranges;
  job.tile_mask = tile_mask;
  job.exclude = -1;
  job.target = target;
  job.tiles_x = (cam->width + cfg->tile_w - 1) / cfg->tile_w;
  job.tiles_y = (cam->height + cfg->tile_h - 1) / cfg->tile_h;
  const int64_t n_tiles = (int64_t)job.tiles_x * job.tiles_y;
  job.cap = max_list(ranges, n_tiles);
  uint32_t m = 0;
  for (int64_t t = 0; t < n_tiles; ++t)
    if (ranges[2 * t + 1] > m) m = ranges[2 * t + 1];
  job.part_dse = (double*)calloc((size_t)m + 1, sizeof(double));
  job.part_imp = (double*)calloc((size_t)m + 1, sizeof(double));
  job.part_mag = (mag || inst_mag) ? (double*)calloc((size_t)m + 1, sizeof(double)) : NULL;
  job.tile_fn = removal_tile;
  run_tiles(&job);
  for (int64_t t = 0; t < n_tiles; ++t) {
    if (tile_mask && !tile_mask[t]) continue;
    for (uint32_t i = ranges[2 * t]; i < ranges[2 * t + 1]; ++i) {
      uint32_t k = vals[i];
      if (dsse) dsse[k] += job.part_dse[i];
      if (imp) imp[k] += job.part_imp[i];
      if (inst_dse) inst_dse[i] = job.part_dse[i];
      if (inst_imp) inst_imp[i] = job.part_imp[i];
      if (mag) mag[k] += job.part_mag[i];
      if (inst_mag) inst_mag[i] = job.part_mag[i];
    }
  }
  free(job.part_dse);
  free(job.part_imp);
  free(job.part_mag);
}

void orc_removal_effect(const orc_camera* cam, const orc_config* cfg, int64_t n,
                        const float* mean2d, const float* qcoef, const float* opacity,
                        const double* rgb, const uint32_t* vals, const uint32_t* ranges,
                        const float* target, const uint8_t* tile_mask, double* dsse, double* imp,
                        double* inst_dse, double* inst_imp) {
  removal_effect_impl(cam, cfg, n, mean2d, qcoef, opacity, rgb, vals, ranges, target, tile_mask, dsse, imp,
                      inst_dse, inst_imp, NULL, NULL);
}

/*
 * The scale of the rounding of a binary32 evaluation of the removal effect: per splat (mag,
 * accumulated) and per tile instance (inst_mag), the sum over the composited pixels of
 * sum_ch (|alpha/(1 - alpha) S_>| + |T alpha c|) (2 |PD| + 2 |c - c_t|) -- the magnitudes of the
 * two parts of PD times the bound of the factor that multiplies an error of PD in dSE.  A
 * quantity for tolerances, not part of the method; both outputs nullable.
 */
void orc_removal_magnitude(const orc_camera* cam, const orc_config* cfg, int64_t n,
                           const float* mean2d, const float* qcoef, const float* opacity,
                           const double* rgb, const uint32_t* vals, const uint32_t* ranges,
                           const float* target, const uint8_t* tile_mask, double* mag, double* inst_mag) {
  removal_effect_impl(cam, cfg, n, mean2d, qcoef, opacity, rgb, vals, ranges, target, tile_mask, NULL, NULL,
                      NULL, NULL, mag, inst_mag);
}

/*
 * The definition itself (Eq. pixel squared error, first line): for splat `exclude`,
 * sum over pixels and channels of (c~ - c_t)^2 - (c - c_t)^2, where c~ is the binary64
 * re-render without that splat.  image (binary64 planar) is the full render.
 */
double orc_removal_bruteforce(const orc_camera* cam, const orc_config* cfg, int64_t n,
                              const float* mean2d, const float* qcoef, const float* opacity,
                              const double* rgb, const uint32_t* vals, const uint32_t* ranges,
                              const float* target, const double* image, int64_t exclude) {
  const int W = cam->width, H = cam->height;
  double* img2 = (double*)malloc(sizeof(double) * 3 * (size_t)W * (size_t)H);
  orc_render(cam, cfg, n, mean2d, qcoef, opacity, rgb, vals, ranges, exclude, NULL, img2, NULL,
             NULL, NULL);
  double acc = 0.0;
  for (int64_t i = 0; i < 3 * (int64_t)W * H; ++i) {
    double t = (double)target[i];
    double d1 = img2[i] - t, d0 = image[i] - t;
    acc += d1 * d1 - d0 * d0;
  }
  free(img2);
  return acc;
}

/*
 * The composited splats of every pixel, in compositing order (the decisions of the walk
 * above).  Pixels are visited tile by tile, row-major inside a tile; entry e has pixel index
 * pix[e] = y * W + x, splat k[e] and list position pos[e].  Returns the number of entries,
 * or -(count) when it exceeds cap (outputs then hold the first cap entries).
 */
int64_t orc_pixel_lists(const orc_camera* cam, const orc_config* cfg, int64_t n, const float* mean2d,
                        const float* qcoef, const float* opacity, const uint32_t* vals,
                        const uint32_t* ranges, int64_t cap, int64_t* pix, uint32_t* k_out,
                        uint32_t* pos_out) {
  const int W = cam->width, H = cam->height;
  const int tiles_x = (W + cfg->tile_w - 1) / cfg->tile_w;
  const int tiles_y = (H + cfg->tile_h - 1) / cfg->tile_h;
  orc_splats sp = {n, mean2d, qcoef, opacity, NULL};
  uint32_t mx = max_list(ranges, (int64_t)tiles_x * tiles_y);
  orc_entry* ent = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)(mx > 0 ? mx : 1));
  int64_t count = 0;
  for (int ty = 0; ty < tiles_y; ++ty)
    for (int tx = 0; tx < tiles_x; ++tx) {
      int64_t t = (int64_t)ty * tiles_x + tx;
      for (int y = ty * cfg->tile_h; y < (ty + 1) * cfg->tile_h && y < H; ++y)
        for (int x = tx * cfg->tile_w; x < (tx + 1) * cfg->tile_w && x < W; ++x) {
          float T32;
          uint32_t nl;
          int64_t K = walk_pixel(&sp, cfg, vals, ranges[2 * t], ranges[2 * t + 1], (float)x + 0.5f,
                                 (float)y + 0.5f, -1, ent, &T32, &nl);
          for (int64_t i = 0; i < K; ++i, ++count) {
            if (count < cap) {
              pix[count] = (int64_t)y * W + x;
              k_out[count] = ent[i].k;
              pos_out[count] = ent[i].pos;
            }
          }
        }
    }
  free(ent);
  return count <= cap ? count : -count;
}