// adam.cu -- fused Adam step over all parameter planes of a scene (the optimiser of the
// fine-tuning loop: the original 3DGS training routine, Section IV-F).  One thread per scalar,
// six learning-rate groups (means, log-scales, quaternions, opacity logits, SH DC, SH rest):
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   p <- p - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)     (Kingma & Ba 2015)
// A parameter whose gradient is 0 and whose moments are 0 does not move (an infinite opacity
// logit of a pruned splat stays infinite).  The scheduled form reads t from a device counter and
// the per-step factors from a table the host filled (potr_adam_schedule), so a fine-tuning step
// can be captured once in a CUDA graph and replayed.
#include "potr_device.cuh"

namespace potr {
namespace {

struct AdamGroup {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t count;
  float step_size;  // lr / (1 - b1^t)
};

struct AdamGroups {
  AdamGroup g[6];
};

constexpr int kSchedWords = 7;  // per step: the six groups' lr / (1 - b1^t), then 1 / sqrt(1 - b2^t)

// sched (nullable): the factors of step *d_step + 1 are row *d_step of sched (n_sched rows);
// past the table nothing is updated.
__global__ void __launch_bounds__(256) adam_kernel(AdamGroups groups, float b1, float b2, float inv_sqrt_bc2,
                                                   float eps, const float* __restrict__ sched,
                                                   const uint32_t* __restrict__ d_step, int64_t n_sched) {
  const float* row = nullptr;
  if (sched) {
    const uint32_t t = *d_step;
    if ((int64_t)t >= n_sched) return;
    row = sched + (int64_t)t * kSchedWords;
    inv_sqrt_bc2 = row[6];
  }
  for (int gi = 0; gi < 6; ++gi) {
    const AdamGroup& G = groups.g[gi];
    const float step_size = row ? row[gi] : G.step_size;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.count; i += (int64_t)gridDim.x * blockDim.x) {
      const float g = G.g[i];
      const float m = b1 * G.m[i] + (1.0f - b1) * g;
      const float v = b2 * G.v[i] + (1.0f - b2) * g * g;
      G.m[i] = m;
      G.v[i] = v;
      if (m != 0.0f) G.p[i] -= step_size * m / (sqrtf(v) * inv_sqrt_bc2 + eps);
    }
  }
}

__global__ void adam_count_kernel(uint32_t* d_step) { *d_step += 1u; }

// The factors of one step, as the host computes them for both forms.
void step_factors(int64_t step, const float* lr, float beta1, float beta2, float* out) {
  const double bc1 = 1.0 - pow((double)beta1, (double)step);
  const double bc2 = 1.0 - pow((double)beta2, (double)step);
  for (int i = 0; i < 6; ++i) out[i] = (float)((double)lr[i] / bc1);
  out[6] = (float)(1.0 / sqrt(bc2));
}

bool groups_for(const potr_scene_grads* params, const potr_scene_grads* grads, const potr_scene_grads* m,
                const potr_scene_grads* v, int64_t n, AdamGroups& G) {
  const potr_scene_grads* s4[4] = {params, grads, m, v};
  for (const potr_scene_grads* s : s4)
    if (!s || !s->means || !s->log_scales || !s->quats || !s->opacity_logits || !s->sh) return false;
  // groups: means, log-scales, quaternions, opacity logits, SH DC (planes 0..2), SH rest (3..47)
  auto groups_of = [n](const potr_scene_grads* s, float** out) {
    out[0] = s->means;
    out[1] = s->log_scales;
    out[2] = s->quats;
    out[3] = s->opacity_logits;
    out[4] = s->sh;
    out[5] = s->sh + 3 * n;
  };
  float *P[6], *Gr[6], *M[6], *V[6];
  groups_of(params, P);
  groups_of(grads, Gr);
  groups_of(m, M);
  groups_of(v, V);
  const int64_t cnt[6] = {3 * n, 3 * n, 4 * n, n, 3 * n, 45 * n};
  for (int i = 0; i < 6; ++i) {
    G.g[i].p = P[i];
    G.g[i].g = Gr[i];
    G.g[i].m = M[i];
    G.g[i].v = V[i];
    G.g[i].count = cnt[i];
    G.g[i].step_size = 0.0f;
  }
  return true;
}

unsigned adam_blocks(int64_t n) {
  int64_t blocks = (59 * n / 6 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

}  // namespace
}  // namespace potr

extern "C" potr_status potr_adam_step(const potr_scene_grads* params, const potr_scene_grads* grads,
                                      const potr_scene_grads* m, const potr_scene_grads* v, int64_t n, int64_t step,
                                      const float* lr, float beta1, float beta2, float eps, potr_stream_t stream) {
  using namespace potr;
  if (!params || !grads || !m || !v || !lr || n <= 0 || step < 1) return POTR_ERR_INVALID_ARGUMENT;
  if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
    return POTR_ERR_INVALID_ARGUMENT;
  AdamGroups G;
  if (!groups_for(params, grads, m, v, n, G)) return POTR_ERR_INVALID_ARGUMENT;
  float f[kSchedWords];
  step_factors(step, lr, beta1, beta2, f);
  for (int i = 0; i < 6; ++i) G.g[i].step_size = f[i];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  adam_kernel<<<adam_blocks(n), 256, 0, s>>>(G, beta1, beta2, f[6], eps, nullptr, nullptr, 0);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}

extern "C" potr_status potr_adam_schedule(int64_t first_step, int64_t count, const float* lr, float beta1,
                                          float beta2, float* out) {
  using namespace potr;
  if (!lr || !out || first_step < 1 || count < 0) return POTR_ERR_INVALID_ARGUMENT;
  if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f)) return POTR_ERR_INVALID_ARGUMENT;
  for (int64_t i = 0; i < count; ++i) step_factors(first_step + i, lr, beta1, beta2, out + i * kSchedWords);
  return POTR_OK;
}

extern "C" potr_status potr_adam_step_scheduled(const potr_scene_grads* params, const potr_scene_grads* grads,
                                                const potr_scene_grads* m, const potr_scene_grads* v, int64_t n,
                                                const float* d_sched, int64_t n_sched, uint32_t* d_step, float beta1,
                                                float beta2, float eps, potr_stream_t stream) {
  using namespace potr;
  if (!params || !grads || !m || !v || !d_sched || !d_step || n <= 0 || n_sched < 1) return POTR_ERR_INVALID_ARGUMENT;
  if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
    return POTR_ERR_INVALID_ARGUMENT;
  AdamGroups G;
  if (!groups_for(params, grads, m, v, n, G)) return POTR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  adam_kernel<<<adam_blocks(n), 256, 0, s>>>(G, beta1, beta2, 0.0f, eps, d_sched, d_step, n_sched);
  POTR_CHECK_LAUNCH();
  adam_count_kernel<<<1, 1, 0, s>>>(d_step);
  POTR_CHECK_LAUNCH();
  return POTR_OK;
}
