// fz_train.cu -- training of the per-block predictor selector network on
// labels produced by the exhaustive trial (the auto-selection of modules
// named as future work in FZModules §5).
//
// Objective: mean softmax cross-entropy of the 4 predictor logits at the
// exhaustive label.  The forward pass uses the bfloat16 rounding of the
// float32 master weights (the weights inference will see) and float32
// accumulation; the gradient is taken with respect to the master weights.
//
//   k_mlp_grad    -- one CTA per 64 samples: forward, softmax, backward and
//                    the CTA's partial gradient, each parameter summed over
//                    the CTA's samples in sample order (no float atomics)
//   k_mlp_reduce  -- one thread per parameter: partials summed in CTA order
//   k_adam        -- Adam update of the master weights and their bf16 copy
// The result is deterministic: the same inputs give the same bits.
#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr int kGradThreads = 256;
constexpr int kSamplesPerCta = 64;

struct GradSmem {
  float w[kNWeights];
  float f[kSamplesPerCta][kNFeat];
  float z[kSamplesPerCta][kNHid];
  float dh[kSamplesPerCta][kNHid];
  float dl[kSamplesPerCta][kNPred];
  float loss[kSamplesPerCta];
};

__global__ void __launch_bounds__(kGradThreads) k_mlp_grad(const float *__restrict__ wm,
                                                            const uint16_t *__restrict__ feat,
                                                            const uint8_t *__restrict__ labels, uint32_t n,
                                                            float *partial) {
  extern __shared__ __align__(16) unsigned char g_smem[];
  GradSmem &sm = *reinterpret_cast<GradSmem *>(g_smem);
  const int t = threadIdx.x;
  const uint32_t s0 = blockIdx.x * kSamplesPerCta;
  const int ns = (int)min((uint32_t)kSamplesPerCta, n - s0);
  const float inv_n = 1.0f / (float)n;
  for (int i = t; i < kNWeights; i += kGradThreads) sm.w[i] = bf16_to_f32(f32_to_bf16_rne(wm[i]));
  for (int i = t; i < kSamplesPerCta * kNFeat; i += kGradThreads) {
    const int s = i / kNFeat, k = i % kNFeat;
    sm.f[s][k] = s < ns ? bf16_to_f32(feat[(uint64_t)(s0 + s) * kNFeat + k]) : 0.0f;
  }
  __syncthreads();
  // forward: hidden pre-activations
  for (int i = t; i < kSamplesPerCta * kNHid; i += kGradThreads) {
    const int s = i / kNHid, j = i % kNHid;
    float acc = sm.w[kOffB1 + j];
#pragma unroll 8
    for (int k = 0; k < kNFeat; ++k) acc = __fmaf_rn(sm.w[kOffW1 + j * kNFeat + k], sm.f[s][k], acc);
    sm.z[s][j] = acc;
  }
  __syncthreads();
  // logits, softmax and loss: one thread per sample
  if (t < kSamplesPerCta) {
    const int s = t;
    float lg[kNPred], mx = -3.0e38f;
    for (int i = 0; i < kNPred; ++i) {
      float acc = sm.w[kOffB2 + i];
      for (int j = 0; j < kNHid; ++j) acc = __fmaf_rn(sm.w[kOffW2 + i * kNHid + j], fmaxf(sm.z[s][j], 0.0f), acc);
      lg[i] = acc;
      mx = fmaxf(mx, acc);
    }
    float den = 0.0f, p[kNPred];
    for (int i = 0; i < kNPred; ++i) { p[i] = expf(lg[i] - mx); den += p[i]; }
    const int lab = s < ns ? labels[s0 + s] : 0;
    for (int i = 0; i < kNPred; ++i) {
      p[i] /= den;
      sm.dl[s][i] = s < ns ? (p[i] - (i == lab ? 1.0f : 0.0f)) * inv_n : 0.0f;
    }
    sm.loss[s] = s < ns ? -(lg[lab] - mx - logf(den)) : 0.0f;
  }
  __syncthreads();
  // hidden gradients
  for (int i = t; i < kSamplesPerCta * kNHid; i += kGradThreads) {
    const int s = i / kNHid, j = i % kNHid;
    float a = 0.0f;
    for (int k = 0; k < kNPred; ++k) a = __fmaf_rn(sm.w[kOffW2 + k * kNHid + j], sm.dl[s][k], a);
    sm.dh[s][j] = sm.z[s][j] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  // this CTA's partial gradient: each parameter summed over samples in order
  float *out = partial + (uint64_t)blockIdx.x * (kNWeights + 1);
  for (int q = t; q < kNWeights; q += kGradThreads) {
    float acc = 0.0f;
    if (q < kOffB1) {
      const int j = q / kNFeat, k = q % kNFeat;
      for (int s = 0; s < ns; ++s) acc = __fmaf_rn(sm.dh[s][j], sm.f[s][k], acc);
    } else if (q < kOffW2) {
      const int j = q - kOffB1;
      for (int s = 0; s < ns; ++s) acc += sm.dh[s][j];
    } else if (q < kOffB2) {
      const int i = (q - kOffW2) / kNHid, j = (q - kOffW2) % kNHid;
      for (int s = 0; s < ns; ++s) acc = __fmaf_rn(sm.dl[s][i], fmaxf(sm.z[s][j], 0.0f), acc);
    } else {
      const int i = q - kOffB2;
      for (int s = 0; s < ns; ++s) acc += sm.dl[s][i];
    }
    out[q] = acc;
  }
  if (t == 0) {
    float l = 0.0f;
    for (int s = 0; s < ns; ++s) l += sm.loss[s];
    out[kNWeights] = l;
  }
}

__global__ void k_mlp_reduce(const float *partial, uint32_t n_cta, uint32_t n, float *grad, float *loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > kNWeights) return;
  float acc = 0.0f;
  for (uint32_t c = 0; c < n_cta; ++c) acc += partial[(uint64_t)c * (kNWeights + 1) + q];
  if (q < kNWeights) grad[q] = acc;
  else if (loss) *loss = acc / (float)n;
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, uint16_t *wb, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kNWeights) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.0f - b1) * gq;
  const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  w[q] = wq;
  if (wb) wb[q] = f32_to_bf16_rne(wq);
}

}  // namespace

size_t mlp_partial_floats(uint32_t n) {
  return (size_t)((n + kSamplesPerCta - 1) / kSamplesPerCta) * (kNWeights + 1);
}

cudaError_t launch_mlp_grad(const float *w, const uint16_t *feat, const uint8_t *labels, uint32_t n,
                            float *partial, float *grad, float *loss, cudaStream_t s) {
  const uint32_t n_cta = (n + kSamplesPerCta - 1) / kSamplesPerCta;
  const int smem = (int)sizeof(GradSmem);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_mlp_grad<<<n_cta, kGradThreads, smem, s>>>(w, feat, labels, n, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_mlp_reduce<<<(kNWeights + 1 + 255) / 256, 256, 0, s>>>(partial, n_cta, n, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *w, const float *grad, float *m, float *v, uint16_t *w_bf16, uint32_t step, float lr,
                        float beta1, float beta2, float eps, cudaStream_t s) {
  // bias corrections 1 - beta^t in double: in float the subtraction cancels
  // most of the digits of beta^t for small t
  const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
  k_adam<<<(kNWeights + 255) / 256, 256, 0, s>>>(w, grad, m, v, w_bf16, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace fz
