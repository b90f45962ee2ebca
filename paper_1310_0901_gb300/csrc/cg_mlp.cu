// cg_mlp.cu -- training kernels of the batch-split cost model: a small
// one-hidden-layer ReLU network, y = b2 + sum_j w2[j] relu(b1[j] +
// sum_k x[k] W1[k][j]), fitted to log2(batch ms) by mean squared error with
// full-batch Adam.  Forward and backward are this file's own kernels:
// block b computes the loss and gradient contributions of its share of the
// samples into its own slot (no atomics), and one reduction kernel sums
// the slots in a fixed order and applies the Adam step.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <random>
#include <vector>

#include "cg_ctx.h"

namespace cgi {

constexpr int kMlpBlocks = 64;

// parameters, packed: W1[D][H] | b1[H] | w2[H] | b2
__host__ __device__ inline int mlp_nparams(int D, int H) { return D * H + 2 * H + 1; }

__global__ void mlp_grad_kernel(const float *__restrict__ x, const float *__restrict__ t, int n,
                                int D, int H, const float *__restrict__ p,
                                float *__restrict__ part /* [blocks][P + 1] */) {
  extern __shared__ float red[];  // one partial sum per warp
  const int P = mlp_nparams(D, H);
  const int j = threadIdx.x;  // hidden unit
  const float *W1 = p, *b1 = p + D * H, *w2 = b1 + H, *b2 = w2 + H;
  float *g = part + (size_t)blockIdx.x * (P + 1);
  // this thread's gradient accumulators live in the block's slot
  float gb1 = 0.f, gw2 = 0.f;
  for (int k = 0; k < D; k++) g[k * H + j] = 0.f;
  float gb2 = 0.f, loss = 0.f;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  for (int i = i0; i < i1; i++) {
    const float *xi = x + (size_t)i * D;
    float z = b1[j];
    for (int k = 0; k < D; k++) z += xi[k] * W1[k * H + j];
    const float h = z > 0.f ? z : 0.f;
    // y = b2 + sum_j h_j w2_j (block reduction)
    float v = h * w2[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((j & 31) == 0) red[j >> 5] = v;
    __syncthreads();
    float y = b2[0];
    for (int w = 0; w < (H + 31) / 32; w++) y += red[w];
    __syncthreads();
    const float r = y - t[i];
    const float d = 2.f * r / (float)n;  // d loss / d y
    if (j == 0) {
      loss += r * r / (float)n;
      gb2 += d;
    }
    gw2 += d * h;
    const float dz = z > 0.f ? d * w2[j] : 0.f;
    gb1 += dz;
    for (int k = 0; k < D; k++) g[k * H + j] += xi[k] * dz;
  }
  g[D * H + j] = gb1;
  g[D * H + H + j] = gw2;
  if (j == 0) {
    g[D * H + 2 * H] = gb2;
    g[P] = loss;
  }
}

// Sum the block slots (fixed order) into grad[P + 1]; with lr > 0 also
// take one Adam step on p (moments m, v; step count t).
__global__ void mlp_reduce_adam_kernel(const float *__restrict__ part, int blocks, int P,
                                       float *__restrict__ grad, float *__restrict__ p,
                                       float *__restrict__ m, float *__restrict__ v, int t,
                                       float lr) {
  for (int q = threadIdx.x; q <= P; q += blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < blocks; b++) s += part[(size_t)b * (P + 1) + q];
    grad[q] = s;
    if (lr > 0.f && q < P) {
      const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
      m[q] = b1 * m[q] + (1.f - b1) * s;
      v[q] = b2 * v[q] + (1.f - b2) * s * s;
      const float mh = m[q] / (1.f - powf(b1, (float)t));
      const float vh = v[q] / (1.f - powf(b2, (float)t));
      p[q] -= lr * mh / (sqrtf(vh) + eps);
    }
  }
}

}  // namespace cgi

using namespace cgi;

namespace {

// inputs standardised on the host: (x - mu) / sigma per column
void standardise(const float *x, uint32_t n, int D, std::vector<float> &mu, std::vector<float> &sd,
                 std::vector<float> &xs, bool fit) {
  if (fit) {
    mu.assign(D, 0.f);
    sd.assign(D, 0.f);
    for (uint32_t i = 0; i < n; i++)
      for (int k = 0; k < D; k++) mu[k] += x[(size_t)i * D + k] / (float)n;
    for (uint32_t i = 0; i < n; i++)
      for (int k = 0; k < D; k++) {
        const float d = x[(size_t)i * D + k] - mu[k];
        sd[k] += d * d / (float)n;
      }
    for (int k = 0; k < D; k++) sd[k] = sd[k] > 1e-12f ? std::sqrt(sd[k]) : 1.f;
  }
  xs.resize((size_t)n * D);
  for (uint32_t i = 0; i < n; i++)
    for (int k = 0; k < D; k++) xs[(size_t)i * D + k] = (x[(size_t)i * D + k] - mu[k]) / sd[k];
}

struct MlpDev {
  float *x = nullptr, *t = nullptr, *p = nullptr, *m = nullptr, *v = nullptr, *part = nullptr,
        *grad = nullptr;
  ~MlpDev() {
    for (float *q : {x, t, p, m, v, part, grad})
      if (q) cudaFree(q);
  }
};

cg_status mlp_setup(MlpDev &d, const std::vector<float> &xs, const float *t, uint32_t n, int P) {
  CG_CUDA(cudaMalloc(&d.x, xs.size() * sizeof(float)));
  CG_CUDA(cudaMalloc(&d.t, (size_t)n * sizeof(float)));
  CG_CUDA(cudaMalloc(&d.p, (size_t)P * sizeof(float)));
  CG_CUDA(cudaMalloc(&d.m, (size_t)P * sizeof(float)));
  CG_CUDA(cudaMalloc(&d.v, (size_t)P * sizeof(float)));
  CG_CUDA(cudaMalloc(&d.part, (size_t)kMlpBlocks * (P + 1) * sizeof(float)));
  CG_CUDA(cudaMalloc(&d.grad, (size_t)(P + 1) * sizeof(float)));
  CG_CUDA(cudaMemcpy(d.x, xs.data(), xs.size() * sizeof(float), cudaMemcpyHostToDevice));
  CG_CUDA(cudaMemcpy(d.t, t, (size_t)n * sizeof(float), cudaMemcpyHostToDevice));
  CG_CUDA(cudaMemset(d.m, 0, (size_t)P * sizeof(float)));
  CG_CUDA(cudaMemset(d.v, 0, (size_t)P * sizeof(float)));
  return CG_OK;
}

cg_status mlp_step(const MlpDev &d, uint32_t n, int D, int H, int step, float lr,
                   cudaStream_t st) {
  const int P = mlp_nparams(D, H);
  const int blocks = (int)std::min<uint32_t>(kMlpBlocks, std::max<uint32_t>(1, n));
  const size_t smem = 32 * sizeof(float);
  mlp_grad_kernel<<<blocks, H, smem, st>>>(d.x, d.t, (int)n, D, H, d.p, d.part);
  CG_CUDA(cudaGetLastError());
  mlp_reduce_adam_kernel<<<1, 256, 0, st>>>(d.part, blocks, P, d.grad, d.p, d.m, d.v, step, lr);
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

}  // namespace

extern "C" {

cg_status cg_mlp_grad(const float *x, const float *t, uint32_t n, uint32_t hidden,
                      const float *weights, float *grads, float *loss, void *stream) {
  if (!x || !t || !weights || !grads || !n) return set_error(CG_E_ARG, "NULL argument");
  if (hidden == 0 || hidden > 1024 || hidden % 32)
    return set_error(CG_E_ARG, "hidden must be a multiple of 32 in 32..1024");
  const int D = CG_NFEAT + 1, H = (int)hidden, P = mlp_nparams(D, H);
  std::vector<float> mu(weights, weights + D), sd(weights + D, weights + 2 * D), xs;
  standardise(x, n, D, mu, sd, xs, false);
  MlpDev d;
  CG_TRY(mlp_setup(d, xs, t, n, P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_CUDA(cudaMemcpy(d.p, weights + 2 * D, (size_t)P * sizeof(float), cudaMemcpyHostToDevice));
  CG_TRY(mlp_step(d, n, D, H, 1, 0.f, st));
  std::vector<float> g(P + 1);
  CG_CUDA(cudaStreamSynchronize(st));
  CG_CUDA(cudaMemcpy(g.data(), d.grad, (size_t)(P + 1) * sizeof(float), cudaMemcpyDeviceToHost));
  for (int k = 0; k < 2 * D; k++) grads[k] = 0.f;  // mu and sigma are not trained
  for (int k = 0; k < P; k++) grads[2 * D + k] = g[k];
  if (loss) *loss = g[P];
  return CG_OK;
}

cg_status cg_mlp_fit(const float *x, const float *t, uint32_t n, uint32_t hidden,
                     uint32_t epochs, float lr, uint64_t seed, float *weights, float *losses,
                     void *stream) {
  if (!x || !t || !weights || !n) return set_error(CG_E_ARG, "NULL argument");
  if (hidden == 0 || hidden > 1024 || hidden % 32)
    return set_error(CG_E_ARG, "hidden must be a multiple of 32 in 32..1024");
  const int D = CG_NFEAT + 1, H = (int)hidden, P = mlp_nparams(D, H);
  std::vector<float> mu, sd, xs;
  standardise(x, n, D, mu, sd, xs, true);
  // He-style initialisation from a seeded generator; b2 starts at mean(t)
  std::vector<float> p0(P, 0.f);
  std::mt19937_64 gen(seed);
  std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (float)D));
  for (int k = 0; k < D * H; k++) p0[k] = nd(gen);
  std::normal_distribution<float> nd2(0.f, std::sqrt(1.f / (float)H));
  for (int j = 0; j < H; j++) p0[D * H + H + j] = nd2(gen);
  double tm = 0;
  for (uint32_t i = 0; i < n; i++) tm += t[i];
  p0[D * H + 2 * H] = (float)(tm / n);
  MlpDev d;
  CG_TRY(mlp_setup(d, xs, t, n, P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_CUDA(cudaMemcpy(d.p, p0.data(), (size_t)P * sizeof(float), cudaMemcpyHostToDevice));
  for (uint32_t e = 0; e < epochs; e++) {
    CG_TRY(mlp_step(d, n, D, H, (int)e + 1, lr, st));
    if (losses)
      CG_CUDA(cudaMemcpyAsync(losses + e, d.grad + P, sizeof(float), cudaMemcpyDeviceToHost, st));
  }
  CG_CUDA(cudaStreamSynchronize(st));
  std::vector<float> p(P);
  CG_CUDA(cudaMemcpy(p.data(), d.p, (size_t)P * sizeof(float), cudaMemcpyDeviceToHost));
  for (int k = 0; k < D; k++) {
    weights[k] = mu[k];
    weights[D + k] = sd[k];
  }
  for (int k = 0; k < P; k++) weights[2 * D + k] = p[k];
  return CG_OK;
}

}  // extern "C"
