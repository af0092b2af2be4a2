// Training of the per-site noise-scale network (learned extension, not in the
// paper): forward/backward in FP32 over sampled per-site inputs, the correlator
// loss in its Gram form, deterministic gradient reduction, and Adam.
//
// Loss (runs r, included wave vectors k, hydrodynamic pairs p):
//   L = 1/(R P K) sum_r sum_{k,p} | D_rp(k) + sum_c (m_rc - 1) G^c_rp(k) |^2,
//   D = S^plain - delta_p,  m_rc = mean_b s_c(x_rb)^2,
// which expands per run into d0 + 2 g.(m-1) + (m-1)^T H (m-1) with
//   d0 = sum |D|^2,  g_c = Re sum D^* G^c,  H_cc' = Re sum G^c* G^c'.
// flb_mlp_gram computes (d0, g, H) once; every training step then needs only
// the network.  Weight vector layout: W1 (32x3), W2 (32x32), W3 (6x32), b1, b2, b3.
#include <algorithm>
#include <cstring>

#include "flb_internal.cuh"

namespace flb {

constexpr int kH = kMlpHidden, kO = kMlpOut;
constexpr int kOffW1 = 0, kOffW2 = kOffW1 + kH * 3, kOffW3 = kOffW2 + kH * kH;
constexpr int kOffB1 = kOffW3 + kO * kH, kOffB2 = kOffB1 + kH, kOffB3 = kOffB2 + kH;
constexpr int kNParams = kOffB3 + kO;                       // 1382
constexpr int kGram = 1 + kO + kO * kO;                     // d0, g[6], H[6][6]
constexpr int kInter = 3 + kH + kH + kH + kH + kO;          // X, h1, h2, dz1, dz2, do per sample
constexpr int kPairs = 6;
constexpr int kTrainBlock = 256;

// (d0, g, H) per run.  Splain: [R][P][K] complex, G: [R][C][P][K] complex (re, im).
// One block per run; fixed-order block reduction.
__global__ void k_mlp_gram(const double* __restrict__ Sp, const double* __restrict__ G, int P, int K,
                           double* __restrict__ out) {
  const int r = blockIdx.x;
  __shared__ double red[kTrainBlock];
  const int n_terms = kGram;
  for (int term = 0; term < n_terms; ++term) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < P * K; i += blockDim.x) {
      const int p = i / K;
      const double tgt = (p == 0 || p == 3 || p == 5) ? 1.0 : 0.0;
      const double* s = Sp + 2 * ((size_t)r * P * K + i);
      const double dr = s[0] - tgt, di = s[1];
      if (term == 0) {
        acc += dr * dr + di * di;
      } else if (term <= kO) {
        const int c = term - 1;
        const double* gc = G + 2 * (((size_t)r * kO + c) * P * K + i);
        acc += dr * gc[0] + di * gc[1];
      } else {
        const int c = (term - 1 - kO) / kO, c2 = (term - 1 - kO) % kO;
        const double* ga = G + 2 * (((size_t)r * kO + c) * P * K + i);
        const double* gb = G + 2 * (((size_t)r * kO + c2) * P * K + i);
        acc += ga[0] * gb[0] + ga[1] * gb[1];
      }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)r * kGram + term] = red[0];
    __syncthreads();
  }
}

struct Fwd {
  float z1[kH], h1[kH], z2[kH], h2[kH], s[kO];
};

__device__ __forceinline__ void forward(const float* __restrict__ W, const float x[3], Fwd& f) {
  for (int h = 0; h < kH; ++h) {
    float z = W[kOffB1 + h];
    for (int i = 0; i < 3; ++i) z = fmaf(W[kOffW1 + 3 * h + i], x[i], z);
    f.z1[h] = z;
    f.h1[h] = fmaxf(z, 0.f);
  }
  for (int h = 0; h < kH; ++h) {
    float z = W[kOffB2 + h];
    for (int k = 0; k < kH; ++k) z = fmaf(W[kOffW2 + kH * h + k], f.h1[k], z);
    f.z2[h] = z;
    f.h2[h] = fmaxf(z, 0.f);
  }
  for (int c = 0; c < kO; ++c) {
    float o = W[kOffB3 + c];
    for (int h = 0; h < kH; ++h) o = fmaf(W[kOffW3 + kH * c + h], f.h2[h], o);
    f.s[c] = 1.f + o;
  }
}

// Pass 1: forward of every sample, block partial sums of s_c^2 per run.
// grid = R * blocks_per_run; block b of run r covers samples [b*256, b*256+256).
__global__ void k_mlp_fwd_stats(const float* __restrict__ Wg, const float* __restrict__ X, int B,
                                int blocks_per_run, double* __restrict__ partial) {
  __shared__ float W[kNParams];
  __shared__ double red[kTrainBlock / 32][kO];
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) W[i] = Wg[i];
  __syncthreads();
  const int r = blockIdx.x / blocks_per_run, bb = blockIdx.x % blocks_per_run;
  const int b = bb * blockDim.x + threadIdx.x;
  double s2[kO] = {0, 0, 0, 0, 0, 0};
  if (b < B) {
    const float* xp = X + 3 * ((size_t)r * B + b);
    const float x[3] = {xp[0], xp[1], xp[2]};
    Fwd f;
    forward(W, x, f);
    for (int c = 0; c < kO; ++c) s2[c] = (double)f.s[c] * (double)f.s[c];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < kO; ++c) {
    double v = s2[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kO) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[w][threadIdx.x];
    partial[(size_t)blockIdx.x * kO + threadIdx.x] = v;
  }
}

// Pass 2 (one block): m_rc, the per-run loss and dL/dm_rc from the Gram terms;
// thread 0 then adds the per-run losses in order.
__global__ void k_mlp_loss(const double* __restrict__ partial, int R, int B, int blocks_per_run,
                           const double* __restrict__ gram, double norm, double* __restrict__ m_out,
                           double* __restrict__ dm, double* __restrict__ loss_r, double* __restrict__ loss) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double m[kO];
    for (int c = 0; c < kO; ++c) {
      double v = 0.0;
      for (int bb = 0; bb < blocks_per_run; ++bb) v += partial[((size_t)r * blocks_per_run + bb) * kO + c];
      m[c] = v / B;
      m_out[r * kO + c] = m[c];
    }
    const double* gm = gram + (size_t)r * kGram;
    double L = gm[0];
    for (int c = 0; c < kO; ++c) {
      double hd = 0.0;
      for (int c2 = 0; c2 < kO; ++c2) hd += gm[1 + kO + c * kO + c2] * (m[c2] - 1.0);
      L += 2.0 * gm[1 + c] * (m[c] - 1.0) + (m[c] - 1.0) * hd;
      dm[r * kO + c] = norm * (2.0 * gm[1 + c] + 2.0 * hd);
    }
    loss_r[r] = L;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double L = 0.0;
    for (int r = 0; r < R; ++r) L += loss_r[r];
    *loss = norm * L;
  }
}

// Pass 3: per-sample backward; stores the intermediates the weight gradients need.
__global__ void k_mlp_backward(const float* __restrict__ Wg, const float* __restrict__ X, int R, int B,
                               const double* __restrict__ dm, float* __restrict__ inter) {
  __shared__ float W[kNParams];
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) W[i] = Wg[i];
  __syncthreads();
  const int64_t n = (int64_t)R * B;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / B);
    const float* xp = X + 3 * i;
    const float x[3] = {xp[0], xp[1], xp[2]};
    Fwd f;
    forward(W, x, f);
    float dout[kO];
    for (int c = 0; c < kO; ++c) dout[c] = (float)(dm[r * kO + c] * 2.0 * (double)f.s[c] / (double)B);
    float dz2[kH], dz1[kH];
    for (int h = 0; h < kH; ++h) {
      float v = 0.f;
      for (int c = 0; c < kO; ++c) v = fmaf(W[kOffW3 + kH * c + h], dout[c], v);
      dz2[h] = f.z2[h] > 0.f ? v : 0.f;
    }
    for (int k = 0; k < kH; ++k) {
      float v = 0.f;
      for (int h = 0; h < kH; ++h) v = fmaf(W[kOffW2 + kH * h + k], dz2[h], v);
      dz1[k] = f.z1[k] > 0.f ? v : 0.f;
    }
    float* o = inter + i;                       // structure of arrays: [field][R*B]
    for (int j = 0; j < 3; ++j) o[(int64_t)j * n] = x[j];
    for (int h = 0; h < kH; ++h) {
      o[(int64_t)(3 + h) * n] = f.h1[h];
      o[(int64_t)(3 + kH + h) * n] = f.h2[h];
      o[(int64_t)(3 + 2 * kH + h) * n] = dz1[h];
      o[(int64_t)(3 + 3 * kH + h) * n] = dz2[h];
    }
    for (int c = 0; c < kO; ++c) o[(int64_t)(3 + 4 * kH + c) * n] = dout[c];
  }
}

// Pass 4: one block per parameter, fixed-order sum over all samples.
__global__ void k_mlp_grad_reduce(const float* __restrict__ inter, int64_t n, float* __restrict__ grad) {
  const int p = blockIdx.x;
  int ga, gb = -1;           // gradient = sum_b inter[ga][b] * inter[gb][b]  (gb < 0: plain sum)
  constexpr int X0 = 0, H1 = 3, H2 = 3 + kH, DZ1 = 3 + 2 * kH, DZ2 = 3 + 3 * kH, DO = 3 + 4 * kH;
  if (p < kOffW2) { ga = DZ1 + p / 3; gb = X0 + p % 3; }
  else if (p < kOffW3) { const int q = p - kOffW2; ga = DZ2 + q / kH; gb = H1 + q % kH; }
  else if (p < kOffB1) { const int q = p - kOffW3; ga = DO + q / kH; gb = H2 + q % kH; }
  else if (p < kOffB2) { ga = DZ1 + (p - kOffB1); }
  else if (p < kOffB3) { ga = DZ2 + (p - kOffB2); }
  else { ga = DO + (p - kOffB3); }
  __shared__ double red[kTrainBlock];
  double acc = 0.0;
  const float* A = inter + (int64_t)ga * n;
  const float* Bv = gb >= 0 ? inter + (int64_t)gb * n : nullptr;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += (double)A[i] * (Bv ? (double)Bv[i] : 1.0);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad[p] = (float)red[0];
}

// Adam (Kingma & Ba, 2015) with bias correction.
__global__ void k_adam(float* __restrict__ W, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float mi = b1 * m[i] + (1.f - b1) * g[i];
  const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  W[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static int64_t a256(int64_t x) { return (x + 255) & ~int64_t(255); }

struct TrainLayout {
  int blocks_per_run;
  int64_t off_partial, off_dm, off_lossr, off_inter, off_grad, total;
};

static TrainLayout train_layout(int R, int B) {
  TrainLayout t;
  t.blocks_per_run = (B + kTrainBlock - 1) / kTrainBlock;
  int64_t off = 0;
  t.off_partial = off; off = a256(off + 8 * (int64_t)R * t.blocks_per_run * kO);
  t.off_dm = off; off = a256(off + 8 * (int64_t)R * kO);
  t.off_lossr = off; off = a256(off + 8 * (int64_t)R);
  t.off_grad = off; off = a256(off + 4 * (int64_t)kNParams);
  t.off_inter = off; off = a256(off + 4 * (int64_t)kInter * R * B);
  t.total = off;
  return t;
}

}  // namespace flb

using namespace flb;

extern "C" {

int flb_mlp_param_count(void) { return kNParams; }

int flb_mlp_gram(const double* splain_dev, const double* g_dev, int R, int P, int K, double* gram_dev,
                 void* cuda_stream) {
  if (R < 1 || P != kPairs || K < 1) return set_error(FLB_EINVAL, "need R >= 1, P = 6 pairs, K >= 1");
  if (!splain_dev || !g_dev || !gram_dev) return set_error(FLB_EINVAL, "NULL pointer");
  k_mlp_gram<<<R, kTrainBlock, 0, static_cast<cudaStream_t>(cuda_stream)>>>(splain_dev, g_dev, P, K, gram_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FLB_OK : set_error(FLB_ECUDA, "flb_mlp_gram: %s", cudaGetErrorString(e));
}

int flb_mlp_scratch_bytes(int R, int B, size_t* bytes) {
  if (R < 1 || B < 1 || !bytes) return set_error(FLB_EINVAL, "need R, B >= 1");
  *bytes = (size_t)train_layout(R, B).total;
  return FLB_OK;
}

int flb_mlp_train_step(float* w_dev, float* adam_m_dev, float* adam_v_dev, int t, float lr, float beta1,
                       float beta2, float eps, const float* x_dev, int R, int B, const double* gram_dev,
                       int P, int K, double* loss_dev, double* m_dev, float* grad_dev, void* scratch_dev,
                       size_t scratch_bytes, void* cuda_stream) {
  if (!w_dev || !x_dev || !gram_dev || !loss_dev || !m_dev || !scratch_dev) return set_error(FLB_EINVAL, "NULL pointer");
  if (R < 1 || B < 1 || P != kPairs || K < 1) return set_error(FLB_EINVAL, "need R, B, K >= 1 and P = 6");
  if (lr > 0.f && (!adam_m_dev || !adam_v_dev || t < 1)) return set_error(FLB_EINVAL, "Adam needs m, v and t >= 1");
  const TrainLayout T = train_layout(R, B);
  if (scratch_bytes < (size_t)T.total) return set_error(FLB_ENOMEM, "scratch %zu < %lld bytes", scratch_bytes, (long long)T.total);
  if (((uintptr_t)scratch_dev) & 255) return set_error(FLB_EINVAL, "scratch must be 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  char* s = static_cast<char*>(scratch_dev);
  double* partial = reinterpret_cast<double*>(s + T.off_partial);
  double* dm = reinterpret_cast<double*>(s + T.off_dm);
  float* inter = reinterpret_cast<float*>(s + T.off_inter);
  float* grad = grad_dev ? grad_dev : reinterpret_cast<float*>(s + T.off_grad);
  const double norm = 1.0 / ((double)R * P * K);
  k_mlp_fwd_stats<<<R * T.blocks_per_run, kTrainBlock, 0, st>>>(w_dev, x_dev, B, T.blocks_per_run, partial);
  k_mlp_loss<<<1, 64, 0, st>>>(partial, R, B, T.blocks_per_run, gram_dev, norm, m_dev, dm,
                               reinterpret_cast<double*>(s + T.off_lossr), loss_dev);
  const int64_t n = (int64_t)R * B;
  const int bgrid = (int)std::min<int64_t>((n + kTrainBlock - 1) / kTrainBlock, 4096);
  k_mlp_backward<<<bgrid, kTrainBlock, 0, st>>>(w_dev, x_dev, R, B, dm, inter);
  k_mlp_grad_reduce<<<kNParams, kTrainBlock, 0, st>>>(inter, n, grad);
  if (lr > 0.f) {
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam<<<(kNParams + 255) / 256, 256, 0, st>>>(w_dev, grad, adam_m_dev, adam_v_dev, kNParams, lr, beta1, beta2,
                                                    eps, c1, c2);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FLB_OK : set_error(FLB_ECUDA, "flb_mlp_train_step: %s", cudaGetErrorString(e));
}

}  // extern "C"
