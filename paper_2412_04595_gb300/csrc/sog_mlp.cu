// Small multilayer perceptron that proposes the near-field neighbour count
// (hence r_c and the rest of the split) from features of a system, with its
// own forward, backward and Adam kernels (sog_mlp_* and sog_features in
// sog.h).  The paper selects parameters analytically (Sec. 4.3); that
// selection stays the fallback and decides feasibility.
//
// Network: x (n_in) -> tanh(W1 x + b1) (H) -> tanh(W2 h1 + b2) (H) ->
// y = w3 . h2 + b3.  Parameters in one FP32 array:
//   W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1].
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/sog.h"

struct sog_mlp {
  int n_in = 0, H = 0;
  int64_t np = 0;
  float* d_p = nullptr;  // parameters
  float* d_g = nullptr;  // gradient
  float* d_m = nullptr;  // Adam moments
  float* d_v = nullptr;
  float* d_loss = nullptr;
  int64_t step = 0;
};

namespace {

constexpr int kMaxIn = 16, kMaxH = 64, kMlpThreads = 128;

__host__ __device__ inline int64_t n_params(int n_in, int H) {
  return (int64_t)H * n_in + H + (int64_t)H * H + H + H + 1;
}

// Forward pass of one sample; returns y and keeps the activations.
__device__ __forceinline__ float mlp_forward(const float* __restrict__ p, int n_in, int H,
                                             const float* x, float* h1, float* h2) {
  const float* W1 = p;
  const float* b1 = W1 + H * n_in;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const float b3 = w3[H];
  for (int j = 0; j < H; ++j) {
    float a = b1[j];
    for (int i = 0; i < n_in; ++i) a += W1[j * n_in + i] * x[i];
    h1[j] = tanhf(a);
  }
  float y = b3;
  for (int j = 0; j < H; ++j) {
    float a = b2[j];
    for (int i = 0; i < H; ++i) a += W2[j * H + i] * h1[i];
    h2[j] = tanhf(a);
    y += w3[j] * h2[j];
  }
  return y;
}

__global__ void k_mlp_forward(const float* __restrict__ p, int n_in, int H, int64_t np,
                              const float* __restrict__ X, int n, float* __restrict__ Y) {
  extern __shared__ float sp[];
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) sp[i] = p[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[kMaxIn], h1[kMaxH], h2[kMaxH];
  for (int i = 0; i < n_in; ++i) x[i] = X[(size_t)s * n_in + i];
  Y[s] = mlp_forward(sp, n_in, H, x, h1, h2);
}

// Mean squared error (1/n) sum (y - t)^2 and its gradient: each thread
// back-propagates one sample into a block-shared gradient, blocks add theirs
// to the global one.  grad and loss must be zero on entry.
__global__ void k_mlp_loss_grad(const float* __restrict__ p, int n_in, int H, int64_t np,
                                const float* __restrict__ X, const float* __restrict__ T, int n,
                                float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* sp = sm;
  float* sg = sm + np;
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) {
    sp[i] = p[i];
    sg[i] = 0.f;
  }
  __shared__ float sl;
  if (threadIdx.x == 0) sl = 0.f;
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    float x[kMaxIn], h1[kMaxH], h2[kMaxH], d2[kMaxH];
    for (int i = 0; i < n_in; ++i) x[i] = X[(size_t)s * n_in + i];
    const float y = mlp_forward(sp, n_in, H, x, h1, h2);
    const float r = y - T[s];
    atomicAdd(&sl, r * r / n);
    const float dy = 2.f * r / n;
    float* gW1 = sg;
    float* gb1 = gW1 + H * n_in;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gw3 = gb2 + H;
    const float* W2 = sp + H * n_in + H;
    const float* w3 = W2 + H * H + H;
    atomicAdd(&gw3[H], dy);  // b3
    for (int j = 0; j < H; ++j) {
      atomicAdd(&gw3[j], dy * h2[j]);
      d2[j] = dy * w3[j] * (1.f - h2[j] * h2[j]);
      atomicAdd(&gb2[j], d2[j]);
      for (int i = 0; i < H; ++i) atomicAdd(&gW2[j * H + i], d2[j] * h1[i]);
    }
    for (int i = 0; i < H; ++i) {
      float a = 0.f;
      for (int j = 0; j < H; ++j) a += W2[j * H + i] * d2[j];
      const float d1 = a * (1.f - h1[i] * h1[i]);
      atomicAdd(&gb1[i], d1);
      for (int k = 0; k < n_in; ++k) atomicAdd(&gW1[i * n_in + k], d1 * x[k]);
    }
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x)
    if (sg[i] != 0.f) atomicAdd(&grad[i], sg[i]);
  if (threadIdx.x == 0) atomicAdd(loss, sl);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t np, float lr, float b1c, float b2c) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float b1 = 0.9f, b2 = 0.999f;
  const float mi = b1 * m[i] + (1.f - b1) * g[i];
  const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
}

// Uniform init in +-sqrt(6/(fan_in + fan_out)) (Glorot) from a 64-bit LCG.
void init_params(std::vector<float>& p, int n_in, int H, uint64_t seed) {
  uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(st >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  };
  size_t k = 0;
  const double a1 = sqrt(6.0 / (n_in + H)), a2 = sqrt(6.0 / (2.0 * H)), a3 = sqrt(6.0 / (H + 1));
  for (int i = 0; i < H * n_in; ++i) p[k++] = (float)(a1 * uni());
  for (int i = 0; i < H; ++i) p[k++] = 0.f;
  for (int i = 0; i < H * H; ++i) p[k++] = (float)(a2 * uni());
  for (int i = 0; i < H; ++i) p[k++] = 0.f;
  for (int i = 0; i < H; ++i) p[k++] = (float)(a3 * uni());
  p[k++] = 0.f;
}

size_t smem_params(const sog_mlp* m) { return (size_t)m->np * sizeof(float); }

// z histogram of the particles: 16 bins over [-Lz/2, Lz/2].
template <typename T>
__global__ void k_zhist(const T* __restrict__ r, int64_t N, double Lz, unsigned* __restrict__ hist) {
  __shared__ unsigned sh[16];
  if (threadIdx.x < 16) sh[threadIdx.x] = 0;
  __syncthreads();
  const double inv = 16.0 / Lz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int b = (int)floor(((double)r[3 * i + 2] + 0.5 * Lz) * inv);
    b = b < 0 ? 0 : (b > 15 ? 15 : b);
    atomicAdd(&sh[b], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 16) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

}  // namespace

extern "C" {

sog_status sog_mlp_create(sog_mlp** out, int32_t n_in, int32_t n_hidden, uint64_t seed) {
  if (!out || n_in < 1 || n_in > kMaxIn || n_hidden < 1 || n_hidden > kMaxH) return SOG_ERR_ARG;
  *out = nullptr;
  sog_mlp* m = new sog_mlp;
  m->n_in = n_in;
  m->H = n_hidden;
  m->np = n_params(n_in, n_hidden);
  std::vector<float> p((size_t)m->np);
  init_params(p, n_in, n_hidden, seed);
  const size_t b = (size_t)m->np * sizeof(float);
  if (cudaMalloc(&m->d_p, 4 * b + 256) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return SOG_ERR_NOMEM;
  }
  m->d_g = m->d_p + m->np;
  m->d_m = m->d_g + m->np;
  m->d_v = m->d_m + m->np;
  m->d_loss = m->d_v + m->np;
  if (cudaMemcpy(m->d_p, p.data(), b, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->d_m, 0, 2 * b) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(m->d_p);
    delete m;
    return SOG_ERR_CUDA;
  }
  *out = m;
  return SOG_OK;
}

int64_t sog_mlp_num_params(const sog_mlp* m) { return m ? m->np : 0; }

sog_status sog_mlp_get_params(const sog_mlp* m, float* host, int64_t n) {
  if (!m || !host || n != m->np) return SOG_ERR_ARG;
  return cudaMemcpy(host, m->d_p, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
             ? SOG_OK
             : SOG_ERR_CUDA;
}

sog_status sog_mlp_set_params(sog_mlp* m, const float* host, int64_t n) {
  if (!m || !host || n != m->np) return SOG_ERR_ARG;
  if (cudaMemcpy(m->d_p, host, (size_t)n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return SOG_ERR_CUDA;
  m->step = 0;
  return cudaMemset(m->d_m, 0, 2 * (size_t)n * sizeof(float)) == cudaSuccess ? SOG_OK
                                                                              : SOG_ERR_CUDA;
}

sog_status sog_mlp_forward(const sog_mlp* m, const float* X, int32_t n, float* Y, void* stream) {
  if (!m || !X || !Y || n < 1) return SOG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_mlp_forward<<<(n + kMlpThreads - 1) / kMlpThreads, kMlpThreads, smem_params(m), s>>>(
      m->d_p, m->n_in, m->H, m->np, X, n, Y);
  return cudaGetLastError() == cudaSuccess ? SOG_OK : SOG_ERR_CUDA;
}

sog_status sog_mlp_loss_grad(const sog_mlp* m, const float* X, const float* T, int32_t n,
                             float* grad, float* loss, void* stream) {
  if (!m || !X || !T || !grad || !loss || n < 1) return SOG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(grad, 0, (size_t)m->np * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess)
    return SOG_ERR_CUDA;
  k_mlp_loss_grad<<<(n + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 2 * smem_params(m), s>>>(
      m->d_p, m->n_in, m->H, m->np, X, T, n, grad, loss);
  return cudaGetLastError() == cudaSuccess ? SOG_OK : SOG_ERR_CUDA;
}

sog_status sog_mlp_train(sog_mlp* m, const float* X, const float* T, int32_t n, int32_t iters,
                         float lr, float* loss_out, void* stream) {
  if (!m || !X || !T || n < 1 || iters < 0 || !(lr > 0.f)) return SOG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int tb = 256;
  const int gb = (int)((m->np + tb - 1) / tb);
  for (int it = 0; it < iters; ++it) {
    const sog_status st = sog_mlp_loss_grad(m, X, T, n, m->d_g, m->d_loss, stream);
    if (st != SOG_OK) return st;
    ++m->step;
    const float b1c = 1.f - powf(0.9f, (float)m->step), b2c = 1.f - powf(0.999f, (float)m->step);
    k_adam<<<gb, tb, 0, s>>>(m->d_p, m->d_g, m->d_m, m->d_v, m->np, lr, b1c, b2c);
    if (cudaGetLastError() != cudaSuccess) return SOG_ERR_CUDA;
  }
  if (loss_out) {
    if (iters == 0) {
      const sog_status st = sog_mlp_loss_grad(m, X, T, n, m->d_g, m->d_loss, stream);
      if (st != SOG_OK) return st;
    }
    if (cudaMemcpyAsync(loss_out, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SOG_ERR_CUDA;
  }
  return SOG_OK;
}

void sog_mlp_destroy(sog_mlp* m) {
  if (!m) return;
  cudaFree(m->d_p);
  delete m;
}

sog_status sog_features(int64_t N, double Lx, double Ly, double Lz, double tol, const void* r,
                        int32_t precision, float* feat) {
  if (N < 2 || !(Lx > 0) || !(Ly > 0) || !(Lz > 0) || !(tol > 0) || !r || !feat ||
      (precision != SOG_PREC_FP64 && precision != SOG_PREC_MIXED))
    return SOG_ERR_ARG;
  unsigned* d_hist = nullptr;
  if (cudaMalloc(&d_hist, 16 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return SOG_ERR_NOMEM;
  }
  cudaMemset(d_hist, 0, 16 * sizeof(unsigned));
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  const int blocks = (int)std::min<int64_t>(2 * (int64_t)sms, (N + 255) / 256);
  if (precision == SOG_PREC_FP64)
    k_zhist<double><<<blocks, 256>>>(static_cast<const double*>(r), N, Lz, d_hist);
  else
    k_zhist<float><<<blocks, 256>>>(static_cast<const float*>(r), N, Lz, d_hist);
  unsigned h[16];
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpy(h, d_hist, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d_hist);
  if (!ok) return SOG_ERR_CUDA;
  const double mean = (double)N / 16.0;
  double mx = 0.0, var = 0.0;
  for (int b = 0; b < 16; ++b) {
    mx = std::max(mx, (double)h[b]);
    var += ((double)h[b] - mean) * ((double)h[b] - mean) / 16.0;
  }
  const double rho = (double)N / (Lx * Ly * Lz);
  feat[0] = (float)log10((double)N);
  feat[1] = (float)log10(sqrt(Lx * Ly));
  feat[2] = (float)log10(Lz / sqrt(Lx * Ly));
  feat[3] = (float)log10(tol);
  feat[4] = (float)log10(rho);
  feat[5] = (float)(mx / mean);
  feat[6] = (float)(((double)h[0] + (double)h[15]) / (2.0 * mean));
  feat[7] = (float)(sqrt(var) / mean);
  return SOG_OK;
}

}  // extern "C"
