// Plan-free, allocation-free assembly of the potential, forces and energy
// from the four parts of the potential (sog_assemble_noalloc in sog.h).
//
// The energy reduction needs per-block partial sums.  They live in a
// file-scope device array of fixed size instead of plan memory or a
// temporary allocation, so that the call performs no cudaMalloc, cudaFree or
// allocating library call.  Its device address is looked up once per device
// (cudaGetSymbolAddress, with that device current) on the first call.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "sog_internal.h"

namespace {

// Partial sums of q_i Phi_i: one per block, at most 1024 blocks (two per SM
// of the device, capped); 1024 doubles = 8 KB.  The grid-stride loop lets any
// N use them.
constexpr int kNoAllocBlocks = 1024;
constexpr int kNoAllocThreads = 256;
// Element indices are 32-bit in the kernel (3 i + d < 2^31).
constexpr int64_t kNoAllocMaxN = 715827882;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_energy_partials[kNoAllocBlocks];

std::mutex g_setup_mu;
double* g_partials_ptr[kMaxDevices] = {};
int g_blocks[kMaxDevices] = {};

__device__ __forceinline__ double warp_add(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Phi_i = sum of the four parts - q_i sum_l w_l (self term), F_i = -q_i grad
// Phi, and one partial sum of q_i Phi_i per block written to part[blockIdx.x]
// (every block writes its slot, so nothing needs to start at zero).  A
// non-finite charge counts as 0, as in the plans' own assembly; the plan whose
// sog_eval_components produced the parts reports it through sog_plan_check.
template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads)
    k_assemble_noalloc(const T* __restrict__ q, int N, const double* __restrict__ pp,
                       const double* __restrict__ pg, double selfsum, T* __restrict__ phi,
                       T* __restrict__ F, double* __restrict__ part) {
  __shared__ double sh[kNoAllocThreads / 32];
  double e = 0.0;
  const size_t n = (size_t)N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double qi = (double)q[i];
    if (!isfinite(qi)) qi = 0.0;
    const double ph = pp[i] + pp[n + i] + pp[2 * n + i] + pp[3 * n + i] - qi * selfsum;
    if (phi) phi[i] = (T)ph;
    if (F)
      for (int d = 0; d < 3; ++d) {
        const double g = pg[3 * i + d] + pg[3 * (n + i) + d] + pg[3 * (2 * n + i) + d] +
                         pg[3 * (3 * n + i) + d];
        F[3 * i + d] = (T)(-qi * g);
      }
    e += qi * ph;
  }
  e = warp_add(e);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// U = 1/2 sum of the partials, in a fixed order (one warp).
__global__ void k_energy_noalloc(const double* __restrict__ part, int nblk, double* __restrict__ E) {
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[b];
  s = warp_add(s);
  if (lane == 0) *E = 0.5 * s;
}

// Device address of g_energy_partials on the current device and the block
// count of the assembly there (two per SM, at most kNoAllocBlocks), looked
// up once per device.
sog_status partials_ptr(double** out, int* max_blocks) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SOG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SOG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_energy_partials) != cudaSuccess || !p) return SOG_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
      return SOG_ERR_CUDA;
    g_blocks[dev] = 2 * sms < kNoAllocBlocks ? 2 * sms : kNoAllocBlocks;
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  *max_blocks = g_blocks[dev];
  return SOG_OK;
}

// sum_l w_l of Eq. (2.22) with w_0 scaled by omega (Eq. 2.25): the
// coefficient of the self term, term by term from the weights the plans'
// tables use (no host or device allocation).
double self_coefficient(const sog_params& prm) {
  double s = 0.0;
  for (int l = 0; l <= prm.M; ++l) s += sogk::sog_weight(prm.b, prm.sigma, prm.omega, l);
  return s;
}

template <typename T>
sog_status launch(int N, const void* q, const double* pp, const double* pg, double selfsum,
                  void* phi, double* E, void* F, cudaStream_t s) {
  double* part = nullptr;
  int max_blocks = 0;
  const sog_status st = partials_ptr(&part, &max_blocks);
  if (st != SOG_OK) return st;
  int blocks = (N + kNoAllocThreads - 1) / kNoAllocThreads;
  if (blocks > max_blocks) blocks = max_blocks;
  k_assemble_noalloc<T><<<blocks, kNoAllocThreads, 0, s>>>(
      static_cast<const T*>(q), N, pp, pg, selfsum, static_cast<T*>(phi), static_cast<T*>(F), part);
  if (cudaGetLastError() != cudaSuccess) return SOG_ERR_CUDA;
  if (E) {
    k_energy_noalloc<<<1, 32, 0, s>>>(part, blocks, E);
    if (cudaGetLastError() != cudaSuccess) return SOG_ERR_CUDA;
  }
  return SOG_OK;
}

}  // namespace

extern "C" sog_status sog_assemble_noalloc(int64_t N, int32_t precision, const sog_params* prm,
                                           const void* q, const double* phi_parts,
                                           const double* grad_parts, void* phi, double* E,
                                           void* F, void* stream) {
  if (!prm || !q || !phi_parts) return SOG_ERR_ARG;
  if (N < 1 || N > kNoAllocMaxN) return SOG_ERR_ARG;
  if (precision != SOG_PREC_FP64 && precision != SOG_PREC_MIXED) return SOG_ERR_ARG;
  if (F && !grad_parts) return SOG_ERR_ARG;
  if (!(prm->b > 1.0) || !(prm->sigma > 0.0) || !(prm->omega > 0.0) || prm->M < 0 ||
      prm->M > 4000 || !isfinite(prm->b) || !isfinite(prm->sigma) || !isfinite(prm->omega))
    return SOG_ERR_ARG;
  const double selfsum = self_coefficient(*prm);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == SOG_PREC_FP64)
    return launch<double>((int)N, q, phi_parts, grad_parts, selfsum, phi, E, F, s);
  return launch<float>((int)N, q, phi_parts, grad_parts, selfsum, phi, E, F, s);
}
