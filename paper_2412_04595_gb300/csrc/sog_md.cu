// Repeated evaluation for molecular dynamics (sog_md_* in sog.h): velocity
// Verlet with the plan's forces.  The SOG split of Sec. 2.2 is built C^1 at
// the cutoff (Eq. 2.23, 2.24), so the forces are continuous in the pair
// distance, and the evaluation's forces are the gradient of its energy (the
// gridding is the transpose of the gathering), which is what an energy
// conserving integrator needs.
//
// Every step reuses the plan (tables, workspaces, the captured evaluation
// graph).  Every `sort_every` steps the particle arrays are permuted into the
// near-field cell order of the last evaluation, so that the next steps' bin
// counting sorts run on nearly sorted input (few distinct bins per warp, near
// contiguous scatters): the re-binning starts from the previous sort.
#include <cuda_runtime.h>

#include <new>

#include "sog_internal.h"

struct sog_md {
  sog_plan* plan = nullptr;
  void* scratch = nullptr;  // N x 3 elements of the plan's type: the array being permuted
  int64_t steps = 0;
};

namespace {

constexpr int kMdThreads = 256;

// v += h F / m (inv_mass NULL: unit masses); then, with dt != 0, r += dt v,
// x and y wrapped into [-L/2, L/2) by one period, z reflected at the walls
// z = +-Lz/2 (v_z reversed).
template <typename T>
__global__ void k_md_kick_drift(int N, T h, T dt, const T* __restrict__ F,
                                const T* __restrict__ inv_mass, T* __restrict__ v,
                                T* __restrict__ r, T Lx, T Ly, T hz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T im = inv_mass ? inv_mass[i] : T(1);
  T vx = v[3 * i] + h * F[3 * i] * im;
  T vy = v[3 * i + 1] + h * F[3 * i + 1] * im;
  T vz = v[3 * i + 2] + h * F[3 * i + 2] * im;
  if (dt != T(0)) {
    T x = r[3 * i] + dt * vx, y = r[3 * i + 1] + dt * vy, z = r[3 * i + 2] + dt * vz;
    if (x >= T(0.5) * Lx) x -= Lx;
    else if (x < T(-0.5) * Lx) x += Lx;
    if (y >= T(0.5) * Ly) y -= Ly;
    else if (y < T(-0.5) * Ly) y += Ly;
    if (z > hz) {
      z = T(2) * hz - z;
      vz = -vz;
    } else if (z < -hz) {
      z = T(-2) * hz - z;
      vz = -vz;
    }
    r[3 * i] = x;
    r[3 * i + 1] = y;
    r[3 * i + 2] = z;
  }
  v[3 * i] = vx;
  v[3 * i + 1] = vy;
  v[3 * i + 2] = vz;
}

// dst[pos * w + k] = src[perm[pos] * w + k]: gather into the sorted order.
template <typename T>
__global__ void k_md_gather(int N, int w, const int* __restrict__ perm, const T* __restrict__ src,
                            T* __restrict__ dst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * w) return;
  const int pos = t / w, k = t - pos * w;
  dst[t] = src[(size_t)perm[pos] * w + k];
}

template <typename T>
cudaError_t permute(sog_md* md, T* a, int w, cudaStream_t s) {
  if (!a) return cudaSuccess;
  const int N = (int)md->plan->N;
  cudaError_t e = cudaMemcpyAsync(md->scratch, a, (size_t)N * w * sizeof(T),
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  const int n = N * w;
  k_md_gather<T><<<(n + kMdThreads - 1) / kMdThreads, kMdThreads, 0, s>>>(
      N, w, md->plan->d_perm, static_cast<const T*>(md->scratch), a);
  return cudaGetLastError();
}

template <typename T>
sog_status md_steps(sog_md* md, void* q, void* r, void* v, void* F, void* inv_mass, double dt,
                    int nsteps, int sort_every, double* E, int32_t* order, cudaStream_t s) {
  sog_plan* p = md->plan;
  const int N = (int)p->N;
  const int blocks = (N + kMdThreads - 1) / kMdThreads;
  const T h = (T)(0.5 * dt), d = (T)dt;
  const T Lx = (T)p->prm.L[0], Ly = (T)p->prm.L[1], hz = (T)(0.5 * p->prm.L[2]);
  for (int k = 0; k < nsteps; ++k) {
    k_md_kick_drift<T><<<blocks, kMdThreads, 0, s>>>(N, h, d, static_cast<const T*>(F),
                                                     static_cast<const T*>(inv_mass),
                                                     static_cast<T*>(v), static_cast<T*>(r), Lx,
                                                     Ly, hz);
    if (cudaGetLastError() != cudaSuccess) return SOG_ERR_CUDA;
    const sog_status st = sogk::eval_device(p, q, r, nullptr, E, F, nullptr, nullptr, s);
    if (st != SOG_OK) return st;
    k_md_kick_drift<T><<<blocks, kMdThreads, 0, s>>>(N, h, T(0), static_cast<const T*>(F),
                                                     static_cast<const T*>(inv_mass),
                                                     static_cast<T*>(v), static_cast<T*>(r), Lx,
                                                     Ly, hz);
    if (cudaGetLastError() != cudaSuccess) return SOG_ERR_CUDA;
    ++md->steps;
    if (sort_every > 0 && md->steps % sort_every == 0) {
      // the last evaluation's near-field cell order: perm[pos] = index
      if (permute<T>(md, static_cast<T*>(q), 1, s) != cudaSuccess ||
          permute<T>(md, static_cast<T*>(r), 3, s) != cudaSuccess ||
          permute<T>(md, static_cast<T*>(v), 3, s) != cudaSuccess ||
          permute<T>(md, static_cast<T*>(F), 3, s) != cudaSuccess ||
          permute<T>(md, static_cast<T*>(inv_mass), 1, s) != cudaSuccess ||
          permute<int32_t>(md, order, 1, s) != cudaSuccess)
        return SOG_ERR_CUDA;
    }
  }
  p->last_stream = s;
  return SOG_OK;
}

}  // namespace

extern "C" {

sog_status sog_md_create(sog_md** md, sog_plan* plan) {
  if (!md || !plan) return SOG_ERR_ARG;
  *md = nullptr;
  sog_md* m = new (std::nothrow) sog_md();
  if (!m) return SOG_ERR_NOMEM;
  m->plan = plan;
  const size_t es = plan->prec == SOG_PREC_FP64 ? sizeof(double) : sizeof(float);
  if (cudaMalloc(&m->scratch, (size_t)plan->N * 3 * es) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return SOG_ERR_NOMEM;
  }
  *md = m;
  return SOG_OK;
}

sog_status sog_md_step(sog_md* md, void* q, void* r, void* v, void* F, void* inv_mass,
                       double dt, int32_t nsteps, int32_t sort_every, double* E, int32_t* order,
                       void* stream) {
  if (!md || !q || !r || !v || !F || nsteps < 0 || sort_every < 0 || !(dt == dt)) return SOG_ERR_ARG;
  if (sort_every > 0 && !order) return SOG_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (md->plan->prec == SOG_PREC_FP64)
    return md_steps<double>(md, q, r, v, F, inv_mass, dt, nsteps, sort_every, E, order, s);
  return md_steps<float>(md, q, r, v, F, inv_mass, dt, nsteps, sort_every, E, order, s);
}

void sog_md_destroy(sog_md* md) {
  if (!md) return;
  cudaStreamSynchronize(md->plan->last_stream);
  cudaFree(md->scratch);
  delete md;
}

}  // extern "C"
