// Batched mixed-radix FFTs of the spectral SOG solvers, in shared memory.
//
// Algorithm 1 needs a forward 3D FFT, the scaling of Eq. (3.8) and a
// backward 3D FFT on the real grid; Algorithm 2 needs forward and backward 2D
// FFTs of every Chebyshev proxy plane with a z-contraction in between.  Both
// are done as passes over lines:
//   x pass:  real rows, two rows packed into one complex line (R2C / C2R),
//            half spectrum written in place (row pitch Ix + 2 reals);
//   y pass:  complex lines along y;
//   z pass:  forward FFT along z, multiplication by the precomputed scaling
//            factor, backward FFT along z, in one kernel (Algorithm 1 steps
//            2-4 for the z direction without a round trip through memory).
// Each CTA holds a batch of lines in shared memory and runs self-sorting
// Stockham stages of radix 2, 3, 4, 5, 7 or 8.  Transforms are unnormalised;
// the 1/n factors live in the scaling tables.
#include "sog_internal.h"

namespace sogk {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) { return T2{a.x + b.x, a.y + b.y}; }
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) { return T2{a.x - b.x, a.y - b.y}; }
template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  return T2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by -i (forward) or +i (inverse)
template <typename T2>
__device__ __forceinline__ T2 rot(T2 a, bool inv) {
  return inv ? T2{-a.y, a.x} : T2{a.y, -a.x};
}

// One Stockham stage of radix R on nl lines of length n stored with line
// stride ls in a (input) and b (output).  L = product of earlier radices.
template <typename T2, int R>
__device__ void stage(const T2* __restrict__ a, T2* __restrict__ b, int n, int L, int nl,
                      int ls, const T2* __restrict__ tw, bool inv) {
  const int nb = n / R;
  const int m = nb / L;
  const int tot = nl * nb;
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int line = idx / nb;
    const int t = idx - line * nb;
    const int j = t % L;
    const int k = t / L;
    const T2* al = a + line * ls;
    T2* bl = b + line * ls;
    T2 x[R];
#pragma unroll
    for (int p = 0; p < R; ++p) x[p] = al[(k + m * p) * L + j];
#pragma unroll
    for (int p = 1; p < R; ++p) {
      T2 w = tw[j * p * m];
      if (inv) w.y = -w.y;
      x[p] = cmul(x[p], w);
    }
    T2 y[R];
    if (R == 2) {
      y[0] = cadd(x[0], x[1]);
      y[1] = csub(x[0], x[1]);
    } else if (R == 4) {
      const T2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
      const T2 s13 = cadd(x[1], x[3]), d13 = rot(csub(x[1], x[3]), inv);
      y[0] = cadd(s02, s13);
      y[2] = csub(s02, s13);
      y[1] = cadd(d02, d13);
      y[3] = csub(d02, d13);
    } else {
      const int step = n / R;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        T2 s = x[0];
#pragma unroll
        for (int p = 1; p < R; ++p) {
          T2 w = tw[((q * p) % R) * step];
          if (inv) w.y = -w.y;
          s = cadd(s, cmul(x[p], w));
        }
        y[q] = s;
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) bl[k * L * R + j + L * q] = y[q];
  }
}

// Runs all stages; returns the buffer holding the result (a or b).
template <typename T2>
__device__ T2* run_fft(T2* a, T2* b, const FftLen& f, int nl, int ls, const T2* tw, bool inv) {
  int L = 1;
  for (int s = 0; s < f.nst; ++s) {
    const int R = f.radix[s];
    switch (R) {
      case 2: stage<T2, 2>(a, b, f.n, L, nl, ls, tw, inv); break;
      case 3: stage<T2, 3>(a, b, f.n, L, nl, ls, tw, inv); break;
      case 4: stage<T2, 4>(a, b, f.n, L, nl, ls, tw, inv); break;
      case 5: stage<T2, 5>(a, b, f.n, L, nl, ls, tw, inv); break;
      case 7: stage<T2, 7>(a, b, f.n, L, nl, ls, tw, inv); break;
      default: stage<T2, 8>(a, b, f.n, L, nl, ls, tw, inv); break;
    }
    __syncthreads();
    T2* t = a;
    a = b;
    b = t;
    L *= R;
  }
  return a;
}

// x pass.  Rows r = 0..nrows-1 (nrows even) of n reals with pitch n + 2;
// rows 2p and 2p+1 travel as one complex line.  Forward: real rows in,
// half spectra (n/2 + 1 complex) out, in place.  Inverse: the reverse.
template <typename T>
__global__ void k_fft_x(T* __restrict__ data, FftLen f, const typename C2<T>::t* __restrict__ twg,
                        int npairs, int B, bool inv) {
  using T2 = typename C2<T>::t;
  extern __shared__ unsigned char smraw[];
  const int n = f.n;
  const int ls = n + 1;
  T2* a = reinterpret_cast<T2*>(smraw);
  T2* b = a + B * ls;
  const int p0 = blockIdx.x * B;
  const int nl = min(B, npairs - p0);
  const int pitch = n + 2;
  const T2* tw = twg + f.tw_off;
  if (!inv) {
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
      const int l = idx / n, t = idx - l * n;
      const T* r0 = data + (size_t)(2 * (p0 + l)) * pitch;
      a[l * ls + t] = T2{r0[t], r0[pitch + t]};
    }
  } else {
    const int nh = n / 2;
    for (int idx = threadIdx.x; idx < nl * (nh + 1); idx += blockDim.x) {
      const int l = idx / (nh + 1), fq = idx - l * (nh + 1);
      const T2* ra = reinterpret_cast<const T2*>(data + (size_t)(2 * (p0 + l)) * pitch);
      const T2* rb = reinterpret_cast<const T2*>(data + (size_t)(2 * (p0 + l) + 1) * pitch);
      const T2 A = ra[fq], Bv = rb[fq];
      a[l * ls + fq] = T2{A.x - Bv.y, A.y + Bv.x};
      if (fq > 0 && fq < nh) a[l * ls + n - fq] = T2{A.x + Bv.y, Bv.x - A.y};
    }
  }
  __syncthreads();
  T2* res = run_fft<T2>(a, b, f, nl, ls, tw, inv);
  if (!inv) {
    const int nh = n / 2;
    for (int idx = threadIdx.x; idx < nl * (nh + 1); idx += blockDim.x) {
      const int l = idx / (nh + 1), fq = idx - l * (nh + 1);
      const T2 Z = res[l * ls + fq];
      const T2 Zc = res[l * ls + (fq == 0 ? 0 : n - fq)];
      const T h = T(0.5);
      T2* ra = reinterpret_cast<T2*>(data + (size_t)(2 * (p0 + l)) * pitch);
      T2* rb = reinterpret_cast<T2*>(data + (size_t)(2 * (p0 + l) + 1) * pitch);
      ra[fq] = T2{h * (Z.x + Zc.x), h * (Z.y - Zc.y)};
      rb[fq] = T2{h * (Z.y + Zc.y), h * (Zc.x - Z.x)};
    }
  } else {
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
      const int l = idx / n, t = idx - l * n;
      T* r0 = data + (size_t)(2 * (p0 + l)) * pitch;
      const T2 z = res[l * ls + t];
      r0[t] = z.x;
      r0[pitch + t] = z.y;
    }
  }
}

// Complex line pass.  Line (o, c), o < O, c < C: element i at
// o*os + c + i*es (complex units).  A CTA takes B consecutive c of one o.
// With mult != nullptr (z pass of Algorithm 1): forward FFT, multiply element
// (o, c, i) by mult[(i*O + o)*C + c], backward FFT.
template <typename T>
__global__ void k_fft_lines(typename C2<T>::t* __restrict__ data, FftLen f,
                            const typename C2<T>::t* __restrict__ twg, int C, int O, long os,
                            long es, int B, bool inv, const T* __restrict__ mult) {
  using T2 = typename C2<T>::t;
  extern __shared__ unsigned char smraw[];
  const int n = f.n;
  const int ls = n + 1;
  T2* a = reinterpret_cast<T2*>(smraw);
  T2* b = a + B * ls;
  const int gpo = (C + B - 1) / B;
  const int o = blockIdx.x / gpo;
  const int c0 = (blockIdx.x - o * gpo) * B;
  const int nl = min(B, C - c0);
  const T2* tw = twg + f.tw_off;
  T2* base = data + (size_t)o * os + c0;
  for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
    const int i = idx / nl, c = idx - i * nl;
    a[c * ls + i] = base[(size_t)i * es + c];
  }
  __syncthreads();
  T2* res = run_fft<T2>(a, b, f, nl, ls, tw, mult ? false : inv);
  if (mult) {
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
      const int i = idx / nl, c = idx - i * nl;
      const T s = mult[((size_t)i * O + o) * C + c0 + c];
      T2 v = res[c * ls + i];
      res[c * ls + i] = T2{v.x * s, v.y * s};
    }
    __syncthreads();
    T2* other = (res == a) ? b : a;
    res = run_fft<T2>(res, other, f, nl, ls, tw, true);
  }
  for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
    const int i = idx / nl, c = idx - i * nl;
    base[(size_t)i * es + c] = res[c * ls + i];
  }
}

static int lines_per_cta(int n, size_t elem, int maxB) {
  const size_t budget = 96 * 1024;
  int B = (int)(budget / (2 * (size_t)(n + 1) * elem));
  if (B > maxB) B = maxB;
  if (B < 1) B = 1;
  return B;
}

template <typename T>
static cudaError_t launch_x(T* data, const FftLen& f, const void* tw, int nrows, bool inv,
                            cudaStream_t s) {
  using T2 = typename C2<T>::t;
  const int npairs = nrows / 2;
  const int B = lines_per_cta(f.n, sizeof(T2), 8);
  const size_t sm = 2 * (size_t)B * (f.n + 1) * sizeof(T2);
  const int grid = (npairs + B - 1) / B;
  k_fft_x<T><<<grid, 256, sm, s>>>(data, f, reinterpret_cast<const T2*>(tw), npairs, B, inv);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_lines(T* data, const FftLen& f, const void* tw, int C, int O, long os,
                                long es, bool inv, const T* mult, cudaStream_t s) {
  using T2 = typename C2<T>::t;
  const int B = lines_per_cta(f.n, sizeof(T2), 16);
  const size_t sm = 2 * (size_t)B * (f.n + 1) * sizeof(T2);
  const int grid = O * ((C + B - 1) / B);
  k_fft_lines<T><<<grid, 256, sm, s>>>(reinterpret_cast<T2*>(data), f,
                                       reinterpret_cast<const T2*>(tw), C, O, os, es, B, inv,
                                       mult);
  return cudaGetLastError();
}

// Algorithm 1 steps 2-4 on the mid grid (layout [z][y][x], pitch Ix + 2).
template <typename T>
cudaError_t fft_mid_forward_conv_inverse(const sog_plan* p, cudaStream_t s) {
  T* g = reinterpret_cast<T*>(p->d_grid);
  const int Ix = p->prm.I[0], Iy = p->prm.I[1], Iz = p->prm.I[2];
  const int C = Ix / 2 + 1;
  cudaError_t e;
  if ((e = launch_x<T>(g, p->fx, p->d_tw, Iy * Iz, false, s))) return e;
  if ((e = launch_lines<T>(g, p->fy, p->d_tw, C, Iz, (long)Iy * C, C, false, nullptr, s))) return e;
  if ((e = launch_lines<T>(g, p->fz, p->d_tw, C, Iy, C, (long)Iy * C, false,
                           reinterpret_cast<const T*>(p->d_mult), s)))
    return e;
  if ((e = launch_lines<T>(g, p->fy, p->d_tw, C, Iz, (long)Iy * C, C, true, nullptr, s))) return e;
  return launch_x<T>(g, p->fx, p->d_tw, Iy * Iz, true, s);
}

// Algorithm 2 steps 2 and 4: 2D FFTs of the Chebyshev proxy planes (layout
// [n][y][x], pitch Ix_long + 2), forward (inv = false) or backward.
template <typename T>
static cudaError_t fft_long_half(const sog_plan* p, T* g, bool inv, cudaStream_t s) {
  const int Ix = p->prm.I_long[0], Iy = p->prm.I_long[1], P = p->prm.P_cheb;
  const int C = Ix / 2 + 1;
  cudaError_t e;
  if (!inv) {
    if ((e = launch_x<T>(g, p->flx, p->d_tw, Iy * P, false, s))) return e;
    return launch_lines<T>(g, p->fly, p->d_tw, C, P, (long)Iy * C, C, false, nullptr, s);
  }
  if ((e = launch_lines<T>(g, p->fly, p->d_tw, C, P, (long)Iy * C, C, true, nullptr, s))) return e;
  return launch_x<T>(g, p->flx, p->d_tw, Iy * P, true, s);
}

// Allow the FFT kernels the full dynamic shared memory of an SM (set once per
// process before any launch or stream capture).
template <typename T>
cudaError_t fft_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_fft_x<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxDynSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_lines<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem);
  return e;
}
template cudaError_t fft_prepare<float>();
template cudaError_t fft_prepare<double>();

template cudaError_t fft_mid_forward_conv_inverse<float>(const sog_plan*, cudaStream_t);
template cudaError_t fft_mid_forward_conv_inverse<double>(const sog_plan*, cudaStream_t);

// Exposed to the kernel driver: forward (inv = false) on d_lA, backward on d_lB.
template <typename T>
cudaError_t fft_long_pass(const sog_plan* p, bool inv, cudaStream_t s) {
  return fft_long_half<T>(p, reinterpret_cast<T*>(inv ? p->d_lB : p->d_lA), inv, s);
}
template cudaError_t fft_long_pass<float>(const sog_plan*, bool, cudaStream_t);
template cudaError_t fft_long_pass<double>(const sog_plan*, bool, cudaStream_t);

}  // namespace sogk
