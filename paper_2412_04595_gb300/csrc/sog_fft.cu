// Batched mixed-radix FFTs of the spectral SOG solvers, in shared memory.
//
// Algorithm 1 needs a forward 3D FFT, the scaling of Eq. (3.8) and a
// backward 3D FFT on the real grid; Algorithm 2 needs forward and backward 2D
// FFTs of every Chebyshev proxy plane with a z-contraction in between.
//
// Engine: a CTA (FftCfg: threads, values per thread) holds a set of lines in
// shared memory and transforms them in place with self-sorting (Stockham)
// stages of radix 2, 3, 4, 5, 7, 8, and for FP32 also 15 (3 x 5) and 16
// (4 x 4).  In a stage every thread reads the inputs of its butterflies into
// registers, applies twiddles and the butterfly, waits at a barrier and
// writes the outputs, so one buffer suffices; a thread holds at most
// FftCfg::cap complex values.  Index arithmetic uses exact float
// reciprocals instead of integer division.  Transforms are unnormalised; the
// 1/n factors live in the scaling tables.
//
// Kernels:
//   k_fft_plane  one CTA per xy plane: real rows packed in pairs as complex
//                lines, x FFT, split into half spectra, y FFT (forward), or
//                the reverse; used when a plane fits one CTA.
//   k_fft_rows   x pass alone (pairs of real rows), for planes that do not fit.
//   k_fft_cols   complex lines with a stride (y pass), or the z pass of
//                Algorithm 1: forward FFT, multiplication by the scaling
//                factor, backward FFT without a round trip through memory.
#include "sog_internal.h"

namespace sogk {

// Twiddle table entry: FP32 (cos, sin) and the parts lost to their
// rounding; FP64 (cos, sin).
struct alignas(16) TwF {
  float x, y, z, w;
};
struct alignas(16) TwD {
  double x, y;
};

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; using tw = TwF; };
template <> struct C2<double> { using t = double2; using tw = TwD; };

// Threads per CTA, complex values a thread holds in a stage, and CTAs per
// SM the register budget is sized for: FP32 runs two CTAs of 512 threads per
// SM (one CTA's barriers overlap the other's work), FP64 one of 1024.
template <typename T> struct FftCfg;
template <> struct FftCfg<float> { static constexpr int threads = 512, cap = 16, minb = 2; };
template <> struct FftCfg<double> { static constexpr int threads = 1024, cap = 8, minb = 1; };

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

// a times the twiddle w = (cos, sin) + (cos_lo, sin_lo) (its conjugate for
// the inverse): the rounding-error parts are applied first
__device__ __forceinline__ float2 cmul_tw(float2 a, TwF w, bool inv) {
  const float sh = inv ? -w.y : w.y;
  const float sl = inv ? -w.w : w.w;
  const float re_lo = a.x * w.z - a.y * sl;
  const float im_lo = a.x * sl + a.y * w.z;
  return float2{fmaf(a.x, w.x, fmaf(-a.y, sh, re_lo)), fmaf(a.x, sh, fmaf(a.y, w.x, im_lo))};
}
__device__ __forceinline__ double2 cmul_tw(double2 a, TwD w, bool inv) {
  const double sh = inv ? -w.y : w.y;
  return double2{a.x * w.x - a.y * sh, a.x * sh + a.y * w.x};
}

// floor(a / b) for 0 <= a < 2^22 from rb = 1/b rounded to float: the
// fractional part of (a + 1/2) / b is at least 1/(2b) away from an integer
// and the relative error of the product is below 2^-23.
__device__ __forceinline__ int fdiv(int a, float rb) { return (int)(((float)a + 0.5f) * rb); }

// A set of nl lines of length n in shared memory: element i of line l at
// l * ls + i * es.  line_fast: consecutive threads take consecutive lines
// (lines adjacent in memory), else consecutive elements of one line.
struct LineSet {
  int n, nl, ls, es;
  bool line_fast;
};

// a / sqrt(2) to within the rounding of the result
__device__ __forceinline__ float div_sqrt2(float a) {
  return fmaf(a, 0.70710676908493042f, a * 1.2101617e-8f);
}
__device__ __forceinline__ double div_sqrt2(double a) {
  return fma(a, 0.70710678118654746, a * 6.2685835895251089e-17);
}

// a times a constant given as a rounded value hi plus its rounding error lo
// (FP32); FP64 uses the double constant.
__device__ __forceinline__ float mulc(float a, float hi, float lo, double) {
  return fmaf(a, hi, a * lo);
}
__device__ __forceinline__ double mulc(double a, float, float, double v) { return a * v; }

// a + i b (inv) or a - i b
template <typename T2>
__device__ __forceinline__ T2 pm_i(T2 a, T2 b, bool plus) {
  return plus ? T2{a.x - b.y, a.y + b.x} : T2{a.x + b.y, a.y - b.x};
}

template <typename T2, int R, typename T4>
__device__ __forceinline__ void dft(T2* x, bool inv, const T4* tw, int n) {
  if constexpr (R == 2) {
    const T2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const T2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    const T2 s13 = cadd(x[1], x[3]), d13 = rot(csub(x[1], x[3]), inv);
    x[0] = cadd(s02, s13);
    x[2] = csub(s02, s13);
    x[1] = cadd(d02, d13);
    x[3] = csub(d02, d13);
  } else if constexpr (R == 8) {
    // two DFT4 on even and odd samples, odd part rotated by w8^k
    T2 e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
    dft<T2, 4>(e, inv, tw, n);
    dft<T2, 4>(o, inv, tw, n);
    // w8^1 = (1 - i)/sqrt2 forward, (1 + i)/sqrt2 inverse; w8^2 = -i / +i.
    // 1/sqrt2 is applied as a rounded value plus its rounding error (no
    // floating-point number h has 2 h^2 = 1, and a biased rotation would
    // shrink every transform by a few 1e-8).
    const T2 o1 = inv ? T2{div_sqrt2(o[1].x - o[1].y), div_sqrt2(o[1].x + o[1].y)}
                      : T2{div_sqrt2(o[1].x + o[1].y), div_sqrt2(o[1].y - o[1].x)};
    const T2 o2 = rot(o[2], inv);
    const T2 o3 = inv ? T2{-div_sqrt2(o[3].x + o[3].y), div_sqrt2(o[3].x - o[3].y)}
                      : T2{div_sqrt2(o[3].y - o[3].x), -div_sqrt2(o[3].x + o[3].y)};
    x[0] = cadd(e[0], o[0]);
    x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[5] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[6] = csub(e[2], o2);
    x[3] = cadd(e[3], o3);
    x[7] = csub(e[3], o3);
  } else if constexpr (R == 3) {
    // w = e^(-2 pi i / 3) = -1/2 - i sqrt3/2
    const T2 t = cadd(x[1], x[2]), d = csub(x[1], x[2]);
    const T2 a = T2{x[0].x - 0.5f * t.x, x[0].y - 0.5f * t.y};
    const T2 b = T2{mulc(d.x, 8.660253882e-01f, 1.554362505e-08f, 0.8660254037844386),
                    mulc(d.y, 8.660253882e-01f, 1.554362505e-08f, 0.8660254037844386)};
    x[0] = cadd(x[0], t);
    x[1] = pm_i(a, b, inv);
    x[2] = pm_i(a, b, !inv);
  } else if constexpr (R == 5) {
    // w = e^(-2 pi i / 5) = c1 - i s1, w^2 = c2 - i s2
    const T2 t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
    const T2 t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
#define SOG_C1(v) mulc(v, 3.090170026e-01f, -8.207602598e-09f, 0.30901699437494745)
#define SOG_C2(v) mulc(v, -8.090170026e-01f, 8.207602598e-09f, -0.8090169943749473)
#define SOG_S1(v) mulc(v, 9.510565400e-01f, -2.371720598e-08f, 0.9510565162951535)
#define SOG_S2(v) mulc(v, 5.877852440e-01f, 8.304436250e-09f, 0.5877852522924732)
    const T2 a1 = T2{x[0].x + SOG_C1(t1.x) + SOG_C2(t2.x), x[0].y + SOG_C1(t1.y) + SOG_C2(t2.y)};
    const T2 a2 = T2{x[0].x + SOG_C2(t1.x) + SOG_C1(t2.x), x[0].y + SOG_C2(t1.y) + SOG_C1(t2.y)};
    const T2 b1 = T2{SOG_S1(t3.x) + SOG_S2(t4.x), SOG_S1(t3.y) + SOG_S2(t4.y)};
    const T2 b2 = T2{SOG_S2(t3.x) - SOG_S1(t4.x), SOG_S2(t3.y) - SOG_S1(t4.y)};
#undef SOG_C1
#undef SOG_C2
#undef SOG_S1
#undef SOG_S2
    x[0] = cadd(x[0], cadd(t1, t2));
    x[1] = pm_i(a1, b1, inv);
    x[4] = pm_i(a1, b1, !inv);
    x[2] = pm_i(a2, b2, inv);
    x[3] = pm_i(a2, b2, !inv);
  } else if constexpr (R == 16) {
    // 4 x 4: DFT4 over x[j2 + 4 j1] for each j2, twiddles w16^(j2 k1) from
    // the length-n table (entry j2 k1 n / 16), DFT4 over j2 for each k1;
    // output k1 + 4 k2
    T2 a[4][4];
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
      T2 v[4] = {x[j2], x[4 + j2], x[8 + j2], x[12 + j2]};
      dft<T2, 4>(v, inv, tw, n);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1)
        a[j2][k1] = (j2 == 0 || k1 == 0) ? v[k1] : cmul_tw(v[k1], tw[j2 * k1 * (n / 16)], inv);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      T2 v[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      dft<T2, 4>(v, inv, tw, n);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = v[k2];
    }
  } else if constexpr (R == 15) {
    // 3 x 5: DFT3 over x[j2 + 5 j1] for each j2, twiddles w15^(j2 k1) from
    // the length-n table, DFT5 over j2 for each k1; output k1 + 3 k2
    T2 a[5][3];
#pragma unroll
    for (int j2 = 0; j2 < 5; ++j2) {
      T2 v[3] = {x[j2], x[5 + j2], x[10 + j2]};
      dft<T2, 3>(v, inv, tw, n);
#pragma unroll
      for (int k1 = 0; k1 < 3; ++k1)
        a[j2][k1] = (j2 == 0 || k1 == 0) ? v[k1] : cmul_tw(v[k1], tw[j2 * k1 * (n / 15)], inv);
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      T2 v[5] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1], a[4][k1]};
      dft<T2, 5>(v, inv, tw, n);
#pragma unroll
      for (int k2 = 0; k2 < 5; ++k2) x[k1 + 3 * k2] = v[k2];
    }
  } else {
    // other odd radix (7): y_q = sum_p x_p w^(qp), w = exp(-+2 pi i / R) from
    // the length-n table (entry (qp mod R) n / R)
    const int step = n / R;
    T2 y[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T2 s = x[0];
#pragma unroll
      for (int p = 1; p < R; ++p) {
        s = cadd(s, cmul_tw(x[p], tw[((q * p) % R) * step], inv));
      }
      y[q] = s;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = y[q];
  }
}

// One in-place Stockham stage of radix R; L = product of earlier radices.
template <typename T2, int CAP, int R, typename T4>
__device__ __forceinline__ void stage(T2* buf, const LineSet s, int L, const T4* tw, bool inv) {
  constexpr int KB = CAP / R;
  const int nb = s.n / R, m = nb / L;
  const int tot = s.nl * nb;
  const float rq = s.line_fast ? 1.f / (float)s.nl : 1.f / (float)nb;
  const float rL = 1.f / (float)L;
  T2 x[KB][R];
  int wb[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int id = threadIdx.x + k * (int)blockDim.x;
    wb[k] = -1;
    if (id < tot) {
      int line, t;
      if (s.line_fast) {
        t = fdiv(id, rq);
        line = id - t * s.nl;
      } else {
        line = fdiv(id, rq);
        t = id - line * nb;
      }
      const int kk = fdiv(t, rL), j = t - kk * L;
      const T2* a = buf + line * s.ls + (kk * L + j) * s.es;
      const int st = m * L * s.es;
#pragma unroll
      for (int p = 0; p < R; ++p) x[k][p] = a[p * st];
#pragma unroll
      for (int p = 1; p < R; ++p) x[k][p] = cmul_tw(x[k][p], tw[j * p * m], inv);
      dft<T2, R>(x[k], inv, tw, s.n);
      wb[k] = line * s.ls + (kk * L * R + j) * s.es;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    if (wb[k] >= 0) {
      T2* b = buf + wb[k];
      const int st = L * s.es;
#pragma unroll
      for (int q = 0; q < R; ++q) b[q * st] = x[k][q];
    }
  }
  __syncthreads();
}

// All stages of one length.  The factorisation orders the radices 16..16,
// 15..15 (engines holding at least 16 values per thread), 8..8, 4, 2, 3..3,
// 5..5, 7..7; each group is a separate straight-line block so that the
// registers of one stage are free for the next.
template <typename T2, int CAP, typename T4>
__device__ void fft_lines(T2* buf, const LineSet s, const FftLen& f, const T4* tw, bool inv) {
  const int n16 = f.n16, n15 = f.n15, n8 = f.n8, n4 = f.n4, n2 = f.n2, n3 = f.n3, n5 = f.n5,
            n7 = f.n7;
  int L = 1;
  if constexpr (CAP >= 16) {
    for (int i = 0; i < n16; ++i, L *= 16) stage<T2, CAP, 16>(buf, s, L, tw, inv);
    for (int i = 0; i < n15; ++i, L *= 15) stage<T2, CAP, 15>(buf, s, L, tw, inv);
  }
  for (int i = 0; i < n8; ++i, L *= 8) stage<T2, CAP, 8>(buf, s, L, tw, inv);
  if (n4) { stage<T2, CAP, 4>(buf, s, L, tw, inv); L *= 4; }
  if (n2) { stage<T2, CAP, 2>(buf, s, L, tw, inv); L *= 2; }
  for (int i = 0; i < n3; ++i, L *= 3) stage<T2, CAP, 3>(buf, s, L, tw, inv);
  for (int i = 0; i < n5; ++i, L *= 5) stage<T2, CAP, 5>(buf, s, L, tw, inv);
  for (int i = 0; i < n7; ++i, L *= 7) stage<T2, CAP, 7>(buf, s, L, tw, inv);
}

// Largest nl for which nl lines of length n fit the engine.
static int max_lines(const FftLen& f, int cap, int nt) {
  int best = 1 << 30;
  for (int st = 0; st < f.nst; ++st) {
    const int R = f.radix[st];
    best = std::min(best, nt * (cap / R) / (f.n / R));
  }
  return best;
}

template <typename T4>
__device__ __forceinline__ void load_tw(T4* dst, const T4* src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Split Z = FFT(row 2p + i row 2p+1) into the half spectra of both rows,
// in place: Z in [p][x] (pitch Ix) -> H in [y][k] (pitch C = Ix/2 + 1).
template <typename T2, int CAP>
__device__ __forceinline__ void split_pairs(T2* buf, int Ix, int npairs) {
  using T = decltype(buf[0].x);
  const int C = Ix / 2 + 1;
  const int tot = npairs * C;
  const float rC = 1.f / (float)C;
  constexpr int KB = CAP / 2;
  T2 a[KB], b[KB];
  int pr[KB], fq[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int id = threadIdx.x + k * (int)blockDim.x;
    pr[k] = -1;
    if (id < tot) {
      const int p = fdiv(id, rC), f = id - p * C;
      const T2 Z = buf[p * Ix + f], Zc = buf[p * Ix + (f == 0 ? 0 : Ix - f)];
      const T h = T(0.5);
      a[k] = T2{h * (Z.x + Zc.x), h * (Z.y - Zc.y)};
      b[k] = T2{h * (Z.y + Zc.y), h * (Zc.x - Z.x)};
      pr[k] = p;
      fq[k] = f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < KB; ++k)
    if (pr[k] >= 0) {
      buf[(2 * pr[k]) * C + fq[k]] = a[k];
      buf[(2 * pr[k] + 1) * C + fq[k]] = b[k];
    }
  __syncthreads();
}

// Inverse of split_pairs: H [y][k] -> Z [p][x] with Z = X_2p + i X_2p+1 over
// the full length (Hermitian symmetry for k > Ix/2).
template <typename T2, int CAP>
__device__ __forceinline__ void join_pairs(T2* buf, int Ix, int npairs) {
  const int C = Ix / 2 + 1, nh = Ix / 2;
  const int tot = npairs * C;
  const float rC = 1.f / (float)C;
  constexpr int KB = CAP / 2;
  T2 a[KB], b[KB];
  int pr[KB], fq[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int id = threadIdx.x + k * (int)blockDim.x;
    pr[k] = -1;
    if (id < tot) {
      const int p = fdiv(id, rC), f = id - p * C;
      const T2 A = buf[(2 * p) * C + f], B = buf[(2 * p + 1) * C + f];
      a[k] = T2{A.x - B.y, A.y + B.x};
      b[k] = T2{A.x + B.y, B.x - A.y};
      pr[k] = p;
      fq[k] = f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < KB; ++k)
    if (pr[k] >= 0) {
      buf[pr[k] * Ix + fq[k]] = a[k];
      if (fq[k] > 0 && fq[k] < nh) buf[pr[k] * Ix + Ix - fq[k]] = b[k];
    }
  __syncthreads();
}

// 2D real FFT of one plane per CTA.  Plane z: Iy rows of Ix reals with pitch
// Ix + 2 at data + z * Iy * (Ix + 2); the half spectrum [ky][kx] (C complex
// per row) is stored over the same memory.
template <typename T>
__global__ void __launch_bounds__(FftCfg<T>::threads, FftCfg<T>::minb)
    k_fft_plane(T* __restrict__ data, FftLen fx, FftLen fy, const typename C2<T>::tw* __restrict__ twg,
                bool inv) {
  using T2 = typename C2<T>::t;
  using T4 = typename C2<T>::tw;
  constexpr int CAP = FftCfg<T>::cap;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Ix = fx.n, Iy = fy.n, C = Ix / 2 + 1, pitch = Ix + 2;
  const int np = Iy / 2;
  T4* twx = reinterpret_cast<T4*>(smraw);
  T4* twy = twx + Ix;
  T2* buf = reinterpret_cast<T2*>(twy + Iy);
  load_tw(twx, twg + fx.tw_off, Ix);
  load_tw(twy, twg + fy.tw_off, Iy);
  T* pl = data + (size_t)blockIdx.x * Iy * pitch;
  T2* plc = reinterpret_cast<T2*>(pl);
  const LineSet xs{Ix, np, Ix, 1, false};
  const LineSet ys{Iy, C, 1, C, true};
  if (!inv) {
    const float rI = 1.f / (float)Ix;
    for (int id = threadIdx.x; id < np * Ix; id += blockDim.x) {
      const int p = fdiv(id, rI), x = id - p * Ix;
      const T* r0 = pl + (size_t)(2 * p) * pitch + x;
      buf[id] = T2{r0[0], r0[pitch]};
    }
    __syncthreads();
    fft_lines<T2, CAP>(buf, xs, fx, twx, false);
    split_pairs<T2, CAP>(buf, Ix, np);
    fft_lines<T2, CAP>(buf, ys, fy, twy, false);
    for (int id = threadIdx.x; id < Iy * C; id += blockDim.x) plc[id] = buf[id];
  } else {
    for (int id = threadIdx.x; id < Iy * C; id += blockDim.x) buf[id] = plc[id];
    __syncthreads();
    fft_lines<T2, CAP>(buf, ys, fy, twy, true);
    join_pairs<T2, CAP>(buf, Ix, np);
    fft_lines<T2, CAP>(buf, xs, fx, twx, true);
    const float rI = 1.f / (float)Ix;
    for (int id = threadIdx.x; id < np * Ix; id += blockDim.x) {
      const int p = fdiv(id, rI), x = id - p * Ix;
      T* r0 = pl + (size_t)(2 * p) * pitch + x;
      const T2 z = buf[id];
      r0[0] = z.x;
      r0[pitch] = z.y;
    }
  }
}

// x pass alone: rows 2p, 2p+1 (pitch Ix + 2) of pairs p0 .. p0 + B - 1.
template <typename T>
__global__ void __launch_bounds__(FftCfg<T>::threads, FftCfg<T>::minb)
    k_fft_rows(T* __restrict__ data, FftLen fx, const typename C2<T>::tw* __restrict__ twg,
               int npairs, int B, bool inv) {
  using T2 = typename C2<T>::t;
  constexpr int CAP = FftCfg<T>::cap;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Ix = fx.n, C = Ix / 2 + 1, pitch = Ix + 2;
  using T4 = typename C2<T>::tw;
  T4* twx = reinterpret_cast<T4*>(smraw);
  T2* buf = reinterpret_cast<T2*>(twx + Ix);
  load_tw(twx, twg + fx.tw_off, Ix);
  const int p0 = blockIdx.x * B;
  const int nl = min(B, npairs - p0);
  T* base = data + (size_t)(2 * p0) * pitch;
  const LineSet xs{Ix, nl, Ix, 1, false};
  const float rI = 1.f / (float)Ix, rC = 1.f / (float)C;
  if (!inv) {
    for (int id = threadIdx.x; id < nl * Ix; id += blockDim.x) {
      const int p = fdiv(id, rI), x = id - p * Ix;
      const T* r0 = base + (size_t)(2 * p) * pitch + x;
      buf[id] = T2{r0[0], r0[pitch]};
    }
    __syncthreads();
    fft_lines<T2, CAP>(buf, xs, fx, twx, false);
    split_pairs<T2, CAP>(buf, Ix, nl);
    for (int id = threadIdx.x; id < 2 * nl * C; id += blockDim.x) {
      const int y = fdiv(id, rC), f = id - y * C;
      reinterpret_cast<T2*>(base + (size_t)y * pitch)[f] = buf[id];
    }
  } else {
    for (int id = threadIdx.x; id < 2 * nl * C; id += blockDim.x) {
      const int y = fdiv(id, rC), f = id - y * C;
      buf[id] = reinterpret_cast<const T2*>(base + (size_t)y * pitch)[f];
    }
    __syncthreads();
    join_pairs<T2, CAP>(buf, Ix, nl);
    fft_lines<T2, CAP>(buf, xs, fx, twx, true);
    for (int id = threadIdx.x; id < nl * Ix; id += blockDim.x) {
      const int p = fdiv(id, rI), x = id - p * Ix;
      T* r0 = base + (size_t)(2 * p) * pitch + x;
      const T2 z = buf[id];
      r0[0] = z.x;
      r0[pitch] = z.y;
    }
  }
}

// Complex lines (o, c), o < O, c < Cn: element i at o*os + c + i*es (complex
// units).  A CTA takes B consecutive c of one o, held as [i][c].  With mult
// (z pass of Algorithm 1): forward FFT, multiply element (o, c, i) by
// mult[(i*O + o)*Cn + c], backward FFT.
template <typename T>
__global__ void __launch_bounds__(FftCfg<T>::threads, FftCfg<T>::minb)
    k_fft_cols(typename C2<T>::t* __restrict__ data, FftLen f, const typename C2<T>::tw* __restrict__ twg,
               int Cn, int O, long os, long es, int B, bool inv, const T* __restrict__ mult) {
  using T2 = typename C2<T>::t;
  constexpr int CAP = FftCfg<T>::cap;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = f.n;
  using T4 = typename C2<T>::tw;
  T4* tw = reinterpret_cast<T4*>(smraw);
  T2* buf = reinterpret_cast<T2*>(tw + n);
  load_tw(tw, twg + f.tw_off, n);
  const int gpo = (Cn + B - 1) / B;
  const int o = blockIdx.x / gpo;
  const int c0 = (blockIdx.x - o * gpo) * B;
  const int nl = min(B, Cn - c0);
  T2* base = data + (size_t)o * os + c0;
  const float rl = 1.f / (float)nl;
  for (int id = threadIdx.x; id < nl * n; id += blockDim.x) {
    const int i = fdiv(id, rl), c = id - i * nl;
    buf[id] = base[(size_t)i * es + c];
  }
  __syncthreads();
  const LineSet cs{n, nl, 1, nl, true};
  fft_lines<T2, CAP>(buf, cs, f, tw, mult ? false : inv);
  if (mult) {
    for (int id = threadIdx.x; id < nl * n; id += blockDim.x) {
      const int i = fdiv(id, rl), c = id - i * nl;
      const T sc = mult[((size_t)i * O + o) * Cn + c0 + c];
      const T2 v = buf[id];
      buf[id] = T2{v.x * sc, v.y * sc};
    }
    __syncthreads();
    fft_lines<T2, CAP>(buf, cs, f, tw, true);
  }
  for (int id = threadIdx.x; id < nl * n; id += blockDim.x) {
    const int i = fdiv(id, rl), c = id - i * nl;
    base[(size_t)i * es + c] = buf[id];
  }
}

// True when a whole Ix x Iy plane fits one CTA of k_fft_plane with nt
// threads.
template <typename T>
static bool plane_fits(const FftLen& fx, const FftLen& fy, int nt = FftCfg<T>::threads) {
  constexpr int CAP = FftCfg<T>::cap;
  const int C = fx.n / 2 + 1;
  const size_t smem = (size_t)(fx.n + fy.n) * sizeof(typename C2<T>::tw) +
                      (size_t)std::max((fy.n / 2) * fx.n, fy.n * C) * sizeof(typename C2<T>::t);
  return max_lines(fx, CAP, nt) >= fy.n / 2 && max_lines(fy, CAP, nt) >= C &&
         (fy.n / 2) * C <= nt * (CAP / 2) && smem <= (size_t)kMaxDynSmem;
}

// Fewest threads (a multiple of 128) whose CTA holds the whole plane: small
// planes (the long range's proxy planes) do not need 1024 threads.
template <typename T>
static int plane_threads(const FftLen& fx, const FftLen& fy) {
  for (int nt = 128; nt < FftCfg<T>::threads; nt *= 2)
    if (plane_fits<T>(fx, fy, nt)) return nt;
  return FftCfg<T>::threads;
}

template <typename T>
static cudaError_t launch_plane(T* data, const FftLen& fx, const FftLen& fy, const void* tw,
                                int nplanes, bool inv, cudaStream_t s) {
  using T2 = typename C2<T>::t;
  const int C = fx.n / 2 + 1;
  using T4 = typename C2<T>::tw;
  const size_t sm = (size_t)(fx.n + fy.n) * sizeof(T4) +
                    (size_t)std::max((fy.n / 2) * fx.n, fy.n * C) * sizeof(T2);
  k_fft_plane<T><<<nplanes, plane_threads<T>(fx, fy), sm, s>>>(data, fx, fy,
                                                                reinterpret_cast<const T4*>(tw),
                                                  inv);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_rows(T* data, const FftLen& fx, const void* tw, int nrows, bool inv,
                               cudaStream_t s) {
  using T2 = typename C2<T>::t;
  constexpr int CAP = FftCfg<T>::cap;
  const int npairs = nrows / 2;
  const int C = fx.n / 2 + 1;
  constexpr int NT = FftCfg<T>::threads;
  int B = std::min(max_lines(fx, CAP, NT), NT * (CAP / 2) / C);
  B = std::max(1, std::min(B, npairs));
  using T4 = typename C2<T>::tw;
  const size_t sm = (size_t)fx.n * sizeof(T4) + (size_t)B * std::max(fx.n, 2 * C) * sizeof(T2);
  const int grid = (npairs + B - 1) / B;
  k_fft_rows<T><<<grid, NT, sm, s>>>(data, fx, reinterpret_cast<const T4*>(tw), npairs,
                                              B, inv);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_cols(T* data, const FftLen& f, const void* tw, int Cn, int O, long os,
                               long es, bool inv, const T* mult, cudaStream_t s) {
  using T2 = typename C2<T>::t;
  constexpr int CAP = FftCfg<T>::cap;
  constexpr int NT = FftCfg<T>::threads;
  int B = std::max(1, std::min(max_lines(f, CAP, NT), Cn));
  // balance the groups of one o
  const int groups = (Cn + B - 1) / B;
  B = (Cn + groups - 1) / groups;
  using T4 = typename C2<T>::tw;
  const size_t sm = (size_t)f.n * sizeof(T4) + (size_t)B * f.n * sizeof(T2);
  const int grid = O * groups;
  k_fft_cols<T><<<grid, NT, sm, s>>>(reinterpret_cast<T2*>(data), f,
                                              reinterpret_cast<const T4*>(tw), Cn, O, os, es, B,
                                              inv, mult);
  return cudaGetLastError();
}

// Forward 2D FFT of nplanes planes of Ix x Iy (pitch Ix + 2), or backward.
template <typename T>
static cudaError_t fft_planes(T* g, const FftLen& fx, const FftLen& fy, const void* tw,
                              int nplanes, bool inv, cudaStream_t s, int& launches) {
  const int Ix = fx.n, Iy = fy.n, C = Ix / 2 + 1;
  if (plane_fits<T>(fx, fy)) {
    launches += 1;
    return launch_plane<T>(g, fx, fy, tw, nplanes, inv, s);
  }
  cudaError_t e;
  launches += 2;
  if (!inv) {
    if ((e = launch_rows<T>(g, fx, tw, Iy * nplanes, false, s))) return e;
    return launch_cols<T>(g, fy, tw, C, nplanes, (long)Iy * C, C, false, nullptr, s);
  }
  if ((e = launch_cols<T>(g, fy, tw, C, nplanes, (long)Iy * C, C, true, nullptr, s))) return e;
  return launch_rows<T>(g, fx, tw, Iy * nplanes, true, s);
}

// Algorithm 1 steps 2-4 on the mid grid (layout [z][y][x], pitch Ix + 2).
template <typename T>
cudaError_t fft_mid_forward_conv_inverse(const sog_plan* p, cudaStream_t s, int& launches) {
  T* g = reinterpret_cast<T*>(p->d_grid);
  const int Ix = p->prm.I[0], Iy = p->prm.I[1], Iz = p->prm.I[2];
  const int C = Ix / 2 + 1;
  cudaError_t e;
  if ((e = fft_planes<T>(g, p->fx, p->fy, p->d_tw, Iz, false, s, launches))) return e;
  if ((e = launch_cols<T>(g, p->fz, p->d_tw, C, Iy, C, (long)Iy * C, false,
                          reinterpret_cast<const T*>(p->d_mult), s)))
    return e;
  launches += 1;
  return fft_planes<T>(g, p->fx, p->fy, p->d_tw, Iz, true, s, launches);
}
template cudaError_t fft_mid_forward_conv_inverse<float>(const sog_plan*, cudaStream_t, int&);
template cudaError_t fft_mid_forward_conv_inverse<double>(const sog_plan*, cudaStream_t, int&);

// Algorithm 2 steps 2 and 4: 2D FFTs of the Chebyshev proxy planes (layout
// [n][y][x], pitch Ix_long + 2), forward on d_lA (inv = false) or backward
// on d_lB.
template <typename T>
cudaError_t fft_long_pass(const sog_plan* p, bool inv, cudaStream_t s, int& launches) {
  T* g = reinterpret_cast<T*>(inv ? p->d_lB : p->d_lA);
  return fft_planes<T>(g, p->flx, p->fly, p->d_tw, p->prm.P_cheb, inv, s, launches);
}
template cudaError_t fft_long_pass<float>(const sog_plan*, bool, cudaStream_t, int&);
template cudaError_t fft_long_pass<double>(const sog_plan*, bool, cudaStream_t, int&);

// True when transforms of this length fit the engine (at least one line per
// CTA; the x pass also needs its half spectrum to fit one CTA).
bool fft_len_ok(int prec, const FftLen& f) {
  const int cap = prec == SOG_PREC_FP64 ? FftCfg<double>::cap : FftCfg<float>::cap;
  const int nt = prec == SOG_PREC_FP64 ? FftCfg<double>::threads : FftCfg<float>::threads;
  const size_t elem = prec == SOG_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t twe = prec == SOG_PREC_FP64 ? sizeof(TwD) : sizeof(TwF);
  return f.n >= 2 && max_lines(f, cap, nt) >= 1 && (f.n / 2 + 1) <= nt * (cap / 2) &&
         (size_t)f.n * twe + (size_t)(f.n + 2) * elem <= (size_t)kMaxDynSmem;
}

// Allow the FFT kernels the dynamic shared memory they may need (set once per
// process before any launch or stream capture).
template <typename T>
cudaError_t fft_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_fft_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxDynSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem);
  return e;
}
template cudaError_t fft_prepare<float>();
template cudaError_t fft_prepare<double>();

}  // namespace sogk
