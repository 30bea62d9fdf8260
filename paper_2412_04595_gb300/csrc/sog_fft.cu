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

// Threads of the fused y pass of Algorithm 2 (one CTA per SM).
constexpr int kYpassThreads = 1024;

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

// ---------------------------------------------------------------------------
// Asynchronous copies.  cp.async moves 4, 8 or 16 bytes per thread without
// blocking, so a CTA keeps its whole tile's loads in flight at once;
// cp.async.bulk (the TMA's bulk copy) moves a contiguous block, completing on
// an mbarrier (loads) or a bulk group (stores).
// ---------------------------------------------------------------------------

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes)
               : "memory");
}
// Bulk copy global -> shared of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing on bar.
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, unsigned bytes,
                                         unsigned long long* bar) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const unsigned ba = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(sa), "l"(gmem), "r"(bytes), "r"(ba)
      : "memory");
}
// Wait for phase `phase` of bar to complete, at most kMbarSpins polls; false
// when the limit ran out.
constexpr long kMbarSpins = 1L << 24;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  for (long it = 0; it < kMbarSpins; ++it) {
    unsigned done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}
// Bulk copy shared -> global (sizes and alignment as bulk_g2s), then wait
// until the shared memory has been read (the issuing thread only).
__device__ __forceinline__ void bulk_s2g_wait(void* gmem, const void* smem, unsigned bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem),
               "r"(sa), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// Make this thread's generic-proxy shared-memory writes visible to the bulk
// copies (the async proxy).
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
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
        a[j2][k1] = (j2 == 0 || k1 == 0) ? v[k1] : cmul_tw(v[k1], tw[j2 * k1], inv);
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
        a[j2][k1] = (j2 == 0 || k1 == 0) ? v[k1] : cmul_tw(v[k1], tw[16 + j2 * k1], inv);
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      T2 v[5] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1], a[4][k1]};
      dft<T2, 5>(v, inv, tw, n);
#pragma unroll
      for (int k2 = 0; k2 < 5; ++k2) x[k1 + 3 * k2] = v[k2];
    }
  } else if constexpr (R == 7) {
    // w = e^(-2 pi i / 7): with t_k = x_k + x_(7-k), d_k = x_k - x_(7-k) and
    // c_k = cos(2 pi k / 7), s_k = sin(2 pi k / 7),
    //   y_1 = x_0 + c1 t1 + c2 t2 + c3 t3 - i (s1 d1 + s2 d2 + s3 d3),
    //   y_2 = x_0 + c2 t1 + c3 t2 + c1 t3 - i (s2 d1 - s3 d2 - s1 d3),
    //   y_3 = x_0 + c3 t1 + c1 t2 + c2 t3 - i (s3 d1 - s1 d2 + s2 d3),
    //   y_(7-k) the same with + i (constants as value plus rounding error)
    const T2 t1 = cadd(x[1], x[6]), t2 = cadd(x[2], x[5]), t3 = cadd(x[3], x[4]);
    const T2 d1 = csub(x[1], x[6]), d2 = csub(x[2], x[5]), d3 = csub(x[3], x[4]);
#define SOG_C1(v) mulc(v, 6.234897971e-01f, 4.743407445e-09f, 0.6234898018587336)
#define SOG_C2(v) mulc(v, -2.225209326e-01f, -1.401115668e-09f, -0.22252093395631434)
#define SOG_C3(v) mulc(v, -9.009688497e-01f, -1.824345297e-08f, -0.900968867902419)
#define SOG_S1(v) mulc(v, 7.818315029e-01f, -2.044639835e-08f, 0.7818314824680298)
#define SOG_S2(v) mulc(v, 9.749279022e-01f, 9.960143821e-09f, 0.9749279121818236)
#define SOG_S3(v) mulc(v, 4.338837266e-01f, 1.252072579e-08f, 0.43388373911755823)
    const T2 a1 = T2{x[0].x + SOG_C1(t1.x) + SOG_C2(t2.x) + SOG_C3(t3.x),
                     x[0].y + SOG_C1(t1.y) + SOG_C2(t2.y) + SOG_C3(t3.y)};
    const T2 a2 = T2{x[0].x + SOG_C2(t1.x) + SOG_C3(t2.x) + SOG_C1(t3.x),
                     x[0].y + SOG_C2(t1.y) + SOG_C3(t2.y) + SOG_C1(t3.y)};
    const T2 a3 = T2{x[0].x + SOG_C3(t1.x) + SOG_C1(t2.x) + SOG_C2(t3.x),
                     x[0].y + SOG_C3(t1.y) + SOG_C1(t2.y) + SOG_C2(t3.y)};
    const T2 b1 = T2{SOG_S1(d1.x) + SOG_S2(d2.x) + SOG_S3(d3.x),
                     SOG_S1(d1.y) + SOG_S2(d2.y) + SOG_S3(d3.y)};
    const T2 b2 = T2{SOG_S2(d1.x) - SOG_S3(d2.x) - SOG_S1(d3.x),
                     SOG_S2(d1.y) - SOG_S3(d2.y) - SOG_S1(d3.y)};
    const T2 b3 = T2{SOG_S3(d1.x) - SOG_S1(d2.x) + SOG_S2(d3.x),
                     SOG_S3(d1.y) - SOG_S1(d2.y) + SOG_S2(d3.y)};
#undef SOG_C1
#undef SOG_C2
#undef SOG_C3
#undef SOG_S1
#undef SOG_S2
#undef SOG_S3
    x[0] = cadd(x[0], cadd(cadd(t1, t2), t3));
    x[1] = pm_i(a1, b1, inv);
    x[6] = pm_i(a1, b1, !inv);
    x[2] = pm_i(a2, b2, inv);
    x[5] = pm_i(a2, b2, !inv);
    x[3] = pm_i(a3, b3, inv);
    x[4] = pm_i(a3, b3, !inv);
  } else {
    static_assert(R == 2, "radix without a butterfly");
  }
}

// One in-place Stockham stage of radix R; L = product of earlier radices.
template <typename T2, int CAP, int R, typename T4>
__device__ __forceinline__ void stage(T2* buf, const LineSet s, int L, const T4* tw,
                                      const T4* __restrict__ stw, bool inv) {
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
      for (int p = 1; p < R; ++p) x[k][p] = cmul_tw(x[k][p], stw[(p - 1) * L + j], inv);
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

// All stages of one length (a Stockham stage is correct in any order of the
// radices, given L = the product of the earlier ones).  Odd radices run
// first: with contiguous lines, a stage writes its outputs R elements apart
// across consecutive threads while L is small, which for an even R maps a
// warp onto few shared-memory banks; the even radices come once L is large.
// Each group is a separate straight-line block so that the registers of one
// stage are free for the next.
template <typename T2, int CAP, typename T4>
__device__ void fft_lines(T2* buf, const LineSet s, const FftLen& f, const T4* tw, bool inv) {
  const int n16 = f.n16, n15 = f.n15, n8 = f.n8, n4 = f.n4, n2 = f.n2, n3 = f.n3, n5 = f.n5,
            n7 = f.n7;
  // the stage tables follow the length-n table: stage by stage, in this
  // order, (R - 1) L entries [p - 1][j] = w_n^(j p n / (R L))
  const T4* stw = tw + kTwConst;
  int L = 1;
  if constexpr (CAP >= 16)
    for (int i = 0; i < n15; ++i, stw += 14 * L, L *= 15) stage<T2, CAP, 15>(buf, s, L, tw, stw, inv);
  for (int i = 0; i < n3; ++i, stw += 2 * L, L *= 3) stage<T2, CAP, 3>(buf, s, L, tw, stw, inv);
  for (int i = 0; i < n5; ++i, stw += 4 * L, L *= 5) stage<T2, CAP, 5>(buf, s, L, tw, stw, inv);
  for (int i = 0; i < n7; ++i, stw += 6 * L, L *= 7) stage<T2, CAP, 7>(buf, s, L, tw, stw, inv);
  if constexpr (CAP >= 16)
    for (int i = 0; i < n16; ++i, stw += 15 * L, L *= 16) stage<T2, CAP, 16>(buf, s, L, tw, stw, inv);
  for (int i = 0; i < n8; ++i, stw += 7 * L, L *= 8) stage<T2, CAP, 8>(buf, s, L, tw, stw, inv);
  if (n4) {
    stage<T2, CAP, 4>(buf, s, L, tw, stw, inv);
    stw += 3 * L;
    L *= 4;
  }
  if (n2) stage<T2, CAP, 2>(buf, s, L, tw, stw, inv);
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
  T4* twy = twx + tw_len(Ix);
  T2* buf = reinterpret_cast<T2*>(twy + tw_len(Iy));
  load_tw(twx, twg + fx.tw_off, tw_len(Ix));
  load_tw(twy, twg + fy.tw_off, tw_len(Iy));
  T* pl = data + (size_t)blockIdx.x * Iy * pitch;
  T2* plc = reinterpret_cast<T2*>(pl);
  const LineSet xs{Ix, np, Ix, 1, false};
  const LineSet ys{Iy, C, 1, C, true};
  if (!inv) {
    const float rI = 1.f / (float)Ix;
    for (int id = threadIdx.x; id < np * Ix; id += blockDim.x) {
      const int p = fdiv(id, rI), x = id - p * Ix;
      const T* r0 = pl + (size_t)(2 * p) * pitch + x;
      cp_async<sizeof(T)>(&buf[id].x, r0);
      cp_async<sizeof(T)>(&buf[id].y, r0 + pitch);
    }
    cp_async_wait();
    __syncthreads();
    fft_lines<T2, CAP>(buf, xs, fx, twx, false);
    split_pairs<T2, CAP>(buf, Ix, np);
    fft_lines<T2, CAP>(buf, ys, fy, twy, false);
    for (int id = threadIdx.x; id < Iy * C; id += blockDim.x) plc[id] = buf[id];
  } else {
    for (int id = threadIdx.x; id < Iy * C; id += blockDim.x) cp_async<sizeof(T2)>(buf + id, plc + id);
    cp_async_wait();
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
// With tdata, the half spectrum lives there transposed instead of in place:
// column f of row y of plane n at tdata[f * NR + R'], R' = (i + par np0) Iy
// + y for n = 2 i + par (planes of each parity contiguous within a column),
// written by the forward pass and read by the backward pass.
template <typename T>
__global__ void __launch_bounds__(FftCfg<T>::threads, FftCfg<T>::minb)
    k_fft_rows(T* __restrict__ data, FftLen fx, const typename C2<T>::tw* __restrict__ twg,
               int npairs, int B, bool inv, typename C2<T>::t* __restrict__ tdata, long NR,
               int Iy, int np0) {
  using T2 = typename C2<T>::t;
  constexpr int CAP = FftCfg<T>::cap;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Ix = fx.n, C = Ix / 2 + 1, pitch = Ix + 2;
  using T4 = typename C2<T>::tw;
  T4* twx = reinterpret_cast<T4*>(smraw);
  T2* buf = reinterpret_cast<T2*>(twx + tw_len(Ix));
  load_tw(twx, twg + fx.tw_off, tw_len(Ix));
  const int p0 = blockIdx.x * B;
  const int nl = min(B, npairs - p0);
  T* base = data + (size_t)(2 * p0) * pitch;
  const LineSet xs{Ix, nl, Ix, 1, false};
  const float rI = 1.f / (float)Ix, rC = 1.f / (float)C;
  if (!inv) {
    for (int id = threadIdx.x; id < nl * Ix; id += blockDim.x) {
      const int p = fdiv(id, rI), x = id - p * Ix;
      const T* r0 = base + (size_t)(2 * p) * pitch + x;
      cp_async<sizeof(T)>(&buf[id].x, r0);
      cp_async<sizeof(T)>(&buf[id].y, r0 + pitch);
    }
    cp_async_wait();
    __syncthreads();
    fft_lines<T2, CAP>(buf, xs, fx, twx, false);
    split_pairs<T2, CAP>(buf, Ix, nl);
    if (tdata) {
      // consecutive threads take consecutive rows of one column: runs of
      // contiguous elements in the transposed layout
      const float r2 = 1.f / (float)(2 * nl), rIy = 1.f / (float)Iy;
      for (int id = threadIdx.x; id < 2 * nl * C; id += blockDim.x) {
        const int f = fdiv(id, r2), y = id - f * 2 * nl;
        const int R = 2 * p0 + y, n = fdiv(R, rIy), yy = R - n * Iy;
        tdata[(size_t)f * NR + (size_t)((n >> 1) + (n & 1) * np0) * Iy + yy] = buf[y * C + f];
      }
      return;
    }
    for (int id = threadIdx.x; id < 2 * nl * C; id += blockDim.x) {
      const int y = fdiv(id, rC), f = id - y * C;
      reinterpret_cast<T2*>(base + (size_t)y * pitch)[f] = buf[id];
    }
  } else {
    if (tdata) {
      const float r2 = 1.f / (float)(2 * nl), rIy = 1.f / (float)Iy;
      for (int id = threadIdx.x; id < 2 * nl * C; id += blockDim.x) {
        const int f = fdiv(id, r2), y = id - f * 2 * nl;
        const int R = 2 * p0 + y, n = fdiv(R, rIy), yy = R - n * Iy;
        cp_async<sizeof(T2)>(buf + y * C + f,
                             tdata + (size_t)f * NR + (size_t)((n >> 1) + (n & 1) * np0) * Iy + yy);
      }
    } else {
      for (int id = threadIdx.x; id < 2 * nl * C; id += blockDim.x) {
        const int y = fdiv(id, rC), f = id - y * C;
        cp_async<sizeof(T2)>(buf + id, reinterpret_cast<const T2*>(base + (size_t)y * pitch) + f);
      }
    }
    cp_async_wait();
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
  T2* buf = reinterpret_cast<T2*>(tw + tw_len(n));
  load_tw(tw, twg + f.tw_off, tw_len(n));
  const int gpo = (Cn + B - 1) / B;
  const int o = blockIdx.x / gpo;
  const int c0 = (blockIdx.x - o * gpo) * B;
  const int nl = min(B, Cn - c0);
  T2* base = data + (size_t)o * os + c0;
  const float rl = 1.f / (float)nl;
  for (int id = threadIdx.x; id < nl * n; id += blockDim.x) {
    const int i = fdiv(id, rl), c = id - i * nl;
    cp_async<sizeof(T2)>(buf + id, base + (size_t)i * es + c);
  }
  cp_async_wait();
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

// ---------------------------------------------------------------------------
// Algorithm 2, z-contraction (Eq. 3.13 / 4.40 in the Chebyshev basis of the
// proxy planes), factorised over the long-range Gaussians l = m+1..M:
//   nu_n(k) = fx(kx) fy(ky) sum_l c1_l e^{-c2_l |k|^2} sum_n' B_l[n][n'] mu_n'(k)
// with B_l = C^T E_l C, E_l[c][c'] = e^{-(z_c - z_c')^2 / s_l^2}.  B_l[n][n']
// is zero when n + n' is odd (the proxy points are symmetric about z = 0),
// so orders of each parity form their own block (row stride pst, zero
// padded).  s_l grows with l: once c2_l |k|^2 > 80 that term and every later
// one is below e^-80 of the earlier ones, and the sum stops.  No per-mode
// matrix is stored.
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T dexp_(T x);
template <>
__device__ __forceinline__ float dexp_(float x) { return expf(x); }
template <>
__device__ __forceinline__ double dexp_(double x) { return exp(x); }

// t = sum_j B[j] v[j], j < np, for a B row padded with zeros to a multiple
// of four (the rows start 16-byte aligned): vector loads of four.
template <int PH>
__device__ __forceinline__ void brow_dot(const float* __restrict__ B, const float2 (&v)[PH], int np,
                                         float& tx, float& ty) {
  const float4* B4 = reinterpret_cast<const float4*>(B);
#pragma unroll
  for (int q = 0; q < PH / 4; ++q) {
    if (4 * q < np) {
      const float4 b = B4[q];
      tx = fmaf(b.x, v[4 * q].x, tx);
      ty = fmaf(b.x, v[4 * q].y, ty);
      tx = fmaf(b.y, v[4 * q + 1].x, tx);
      ty = fmaf(b.y, v[4 * q + 1].y, ty);
      tx = fmaf(b.z, v[4 * q + 2].x, tx);
      ty = fmaf(b.z, v[4 * q + 2].y, ty);
      tx = fmaf(b.w, v[4 * q + 3].x, tx);
      ty = fmaf(b.w, v[4 * q + 3].y, ty);
    }
  }
}
template <int PH>
__device__ __forceinline__ void brow_dot(const double* __restrict__ B, const double2 (&v)[PH],
                                         int np, double& tx, double& ty) {
#pragma unroll
  for (int j = 0; j < PH; ++j) {
    if (j < np) {
      tx = fma(B[j], v[j].x, tx);
      ty = fma(B[j], v[j].y, ty);
    }
  }
}

// One mode, one parity block: orders n = 2 i + par, i < np; get(i) returns
// mu_n, put(i, v) stores nu_n.  PH bounds np; the outputs are computed OH at
// a time (inputs held in registers, the exponentials recomputed per chunk).
template <typename T, int PH, int OH, typename GET, typename PUT>
__device__ __forceinline__ void long_contract_parity(GET get, PUT put, int np, int par, int ps,
                                                     int pst, int nl, const T* __restrict__ lbl,
                                                     const typename C2<T>::t* __restrict__ lcl,
                                                     T k2, T fac, T xmax) {
  using T2 = typename C2<T>::t;
  T2 v[PH];
#pragma unroll
  for (int i = 0; i < PH; ++i) v[i] = i < np ? get(i) : T2{T(0), T(0)};
#pragma unroll 1
  for (int i0 = 0; i0 < np; i0 += OH) {
    T2 acc[OH];
#pragma unroll
    for (int o = 0; o < OH; ++o) acc[o] = T2{T(0), T(0)};
#pragma unroll 1
    for (int l = 0; l < nl; ++l) {
      const T2 c = lcl[l];
      const T x = c.y * k2;
      if (x > xmax) break;
      const T a = fac * c.x * dexp_(-x);
      const T* B = lbl + ((size_t)l * 2 + par) * ps * pst + (size_t)i0 * pst;
#pragma unroll
      for (int o = 0; o < OH; ++o) {
        if (i0 + o < np) {
          T tx = T(0), ty = T(0);
          brow_dot<PH>(B + o * pst, v, np, tx, ty);
          acc[o].x = fma(a, tx, acc[o].x);
          acc[o].y = fma(a, ty, acc[o].y);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < OH; ++o)
      if (i0 + o < np) put(i0 + o, acc[o]);
  }
}

// Contraction in place on the half spectra of the P proxy planes (layout
// [n][y][c], plane stride Iy C complex): a thread per mode (y, c); the k = 0
// mode is zeroed (it is the separate FP64 step).
template <typename T, int PH>
__global__ void __launch_bounds__(128)
    k_long_contract(typename C2<T>::t* __restrict__ A, int P, int Iy, int C,
                    const T* __restrict__ lbl, const typename C2<T>::t* __restrict__ lcl,
                    const typename C2<T>::t* __restrict__ lfx,
                    const typename C2<T>::t* __restrict__ lfy, int nl, int ps, int pst, T xmax) {
  using T2 = typename C2<T>::t;
  const int mode = blockIdx.x * blockDim.x + threadIdx.x;
  if (mode >= Iy * C) return;
  const int y = mode / C, c = mode - y * C;
  const size_t pstr = (size_t)Iy * C;
  T2* a = A + mode;
  if (mode == 0) {
    for (int n = 0; n < P; ++n) a[n * pstr] = T2{T(0), T(0)};
    return;
  }
  const T2 fx = lfx[c], fy = lfy[y];
#pragma unroll 1
  for (int par = 0; par < 2; ++par)
    long_contract_parity<T, PH, PH>([&](int i) { return a[(2 * i + par) * pstr]; },
                                [&](int i, T2 v) { a[(2 * i + par) * pstr] = v; },
                                (P + 1 - par) / 2, par, ps, pst, nl, lbl, lcl, fx.x + fy.x,
                                fx.y * fy.y, xmax);
}

// Outputs of one contraction work item in the fused y pass.
constexpr int kYpassOut = 4;

// Fused y pass of Algorithm 2 for one half-spectrum column c and one parity
// par of the Chebyshev order (orders of different parity do not couple in the
// contraction): the np planes n = 2 i + par of the column (transposed layout
// [c][par][i][y], written by the x pass) are brought into shared memory by
// bulk copies, with this parity's B_l and (c1_l, c2_l) beside them; the np
// forward y FFTs run in one pass of the engine; the contraction runs in
// rounds, each over a range of modes y, one thread per (mode, chunk of
// kYpassOut orders), threads of a warp sharing a chunk so that their B_l
// reads are broadcasts; every round reads its modes' inputs, waits, then
// writes the outputs in place; then the backward y FFTs, and one bulk copy
// writes the block back.  A bulk copy that does not complete within the
// bounded wait sets bit 2 of *status and the CTA returns.
template <typename T, int PH>
__global__ void __launch_bounds__(kYpassThreads, 1)
    k_long_ypass(typename C2<T>::t* __restrict__ data, FftLen fy,
                 const typename C2<T>::tw* __restrict__ twg, int P,
                 const T* __restrict__ lbl, const typename C2<T>::t* __restrict__ lcl,
                 const typename C2<T>::t* __restrict__ lfx,
                 const typename C2<T>::t* __restrict__ lfy, int nl, int ps, int pst,
                 T xmax, int* __restrict__ status) {
  using T2 = typename C2<T>::t;
  using T4 = typename C2<T>::tw;
  constexpr int CAP = FftCfg<T>::cap;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int ynext;
  T2* buf = reinterpret_cast<T2*>(smraw);
  const int c = blockIdx.x >> 1, par = blockIdx.x & 1, Iy = fy.n;
  const int np0 = (P + 1) / 2, np = par ? P / 2 : np0;
  const int tot = np * Iy;
  T4* tw = reinterpret_cast<T4*>(buf + (size_t)np0 * Iy);
  T* sB = reinterpret_cast<T*>(tw + tw_len(Iy));      // [l][i][j], row stride pst
  T2* sC = reinterpret_cast<T2*>(sB + (size_t)nl * ps * pst);
  T2* blk = data + (size_t)c * P * Iy + (size_t)(par ? np0 : 0) * Iy;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    const unsigned bytes = (unsigned)(tot * sizeof(T2));
    mbar_expect_tx(&bar, bytes);
    for (unsigned o = 0; o < bytes; o += 32768u)
      bulk_g2s(reinterpret_cast<char*>(buf) + o, reinterpret_cast<const char*>(blk) + o,
               bytes - o < 32768u ? bytes - o : 32768u, &bar);
  }
  for (int i = threadIdx.x; i < tw_len(Iy); i += blockDim.x) tw[i] = twg[fy.tw_off + i];
  const int bsz = ps * pst;
  for (int i = threadIdx.x; i < nl * bsz; i += blockDim.x) {
    const int l = i / bsz;
    sB[i] = lbl[((size_t)l * 2 + par) * bsz + (i - l * bsz)];
  }
  for (int l = threadIdx.x; l < nl; l += blockDim.x) sC[l] = lcl[l];
  if (threadIdx.x == 0) ynext = 0;
  __syncthreads();
  if (!mbar_wait(&bar, 0)) {
    if (threadIdx.x == 0) atomicOr(status, 4);
    // the copy may still land in this CTA's shared memory: wait once more, bounded
    mbar_wait(&bar, 0);
    return;
  }
  const LineSet ls{Iy, np, Iy, 1, false};
  fft_lines<T2, CAP>(buf, ls, fy, tw, false);
  const T2 fx = lfx[c];
  // contraction: a warp takes a group of G modes at a time, its lanes over
  // (mode, chunk of kYpassOut orders); all reads and writes of a mode stay
  // inside one warp, so groups need no block-wide barrier.  Groups are
  // handed out in the order 0, last, 1, last - 1, ... (the modes of small
  // |k_y|, which keep the most Gaussians, first) from a shared counter.
  const int nsplit = (np + kYpassOut - 1) / kYpassOut;
  const int G = 32 / nsplit;
  const int lane = threadIdx.x & 31;
  const int ml = lane / nsplit, ch = lane - ml * nsplit, i0 = ch * kYpassOut;
  const int ngroups = (Iy + G - 1) / G;
  for (;;) {
    int gi = 0;
    if (lane == 0) gi = atomicAdd(&ynext, 1);
    gi = __shfl_sync(0xffffffffu, gi, 0);
    if (gi >= ngroups) break;
    const int grp = (gi & 1) ? ngroups - 1 - (gi >> 1) : (gi >> 1);
    const int y = grp * G + ml;
    const bool act = ml < G && y < Iy;
    T2 acc[kYpassOut];
#pragma unroll
    for (int o = 0; o < kYpassOut; ++o) acc[o] = T2{T(0), T(0)};
    if (act && !(c == 0 && y == 0)) {
      const T2* a = buf + y;
      T2 v[PH];
#pragma unroll
      for (int i = 0; i < PH; ++i) v[i] = i < np ? a[i * Iy] : T2{T(0), T(0)};
      const T2 fyv = lfy[y];
      const T k2 = fx.x + fyv.x, fac = fx.y * fyv.y;
#pragma unroll 1
      for (int l = 0; l < nl; ++l) {
        const T2 cl = sC[l];
        const T xx = cl.y * k2;
        if (xx > xmax) break;
        const T al = fac * cl.x * dexp_(-xx);
        const T* B = sB + (size_t)l * bsz + (size_t)i0 * pst;
#pragma unroll
        for (int o = 0; o < kYpassOut; ++o) {
          if (i0 + o < np) {
            T tx = T(0), ty = T(0);
            brow_dot<PH>(B + o * pst, v, np, tx, ty);
            acc[o].x = fma(al, tx, acc[o].x);
            acc[o].y = fma(al, ty, acc[o].y);
          }
        }
      }
    }
    __syncwarp();  // every input of this group's modes has been read
    if (act) {
#pragma unroll
      for (int o = 0; o < kYpassOut; ++o)
        if (i0 + o < np) buf[(size_t)(i0 + o) * Iy + y] = acc[o];
    }
    __syncwarp();
  }
  __syncthreads();
  fft_lines<T2, CAP>(buf, ls, fy, tw, true);
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) bulk_s2g_wait(blk, buf, (unsigned)(tot * sizeof(T2)));
}

// True when a whole Ix x Iy plane fits one CTA of k_fft_plane with nt
// threads.
template <typename T>
static bool plane_fits(const FftLen& fx, const FftLen& fy, int nt = FftCfg<T>::threads) {
  constexpr int CAP = FftCfg<T>::cap;
  const int C = fx.n / 2 + 1;
  const size_t smem = (size_t)(tw_len(fx.n) + tw_len(fy.n)) * sizeof(typename C2<T>::tw) +
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
  const size_t sm = (size_t)(tw_len(fx.n) + tw_len(fy.n)) * sizeof(T4) +
                    (size_t)std::max((fy.n / 2) * fx.n, fy.n * C) * sizeof(T2);
  k_fft_plane<T><<<nplanes, plane_threads<T>(fx, fy), sm, s>>>(data, fx, fy,
                                                                reinterpret_cast<const T4*>(tw),
                                                  inv);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_rows(T* data, const FftLen& fx, const void* tw, int nrows, bool inv,
                               cudaStream_t s, typename C2<T>::t* tdata = nullptr, int Iy = 1,
                               int np0 = 0) {
  using T2 = typename C2<T>::t;
  constexpr int CAP = FftCfg<T>::cap;
  const int npairs = nrows / 2;
  const int C = fx.n / 2 + 1;
  constexpr int NT = FftCfg<T>::threads;
  int B = std::min(max_lines(fx, CAP, NT), NT * (CAP / 2) / C);
  B = std::max(1, std::min(B, npairs));
  using T4 = typename C2<T>::tw;
  const size_t sm =
      (size_t)tw_len(fx.n) * sizeof(T4) + (size_t)B * std::max(fx.n, 2 * C) * sizeof(T2);
  const int grid = (npairs + B - 1) / B;
  k_fft_rows<T><<<grid, NT, sm, s>>>(data, fx, reinterpret_cast<const T4*>(tw), npairs,
                                              B, inv, tdata, (long)nrows, Iy, np0);
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
  const size_t sm = (size_t)tw_len(f.n) * sizeof(T4) + (size_t)B * f.n * sizeof(T2);
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

// Shared memory of the fused y pass: one parity block of a column, the y
// twiddles, one parity's B_l for the nl Gaussians a mode can use, (c1, c2).
size_t long_fused_smem(int P, const FftLen& fy, int nl, size_t es) {
  const int np0 = (P + 1) / 2, ps = np0, pst = (ps + 3) / 4 * 4;
  return (size_t)np0 * fy.n * 2 * es +
         (size_t)tw_len(fy.n) * (es == 4 ? sizeof(TwF) : sizeof(TwD)) +
         (size_t)nl * ps * pst * es + (size_t)nl * 2 * es;
}

// FP32 plans: the fused y pass's shared memory must fit one CTA, the block's
// lines one pass of the engine, and the block the register budget
// (P <= 32).  FP64 plans use the separate passes.
bool long_fused_fits(int P, const FftLen& fy, int nl, size_t es) {
  const int np0 = (P + 1) / 2;
  return es == sizeof(float) && P <= 32 && long_fused_smem(P, fy, nl, es) + 64 <= (size_t)kMaxDynSmem &&
         max_lines(fy, FftCfg<float>::cap, kYpassThreads) >= np0;
}

template <typename T, int PH>
static void launch_contract(const sog_plan* p, T* A, cudaStream_t s) {
  using T2 = typename C2<T>::t;
  const int P = p->prm.P_cheb, Iy = p->prm.I_long[1], C = p->prm.I_long[0] / 2 + 1;
  const int modes = Iy * C;
  k_long_contract<T, PH><<<(modes + 127) / 128, 128, 0, s>>>(
      reinterpret_cast<T2*>(A), P, Iy, C, reinterpret_cast<const T*>(p->d_lbl),
      reinterpret_cast<const T2*>(p->d_lcl), reinterpret_cast<const T2*>(p->d_lfx),
      reinterpret_cast<const T2*>(p->d_lfy), p->n_lg_used, p->lps, p->lpst, (T)p->lg_xmax);
}

template <typename T, int PH>
static void launch_ypass(const sog_plan* p, typename C2<T>::t* col, cudaStream_t s) {
  using T2 = typename C2<T>::t;
  using T4 = typename C2<T>::tw;
  const int P = p->prm.P_cheb, C = p->prm.I_long[0] / 2 + 1;
  const size_t sm = long_fused_smem(P, p->fly, p->n_lg_used, sizeof(T));
  k_long_ypass<T, PH><<<2 * C, kYpassThreads, sm, s>>>(
      col, p->fly, reinterpret_cast<const T4*>(p->d_tw), P,
      reinterpret_cast<const T*>(p->d_lbl), reinterpret_cast<const T2*>(p->d_lcl),
      reinterpret_cast<const T2*>(p->d_lfx), reinterpret_cast<const T2*>(p->d_lfy), p->n_lg_used,
      p->lps, p->lpst, (T)p->lg_xmax, p->d_status);
}

// Algorithm 2 steps 2-4 on the proxy planes in d_lA.  Fused: x pass with the
// half spectrum written transposed to d_lB, the y pass / contraction /
// backward y pass per column, backward x pass back into d_lA.  Otherwise:
// forward 2D FFTs, the contraction kernel and backward 2D FFTs, in place.
template <typename T>
cudaError_t fft_long_solve(const sog_plan* p, cudaStream_t s, int& launches) {
  using T2 = typename C2<T>::t;
  T* A = reinterpret_cast<T*>(p->d_lA);
  const int P = p->prm.P_cheb, Iy = p->prm.I_long[1];
  const int ph = (P + 1) / 2;
  cudaError_t e;
  if constexpr (sizeof(T) == 4) if (p->long_fused) {
    T2* col = reinterpret_cast<T2*>(p->d_lB);
    if ((e = launch_rows<T>(A, p->flx, p->d_tw, Iy * P, false, s, col, Iy, ph))) return e;
    if (ph <= 4) launch_ypass<T, 4>(p, col, s);
    else if (ph <= 8) launch_ypass<T, 8>(p, col, s);
    else if (ph <= 12) launch_ypass<T, 12>(p, col, s);
    else launch_ypass<T, 16>(p, col, s);
    if ((e = cudaGetLastError())) return e;
    if ((e = launch_rows<T>(A, p->flx, p->d_tw, Iy * P, true, s, col, Iy, ph))) return e;
    launches += 3;
    return cudaSuccess;
  }
  if ((e = fft_planes<T>(A, p->flx, p->fly, p->d_tw, P, false, s, launches))) return e;
  if (ph <= 4) launch_contract<T, 4>(p, A, s);
  else if (ph <= 8) launch_contract<T, 8>(p, A, s);
  else if (ph <= 12) launch_contract<T, 12>(p, A, s);
  else if (ph <= 16) launch_contract<T, 16>(p, A, s);
  else launch_contract<T, 32>(p, A, s);
  if ((e = cudaGetLastError())) return e;
  launches += 1;
  return fft_planes<T>(A, p->flx, p->fly, p->d_tw, P, true, s, launches);
}
template cudaError_t fft_long_solve<float>(const sog_plan*, cudaStream_t, int&);
template cudaError_t fft_long_solve<double>(const sog_plan*, cudaStream_t, int&);

// True when transforms of this length fit the engine (at least one line per
// CTA; the x pass also needs its half spectrum to fit one CTA).
bool fft_len_ok(int prec, const FftLen& f) {
  const int cap = prec == SOG_PREC_FP64 ? FftCfg<double>::cap : FftCfg<float>::cap;
  const int nt = prec == SOG_PREC_FP64 ? FftCfg<double>::threads : FftCfg<float>::threads;
  const size_t elem = prec == SOG_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t twe = prec == SOG_PREC_FP64 ? sizeof(TwD) : sizeof(TwF);
  return f.n >= 2 && max_lines(f, cap, nt) >= 1 && (f.n / 2 + 1) <= nt * (cap / 2) &&
         (size_t)tw_len(f.n) * twe + (size_t)(f.n + 2) * elem <= (size_t)kMaxDynSmem;
}

// The largest dynamic shared memory a kernel's static shared memory leaves.
template <typename K>
static cudaError_t allow_dyn_smem(K* kernel) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kMaxDynSmem - (int)a.sharedSizeBytes);
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
  if constexpr (sizeof(T) == 4) {
    // the y pass holds its mbarrier in static shared memory
    if (e == cudaSuccess) e = allow_dyn_smem(k_long_ypass<T, 4>);
    if (e == cudaSuccess) e = allow_dyn_smem(k_long_ypass<T, 8>);
    if (e == cudaSuccess) e = allow_dyn_smem(k_long_ypass<T, 12>);
    if (e == cudaSuccess) e = allow_dyn_smem(k_long_ypass<T, 16>);
  }
  return e;
}
template cudaError_t fft_prepare<float>();
template cudaError_t fft_prepare<double>();

}  // namespace sogk
