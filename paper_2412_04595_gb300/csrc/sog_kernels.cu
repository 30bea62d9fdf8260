// Device kernels of the spectral SOG method and the host code that enqueues them.
//
// One evaluation (sog_eval) runs, on one stream:
//   1. binning: every particle gets a near-field cell (cells >= r_c, Sec. 2.2
//      cell list), a mid-grid tile and a long-grid tile; three counting sorts
//      produce cell-/tile-sorted particle records;
//   2. near field Phi^N (Eq. 2.28) over the 27 neighbouring cells, kernel
//      1/r - F_M(r) from a piecewise-polynomial table (Remark 2.4);
//   3. mid range, Algorithm 1: gridding (Eq. 3.7) tile by tile in shared
//      memory, FFT / scaling (Eq. 3.8) / inverse FFT, gathering (Eq. 3.10)
//      with the window gradient for the forces;
//   4. long range, Algorithm 2 (anterpolation form): charges times the
//      Chebyshev polynomials T_n(2z/Lz) spread in x,y onto P proxy planes,
//      2D FFTs, per-mode z-contraction with the kernel of Eq. 3.13 / 4.40
//      written in the Chebyshev basis, inverse 2D FFTs, gathering with
//      T_n(2 z_i/Lz) (and T_n' for the z force);
//   5. the k = 0 mode of the long range in FP64 from exact Chebyshev moments;
//   6. assembly Phi = sum of parts - q sum_l w_l (Eq. 3.22, 2.28), forces,
//      energy U = 1/2 sum q Phi reduced in FP64 in a fixed order.
// The element type T is float (mixed precision) or double (FP64).
#include <math.h>

#include <cmath>

#include "sog_internal.h"

namespace sogk {

// ---------------------------------------------------------------------------
// geometry passed to the kernels
// ---------------------------------------------------------------------------

struct PrepGeom {
  double L[3], halfL[3];
  int nc[3];
  double icell[3];   // 1 / cell edge
  int has_mid, has_long;
  double ih[3], Lzs_half;  // 1 / mid grid spacing
  int Tm[3], ntm[3];
  double iTm[3];
  double ihl[2];     // 1 / long grid spacing
  double h[3], hl[2];  // grid spacings (FP64 plans divide by them, as the oracle does)
  int Tl[2], ntl[2];
  double iTl[2];
  double ihalfLz;
  // FP32 plans: the same quantities for arithmetic in float pairs (value
  // rounded to float, plus the rounding error), and float thresholds that
  // decide the comparisons with the FP64 half box lengths exactly
  float wrap_hi[2], wrap_lo[2];  // c >= L/2  <=>  c >= wrap_hi;  c < -L/2  <=>  c < wrap_lo
  float z_lo, z_hi;              // -Lz/2 <= z <= Lz/2  <=>  z_lo <= z <= z_hi
  float halfLf[3];               // L/2 rounded (clamp values)
  float2 halfLp[3], icellp[3], ihp[3], Lzs_halfp, iTmp[3], ihlp[2], iTlp[2], ihalfLzp;
};

// Float pairs: value h plus error l (|l| <= ulp(h) / 2).
struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_fast2(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return FF{s, b - (s - a)};
}
// c + H exactly up to the rounding of H's pair
__device__ __forceinline__ FF ff_add(float c, float2 H) {
  const float s = c + H.x;
  const float bb = s - c;
  const float e = (c - (s - bb)) + (H.x - bb);
  return ff_fast2(s, e + H.y);
}
__device__ __forceinline__ FF ff_mul(FF a, float2 b) {
  const float p = a.h * b.x;
  float e = fmaf(a.h, b.x, -p);
  e = fmaf(a.h, b.y, e);
  e = fmaf(a.l, b.x, e);
  return ff_fast2(p, e);
}
// floor(a.h + a.l) clamped to [0, n - 1] (0 for NaN)
__device__ __forceinline__ int ff_floor_clamp(FF a, int n) {
  if (!(a.h >= 0.0f)) return 0;
  float k = floorf(a.h);
  if (k == a.h && a.l < 0.0f) k -= 1.0f;
  if (k >= (float)n) return n - 1;
  return k < 0.0f ? 0 : (int)k;
}
// (a.h + a.l) - k m rounded once (k m exact: both small integers)
__device__ __forceinline__ float ff_sub_int(FF a, int k, int m) { return (a.h - (float)(k * m)) + a.l; }

// KB: I0(beta sqrt(1 - v^2)) / I0(beta) = sum_k kbc[k] u^k, u = 1 - v^2, from
// the power series of I0 (kbc[k] = (beta^2/4)^k / (k!)^2 / I0(beta); all
// terms positive, so Horner in u in [0, 1] is accurate in FP32 too).
constexpr int kKbTerms = 64;
template <typename T>
struct WinT {
  int P, kind;
  T half, inv_half, shape;
  int kbn;           // KB: number of series terms
  T kbc[kKbTerms];   // KB: series coefficients for the rounded shape
  int nu;            // > 0: polynomial windows of this degree
  T pc[kMaxWin * (kPolyMax + 1)];  // their monomial coefficients [d][j] (win_poly_coeffs)
};

template <typename T>
__host__ WinT<T> wint(const WinPar& w) {
  WinT<T> o;
  o.P = w.P;
  o.kind = w.kind;
  o.half = (T)w.half;
  o.inv_half = (T)(1.0 / w.half);
  o.shape = (T)w.shape;
  o.kbn = 0;
  for (int k = 0; k < kKbTerms; ++k) o.kbc[k] = T(0);
  if (w.kind == SOG_WIN_KB) o.kbn = kb_series<T>((double)o.shape, o.kbc, kKbTerms);
  o.nu = w.nu;
  double a[kMaxWin * (kPolyMax + 1)] = {};
  if (w.nu > 0) win_poly_coeffs(w, a);
  for (int i = 0; i < kMaxWin * (kPolyMax + 1); ++i) o.pc[i] = (T)a[i];
  return o;
}

// Window argument v = offset / half-width: FP64 divides (bit for bit the
// oracle's value), FP32 multiplies by the rounded reciprocal.
template <typename T>
__device__ __forceinline__ T win_arg(T d, const WinT<T>& w) {
  if constexpr (sizeof(T) == 8) return d / w.half;
  else return d * w.inv_half;
}

__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dceil(float x) { return ceilf(x); }
__device__ __forceinline__ double dceil(double x) { return ceil(x); }
__device__ __forceinline__ float drint(float x) { return rintf(x); }
__device__ __forceinline__ double drint(double x) { return rint(x); }
__device__ __forceinline__ float drsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double drsqrt(double x) { return rsqrt(x); }

// Window phi(v) (v = offset / half-width) and d phi / dv; zero outside |v| <= 1.
// KB: whether the Kaiser-Bessel branch is compiled in (only the kernels for a
// run-time support take it, so that the fixed-support kernels of the ES and
// Gaussian windows keep their code).
template <typename T, bool KB>
__device__ __forceinline__ void win_eval(const WinT<T>& w, T v, T& val, T& dval) {
  const T one = T(1);
  val = T(0);
  dval = T(0);
  if (!(v >= -one && v <= one)) return;
  if (w.kind == SOG_WIN_ES) {
    // beta (sqrt(1 - v^2) - 1) written as -beta v^2 / (1 + sqrt(1 - v^2)):
    // no cancellation near the window centre, where the weights are largest
    const T a2 = (one - v) * (one + v);
    const T a = dsqrt(a2);
    val = dexp(-w.shape * (v * v / (one + a)));
    if (a2 > T(0)) dval = -val * w.shape * v * drsqrt(a2);
  } else if (KB && w.kind == SOG_WIN_KB) {
    // series in u = 1 - v^2 and its u-derivative by Horner; d/dv = -2 v d/du
    const T u = (one - v) * (one + v);
    T p = w.kbc[w.kbn - 1], dp = T(0);
    for (int k = w.kbn - 2; k >= 0; --k) {
      dp = dp * u + p;
      p = p * u + w.kbc[k];
    }
    val = p;
    dval = T(-2) * v * dp;
  } else {
    val = dexp(-w.shape * v * v);
    dval = T(-2) * w.shape * v * val;
  }
}

// A complex number (or a pair of values) in the element type.
template <typename T>
struct alignas(2 * sizeof(T)) Cx {
  T x, y;
};
template <typename T>
__device__ __forceinline__ Cx<T> cxmul(Cx<T> a, Cx<T> b) {
  return Cx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Window value only (same arithmetic as win_eval's value).
template <typename T, bool KB>
__device__ __forceinline__ T win_val(const WinT<T>& w, T v) {
  const T one = T(1);
  if (!(v >= -one && v <= one)) return T(0);
  if (w.kind == SOG_WIN_ES) {
    const T a2 = (one - v) * (one + v);
    return dexp(-w.shape * (v * v / (one + dsqrt(a2))));
  }
  if (KB && w.kind == SOG_WIN_KB) {
    const T u = (one - v) * (one + v);
    T p = w.kbc[w.kbn - 1];
    for (int k = w.kbn - 2; k >= 0; --k) p = p * u + w.kbc[k];
    return p;
  }
  return dexp(-w.shape * v * v);
}

// Window weight of support point k of a particle at grid coordinate c
// (g0 = ceil(c - half)) and d phi / dv: directly at v = (g0 + k - c) / half,
// or, for polynomial windows, by Horner in sigma = 2 (g0 - c) + P - 2 (the
// same number as 2 (g0 - c + half) - 1, exact in both types) on point k's
// coefficients; d phi / dv = 2 half d p / d sigma.
template <typename T>
__device__ __forceinline__ T win_sigma(int g0, T c, const WinT<T>& w) {
  return T(2) * ((T)g0 - c) + (T)(w.P - 2);
}
template <typename T, bool KB>
__device__ __forceinline__ void win_eval_pt(const WinT<T>& w, int g0, T c, int k, T& val, T& dval) {
  if (w.nu > 0) {
    const T sg = win_sigma(g0, c, w);
    const T* a = w.pc + k * (kPolyMax + 1);
    T p = a[w.nu], dp = T(0);
    for (int j = w.nu - 1; j >= 0; --j) {
      dp = dp * sg + p;
      p = p * sg + a[j];
    }
    val = p;
    dval = (T)(w.P - 1) * dp;
    return;
  }
  win_eval<T, KB>(w, win_arg(((T)(g0 + k) - c), w), val, dval);
}
template <typename T, bool KB>
__device__ __forceinline__ T win_val_pt(const WinT<T>& w, int g0, T c, int k) {
  if (w.nu > 0) {
    const T sg = win_sigma(g0, c, w);
    const T* a = w.pc + k * (kPolyMax + 1);
    T p = a[w.nu];
    for (int j = w.nu - 1; j >= 0; --j) p = p * sg + a[j];
    return p;
  }
  return win_val<T, KB>(w, win_arg(((T)(g0 + k) - c), w));
}

// ---------------------------------------------------------------------------
// 1. binning
// ---------------------------------------------------------------------------


__device__ __forceinline__ int floor_clamp(double t, int n) {
  if (!(t >= 0.0)) return 0;  // also NaN
  if (t >= (double)n) return n - 1;
  return (int)t;
}

// FP32 plans: prep_particle in float and float-pair arithmetic (the FP64
// pipe of this GPU is slow): the wrap and range decisions are exact, bins
// follow the rounded pair sums, and the tile-local coordinates carry one
// rounding, as when they are computed in FP64 and rounded.
__device__ void prep_particle_f(const PrepGeom& g, const float* __restrict__ q,
                                const float* __restrict__ r, int i, int& bits, P4<float>& rn,
                                int& kn, int& km, P4<float>& rm, int& kl, P4<float>& rl) {
  float c[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]};
  float qi = q[i];
  for (int d = 0; d < 2; ++d) {
    const float Ld = (float)g.L[d];
    if (c[d] >= g.wrap_hi[d]) c[d] = c[d] - Ld;
    else if (c[d] < g.wrap_lo[d]) c[d] = c[d] + Ld;
    if (!(c[d] >= g.wrap_lo[d] && c[d] < g.wrap_hi[d])) {
      bits |= 2;
      c[d] = isfinite(c[d]) ? (c[d] < 0.0f ? -g.halfLf[d] : 0.0f) : 0.0f;
    }
  }
  if (!(c[2] >= g.z_lo && c[2] <= g.z_hi)) {
    bits |= 2;
    c[2] = isfinite(c[2]) ? (c[2] < 0.0f ? -g.halfLf[2] : g.halfLf[2]) : 0.0f;
  }
  if (!isfinite(qi)) {
    bits |= 2;
    qi = 0.0f;
  }
  rn = P4<float>{c[0], c[1], c[2], qi};
  FF s[3];
  int cc[3];
  for (int d = 0; d < 3; ++d) {
    s[d] = ff_add(c[d], g.halfLp[d]);
    cc[d] = ff_floor_clamp(ff_mul(s[d], g.icellp[d]), g.nc[d]);
  }
  kn = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
  km = 0;
  kl = 0;
  if (g.has_mid) {
    FF t[3];
    t[0] = ff_mul(s[0], g.ihp[0]);
    t[1] = ff_mul(s[1], g.ihp[1]);
    t[2] = ff_mul(ff_add(c[2], g.Lzs_halfp), g.ihp[2]);
    int tt[3];
    float loc[3];
    for (int d = 0; d < 3; ++d) {
      tt[d] = ff_floor_clamp(ff_mul(t[d], g.iTmp[d]), g.ntm[d]);
      loc[d] = ff_sub_int(t[d], tt[d], g.Tm[d]);
    }
    km = (tt[2] * g.ntm[1] + tt[1]) * g.ntm[0] + tt[0];
    rm = P4<float>{loc[0], loc[1], loc[2], qi};
  }
  if (g.has_long) {
    FF t[2];
    int tt[2];
    float loc[2];
    for (int d = 0; d < 2; ++d) {
      t[d] = ff_mul(s[d], g.ihlp[d]);
      tt[d] = ff_floor_clamp(ff_mul(t[d], g.iTlp[d]), g.ntl[d]);
      loc[d] = ff_sub_int(t[d], tt[d], g.Tl[d]);
    }
    kl = tt[1] * g.ntl[0] + tt[0];
    const FF zz = ff_mul(FF{c[2], 0.0f}, g.ihalfLzp);
    rl = P4<float>{loc[0], loc[1], zz.h + zz.l, qi};
  }
}

// Wrap / clamp one particle and compute its bins and tile-local records.
template <typename T>
__device__ void prep_particle(const PrepGeom& g, const T* __restrict__ q, const T* __restrict__ r,
                              int i, int& bits, P4<T>& rn, int& kn, int& km, P4<T>& rm, int& kl,
                              P4<T>& rl) {
  if constexpr (sizeof(T) == 4) {
    prep_particle_f(g, q, r, i, bits, rn, kn, km, rm, kl, rl);
    return;
  }
  T x = r[3 * i], y = r[3 * i + 1], z = r[3 * i + 2], qi = q[i];
  T c[3] = {x, y, z};
  for (int d = 0; d < 2; ++d) {
    const T Ld = (T)g.L[d];
    if ((double)c[d] >= g.halfL[d]) c[d] = c[d] - Ld;
    else if ((double)c[d] < -g.halfL[d]) c[d] = c[d] + Ld;
    if (!((double)c[d] >= -g.halfL[d] && (double)c[d] < g.halfL[d])) {
      bits |= 2;
      c[d] = isfinite((double)c[d]) ? ((double)c[d] < 0 ? (T)(-g.halfL[d]) : (T)0) : (T)0;
    }
  }
  if (!((double)c[2] >= -g.halfL[2] && (double)c[2] <= g.halfL[2])) {
    bits |= 2;
    c[2] = isfinite((double)c[2]) ? ((double)c[2] < 0 ? (T)(-g.halfL[2]) : (T)(g.halfL[2])) : (T)0;
  }
  if (!isfinite((double)qi)) {
    bits |= 2;
    qi = (T)0;
  }
  rn = P4<T>{c[0], c[1], c[2], qi};
  // near-field cell (cells of edge >= r_c; z cells clamp at the open walls)
  int cc[3];
  for (int d = 0; d < 3; ++d) cc[d] = floor_clamp(((double)c[d] + g.halfL[d]) * g.icell[d], g.nc[d]);
  kn = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
  km = 0;
  kl = 0;
  if (g.has_mid) {
    double t[3];
    // grid coordinates by IEEE division: a particle on a grid line gets
    // exactly the coordinate the FP64 oracle computes (the ES window's
    // derivative is unbounded at its support edge, so the last bit matters)
    t[0] = ((double)c[0] + g.halfL[0]) / g.h[0];
    t[1] = ((double)c[1] + g.halfL[1]) / g.h[1];
    t[2] = ((double)c[2] + g.Lzs_half) / g.h[2];
    int tt[3];
    double loc[3];
    for (int d = 0; d < 3; ++d) {
      tt[d] = floor_clamp(t[d] * g.iTm[d], g.ntm[d]);
      loc[d] = t[d] - (double)tt[d] * g.Tm[d];
    }
    km = (tt[2] * g.ntm[1] + tt[1]) * g.ntm[0] + tt[0];
    rm = P4<T>{(T)loc[0], (T)loc[1], (T)loc[2], qi};
  }
  if (g.has_long) {
    double t[2];
    t[0] = ((double)c[0] + g.halfL[0]) / g.hl[0];
    t[1] = ((double)c[1] + g.halfL[1]) / g.hl[1];
    int tt[2];
    double loc[2];
    for (int d = 0; d < 2; ++d) {
      tt[d] = floor_clamp(t[d] * g.iTl[d], g.ntl[d]);
      loc[d] = t[d] - (double)tt[d] * g.Tl[d];
    }
    kl = tt[1] * g.ntl[0] + tt[0];
    rl = P4<T>{(T)loc[0], (T)loc[1], (T)((double)c[2] * g.ihalfLz), qi};
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of four values over the warp by halving exchanges (6 shuffles instead
// of 20): on return lanes 0-7 hold the sum of a, 8-15 of b, 16-23 of c,
// 24-31 of d.
template <typename T>
__device__ __forceinline__ T warp_sum4(T a, T b, T c, T d) {
  const int lane = threadIdx.x & 31;
  const bool hi16 = lane & 16, hi8 = lane & 8;
  T k0 = hi16 ? c : a, k1 = hi16 ? d : b;
  k0 += __shfl_xor_sync(0xffffffffu, hi16 ? a : c, 16);
  k1 += __shfl_xor_sync(0xffffffffu, hi16 ? b : d, 16);
  T k = hi8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

// Per-particle results (potential and three gradient components) of up to
// 8 particles of a warp, held one per lane: lane 8 v + s keeps value v of
// the particle in slot s.  Writing them out in FP64 then costs one
// conversion for 8 particles (a warp-wide FP64 instruction occupies the FP64
// pipe for many cycles however few lanes are active).
template <typename T>
struct OutSlots {
  T val;
  int o, n;
  // tot: value (lane >> 3) of the current particle, as left by warp_sum4
  __device__ __forceinline__ void put(T tot, int out_index) {
    if (((threadIdx.x & 31) & 7) == n) {
      val = tot;
      o = out_index;
    }
    ++n;
  }
  // add: accumulate into the outputs instead of overwriting them
  __device__ __forceinline__ void flush(double* __restrict__ phi, double* __restrict__ grad,
                                        bool add) {
    const int lane = threadIdx.x & 31, which = lane >> 3;
    if ((lane & 7) < n) {
      double* dst = which == 0 ? phi + o : grad + 3 * (size_t)o + which - 1;
      if (add) *dst += (double)val;
      else *dst = (double)val;
    }
    n = 0;
  }
};

// Block-wide sum of a double; result valid in thread 0.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

template <typename T>
__global__ void k_bin_count(PrepGeom g, const T* __restrict__ q, const T* __restrict__ r, int N,
                            int* __restrict__ key, int* __restrict__ rank, int* __restrict__ cnt,
                            int3 off, P4<T>* __restrict__ tmp, double* __restrict__ red,
                            int* __restrict__ status) {
  __shared__ double2 sh2[256];
  double sq = 0.0, sa = 0.0;
  int bits = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    P4<T> rn, rm, rl;
    int kn, km, kl;
    prep_particle<T>(g, q, r, i, bits, rn, kn, km, rm, kl, rl);
    // ranks in the three binnings: the atomics of all three are issued
    // before any result is used, so their latencies overlap
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const unsigned pn = __match_any_sync(act, kn);
    const unsigned pm = g.has_mid ? __match_any_sync(act, km) : 0u;
    const unsigned pl = g.has_long ? __match_any_sync(act, kl) : 0u;
    const int ln = __ffs(pn) - 1, lm = __ffs(pm) - 1, ll = __ffs(pl) - 1;
    int bn = 0, bm = 0, bl = 0;
    if (lane == ln) bn = atomicAdd(cnt + off.x + kn, __popc(pn));
    if (g.has_mid && lane == lm) bm = atomicAdd(cnt + off.y + km, __popc(pm));
    if (g.has_long && lane == ll) bl = atomicAdd(cnt + off.z + kl, __popc(pl));
    key[i] = kn;
    tmp[i] = rn;
    rank[i] = __shfl_sync(pn, bn, ln) + __popc(pn & below);
    if (g.has_mid) {
      key[N + i] = km;
      tmp[N + i] = rm;
      rank[N + i] = __shfl_sync(pm, bm, lm) + __popc(pm & below);
    }
    if (g.has_long) {
      key[2 * N + i] = kl;
      tmp[2 * N + i] = rl;
      rank[2 * N + i] = __shfl_sync(pl, bl, ll) + __popc(pl & below);
    }
    sq += (double)rn.q;
    sa += fabs((double)rn.q);
  }
  if (bits) atomicOr(status, bits);
  // block sums of q and |q| in a fixed order: warp 0 adds the threads'
  // values from shared memory (few warp-wide FP64 instructions)
  sh2[threadIdx.x] = make_double2(sq, sa);
  __syncthreads();
  if (threadIdx.x < 32) {
    double tq = 0.0, ta = 0.0;
    for (int k = threadIdx.x; k < (int)blockDim.x; k += 32) {
      tq += sh2[k].x;
      ta += sh2[k].y;
    }
    tq = warp_sum(tq);
    ta = warp_sum(ta);
    if (threadIdx.x == 0) {
      red[2 * blockIdx.x] = tq;
      red[2 * blockIdx.x + 1] = ta;
    }
  }
}

// Exclusive scan of three count arrays (one CTA each): cnt[off + k] for
// k < n becomes the start of bin k, cnt[off + n] the total.
__global__ void k_scan3(int* __restrict__ cnt, int3 off, int3 nbins) {
  // each thread takes kScanItems consecutive counts per round (their loads
  // in flight together), scans them serially; the threads' totals are
  // scanned across the block and carried from round to round
  constexpr int kScanItems = 8;
  const int which = blockIdx.x;
  const int o = which == 0 ? off.x : (which == 1 ? off.y : off.z);
  const int n = which == 0 ? nbins.x : (which == 1 ? nbins.y : nbins.z);
  if (n <= 0) return;
  int* a = cnt + o;
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base <= n; base += (int)blockDim.x * kScanItems) {
    const int i0 = base + (int)threadIdx.x * kScanItems;
    int v[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = (i0 + k < n) ? a[i0 + k] : 0;
    int tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const int t = v[k];
      v[k] = tsum;
      tsum += t;
    }
    int x = tsum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int sw = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, sw, d);
        if (lane >= d) sw += y;
      }
      wsum[lane] = sw;
    }
    __syncthreads();
    const int excl = carry + (wid > 0 ? wsum[wid - 1] : 0) + x - tsum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
      if (i0 + k <= n) a[i0 + k] = excl + v[k];
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + tsum;
    __syncthreads();
  }
}

template <typename T>
__global__ void k_bin_scatter(int N, int has_mid, int has_long, const int* __restrict__ key,
                              const int* __restrict__ rank, const int* __restrict__ cnt, int3 off,
                              const P4<T>* __restrict__ tmp, P4<T>* __restrict__ rec_n,
                              P4<T>* __restrict__ rec_m, P4<T>* __restrict__ rec_l,
                              int* __restrict__ perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int pos = cnt[off.x + key[i]] + rank[i];
    rec_n[pos] = tmp[i];
    perm[pos] = i;
    if (has_mid) {
      pos = cnt[off.y + key[N + i]] + rank[N + i];
      rec_m[pos] = tmp[N + i];
      perm[N + pos] = i;
    }
    if (has_long) {
      pos = cnt[off.z + key[2 * N + i]] + rank[2 * N + i];
      rec_l[pos] = tmp[2 * N + i];
      perm[2 * N + pos] = i;
    }
  }
}

// ---------------------------------------------------------------------------
// 2. near field
// ---------------------------------------------------------------------------

struct NearGeom {
  double halfL[3];
  double cell[3];
  int nc[3];
  double L[2];
  double rc;
  int K, D;
  // per-launch constants in both element types (no FP64 work per thread):
  // r_c^2, table interval h_K and 1/h_K, Lx, Ly, 1/Lx, 1/Ly, Lx/2, Ly/2
  float cf[9];
  double cd[9];
};
enum { kNcRc2, kNcHK, kNcIhK, kNcLx, kNcLy, kNcILx, kNcILy, kNcHLx, kNcHLy };
template <typename T>
__device__ __forceinline__ T near_const(const NearGeom& g, int i) {
  if constexpr (sizeof(T) == 4) return g.cf[i];
  else return g.cd[i];
}
// The same constants computed as the kernels would in the element type.
template <typename T>
__host__ void near_consts(NearGeom& g, T* out) {
  const T rc = (T)g.rc;
  out[kNcRc2] = rc * rc;
  out[kNcHK] = rc / (T)g.K;
  out[kNcIhK] = (T)g.K / rc;
  out[kNcLx] = (T)g.L[0];
  out[kNcLy] = (T)g.L[1];
  out[kNcILx] = (T)(1.0 / g.L[0]);
  out[kNcILy] = (T)(1.0 / g.L[1]);
  out[kNcHLx] = (T)g.halfL[0];
  out[kNcHLy] = (T)g.halfL[1];
}

// Compensated accumulation for the FP32 path: the near-field sum
// adds ~100 terms whose largest (1/r of a close pair) sets the rounding of
// every later addition; the compensation keeps the sum at one rounding.
template <typename T>
struct Acc {
  T s, c;
  __device__ __forceinline__ void add(T v) {
    // error of s + v by the branch-free two-sum (adds only)
    const T t = s + v;
    const T bv = t - s;
    c += (s - (t - bv)) + (v - bv);
    s = t;
  }
  __device__ __forceinline__ T get() const { return s + c; }
};

constexpr int kNearThreads = 256;
// source particles staged per pass and table entries kept in shared memory
// (static shared memory stays under 48 KB for both element types)
template <typename T> struct NearCfg;
template <> struct NearCfg<float> { static constexpr int src = 1088, tab = 2304; };
template <> struct NearCfg<double> { static constexpr int src = 448, tab = 576; };

// 1/sqrt and sqrt of the squared distance.  FP32: the hardware reciprocal
// square root (relative error ~1e-7) in place of an IEEE sqrt and division.
__device__ __forceinline__ void inv_dist(float r2, float& rr, float& rinv) {
  rinv = rsqrtf(r2);
  rr = r2 * rinv;
}
__device__ __forceinline__ void inv_dist(double r2, double& rr, double& rinv) {
  rr = sqrt(r2);
  rinv = 1.0 / rr;
}

// Periodic shift (x, y) of a staged source, in the element type (half box
// lengths are exact in FP64, and rounded like the positions in FP32).
template <typename T>
struct alignas(2 * sizeof(T)) S2 {
  T x, y;
};

// Near kernel g(r)/r and its radial derivative from the piecewise
// polynomial table (degree kNearD in u on each of the K intervals).
template <typename T>
__device__ __forceinline__ void near_pair(T r2, T q, T dx, T dy, T dz, const T* __restrict__ tab,
                                          int K, T hK, T ihK, Acc<T>& phi, T& gx, T& gy, T& gz) {
  T rr, rinv;
  inv_dist(r2, rr, rinv);
  int kk = (int)(rr * ihK);
  kk = kk < K ? kk : K - 1;
  const T ihK2 = T(2) * ihK;
  const T u = (rr - (T)kk * hK) * ihK2 - T(1);
  // the interval's coefficients by 16-byte vector loads (rows padded to
  // near_row<T>() elements)
  T c[near_row<T>()];
  if constexpr (sizeof(T) == 4) {
    const float4* v = reinterpret_cast<const float4*>(tab + kk * near_row<T>());
#pragma unroll
    for (int i = 0; i < near_row<T>() / 4; ++i) {
      const float4 t = v[i];
      c[4 * i] = t.x;
      c[4 * i + 1] = t.y;
      c[4 * i + 2] = t.z;
      c[4 * i + 3] = t.w;
    }
  } else {
    const double2* v = reinterpret_cast<const double2*>(tab + kk * near_row<T>());
#pragma unroll
    for (int i = 0; i < near_row<T>() / 2; ++i) {
      const double2 t = v[i];
      c[2 * i] = t.x;
      c[2 * i + 1] = t.y;
    }
  }
  T p = c[kNearD], dp = T(0);
#pragma unroll
  for (int jj = kNearD - 1; jj >= 0; --jj) {
    dp = dp * u + p;
    p = p * u + c[jj];
  }
  // g(r) = 1 - r F_M(r) = p; near kernel G = g/r; dG/dr = (g' - g/r)/r
  const T gp = dp * ihK2;
  phi.add(q * p * rinv);
  const T f = q * (gp - p * rinv) * rinv * rinv;
  gx += f * dx;
  gy += f * dy;
  gz += f * dz;
}

// One warp, one target.  Pass 1 tests the staged sources 32 at a time (one
// ballot per step) and appends the accepted ones to the warp's list of
// source indices, in order; pass 2 hands the listed sources to the lanes, 32
// per round, so that every round but the last has all lanes busy.  The list
// holds kNearList entries: pass 1 runs in chunks of 8 steps and the list is
// evaluated and emptied early when another chunk might not fit.  SHIFT:
// sources carry a periodic shift s (dx = (x_i + s) - (x_j - s), both brackets
// exact).
constexpr int kNearList = 512;

template <typename T, bool SHIFT>
__device__ __forceinline__ void near_target(const P4<T>& a, const P4<T>* __restrict__ src,
                                            const S2<T>* __restrict__ sh, int nsteps, T rc2,
                                            const T* __restrict__ tab, int K, T hK, T ihK,
                                            unsigned short* __restrict__ list, T& o_phi, T& o_gx,
                                            T& o_gy, T& o_gz) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  auto diff = [&](int k, T& dx, T& dy, T& dz, T& q) {
    const P4<T> b = src[k];
    if (SHIFT) {
      const S2<T> s2 = sh[k];
      dx = (a.x + s2.x) - b.x;
      dy = (a.y + s2.y) - b.y;
    } else {
      dx = a.x - b.x;
      dy = a.y - b.y;
    }
    dz = a.z - b.z;
    q = b.q;
  };
  Acc<T> phi{0, 0};
  T gx = 0, gy = 0, gz = 0;
  auto evaluate = [&](int cnt) {
    __syncwarp();
    for (int h0 = 0; h0 < cnt; h0 += 32) {
      if (h0 + lane < cnt) {
        T dx, dy, dz, q;
        diff(list[h0 + lane], dx, dy, dz, q);
        const T r2 = dx * dx + dy * dy + dz * dz;
        // r2 == 0 only for the target itself (coincident charges are invalid input)
        if (r2 > T(0)) near_pair(r2, q, dx, dy, dz, tab, K, hK, ihK, phi, gx, gy, gz);
      }
    }
    __syncwarp();
  };
  int cnt = 0;  // warp-uniform
  for (int s0 = 0; s0 < nsteps; s0 += 8) {
    const int s1 = min(nsteps, s0 + 8);
    for (int st = s0; st < s1; ++st) {
      T dx, dy, dz, q;
      const int k = st * 32 + lane;
      diff(k, dx, dy, dz, q);
      const T r2 = dx * dx + dy * dy + dz * dz;
      const bool in = r2 < rc2;  // the target itself is listed and skipped when evaluated
      const unsigned m = __ballot_sync(full, in);
      if (in) list[cnt + __popc(m & below)] = (unsigned short)k;
      cnt += __popc(m);
    }
    if (cnt > kNearList - 8 * 32) {
      evaluate(cnt);
      cnt = 0;
    }
  }
  evaluate(cnt);
  o_phi = phi.get();
  o_gx = gx;
  o_gy = gy;
  o_gz = gz;
}

// Near field, Eq. (2.28): one CTA per cell.  The particles of the (up to 27)
// neighbouring cells are staged contiguously in shared memory (padded to a
// multiple of 32 with inert far-away sources); warps take the cell's
// targets one at a time (near_target).  Cells away from the periodic edges
// need no shifts; with fewer than three cells per periodic dimension the
// minimum image is found per pair by rounding instead.
template <typename T>
__global__ void __launch_bounds__(kNearThreads) k_near(NearGeom g, const P4<T>* __restrict__ rec,
                                                      const int* __restrict__ cstart,
                                                      const int* __restrict__ perm,
                                                      const T* __restrict__ tab,
                                                      double* __restrict__ phi_out,
                                                      double* __restrict__ grad_out) {
  constexpr int kNearSrc = NearCfg<T>::src, kNearTab = NearCfg<T>::tab;
  __shared__ P4<T> src[kNearSrc];                  // x - s, y - s, z, q
  __shared__ S2<T> shs[kNearSrc];                  // s (periodic shift) per source
  __shared__ unsigned short list[kNearThreads / 32][kNearList];  // accepted sources per warp
  __shared__ __align__(16) T stab[kNearTab];
  __shared__ int cb[27], coff[28];
  __shared__ T csx[27], csy[27];
  __shared__ int ncell, any_shift;
  const int c = blockIdx.x;
  const int tb = cstart[c], te = cstart[c + 1];
  if (tb == te) return;
  const int ntab = g.K * near_row<T>();
  const bool tab_sm = ntab <= kNearTab;
  if (tab_sm)
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) stab[i] = tab[i];
  const bool periodic_cells = g.nc[0] >= 3 && g.nc[1] >= 3;
  const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
  if (threadIdx.x < 32) {
    // warp 0: one lane per neighbouring cell (x fastest, then y, then z)
    const int lane = threadIdx.x;
    const int cc[3] = {cx, cy, cz};
    int lo[3], ext[3];
    for (int d = 0; d < 2; ++d) {
      if (g.nc[d] >= 3) { lo[d] = cc[d] - 1; ext[d] = 3; }
      else { lo[d] = 0; ext[d] = g.nc[d]; }
    }
    lo[2] = max(cz - 1, 0);
    ext[2] = min(cz + 1, g.nc[2] - 1) - lo[2] + 1;
    const int n = ext[0] * ext[1] * ext[2];
    int cnt = 0, st = 0;
    T sx = T(0), sy = T(0);
    if (lane < n) {
      const int ix = lane % ext[0], iy = (lane / ext[0]) % ext[1], iz = lane / (ext[0] * ext[1]);
      const int x0 = lo[0] + ix, y0 = lo[1] + iy, z = lo[2] + iz;
      const int y = (y0 + g.nc[1]) % g.nc[1], x = (x0 + g.nc[0]) % g.nc[0];
      const int k = (z * g.nc[1] + y) * g.nc[0] + x;
      st = cstart[k];
      cnt = cstart[k + 1] - st;
      // source beyond the -L/2 edge sits near +L/2: s = +L/2, and vice versa
      if (periodic_cells) {
        const T hx = near_const<T>(g, kNcHLx), hy = near_const<T>(g, kNcHLy);
        sx = x0 < 0 ? hx : (x0 >= g.nc[0] ? -hx : T(0));
        sy = y0 < 0 ? hy : (y0 >= g.nc[1] ? -hy : T(0));
      }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const bool anys = __any_sync(0xffffffffu, sx != T(0) || sy != T(0));
    if (lane < n) {
      cb[lane] = st;
      coff[lane] = incl - cnt;
      csx[lane] = sx;
      csy[lane] = sy;
    }
    if (lane == n - 1) coff[n] = incl;
    if (lane == 0) {
      ncell = n;
      any_shift = anys;
    }
  }
  __syncthreads();
  const T* tb_ = tab_sm ? stab : tab;
  const T rc2 = near_const<T>(g, kNcRc2);
  const T hK = near_const<T>(g, kNcHK), ihK = near_const<T>(g, kNcIhK);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kNearThreads / 32;
  unsigned short* mylist = list[warp];
  const int ntg = te - tb;
  const int nsrc = coff[ncell];
  const bool shifted = any_shift != 0;
  const T Lx = near_const<T>(g, kNcLx), Ly = near_const<T>(g, kNcLy);
  const T iLx = near_const<T>(g, kNcILx), iLy = near_const<T>(g, kNcILy);
  // sources in passes of at most kNearSrc (one pass in the usual case)
  for (int s0 = 0; s0 < nsrc; s0 += kNearSrc) {
    const int ns = min(kNearSrc, nsrc - s0);
    const int nsteps = (ns + 31) >> 5;
    __syncthreads();
    // a warp per neighbouring cell copies the part of it inside this pass
    for (int cc = warp; cc < ncell; cc += nw) {
      const int a0 = max(coff[cc], s0), a1 = min(coff[cc + 1], s0 + ns);
      const T sx = csx[cc], sy = csy[cc];
      const int shift = cb[cc] - coff[cc];
      for (int gk = a0 + lane; gk < a1; gk += 32) {
        P4<T> b = rec[gk + shift];
        b.x = b.x - (T)sx;
        b.y = b.y - (T)sy;
        src[gk - s0] = b;
        shs[gk - s0] = S2<T>{sx, sy};
      }
    }
    for (int k = ns + threadIdx.x; k < nsteps * 32; k += blockDim.x) {
      src[k] = P4<T>{T(1e30), T(1e30), T(1e30), T(0)};
      shs[k] = S2<T>{T(0), T(0)};
    }
    __syncthreads();
    OutSlots<T> out{T(0), 0, 0};
    // the next target's record and output index are loaded one target ahead
    P4<T> a_next{};
    int o_next = 0;
    if (warp < ntg) {
      a_next = rec[tb + warp];
      o_next = perm[tb + warp];
    }
    for (int t0 = 0; t0 < ntg; t0 += nw) {
      const int tt = t0 + warp;
      if (tt >= ntg) break;
      const P4<T> a = a_next;
      const int oi = o_next;
      if (tt + nw < ntg) {
        a_next = rec[tb + tt + nw];
        o_next = perm[tb + tt + nw];
      }
      T v0, v1, v2, v3;
      if (!periodic_cells) {
        // few cells: minimum image per pair (sources unshifted)
        Acc<T> phi{0, 0};
        T gx = 0, gy = 0, gz = 0;
        for (int k = lane; k < ns; k += 32) {  // padding excluded: rounding would fold it back
          const P4<T> b = src[k];
          T dx = a.x - b.x, dy = a.y - b.y;
          const T dz = a.z - b.z;
          dx -= Lx * drint(dx * iLx);
          dy -= Ly * drint(dy * iLy);
          const T r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < rc2 && r2 > T(0)) near_pair(r2, b.q, dx, dy, dz, tb_, g.K, hK, ihK, phi, gx, gy, gz);
        }
        v0 = phi.get();
        v1 = gx;
        v2 = gy;
        v3 = gz;
      } else if (shifted) {
        near_target<T, true>(a, src, shs, nsteps, rc2, tb_, g.K, hK, ihK, mylist, v0, v1, v2, v3);
      } else {
        near_target<T, false>(a, src, shs, nsteps, rc2, tb_, g.K, hK, ihK, mylist, v0, v1, v2, v3);
      }
      out.put(warp_sum4(v0, v1, v2, v3), oi);
      if (out.n == 8) out.flush(phi_out, grad_out, s0 > 0);
    }
    out.flush(phi_out, grad_out, s0 > 0);
  }
}

// ---------------------------------------------------------------------------
// 3. mid range (Algorithm 1): gridding and gathering
// ---------------------------------------------------------------------------

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Particles [b, e) of a tile, split into contiguous parts when several CTAs
// (blockIdx.y) share the tile; false when this CTA's part is empty.
__device__ __forceinline__ bool chunk_range(int& b, int& e, int chunks) {
  const int len = (e - b + chunks - 1) / chunks;
  b += blockIdx.y * len;
  e = min(e, b + len);
  return b < e;
}

// Offsets in the periodic grid of the rows of a padded tile whose corner is
// (oy, oz): yoff[ly] = ((oy + ly) mod I1) * pitch, zoff[lz] = ((oz + lz) mod
// I2) * I1 * pitch.  zplanes: for proxy planes, lz is the plane index n.
__device__ __forceinline__ void tile_tables(const TileGeom& g, int oy, int oz, int nz, bool zplanes,
                                            int* yoff, long long* zoff) {
  for (int i = threadIdx.x; i < g.W[1]; i += blockDim.x) yoff[i] = pmod(oy + i, g.I[1]) * g.pitch;
  for (int i = threadIdx.x; i < nz; i += blockDim.x)
    zoff[i] = (long long)(zplanes ? i : pmod(oz + i, g.I[2])) * g.I[1] * g.pitch;
}

// Asynchronous global -> shared copy of one element (cp.async): the loads of
// a whole tile are in flight together instead of one row at a time.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Moves the padded tile between shared memory (row pitch rp, plane stride
// ps) and the periodic grid, one warp per row (W0 <= 32): LOAD copies grid
// to tile, otherwise the tile is added to the grid with atomics (tiles
// overlap in their halos).  xw = wrapped x index of this lane.
template <typename T, bool LOAD>
__device__ __forceinline__ void tile_rows(T* __restrict__ grid, T* __restrict__ st, int W0, int W1,
                                          int nz, int rp, int ps, const int* __restrict__ yoff,
                                          const long long* __restrict__ zoff, int xw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int ly = warp, lz = 0;
  while (ly >= W1) { ly -= W1; ++lz; }
  for (int row = warp; row < W1 * nz; row += nw) {
    if (lane < W0) {
      T* gp = grid + zoff[lz] + yoff[ly] + xw;
      T* sp = st + lz * ps + ly * rp + lane;
      if (LOAD) {
        cp_async_elem(sp, gp);
      } else {
        const T v = *sp;
        if (v != T(0)) atomicAdd(gp, v);
      }
    }
    ly += nw;
    while (ly >= W1) { ly -= W1; ++lz; }
  }
  if (LOAD) cp_async_wait_all();
}

// Fixed-point accumulator of the spreading tile: int32 for FP32 plans, int64
// for FP64 plans (integer shared-memory atomics are native; the sum is
// exact and independent of the order of the additions).
template <typename T> struct FixAcc;
template <> struct FixAcc<float> {
  using t = int;
  static constexpr int bits = 30;
  __device__ static int cvt(float v) { return __float2int_rn(v); }
};
template <> struct FixAcc<double> {
  using t = long long;
  static constexpr int bits = 62;
  __device__ static long long cvt(double v) { return __double2ll_rn(v); }
};

__device__ __forceinline__ void fix_add(int* p, int v) { atomicAdd(p, v); }
__device__ __forceinline__ void fix_add(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// Gridding, Eq. (3.7).  One CTA per tile (or part of a tile).  The CTA's
// particles are spread into a padded tile in shared memory held in fixed
// point: the scale S = 2^(bits - e) with sum_j |q_j| < 2^e bounds every
// partial sum by 2^bits, so the integer atomics cannot overflow.  A warp per
// particle, lanes over the (dz, dy) rows of its window.  The padded tile is
// then added to the grid (zero on entry).
template <typename T, int PW>
__global__ void __launch_bounds__(kTileThreads) k_mid_spread(TileGeom g, WinT<T> w,
                                                             const P4<T>* __restrict__ rec,
                                                             const int* __restrict__ start,
                                                             T* __restrict__ grid) {
  using A = typename FixAcc<T>::t;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tile = blockIdx.x;
  int b = start[tile], e = start[tile + 1];
  if (!chunk_range(b, e, g.chunks)) return;
  const int W0 = g.W[0], W1 = g.W[1], W2 = g.W[2];
  const int P = PW > 0 ? PW : w.P;
  const int PP = P * P;
  const int RP = gather_row_pitch(W0);
  const int PS = gather_plane_stride(RP, W1, P);
  long long* zoff = reinterpret_cast<long long*>(smraw);
  int* yoff = reinterpret_cast<int*>(zoff + 64);
  int* bofs = yoff + 32;
  T* red = reinterpret_cast<T*>(bofs + kTileBatch);     // [8] warp sums of |q|
  T* wgt = reinterpret_cast<T*>(smraw + kTileHeader);  // [j][axis][k], q folded into x
  A* st = reinterpret_cast<A*>(wgt + kTileBatch * 3 * kMaxWin);
  const int tz = tile / (g.nt[0] * g.nt[1]);
  const int ty = (tile / g.nt[0]) % g.nt[1];
  const int tx = tile % g.nt[0];
  const int ox = tx * g.T[0] - g.pad_lo, oy = ty * g.T[1] - g.pad_lo, oz = tz * g.T[2] - g.pad_lo;
  {
    // the tile starts 16-byte aligned: zero it in 16-byte stores
    constexpr int V = 16 / sizeof(A);
    const int nv = W2 * PS / V;
    int4* st4 = reinterpret_cast<int4*>(st);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) st4[i] = make_int4(0, 0, 0, 0);
    for (int i = nv * V + threadIdx.x; i < W2 * PS; i += blockDim.x) st[i] = A(0);
  }
  tile_tables(g, oy, oz, W2, false, yoff, zoff);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // scale of the fixed-point tile
  T qa = 0;
  for (int i = b + threadIdx.x; i < e; i += blockDim.x) qa += fabs(rec[i].q);
  qa = warp_sum(qa);
  if (lane == 0) red[warp] = qa;
  __syncthreads();
  T qsum = 0;
  for (int k = 0; k < nw; ++k) qsum += red[k];
  int ex = 0;
  frexp(qsum > T(0) ? qsum : T(1), &ex);  // qsum < 2^ex
  const T S = ldexp(T(1), FixAcc<T>::bits - ex), iS = ldexp(T(1), ex - FixAcc<T>::bits);
  constexpr int NIT = PW > 0 ? (PW * PW + 31) / 32 : (kMaxWin * kMaxWin) / 32;
  constexpr int PR = PW > 0 ? PW : kMaxWin;
  int roff[NIT], rdy[NIT], rdz[NIT];  // this lane's (dz, dy) rows, roff -1: none
#pragma unroll
  for (int it = 0; it < NIT; ++it) {
    const int s2 = lane + 32 * it;
    const int dz = s2 / P, dy = s2 - dz * P;
    const bool ok = s2 < PP;
    roff[it] = ok ? dz * PS + dy * RP : -1;
    rdy[it] = ok ? dy : 0;
    rdz[it] = ok ? dz : 0;
  }
  for (int p0 = b; p0 < e; p0 += kTileBatch) {
    const int nb = min(kTileBatch, e - p0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * 3 * P; idx += blockDim.x) {
      const int j = idx / (3 * P);
      const int r = idx - j * 3 * P;
      const int ax = r / P, k = r - ax * P;
      const P4<T> a = rec[p0 + j];
      const T c = ax == 0 ? a.x : (ax == 1 ? a.y : a.z);
      const int g0 = (int)dceil(c - w.half);
      const T v = win_val_pt<T, PW == 0>(w, g0, c, k);
      wgt[(j * 3 + ax) * kMaxWin + k] = ax == 0 ? v * a.q : v;
      if (r == 0) {
        const int gy0 = (int)dceil(a.y - w.half), gz0 = (int)dceil(a.z - w.half);
        bofs[j] = (gz0 + g.pad_lo) * PS + (gy0 + g.pad_lo) * RP + g0 + g.pad_lo;
      }
    }
    __syncthreads();
    for (int j = warp; j < nb; j += nw) {
      const T* wj = wgt + j * 3 * kMaxWin;
      T rwx[PR];
#pragma unroll
      for (int dx = 0; dx < PR; ++dx) rwx[dx] = dx < P ? wj[dx] : T(0);
      A* bj = st + bofs[j];
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        if (roff[it] >= 0) {
          const T c = wj[kMaxWin + rdy[it]] * wj[2 * kMaxWin + rdz[it]] * S;
          A* rp = bj + roff[it];
#pragma unroll
          for (int dx = 0; dx < PR; ++dx)
            if (dx < P) fix_add(rp + dx, FixAcc<T>::cvt(c * rwx[dx]));
        }
      }
    }
  }
  __syncthreads();
  if (sizeof(T) == 4 && ((g.I[0] | g.pitch) & 1) == 0) {
    // FP32: pairs of columns (x even, x + 1) with one 8-byte atomic; the
    // even grid width keeps a pair inside one row.  Pairs start at the even
    // column ox0 <= ox; columns outside the tile add zero.
    const int ox0 = ox & ~1;
    const int W0h = (ox + W0 - ox0 + 1) >> 1, tot = W0h * W1 * W2;
    const int nt = blockDim.x;
    int lx = threadIdx.x % W0h, rr = threadIdx.x / W0h;
    int ly = rr % W1, lz = rr / W1;
    const int sx = nt % W0h, sr = nt / W0h, sy = sr % W1, sz = sr / W1;
    for (int i = threadIdx.x; i < tot; i += nt) {
      const int c0 = ox0 + 2 * lx - ox;  // tile column of the pair's first element
      const A* sp = st + lz * PS + ly * RP;
      const A v0 = c0 >= 0 ? sp[c0] : A(0), v1 = c0 + 1 < W0 ? sp[c0 + 1] : A(0);
      if ((v0 | v1) != 0) {
        float* gp = reinterpret_cast<float*>(grid) + zoff[lz] + yoff[ly] + pmod(ox0 + 2 * lx, g.I[0]);
        atomicAdd(reinterpret_cast<float2*>(gp), make_float2((float)v0 * (float)iS, (float)v1 * (float)iS));
      }
      lx += sx;
      ly += sy;
      lz += sz;
      if (lx >= W0h) { lx -= W0h; ++ly; }
      if (ly >= W1) { ly -= W1; ++lz; }
    }
    return;
  }
  const int xw = lane < W0 ? pmod(ox + lane, g.I[0]) : 0;
  int ly = warp, lz = 0;
  while (ly >= W1) { ly -= W1; ++lz; }
  for (int row = warp; row < W1 * W2; row += nw) {
    if (lane < W0) {
      const A v = st[lz * PS + ly * RP + lane];
      if (v != A(0)) atomicAdd(grid + zoff[lz] + yoff[ly] + xw, (T)v * iS);
    }
    ly += nw;
    while (ly >= W1) { ly -= W1; ++lz; }
  }
}

// Copies a padded tile (W0 x W1 x nz elements) from the periodic grid into
// shared memory (row pitch rp, plane stride ps), element by element with
// cp.async: xoff, yoff, zoff give the grid offsets of tile column, row and
// plane.
template <typename T>
__device__ __forceinline__ void tile_load(const T* __restrict__ grid, T* __restrict__ st, int W0,
                                          int W1, int nz, int rp, int ps, const int* __restrict__ xoff,
                                          const int* __restrict__ yoff,
                                          const long long* __restrict__ zoff) {
  const int tot = W0 * W1 * nz;
  const int nt = blockDim.x;
  int lx = threadIdx.x % W0, r = threadIdx.x / W0;
  int ly = r % W1, lz = r / W1;
  const int sx = nt % W0, sr = nt / W0, sy = sr % W1, sz = sr / W1;
  for (int i = threadIdx.x; i < tot; i += nt) {
    cp_async_elem(st + lz * ps + ly * rp + lx, grid + zoff[lz] + yoff[ly] + xoff[lx]);
    lx += sx;
    ly += sy;
    lz += sz;
    if (lx >= W0) { lx -= W0; ++ly; }
    if (ly >= W1) { ly -= W1; ++lz; }
  }
  cp_async_wait_all();
}

// Gathering, Eq. (3.10): Phi^mid_i = sum_g u[g] W(r_i - r_g) and its gradient.
// The padded tile is loaded into shared memory once (odd row pitch, plane
// stride = P x pitch mod 32).  A warp per particle: its lanes first evaluate
// the 3P window values and derivatives, then each lane sums whole x rows
// (dz, dy) of the window; lane e reads word e x pitch + dx (mod 32), so the
// 32 rows of a step fall in 32 different banks.  The four sums are combined
// over the warp at the end.
template <typename T, int PW>
__global__ void __launch_bounds__(kTileThreads) k_mid_gather(TileGeom g, WinT<T> w,
                                                             const P4<T>* __restrict__ rec,
                                                             const int* __restrict__ start,
                                                             const int* __restrict__ perm,
                                                             const T* __restrict__ grid, double3 invh,
                                                             double* __restrict__ phi_out,
                                                             double* __restrict__ grad_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tile = blockIdx.x;
  int b = start[tile], e = start[tile + 1];
  if (!chunk_range(b, e, g.chunks)) return;
  const int W0 = g.W[0], W1 = g.W[1], W2 = g.W[2];
  const int P = PW > 0 ? PW : w.P;
  const int PP = P * P;
  const int RP = gather_row_pitch(W0);
  const int PS = gather_plane_stride(RP, W1, P);
  constexpr int PR = PW > 0 ? PW : kMaxWin;
  constexpr int NIT = PW > 0 ? (PW * PW + 31) / 32 : (kMaxWin * kMaxWin) / 32;
  long long* zoff = reinterpret_cast<long long*>(smraw);
  int* yoff = reinterpret_cast<int*>(zoff + 64);
  int* xoff = yoff + 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // per warp: (w, w') of the 3 axes, [axis][k]
  Cx<T>* wsm = reinterpret_cast<Cx<T>*>(smraw + kGatherHeader) + warp * 3 * kMaxWin;
  T* st = reinterpret_cast<T*>(smraw + kGatherHeader + (size_t)kTileThreads / 32 * 3 * kMaxWin * sizeof(Cx<T>));
  const int tz = tile / (g.nt[0] * g.nt[1]);
  const int ty = (tile / g.nt[0]) % g.nt[1];
  const int tx = tile % g.nt[0];
  const int ox = tx * g.T[0] - g.pad_lo, oy = ty * g.T[1] - g.pad_lo, oz = tz * g.T[2] - g.pad_lo;
  tile_tables(g, oy, oz, W2, false, yoff, zoff);
  for (int i = threadIdx.x; i < W0; i += blockDim.x) xoff[i] = pmod(ox + i, g.I[0]);
  __syncthreads();
  tile_load(grid, st, W0, W1, W2, RP, PS, xoff, yoff, zoff);
  __syncthreads();
  // this lane's rows (dz, dy) of the window; roff -1: none
  int roff[NIT], rdy[NIT], rdz[NIT];
#pragma unroll
  for (int it = 0; it < NIT; ++it) {
    const int s2 = lane + 32 * it;
    const int dz = s2 / P, dy = s2 - dz * P;
    const bool ok = s2 < PP;
    roff[it] = ok ? dz * PS + dy * RP : -1;
    rdy[it] = ok ? dy : 0;
    rdz[it] = ok ? dz : 0;
  }
  // this lane's window values: index l = lane (and lane + 32) of [axis][k]
  const int ax0 = lane / P, k0 = lane - ax0 * P;
  const int l1 = lane + 32, ax1 = l1 / P, k1 = l1 - ax1 * P;
  const T ih_lane = (T)((lane >> 3) == 1 ? invh.x : ((lane >> 3) == 2 ? invh.y : invh.z));
  OutSlots<T> out{T(0), 0, 0};
  // the next particle's record and output index are loaded one iteration
  // ahead, so their latency overlaps the current particle's sums
  P4<T> a_next{};
  int o_next = 0;
  if (b + warp < e) {
    a_next = rec[b + warp];
    o_next = perm[b + warp];
  }
  for (int j = b + warp; j < e; j += nw) {
    const P4<T> a = a_next;
    const int oj = o_next;
    if (j + nw < e) {
      a_next = rec[j + nw];
      o_next = perm[j + nw];
    }
    const int gx0 = (int)dceil(a.x - w.half), gy0 = (int)dceil(a.y - w.half),
              gz0 = (int)dceil(a.z - w.half);
    {
      // d/dt of phi((g - t)/half) = -phi'/half
      T v, dv;
      if (ax0 < 3) {
        const T c = ax0 == 0 ? a.x : (ax0 == 1 ? a.y : a.z);
        const int g0 = ax0 == 0 ? gx0 : (ax0 == 1 ? gy0 : gz0);
        win_eval_pt<T, PW == 0>(w, g0, c, k0, v, dv);
        wsm[ax0 * kMaxWin + k0] = Cx<T>{v, -dv * w.inv_half};
      }
      if (3 * P > 32 && ax1 < 3) {
        const T c = ax1 == 0 ? a.x : (ax1 == 1 ? a.y : a.z);
        const int g0 = ax1 == 0 ? gx0 : (ax1 == 1 ? gy0 : gz0);
        win_eval_pt<T, PW == 0>(w, g0, c, k1, v, dv);
        wsm[ax1 * kMaxWin + k1] = Cx<T>{v, -dv * w.inv_half};
      }
    }
    __syncwarp();
    T wx[PR], dwx[PR];
#pragma unroll
    for (int k = 0; k < PR; ++k) {
      const Cx<T> t = k < P ? wsm[k] : Cx<T>{T(0), T(0)};
      wx[k] = t.x;
      dwx[k] = t.y;
    }
    const T* bj = st + (gz0 + g.pad_lo) * PS + (gy0 + g.pad_lo) * RP + gx0 + g.pad_lo;
    T f = 0, fx = 0, fy = 0, fz = 0;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      if (roff[it] >= 0) {
        const T* rp = bj + roff[it];
        T sx = 0, sd = 0;
#pragma unroll
        for (int dx = 0; dx < PR; ++dx) {
          if (dx < P) {
            const T u = rp[dx];
            sx += u * wx[dx];
            sd += u * dwx[dx];
          }
        }
        const Cx<T> wy = wsm[kMaxWin + rdy[it]], wz = wsm[2 * kMaxWin + rdz[it]];
        const T wyz = wy.x * wz.x;
        f += wyz * sx;
        fx += wyz * sd;
        fy += wy.y * wz.x * sx;
        fz += wy.x * wz.y * sx;
      }
    }
    __syncwarp();
    const T tot = warp_sum4(f, fx, fy, fz);
    out.put(lane < 8 ? tot : tot * ih_lane, oj);
    if (out.n == 8) out.flush(phi_out, grad_out, false);
  }
  out.flush(phi_out, grad_out, false);
}

// ---------------------------------------------------------------------------
// 4. long range (Algorithm 2, anterpolation form)
// ---------------------------------------------------------------------------

// Chebyshev polynomials T_0..T_{P-1}(x) into t[].
template <typename T>
__device__ __forceinline__ void cheb_all(T x, int P, T* t) {
  t[0] = T(1);
  if (P > 1) t[1] = x;
  for (int n = 2; n < P; ++n) t[n] = T(2) * x * t[n - 1] - t[n - 2];
}

// Spread q_j T_n(x_j) W2(rho_g - rho_j) onto the P proxy planes (layout
// [n][y][x], pitch Ix + 2) through padded tiles (Algorithm 2, gridding in the
// anterpolation reading); planes zero on entry.  As in the mid-range
// gridding: the padded tile of all P planes is held in shared memory in fixed
// point (scale from sum |q| of the CTA's charges, so no partial sum
// overflows; |T_n| <= 1 and the window is at most 1), window values and
// T_n(x_j) are staged per batch of kTileBatch charges, and a warp takes one
// charge with its lanes over the (n, dy) rows of the window, P_cheb x P rows
// in all, 32 at a time; lane s writes word s x RP + dx (mod 32), so a step's
// 32 rows fall in 32 banks.  The tile is then added to the planes.
// A lane's rows (n, dy) of the P planes x Pw window rows, n Pw + dy = lane,
// lane + 32, lane + 64, ...: the first one and the step between them (32
// rows = dn planes and ddy rows; a row offset o = n PS + dy RP in the tile),
// so that the row loops advance by additions instead of dividing.
struct RowStep {
  int n0, dy0, o0, dn, ddy, dO, wrapO;
  __device__ RowStep(int lane, int Pw, int PS, int RP) {
    n0 = lane / Pw;
    dy0 = lane - n0 * Pw;
    o0 = n0 * PS + dy0 * RP;
    dn = 32 / Pw;
    ddy = 32 - dn * Pw;
    dO = dn * PS + ddy * RP;
    wrapO = PS - Pw * RP;
  }
  __device__ __forceinline__ void next(int& n, int& dy, int& o, int Pw) const {
    dy += ddy;
    n += dn;
    o += dO;
    if (dy >= Pw) {
      dy -= Pw;
      ++n;
      o += wrapO;
    }
  }
};

template <typename T, int PW>
__global__ void __launch_bounds__(kTileThreads) k_long_spread(TileGeom g, WinT<T> w, int P,
                                                              const P4<T>* __restrict__ rec,
                                                              const int* __restrict__ start,
                                                              T* __restrict__ planes) {
  using A = typename FixAcc<T>::t;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tile = blockIdx.x;
  int b = start[tile], e = start[tile + 1];
  if (!chunk_range(b, e, g.chunks)) return;
  const int W0 = g.W[0], W1 = g.W[1];
  const int Pw = PW > 0 ? PW : w.P;
  constexpr int PR = PW > 0 ? PW : kMaxWin;
  const int RP = gather_row_pitch(W0);
  const int PS = gather_plane_stride(RP, W1, Pw);
  long long* zoff = reinterpret_cast<long long*>(smraw);            // [kMaxCheb]
  int* yoff = reinterpret_cast<int*>(zoff + kMaxCheb);             // [32]
  int* bofs = yoff + 32;                                           // [kTileBatch]
  T* red = reinterpret_cast<T*>(bofs + kTileBatch);                // [8]
  T* wgt = reinterpret_cast<T*>(smraw + kLongSpreadHeader);        // [j][2][Pw]
  T* tnb = wgt + kTileBatch * 2 * Pw;                         // [j][P]
  A* st = reinterpret_cast<A*>(tnb + kTileBatch * P);
  const int ty = tile / g.nt[0], tx = tile % g.nt[0];
  const int ox = tx * g.T[0] - g.pad_lo, oy = ty * g.T[1] - g.pad_lo;
  {
    constexpr int V = 16 / sizeof(A);
    const int nv = P * PS / V;
    int4* st4 = reinterpret_cast<int4*>(st);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) st4[i] = make_int4(0, 0, 0, 0);
    for (int i = nv * V + threadIdx.x; i < P * PS; i += blockDim.x) st[i] = A(0);
  }
  tile_tables(g, oy, 0, P, true, yoff, zoff);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T qa = 0;
  for (int i = b + threadIdx.x; i < e; i += blockDim.x) qa += fabs(rec[i].q);
  qa = warp_sum(qa);
  if (lane == 0) red[warp] = qa;
  __syncthreads();
  T qsum = 0;
  for (int k = 0; k < nw; ++k) qsum += red[k];
  int ex = 0;
  frexp(qsum > T(0) ? qsum : T(1), &ex);  // qsum < 2^ex
  const T S = ldexp(T(1), FixAcc<T>::bits - ex), iS = ldexp(T(1), ex - FixAcc<T>::bits);
  const RowStep rs(lane, Pw, PS, RP);
  for (int p0 = b; p0 < e; p0 += kTileBatch) {
    const int nb = min(kTileBatch, e - p0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * 2 * Pw; idx += blockDim.x) {
      const int j = idx / (2 * Pw);
      const int r = idx - j * 2 * Pw;
      const int ax = r / Pw, k = r - ax * Pw;
      const P4<T> a = rec[p0 + j];
      const T c = ax == 0 ? a.x : a.y;
      const int g0 = (int)dceil(c - w.half);
      const T v = win_val_pt<T, PW == 0>(w, g0, c, k);
      wgt[(j * 2 + ax) * Pw + k] = ax == 0 ? v * a.q : v;
      if (r == 0) {
        const int gy0 = (int)dceil(a.y - w.half);
        bofs[j] = (gy0 + g.pad_lo) * RP + g0 + g.pad_lo;
      }
    }
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      // T_n(x_j) by the three-term recurrence (|x_j| <= 1)
      const T x = rec[p0 + j].z;
      T t0 = T(1), t1 = x;
      T* tj = tnb + j * P;
      for (int n = 0; n < P; ++n) {
        tj[n] = t0;
        const T t2 = T(2) * x * t1 - t0;
        t0 = t1;
        t1 = t2;
      }
    }
    __syncthreads();
    for (int j = warp; j < nb; j += nw) {
      const T* wj = wgt + j * 2 * Pw;
      const T* tj = tnb + j * P;
      T rwx[PR];
#pragma unroll
      for (int dx = 0; dx < PR; ++dx) rwx[dx] = dx < Pw ? wj[dx] : T(0);
      A* bj = st + bofs[j];
      // rows n Pw + dy = lane, lane + 32, ...: stepped, not divided
      int n = rs.n0, dy = rs.dy0, o = rs.o0;
      while (n < P) {
        const T c = wj[Pw + dy] * tj[n] * S;
        A* rp = bj + o;
#pragma unroll
        for (int dx = 0; dx < PR; ++dx)
          if (dx < Pw) fix_add(rp + dx, FixAcc<T>::cvt(c * rwx[dx]));
        rs.next(n, dy, o, Pw);
      }
    }
  }
  __syncthreads();
  // add the padded tile to the planes (tiles overlap in their halos)
  const int nt = blockDim.x;
  if (sizeof(T) == 4 && ((g.I[0] | g.pitch) & 1) == 0) {
    // FP32: pairs of columns (x even, x + 1) with one 8-byte atomic, as in
    // the mid-range gridding; columns outside the tile add zero
    const int ox0 = ox & ~1;
    const int W0h = (ox + W0 - ox0 + 1) >> 1, tot = W0h * W1 * P;
    int lx = threadIdx.x % W0h, rr = threadIdx.x / W0h;
    int ly = rr % W1, n = rr / W1;
    const int sx = nt % W0h, sr = nt / W0h, sy = sr % W1, sn = sr / W1;
    for (int i = threadIdx.x; i < tot; i += nt) {
      const int c0 = ox0 + 2 * lx - ox;
      const A* sp = st + n * PS + ly * RP;
      const A v0 = c0 >= 0 ? sp[c0] : A(0), v1 = c0 + 1 < W0 ? sp[c0 + 1] : A(0);
      if ((v0 | v1) != 0) {
        float* gp = reinterpret_cast<float*>(planes) + zoff[n] + yoff[ly] + pmod(ox0 + 2 * lx, g.I[0]);
        atomicAdd(reinterpret_cast<float2*>(gp), make_float2((float)v0 * (float)iS, (float)v1 * (float)iS));
      }
      lx += sx;
      ly += sy;
      n += sn;
      if (lx >= W0h) { lx -= W0h; ++ly; }
      if (ly >= W1) { ly -= W1; ++n; }
    }
    return;
  }
  const int xw = lane < W0 ? pmod(ox + lane, g.I[0]) : 0;
  int ly = warp, n = 0;
  while (ly >= W1) { ly -= W1; ++n; }
  for (int row = warp; row < W1 * P; row += nw) {
    if (lane < W0) {
      const A v = st[n * PS + ly * RP + lane];
      if (v != A(0)) atomicAdd(planes + zoff[n] + yoff[ly] + xw, (T)v * iS);
    }
    ly += nw;
    while (ly >= W1) { ly -= W1; ++n; }
  }
}

// Small long-range grids (I_long <= 16, one tile): each CTA takes a slice
// of the particles; every thread owns grid points of all P planes in
// registers and adds q_j W2 T_n(x_j) for the particles whose window covers
// them (no atomics).  Window values on every grid line (nearest image) and
// the Chebyshev values are staged per batch by all threads.  The per-CTA
// planes go to scratch and k_long_reduce adds them in a fixed order.
constexpr int kSmallBatch = 32;

template <typename T, int PMAX>
__global__ void __launch_bounds__(256) k_long_spread_small(int I0, int I1, WinT<T> w, int P,
                                                           const P4<T>* __restrict__ rec, int N,
                                                           T* __restrict__ partial) {
  __shared__ T wx[kSmallBatch][16], wy[kSmallBatch][16];
  __shared__ __align__(16) T tn[kSmallBatch][PMAX];
  const int G = I0 * I1;
  const int per = (N + gridDim.x - 1) / gridDim.x;
  const int b = blockIdx.x * per, e = min(N, b + per);
  const T iI0 = T(1) / (T)I0, iI1 = T(1) / (T)I1;
  for (int g0 = 0; g0 < G; g0 += blockDim.x) {
    const int gpt = g0 + threadIdx.x;
    const int gy = gpt / I0, gx = gpt - gy * I0;
    T acc[PMAX];
#pragma unroll
    for (int n = 0; n < PMAX; ++n) acc[n] = T(0);
    for (int p0 = b; p0 < e; p0 += kSmallBatch) {
      const int nb = min(kSmallBatch, e - p0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nb * 32; idx += blockDim.x) {
        const int j = idx >> 5, ax = (idx >> 4) & 1, k = idx & 15;
        const int Id = ax ? I1 : I0;
        if (k < Id) {
          const P4<T> a = rec[p0 + j];
          T v, dv;
          if (w.nu > 0) {
            // support point of grid index k, if any (the grid holds P + 4
            // points at least, so one per index)
            const T c = ax ? a.y : a.x;
            const int g0 = (int)dceil(c - w.half);
            const int kk = ((k - g0) % Id + Id) % Id;
            v = T(0);
            if (kk < w.P) win_eval_pt<T, true>(w, g0, c, kk, v, dv);
          } else {
            // nearest image of grid index k relative to the particle
            T d = (T)k - (ax ? a.y : a.x);
            d -= (T)Id * drint(d * (ax ? iI1 : iI0));
            win_eval<T, true>(w, win_arg(d, w), v, dv);
          }
          if (ax) wy[j][k] = v;
          else wx[j][k] = v * a.q;
        }
      }
      for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const T x = rec[p0 + j].z;
        T t0 = T(1), t1 = x;
#pragma unroll
        for (int n = 0; n < PMAX; ++n) {
          tn[j][n] = n < P ? t0 : T(0);
          const T t2 = T(2) * x * t1 - t0;
          t0 = t1;
          t1 = t2;
        }
      }
      __syncthreads();
      if (gpt < G) {
        for (int j = 0; j < nb; ++j) {
          const T c = wx[j][gx] * wy[j][gy];
          if (c != T(0)) {
#pragma unroll
            for (int n = 0; n < PMAX; ++n) acc[n] += c * tn[j][n];
          }
        }
      }
    }
    if (gpt < G) {
      T* out = partial + (size_t)blockIdx.x * P * G + gpt;
#pragma unroll
      for (int n = 0; n < PMAX; ++n)
        if (n < P) out[(size_t)n * G] = acc[n];
    }
  }
}

// planes[n][y][x] = sum over the CTAs b of partial[b][n][y][x], in the
// order b = 0, 1, ...: eight threads per value each sum a contiguous eighth,
// then the eight sums are added in a fixed order.
template <typename T>
__global__ void k_long_reduce(const T* __restrict__ partial, int nblk, int I0, int I1, int P,
                              T* __restrict__ planes) {
  const int G = I0 * I1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t >> 3, part = t & 7;
  const int len = (nblk + 7) / 8;
  const int b0 = part * len, b1 = min(nblk, b0 + len);
  T acc = 0;
  if (i < P * G)
    for (int bb = b0; bb < b1; ++bb) acc += partial[(size_t)bb * P * G + i];
  // fixed-order combination of the eight partial sums (lanes 8k .. 8k+7)
  const int base = threadIdx.x & 24;
  T tot = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) tot += __shfl_sync(0xffffffffu, acc, base + k);
  if (part == 0 && i < P * G) {
    const int n = i / G, gg = i - n * G;
    const int y = gg / I0, x = gg - y * I0;
    planes[((size_t)n * I1 + y) * (I0 + 2) + x] = tot;
  }
}

// Gathering, Eq. (3.19) discretised: Phi_i = sum_n T_n(x_i) sum_g W2 u_n[g],
// with the gradient from W2' in x, y and T_n' in z.  The padded tile of all P
// planes is loaded into shared memory (odd row pitch RP, plane stride =
// P_win x RP mod 32).  Window values and T_n, T_n' (three-term recurrences)
// are staged per batch of kTileBatch charges; a warp takes one charge, its
// lanes over the (n, dy) rows of the window (lane s reads word s x RP + dx
// mod 32, 32 banks per step), each lane summing whole x rows; the four sums
// are combined over the warp at the end.
template <typename T, int PW>
__global__ void __launch_bounds__(kTileThreads) k_long_gather(TileGeom g, WinT<T> w, int P,
                                                              const P4<T>* __restrict__ rec,
                                                              const int* __restrict__ start,
                                                              const int* __restrict__ perm,
                                                              const T* __restrict__ planes, double3 sc,
                                                              double* __restrict__ phi_out,
                                                              double* __restrict__ grad_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tile = blockIdx.x;
  int b = start[tile], e = start[tile + 1];
  if (!chunk_range(b, e, g.chunks)) return;
  const int W0 = g.W[0], W1 = g.W[1];
  const int Pw = PW > 0 ? PW : w.P;
  constexpr int PR = PW > 0 ? PW : kMaxWin;
  const int RP = gather_row_pitch(W0);
  const int PS = gather_plane_stride(RP, W1, Pw);
  long long* zoff = reinterpret_cast<long long*>(smraw);   // [kMaxCheb]
  int* yoff = reinterpret_cast<int*>(zoff + kMaxCheb);    // [32]
  int* xoff = yoff + 32;                                  // [32]
  int* bofs = xoff + 32;                                  // [kTileBatch]
  T* wgt = reinterpret_cast<T*>(smraw + kLongSpreadHeader);  // [j][4][Pw]: w_x, w_x', w_y, w_y'
  T* tnb = wgt + kTileBatch * 4 * Pw;                   // [j][2][P]: T_n, T_n'
  T* st = tnb + kTileBatch * 2 * P;
  const int ty = tile / g.nt[0], tx = tile % g.nt[0];
  const int ox = tx * g.T[0] - g.pad_lo, oy = ty * g.T[1] - g.pad_lo;
  tile_tables(g, oy, 0, P, true, yoff, zoff);
  for (int i = threadIdx.x; i < W0; i += blockDim.x) xoff[i] = pmod(ox + i, g.I[0]);
  __syncthreads();
  tile_load(planes, st, W0, W1, P, RP, PS, xoff, yoff, zoff);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T sc_lane = (T)((lane >> 3) == 1 ? sc.x : ((lane >> 3) == 2 ? sc.y : sc.z));
  const RowStep rs(lane, Pw, PS, RP);
  OutSlots<T> out{T(0), 0, 0};
  for (int p0 = b; p0 < e; p0 += kTileBatch) {
    const int nb = min(kTileBatch, e - p0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * 2 * Pw; idx += blockDim.x) {
      const int j = idx / (2 * Pw);
      const int r = idx - j * 2 * Pw;
      const int ax = r / Pw, k = r - ax * Pw;
      const P4<T> a = rec[p0 + j];
      const T c = ax == 0 ? a.x : a.y;
      const int g0 = (int)dceil(c - w.half);
      T v, dv;
      win_eval_pt<T, PW == 0>(w, g0, c, k, v, dv);
      T* wj = wgt + (j * 4 + 2 * ax) * Pw;
      wj[k] = v;
      wj[Pw + k] = -dv * w.inv_half;  // d/dt of phi((g - t)/half)
      if (r == 0) {
        const int gy0 = (int)dceil(a.y - w.half);
        bofs[j] = (gy0 + g.pad_lo) * RP + g0 + g.pad_lo;
      }
    }
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      // T_n(x) and T_n'(x) by the three-term recurrences
      const T x = rec[p0 + j].z;
      T* tj = tnb + j * 2 * P;
      T t0 = T(1), t1 = x, d0 = T(0), d1 = T(1);
      for (int n = 0; n < P; ++n) {
        tj[n] = t0;
        tj[P + n] = d0;
        const T t2 = T(2) * x * t1 - t0, d2 = T(2) * t1 + T(2) * x * d1 - d0;
        t0 = t1;
        t1 = t2;
        d0 = d1;
        d1 = d2;
      }
    }
    __syncthreads();
    for (int j = warp; j < nb; j += nw) {
      const T* wj = wgt + j * 4 * Pw;
      const T* tj = tnb + j * 2 * P;
      T rwx[PR], rdwx[PR];
#pragma unroll
      for (int dx = 0; dx < PR; ++dx) {
        rwx[dx] = dx < Pw ? wj[dx] : T(0);
        rdwx[dx] = dx < Pw ? wj[Pw + dx] : T(0);
      }
      const T* bj = st + bofs[j];
      T f = 0, fx = 0, fy = 0, fz = 0;
      // rows n Pw + dy = lane, lane + 32, ...: stepped, not divided
      int n = rs.n0, dy = rs.dy0, o = rs.o0;
      while (n < P) {
        const T* rp = bj + o;
        T sx = 0, sd = 0;
#pragma unroll
        for (int dx = 0; dx < PR; ++dx) {
          if (dx < Pw) {
            const T u = rp[dx];
            sx += u * rwx[dx];
            sd += u * rdwx[dx];
          }
        }
        const T wy = wj[2 * Pw + dy], dwy = wj[3 * Pw + dy];
        const T tn = tj[n], dtn = tj[P + n];
        const T tw = tn * wy;
        f += tw * sx;
        fx += tw * sd;
        fy += tn * dwy * sx;
        fz += dtn * wy * sx;
        rs.next(n, dy, o, Pw);
      }
      const T tot = warp_sum4(f, fx, fy, fz);
      out.put(lane < 8 ? tot : tot * sc_lane, perm[p0 + j]);
      if (out.n == 8) out.flush(phi_out, grad_out, false);
    }
  }
  out.flush(phi_out, grad_out, false);
}

// ---------------------------------------------------------------------------
// 4b. long range by direct Fourier sums (Algorithm 3, no FFT), in the same
//     anterpolation reading: moments mu_n(k) = sum_j q_j T_n(x_j) e^{-ik.rho_j}
//     over the half-plane modes, coefficients c_n(k) = K_k mu(k), and
//     Phi_i = sum_k Re[e^{ik.rho_i} sum_n c_n(k) T_n(x_i)] (the conjugate
//     modes are folded into the factor 2 of K_k).
// ---------------------------------------------------------------------------

constexpr int kModeThreads = 256, kModeBatch = 128;

__device__ __forceinline__ void dsincospi(float a, float* s, float* c) { sincospif(a, s, c); }
__device__ __forceinline__ void dsincospi(double a, double* s, double* c) { sincospi(a, s, c); }

// Geometry of the direct long range in the element type (no FP64 in the
// per-particle work): 2/Lx, 2/Ly, Lz/2, 2/Lz, 2 pi/Lx, 2 pi/Ly.
template <typename T>
struct ModeGeom {
  T tx, ty, hz, ihz, kx1, ky1;
};
template <typename T>
__host__ ModeGeom<T> mode_geom(double Lx, double Ly, double Lz) {
  const double pi = 3.14159265358979323846;
  return ModeGeom<T>{(T)(2.0 / Lx), (T)(2.0 / Ly), (T)(0.5 * Lz), (T)(2.0 / Lz), (T)(2.0 * pi / Lx),
                     (T)(2.0 * pi / Ly)};
}
// z / (Lz/2), clamped to [-1, 1] (0 for non-finite z)
template <typename T>
__device__ __forceinline__ T cheb_x(T z, const ModeGeom<T>& mg) {
  T x = z * mg.ihz;
  if (!(x >= T(-1) && x <= T(1))) x = isfinite(z) ? (x < T(0) ? T(-1) : T(1)) : T(0);
  return x;
}

// e^{sgn i 2 pi n t / L} for n = n0 .. n0 + cnt - 1 (tl = 2/L): the first by
// sincospi, the rest by products with the step.
template <typename T>
__device__ __forceinline__ void cis_run(T t, T tl, int n0, int cnt, T sgn, Cx<T>* out,
                                        int stride) {
  const T a = tl * t;
  T s, c;
  dsincospi(a, &s, &c);
  const Cx<T> step{c, sgn * s};
  dsincospi(a * (T)n0, &s, &c);
  Cx<T> v{c, sgn * s};
  for (int k = 0; k < cnt; ++k) {
    out[k * stride] = v;
    v = cxmul(v, step);
  }
}

// Per-block partial moments.  A batch of nbt particles is staged (q T_n,
// e^{-ik_x x}, e^{-ik_y y}); thread (mode, group) sums the batch's particles
// j = group (mod groups) for its mode in the element type; at the end the
// groups are added in a fixed order in the element type, kModeRed orders at
// a time, and written per block.
constexpr int kModeRed = 16;

template <typename T, int PMAX>
__global__ void __launch_bounds__(kModeThreads) k_lmodes_moments(
    const T* __restrict__ q, const T* __restrict__ r, int N, int P, int Kx, int Ky, int nhalf,
    int nbt, ModeGeom<T> mg, T* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ny_all = 2 * Ky + 1;
  T* tq = reinterpret_cast<T*>(smraw);                   // [j][PMAX]
  Cx<T>* ex = reinterpret_cast<Cx<T>*>(tq + nbt * PMAX);  // [j][Kx + 1]
  Cx<T>* ey = ex + nbt * (Kx + 1);                        // [j][2 Ky + 1]
  const int G = kModeThreads / nhalf;
  const int mode = threadIdx.x % nhalf, grp = threadIdx.x / nhalf;
  const bool active = grp < G;
  int nx = 0, ny = 0;
  half_mode(mode, Ky, nx, ny);
  T acc[PMAX][2];
#pragma unroll
  for (int n = 0; n < PMAX; ++n) acc[n][0] = acc[n][1] = T(0);
  const int per = (N + gridDim.x - 1) / gridDim.x;
  const int b = blockIdx.x * per, e = min(N, b + per);
  for (int p0 = b; p0 < e; p0 += nbt) {
    const int nb = min(nbt, e - p0);
    __syncthreads();
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      const int i = p0 + j;
      const T x = cheb_x(r[3 * i + 2], mg);
      T qi = q[i];
      if (!isfinite(qi)) qi = T(0);
      T t0 = T(1), t1 = x;
#pragma unroll
      for (int n = 0; n < PMAX; ++n) {
        tq[j * PMAX + n] = n < P ? qi * t0 : T(0);
        const T t2 = T(2) * x * t1 - t0;
        t0 = t1;
        t1 = t2;
      }
      cis_run(r[3 * i], mg.tx, 0, Kx + 1, T(-1), ex + j * (Kx + 1), 1);
      cis_run(r[3 * i + 1], mg.ty, -Ky, ny_all, T(-1), ey + j * ny_all, 1);
    }
    __syncthreads();
    if (active) {
      for (int j = grp; j < nb; j += G) {
        const Cx<T> ph = cxmul(ex[j * (Kx + 1) + nx], ey[j * ny_all + ny + Ky]);
        const T* tj = tq + j * PMAX;
#pragma unroll
        for (int n = 0; n < PMAX; ++n) {
          acc[n][0] += ph.x * tj[n];
          acc[n][1] += ph.y * tj[n];
        }
      }
    }
  }
  // groups -> fixed-order sum, kModeRed orders at a time (reuses the staging)
  T* red = reinterpret_cast<T*>(smraw);  // [thread][kModeRed][2]
#pragma unroll
  for (int c0 = 0; c0 < PMAX; c0 += kModeRed) {
    if (c0 < P) {
      __syncthreads();
      if (active) {
#pragma unroll
        for (int k = 0; k < kModeRed; ++k) {
          red[(threadIdx.x * kModeRed + k) * 2] = acc[c0 + k][0];
          red[(threadIdx.x * kModeRed + k) * 2 + 1] = acc[c0 + k][1];
        }
      }
      __syncthreads();
      const int pc = min(kModeRed, P - c0);
      for (int idx = threadIdx.x; idx < nhalf * pc; idx += blockDim.x) {
        const int md = idx / pc, k = idx - md * pc;
        T sr = T(0), si = T(0);
        for (int g = 0; g < G; ++g) {
          sr += red[((g * nhalf + md) * kModeRed + k) * 2];
          si += red[((g * nhalf + md) * kModeRed + k) * 2 + 1];
        }
        T* o = part + (((size_t)blockIdx.x * nhalf + md) * P + c0 + k) * 2;
        o[0] = sr;
        o[1] = si;
      }
    }
  }
}

// Coefficients: one block per half-plane mode.  Thread t takes the value
// t mod 2P (order n, real or imaginary part) of the blocks b = t / 2P (mod
// groups) in a fixed order (FP32 plans: compensated float sums, as precise
// as FP64 here and without the slow FP64 pipe), the groups are added in a
// fixed order in FP64, and the mode's P x P kernel is applied.
constexpr int kCoefThreads = 1024;
template <typename T>
__global__ void __launch_bounds__(kCoefThreads) k_lmodes_coeffs(const T* __restrict__ part,
                                                                int nblk, int nhalf, int P,
                                                                const T* __restrict__ K,
                                                                T* __restrict__ coef) {
  __shared__ double gs[kCoefThreads];
  __shared__ double mu[kMaxCheb * 2];
  const int mode = blockIdx.x;
  const int w = 2 * P, G = blockDim.x / w;
  const int v = threadIdx.x % w, g = threadIdx.x / w;
  T s = T(0), c = T(0);
  if (g < G) {
#pragma unroll 4
    for (int b = g; b < nblk; b += G) {
      const T x = part[((size_t)b * nhalf + mode) * w + v];
      if constexpr (sizeof(T) == 4) {
        const T t = s + x, bx = t - s;
        c += (s - (t - bx)) + (x - bx);
        s = t;
      } else {
        s += x;
      }
    }
  }
  gs[threadIdx.x] = (double)s + (double)c;
  __syncthreads();
  if (threadIdx.x < w) {
    double t = 0.0;
    for (int k = 0; k < G; ++k) t += gs[k * w + threadIdx.x];
    mu[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x < w) {
    const int n = threadIdx.x >> 1, c = threadIdx.x & 1;
    const T* Km = K + ((size_t)mode * P + n) * P;
    double acc = 0.0;
    for (int n2 = 0; n2 < P; ++n2) acc += (double)Km[n2] * mu[2 * n2 + c];
    coef[(size_t)mode * w + threadIdx.x] = (T)acc;
  }
}

// Potential and gradient of the long range at every particle (input order).
template <typename T, int PMAX>
__global__ void __launch_bounds__(kModeThreads) k_lmodes_eval(
    const T* __restrict__ r, int N, int P, int Kx, int Ky, int nhalf, ModeGeom<T> mg,
    const T* __restrict__ coef, double* __restrict__ phi_out, double* __restrict__ grad_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Cx<T>* c = reinterpret_cast<Cx<T>*>(smraw);  // [mode][P]
  for (int i = threadIdx.x; i < nhalf * P; i += blockDim.x)
    c[i] = Cx<T>{coef[2 * i], coef[2 * i + 1]};
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T x = cheb_x(r[3 * i + 2], mg);
  T tn[PMAX], dn[PMAX];
  {
    T t0 = T(1), t1 = x, d0 = T(0), d1 = T(1);
#pragma unroll
    for (int n = 0; n < PMAX; ++n) {
      tn[n] = t0;
      dn[n] = d0;
      const T t2 = T(2) * x * t1 - t0;
      const T d2 = T(2) * t1 + T(2) * x * d1 - d0;
      t0 = t1;
      t1 = t2;
      d0 = d1;
      d1 = d2;
    }
  }
  const T kx1 = mg.kx1, ky1 = mg.ky1;
  const T xv = r[3 * i], yv = r[3 * i + 1];
  T sa, ca, sb, cb;
  dsincospi(mg.tx * xv, &sa, &ca);
  dsincospi(mg.ty * yv, &sb, &cb);
  const Cx<T> stepx{ca, sa}, stepy{cb, sb};
  T f = 0, gx = 0, gy = 0, gz = 0;
  Cx<T> exv{T(1), T(0)};
  int md = 0;
  for (int mx = 0; mx <= Kx; ++mx) {
    // e^{i ky y} from n_y = 1 (mx = 0) or -Ky (mx > 0)
    const int ny0 = mx == 0 ? 1 : -Ky;
    T s0, c0;
    dsincospi(mg.ty * yv * (T)ny0, &s0, &c0);
    Cx<T> eyv{c0, s0};
    for (int my = ny0; my <= Ky; ++my, ++md) {
      const Cx<T> ph = cxmul(exv, eyv);
      const Cx<T>* cm = c + md * P;
      T Sr = 0, Si = 0, Zr = 0, Zi = 0;
#pragma unroll
      for (int n = 0; n < PMAX; ++n) {
        if (n < P) {
          const Cx<T> cn = cm[n];
          Sr += cn.x * tn[n];
          Si += cn.y * tn[n];
          Zr += cn.x * dn[n];
          Zi += cn.y * dn[n];
        }
      }
      const T re = ph.x * Sr - ph.y * Si, im = ph.x * Si + ph.y * Sr;
      f += re;
      gx -= (T)mx * kx1 * im;
      gy -= (T)my * ky1 * im;
      gz += ph.x * Zr - ph.y * Zi;
      eyv = cxmul(eyv, stepy);
    }
    exv = cxmul(exv, stepx);
  }
  phi_out[i] = (double)f;
  grad_out[3 * i] = (double)gx;
  grad_out[3 * i + 1] = (double)gy;
  grad_out[3 * i + 2] = (double)(gz * mg.ihz);
}

// ---------------------------------------------------------------------------
// 5. k = 0 mode of the long range, FP64
// ---------------------------------------------------------------------------

// Per-block partial Chebyshev moments sum_j q_j T_n(x_j), n < P: T_n by the
// recurrence in the element type (|T_n| <= 1 on [-1, 1]); each thread sums
// its few particles (about N / 19,456) in the element type, warps and blocks
// sum in FP64.  The moments are then combined with the FP64 kernel matrix
// and the k = 0 potential is evaluated in FP64 (Clenshaw).
constexpr int kK0Threads = 128;

template <typename T, int PMAX>
__global__ void __launch_bounds__(kK0Threads) k_k0_moments(const T* __restrict__ q,
                                                           const T* __restrict__ r, int N, int P,
                                                           ModeGeom<T> mg, double* __restrict__ part) {
  __shared__ double wsum[kK0Threads / 32][PMAX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a thread sums its few particles in T, the block sums in double
  T mom[PMAX];
#pragma unroll
  for (int n = 0; n < PMAX; ++n) mom[n] = T(0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const T x = cheb_x(r[3 * i + 2], mg);
    T qi = q[i];
    if (!isfinite(qi)) qi = T(0);
    T t0 = T(1), t1 = x;
#pragma unroll
    for (int n = 0; n < PMAX; ++n) {
      mom[n] += qi * t0;
      const T t2 = T(2) * x * t1 - t0;
      t0 = t1;
      t1 = t2;
    }
  }
#pragma unroll
  for (int n = 0; n < PMAX; ++n) {
    if (n < P) {
      double v;
      if constexpr (sizeof(T) == 4) {
        // warp sum as a float pair (two-sum at every level): FP64 precision
        // without warp-wide FP64 instructions
        float hi = mom[n], lo = 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
          const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
          const float sm = hi + h2, bv = sm - hi;
          lo += l2 + ((hi - (sm - bv)) + (h2 - bv));
          hi = sm;
        }
        v = (double)hi + (double)lo;
      } else {
        v = warp_sum((double)mom[n]);
      }
      if (lane == 0) wsum[warp][n] = v;
    }
  }
  __syncthreads();
  for (int n = threadIdx.x; n < P; n += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kK0Threads / 32; ++w) t += wsum[w][n];
    part[(size_t)blockIdx.x * P + n] = t;
  }
}

// Sum of nblk partials of stride P for entry n, by one warp in a fixed order.
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ part, int nblk,
                                                    int P, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * P + n];
  return warp_sum(s);
}

// mu_n = sum of the partial moments, nu = K0 mu; also the charge neutrality
// check of Eq. (2.4) from the binning partials.  One warp per entry.
__global__ void k_k0_finalize(const double* __restrict__ part, int nblk, int P,
                              const double* __restrict__ K0, double* __restrict__ nu,
                              const double* __restrict__ qred, int nblk_q, int* __restrict__ status) {
  __shared__ double mu[kMaxCheb];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int n = warp; n < P; n += nw) {
    const double v = warp_sum_partials(part, nblk, P, n);
    if (lane == 0) mu[n] = v;
  }
  if (warp == nw - 1 && qred) {
    const double sq = warp_sum_partials(qred, nblk_q, 2, 0);
    const double sa = warp_sum_partials(qred, nblk_q, 2, 1);
    if (lane == 0 && fabs(sq) > 1e-10 * sa) atomicOr(status, 1);
  }
  __syncthreads();
  for (int n = threadIdx.x; n < P; n += blockDim.x) {
    double s = 0.0;
    for (int m = 0; m < P; ++m) s += K0[n * P + m] * mu[m];
    nu[n] = s;
  }
}

// Float-pair arithmetic with ~48-bit significands (value + error term).
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return FF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF ff_add2(FF a, FF b) {
  const FF s = ff_two_sum(a.h, b.h);
  return ff_fast2(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ FF ff_mul2(FF a, FF b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return ff_fast2(p, e);
}
__device__ __forceinline__ FF ff_of(double v) {
  const float h = (float)v;
  return FF{h, (float)(v - (double)h)};
}

// The k = 0 potential and its z-derivative at every charge, Clenshaw sums of
// sum_n nu_n T_n(x) and sum_n (n+1) nu_(n+1) U_n(x), x = 2 z / Lz.  FP64
// plans sum in double; FP32 plans in float pairs (about 48-bit precision on
// the FP32 pipe, which this GPU runs at 64 times the FP64 rate): the k = 0
// part can be much larger than the total potential (in a thin slab it
// carries most of each charge's self-interaction), so FP32 alone would not do.
template <typename T>
__global__ void k_k0_eval(const T* __restrict__ r, int N, int P, double halfLz, float2 ihp,
                          const double* __restrict__ nu, double* __restrict__ phi_out,
                          double* __restrict__ grad_out) {
  __shared__ double snu[kMaxCheb], scd[kMaxCheb];
  __shared__ FF fnu[kMaxCheb], fcd[kMaxCheb];
  for (int n = threadIdx.x; n < P; n += blockDim.x) {
    snu[n] = nu[n];
    scd[n] = n + 1 < P ? (double)(n + 1) * nu[n + 1] : 0.0;  // T_n' = n U_(n-1)
    fnu[n] = ff_of(snu[n]);
    fcd[n] = ff_of(scd[n]);
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if constexpr (sizeof(T) == 4) {
    const float z = r[3 * i + 2];
    FF x = ff_mul2(FF{z, 0.0f}, FF{ihp.x, ihp.y});
    if (!(x.h >= -1.0f && x.h <= 1.0f)) x = isfinite(z) ? FF{x.h < 0.0f ? -1.0f : 1.0f, 0.0f} : FF{0.0f, 0.0f};
    const FF x2{2.0f * x.h, 2.0f * x.l};
    FF b1{0.0f, 0.0f}, b2{0.0f, 0.0f}, d1{0.0f, 0.0f}, d2{0.0f, 0.0f};
    for (int k = P - 1; k >= 1; --k) {
      const FF b0 = ff_add2(ff_add2(ff_mul2(x2, b1), FF{-b2.h, -b2.l}), fnu[k]);
      b2 = b1;
      b1 = b0;
      const FF d0 = ff_add2(ff_add2(ff_mul2(x2, d1), FF{-d2.h, -d2.l}), fcd[k - 1]);
      d2 = d1;
      d1 = d0;
    }
    const FF ph = ff_add2(ff_add2(ff_mul2(x, b1), FF{-b2.h, -b2.l}), fnu[0]);
    const FF gz = ff_mul2(d1, FF{ihp.x, ihp.y});
    phi_out[i] = (double)ph.h + (double)ph.l;
    grad_out[3 * i] = 0.0;
    grad_out[3 * i + 1] = 0.0;
    grad_out[3 * i + 2] = (double)gz.h + (double)gz.l;
  } else {
    double z = (double)r[3 * i + 2];
    if (!(z >= -halfLz && z <= halfLz)) z = isfinite(z) ? (z < 0 ? -halfLz : halfLz) : 0.0;
    const double ih = 1.0 / halfLz;
    const double x = z * ih, x2 = 2.0 * x;
    // Clenshaw: sum nu_n T_n(x) and sum (n+1) nu_(n+1) U_n(x)
    double b1 = 0.0, b2 = 0.0, d1 = 0.0, d2 = 0.0;
    for (int k = P - 1; k >= 1; --k) {
      const double b0 = fma(x2, b1, snu[k] - b2);
      b2 = b1;
      b1 = b0;
      const double d0 = fma(x2, d1, scd[k - 1] - d2);
      d2 = d1;
      d1 = d0;
    }
    phi_out[i] = fma(x, b1, snu[0] - b2);
    grad_out[3 * i] = 0.0;
    grad_out[3 * i + 1] = 0.0;
    grad_out[3 * i + 2] = d1 * ih;
  }
}

// ---------------------------------------------------------------------------
// 6. assembly and energy
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_assemble(const T* __restrict__ q, int N, const double* __restrict__ pp,
                           const double* __restrict__ pg, double selfsum, T* __restrict__ phi,
                           T* __restrict__ F, double* __restrict__ part) {
  __shared__ double sh[32];
  double e = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double qi = (double)q[i];
    if (!isfinite(qi)) qi = 0.0;
    const double ph = pp[i] + pp[N + i] + pp[2 * (size_t)N + i] + pp[3 * (size_t)N + i] - qi * selfsum;
    double g[3];
    for (int d = 0; d < 3; ++d)
      g[d] = pg[3 * i + d] + pg[3 * ((size_t)N + i) + d] + pg[3 * (2 * (size_t)N + i) + d] +
             pg[3 * (3 * (size_t)N + i) + d];
    if (phi) phi[i] = (T)ph;
    if (F)
      for (int d = 0; d < 3; ++d) F[3 * i + d] = (T)(-qi * g[d]);
    e += qi * ph;
  }
  const double t = block_sum(e, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_energy(const double* __restrict__ part, int nblk, double* __restrict__ E) {
  if (threadIdx.x < 32) {
    const double v = warp_sum_partials(part, nblk, 1, 0);
    if (threadIdx.x == 0) *E = 0.5 * v;
  }
}

// ---------------------------------------------------------------------------
// host side of one evaluation: the launch sequence
// ---------------------------------------------------------------------------

// Window supports with dedicated (unrolled) kernels; others use the generic
// instantiation (PW = 0).
// Support of the kernel instantiation a window runs on: the KB window runs on
// the run-time-support kernels (0), the others on their fixed support.
static int pw_dispatch(const WinPar& w) { return w.kind == SOG_WIN_KB ? 0 : w.P; }

#define SOG_DISPATCH_PW(P_, KER, GRID, SMEM, STREAM, ...)                 \
  do {                                                                     \
    switch (P_) {                                                          \
      case 6: KER<T, 6><<<GRID, 256, SMEM, STREAM>>>(__VA_ARGS__); break;   \
      case 8: KER<T, 8><<<GRID, 256, SMEM, STREAM>>>(__VA_ARGS__); break;   \
      case 9: KER<T, 9><<<GRID, 256, SMEM, STREAM>>>(__VA_ARGS__); break;   \
      case 12: KER<T, 12><<<GRID, 256, SMEM, STREAM>>>(__VA_ARGS__); break; \
      default: KER<T, 0><<<GRID, 256, SMEM, STREAM>>>(__VA_ARGS__); break;  \
    }                                                                      \
  } while (0)

// Opt a kernel in to the largest dynamic shared memory its static shared
// memory leaves free.
template <typename K>
static cudaError_t allow_smem(K* kernel) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kMaxDynSmem - (int)a.sharedSizeBytes);
}

template <typename T, int PW>
static cudaError_t allow_pw() {
  cudaError_t e = allow_smem(k_mid_spread<T, PW>);
  if (e == cudaSuccess) e = allow_smem(k_mid_gather<T, PW>);
  if (e == cudaSuccess) e = allow_smem(k_long_spread<T, PW>);
  if (e == cudaSuccess) e = allow_smem(k_long_gather<T, PW>);
  return e;
}

size_t mid_smem(const sog_plan* p, size_t es, bool gather) {
  const TileGeom& g = p->gm;
  const int P = p->wm.P;
  const int rp = gather_row_pitch(g.W[0]);
  const size_t tile = (size_t)g.W[2] * gather_plane_stride(rp, g.W[1], P);
  if (gather)  // per-warp window values (w, w') and the tile
    return kGatherHeader + ((size_t)kTileThreads / 32 * 3 * kMaxWin * 2 + tile) * es;
  // fixed-point tile: int32 for FP32, int64 for FP64 (same size as T)
  return kTileHeader + ((size_t)kTileBatch * 3 * kMaxWin + tile) * es;
}
size_t long_smem(const sog_plan* p, size_t es, bool gather) {
  const TileGeom& g = p->gl;
  const int P = p->prm.P_cheb;
  const int rp = gather_row_pitch(g.W[0]);
  const size_t tile = (size_t)P * gather_plane_stride(rp, g.W[1], p->wl.P);
  const size_t pw = (size_t)p->wl.P;
  // gathering: staged window values and derivatives, T_n and T_n', the tile
  // (sized by the plan's support and P_cheb: the smaller footprint lets
  // three CTAs share an SM)
  if (gather) return kLongSpreadHeader + ((size_t)kTileBatch * (4 * pw + 2 * P) + tile) * es;
  // gridding: staged window values and T_n, then the fixed-point tile (int32
  // for FP32, int64 for FP64: the size of T)
  return kLongSpreadHeader + ((size_t)kTileBatch * (2 * pw + P) + tile) * es;
}

#define SOG_CK(x)                      \
  do {                                 \
    cudaError_t e_ = (x);              \
    if (e_ != cudaSuccess) return e_;  \
  } while (0)

// Stage timers: event 2k at the start of stage k, 2k+1 at its end, on the
// stream the stage runs on.  Inside a graph the records are external nodes.
static void mark_ev(sog_plan* p, int idx, cudaStream_t s) {
  if (!p->timing) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(p->ev[idx], s, cudaEventRecordExternal);
  else
    cudaEventRecord(p->ev[idx], s);
  p->ev_used[idx] = 1;
}
static void mark_begin(sog_plan* p, int stage, cudaStream_t s) { mark_ev(p, 2 * stage, s); }
static void mark_end(sog_plan* p, int stage, cudaStream_t s) { mark_ev(p, 2 * stage + 1, s); }

#define LAUNCH_CHECK()                 \
  do {                                 \
    ++p->launches;                     \
    SOG_CK(cudaGetLastError());        \
  } while (0)

// Smallest float >= v, largest float <= v, and v as float plus remainder.
static float float_ceil(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}
static float float_floor(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}
static float2 float_pair(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

template <typename T>
static cudaError_t eval_t(sog_plan* p, const T* q, const T* r, T* phi, double* E, T* F,
                         double* pp, double* pg, cudaStream_t s) {
  p->launches = 0;
  for (int i = 0; i < 2 * SOG_NSTAGES; ++i) p->ev_used[i] = 0;
  const int N = (int)p->N;
  const sog_params& m = p->prm;
  PrepGeom g{};
  for (int d = 0; d < 3; ++d) {
    g.L[d] = m.L[d];
    g.halfL[d] = 0.5 * m.L[d];
    g.nc[d] = p->nc[d];
    g.icell[d] = 1.0 / p->cell[d];
    g.ih[d] = p->has_mid ? 1.0 / p->h[d] : 0.0;
    g.h[d] = p->has_mid ? p->h[d] : 1.0;
    g.Tm[d] = p->gm.T[d];
    g.ntm[d] = p->gm.nt[d];
    g.iTm[d] = p->has_mid ? 1.0 / p->gm.T[d] : 0.0;
  }
  const int long_bins = p->has_long && !p->long_direct;  // direct sums need no tiles
  g.has_mid = p->has_mid;
  g.has_long = long_bins;
  g.Lzs_half = 0.5 * p->Lzs;
  for (int d = 0; d < 2; ++d) {
    g.ihl[d] = p->has_long ? 1.0 / p->hl[d] : 0.0;
    g.hl[d] = long_bins ? p->hl[d] : 1.0;
    g.Tl[d] = p->gl.T[d];
    g.ntl[d] = p->gl.nt[d];
    g.iTl[d] = p->has_long ? 1.0 / p->gl.T[d] : 0.0;
  }
  g.ihalfLz = 2.0 / m.L[2];
  // float forms for FP32 plans
  for (int d = 0; d < 2; ++d) {
    g.wrap_hi[d] = float_ceil(g.halfL[d]);
    g.wrap_lo[d] = float_ceil(-g.halfL[d]);
  }
  g.z_lo = float_ceil(-g.halfL[2]);
  g.z_hi = float_floor(g.halfL[2]);
  for (int d = 0; d < 3; ++d) {
    g.halfLf[d] = (float)g.halfL[d];
    g.halfLp[d] = float_pair(g.halfL[d]);
    g.icellp[d] = float_pair(g.icell[d]);
    g.ihp[d] = float_pair(g.ih[d]);
    g.iTmp[d] = float_pair(g.iTm[d]);
  }
  g.Lzs_halfp = float_pair(g.Lzs_half);
  for (int d = 0; d < 2; ++d) {
    g.ihlp[d] = float_pair(g.ihl[d]);
    g.iTlp[d] = float_pair(g.iTl[d]);
  }
  g.ihalfLzp = float_pair(g.ihalfLz);
  const int3 off = make_int3(p->cnt_off[0], p->cnt_off[1], p->cnt_off[2]);
  const int3 nb = make_int3(p->n_cells, p->has_mid ? p->n_tiles_mid : 0,
                            long_bins ? p->n_tiles_long : 0);
  P4<T>* rn = reinterpret_cast<P4<T>*>(p->d_rec_near);
  P4<T>* rm = reinterpret_cast<P4<T>*>(p->d_rec_mid);
  P4<T>* rl = reinterpret_cast<P4<T>*>(p->d_rec_long);

  // 1. binning
  mark_begin(p, 0, s);
  SOG_CK(cudaMemsetAsync(p->d_cnt, 0, sizeof(int) * p->cnt_off[3], s));
  P4<T>* tmp = reinterpret_cast<P4<T>*>(p->d_rec_tmp);
  k_bin_count<T><<<p->red_blocks, 256, 0, s>>>(g, q, r, N, p->d_key, p->d_rank, p->d_cnt, off, tmp,
                                           p->d_red, p->d_status);
  LAUNCH_CHECK();
  k_scan3<<<3, 1024, 0, s>>>(p->d_cnt, off, nb);
  LAUNCH_CHECK();
  k_bin_scatter<T><<<(N + 255) / 256, 256, 0, s>>>(N, p->has_mid, long_bins, p->d_key,
                                                   p->d_rank, p->d_cnt, off, tmp, rn, rm, rl,
                                                   p->d_perm);
  LAUNCH_CHECK();
  mark_end(p, 0, s);

  // 2. near field
  NearGeom ng{};
  for (int d = 0; d < 3; ++d) {
    ng.halfL[d] = 0.5 * m.L[d];
    ng.cell[d] = p->cell[d];
    ng.nc[d] = p->nc[d];
  }
  ng.L[0] = m.L[0];
  ng.L[1] = m.L[1];
  ng.rc = m.rc;
  ng.K = p->near_K;
  ng.D = p->near_D;
  near_consts<float>(ng, ng.cf);
  near_consts<double>(ng, ng.cd);
  // the near field depends only on the binning: fork it onto the side stream
  // timing mode 2: every stage on the caller's stream, one after another
  const bool serial = p->timing == 2;
  const cudaStream_t sn = serial ? s : p->side_stream;
  SOG_CK(cudaEventRecord(p->ev_fork, s));
  SOG_CK(cudaStreamWaitEvent(sn, p->ev_fork, 0));
  mark_begin(p, 1, sn);
  k_near<T><<<p->n_cells, kNearThreads, 0, sn>>>(ng, rn, p->d_cnt + off.x, p->d_perm,
                                                 reinterpret_cast<const T*>(p->d_near_tab), pp, pg);
  LAUNCH_CHECK();
  mark_end(p, 1, sn);
  SOG_CK(cudaEventRecord(p->ev_join, sn));

  // 3. mid range
  if (p->has_mid) {
    mark_begin(p, 2, s);
    T* grid = reinterpret_cast<T*>(p->d_grid);
    const size_t gbytes = (size_t)m.I[2] * m.I[1] * (m.I[0] + 2) * sizeof(T);
    SOG_CK(cudaMemsetAsync(grid, 0, gbytes, s));
    const WinT<T> w = wint<T>(p->wm);
    const size_t sm = mid_smem(p, sizeof(T), false);
    const dim3 mgrid(p->n_tiles_mid, p->gm.chunks);
    SOG_DISPATCH_PW(pw_dispatch(p->wm), k_mid_spread, mgrid, sm, s, p->gm, w, rm, p->d_cnt + off.y, grid);
    LAUNCH_CHECK();
    mark_end(p, 2, s);
    mark_begin(p, 3, s);
    int nl = 0;
    SOG_CK(fft_mid_forward_conv_inverse<T>(p, s, nl));
    p->launches += nl;
    mark_end(p, 3, s);
    mark_begin(p, 4, s);
    const size_t sm2 = mid_smem(p, sizeof(T), true);
    const double3 invh = make_double3(1.0 / p->h[0], 1.0 / p->h[1], 1.0 / p->h[2]);
    SOG_DISPATCH_PW(pw_dispatch(p->wm), k_mid_gather, mgrid, sm2, s, p->gm, w, rm, p->d_cnt + off.y,
                    p->d_perm + N, grid, invh, pp + N, pg + 3 * (size_t)N);
    LAUNCH_CHECK();
    mark_end(p, 4, s);
  } else {
    SOG_CK(cudaMemsetAsync(pp + N, 0, sizeof(double) * N, s));
    SOG_CK(cudaMemsetAsync(pg + 3 * (size_t)N, 0, sizeof(double) * 3 * N, s));
  }

  // 4. long range on long_stream and 5. its k = 0 mode on k0_stream, after
  // the binning
  // (the direct sums and the k = 0 moments could start with the evaluation,
  // but measured no faster: they compete with the binning that every other
  // part waits for)
  const cudaStream_t sl = serial ? s : p->long_stream;
  SOG_CK(cudaStreamWaitEvent(sl, p->ev_fork, 0));
  bool k0_branch = false;
  if (p->has_long && p->long_direct) {
    const int P = m.P_cheb, Kx = (m.I_long[0] - 1) / 2, Ky = (m.I_long[1] - 1) / 2;
    const int nh = p->n_half;
    const int pmax = P <= 16 ? 16 : (P <= 32 ? 32 : 64);
    // staging batch: kModeBatch particles, fewer if their tables would not fit
    const size_t per_part = (size_t)(pmax + 2 * (Kx + 1) + 2 * (2 * Ky + 1)) * sizeof(T);
    int nbt = kModeBatch;
    while (nbt > 8 && (size_t)nbt * per_part > (size_t)kMaxDynSmem) nbt /= 2;
    const size_t sm1 = std::max((size_t)nbt * per_part,
                                (size_t)kModeThreads * kModeRed * 2 * sizeof(T));
    const size_t sm3 = (size_t)nh * P * 2 * sizeof(T);
    const ModeGeom<T> mg = mode_geom<T>(m.L[0], m.L[1], m.L[2]);
    T* lmom = reinterpret_cast<T*>(p->d_lmom);  // per-block moments in the element type
    mark_begin(p, 5, sl);
    if (pmax == 16)
      k_lmodes_moments<T, 16><<<p->mode_blocks, kModeThreads, sm1, sl>>>(q, r, N, P, Kx, Ky, nh, nbt, mg, lmom);
    else if (pmax == 32)
      k_lmodes_moments<T, 32><<<p->mode_blocks, kModeThreads, sm1, sl>>>(q, r, N, P, Kx, Ky, nh, nbt, mg, lmom);
    else
      k_lmodes_moments<T, 64><<<p->mode_blocks, kModeThreads, sm1, sl>>>(q, r, N, P, Kx, Ky, nh, nbt, mg, lmom);
    LAUNCH_CHECK();
    mark_end(p, 5, sl);
    mark_begin(p, 6, sl);
    k_lmodes_coeffs<T><<<nh, kCoefThreads, 0, sl>>>(lmom, p->mode_blocks, nh, P,
                                                     reinterpret_cast<const T*>(p->d_kmat),
                                                     reinterpret_cast<T*>(p->d_lcoef));
    LAUNCH_CHECK();
    mark_end(p, 6, sl);
    mark_begin(p, 7, sl);
    const T* cf = reinterpret_cast<const T*>(p->d_lcoef);
    if (pmax == 16)
      k_lmodes_eval<T, 16><<<(N + kModeThreads - 1) / kModeThreads, kModeThreads, sm3, sl>>>(r, N, P, Kx, Ky, nh, mg, cf, pp + 2 * (size_t)N, pg + 6 * (size_t)N);
    else if (pmax == 32)
      k_lmodes_eval<T, 32><<<(N + kModeThreads - 1) / kModeThreads, kModeThreads, sm3, sl>>>(r, N, P, Kx, Ky, nh, mg, cf, pp + 2 * (size_t)N, pg + 6 * (size_t)N);
    else
      k_lmodes_eval<T, 64><<<(N + kModeThreads - 1) / kModeThreads, kModeThreads, sm3, sl>>>(r, N, P, Kx, Ky, nh, mg, cf, pp + 2 * (size_t)N, pg + 6 * (size_t)N);
    LAUNCH_CHECK();
    mark_end(p, 7, sl);
  }
  if (p->has_long) {
    const int P = m.P_cheb;
    if (!p->long_direct) {
    mark_begin(p, 5, sl);
    T* A = reinterpret_cast<T*>(p->d_lA);
    const WinT<T> w = wint<T>(p->wl);
    if (p->long_small) {
      const int I0 = m.I_long[0], I1 = m.I_long[1];
      T* part = reinterpret_cast<T*>(p->d_long_partial);
      if (P <= 16)
        k_long_spread_small<T, 16><<<p->long_small_blocks, 256, 0, sl>>>(I0, I1, w, P, rl, N, part);
      else if (P <= 32)
        k_long_spread_small<T, 32><<<p->long_small_blocks, 256, 0, sl>>>(I0, I1, w, P, rl, N, part);
      else
        k_long_spread_small<T, 64><<<p->long_small_blocks, 256, 0, sl>>>(I0, I1, w, P, rl, N, part);
      LAUNCH_CHECK();
      const int tot = P * I0 * I1;
      k_long_reduce<T><<<(8 * tot + 255) / 256, 256, 0, sl>>>(
          reinterpret_cast<const T*>(p->d_long_partial), p->long_small_blocks, I0, I1, P, A);
      LAUNCH_CHECK();
    } else {
      const size_t pbytes = (size_t)P * m.I_long[1] * (m.I_long[0] + 2) * sizeof(T);
      SOG_CK(cudaMemsetAsync(A, 0, pbytes, sl));
      const size_t sm = long_smem(p, sizeof(T), false);
      const dim3 lgrid(p->n_tiles_long, p->gl.chunks);
      SOG_DISPATCH_PW(pw_dispatch(p->wl), k_long_spread, lgrid, sm, sl, p->gl, w, P, rl, p->d_cnt + off.z, A);
      LAUNCH_CHECK();
    }
    mark_end(p, 5, sl);
    mark_begin(p, 6, sl);
    int nl = 0;
    SOG_CK(fft_long_solve<T>(p, sl, nl));
    p->launches += nl;
    mark_end(p, 6, sl);
    mark_begin(p, 7, sl);
    const size_t sm2 = long_smem(p, sizeof(T), true);
    const double3 sc = make_double3(1.0 / p->hl[0], 1.0 / p->hl[1], 2.0 / m.L[2]);
    const dim3 lgrid2(p->n_tiles_long, p->gl.chunks);
    SOG_DISPATCH_PW(pw_dispatch(p->wl), k_long_gather, lgrid2, sm2, sl, p->gl, w, P, rl, p->d_cnt + off.z,
                    p->d_perm + 2 * (size_t)N, A, sc, pp + 2 * (size_t)N, pg + 6 * (size_t)N);
    LAUNCH_CHECK();
    mark_end(p, 7, sl);
    }
    // the k = 0 mode needs only the charges: its own branch (k0_stream),
    // running beside the near field and the gridded long range
    const cudaStream_t sk = serial ? s : p->k0_stream;
    SOG_CK(cudaStreamWaitEvent(sk, p->ev_fork, 0));
    {
    mark_begin(p, 8, sk);
    const int P = m.P_cheb;
    double* mpart = p->d_red + 2 * p->red_blocks;
    const ModeGeom<T> mg0 = mode_geom<T>(m.L[0], m.L[1], m.L[2]);
    if (P <= 16)
      k_k0_moments<T, 16><<<p->k0_blocks, kK0Threads, 0, sk>>>(q, r, N, P, mg0, mpart);
    else if (P <= 32)
      k_k0_moments<T, 32><<<p->k0_blocks, kK0Threads, 0, sk>>>(q, r, N, P, mg0, mpart);
    else
      k_k0_moments<T, 64><<<p->k0_blocks, kK0Threads, 0, sk>>>(q, r, N, P, mg0, mpart);
    LAUNCH_CHECK();
    }
    k_k0_finalize<<<1, 1024, 0, sk>>>(p->d_red + 2 * p->red_blocks, p->k0_blocks, P, p->d_k0mat,
                                     p->d_k0nu, p->d_red, p->red_blocks, p->d_status);
    LAUNCH_CHECK();
    k_k0_eval<T><<<(N + 255) / 256, 256, 0, sk>>>(r, N, P, 0.5 * m.L[2], float_pair(2.0 / m.L[2]),
                                                p->d_k0nu, pp + 3 * (size_t)N, pg + 9 * (size_t)N);
    LAUNCH_CHECK();
    mark_end(p, 8, sk);
    SOG_CK(cudaEventRecord(p->ev_join_k0, sk));
    k0_branch = true;
  } else {
    SOG_CK(cudaMemsetAsync(pp + 2 * (size_t)N, 0, sizeof(double) * 2 * N, sl));
    SOG_CK(cudaMemsetAsync(pg + 6 * (size_t)N, 0, sizeof(double) * 6 * N, sl));
    k_k0_finalize<<<1, 1024, 0, sl>>>(p->d_red + 2 * p->red_blocks, p->k0_blocks, 0, p->d_k0mat,
                                     p->d_k0nu, p->d_red, p->red_blocks, p->d_status);
    LAUNCH_CHECK();
  }

  SOG_CK(cudaEventRecord(p->ev_join_long, sl));

  // join the near field and the long range, then 6. assembly
  SOG_CK(cudaStreamWaitEvent(s, p->ev_join, 0));
  SOG_CK(cudaStreamWaitEvent(s, p->ev_join_long, 0));
  if (k0_branch) SOG_CK(cudaStreamWaitEvent(s, p->ev_join_k0, 0));
  mark_begin(p, 9, s);
  if (phi || F || E) {
    double* epart = p->d_red + 2 * p->red_blocks + (size_t)p->red_blocks * kMaxCheb;
    k_assemble<T><<<p->red_blocks, 256, 0, s>>>(q, N, pp, pg, p->selfsum, phi, F, epart);
    LAUNCH_CHECK();
    if (E) {
      k_energy<<<1, 32, 0, s>>>(epart, p->red_blocks, E);
      LAUNCH_CHECK();
    }
  }
  mark_end(p, 9, s);
  return cudaSuccess;
}

template <typename T>
static cudaError_t prepare_t() {
  {
    cudaError_t e0 = allow_smem(k_lmodes_moments<T, 16>);
    if (e0 == cudaSuccess) e0 = allow_smem(k_lmodes_moments<T, 32>);
    if (e0 == cudaSuccess) e0 = allow_smem(k_lmodes_moments<T, 64>);
    if (e0 == cudaSuccess) e0 = allow_smem(k_lmodes_eval<T, 16>);
    if (e0 == cudaSuccess) e0 = allow_smem(k_lmodes_eval<T, 32>);
    if (e0 == cudaSuccess) e0 = allow_smem(k_lmodes_eval<T, 64>);
    if (e0 != cudaSuccess) return e0;
  }
  cudaError_t e = allow_pw<T, 0>();
  if (e == cudaSuccess) e = allow_pw<T, 6>();
  if (e == cudaSuccess) e = allow_pw<T, 8>();
  if (e == cudaSuccess) e = allow_pw<T, 9>();
  if (e == cudaSuccess) e = allow_pw<T, 12>();
  if (e == cudaSuccess) e = fft_prepare<T>();
  return e;
}

cudaError_t prepare_kernels(int prec) {
  return prec == SOG_PREC_FP64 ? prepare_t<double>() : prepare_t<float>();
}

static cudaError_t eval_direct(sog_plan* p, const void* q, const void* r, void* phi, double* E,
                               void* F, double* pp, double* pg, cudaStream_t s) {
  if (p->prec == SOG_PREC_FP64)
    return eval_t<double>(p, (const double*)q, (const double*)r, (double*)phi, E, (double*)F, pp,
                          pg, s);
  return eval_t<float>(p, (const float*)q, (const float*)r, (float*)phi, E, (float*)F, pp, pg, s);
}

cudaError_t enqueue_eval(sog_plan* p, const void* q, const void* r, void* phi, double* E, void* F,
                         cudaStream_t s) {
  const cudaError_t e = eval_direct(p, q, r, phi, E, F, p->d_parts_phi, p->d_parts_grad, s);
  p->last_stream = s;
  return e;
}

void release_graphs(sog_plan* p) {
  for (int i = 0; i < p->n_graphs; ++i) cudaGraphExecDestroy(p->graphs[i].exec);
  p->n_graphs = 0;
}

// Replays a captured graph of the whole evaluation for this set of caller
// pointers (and timing mode), capturing it on the plan's private stream the
// first time.  With timing on, the stage events are part of the graph.
static cudaError_t eval_graph(sog_plan* p, const void* q, const void* r, void* phi, double* E,
                              void* F, double* pp, double* pg, cudaStream_t s) {
  GraphEntry* hit = nullptr;
  for (int i = 0; i < p->n_graphs; ++i) {
    GraphEntry& g = p->graphs[i];
    if (g.q == q && g.r == r && g.phi == phi && g.E == E && g.F == F && g.pp == pp &&
        g.pg == pg && g.timing == p->timing) {
      hit = &g;
      break;
    }
  }
  if (!hit) {
    int slot = p->n_graphs;
    if (slot == kMaxGraphs) {
      slot = 0;
      for (int i = 1; i < kMaxGraphs; ++i)
        if (p->graphs[i].last_use < p->graphs[slot].last_use) slot = i;
      // the evicted graph may still be running on the caller's stream
      cudaStreamSynchronize(p->last_stream);
      cudaGraphExecDestroy(p->graphs[slot].exec);
      // move the last entry into the hole so entries stay contiguous
      p->graphs[slot] = p->graphs[p->n_graphs - 1];
      slot = --p->n_graphs;
    }
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t e1 = eval_direct(p, q, r, phi, E, F, pp, pg, p->cap_stream);
    e = cudaStreamEndCapture(p->cap_stream, &graph);
    if (e1 != cudaSuccess || e != cudaSuccess) {
      if (e == cudaSuccess) cudaGraphDestroy(graph);
      return e1 != cudaSuccess ? e1 : e;
    }
    GraphEntry& g = p->graphs[slot];
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    ++p->n_graphs;
    g.q = q;
    g.r = r;
    g.phi = phi;
    g.E = E;
    g.F = F;
    g.pp = pp;
    g.pg = pg;
    g.timing = p->timing;
    for (int i = 0; i < 2 * SOG_NSTAGES; ++i) g.ev_used[i] = p->ev_used[i];
    g.launches = p->launches;
    hit = &g;
  }
  hit->last_use = ++p->use_clock;
  p->launches = hit->launches;
  for (int i = 0; i < 2 * SOG_NSTAGES; ++i) p->ev_used[i] = hit->ev_used[i];
  return cudaGraphLaunch(hit->exec, s);
}

sog_status eval_device(sog_plan* p, const void* q, const void* r, void* phi, double* E, void* F,
                       double* phi_parts, double* grad_parts, cudaStream_t s) {
  double* pp = phi_parts ? phi_parts : p->d_parts_phi;
  double* pg = grad_parts ? grad_parts : p->d_parts_grad;
  const cudaError_t e = p->use_graphs ? eval_graph(p, q, r, phi, E, F, pp, pg, s)
                                      : eval_direct(p, q, r, phi, E, F, pp, pg, s);
  p->last_stream = s;
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->launch_error = 1;
    return SOG_ERR_CUDA;
  }
  return SOG_OK;
}

}  // namespace sogk
