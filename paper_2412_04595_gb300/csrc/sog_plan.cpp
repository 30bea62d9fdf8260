// Host side of the GB300 SOG library: parameter selection (Sec. 4.3), the
// FP64 tables every evaluation reads, device memory, and the C ABI of sog.h.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sog_internal.h"

namespace sogk {

// w_l of Eq. (2.22), w_0 scaled by omega (Eq. 2.25).
double sog_weight(double b, double sigma, double omega, int l) {
  const double w = pow(3.14159265358979323846 / 2.0, -0.5) * pow(b, -(double)l) / sigma * log(b);
  return l == 0 ? w * omega : w;
}

// w_l and s_l of Eq. (2.22), w_0 scaled by omega (Eq. 2.25).
void sog_table(double b, double sigma, double omega, int M, std::vector<double>& w,
               std::vector<double>& s) {
  w.resize(M + 1);
  s.resize(M + 1);
  for (int l = 0; l <= M; ++l) {
    w[l] = sog_weight(b, sigma, omega, l);
    s[l] = sqrt(2.0) * pow(b, (double)l) * sigma;
  }
}

}  // namespace sogk

using sogk::sog_table;

namespace {

const double kPi = 3.14159265358979323846;

// Table 1 (Sec. 2.3): b, r0, omega, energy error, M.
const double kTable1[6][5] = {
    {2.0, 1.9892536839080267, 0.9944464927622323, 3.12e-2, 16},
    {1.62976708826776469, 2.7520026668023417, 1.0078069793438068, 2.33e-3, 31},
    {1.48783512395703226, 3.7554672283554990, 0.9919117057598183, 2.29e-4, 46},
    {1.32070036405934420, 4.3914554711638349, 1.0018891411481198, 1.18e-6, 76},
    {1.21812525709410644, 5.6355288151271085, 1.0009014615603334, 7.14e-10, 166},
    {1.14878150173321925, 7.2956245490719404, 1.0000368348358225, 1.30e-15, 271},
};

int fft_size(long n) {
  if (n < 8) n = 8;
  n = (n + 7) / 8 * 8;
  for (;; n += 8) {
    long k = n;
    for (int p : {2, 3, 5, 7})
      while (k % p == 0) k /= p;
    if (k == 1) return (int)n;
  }
}

long clog2(long n) {
  long v = n - 1;
  long b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b < 1 ? 1 : b;
}

// Inverse of erfc on (0, 2) by bisection then Newton, to double rounding.
double erfcinv(double y) {
  double lo = -30.0, hi = 30.0;
  for (int i = 0; i < 200; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (erfc(mid) > y) lo = mid;
    else hi = mid;
  }
  double x = 0.5 * (lo + hi);
  for (int i = 0; i < 3; ++i) {
    const double f = erfc(x) - y;
    const double d = -2.0 / sqrt(kPi) * exp(-x * x);
    if (d == 0.0) break;
    x -= f / d;
  }
  return x;
}

double shape_default(int window, int P) {
  if (window == SOG_WIN_ES) return 1.9 * P;
  if (window == SOG_WIN_KB) return 2.0 * P;
  return 0.35 * kPi * P;  // Gaussian, on grids that are not upsampled
}

sog_status select_params(int64_t N, double Lx, double Ly, double Lz, double tol, int window,
                         double n_nb, sog_params* out) {
  int row = 5;
  for (int i = 0; i < 6; ++i)
    if (kTable1[i][3] <= 1.5 * tol) {
      row = i;
      break;
    }
  const double b = kTable1[row][0], r0 = kTable1[row][1], omega = kTable1[row][2];
  const int M_tab = (int)kTable1[row][4];
  const double rho = (double)N / (Lx * Ly * Lz);
  const double A = Lx * Ly;
  const double eps = 0.3 * tol;
  const double phis = pow(rho, 1.0 / 3.0);
  double rc = pow(3.0 * n_nb / (4.0 * kPi * rho), 1.0 / 3.0);
  rc = std::min(rc, 0.5 * std::min(Lx, Ly));
  const double sigma = rc / r0;
  const double cw = pow(kPi / 2.0, -0.5) * log(b) / sigma;
  int M = M_tab;
  const double lmax = std::max(Lx, std::max(Ly, Lz));
  for (;;) {
    const double tail = cw * pow(b, -(double)(M + 1)) / (1.0 - 1.0 / b);
    const double s_next = sqrt(2.0) * pow(b, (double)(M + 1)) * sigma;
    if (kPi * rho * pow(Lz, 3) / sqrt((double)N) * tail <= 0.1 * eps * phis && s_next >= 20.0 * lmax)
      break;
    ++M;
    if (M > 2000) return SOG_ERR_PARAMS;
  }
  std::vector<double> w, s;
  sog_table(b, sigma, omega, M, w, s);
  // window error erfc(C sqrt(P)): ES and KB 1.226 (Sec. 5.1); Gaussian 0.95
  // on grids that are not upsampled
  const double C = window == SOG_WIN_GAUSS ? 0.95 : 1.226;
  int P_win = (int)ceil(pow(erfcinv(eps) / C, 2));
  P_win = std::min(std::max(P_win, 4), 16);
  const double lne = log(1.0 / eps);

  bool have = false;
  long best_cost = 0;
  int bm = 0, bI[3] = {0, 0, 0}, bPw = 0, bIl[2] = {0, 0}, bPl = 0, bPc = 0, bdirect = 0;
  double bhz = 0.0;
  for (int m = -1; m <= M; ++m) {
    long cost = 0;
    int Ix = 0, Iy = 0, Izs = 0, Pw = 0;
    double hz = 0.0;
    if (m >= 0) {
      const double K = 2.0 * sqrt(lne) / s[0];
      const double nx = ceil(K * Lx / kPi), ny = ceil(K * Ly / kPi);
      const double Izb = std::max(1.0, ceil(Lz * K / kPi));
      hz = Lz / Izb;
      Pw = P_win;
      const double Hz = 0.5 * (Pw - 1) * hz;
      // KB decays slowly towards its support's edge: 2.6 H_z of padding (Sec. 3.4)
      const double pad = std::max((window == SOG_WIN_KB ? 2.6 : 2.0) * Hz, s[m] * sqrt(lne));
      const double nz = ceil((Lz + pad) / hz);
      if (nz > 8192 || nx > 4096 || ny > 4096) continue;
      Ix = fft_size((long)nx);
      Iy = fft_size((long)ny);
      Izs = fft_size((long)nz);
      Pw = std::min(P_win, std::min(Ix, Iy));
      const long G = (long)Ix * Iy * Izs;
      cost += 4 * N * (long)Pw * Pw * Pw + 10 * G * clog2(G);
    }
    int Ilx = 0, Ily = 0, Pl = 0, Pc = 0, direct = 0;
    if (m < M) {
      const double s1 = s[m + 1];
      const double Kl = 2.0 * sqrt(lne) / s1;
      const double nx = std::max(ceil(Kl * Lx / kPi), (double)(P_win + 4));
      const double ny = std::max(ceil(Kl * Ly / kPi), (double)(P_win + 4));
      if (nx > 4096 || ny > 4096) continue;
      Ilx = fft_size((long)nx);
      Ily = fft_size((long)ny);
      Pl = P_win;
      for (int P = 2; P <= 64; ++P) {
        double err = 0.0;
        const double lg = 0.5 * lgamma(P + 1.0);
        for (int l = m + 1; l <= M; ++l) {
          const double amp = w[l] * std::max(1.0, kPi * s[l] * s[l] / A);
          const double x = 2.0 * sqrt(2.0) * s[l] / Lz;
          err += amp * exp(-P * log(x) - lg);
        }
        if (2.0 * err <= eps * phis) {
          Pc = P;
          break;
        }
      }
      if (Pc == 0) continue;
      const long Gl = (long)Ilx * Ily;
      const long cost_grid = 4 * N * (long)Pl * Pl * Pc + 10 * Gl * Pc * clog2(Gl) +
                             2 * Gl * (long)Pc * Pc + N * (long)Pc;
      // Algorithm 3: direct sums over the modes |k| <= Kl (no window, no FFT)
      const long Kdx = (long)ceil(Kl * Lx / (2.0 * kPi)), Kdy = (long)ceil(Kl * Ly / (2.0 * kPi));
      const long nhalf = Kdy + Kdx * (2 * Kdy + 1);
      const long cost_direct = 4 * N * nhalf * (long)Pc;
      if (nhalf >= 1 && nhalf <= sogk::kMaxHalfModes &&
          nhalf * Pc <= sogk::kMaxHalfModeCoefs && cost_direct < cost_grid) {
        direct = 1;
        Ilx = (int)(2 * Kdx + 1);
        Ily = (int)(2 * Kdy + 1);
        cost += cost_direct;
      } else {
        cost += cost_grid;
      }
    }
    if (!have || cost < best_cost) {
      have = true;
      best_cost = cost;
      bm = m;
      bI[0] = Ix;
      bI[1] = Iy;
      bI[2] = Izs;
      bhz = hz;
      bPw = Pw;
      bIl[0] = Ilx;
      bIl[1] = Ily;
      bPl = Pl;
      bPc = Pc;
      bdirect = direct;
    }
  }
  if (!have) return SOG_ERR_PARAMS;
  memset(out, 0, sizeof(*out));
  out->L[0] = Lx;
  out->L[1] = Ly;
  out->L[2] = Lz;
  out->b = b;
  out->r0 = r0;
  out->omega = omega;
  out->sigma = sigma;
  out->rc = rc;
  out->M = M;
  out->m = bm;
  for (int d = 0; d < 3; ++d) out->I[d] = bI[d];
  out->hz = bhz;
  out->P_win = bPw ? bPw : 4;
  out->shape = shape_default(window, out->P_win);
  out->I_long[0] = bIl[0];
  out->I_long[1] = bIl[1];
  out->P_long = bPl ? bPl : 4;
  out->shape_long = shape_default(window, out->P_long);
  out->P_cheb = bPc;
  out->window = window;
  out->long_direct = bdirect;
  out->win_poly = 0;
  return SOG_OK;
}

bool smooth_even(int n) {
  if (n < 2 || n % 2) return false;
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

sog_status check_params(const sog_params& p) {
  for (int d = 0; d < 3; ++d)
    if (!(p.L[d] > 0.0) || !isfinite(p.L[d])) return SOG_ERR_ARG;
  if (!(p.b > 1.0) || !(p.sigma > 0.0) || !(p.rc > 0.0) || !(p.omega > 0.0)) return SOG_ERR_PARAMS;
  if (p.rc > 0.5 * std::min(p.L[0], p.L[1]) * (1.0 + 1e-12)) return SOG_ERR_PARAMS;
  if (p.M < 0 || p.M > 4000 || p.m < -1 || p.m > p.M) return SOG_ERR_PARAMS;
  if (p.window != SOG_WIN_ES && p.window != SOG_WIN_GAUSS && p.window != SOG_WIN_KB)
    return SOG_ERR_PARAMS;
  if (p.win_poly != 0 && (p.win_poly < 2 || p.win_poly > sogk::kPolyMax)) return SOG_ERR_PARAMS;
  if (p.m >= 0) {
    for (int d = 0; d < 3; ++d)
      if (!smooth_even(p.I[d])) return SOG_ERR_PARAMS;
    if (p.P_win < 2 || p.P_win > sogk::kMaxWin || p.P_win > std::min(p.I[0], std::min(p.I[1], p.I[2])))
      return SOG_ERR_PARAMS;
    if (!(p.hz > 0.0) || p.I[2] * p.hz < p.L[2] + (p.P_win - 1) * p.hz - 1e-9 * p.L[2])
      return SOG_ERR_PARAMS;
    if (!(p.shape > 0.0)) return SOG_ERR_PARAMS;
  }
  if (p.long_direct != 0 && p.long_direct != 1) return SOG_ERR_PARAMS;
  if (p.m < p.M) {
    if (p.P_cheb < 2 || p.P_cheb > sogk::kMaxCheb) return SOG_ERR_PARAMS;
    if (p.long_direct) {
      for (int d = 0; d < 2; ++d)
        if (p.I_long[d] < 1 || p.I_long[d] % 2 != 1) return SOG_ERR_PARAMS;
      const int Kx = (p.I_long[0] - 1) / 2, Ky = (p.I_long[1] - 1) / 2;
      const int nhalf = Ky + Kx * (2 * Ky + 1);
      if (nhalf < 1 || nhalf > sogk::kMaxHalfModes ||
          nhalf * p.P_cheb > sogk::kMaxHalfModeCoefs)
        return SOG_ERR_PARAMS;
      return SOG_OK;
    }
    for (int d = 0; d < 2; ++d)
      if (!smooth_even(p.I_long[d])) return SOG_ERR_PARAMS;
    if (p.P_long < 2 || p.P_long > sogk::kMaxWin || p.P_long > std::min(p.I_long[0], p.I_long[1]))
      return SOG_ERR_PARAMS;
    if (!(p.shape_long > 0.0)) return SOG_ERR_PARAMS;
  }
  return SOG_OK;
}

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------

// big: radices 16 and 15 first (engines holding 16 values per thread)
void factorize(int n, sogk::FftLen& f, bool big) {
  f.n = n;
  f.nst = 0;
  int k = n;
  if (big) {
    while (k % 16 == 0) { f.radix[f.nst++] = 16; k /= 16; }
    while (k % 15 == 0) { f.radix[f.nst++] = 15; k /= 15; }
  }
  while (k % 8 == 0 && k > 1) { f.radix[f.nst++] = 8; k /= 8; }
  while (k % 4 == 0) { f.radix[f.nst++] = 4; k /= 4; }
  while (k % 2 == 0) { f.radix[f.nst++] = 2; k /= 2; }
  for (int p : {3, 5, 7})
    while (k % p == 0) { f.radix[f.nst++] = p; k /= p; }
  f.n16 = f.n15 = f.n8 = f.n4 = f.n2 = f.n3 = f.n5 = f.n7 = 0;
  for (int st = 0; st < f.nst; ++st) {
    const int R = f.radix[st];
    f.n16 += R == 16;
    f.n15 += R == 15;
    f.n8 += R == 8;
    f.n4 += R == 4;
    f.n2 += R == 2;
    f.n3 += R == 3;
    f.n5 += R == 5;
    f.n7 += R == 7;
  }
}

// Gauss-Legendre nodes and weights on [-1, 1].
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
  x.resize(n);
  wt.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// hat W(k) of the window W(x) = phi(x/H): Gaussian closed form (Eq. 4.7);
// ES by Gauss-Legendre quadrature of
//   H int_{-pi/2}^{pi/2} exp(beta(cos t - 1)) cos(k H sin t) cos t dt;
// KB by Gauss-Legendre quadrature of the series the kernels evaluate.
struct WinFT {
  int kind;
  double shape, H;
  std::vector<double> gx, gw, kbw;  // KB: node weight x the series the kernels evaluate
  WinFT(int kind_, double shape_, double H_, int prec) : kind(kind_), shape(shape_), H(H_) {
    if (kind == SOG_WIN_KB) {
      gauss_legendre(256, gx, gw);
      std::vector<double> kbc;
      if (prec == SOG_PREC_MIXED) {
        float c[64];
        kbc.assign(c, c + sogk::kb_series<float>(shape, c, 64));
      } else {
        double c[64];
        kbc.assign(c, c + sogk::kb_series<double>(shape, c, 64));
      }
      kbw.resize(gx.size());
      for (size_t i = 0; i < gx.size(); ++i) {
        const double u = (1.0 - gx[i]) * (1.0 + gx[i]);
        double p = 0.0;
        for (size_t j = kbc.size(); j-- > 0;) p = p * u + kbc[j];
        kbw[i] = gw[i] * p;
      }
    }
    if (kind == SOG_WIN_ES) gauss_legendre(256, gx, gw);
  }
  double operator()(double k) const {
    if (kind == SOG_WIN_GAUSS) return sqrt(kPi / shape) * H * exp(-k * k * H * H / (4.0 * shape));
    if (kind == SOG_WIN_KB) {
      // H int_{-1}^{1} sum_j kbc[j] (1 - v^2)^j cos(k H v) dv by Gauss-Legendre
      // (the series with the kernels' rounded coefficients; the closed form
      // 2 sinh(sqrt(b^2 - w^2)) / sqrt(b^2 - w^2) / I0(b) holds for exact ones)
      double acc = 0.0;
      for (size_t i = 0; i < gx.size(); ++i) acc += kbw[i] * cos(k * H * gx[i]);
      return H * acc;
    }
    double acc = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
      const double t = 0.5 * kPi * gx[i];
      acc += gw[i] * exp(shape * (cos(t) - 1.0)) * cos(k * H * sin(t)) * cos(t);
    }
    return H * 0.5 * kPi * acc;
  }
};

// The window the kernels apply, phi((g - x) / half) with the shape and
// 1/half rounded to the element type: its transform (which the scaling
// tables divide by) is taken with the same rounded values, so that a plan
// in FP32 deconvolves exactly the window it spreads with.
double eff_shape(double shape, int prec) {
  return prec == SOG_PREC_MIXED ? (double)(float)shape : shape;
}
double eff_half(double half, int prec) {
  return prec == SOG_PREC_MIXED ? 1.0 / (double)(float)(1.0 / half) : half;
}


// Near kernel table: g(r) = 1 - r F_M(r) on [0, rc], K intervals, degree D
// monomials in u = 2 (r - r_k)/(rc/K) - 1 (fitted at Chebyshev points).
bool near_table(const std::vector<double>& w, const std::vector<double>& s, double rc, int D,
                double target, int& Kout, std::vector<double>& coef) {
  auto gfun = [&](double r) {
    double F = 0.0;
    for (size_t l = 0; l < w.size(); ++l) F += w[l] * exp(-(r * r) / (s[l] * s[l]));
    return 1.0 - r * F;
  };
  for (int K = 16; K <= 8192; K *= 2) {
    const double hK = rc / K;
    coef.assign((size_t)K * (D + 1), 0.0);
    double maxerr = 0.0;
    for (int k = 0; k < K && maxerr <= target; ++k) {
      // Vandermonde solve at D+1 Chebyshev points
      const int n = D + 1;
      std::vector<double> Amat(n * n), rhs(n);
      for (int j = 0; j < n; ++j) {
        const double u = cos(kPi * (j + 0.5) / n);
        double pw = 1.0;
        for (int c = 0; c < n; ++c) {
          Amat[j * n + c] = pw;
          pw *= u;
        }
        rhs[j] = gfun(k * hK + 0.5 * (u + 1.0) * hK);
      }
      for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int rr = c + 1; rr < n; ++rr)
          if (fabs(Amat[rr * n + c]) > fabs(Amat[piv * n + c])) piv = rr;
        for (int cc = 0; cc < n; ++cc) std::swap(Amat[c * n + cc], Amat[piv * n + cc]);
        std::swap(rhs[c], rhs[piv]);
        for (int rr = c + 1; rr < n; ++rr) {
          const double f = Amat[rr * n + c] / Amat[c * n + c];
          for (int cc = c; cc < n; ++cc) Amat[rr * n + cc] -= f * Amat[c * n + cc];
          rhs[rr] -= f * rhs[c];
        }
      }
      for (int c = n - 1; c >= 0; --c) {
        double v = rhs[c];
        for (int cc = c + 1; cc < n; ++cc) v -= Amat[c * n + cc] * coef[(size_t)k * n + cc];
        coef[(size_t)k * n + c] = v / Amat[c * n + c];
      }
      for (int t = 0; t <= 24; ++t) {
        const double u = -1.0 + 2.0 * t / 24.0;
        double p = coef[(size_t)k * n + D];
        for (int c = D - 1; c >= 0; --c) p = p * u + coef[(size_t)k * n + c];
        maxerr = std::max(maxerr, fabs(p - gfun(k * hK + 0.5 * (u + 1.0) * hK)));
      }
    }
    if (maxerr <= target) {
      Kout = K;
      return true;
    }
  }
  return false;
}


// CTAs per tile of the gridding and gathering: enough CTAs in all (about
// 600) while each keeps at least 32 charges; `scale` multiplies the rule.
int tile_chunks(int64_t N, int ntiles, double scale) {
  const double per_tile = (double)N / ntiles;
  int ch = (int)ceil(scale * 600.0 / ntiles);
  ch = std::max(1, std::min(ch, (int)(per_tile / 32.0)));
  return std::max(1, ch);
}

// Mid-range tiling: as many tiles per dimension as edge T needs, their edge
// evened out over the grid (120 = 8 x 15).
void set_mid_tiles(sog_plan* p, int T, double scale) {
  sogk::TileGeom& g = p->gm;
  for (int d = 0; d < 3; ++d) {
    g.I[d] = p->prm.I[d];
    const int nt = (g.I[d] + T - 1) / T;
    g.T[d] = (g.I[d] + nt - 1) / nt;
    g.nt[d] = (g.I[d] + g.T[d] - 1) / g.T[d];
    g.W[d] = g.T[d] + p->prm.P_win;
  }
  g.pad_lo = (int)floor(p->wm.half);
  g.pitch = p->prm.I[0] + 2;
  p->n_tiles_mid = g.nt[0] * g.nt[1] * g.nt[2];
  g.chunks = tile_chunks(p->N, p->n_tiles_mid, scale);
  p->mid_T = T;
  p->mid_cscale = scale;
}

// Long-range tiling of the proxy planes (2D tiles of edge T).
void set_long_tiles(sog_plan* p, int T, double scale) {
  sogk::TileGeom& g = p->gl;
  g.I[0] = p->prm.I_long[0];
  g.I[1] = p->prm.I_long[1];
  g.I[2] = 1;
  for (int d = 0; d < 2; ++d) {
    g.T[d] = std::min(T, g.I[d]);
    g.nt[d] = (g.I[d] + g.T[d] - 1) / g.T[d];
    g.W[d] = g.T[d] + p->prm.P_long;
  }
  g.T[2] = g.nt[2] = g.W[2] = 1;
  g.pad_lo = (int)floor(p->wl.half);
  g.pitch = p->prm.I_long[0] + 2;
  p->n_tiles_long = g.nt[0] * g.nt[1];
  g.chunks = tile_chunks(p->N, p->n_tiles_long, scale);
  p->long_T = T;
  p->long_cscale = scale;
}

// Offsets of the three bin-count arrays in d_cnt for the current tiles.
void set_cnt_offsets(sog_plan* p) {
  p->cnt_off[0] = 0;
  p->cnt_off[1] = p->n_cells + 1;
  p->cnt_off[2] = p->cnt_off[1] + (p->has_mid ? p->n_tiles_mid + 1 : 1);
  p->cnt_off[3] = p->cnt_off[2] + (p->has_long ? p->n_tiles_long + 1 : 1);
}

template <typename T>
void put(std::vector<unsigned char>& buf, size_t off, const std::vector<double>& v) {
  T* d = reinterpret_cast<T*>(buf.data() + off);
  for (size_t i = 0; i < v.size(); ++i) d[i] = (T)v[i];
}

struct Arena {
  size_t size = 0;
  size_t take(size_t bytes) {
    const size_t o = size;
    size += (bytes + 255) / 256 * 256;
    return o;
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* sog_status_str(sog_status s) {
  switch (s) {
    case SOG_OK: return "ok";
    case SOG_ERR_ARG: return "invalid argument";
    case SOG_ERR_NONNEUTRAL: return "charges are not neutral (|sum q| > 1e-10 sum |q|)";
    case SOG_ERR_OUT_OF_BOX: return "a z coordinate is outside [-Lz/2, Lz/2] or a coordinate is not finite";
    case SOG_ERR_NOMEM: return "out of memory";
    case SOG_ERR_CUDA: return "CUDA error";
    case SOG_ERR_PARAMS: return "no feasible or an inconsistent parameter set";
    case SOG_ERR_TIMEOUT: return "a kernel's bounded wait for its asynchronous copies ran out";
  }
  return "unknown status";
}

static sog_status check_args(int64_t N, double Lx, double Ly, double Lz, double tol) {
  if (N < 2 || N > (int64_t)1 << 30) return SOG_ERR_ARG;
  if (!(Lx > 0.0) || !(Ly > 0.0) || !(Lz > 0.0) || !isfinite(Lx) || !isfinite(Ly) || !isfinite(Lz))
    return SOG_ERR_ARG;
  if (!(tol > 0.0) || !(tol <= 0.1)) return SOG_ERR_ARG;
  return SOG_OK;
}

sog_status sog_select_params(int64_t N, double Lx, double Ly, double Lz, double tol,
                             const sog_opts* opts, sog_params* out) {
  if (!out) return SOG_ERR_ARG;
  sog_status st = check_args(N, Lx, Ly, Lz, tol);
  if (st != SOG_OK) return st;
  const int window = opts ? opts->window : SOG_WIN_ES;
  if (window != SOG_WIN_ES && window != SOG_WIN_GAUSS && window != SOG_WIN_KB) return SOG_ERR_ARG;
  const double nnb = (opts && opts->n_nb > 0.0) ? opts->n_nb : 120.0;
  const int nu = opts ? opts->win_poly : 0;
  if (nu != 0 && (nu < 2 || nu > sogk::kPolyMax)) return SOG_ERR_ARG;
  st = select_params(N, Lx, Ly, Lz, tol, window, nnb, out);
  if (st == SOG_OK) out->win_poly = nu;
  return st;
}

sog_status sog_plan_create(sog_plan** plan, int64_t N, double Lx, double Ly, double Lz, double tol,
                           const sog_opts* opts) {
  if (!plan) return SOG_ERR_ARG;
  *plan = nullptr;
  sog_status st = check_args(N, Lx, Ly, Lz, tol);
  if (st != SOG_OK) return st;
  const int prec = opts ? opts->precision : SOG_PREC_MIXED;
  if (prec != SOG_PREC_FP64 && prec != SOG_PREC_MIXED) return SOG_ERR_ARG;
  sog_params prm;
  if (opts && opts->manual) {
    prm = *opts->manual;
    if (prm.L[0] != Lx || prm.L[1] != Ly || prm.L[2] != Lz) return SOG_ERR_ARG;
  } else {
    st = sog_select_params(N, Lx, Ly, Lz, tol, opts, &prm);
    if (st != SOG_OK) return st;
  }
  st = check_params(prm);
  if (st != SOG_OK) return st;

  if (sogk::prepare_kernels(prec) != cudaSuccess) {
    cudaGetLastError();
    return SOG_ERR_CUDA;
  }
  sog_plan* p = new (std::nothrow) sog_plan();
  if (!p) return SOG_ERR_NOMEM;
  p->prm = prm;
  p->prec = prec;
  p->N = N;
  cudaGetDevice(&p->device);
  if (cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
      p->n_sm < 1) {
    cudaGetLastError();
    delete p;
    return SOG_ERR_CUDA;
  }
  p->red_blocks = sogk::kRedBlocksPerSm * p->n_sm;
  p->mode_blocks = sogk::kModeBlocksPerSm * p->n_sm;
  p->k0_blocks = sogk::kK0BlocksPerSm * p->n_sm;
  const size_t es = prec == SOG_PREC_FP64 ? sizeof(double) : sizeof(float);
  const double* L = prm.L;

  // SOG table and derived geometry
  std::vector<double> w, s;
  sog_table(prm.b, prm.sigma, prm.omega, prm.M, w, s);
  p->selfsum = 0.0;
  for (double v : w) p->selfsum += v;
  p->has_mid = prm.m >= 0;
  p->has_long = prm.m < prm.M;
  for (int d = 0; d < 3; ++d) {
    p->nc[d] = std::max(1, (int)floor(L[d] / prm.rc));
    p->cell[d] = L[d] / p->nc[d];
  }
  p->n_cells = p->nc[0] * p->nc[1] * p->nc[2];
  const int Ix = prm.I[0], Iy = prm.I[1], Iz = prm.I[2];
  const int Ilx = prm.I_long[0], Ily = prm.I_long[1];
  const int P = prm.P_cheb;
  if (p->has_mid) {
    p->h[0] = L[0] / Ix;
    p->h[1] = L[1] / Iy;
    p->h[2] = prm.hz;
    p->Lzs = Iz * prm.hz;
    p->wm = sogk::WinPar{prm.P_win, prm.window, 0.5 * (prm.P_win - 1), prm.shape, prm.win_poly};
    int T = 16;
    if (prec == SOG_PREC_FP64 || (size_t)(16 + prm.P_win) * (16 + prm.P_win) * (16 + prm.P_win) * es > 72 * 1024)
      T = 8;
    set_mid_tiles(p, T, 1.0);
  }
  p->long_direct = p->has_long && prm.long_direct;
  if (p->long_direct) {
    p->n_half = (Ily - 1) / 2 + (Ilx - 1) / 2 * Ily;  // Ky + Kx (2 Ky + 1)
    p->long_small = 0;
  }
  if (p->has_long && !p->long_direct) {
    p->hl[0] = L[0] / Ilx;
    p->hl[1] = L[1] / Ily;
    p->wl = sogk::WinPar{prm.P_long, prm.window, 0.5 * (prm.P_long - 1), prm.shape_long, prm.win_poly};
    int T = 16;
    if ((size_t)P * ((16 + prm.P_long) * (16 + prm.P_long) + 1) * es > 96 * 1024) T = 8;
    set_long_tiles(p, T, 1.0);
    // one tile covering the grid and planes that fit shared memory: private
    // copies per CTA plus a reduction instead of atomics on a few addresses
    p->long_small = (p->gl.nt[0] == 1 && p->gl.nt[1] == 1 &&
                     (size_t)P * (Ilx * Ily + 1) * es <= 64 * 1024) ? 1 : 0;
    p->long_small_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(p->red_blocks, N / 128));
  }

  // FFT lengths and twiddles exp(-2 pi i t/n): FP64 (cos, sin); FP32
  // (cos, sin) rounded and their rounding errors, so that FP32 transforms
  // apply twiddles of ~48-bit precision and no FP32-rounded root of unity
  // biases the transform's gain.
  std::vector<double> tw;
  const int tw_vals = prec == SOG_PREC_MIXED ? 4 : 2;
  // Per length: the radix-16 and radix-15 butterfly constants w_16^t and
  // w_15^t (kTwConst entries), then the engine's per-stage tables (in the
  // order the engine runs the radices: 15, 3, 5, 7, 16, 8, 4, 2; stage of
  // radix R after a product L of earlier radices: entries [p - 1][j] =
  // w_n^(j p n / (R L)), p < R, j < L, so that consecutive threads read
  // consecutive entries), padded to n entries.
  auto push_tw = [&](int t, int n) {
    const double c = cos(2.0 * kPi * t / n), sn = -sin(2.0 * kPi * t / n);
    if (prec == SOG_PREC_MIXED) {
      const double ch = (double)(float)c, sh = (double)(float)sn;
      tw.insert(tw.end(), {ch, sh, c - ch, sn - sh});
    } else {
      tw.insert(tw.end(), {c, sn});
    }
  };
  auto add_len = [&](int n, sogk::FftLen& f) {
    factorize(n, f, prec != SOG_PREC_FP64);
    f.tw_off = (int)(tw.size() / tw_vals);
    for (int t = 0; t < 16; ++t) push_tw(t, 16);
    for (int t = 0; t < 16; ++t) push_tw(t % 15, 15);
    int L = 1, used = 0;
    auto stage_tw = [&](int R) {
      const int m = n / (R * L);
      for (int pp = 1; pp < R; ++pp)
        for (int j = 0; j < L; ++j) push_tw(j * pp * m, n);
      used += (R - 1) * L;
      L *= R;
    };
    for (int i = 0; i < f.n15; ++i) stage_tw(15);
    for (int i = 0; i < f.n3; ++i) stage_tw(3);
    for (int i = 0; i < f.n5; ++i) stage_tw(5);
    for (int i = 0; i < f.n7; ++i) stage_tw(7);
    for (int i = 0; i < f.n16; ++i) stage_tw(16);
    for (int i = 0; i < f.n8; ++i) stage_tw(8);
    for (int i = 0; i < f.n4; ++i) stage_tw(4);
    for (int i = 0; i < f.n2; ++i) stage_tw(2);
    for (; used < n; ++used) push_tw(0, n);
  };
  if (p->has_mid) {
    add_len(Ix, p->fx);
    add_len(Iy, p->fy);
    add_len(Iz, p->fz);
  }
  if (p->has_long && !p->long_direct) {
    add_len(Ilx, p->flx);
    add_len(Ily, p->fly);
  }
  if (tw.empty()) tw.assign(4, 0.0);
  if ((p->has_mid && !(sogk::fft_len_ok(prec, p->fx) && sogk::fft_len_ok(prec, p->fy) &&
                       sogk::fft_len_ok(prec, p->fz))) ||
      (p->has_long && !p->long_direct &&
       !(sogk::fft_len_ok(prec, p->flx) && sogk::fft_len_ok(prec, p->fly)))) {
    delete p;
    return SOG_ERR_PARAMS;  // a grid dimension too long for the shared-memory FFT
  }

  // near table
  p->near_D = sogk::kNearD;
  std::vector<double> ntab;
  if (!near_table(w, s, prm.rc, p->near_D, prec == SOG_PREC_FP64 ? 3e-15 : 1e-9, p->near_K, ntab)) {
    delete p;
    return SOG_ERR_PARAMS;
  }
  {
    // rows padded to the kernels' vector stride
    const int D1 = p->near_D + 1, R = prec == SOG_PREC_FP64 ? sogk::near_row<double>()
                                                           : sogk::near_row<float>();
    std::vector<double> padded((size_t)p->near_K * R, 0.0);
    for (int k = 0; k < p->near_K; ++k)
      for (int c = 0; c < D1; ++c) padded[(size_t)k * R + c] = ntab[(size_t)k * D1 + c];
    ntab.swap(padded);
  }

  // mid scaling factors, Eq. (3.8) for unnormalised DFTs
  std::vector<double> mult;
  if (p->has_mid) {
    const int C = Ix / 2 + 1;
    const double shp = eff_shape(prm.shape, prec), hw = eff_half(p->wm.half, prec);
    WinFT fx(prm.window, shp, hw * p->h[0], prec);
    WinFT fy(prm.window, shp, hw * p->h[1], prec);
    WinFT fz(prm.window, shp, hw * p->h[2], prec);
    std::vector<double> kx(C), ky(Iy), kz(Iz), Wx(C), Wy(Iy), Wz(Iz);
    for (int f = 0; f < C; ++f) { kx[f] = 2.0 * kPi * f / L[0]; Wx[f] = fx(kx[f]); }
    for (int f = 0; f < Iy; ++f) { ky[f] = 2.0 * kPi * std::min(f, Iy - f) / L[1]; Wy[f] = fy(ky[f]); }
    for (int f = 0; f < Iz; ++f) { kz[f] = 2.0 * kPi * std::min(f, Iz - f) / p->Lzs; Wz[f] = fz(kz[f]); }
    const double pre = pow(p->h[0] * p->h[1] * p->h[2], 2) / (L[0] * L[1] * p->Lzs);
    mult.resize((size_t)Iz * Iy * C);
    for (int z = 0; z < Iz; ++z)
      for (int y = 0; y < Iy; ++y)
        for (int x = 0; x < C; ++x) {
          const double k2 = kx[x] * kx[x] + ky[y] * ky[y] + kz[z] * kz[z];
          double kh = 0.0;
          for (int l = 0; l <= prm.m; ++l)
            kh += pow(kPi, 1.5) * w[l] * s[l] * s[l] * s[l] * exp(-s[l] * s[l] * k2 / 4.0);
          const double W2 = pow(Wx[x] * Wy[y] * Wz[z], 2);
          mult[((size_t)z * Iy + y) * C + x] = (x == 0 && y == 0 && z == 0) ? 0.0 : pre * kh / W2;
        }
  }

  // long range: per-mode z-kernel in the Chebyshev basis and the k = 0 kernel
  std::vector<double> kmat, lbl, lcl, lfx, lfy,
      k0mat((size_t)std::max(P, 1) * std::max(P, 1), 0.0);
  if (p->has_long) {
    const double A = L[0] * L[1];
    std::vector<double> zc(P), Cm((size_t)P * P);
    for (int c = 0; c < P; ++c) {
      const double x = cos((c + 0.5) * kPi / P);
      zc[c] = 0.5 * L[2] * x;
      double t0 = 1.0, t1 = x;
      for (int n = 0; n < P; ++n) {
        double tn = n == 0 ? 1.0 : (n == 1 ? x : 0.0);
        if (n >= 2) {
          tn = 2.0 * x * t1 - t0;
          t0 = t1;
          t1 = tn;
        }
        Cm[(size_t)c * P + n] = (n == 0 ? 1.0 : 2.0) / P * tn;
      }
    }
    // B_l = C^T E_l C with E_l[c][c'] = exp(-(z_c - z_c')^2 / s_l^2)
    const int nl = prm.M - prm.m;
    std::vector<double> Bl((size_t)nl * P * P);
    std::vector<double> E((size_t)P * P), tmp((size_t)P * P);
    for (int li = 0; li < nl; ++li) {
      const int l = prm.m + 1 + li;
      for (int c = 0; c < P; ++c)
        for (int c2 = 0; c2 < P; ++c2) {
          const double d = zc[c] - zc[c2];
          E[(size_t)c * P + c2] = exp(-d * d / (s[l] * s[l]));
        }
      for (int c = 0; c < P; ++c)
        for (int n2 = 0; n2 < P; ++n2) {
          double a = 0.0;
          for (int c2 = 0; c2 < P; ++c2) a += E[(size_t)c * P + c2] * Cm[(size_t)c2 * P + n2];
          tmp[(size_t)c * P + n2] = a;
        }
      for (int n = 0; n < P; ++n)
        for (int n2 = 0; n2 < P; ++n2) {
          double a = 0.0;
          for (int c = 0; c < P; ++c) a += Cm[(size_t)c * P + n] * tmp[(size_t)c * P + n2];
          Bl[((size_t)li * P + n) * P + n2] = a;
        }
    }
    if (p->long_direct) {
      // Algorithm 3: per half-plane mode (pi/A) sum_l w_l s_l^2 e^{-s_l^2 k^2/4} B_l,
      // doubled for the conjugate mode (the potential is the real part)
      const int Ky = (Ily - 1) / 2;
      kmat.assign((size_t)p->n_half * P * P, 0.0);
      for (int h = 0; h < p->n_half; ++h) {
        int nx, ny;
        sogk::half_mode(h, Ky, nx, ny);
        const double kxv = 2.0 * kPi * nx / L[0], kyv = 2.0 * kPi * ny / L[1];
        const double k2 = kxv * kxv + kyv * kyv;
        double* K = &kmat[(size_t)h * P * P];
        for (int li = 0; li < nl; ++li) {
          const int l = prm.m + 1 + li;
          const double ex = s[l] * s[l] * k2 / 4.0;
          if (ex > 80.0) break;
          const double al = 2.0 * kPi / A * w[l] * s[l] * s[l] * exp(-ex);
          const double* B = &Bl[(size_t)li * P * P];
          for (int i = 0; i < P * P; ++i) K[i] += al * B[i];
        }
      }
    }
    if (!p->long_direct) {
      // Algorithm 2: K_k = fx(kx) fy(ky) sum_l c1_l e^{-c2_l k^2} B_l, applied
      // factor by factor in the contraction.  B_l[n][n'] vanishes when n + n'
      // is odd (the proxy points are symmetric about z = 0 and T_n has the
      // parity of n), so each B_l is stored as its even and odd blocks.
      const int C = Ilx / 2 + 1;
      const int ps = (P + 1) / 2, pst = (ps + 3) / 4 * 4;
      p->n_lg = nl;
      p->lps = ps;
      p->lpst = pst;
      lbl.assign((size_t)nl * 2 * ps * pst, 0.0);
      for (int li = 0; li < nl; ++li)
        for (int par = 0; par < 2; ++par)
          for (int i = 0; 2 * i + par < P; ++i)
            for (int j = 0; 2 * j + par < P; ++j)
              lbl[(((size_t)li * 2 + par) * ps + i) * pst + j] =
                  Bl[((size_t)li * P + 2 * i + par) * P + 2 * j + par];
      lcl.resize((size_t)2 * nl);
      // the smallest mode k != 0 bounds the Gaussians any mode uses: s_l grows
      // with l, and terms with c2_l k^2 > 80 are dropped
      const double kmin = 2.0 * kPi / std::max(L[0], L[1]);
      // a term with c2_l k^2 = x weighs about b^dl e^-x against the mode's
      // largest (x of order 1; the weights w_l s_l^2 grow like b^l): x = 20
      // leaves it below 1e-8 of that term, under FP32 rounding
      p->lg_xmax = prec == SOG_PREC_FP64 ? 80.0 : 20.0;
      p->n_lg_used = 0;
      for (int li = 0; li < nl; ++li) {
        const int l = prm.m + 1 + li;
        lcl[2 * li] = kPi / (L[0] * L[1]) * w[l] * s[l] * s[l];
        lcl[2 * li + 1] = 0.25 * s[l] * s[l];
        if (lcl[2 * li + 1] * kmin * kmin <= p->lg_xmax) p->n_lg_used = li + 1;
      }
      p->long_fused = sogk::long_fused_fits(P, p->fly, p->n_lg_used, es) ? 1 : 0;
      const double shp = eff_shape(prm.shape_long, prec), hw = eff_half(p->wl.half, prec);
      WinFT fx(prm.window, shp, hw * p->hl[0], prec);
      WinFT fy(prm.window, shp, hw * p->hl[1], prec);
      lfx.resize((size_t)2 * C);
      lfy.resize((size_t)2 * Ily);
      for (int f = 0; f < C; ++f) {
        const double k = 2.0 * kPi * f / L[0], W = fx(k);
        lfx[2 * f] = k * k;
        lfx[2 * f + 1] = p->hl[0] * p->hl[0] / (W * W);
      }
      for (int f = 0; f < Ily; ++f) {
        const double k = 2.0 * kPi * std::min(f, Ily - f) / L[1], W = fy(k);
        lfy[2 * f] = k * k;
        lfy[2 * f + 1] = p->hl[1] * p->hl[1] / (W * W);
      }

    }
    // k = 0: (pi/A) C^T K0 C, K0(d) = -sum_{l>m} w_l d^2 phi1(d^2/s_l^2)
    std::vector<double> K0((size_t)P * P, 0.0);
    for (int c = 0; c < P; ++c)
      for (int c2 = 0; c2 < P; ++c2) {
        const double d = zc[c] - zc[c2];
        double acc = 0.0;
        for (int l = prm.m + 1; l <= prm.M; ++l) {
          const double x = d * d / (s[l] * s[l]);
          const double ph1 = x == 0.0 ? 1.0 : -expm1(-x) / x;
          acc -= w[l] * d * d * ph1;
        }
        K0[(size_t)c * P + c2] = acc;
      }
    for (int c = 0; c < P; ++c)
      for (int n2 = 0; n2 < P; ++n2) {
        double acc = 0.0;
        for (int c2 = 0; c2 < P; ++c2) acc += K0[(size_t)c * P + c2] * Cm[(size_t)c2 * P + n2];
        tmp[(size_t)c * P + n2] = acc;
      }
    for (int n = 0; n < P; ++n)
      for (int n2 = 0; n2 < P; ++n2) {
        double acc = 0.0;
        for (int c = 0; c < P; ++c) acc += Cm[(size_t)c * P + n] * tmp[(size_t)c * P + n2];
        k0mat[(size_t)n * P + n2] = kPi / A * acc;
      }
  }

  // device arena
  Arena ar;
  const size_t o_tw = ar.take(tw.size() * es);
  const size_t o_near = ar.take(ntab.size() * es);
  const size_t o_mult = ar.take(mult.size() * es);
  const size_t o_kmat = ar.take(kmat.size() * es);
  const size_t o_lbl = ar.take(lbl.size() * es);
  const size_t o_lcl = ar.take(lcl.size() * es);
  const size_t o_lfx = ar.take(lfx.size() * es);
  const size_t o_lfy = ar.take(lfy.size() * es);
  const size_t o_k0 = ar.take(k0mat.size() * sizeof(double));
  const size_t tables_end = ar.size;
  const size_t o_grid = ar.take(p->has_mid ? (size_t)Iz * Iy * (Ix + 2) * es : 0);
  const size_t lbytes = p->has_long ? (size_t)P * Ily * (Ilx + 2) * es : 0;
  const size_t o_lA = ar.take(lbytes);
  const size_t o_lB = ar.take(p->long_fused ? lbytes : 0);  // transposed spectrum of the fused path
  const size_t o_rn = ar.take((size_t)N * 4 * es);
  const size_t o_rm = ar.take(p->has_mid ? (size_t)N * 4 * es : 0);
  const size_t o_rl = ar.take(p->has_long ? (size_t)N * 4 * es : 0);
  const size_t o_rt = ar.take((size_t)3 * N * 4 * es);
  const size_t o_perm = ar.take((size_t)3 * N * sizeof(int));
  const size_t o_key = ar.take((size_t)3 * N * sizeof(int));
  const size_t o_rank = ar.take((size_t)3 * N * sizeof(int));
  set_cnt_offsets(p);
  // room for the smallest tiles the autotuner tries (edge 8)
  {
    auto ntiles = [](const int* I, int nd, int T) {
      long n = 1;
      for (int d = 0; d < nd; ++d) n *= (I[d] + T - 1) / T;
      return n;
    };
    const long mid_max = p->has_mid ? ntiles(prm.I, 3, 8) : 0;
    const long long_max = (p->has_long && !p->long_direct) ? ntiles(prm.I_long, 2, 8) : 0;
    p->cnt_cap = (int)(p->n_cells + 1 + std::max<long>(mid_max, p->n_tiles_mid) + 1 +
                       std::max<long>(long_max, p->n_tiles_long) + 1);
  }
  const size_t o_cnt = ar.take((size_t)p->cnt_cap * sizeof(int));
  const size_t o_pp = ar.take((size_t)4 * N * sizeof(double));
  const size_t o_pg = ar.take((size_t)12 * N * sizeof(double));
  const size_t o_red = ar.take((size_t)p->red_blocks * (3 + sogk::kMaxCheb) * sizeof(double));
  const size_t o_nu = ar.take(sogk::kMaxCheb * sizeof(double));
  const size_t o_st = ar.take(sizeof(int));
  const size_t o_host = ar.take((size_t)N * 8 * es + sizeof(double));
  const size_t o_lpart = ar.take(p->has_long && p->long_small
                                     ? (size_t)p->long_small_blocks * P * Ilx * Ily * es : 0);
  // direct long range: per-block partial moments (FP64) and the coefficients
  const size_t o_lmom = ar.take(p->long_direct
                                    ? (size_t)p->mode_blocks * p->n_half * P * 2 * sizeof(double)
                                    : 0);
  const size_t o_lcoef = ar.take(p->long_direct ? (size_t)p->n_half * P * 2 * es : 0);
  void* base = nullptr;
  if (cudaMalloc(&base, ar.size) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return SOG_ERR_NOMEM;
  }
  p->arena = base;
  p->arena_bytes = (int64_t)ar.size;
  char* b = static_cast<char*>(base);
  p->d_tw = b + o_tw;
  p->d_near_tab = b + o_near;
  p->d_mult = b + o_mult;
  p->d_kmat = b + o_kmat;
  p->d_lbl = b + o_lbl;
  p->d_lcl = b + o_lcl;
  p->d_lfx = b + o_lfx;
  p->d_lfy = b + o_lfy;
  p->d_k0mat = reinterpret_cast<double*>(b + o_k0);
  p->d_grid = b + o_grid;
  p->d_lA = b + o_lA;
  p->d_lB = b + o_lB;
  p->d_rec_near = b + o_rn;
  p->d_rec_mid = b + o_rm;
  p->d_rec_long = b + o_rl;
  p->d_rec_tmp = b + o_rt;
  p->d_perm = reinterpret_cast<int*>(b + o_perm);
  p->d_key = reinterpret_cast<int*>(b + o_key);
  p->d_rank = reinterpret_cast<int*>(b + o_rank);
  p->d_cnt = reinterpret_cast<int*>(b + o_cnt);
  p->d_parts_phi = reinterpret_cast<double*>(b + o_pp);
  p->d_parts_grad = reinterpret_cast<double*>(b + o_pg);
  p->d_red = reinterpret_cast<double*>(b + o_red);
  p->d_k0nu = reinterpret_cast<double*>(b + o_nu);
  p->d_status = reinterpret_cast<int*>(b + o_st);
  p->d_host_stage = b + o_host;
  p->d_long_partial = b + o_lpart;
  p->d_lmom = reinterpret_cast<double*>(b + o_lmom);
  p->d_lcoef = b + o_lcoef;

  // upload tables (one host staging buffer)
  std::vector<unsigned char> host(tables_end, 0);
  if (es == sizeof(double)) {
    put<double>(host, o_tw, tw);
    put<double>(host, o_near, ntab);
    put<double>(host, o_mult, mult);
    put<double>(host, o_kmat, kmat);
    put<double>(host, o_lbl, lbl);
    put<double>(host, o_lcl, lcl);
    put<double>(host, o_lfx, lfx);
    put<double>(host, o_lfy, lfy);
  } else {
    put<float>(host, o_tw, tw);
    put<float>(host, o_near, ntab);
    put<float>(host, o_mult, mult);
    put<float>(host, o_kmat, kmat);
    put<float>(host, o_lbl, lbl);
    put<float>(host, o_lcl, lcl);
    put<float>(host, o_lfx, lfx);
    put<float>(host, o_lfy, lfy);
  }
  put<double>(host, o_k0, k0mat);
  cudaError_t e = cudaMemcpy(base, host.data(), tables_end, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_k0nu, 0, sogk::kMaxCheb * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(base);
    delete p;
    return SOG_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->long_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->k0_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join_long, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join_k0, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(base);
    delete p;
    return SOG_ERR_CUDA;
  }
  p->use_graphs = 1;
  p->last_stream = nullptr;
  p->launch_error = 0;
  *plan = p;
  return SOG_OK;
}

sog_status sog_plan_get_params(const sog_plan* plan, sog_params* out) {
  if (!plan || !out) return SOG_ERR_ARG;
  *out = plan->prm;
  return SOG_OK;
}

int32_t sog_plan_precision(const sog_plan* plan) { return plan ? plan->prec : -1; }

int64_t sog_plan_device_bytes(const sog_plan* plan) { return plan ? plan->arena_bytes : 0; }

sog_status sog_eval(sog_plan* plan, const void* q, const void* r, void* phi, double* E, void* F,
                    void* stream) {
  if (!plan || !q || !r) return SOG_ERR_ARG;
  return sogk::eval_device(plan, q, r, phi, E, F, nullptr, nullptr, (cudaStream_t)stream);
}

sog_status sog_eval_components(sog_plan* plan, const void* q, const void* r, double* phi_parts,
                               double* grad_parts, void* stream) {
  if (!plan || !q || !r) return SOG_ERR_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  sog_status st = sogk::eval_device(plan, q, r, nullptr, nullptr, nullptr, phi_parts, grad_parts, s);
  return st;
}

sog_status sog_eval_host(sog_plan* plan, const void* q, const void* r, void* phi, double* E, void* F) {
  if (!plan || !q || !r) return SOG_ERR_ARG;
  const size_t es = plan->prec == SOG_PREC_FP64 ? sizeof(double) : sizeof(float);
  const size_t N = (size_t)plan->N;
  void* buf = plan->d_host_stage;
  char* b = static_cast<char*>(buf);
  void* dq = b;
  void* dr = b + N * es;
  void* dphi = b + 4 * N * es;
  void* dF = b + 5 * N * es;
  double* dE = reinterpret_cast<double*>(b + ((8 * N * es + 7) / 8) * 8);
  cudaStream_t s = nullptr;
  cudaError_t e = cudaMemcpyAsync(dq, q, N * es, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dr, r, 3 * N * es, cudaMemcpyHostToDevice, s);
  sog_status st = SOG_OK;
  if (e == cudaSuccess)
    st = sogk::eval_device(plan, dq, dr, phi ? dphi : nullptr, E ? dE : nullptr, F ? dF : nullptr,
                           nullptr, nullptr, s);
  if (e == cudaSuccess && st == SOG_OK) {
    if (phi) e = cudaMemcpyAsync(phi, dphi, N * es, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && F) e = cudaMemcpyAsync(F, dF, 3 * N * es, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && E) e = cudaMemcpyAsync(E, dE, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return SOG_ERR_CUDA;
  if (st != SOG_OK) return st;
  return sog_plan_check(plan);
}

sog_status sog_plan_check(sog_plan* plan) {
  if (!plan) return SOG_ERR_ARG;
  if (cudaStreamSynchronize(plan->last_stream) != cudaSuccess) return SOG_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SOG_ERR_CUDA;
  if (cudaMemset(plan->d_status, 0, sizeof(int)) != cudaSuccess) return SOG_ERR_CUDA;
  if (plan->launch_error) {
    plan->launch_error = 0;
    return SOG_ERR_CUDA;
  }
  if (st & 4) return SOG_ERR_TIMEOUT;
  if (st & 2) return SOG_ERR_OUT_OF_BOX;
  if (st & 1) return SOG_ERR_NONNEUTRAL;
  return SOG_OK;
}

sog_status sog_plan_set_timing(sog_plan* plan, int32_t enable) {
  if (!plan) return SOG_ERR_ARG;
  if (enable && !plan->events_ready) {
    for (int i = 0; i < 2 * SOG_NSTAGES; ++i)
      if (cudaEventCreate(&plan->ev[i]) != cudaSuccess) return SOG_ERR_CUDA;
    plan->events_ready = 1;
  }
  if (enable < 0 || enable > 2) return SOG_ERR_ARG;
  plan->timing = enable;
  return SOG_OK;
}

sog_status sog_plan_get_timing(sog_plan* plan, float* ms) {
  if (!plan || !ms) return SOG_ERR_ARG;
  for (int i = 0; i < SOG_NSTAGES; ++i) ms[i] = 0.0f;
  if (!plan->events_ready) return SOG_OK;
  for (int k = 0; k < SOG_NSTAGES; ++k) {
    if (!plan->ev_used[2 * k] || !plan->ev_used[2 * k + 1]) continue;
    if (cudaEventSynchronize(plan->ev[2 * k + 1]) != cudaSuccess) return SOG_ERR_CUDA;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, plan->ev[2 * k], plan->ev[2 * k + 1]) != cudaSuccess)
      return SOG_ERR_CUDA;
    ms[k] = t;
  }
  return SOG_OK;
}

int64_t sog_plan_launches(const sog_plan* plan) { return plan ? plan->launches : 0; }

sog_status sog_plan_tiles(const sog_plan* plan, int32_t* out) {
  if (!plan || !out) return SOG_ERR_ARG;
  out[0] = plan->has_mid ? plan->mid_T : 0;
  out[1] = plan->has_mid ? plan->gm.chunks : 0;
  out[2] = (plan->has_long && !plan->long_direct) ? plan->long_T : 0;
  out[3] = (plan->has_long && !plan->long_direct) ? plan->gl.chunks : 0;
  return SOG_OK;
}

sog_status sog_plan_autotune(sog_plan* plan, const void* q, const void* r, int32_t reps,
                             void* stream) {
  if (!plan || !q || !r || reps < 1 || reps > 100) return SOG_ERR_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  const int saved = plan->timing;
  sog_status st = sog_plan_set_timing(plan, 2);
  if (st != SOG_OK) return st;
  const size_t es = plan->prec == SOG_PREC_FP64 ? sizeof(double) : sizeof(float);
  // isolated time of stages a and b (gridding and gathering), median of reps
  auto measure = [&](int a, int b, float* out) -> sog_status {
    std::vector<float> v;
    for (int i = 0; i <= reps; ++i) {
      sog_status e = sogk::eval_device(plan, q, r, nullptr, nullptr, nullptr, nullptr, nullptr, s);
      if (e != SOG_OK) return e;
      float ms[SOG_NSTAGES];
      e = sog_plan_get_timing(plan, ms);
      if (e != SOG_OK) return e;
      if (i > 0) v.push_back(ms[a] + ms[b]);  // the first run captures the graph
    }
    std::sort(v.begin(), v.end());
    *out = v[v.size() / 2];
    return SOG_OK;
  };
  const int Ts[] = {8, 12, 16, 20, 23};
  const double scales[] = {0.5, 1.0, 2.0};
  const size_t smem_cap = (size_t)sogk::kMaxDynSmem - 4096;
  // mid range: stages 2 (gridding) and 4 (gathering)
  if (plan->has_mid && st == SOG_OK) {
    int bT = plan->mid_T;
    double bs = plan->mid_cscale;
    float best = 0.0f;
    st = measure(2, 4, &best);
    for (int T : Ts) {
      if (st != SOG_OK) break;
      if (T + plan->prm.P_win > 32) continue;  // row tables of 32 entries
      for (double sc : scales) {
        if (T == bT && sc == bs) continue;
        set_mid_tiles(plan, T, sc);
        set_cnt_offsets(plan);
        if (plan->cnt_off[3] > plan->cnt_cap || sogk::mid_smem(plan, es, false) > smem_cap ||
            sogk::mid_smem(plan, es, true) > smem_cap)
          continue;
        sogk::release_graphs(plan);
        float t = 0.0f;
        st = measure(2, 4, &t);
        if (st != SOG_OK) break;
        if (t < best) {
          best = t;
          bT = T;
          bs = sc;
        }
      }
    }
    set_mid_tiles(plan, bT, bs);
    set_cnt_offsets(plan);
  }
  // long range (gridded form, several tiles): stages 5 and 7
  if (plan->has_long && !plan->long_direct && !plan->long_small && st == SOG_OK) {
    int bT = plan->long_T;
    double bs = plan->long_cscale;
    sogk::release_graphs(plan);
    float best = 0.0f;
    st = measure(5, 7, &best);
    for (int T : Ts) {
      if (st != SOG_OK) break;
      if (T + plan->prm.P_long > 32) continue;
      for (double sc : scales) {
        if (T == bT && sc == bs) continue;
        set_long_tiles(plan, T, sc);
        set_cnt_offsets(plan);
        if (plan->cnt_off[3] > plan->cnt_cap || plan->gl.nt[0] * plan->gl.nt[1] < 2 ||
            sogk::long_smem(plan, es, false) > smem_cap ||
            sogk::long_smem(plan, es, true) > smem_cap)
          continue;
        sogk::release_graphs(plan);
        float t = 0.0f;
        st = measure(5, 7, &t);
        if (st != SOG_OK) break;
        if (t < best) {
          best = t;
          bT = T;
          bs = sc;
        }
      }
    }
    set_long_tiles(plan, bT, bs);
    set_cnt_offsets(plan);
  }
  sogk::release_graphs(plan);
  const sog_status st2 = sog_plan_set_timing(plan, saved);
  return st != SOG_OK ? st : st2;
}

void sog_plan_destroy(sog_plan* plan) {
  if (!plan) return;
  cudaStreamSynchronize(plan->last_stream);
  if (plan->events_ready)
    for (int i = 0; i < 2 * SOG_NSTAGES; ++i) cudaEventDestroy(plan->ev[i]);
  sogk::release_graphs(plan);
  cudaStreamDestroy(plan->cap_stream);
  cudaStreamDestroy(plan->side_stream);
  cudaStreamDestroy(plan->long_stream);
  cudaStreamDestroy(plan->k0_stream);
  cudaEventDestroy(plan->ev_fork);
  cudaEventDestroy(plan->ev_join);
  cudaEventDestroy(plan->ev_join_long);
  cudaEventDestroy(plan->ev_join_k0);
  cudaFree(plan->arena);
  delete plan;
}

sog_status sog_tune_cutoff(int64_t N, double Lx, double Ly, double Lz, double tol,
                           const sog_opts* opts, const void* q, const void* r, const double* n_nb,
                           int32_t ncand, int32_t reps, double* best, float* ms, void* stream) {
  if (!q || !r || !n_nb || !best || ncand < 1 || ncand > 32 || reps < 1 || reps > 100)
    return SOG_ERR_ARG;
  if (opts && opts->manual) return SOG_ERR_ARG;
  for (int c = 0; c < ncand; ++c)
    if (!(n_nb[c] > 0.0) || !std::isfinite(n_nb[c])) return SOG_ERR_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  sog_opts o = opts ? *opts : sog_opts{SOG_PREC_MIXED, SOG_WIN_ES, 0.0, nullptr, 0};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return SOG_ERR_CUDA;
  }
  float best_ms = -1.0f;
  sog_status st = SOG_OK;
  for (int c = 0; c < ncand && st == SOG_OK; ++c) {
    if (ms) ms[c] = -1.0f;
    o.n_nb = n_nb[c];
    sog_plan* p = nullptr;
    const sog_status cs = sog_plan_create(&p, N, Lx, Ly, Lz, tol, &o);
    if (cs == SOG_ERR_PARAMS) continue;  // infeasible candidate
    if (cs != SOG_OK) {
      st = cs;
      break;
    }
    std::vector<float> v;
    for (int i = 0; i <= reps && st == SOG_OK; ++i) {
      cudaEventRecord(e0, s);
      st = sogk::eval_device(p, q, r, nullptr, nullptr, nullptr, nullptr, nullptr, s);
      cudaEventRecord(e1, s);
      if (st != SOG_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        cudaGetLastError();
        st = SOG_ERR_CUDA;
        break;
      }
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      if (i > 0) v.push_back(t);  // the first run captures the graph
    }
    if (st == SOG_OK) st = sog_plan_check(p);
    sog_plan_destroy(p);
    if (st != SOG_OK) break;
    std::sort(v.begin(), v.end());
    const float t = v[v.size() / 2];
    if (ms) ms[c] = t;
    if (best_ms < 0.0f || t < best_ms) {
      best_ms = t;
      *best = n_nb[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SOG_OK) return st;
  return best_ms < 0.0f ? SOG_ERR_PARAMS : SOG_OK;
}

}  // extern "C"
