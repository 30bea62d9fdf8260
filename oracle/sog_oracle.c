/*
 * FP64 CPU oracle: the slow, plain reference sums used to check the GPU path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may link, load or call this file; only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark use it.  It shares no
 * code, header or table with the CUDA path.
 *
 * Contents (each a direct transcription of a definition, no acceleration
 * beyond OpenMP over independent targets):
 *   oracle_ewald2d        Ewald2D reference solution for the quasi-2D sum
 *                         (the "true" solution of Sec. 5; textbook Ewald
 *                         splitting of Eq. (2.6) with the 2D-periodic
 *                         reciprocal sum done in closed form in z).
 *   oracle_brute_images   Eq. (2.6) summed literally over a square of images.
 *   oracle_near           near-field sum Phi^N of Eq. (2.28): minimum image,
 *                         kernel 1/r - F_M(r) for r < r_c, F_M of Eq. (2.21)
 *                         evaluated term by term.
 *   oracle_gauss_images   sum_j q_j sum_n sum_l w_l exp(-|r_ij+n L|^2/s_l^2)
 *                         in real space (the mid-range kernel of Eq. (1.1),
 *                         without the z-periodisation of Algorithm 1).
 *
 * Positions are in the paper's centred box (Sec. 2.1): x in [-Lx/2, Lx/2],
 * periodic in x and y, free in z.  Arrays are row-major N x 3.
 * "grad" outputs are the gradient of the potential at each target; the force
 * on a charge q_i at that target is -q_i * grad.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846;

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* exp(a) * erfc(u) without overflow of exp(a) when erfc(u) is tiny.
 * erfc(u) underflowing to zero makes the product zero, which is its
 * double-precision value whenever that happens for the arguments used here
 * (the exact product is bounded by exp(-u^2/2)). */
static double exp_erfc(double a, double u) {
  double e = erfc(u);
  if (e <= 0.0) return 0.0;
  return exp(a + log(e));
}

/*
 * Ewald2D (Parry's quasi-2D Ewald sum).  For a target at r_i:
 *   Phi = sum_j sum_n' q_j erfc(a|d|)/|d|,  d = r_i - r_j + n o L, |d| < rcut
 *       + (pi/A) sum_j q_j sum_{k != 0, |k| <= kmax} cos(k.rho_ij)/|k|
 *              [e^{k z} erfc(k/(2a) + a z) + e^{-k z} erfc(k/(2a) - a z)]
 *       - (2 pi/A) sum_j q_j [z erf(a z) + e^{-a^2 z^2}/(a sqrt(pi))]
 *       - (2 a/sqrt(pi)) q_self
 * with z = z_i - z_j, A = Lx Ly.  tself[i] >= 0 names the source index that
 * coincides with target i (excluded from the n = 0 real-space term, and the
 * self term added); -1 means the target is not a source.
 */
void oracle_ewald2d(int nt, const double* tr, const int64_t* tself, int ns,
                    const double* q, const double* sr, double Lx, double Ly,
                    double alpha, double rcut, double kmax, double* phi,
                    double* grad) {
  const double A = Lx * Ly;
  const int nxm = (int)ceil(rcut / Lx) + 1;
  const int nym = (int)ceil(rcut / Ly) + 1;
  const int kxm = (int)ceil(kmax * Lx / (2.0 * PI));
  const int kym = (int)ceil(kmax * Ly / (2.0 * PI));
  const double two_a_sqpi = 2.0 * alpha / sqrt(PI);

#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < nt; ++i) {
    const double xi = tr[3 * i], yi = tr[3 * i + 1], zi = tr[3 * i + 2];
    double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int j = 0; j < ns; ++j) {
      const double qj = q[j];
      const double dx0 = xi - sr[3 * j], dy0 = yi - sr[3 * j + 1];
      const double z = zi - sr[3 * j + 2];
      /* real space */
      for (int nx = -nxm; nx <= nxm; ++nx) {
        for (int ny = -nym; ny <= nym; ++ny) {
          if (nx == 0 && ny == 0 && tself[i] == j) continue;
          const double dx = dx0 + nx * Lx, dy = dy0 + ny * Ly;
          const double r2 = dx * dx + dy * dy + z * z;
          if (r2 >= rcut * rcut) continue;
          const double r = sqrt(r2);
          const double e = erfc(alpha * r) / r;
          p += qj * e;
          /* d/dr [erfc(a r)/r] */
          const double de = -e / r - two_a_sqpi * exp(-alpha * alpha * r2) / r;
          gx += qj * de * dx / r;
          gy += qj * de * dy / r;
          gz += qj * de * z / r;
        }
      }
      /* reciprocal space, k != 0 (pairs +k/-k summed together) */
      for (int mx = -kxm; mx <= kxm; ++mx) {
        for (int my = -kym; my <= kym; ++my) {
          if (mx < 0 || (mx == 0 && my <= 0)) continue; /* half plane */
          const double kx = 2.0 * PI * mx / Lx, ky = 2.0 * PI * my / Ly;
          const double k = sqrt(kx * kx + ky * ky);
          if (k > kmax) continue;
          const double fp = exp_erfc(k * z, k / (2.0 * alpha) + alpha * z);
          const double fm = exp_erfc(-k * z, k / (2.0 * alpha) - alpha * z);
          const double ph = kx * dx0 + ky * dy0;
          const double c = cos(ph), s = sin(ph);
          const double pre = 2.0 * PI / A * qj / k; /* x2 for the -k partner */
          p += pre * c * (fp + fm);
          gx += -pre * s * kx * (fp + fm);
          gy += -pre * s * ky * (fp + fm);
          gz += pre * c * k * (fp - fm);
        }
      }
      /* k = 0 */
      p += -2.0 * PI / A * qj *
           (z * erf(alpha * z) + exp(-alpha * alpha * z * z) / (alpha * sqrt(PI)));
      gz += -2.0 * PI / A * qj * erf(alpha * z);
    }
    if (tself[i] >= 0) p -= two_a_sqpi * q[tself[i]];
    phi[i] = p;
    if (grad) {
      grad[3 * i] = gx;
      grad[3 * i + 1] = gy;
      grad[3 * i + 2] = gz;
    }
  }
}

/*
 * Eq. (2.6) summed over the square of images |nx|, |ny| <= R (n = 0 with
 * j = tself[i] excluded).  Converges like 1/R for a neutral system; the
 * caller extrapolates in R.
 */
void oracle_brute_images(int nt, const double* tr, const int64_t* tself, int ns,
                         const double* q, const double* sr, double Lx,
                         double Ly, int R, double* phi) {
  for (int i = 0; i < nt; ++i) {
    double p = 0.0;
#pragma omp parallel for reduction(+ : p) schedule(static)
    for (int nx = -R; nx <= R; ++nx) {
      double pl = 0.0;
      for (int ny = -R; ny <= R; ++ny) {
        for (int j = 0; j < ns; ++j) {
          if (nx == 0 && ny == 0 && tself[i] == j) continue;
          const double dx = tr[3 * i] - sr[3 * j] + nx * Lx;
          const double dy = tr[3 * i + 1] - sr[3 * j + 1] + ny * Ly;
          const double dz = tr[3 * i + 2] - sr[3 * j + 2];
          pl += q[j] / sqrt(dx * dx + dy * dy + dz * dz);
        }
      }
      p += pl;
    }
    phi[i] = p;
  }
}

/* F_M(r) = sum_{l=0}^{M} w_l exp(-r^2/s_l^2)  (Eq. (2.21)), and dF_M/dr. */
static void sog_far(double r, int nl, const double* w, const double* s,
                    double* F, double* dF) {
  double f = 0.0, d = 0.0;
  for (int l = 0; l < nl; ++l) {
    const double e = w[l] * exp(-(r * r) / (s[l] * s[l]));
    f += e;
    d += -2.0 * r / (s[l] * s[l]) * e;
  }
  *F = f;
  *dF = d;
}

/*
 * Near field of Eq. (2.28): Phi^N_i = sum_{j != i} q_j (1/r - F_M(r)) over
 * pairs with r < rc, minimum image in x and y (valid for rc <= min(Lx,Ly)/2).
 * nl = M + 1 Gaussians (w, s).  Every source is visited for every target.
 */
void oracle_near(int nt, const double* tr, const int64_t* tself, int ns,
                 const double* q, const double* sr, double Lx, double Ly,
                 double rc, int nl, const double* w, const double* s,
                 double* phi, double* grad) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < nt; ++i) {
    double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int j = 0; j < ns; ++j) {
      if (tself[i] == j) continue;
      double dx = tr[3 * i] - sr[3 * j];
      double dy = tr[3 * i + 1] - sr[3 * j + 1];
      const double dz = tr[3 * i + 2] - sr[3 * j + 2];
      dx -= Lx * nearbyint(dx / Lx);
      dy -= Ly * nearbyint(dy / Ly);
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 < rc * rc)) continue;
      const double r = sqrt(r2);
      double F, dF;
      sog_far(r, nl, w, s, &F, &dF);
      p += q[j] * (1.0 / r - F);
      const double dG = -1.0 / r2 - dF; /* d/dr (1/r - F_M) */
      gx += q[j] * dG * dx / r;
      gy += q[j] * dG * dy / r;
      gz += q[j] * dG * dz / r;
    }
    phi[i] = p;
    if (grad) {
      grad[3 * i] = gx;
      grad[3 * i + 1] = gy;
      grad[3 * i + 2] = gz;
    }
  }
}

/*
 * Real-space image sum of a set of Gaussians, self term included:
 *   Phi_i = sum_j q_j sum_{n in Z^2 x {0}} sum_l w_l exp(-|r_ij + n o L|^2/s_l^2).
 * Images are taken while the widest Gaussian is above 1e-300 of its peak.
 */
void oracle_gauss_images(int nt, const double* tr, int ns, const double* q,
                         const double* sr, double Lx, double Ly, int nl,
                         const double* w, const double* s, double* phi,
                         double* grad) {
  double smax = 0.0;
  for (int l = 0; l < nl; ++l) smax = s[l] > smax ? s[l] : smax;
  const double reach = smax * sqrt(log(1e300));
  const int nxm = (int)ceil(reach / Lx) + 1;
  const int nym = (int)ceil(reach / Ly) + 1;
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < nt; ++i) {
    double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int j = 0; j < ns; ++j) {
      const double dz = tr[3 * i + 2] - sr[3 * j + 2];
      for (int nx = -nxm; nx <= nxm; ++nx) {
        const double dx = tr[3 * i] - sr[3 * j] + nx * Lx;
        for (int ny = -nym; ny <= nym; ++ny) {
          const double dy = tr[3 * i + 1] - sr[3 * j + 1] + ny * Ly;
          const double r2 = dx * dx + dy * dy + dz * dz;
          for (int l = 0; l < nl; ++l) {
            const double e = q[j] * w[l] * exp(-r2 / (s[l] * s[l]));
            p += e;
            const double c = -2.0 / (s[l] * s[l]) * e;
            gx += c * dx;
            gy += c * dy;
            gz += c * dz;
          }
        }
      }
    }
    phi[i] = p;
    if (grad) {
      grad[3 * i] = gx;
      grad[3 * i + 1] = gy;
      grad[3 * i + 2] = gz;
    }
  }
}
