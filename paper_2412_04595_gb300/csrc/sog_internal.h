// Internal declarations of the GB300 SOG library: the plan, device-side
// geometry records and the launch helpers shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/sog.h"

namespace sogk {

constexpr int kMaxFftStages = 16;
constexpr int kMaxCheb = 64;
constexpr int kMaxWin = 16;
constexpr int kNearD = 8;  // degree of the near-field table polynomials
// Row stride of the near-field table in elements: the kNearD + 1
// coefficients padded to whole 16-byte vectors (FP32: 12 floats = three
// float4, FP64: 10 doubles = five double2), read with vector loads.
template <typename T>
__host__ __device__ constexpr int near_row() { return sizeof(T) == 4 ? 12 : 10; }
constexpr int kMaxHalfModes = 256;  // long range by direct sums: half-plane modes
constexpr int kModeBlocksPerSm = 4;  // CTAs of its moment sums per SM
constexpr int kMaxHalfModeCoefs = 8192;  // half-plane modes x P_cheb (on-chip table)

// Half-plane mode idx of the direct long range: n_x = 0 with n_y = 1..Ky,
// then n_x = 1..Kx with n_y = -Ky..Ky (the other half are the conjugates).
__host__ __device__ inline void half_mode(int idx, int Ky, int& nx, int& ny) {
  if (idx < Ky) {
    nx = 0;
    ny = idx + 1;
  } else {
    const int i = idx - Ky;
    nx = 1 + i / (2 * Ky + 1);
    ny = i % (2 * Ky + 1) - Ky;
  }
}

// One FFT length: radix sequence of the Stockham stages and the offset of its
// n roots of unity exp(-2 pi i t / n) in the twiddle table.
// Twiddle entries per transform length in the plan's table: the constants
// of the radix-16 and radix-15 butterflies (w_16^t, t < 16, then w_15^t,
// t < 15, and one unused entry), then the engine's per-stage tables (n
// entries reserved, n - 1 used).
constexpr int kTwConst = 32;
inline __host__ __device__ int tw_len(int n) { return kTwConst + n; }

struct FftLen {
  int n;
  int nst;
  int radix[kMaxFftStages];
  int tw_off;
  int n16, n15, n8, n4, n2, n3, n5, n7;  // stages of each radix, in this order
};

// Particle record (x, y, z, q) or (local grid coordinates, q).
template <typename T>
struct alignas(4 * sizeof(T)) P4 {
  T x, y, z, q;
};

// Window of Sec. 3.4 / Remark 3.4 on a support of P grid points,
// half-width `half` = (P-1)/2 grid units, shape beta (ES) or S (Gaussian).
// Kaiser-Bessel window I0(beta sqrt(1 - v^2)) / I0(beta) as a power series
// in u = 1 - v^2 (the series of I0): c[k] = (beta^2/4)^k / (k!)^2 / I0(beta),
// rounded to T, up to cap terms; returns the number of terms.  The kernels
// evaluate this series and the plan transforms this same series, so that a
// plan deconvolves exactly the window it applies (coefficients included).
template <typename T>
inline int kb_series(double beta, T* c, int cap) {
  const double x = 0.25 * beta * beta, norm = 1.0 / std::cyl_bessel_i(0.0, beta);
  double t = norm;
  int n = 0;
  for (int k = 0; k < cap; ++k) {
    c[k] = (T)t;
    n = k + 1;
    if (k * k > x && t < 1e-20) break;  // past the peak term (k^2 ~ x) and negligible
    t *= x / ((k + 1.0) * (k + 1.0));
  }
  return n;
}

struct WinPar {
  int P;
  int kind;          // SOG_WIN_ES, SOG_WIN_GAUSS or SOG_WIN_KB
  double half;
  double shape;
  int nu = 0;        // > 0: evaluated through per-point polynomials of degree nu
};

// Largest degree of the polynomial windows.
constexpr int kPolyMax = 12;

// Window phi(v) in FP64 on the host (zero outside |v| <= 1).
inline double win_phi_host(const WinPar& w, double v) {
  if (!(v >= -1.0 && v <= 1.0)) return 0.0;
  const double a = std::sqrt(std::max(0.0, (1.0 - v) * (1.0 + v)));
  if (w.kind == SOG_WIN_ES) return std::exp(w.shape * (a - 1.0));
  if (w.kind == SOG_WIN_KB) return std::cyl_bessel_i(0.0, w.shape * a) / std::cyl_bessel_i(0.0, w.shape);
  return std::exp(-w.shape * v * v);
}

// Polynomial windows (Sec. 3.4, 5.1: Chebyshev interpolation of order nu).
// A particle at grid coordinate t touches g0 + d, d = 0..P-1, g0 =
// ceil(t - half); as a function of sigma = 2 (g0 - t + half) - 1 in [-1, 1)
// the weight of point d is phi((s - half + d) / half), s = (sigma + 1) / 2.
// Its interpolant at the nu + 1 Chebyshev points of the first kind is
// written in monomials of sigma: a[d * (kPolyMax + 1) + j], j = 0..nu
// (coefficients from the discrete orthogonality of T_j at those points,
// then T_j expanded by T_{j+1} = 2 sigma T_j - T_{j-1}; all in FP64).
inline void win_poly_coeffs(const WinPar& w, double* a) {
  const int n = w.nu + 1;
  const double pi = 3.14159265358979323846;
  double T[kPolyMax + 1][kPolyMax + 1] = {};  // monomial coefficients of T_j
  T[0][0] = 1.0;
  if (w.nu >= 1) T[1][1] = 1.0;
  for (int j = 1; j + 1 <= w.nu; ++j)
    for (int i = 0; i <= j + 1; ++i)
      T[j + 1][i] = (i > 0 ? 2.0 * T[j][i - 1] : 0.0) - T[j - 1][i];
  for (int d = 0; d < w.P; ++d) {
    double c[kPolyMax + 1] = {};
    for (int i = 0; i < n; ++i) {
      const double th = (i + 0.5) * pi / n, sg = std::cos(th);
      const double f = win_phi_host(w, (0.5 * (sg + 1.0) - w.half + d) / w.half);
      for (int j = 0; j < n; ++j) c[j] += f * std::cos(j * th);
    }
    for (int j = 0; j < n; ++j) c[j] *= (j == 0 ? 1.0 : 2.0) / n;
    double* ad = a + d * (kPolyMax + 1);
    for (int i = 0; i <= kPolyMax; ++i) ad[i] = 0.0;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i <= j; ++i) ad[i] += c[j] * T[j][i];
  }
}

// Tiling of a periodic grid for spreading / gathering.
struct TileGeom {
  int I[3];          // grid sizes (z unused in 2D)
  int T[3];          // tile edge
  int nt[3];         // tiles per dimension
  int W[3];          // padded tile edge = T + P
  int pad_lo;        // floor(half): padded tile starts pad_lo before the tile
  int pitch;         // row pitch of the real grid (I[0] + 2)
  int chunks;        // CTAs per tile
};

// Tile kernels of the spreading and gathering steps.
constexpr int kTileThreads = 256;  // 8 warps; the spread's row ownership relies on it
constexpr int kTileBatch = 32;     // particles whose window weights are staged at once
constexpr int kTileHeader = 896;   // bytes of row tables and per-particle offsets
constexpr int kLongSpreadHeader = 1024;  // the same for the long-range gridding (P_cheb planes)
constexpr int kGatherBatch = 128;  // particles per batch of the gathers (two threads each)
constexpr int kGatherHeader = 1280;

__host__ __device__ inline int mod32(int a) { return ((a % 32) + 32) % 32; }
// Shared-memory strides of the padded tile (in elements), chosen so that the
// 32 lanes of a warp touch 32 different banks:
//   spreading: lanes over (dz, dx) of a window row, plane stride = P (mod 32);
//   gathering: lanes over (dz, dy) rows, odd row pitch rp and plane stride
//   = P rp (mod 32), so that lane e reads word e rp + dx (mod 32).
__host__ __device__ inline int spread_plane_stride(int W0, int W1, int P) {
  return W0 * W1 + mod32(P - W0 * W1);
}
__host__ __device__ inline int gather_row_pitch(int W0) { return W0 | 1; }
__host__ __device__ inline int gather_plane_stride(int rp, int W1, int P) {
  return rp * W1 + mod32(P * rp - rp * W1);
}

// Blocks of the grid-stride reductions (binning sums, assembly / energy)
// and of the k = 0 moments, per SM of the plan's device.
constexpr int kRedBlocksPerSm = 2;
constexpr int kK0BlocksPerSm = 1;
// Largest dynamic shared memory of one CTA on sm_100-class GPUs (227 KB).
constexpr int kMaxDynSmem = 232448;
// Captured evaluations kept per plan (keyed by the caller's pointers).
constexpr int kMaxGraphs = 4;

struct GraphEntry {
  const void* q;
  const void* r;
  void* phi;
  double* E;
  void* F;
  double* pp;
  double* pg;
  int timing;                      // stage events captured in the graph
  int ev_used[2 * SOG_NSTAGES];
  cudaGraphExec_t exec;
  int64_t launches;
  uint64_t last_use;
};

}  // namespace sogk

struct sog_plan {
  sog_params prm;
  int prec;
  int64_t N;
  int device;
  int n_sm;           // SMs of the device; the block counts below follow it
  int red_blocks;     // kRedBlocksPerSm x n_sm
  int mode_blocks;    // kModeBlocksPerSm x n_sm
  int k0_blocks;      // kK0BlocksPerSm x n_sm
  // derived geometry
  double h[3];        // mid grid spacing
  double Lzs;         // padded box Lz*
  double hl[2];       // long grid spacing
  bool has_mid, has_long;
  int nc[3];          // near-field cells
  double cell[3];
  int n_cells;
  sogk::TileGeom gm, gl;
  int n_tiles_mid, n_tiles_long;
  sogk::WinPar wm, wl;
  sogk::FftLen fx, fy, fz, flx, fly;
  int near_K, near_D;
  double selfsum;
  // device arena and typed views (element type T = plan precision)
  void* arena;
  int64_t arena_bytes;
  void* d_tw;          // twiddles, T2
  void* d_near_tab;    // near table, T
  void* d_mult;        // mid scaling factors, T
  void* d_kmat;        // long z-kernels per half-plane mode (Algorithm 3), T
  // Algorithm 2 z-kernel in factorised form (no per-mode table):
  //   K_k = fx(kx) fy(ky) sum_l c1_l e^{-c2_l |k|^2} B_l
  void* d_lbl;         // B_l, l = m+1..M: even and odd parity blocks [2][lps][lps], T
  void* d_lcl;         // (c1_l, c2_l) = ((pi/A) w_l s_l^2, s_l^2 / 4), T pairs
  void* d_lfx;         // (kx^2, hx^2 / What_x(kx)^2) per half-spectrum column, T pairs
  void* d_lfy;         // (ky^2, hy^2 / What_y(ky)^2) per row, T pairs
  int n_lg;            // long-range Gaussians M - m
  int n_lg_used;       // those with c2_l k_min^2 <= lg_xmax for the smallest mode k != 0
  double lg_xmax;      // terms with c2_l |k|^2 > lg_xmax are dropped: 80 in FP64,
                       // 20 in FP32 (below 1e-8 of the mode's largest term)
  int lps;             // parity block edge ceil(P_cheb / 2)
  int lpst;            // row stride of a parity block (lps rounded up to 4)
  int long_fused;      // y pass, contraction and inverse y pass in one kernel
  double* d_k0mat;     // k = 0 z-kernel, P x P, double
  void* d_grid;        // mid grid, T
  void* d_lA;          // long planes, T
  void* d_lB;          // long planes after the z-contraction, T
  void* d_rec_near;    // P4<T>
  void* d_rec_mid;
  void* d_rec_long;
  void* d_rec_tmp;     // 3 x N records in input order (binning)
  int* d_perm;         // 3 x N
  int* d_key;          // 3 x N
  int* d_rank;         // 3 x N
  int* d_cnt;          // counts / starts of the three bin sets
  int cnt_off[4];
  int cnt_cap;         // entries of d_cnt (sized for the smallest tiles the autotuner tries)
  int mid_T, long_T;   // nominal tile edges of the current tiling
  double mid_cscale, long_cscale;  // CTAs per tile relative to the default rule
  double* d_parts_phi;   // 4 x N
  double* d_parts_grad;  // 4 x N x 3
  double* d_red;         // reduction partials
  double* d_k0nu;        // P
  int* d_status;         // latched errors (bit 0 non-neutral, bit 1 out of box, bit 2 timeout)
  void* d_host_stage;    // device copies of q, r, phi, F, E for sog_eval_host
  int long_small;        // long planes small enough for one private copy per CTA
  int long_small_blocks;
  void* d_long_partial;  // per-CTA copies of the long planes (small path)
  int long_direct;       // long range by direct Fourier sums (Algorithm 3)
  int n_half;            // its half-plane modes
  double* d_lmom;        // per-block partial moments [block][mode][n][re, im]
  void* d_lcoef;         // coefficients [mode][n][re, im] in the element type
  int launch_error;
  cudaStream_t last_stream;
  // stage timers (sog_plan_set_timing) and kernel launch count of the last eval
  int timing, events_ready;
  cudaEvent_t ev[2 * SOG_NSTAGES];   // start and end of each stage
  int ev_used[2 * SOG_NSTAGES];
  int64_t launches;
  // captured evaluations replayed with one cudaGraphLaunch; after the
  // binning the near field (side_stream), the long range (long_stream) and
  // its k = 0 mode (k0_stream) run concurrently with the mid range
  cudaStream_t cap_stream;
  cudaStream_t side_stream, long_stream, k0_stream;
  cudaEvent_t ev_fork, ev_join, ev_join_long, ev_join_k0;
  sogk::GraphEntry graphs[sogk::kMaxGraphs];
  int n_graphs;
  uint64_t use_clock;
  int use_graphs;
};

namespace sogk {

// SOG weight w_l of Eq. (2.22) (w_0 scaled by omega, Eq. 2.25), and the
// weights and bandwidths s_l, l = 0..M, built from it (sog_plan.cpp).
double sog_weight(double b, double sigma, double omega, int l);
void sog_table(double b, double sigma, double omega, int M, std::vector<double>& w,
               std::vector<double>& s);

// Host-side launchers (sog_fft.cu).
// Each adds the number of kernels it launched to `launches`.
template <typename T>
cudaError_t fft_mid_forward_conv_inverse(const sog_plan* p, cudaStream_t s, int& launches);
// Algorithm 2 steps 2-4 on the proxy planes d_lA (layout [n][y][x], pitch
// Ix_long + 2): forward 2D FFTs, the factorised z-contraction, backward 2D
// FFTs; the result is left in d_lA (d_lB is scratch).
template <typename T>
cudaError_t fft_long_solve(const sog_plan* p, cudaStream_t s, int& launches);
template <typename T>
cudaError_t fft_prepare();
bool fft_len_ok(int prec, const FftLen& f);
// Whether the fused y pass (all P_cheb planes of one half-spectrum column in
// one CTA's shared memory) fits, for element size es.
bool long_fused_fits(int P, const FftLen& fy, int nl, size_t es);
size_t long_fused_smem(int P, const FftLen& fy, int nl, size_t es);

// Dynamic shared memory of the mid / long gridding (gather = false) and
// gathering kernels for the plan's current tiles (sog_kernels.cu).
size_t mid_smem(const sog_plan* p, size_t es, bool gather);
size_t long_smem(const sog_plan* p, size_t es, bool gather);

// One-time kernel attributes for the plan's element type (sog_kernels.cu).
cudaError_t prepare_kernels(int prec);
void release_graphs(sog_plan* p);
// Enqueue one evaluation's kernels on s without a graph of the plan's own
// (used while a batch of plans is being captured into one graph).
cudaError_t enqueue_eval(sog_plan* p, const void* q, const void* r, void* phi, double* E, void* F,
                         cudaStream_t s);

// Host side of one evaluation (sog_kernels.cu).
sog_status eval_device(sog_plan* p, const void* q, const void* r, void* phi, double* E, void* F,
                       double* phi_parts, double* grad_parts, cudaStream_t s);

}  // namespace sogk
