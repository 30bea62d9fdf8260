/*
 * sog.h -- C ABI of the GB300 spectral sum-of-Gaussians (SOG) library.
 *
 * Computes, for N point charges q_i at r_i in a box that is periodic in x and
 * y and free in z, the potential of Eq. (2.6),
 *     Phi_i = sum_j sum'_{n in Z^2 x {0}} q_j / |r_i - r_j + n o L|,
 * the energy U = 1/2 sum_i q_i Phi_i and the forces F_i = -q_i grad Phi(r_i)
 * (Sec. 2.3), by the spectral SOG method: the kernel split of Eq. (1.1) into
 * a near field (direct sum over cell lists, Eq. 2.28), a mid range (3D
 * spectral solver, Algorithm 1) and a long range (2D spectral solver with
 * Chebyshev proxy points in z, Algorithm 2), minus the self term (Eq. 2.28).
 * Gaussian units: no 1/(4 pi eps0) factor.
 *
 * Conventions shared by every entry point
 *   - Box: the centred box of Sec. 2.1, x in [-Lx/2, Lx/2), y in
 *     [-Ly/2, Ly/2), z in [-Lz/2, Lz/2].  x and y outside their interval
 *     are wrapped by one period; z must lie inside its interval.
 *   - The system must be neutral (Eq. 2.4): |sum q| <= 1e-10 sum |q|.
 *   - Precision: the plan fixes the element type of q, r, phi and F:
 *     double for SOG_PREC_FP64, float for SOG_PREC_MIXED.  E is always a
 *     double.  r is N x 3 row-major (x0 y0 z0 x1 ...), F likewise.
 *   - Memory: unless an entry point says "host", every array argument is a
 *     device pointer on the plan's device, owned by the caller, and must stay
 *     valid until the work enqueued on `stream` has finished.  The plan owns
 *     all workspace memory, allocated once by sog_plan_create.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL: the legacy
 *     default stream).  Device entry points only enqueue work and return; a
 *     plan must not be used by two streams at the same time.
 *   - Errors: argument errors are returned at once.  Data errors found on
 *     the device (non-neutral charges, z outside the box, non-finite
 *     coordinates) are latched in the plan and returned by sog_plan_check;
 *     the outputs of such a call are unspecified but finite memory accesses
 *     are guaranteed (coordinates are clamped into the grid).
 */
#ifndef SOG_H
#define SOG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sog_plan sog_plan;

typedef enum {
  SOG_OK = 0,
  SOG_ERR_ARG = 1,          /* invalid argument: NULL pointer, N < 2, L <= 0, tol not in (0, 0.1] */
  SOG_ERR_NONNEUTRAL = 2,   /* |sum q| > 1e-10 sum |q| (Eq. 2.4); from sog_plan_check */
  SOG_ERR_OUT_OF_BOX = 3,   /* a z outside [-Lz/2, Lz/2] or a non-finite coordinate; from sog_plan_check */
  SOG_ERR_NOMEM = 4,        /* device or host allocation failed */
  SOG_ERR_CUDA = 5,         /* a CUDA call or kernel launch failed */
  SOG_ERR_PARAMS = 6,       /* no feasible or an inconsistent parameter set */
  SOG_ERR_TIMEOUT = 7       /* a kernel's bounded wait for its own asynchronous copies ran out;
                               from sog_plan_check (the outputs of that call are unspecified) */
} sog_status;

enum { SOG_PREC_FP64 = 0, SOG_PREC_MIXED = 1 };
enum { SOG_WIN_ES = 0, SOG_WIN_GAUSS = 1, SOG_WIN_KB = 2 };

/*
 * Method parameters (Sec. 4.3 names).  Filled by sog_select_params or by the
 * caller (sog_opts.manual).
 *   L        box lengths (Lx, Ly, Lz)
 *   b, r0, omega   SOG row (Table 1): bandwidth ratio, scaled cutoff, w_0 factor
 *   sigma    = rc / r0; w_l, s_l of Eq. (2.22), (2.25), l = 0..M
 *   rc       near-field cutoff, rc <= min(Lx, Ly)/2 (minimum image)
 *   M        last Gaussian; m last mid-range Gaussian (Def. 3.2), -1: none;
 *            Gaussians m+1..M are long range
 *   I        mid grid Ix, Iy, Iz* (Iz* spans the padded box, Eq. 3.20)
 *   hz       mid grid spacing in z; Lz* = Iz* hz
 *   P_win    window support in grid points (Sec. 3.4), 2..16
 *   shape    window shape: ES or KB beta, or Gaussian S (Eq. 4.7)
 *   I_long   long-range grid Ix_long, Iy_long (Sec. 3.4)
 *   P_long, shape_long   long-range window support and shape
 *   P_cheb   number of Chebyshev proxy points in z (Eq. A.6), 2..64
 *   window   SOG_WIN_ES, SOG_WIN_GAUSS or SOG_WIN_KB (Kaiser-Bessel,
 *            I0(beta sqrt(1 - v^2)) / I0(beta); Remark 3.4, Sec. 5.1)
 *   long_direct  0: long range by window gridding and 2D FFTs (Algorithm 2);
 *            1: by direct Fourier sums without FFT (Algorithm 3) over the
 *            modes |n_x| <= (Ix_long-1)/2, |n_y| <= (Iy_long-1)/2 (odd
 *            counts; P_long and shape_long unused)
 *   win_poly 0: windows evaluated directly; 2..12: through polynomials of
 *            this degree nu (Sec. 3.4, 5.1): a particle at grid coordinate t
 *            touches points g0 + d, d = 0..P-1, g0 = ceil(t - half), and the
 *            weight of point d is the Chebyshev interpolant, at nu + 1
 *            first-kind points, of the window as a function of
 *            sigma = 2 (g0 - t + half) - 1 in [-1, 1), evaluated by Horner.
 *            The spectral scaling keeps the exact window's transform; the
 *            approximation error is about 4e-8 (P = 9, nu >= 8) to 1e-12
 *            (P = 16, nu = 10) of the window's peak for ES.
 * Grid sizes must be even; Ix, Iy, Iz*, Ix_long, Iy_long factor into 2,3,5,7
 * Long-range mode counts of long_direct: odd; the half-plane modes
 * Ky + Kx (2 Ky + 1) (K = (I_long - 1) / 2) at most 256, and times P_cheb
 * at most 8192 (the coefficient table is held on chip).
 */
typedef struct sog_params {
  double L[3];
  double b, r0, omega, sigma, rc;
  int32_t M, m;
  int32_t I[3];
  double hz;
  int32_t P_win;
  double shape;
  int32_t I_long[2];
  int32_t P_long;
  double shape_long;
  int32_t P_cheb;
  int32_t window;
  int32_t long_direct;
  int32_t win_poly;
} sog_params;

/*
 * Plan options.  precision: SOG_PREC_*.  window: window of the analytic
 * selection.  n_nb: neighbours per particle the cutoff is sized for
 * ((4/3) pi rc^3 rho = n_nb); <= 0 selects 120.  manual: when non-NULL the
 * parameters are used verbatim (N, L and tol arguments still checked).
 * win_poly: the analytic selection's win_poly (0 or 2..12, see sog_params).
 */
typedef struct sog_opts {
  int32_t precision;
  int32_t window;
  double n_nb;
  const sog_params* manual;
  int32_t win_poly;
} sog_opts;

/*
 * Analytic parameter selection of Sec. 4.3 (host only, no device work):
 * Table 1 row, cutoff from the density, M, mid grid from K_max (Theorem 4.2),
 * window support, then the split index m, padding Lz* and Chebyshev order P
 * chosen by minimising an operation count (the role of Eq. 4.49) under the
 * error constraints of Theorems 3.1, 4.4 and 4.7.  opts may be NULL.
 * Returns SOG_ERR_ARG or SOG_ERR_PARAMS on failure; `out` is host memory.
 */
sog_status sog_select_params(int64_t N, double Lx, double Ly, double Lz, double tol,
                             const sog_opts* opts, sog_params* out);

/*
 * Create a plan for N charges in the box (Lx, Ly, Lz) at relative tolerance
 * tol on the current CUDA device: selects (or takes) the parameters, builds
 * the FP64 tables (SOG weights, window transforms, spectral scaling factors,
 * Chebyshev z-kernels, near-field kernel table) and allocates every
 * workspace.  *plan is owned by the caller and released by sog_plan_destroy.
 * opts may be NULL (mixed precision, ES window, n_nb = 120).
 */
sog_status sog_plan_create(sog_plan** plan, int64_t N, double Lx, double Ly, double Lz,
                           double tol, const sog_opts* opts);

/* Copy the plan's parameters to host memory `out`. */
sog_status sog_plan_get_params(const sog_plan* plan, sog_params* out);

/* Element type of the plan's q, r, phi, F: SOG_PREC_FP64 or SOG_PREC_MIXED. */
int32_t sog_plan_precision(const sog_plan* plan);

/* Bytes of device memory the plan holds. */
int64_t sog_plan_device_bytes(const sog_plan* plan);

/*
 * Evaluate potentials, energy and forces (Eq. 3.22 with the self term
 * subtracted; U and F as in Sec. 2.3).
 *   q    [N]      charges                         (device, plan type)
 *   r    [N x 3]  positions                       (device, plan type)
 *   phi  [N]      potentials Phi_i, or NULL       (device, plan type)
 *   E    [1]      energy U, or NULL               (device, double)
 *   F    [N x 3]  forces, or NULL                 (device, plan type)
 * Enqueued on `stream`; returns without waiting.
 */
sog_status sog_eval(sog_plan* plan, const void* q, const void* r, void* phi, double* E,
                    void* F, void* stream);

/*
 * Same work as sog_eval, but also (or only) returns the four parts of the
 * potential before the self term, in double: part 0 near field (Eq. 2.28),
 * 1 mid range (Algorithm 1), 2 long range without its k = 0 mode
 * (Algorithm 2), 3 the k = 0 mode of the long range.
 *   phi_parts  [4 x N]      device, double (NULL to skip)
 *   grad_parts [4 x N x 3]  gradients of the parts, device, double (NULL to skip)
 */
sog_status sog_eval_components(sog_plan* plan, const void* q, const void* r,
                               double* phi_parts, double* grad_parts, void* stream);

/*
 * sog_eval on host buffers: copies q and r to the device, evaluates, copies
 * phi, E and F back (any of them may be NULL) and waits for completion.
 * All pointers are host pointers of the plan's element type (E: double).
 * Returns the data status of the call as sog_plan_check would.
 */
sog_status sog_eval_host(sog_plan* plan, const void* q, const void* r, void* phi, double* E,
                         void* F);

/*
 * Wait for the plan's last stream, then return and clear the data status
 * latched by the device since the previous check (SOG_ERR_NONNEUTRAL,
 * SOG_ERR_OUT_OF_BOX, SOG_ERR_TIMEOUT), or SOG_ERR_CUDA if a launch failed.
 */
sog_status sog_plan_check(sog_plan* plan);

/*
 * Stage timers.  With timing enabled (enable = 1), every evaluation records
 * CUDA events on its stream at the start and end of each stage; the stages
 * run concurrently as usual, so a stage's time includes any wait for SMs held
 * by the others.  With enable = 2 every stage runs on the caller's stream one
 * after another (no concurrency), so each time is the isolated duration of
 * that stage's kernels.  sog_plan_get_timing waits for the last evaluation
 * and writes the device time of each stage in milliseconds to
 * ms[SOG_NSTAGES] (host memory; 0 for stages that did not run):
 *   0 binning and sorts        1 near field (Eq. 2.28)
 *   2 mid gridding (Eq. 3.7)   3 mid FFT / scaling / inverse FFT (Eq. 3.8)
 *   4 mid gathering (Eq. 3.10) 5 long gridding onto proxy planes
 *   6 long 2D FFTs and z-contraction (Eq. 3.17)
 *   7 long gathering (Eq. 3.19) 8 k = 0 mode       9 assembly and energy
 * With long_direct (Algorithm 3) stages 5-7 are the mode moments, the mode
 * coefficients and the evaluation at the particles.
 */
#define SOG_NSTAGES 10
sog_status sog_plan_set_timing(sog_plan* plan, int32_t enable);
sog_status sog_plan_get_timing(sog_plan* plan, float* ms);

/* Number of kernels the last evaluation launched. */
int64_t sog_plan_launches(const sog_plan* plan);

/*
 * Autotuner of the gridding and gathering tiles (the paper selects no tiles;
 * an implementation choice timed on this GPU).  Tries mid-range tile edges
 * {8, 12, 16, 20, 23} (evened out over the grid, tile edge + window support
 * <= 32) and 0.5, 1 and 2 times the default number of CTAs per tile, timing
 * the mid gridding plus gathering stages of `reps` evaluations of (q, r)
 * (device arrays as in sog_eval) each in isolation (timing mode 2), and
 * keeps the fastest; then the same for the long-range tiles (gridded form
 * with several tiles).  Results are unchanged up to rounding.  Synchronous;
 * on return the plan's timing mode is restored and its captured evaluations
 * are released.  reps in 1..100.
 * sog_plan_tiles writes to host out[4]: mid tile edge, mid CTAs per tile,
 * long tile edge, long CTAs per tile (0 where the part is absent).
 */
sog_status sog_plan_autotune(sog_plan* plan, const void* q, const void* r, int32_t reps,
                             void* stream);
sog_status sog_plan_tiles(const sog_plan* plan, int32_t* out);

/*
 * Cutoff selection by run time (Sec. 4.3: r_c is chosen to optimise the run
 * time of the near field and the far field, ~ rho^(-1/3) as the rough
 * estimate).  For each candidate neighbour count n_nb[c] (the analytic
 * selection of sog_select_params with opts->n_nb = n_nb[c], every other
 * parameter following from the tolerance as there), a plan is created,
 * evaluated reps + 1 times on q, r (the first run captures its graph) and
 * timed with CUDA events on `stream`, then destroyed; the fastest
 * candidate's n_nb is written to host *best, the median times to host
 * ms[c] (may be NULL; a candidate whose parameters are infeasible gets -1).
 * Every candidate meets the tolerance by construction.  Synchronous;
 * allocates and frees one plan at a time.
 *   N, L, tol, opts   as for sog_plan_create (opts->manual must be NULL;
 *                     opts->n_nb is ignored)
 *   q, r              device, the plan type's element type, as in sog_eval
 *   n_nb, ncand       host array of 1 <= ncand <= 32 candidates, each > 0
 *   reps              1..100
 * Errors: SOG_ERR_ARG for bad arguments; SOG_ERR_PARAMS when no candidate is
 * feasible; the first CUDA or data error of an evaluation otherwise.
 */
sog_status sog_tune_cutoff(int64_t N, double Lx, double Ly, double Lz, double tol,
                           const sog_opts* opts, const void* q, const void* r, const double* n_nb,
                           int32_t ncand, int32_t reps, double* best, float* ms, void* stream);

/*
 * Measured fused multiply-add rate of the current device (a measurement
 * utility; the paper has no counterpart): FP32 (precision SOG_PREC_MIXED) or
 * FP64 (SOG_PREC_FP64) FMAs in independent chains on every SM, timed with
 * CUDA events, in TFLOP/s (2 flop per FMA), written to host *tflops.  It is
 * the peak that the ALU-bound steps (near field, gridding, gathering) are
 * reported against.  Synchronous; allocates 8 bytes of device memory for the
 * duration of the call.
 */
sog_status sog_measure_fma_peak(int32_t precision, double* tflops);

/*
 * Batches of independent systems (row "batching" of the hot path; the paper
 * evaluates one system at a time).  Each system i has its own plan, with
 * parameters selected for (N[i], L[3i..3i+2], tol[i]); one sog_batch_eval
 * replays all systems' evaluations as one CUDA graph, the systems running
 * concurrently.
 *   sog_batch_create: nsys >= 1; N [nsys], L [nsys x 3], tol [nsys] host
 *     arrays; opts as for sog_plan_create (opts->manual must be NULL).
 *     Returns the first failing plan's status.  *batch owned by the caller.
 *   sog_batch_eval: q, r, phi, F are host arrays of nsys device pointers
 *     (each as in sog_eval for its system; phi and F may be NULL arrays, or
 *     hold NULL entries only if all systems do the same across calls); E is
 *     a device array of nsys doubles or NULL.  Enqueued on `stream`.  The
 *     graph is captured on the first call and reused while the pointers stay
 *     the same (a change of pointers re-captures it).
 *   sog_batch_check: waits, returns the first data status of any system (as
 *     sog_plan_check) and its index in *first_bad (-1 if none; may be NULL).
 *   sog_batch_plan: the plan of system i (owned by the batch), e.g. for
 *     sog_plan_get_params; NULL if out of range.
 */
typedef struct sog_batch sog_batch;
sog_status sog_batch_create(sog_batch** batch, int32_t nsys, const int64_t* N, const double* L,
                            const double* tol, const sog_opts* opts);
sog_status sog_batch_eval(sog_batch* batch, const void* const* q, const void* const* r,
                          void* const* phi, double* E, void* const* F, void* stream);
sog_status sog_batch_check(sog_batch* batch, int32_t* first_bad);
int32_t sog_batch_size(const sog_batch* batch);
sog_plan* sog_batch_plan(sog_batch* batch, int32_t i);
int64_t sog_batch_launches(const sog_batch* batch);
void sog_batch_destroy(sog_batch* batch);

/*
 * Learned parameter proposer (the paper selects parameters analytically,
 * Sec. 4.3; that selection remains the fallback).  A multilayer perceptron
 * with two tanh hidden layers of n_hidden units and one output, in FP32 on
 * the device, with its own forward, backward and Adam kernels.  Parameters
 * form one array: W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1].
 *   sog_mlp_create: 1 <= n_in <= 16, 1 <= n_hidden <= 64; Glorot-uniform
 *     weights from `seed`, zero biases.  *mlp owned by the caller.
 *   sog_mlp_get_params / sog_mlp_set_params: host array of exactly
 *     sog_mlp_num_params values (set also resets the Adam state).
 *   sog_mlp_forward: X [n x n_in] and Y [n], device FP32.
 *   sog_mlp_loss_grad: loss = (1/n) sum_s (y_s - T_s)^2 and its gradient
 *     with respect to the parameters; X, T, grad [num_params], loss [1] are
 *     device FP32 (grad and loss are overwritten).
 *   sog_mlp_train: `iters` full-batch Adam steps (beta 0.9, 0.999, eps 1e-8,
 *     learning rate lr) on (X, T); *loss_out (host, may be NULL) receives the
 *     loss of the last step (waits for the stream then).
 * All enqueue on `stream`.
 *
 * sog_features: eight features of a system for the proposer, written to host
 * memory `feat`: log10 N, log10 sqrt(Lx Ly), log10 (Lz / sqrt(Lx Ly)),
 * log10 tol, log10 density, and of a 16-bin histogram of z (computed on the
 * device from r, N x 3 of the precision's type): max / mean, mean of the two
 * wall bins / mean, standard deviation / mean.  Synchronous.
 */
typedef struct sog_mlp sog_mlp;
sog_status sog_mlp_create(sog_mlp** mlp, int32_t n_in, int32_t n_hidden, uint64_t seed);
int64_t sog_mlp_num_params(const sog_mlp* mlp);
sog_status sog_mlp_get_params(const sog_mlp* mlp, float* params, int64_t n);
sog_status sog_mlp_set_params(sog_mlp* mlp, const float* params, int64_t n);
sog_status sog_mlp_forward(const sog_mlp* mlp, const float* X, int32_t n, float* Y, void* stream);
sog_status sog_mlp_loss_grad(const sog_mlp* mlp, const float* X, const float* T, int32_t n,
                             float* grad, float* loss, void* stream);
sog_status sog_mlp_train(sog_mlp* mlp, const float* X, const float* T, int32_t n, int32_t iters,
                         float lr, float* loss_out, void* stream);
void sog_mlp_destroy(sog_mlp* mlp);
sog_status sog_features(int64_t N, double Lx, double Ly, double Lz, double tol, const void* r,
                        int32_t precision, float* feat);

/*
 * Assembly of Phi, F and U from the four parts that sog_eval_components
 * returns, with no plan and no memory allocation.  The paper has no
 * counterpart: it is a library convenience for callers that must not allocate
 * device memory during a run, e.g. an integrator that has handed all free
 * device memory to its own pools, or a loop on several streams that cannot
 * afford the device-wide synchronisation of cudaMalloc / cudaFree.
 *   N           number of charges, 1 <= N <= 715827882 (else SOG_ERR_ARG)
 *   precision   SOG_PREC_FP64 or SOG_PREC_MIXED: element type of q, phi, F
 *   prm         host; b, sigma, omega, M give the self-term coefficient
 *               sum_l w_l (Eq. 2.22, 2.25); b > 1, sigma > 0, omega > 0
 *               finite and 0 <= M <= 4000, else SOG_ERR_ARG
 *   q           [N]          device, plan type; a non-finite charge counts
 *                            as 0 (no status is latched here: the plan whose
 *                            sog_eval_components produced the parts reports
 *                            it through sog_plan_check)
 *   phi_parts   [4 x N]      device, double, as from sog_eval_components
 *   grad_parts  [4 x N x 3]  device, double; may be NULL when F is NULL
 *   phi, E, F   outputs as in sog_eval; any may be NULL
 * Enqueued on `stream`; returns without waiting.  The energy's partial sums
 * go to a fixed device array of 1024 doubles (8 KB) inside the library, one
 * per block of the assembly (two blocks per SM, at most 1024; any N uses
 * it; nothing in it has to start at zero).  Its address is looked up on the
 * first call on each device, which should come before any stream capture is
 * begun on that device.  Calls that may run at the same time on one device
 * (different streams or host threads without ordering) share that array and
 * race on E; calls ordered on one stream do not.
 */
sog_status sog_assemble_noalloc(int64_t N, int32_t precision, const sog_params* prm,
                                const void* q, const double* phi_parts, const double* grad_parts,
                                void* phi, double* E, void* F, void* stream);

/*
 * Molecular dynamics with repeated evaluations (the use the paper's C^1
 * split of Sec. 2.2, Eq. 2.23-2.24, is built for).  A sog_md drives one plan
 * through velocity-Verlet steps of length dt:
 *   v += dt/2 F/m;  r += dt v (x, y wrapped by one period, z reflected at
 *   the walls z = +-Lz/2 with v_z reversed);  F = forces at r (sog_eval, the
 *   energy of the step to *E);  v += dt/2 F/m.
 * The plan, its workspaces and its captured evaluation are reused by every
 * step.  With sort_every > 0, after every sort_every-th step the arrays q,
 * r, v, F, inv_mass and order are permuted in place into the near-field cell
 * order of that step's evaluation, so that the next steps' binning sorts
 * nearly sorted input; order[] (initialise it to 0..N-1) then tells the
 * original index of each slot.
 *   sog_md_create: allocates N x 3 elements of scratch; *md owned by the
 *     caller, released by sog_md_destroy (before the plan).
 *   sog_md_step: nsteps steps; q [N], r [N x 3], v [N x 3], F [N x 3] device
 *     arrays of the plan's type, F holding the forces at r on entry (one
 *     sog_eval before the first call) and on return; inv_mass [N] (plan
 *     type) or NULL for unit masses; E device double or NULL; order [N]
 *     int32 device, required when sort_every > 0.  Enqueued on `stream`.
 *     Data errors (a z outside the box after a step cannot occur; charges
 *     not neutral, non-finite values) are reported by sog_plan_check.
 */
typedef struct sog_md sog_md;
sog_status sog_md_create(sog_md** md, sog_plan* plan);
sog_status sog_md_step(sog_md* md, void* q, void* r, void* v, void* F, void* inv_mass, double dt,
                       int32_t nsteps, int32_t sort_every, double* E, int32_t* order,
                       void* stream);
void sog_md_destroy(sog_md* md);

/* Release the plan and its device memory (waits for its pending work). */
void sog_plan_destroy(sog_plan* plan);

/* Static description of a status code. */
const char* sog_status_str(sog_status s);

#ifdef __cplusplus
}
#endif

#endif /* SOG_H */
