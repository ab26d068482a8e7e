/*
 * mujica_pm.h -- C ABI of the GB300 particle-mesh forward model, its adjoint,
 * the projected L-BFGS step and the projection / rank-order-matching
 * operator of MujicΛ ("Initial Condition Reconstruction on Realistic Redshift
 * Surveys with Augmented Optimization").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns a pm_status (0 = PM_OK) and never throws.  On an
 *   error, pm_last_error() returns a message for the calling host thread.
 * - Meshes and the white-noise parameter s are caller-owned DEVICE buffers,
 *   contiguous, C order [n][n][n] (x slowest, z fastest), of the plan's
 *   element type: float for PM_PREC_F32, double for PM_PREC_F64.
 * - Particle arrays are SoA [3][n^3] of the same type; particle
 *   p = (i*n + j)*n + l starts at the Lagrangian node (i, j, l) * L / n.
 * - The library allocates no device memory: each object reports the size of
 *   the device workspace it needs and the caller passes that workspace in.
 *   The host-side plan / state objects are small malloc'ed structs.
 * - Calls are asynchronous on the given cudaStream_t (pass 0 for the legacy
 *   default stream) except those that return a host scalar (loss, dot
 *   products, counts): those synchronise that stream before returning.
 * - Units: comoving Mpc/h, wavenumbers h/Mpc, H0 = 1, momentum
 *   p = a^3 E(a) dx/da.
 * - Citations are to sections and equations of the paper.
 */
#ifndef MUJICA_PM_H
#define MUJICA_PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pm_stream_t; /* a cudaStream_t */

typedef enum {
  PM_OK = 0,
  PM_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad enum value */
  PM_ERR_UNSUPPORTED = 2,   /* mesh not a power of two in [16, 512], bad option combination */
  PM_ERR_CUDA = 3,          /* a CUDA runtime call failed; message has the CUDA error string */
  PM_ERR_NONFINITE = 4,     /* NaN / Inf in an input or in the evaluated loss */
  PM_ERR_WORKSPACE = 5,     /* workspace too small or misaligned (256-byte alignment required) */
  PM_ERR_LINESEARCH = 6,    /* reserved for the reconstruction driver: line search exhausted */
  PM_ERR_DEVICE_STATUS = 7  /* a kernel reported an internal inconsistency */
} pm_status;

typedef enum { PM_PREC_F32 = 0, PM_PREC_F64 = 1 } pm_precision;
typedef enum { PM_LIK_GAUSSIAN = 0, PM_LIK_POISSON = 1 } pm_likelihood;
/* Galaxy bias model (Sec. 2.2.1 item 4), chosen apart from the likelihood.
 * AUTO: linear for PM_LIK_GAUSSIAN, power law + sigmoid for PM_LIK_POISSON
 * (the pairs Sec. 2.2.2 describes; a zero-initialised config gets them). */
typedef enum { PM_BIAS_AUTO = 0, PM_BIAS_LINEAR = 1, PM_BIAS_POWERLAW_SIGMOID = 2 } pm_bias;

/* Model configuration (Sec. 2.2.1 items 1-5, Sec. 2.2.2). */
typedef struct {
  int32_t n;                /* mesh cells per side = particles per side; power of two, 16..512 */
  int32_t n_steps;          /* leapfrog steps, uniform in a from a_init to 1 (Sec. 2.2.1 item 2); >= 1 */
  int32_t lpt_order;        /* 1 (Zel'dovich) or 2 (2LPT, the paper's choice) */
  int32_t rsd_axis;         /* redshift-space shift at a = 1 (Sec. 2.2.1 item 3): -1 none; 0, 1, 2:
                               plane parallel along x, y, z; 3: radial, along the line of sight from
                               `observer` (x_s = x + (p . d) d / (a^2 E), d the unit vector) */
  int32_t likelihood;       /* PM_LIK_GAUSSIAN: 1/2 sum R (f(delta) - d)^2 / sigma^2
                               PM_LIK_POISSON: sum over R > 0 of lambda - N log lambda, lambda = R nbar g(delta)
                               (the Poisson likelihood of Sec. 2.2.2 without log N!) */
  int32_t precision;        /* PM_PREC_F32 (FP32 mesh / FFT / particles, FP64 reductions) or PM_PREC_F64 */
  int32_t checkpoint_every; /* 0: pm_adjoint keeps every step's particle state; c > 0: keeps (x, p)
                               every c steps and recomputes the steps in between (same result) */
  int32_t lightcone;        /* 1: observe each particle on the observer's past light cone (Appendix A):
                               snapshots at a = 0.8, 0.9, 1 (the uniform step grid must hold them, e.g.
                               a_init = 0.1 with 9 or 18 steps), scale factor from three fixed-point
                               iterations of DistToScaleFactor, linear interpolation between snapshots,
                               radial shift at that scale factor; needs rsd_axis = 3.  0: off */
  int32_t bias;             /* pm_bias.  Linear: f = b delta (Gaussian), g = max(1 + b delta, rho_floor)
                               (Poisson; zero derivative below the floor).  Power law + sigmoid (Eq.
                               galaxy_bias): g = max(1 + delta, rho_floor)^alpha sigmoid(K (delta - delta_th)),
                               f = nbar g (Gaussian) */
  double box;               /* side of the periodic box, Mpc/h */
  double omega_m;           /* flat LCDM matter density (E(a) and the Poisson source) */
  double a_init;            /* scale factor of the 2LPT initial condition, 0 < a_init < 1 */
  double bias_b;            /* linear bias: b */
  double sigma;             /* Gaussian: noise standard deviation per cell */
  double alpha;             /* power-law bias: index (paper: 0.7) */
  double delta_th;          /* power-law bias: sigmoid threshold (paper: 1.2) */
  double K;                 /* power-law bias: sigmoid steepness (paper: 3.0) */
  double nbar_cell;         /* Poisson, and the Gaussian with the power-law bias: normalisation N_G of
                               Eq. galaxy_bias, galaxies per cell */
  double rho_floor;         /* Poisson, and the power-law bias: floor on 1 + delta (power law) or
                               1 + b delta (linear Poisson rate), 1e-3 */
  double prior_weight;      /* weight w of the Gaussian prior (w/2) sum s^2; 0 = likelihood only */
  double observer[3];       /* rsd_axis = 3: observer position in box coordinates, Mpc/h (may lie
                               outside the box; no particle may sit on it) */
} pm_config;

typedef struct pm_plan pm_plan;
typedef struct lbfgs_state lbfgs_state;

/* Message describing the last error on this host thread ("" if none). */
const char *pm_last_error(void);
/* Library version string. */
const char *pm_version(void);
/* Number of CUDA kernel launches this library has issued since it was loaded
 * (all plans and threads; diagnostics, no counterpart in the paper). */
int64_t pm_launch_count(void);
/* Measured fused multiply-add rate of this GPU in the given precision
 * (diagnostics: the arithmetic ceiling of the all-FP64 path, no counterpart in
 * the paper).  One launch of 8 blocks per SM x 256 threads, each running 8
 * independent FMA chains of `iters` steps (1 <= iters <= 1e6), timed with CUDA
 * events on the stream after an untimed one-step launch of the same kernel;
 * *tflops_out = 2 x FMAs / time in TFLOP/s.  scratch:
 * device buffer of >= 8 bytes, written only in a case the arithmetic never
 * reaches (it keeps the chains live).  Synchronises.  Errors:
 * PM_ERR_INVALID_ARG, PM_ERR_CUDA. */
pm_status pm_fma_rate(int32_t precision, int64_t iters, void *scratch, double *tflops_out, pm_stream_t stream);

/* ---- host-side coefficients (no GPU) ----------------------------------- */

/* Linear matter power spectrum at z = 0 (Sec. 2.2.1 item 1: P_k of the fiducial
 * cosmology): Eisenstein & Hu (1998) no-wiggle transfer function, spectral
 * index n_s, normalised to sigma8 with an 8 Mpc/h top hat.  Writes n_k
 * log-spaced points k in [k_min, k_max] (h/Mpc) as (ln k, ln P) into the host
 * arrays lnk, lnp.  Errors: PM_ERR_INVALID_ARG. */
pm_status pm_linear_power_table(double omega_m, double omega_b, double h, double sigma8,
                                double n_s, double k_min, double k_max, int32_t n_k,
                                double *lnk, double *lnp);

/* Growth factors of flat LCDM at n_a scale factors (host arrays): linear D1
 * (D1(1) = 1), second order D2 (-3/7 D1^2 in the EdS limit) and the momentum
 * growth Gp1 = a^3 E dD1/da, Gp2 = a^3 E dD2/da used by 2LPT and the FastPM
 * kick / drift factors (Sec. 2.2.1 item 2).  Any output may be NULL. */
pm_status pm_growth(double omega_m, int32_t n_a, const double *a, double *D1, double *D2,
                    double *Gp1, double *Gp2);

/* Comoving distance table of the lightcone (Appendix A, DistToScaleFactor):
 * a_j = a_min + j (1 - a_min) / (n - 1) and chi_j = (c/H0) int_{a_j}^1 da / (a^2 E(a))
 * in Mpc/h, j = 0..n-1 (host arrays of n >= 2 doubles, caller-owned).  A plan with
 * lightcone = 1 builds this table with a_min = 0.5, n = 2049.  Errors:
 * PM_ERR_INVALID_ARG (NULL output, n < 2, a_min outside (0, 1), omega_m outside (0, 1]). */
pm_status pm_distance_table(double omega_m, double a_min, int32_t n, double *a, double *chi);

/* ---- plan: the forward model and its adjoint --------------------------- */

/* Device workspace bytes a plan with this configuration needs. */
pm_status pm_workspace_bytes(const pm_config *cfg, size_t *bytes);

/* Create a plan.  lnk / lnp: host table (n_pk >= 2 points, ln k increasing) of
 * the linear power spectrum, interpolated linearly in (ln k, ln P) and clamped
 * at its ends.  workspace: caller-owned device buffer of at least
 * pm_workspace_bytes() bytes, 256-byte aligned, that must outlive the plan;
 * it is not cleared by the caller.  Synchronous (uploads tables).  Errors:
 * PM_ERR_INVALID_ARG, PM_ERR_UNSUPPORTED, PM_ERR_WORKSPACE, PM_ERR_CUDA. */
pm_status pm_plan_create(const pm_config *cfg, const double *lnk, const double *lnp, int32_t n_pk,
                         void *workspace, size_t bytes, pm_plan **out);
pm_status pm_plan_destroy(pm_plan *plan);

/* Forward model and loss (Sec. 2.2.1 items 1-5, Sec. 2.2.2, plus the prior):
 *   loss = -log L(data | delta(s)) + (w/2) sum s^2
 * s: white noise [n^3]; data: Gaussian d or Poisson counts N_G [n^3]; R: survey
 * response [n^3] (Gaussian: per-cell weight; Poisson: cells with R > 0 enter
 * the likelihood).  loss_out: host double.  delta_out (nullable): final
 * matter density contrast after the redshift-space shift, [n^3].
 * Synchronises the stream.  Errors: PM_ERR_INVALID_ARG, PM_ERR_NONFINITE (loss
 * not finite), PM_ERR_CUDA. */
pm_status pm_forward(pm_plan *plan, const void *s, const void *data, const void *R,
                     double *loss_out, void *delta_out, pm_stream_t stream);

/* Vector-Jacobian product of loss_weight * loss + <cot_delta, delta> with
 * respect to s (the gradient the L-BFGS iterations of Sec. 2.3.1 consume),
 * by the hand-derived reverse of every stage.  cot_delta (nullable): [n^3].
 * grad_out: [n^3].  loss_out (nullable): host double, the loss (unweighted).
 * Synchronises the stream.  Errors: as pm_forward. */
pm_status pm_adjoint(pm_plan *plan, const void *s, const void *data, const void *R,
                     double loss_weight, const void *cot_delta, double *loss_out,
                     void *grad_out, pm_stream_t stream);

/* Likelihood and prior parts of the last loss this plan evaluated. */
pm_status pm_last_terms(const pm_plan *plan, double *likelihood, double *prior);

/* ---- stage probes (same kernels as the forward model) ------------------ */

/* delta_L = IFFT[ sqrt(P(|k|)/Delta^3) FFT[s] ], DC = 0 (Sec. 2.2.1 item 1). */
pm_status pm_linear_field(pm_plan *plan, const void *s, void *delta_l_out, pm_stream_t stream);
/* 2LPT displacement (Mpc/h) and momentum at a_init (Sec. 2.2.1 item 2), SoA [3][n^3]. */
pm_status pm_lpt(pm_plan *plan, const void *s, void *disp_out, void *mom_out, pm_stream_t stream);
/* PM force F = -grad phi, lap phi = 1.5 Omega_m delta, read out at the particles
 * displaced by disp (Mpc/h, SoA), SoA [3][n^3] output; density_out (nullable)
 * receives delta = rho - 1 painted from disp. */
pm_status pm_force(pm_plan *plan, const void *disp, void *force_out, void *density_out,
                   pm_stream_t stream);
/* Displacement and momentum at a = 1 after 2LPT and the leapfrog steps. */
pm_status pm_evolve(pm_plan *plan, const void *s, void *disp_out, void *mom_out, pm_stream_t stream);

/* Model mean per cell at s, the rate the mock galaxies are drawn from:
 * Poisson: lambda = R nbar g(delta) (g of the bias model: Eq. galaxy_bias or
 * the floored linear rate, times the survey response of Sec. 2.2.1 item 5);
 * Gaussian: f(delta) (b delta, or nbar g(delta)).  out: [n^3]. */
pm_status pm_expected_counts(pm_plan *plan, const void *s, const void *R, void *out, pm_stream_t stream);

/* ---- annealing: low-resolution stage feeding the full-resolution start (Sec. 3, opening) ---- */

/* White noise of the plan's mesh (n per side) from a coarse one (n_coarse per
 * side, a power of two below n, same box): with r = n / n_coarse,
 * out(k) = r^{3/2} s_coarse(k) on the modes with every |n_i| < n_coarse / 2 and
 * out(k) = fresh(k) on all others, so the linear density of the coarse field
 * (delta_L = s sqrt(P / Delta^3)) is kept and out stays unit white noise when
 * fresh is.  s_coarse [n_coarse^3], fresh [n^3] (caller's N(0,1) draws), out
 * [n^3]: device arrays of the plan's precision, caller-owned; out may not alias
 * the inputs.  Uses the plan's workspace (call between, not during, forward /
 * adjoint calls on the stream).  Errors: PM_ERR_INVALID_ARG, PM_ERR_CUDA. */
pm_status pm_refine_noise(pm_plan *plan, const void *s_coarse, int32_t n_coarse, const void *fresh, void *out,
                          pm_stream_t stream);

/* ---- analysis of fields (Sec. 3.2: r_c(k); Sec. 3.3: the T-web) ---------- */

/* Binned power spectra of one or two real fields on the plan's mesh (device
 * arrays [n^3] of the plan's precision; b may be NULL): with the DFT
 * X(k) = sum_x x e^{-ikx}, P(k) = (V / n^6) sum |X|^2 over the modes of a bin
 * divided by their number (cross spectrum: Re(A conj B)), V = box^3; the mode
 * of integer wave vector m, |k| = (2 pi / box) |m|, falls in bin
 * floor((|k| - k_min) / dk), dk = (k_max - k_min) / n_bins, when that lies in
 * [0, n_bins).  Host outputs of n_bins doubles: p_aa, counts (required), p_bb,
 * p_ab (nullable; 0 when b is NULL), r_c (nullable): the cross-correlation
 * coefficient r_c = p_ab / sqrt(p_aa p_bb) of Sec. 3.2 (NaN when b is NULL);
 * empty bins give NaN.  Uses the plan's workspace; synchronises the stream.
 * Bin sums are FP64 atomics, so the last bits may differ between calls.
 * Errors: PM_ERR_INVALID_ARG (n_bins outside [1, 1024], k_max <= k_min),
 * PM_ERR_CUDA. */
pm_status pm_power_spectra(pm_plan *plan, const void *a, const void *b, int32_t n_bins, double k_min, double k_max,
                           double *p_aa, double *p_bb, double *p_ab, double *counts, double *r_c,
                           pm_stream_t stream);

/* Gaussian smoothing out = IFFT[exp(-|k|^2 r_sm^2 / 2) FFT(in)] (r_sm in Mpc/h,
 * >= 0), device arrays [n^3] of the plan's precision (in-place allowed). */
pm_status pm_smooth(pm_plan *plan, const void *in, double r_sm, void *out, pm_stream_t stream);

/* T-web classification of a density contrast field (device [n^3], plan's
 * precision): psi_ij(k) = k_i k_j / |k|^2 exp(-|k|^2 r_sm^2 / 2) delta(k) (k_i = 0 at
 * axis i's Nyquist index, psi(0) = 0), per cell eigenvalues
 * lambda_1 <= lambda_2 <= lambda_3 (FP64 closed form of the cubic) and unit
 * eigenvectors; labels[c] = number of eigenvalues above lambda_th (0 void,
 * 1 sheet, 2 filament, 3 knot; the paper: r_sm = 2 Mpc/h, lambda_th = 0.16).
 * Outputs (device, caller-owned): labels int32 [n^3] (required), eig [3][n^3]
 * and evec [3 (which) x 3 (component)][n^3] in the plan's precision (nullable).
 * Uses the plan's workspace. */
pm_status pm_tweb(pm_plan *plan, const void *delta, double r_sm, double lambda_th, int32_t *labels, void *eig,
                  void *evec, pm_stream_t stream);

/* Cosine similarity |e_i,a . e_i,b| (i = 1, 2, 3) of two eigenvector fields in
 * pm_tweb's layout; out [3][n_cells]; device arrays of the given precision. */
pm_status pm_eigvec_cosines(int64_t n_cells, int32_t precision, const void *va, const void *vb, void *out,
                            pm_stream_t stream);

/* Confusion matrix of two T-web labelings over the cells with R > 0 (all
 * cells when R is NULL; R in the given precision): counts_out (device int64
 * [16], overwritten) [4 * truth + reconstructed]; labels outside 0..3 are not
 * counted. */
pm_status pm_confusion(int64_t n_cells, int32_t precision, const int32_t *labels_truth, const int32_t *labels_rec,
                       const void *R, int64_t *counts_out, pm_stream_t stream);

/* Coarse mesh of (n / factor)^3 cells from a mesh of n^3 cells: the sum
 * (mean = 0, e.g. galaxy counts) or the mean (mean = 1, e.g. the survey
 * response R) of each factor^3 block, added in FP64.  n and factor powers of
 * two, factor <= n <= 1024; in [n^3], out [(n/factor)^3] device arrays of the
 * given precision, caller-owned.  Errors: PM_ERR_INVALID_ARG, PM_ERR_CUDA. */
pm_status pm_coarsen(int32_t n, int32_t factor, int32_t precision, int32_t mean, const void *in, void *out,
                     pm_stream_t stream);

/* ---- kernel timing (no counterpart in the paper; diagnostics) ----------
 * pm_profile(plan, 1, capacity) creates 2*capacity CUDA events and from then
 * on brackets every launch of the profiled kernel classes on its stream
 * (up to capacity launches); pm_profile(plan, 0, 0) stops recording.
 * pm_profile_read sums, over the recorded launches of one class, the elapsed
 * time, the launch count, the algorithmic bytes each launch must move (the
 * method's inputs read once and outputs written once, meshes and particle
 * arrays as FP32 / FP64 words) and (impl_bytes_total, nullable) the bytes of
 * the implementation's own arrays (64-bit fixed-point meshes, the padded
 * force mesh) and (flops_total, nullable) the floating-point
 * operations of the FFT passes (5 L log2 L per complex FFT of length L, half
 * for a real one; 0 for the other classes) (synchronises).
 * Classes: 0 fused readout+kick+drift+paint, 1 z-pass r2c, 2 column pass,
 * 3 x-pass with multipliers, 4 z-pass c2r, 5 adjoint 3-channel paint,
 * 6 adjoint gather, 7 likelihood. */
pm_status pm_profile(pm_plan *plan, int32_t enable, int32_t capacity);
pm_status pm_profile_read(pm_plan *plan, int32_t kernel_class, double *ms_total, int64_t *launches,
                          double *bytes_total, double *impl_bytes_total, double *flops_total);

/* ---- projection and rank-order matching (Sec. 2.3.1, Sec. 2.3.2) ------- */

#define PM_PROJECT 1u       /* z-score, then reset |s_hat| > 10 to counter-based N(0,1) draws */
#define PM_ROM_FOURIER 2u   /* rank-order matching of Fourier modes in 100 |k| bins, k >= 0.1 h/Mpc */
#define PM_ROM_REAL 4u      /* rank-order matching of s over the cells with R > 0 */

/* Number of values Fourier matching touches in each of the 100 bins (host
 * int64[100]); the caller draws that many sorted N(0,1) targets per bin. */
pm_status pm_rom_fourier_counts(const pm_plan *plan, int64_t *counts_out);
/* Number of cells with R > 0 (synchronises). */
pm_status pm_count_positive(pm_plan *plan, const void *R, int64_t *count_out, pm_stream_t stream);

/* Applies, in this order and each only when its bit is in mode: Fourier
 * matching, real-space matching, projection.  s_inout [n^3] in place.
 * targets_real: device [count of R > 0], sorted descending (plan type);
 * targets_fourier: device, the per-bin target lists concatenated in bin
 * order, each sorted descending (plan type).  Ranks break ties by index
 * (lower index = larger).  rng_seed / rng_counter key the reset draws.
 * n_reset_out (nullable host): number of reset values; when non-NULL the call
 * synchronises.  rank_out (nullable, device int32 [n^3], caller-owned): with
 * PM_ROM_REAL in mode, the rank pi of Sec. 2.3.2 step 1 of every cell with
 * R > 0 by its value before matching (0 = largest, ties as above; that cell
 * received targets_real[rank]), -1 for the cells with R <= 0; without
 * PM_ROM_REAL it is not written.  Errors: PM_ERR_INVALID_ARG,
 * PM_ERR_NONFINITE (NaN in s), PM_ERR_CUDA. */
pm_status project_rank_match(pm_plan *plan, void *s_inout, uint32_t mode, const void *R,
                             const void *targets_real, const void *targets_fourier,
                             uint64_t rng_seed, uint64_t rng_counter, int64_t *n_reset_out,
                             int32_t *rank_out, pm_stream_t stream);

/* Projection step only (z-score, then reset |s_hat| > 10 to the same
 * counter-based N(0,1) draws as PM_PROJECT) on n elements of the given
 * precision, in place, WITHOUT any workspace: for callers that cannot give
 * the library device memory (their GPU memory is owned by another allocator,
 * or they must not allocate mid-run).  The paper has no counterpart of this
 * entry point; it repeats the projection of project_rank_match.
 * Scratch: a file-scope device array of about 512 KB held by every GPU that
 * loads the library until exit; n must not exceed 2^28 elements
 * (PM_ERR_UNSUPPORTED otherwise).  The first call on each device looks up the
 * array's device address (with that device current); make that first call
 * before any stream capture.  All calls share the array: calls that overlap on
 * the GPU race and must be serialised.  Allocates nothing; synchronises the
 * stream.  n_reset_out (nullable host): number of reset values. */
pm_status pm_project_noalloc(int64_t n, int32_t precision, void *s_inout, uint64_t rng_seed,
                             uint64_t rng_counter, int64_t *n_reset_out, pm_stream_t stream);

/* ---- L-BFGS (Sec. 2.3.1) ------------------------------------------------ */

pm_status lbfgs_workspace_bytes(int64_t n_elems, int32_t m, int32_t precision, size_t *bytes);
pm_status lbfgs_create(int64_t n_elems, int32_t m, int32_t precision, void *workspace,
                       size_t bytes, lbfgs_state **out);
pm_status lbfgs_destroy(lbfgs_state *st);
/* Forget the stored pairs and the previous point. */
pm_status lbfgs_reset(lbfgs_state *st);
/* If a previous point exists, store the pair (x_new - x_prev, g_new - g_prev)
 * when s.y > 1e-10 |s| |y|; then d_out = -H g_new by the two-loop recursion
 * with H0 = gamma I (gamma = s.y / y.y of the newest pair, 1 without pairs);
 * if g.d >= 0 the pairs are dropped and d = -g.  Host outputs (nullable):
 * gdotd_out = g.d, dnorm_out = |d|, pushed_out = whether a pair was stored.
 * Dot products: FP64 vectors accumulate in FP64; FP32 vectors form each
 * product exactly (p + e by FMA) and sum it per thread in a compensated FP32
 * pair (Knuth's TwoSum), converted to FP64 once per thread, then every thread's
 * partial is added in FP64 in a fixed order (deterministic; within ~1e-13 of
 * sum |x y|, far below the 6e-8 rounding of the FP32 vectors).  Synchronises. */
pm_status lbfgs_step(lbfgs_state *st, const void *x_new, const void *g_new, void *d_out,
                     double *gdotd_out, double *dnorm_out, int32_t *pushed_out,
                     pm_stream_t stream);

/* out = y + alpha * x over n elements of the given precision (device). */
pm_status pm_axpy(int64_t n, int32_t precision, double alpha, const void *x, const void *y,
                  void *out, pm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MUJICA_PM_H */
