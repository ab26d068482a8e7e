// C ABI of the particle-mesh model: plan lifecycle, forward, adjoint,
// stage probes and the host-side coefficient helpers.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>
#include <string>

#include "api_internal.h"
#include "rom.cuh"

extern template struct pm::Engine<float>;
extern template struct pm::Engine<double>;
extern template struct pm::rom::Rom<float>;
extern template struct pm::rom::Rom<double>;

namespace {
thread_local std::string g_err;
}

namespace pm {
void set_error(const std::string &msg) { g_err = msg; }
}  // namespace pm

struct pm_plan {
  pm_config cfg;
  pm::Engine<float> *f32 = nullptr;
  pm::Engine<double> *f64 = nullptr;
};

pm_status pm_validate_config(const pm_config *c) {
  if (!c) {
    pm::set_error("config is NULL");
    return PM_ERR_INVALID_ARG;
  }
  const int n = c->n;
  if (n < 16 || n > 512 || (n & (n - 1))) {
    pm::set_error("n must be a power of two in [16, 512]");
    return PM_ERR_UNSUPPORTED;
  }
  if (c->n_steps < 1 || c->n_steps > 1000 || (c->lpt_order != 1 && c->lpt_order != 2) || c->rsd_axis < -1 ||
      c->rsd_axis > 3 || (c->likelihood != PM_LIK_GAUSSIAN && c->likelihood != PM_LIK_POISSON) ||
      (c->precision != PM_PREC_F32 && c->precision != PM_PREC_F64) || c->checkpoint_every < 0 ||
      (c->bias != PM_BIAS_AUTO && c->bias != PM_BIAS_LINEAR && c->bias != PM_BIAS_POWERLAW_SIGMOID)) {
    pm::set_error("invalid enum / step count / checkpoint setting");
    return PM_ERR_INVALID_ARG;
  }
  if (!(c->box > 0) || !(c->a_init > 0) || !(c->a_init < 1) || !(c->omega_m > 0) || !(c->omega_m <= 1) ||
      !std::isfinite(c->prior_weight)) {
    pm::set_error("invalid box / a_init / omega_m / prior_weight");
    return PM_ERR_INVALID_ARG;
  }
  if (c->rsd_axis == 3 &&
      !(std::isfinite(c->observer[0]) && std::isfinite(c->observer[1]) && std::isfinite(c->observer[2]))) {
    pm::set_error("radial redshift-space shift needs a finite observer position");
    return PM_ERR_INVALID_ARG;
  }
  if (c->lightcone != 0) {
    if (c->lightcone != 1 || c->rsd_axis != 3) {
      pm::set_error("lightcone must be 0 or 1, and the lightcone needs rsd_axis = 3 (radial)");
      return PM_ERR_INVALID_ARG;
    }
    int ks[2];
    if (!pm::lightcone_states(*c, ks)) {
      pm::set_error("lightcone: the uniform step grid has no state at a = 0.8 or a = 0.9");
      return PM_ERR_UNSUPPORTED;
    }
  }
  if (c->likelihood == PM_LIK_GAUSSIAN && !(c->sigma > 0)) {
    pm::set_error("Gaussian likelihood needs sigma > 0");
    return PM_ERR_INVALID_ARG;
  }
  const bool powerlaw = c->bias == PM_BIAS_POWERLAW_SIGMOID || (c->bias == PM_BIAS_AUTO && c->likelihood == PM_LIK_POISSON);
  if ((c->likelihood == PM_LIK_POISSON || powerlaw) && (!(c->nbar_cell > 0) || !(c->rho_floor > 0))) {
    pm::set_error("the Poisson likelihood and the power-law bias need nbar_cell > 0 and rho_floor > 0");
    return PM_ERR_INVALID_ARG;
  }
  return PM_OK;
}

extern "C" {

const char *pm_last_error(void) { return g_err.c_str(); }
const char *pm_version(void) { return "mujica-pm 0.1 (sm_103a)"; }
int64_t pm_launch_count(void) { return pm::g_launches.load(); }

pm_status pm_fma_rate(int32_t precision, int64_t iters, void *scratch, double *tflops_out, pm_stream_t stream) {
  if (!scratch || !tflops_out || iters < 1 || iters > 1000000 ||
      (precision != PM_PREC_F32 && precision != PM_PREC_F64)) {
    pm::set_error("invalid FMA-rate arguments");
    return PM_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  PM_CUDA_TRY(cudaGetDevice(&dev));
  PM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int grid = 8 * sms, block = 256;
  cudaEvent_t e0, e1;
  PM_CUDA_TRY(cudaEventCreate(&e0));
  PM_CUDA_TRY(cudaEventCreate(&e1));
  float ms = 0.f;
  // one untimed launch first: the first launch of a kernel in a process loads
  // its module on the host, which would otherwise open a gap between the events
  auto launch = [&](int64_t it) {
    ::pm::note_launch();
    if (precision == PM_PREC_F32)
      pm::pw::k_fma_probe<float><<<grid, block, 0, s>>>(it, (float *)scratch);
    else
      pm::pw::k_fma_probe<double><<<grid, block, 0, s>>>(it, (double *)scratch);
  };
  launch(1);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaEventRecord(e0, s);
  if (err == cudaSuccess) launch(iters);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaEventRecord(e1, s);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    pm::set_error(cudaGetErrorString(err));
    return PM_ERR_CUDA;
  }
  const double fmas = (double)grid * block * 8.0 * (double)iters;
  *tflops_out = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return PM_OK;
}

pm_status pm_linear_power_table(double omega_m, double omega_b, double h, double sigma8, double n_s,
                                double k_min, double k_max, int32_t n_k, double *lnk, double *lnp) {
  if (!lnk || !lnp || n_k < 2 || !(k_min > 0) || !(k_max > k_min) || !(omega_m > 0) || !(omega_b >= 0) ||
      !(omega_b < omega_m) || !(h > 0) || !(sigma8 > 0)) {
    pm::set_error("invalid power-table arguments");
    return PM_ERR_INVALID_ARG;
  }
  pmhost::power_table(omega_m, omega_b, h, sigma8, n_s, k_min, k_max, n_k, lnk, lnp);
  return PM_OK;
}

pm_status pm_growth(double omega_m, int32_t n_a, const double *a, double *D1, double *D2, double *Gp1,
                    double *Gp2) {
  if (!a || n_a < 1 || !(omega_m > 0) || !(omega_m <= 1)) {
    pm::set_error("invalid growth arguments");
    return PM_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_a; ++i)
    if (!(a[i] > 1e-5) || !(a[i] <= 1.0)) {
      pm::set_error("scale factors must lie in (1e-5, 1]");
      return PM_ERR_INVALID_ARG;
    }
  std::vector<pmhost::GrowthPoint> g(n_a);
  pmhost::growth(omega_m, n_a, a, g.data());
  for (int i = 0; i < n_a; ++i) {
    if (D1) D1[i] = g[i].D1;
    if (D2) D2[i] = g[i].D2;
    if (Gp1) Gp1[i] = g[i].Gp1;
    if (Gp2) Gp2[i] = g[i].Gp2;
  }
  return PM_OK;
}

pm_status pm_distance_table(double omega_m, double a_min, int32_t n, double *a, double *chi) {
  if (!a || !chi || n < 2 || !(a_min > 0) || !(a_min < 1) || !(omega_m > 0) || !(omega_m <= 1)) {
    pm::set_error("invalid distance table arguments");
    return PM_ERR_INVALID_ARG;
  }
  pmhost::distance_table(omega_m, a_min, n, a, chi);
  return PM_OK;
}

pm_status pm_workspace_bytes(const pm_config *cfg, size_t *bytes) {
  const pm_status s = pm_validate_config(cfg);
  if (s) return s;
  if (!bytes) {
    pm::set_error("bytes is NULL");
    return PM_ERR_INVALID_ARG;
  }
  *bytes = pm::make_layout(*cfg).total + pm_sort_workspace_bytes(*cfg);
  return PM_OK;
}

pm_status pm_plan_create(const pm_config *cfg, const double *lnk, const double *lnp, int32_t n_pk, void *workspace,
                         size_t bytes, pm_plan **out) {
  pm_status s = pm_validate_config(cfg);
  if (s) return s;
  if (!lnk || !lnp || n_pk < 2 || !out || !workspace) {
    pm::set_error("NULL table / workspace / out, or fewer than 2 table points");
    return PM_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_pk; ++i) {
    if (!std::isfinite(lnk[i]) || !std::isfinite(lnp[i]) || (i && !(lnk[i] > lnk[i - 1]))) {
      pm::set_error("power table must be finite with increasing ln k");
      return PM_ERR_INVALID_ARG;
    }
  }
  size_t need = 0;
  pm_workspace_bytes(cfg, &need);
  if (bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    pm::set_error("workspace too small or not 256-byte aligned: need " + std::to_string(need) + " bytes");
    return PM_ERR_WORKSPACE;
  }
  pm_plan *p = new (std::nothrow) pm_plan;
  if (!p) {
    pm::set_error("host allocation failed");
    return PM_ERR_INVALID_ARG;
  }
  p->cfg = *cfg;
  const size_t model_bytes = pm::make_layout(*cfg).total;
  void *sort_ws = static_cast<char *>(workspace) + model_bytes;
  if (cfg->precision == PM_PREC_F32) {
    p->f32 = new pm::Engine<float>();
    s = p->f32->init(*cfg, lnk, lnp, n_pk, workspace);
    p->f32->sort_ws = sort_ws;
  } else {
    p->f64 = new pm::Engine<double>();
    s = p->f64->init(*cfg, lnk, lnp, n_pk, workspace);
    p->f64->sort_ws = sort_ws;
  }
  if (s) {
    pm_plan_destroy(p);
    return s;
  }
  *out = p;
  return PM_OK;
}

pm_status pm_plan_destroy(pm_plan *plan) {
  if (!plan) return PM_OK;
  delete plan->f32;
  delete plan->f64;
  delete plan;
  return PM_OK;
}

#define PM_PLAN_CALL(plan, stream, call32, call64)                   \
  do {                                                               \
    if (!(plan)) {                                                   \
      pm::set_error("plan is NULL");                                 \
      return PM_ERR_INVALID_ARG;                                     \
    }                                                                \
    if ((plan)->f32) {                                               \
      auto &E = *(plan)->f32;                                        \
      using T = float;                                               \
      E.st = reinterpret_cast<cudaStream_t>(stream);                 \
      return call32;                                                 \
    } else {                                                         \
      auto &E = *(plan)->f64;                                        \
      using T = double;                                              \
      E.st = reinterpret_cast<cudaStream_t>(stream);                 \
      return call64;                                                 \
    }                                                                \
  } while (0)

#define PM_BOTH(expr) PM_PLAN_CALL(plan, stream, expr, expr)

pm_status pm_forward(pm_plan *plan, const void *s, const void *data, const void *R, double *loss_out,
                     void *delta_out, pm_stream_t stream) {
  if (!s || !data || !R || !loss_out) {
    pm::set_error("NULL s / data / R / loss_out");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.forward((const T *)s, (const T *)data, (const T *)R, loss_out, (T *)delta_out));
}

pm_status pm_adjoint(pm_plan *plan, const void *s, const void *data, const void *R, double loss_weight,
                     const void *cot_delta, double *loss_out, void *grad_out, pm_stream_t stream) {
  if (!s || !data || !R || !grad_out || !std::isfinite(loss_weight)) {
    pm::set_error("NULL s / data / R / grad_out, or non-finite loss_weight");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.adjoint((const T *)s, (const T *)data, (const T *)R, loss_weight, (const T *)cot_delta, loss_out,
                    (T *)grad_out));
}

pm_status pm_last_terms(const pm_plan *plan, double *likelihood, double *prior) {
  if (!plan) {
    pm::set_error("plan is NULL");
    return PM_ERR_INVALID_ARG;
  }
  const double l = plan->f32 ? plan->f32->last_lik : plan->f64->last_lik;
  const double p = plan->f32 ? plan->f32->last_prior : plan->f64->last_prior;
  if (likelihood) *likelihood = l;
  if (prior) *prior = p;
  return PM_OK;
}

pm_status pm_linear_field(pm_plan *plan, const void *s, void *out, pm_stream_t stream) {
  if (!s || !out) {
    pm::set_error("NULL s / out");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.linear_field((const T *)s, (T *)out));
}

pm_status pm_lpt(pm_plan *plan, const void *s, void *disp_out, void *mom_out, pm_stream_t stream) {
  if (!s || !disp_out || !mom_out) {
    pm::set_error("NULL s / disp_out / mom_out");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.probe_lpt((const T *)s, (T *)disp_out, (T *)mom_out));
}

pm_status pm_force(pm_plan *plan, const void *disp, void *force_out, void *density_out, pm_stream_t stream) {
  if (!disp || !force_out) {
    pm::set_error("NULL disp / force_out");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.probe_force((const T *)disp, (T *)force_out, (T *)density_out));
}

pm_status pm_evolve(pm_plan *plan, const void *s, void *disp_out, void *mom_out, pm_stream_t stream) {
  if (!s || !disp_out || !mom_out) {
    pm::set_error("NULL s / disp_out / mom_out");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.probe_evolve((const T *)s, (T *)disp_out, (T *)mom_out));
}

pm_status pm_expected_counts(pm_plan *plan, const void *s, const void *R, void *out, pm_stream_t stream) {
  if (!s || !R || !out) {
    pm::set_error("NULL s / R / out");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.expected_counts((const T *)s, (const T *)R, (T *)out));
}

pm_status pm_refine_noise(pm_plan *plan, const void *s_coarse, int32_t n_coarse, const void *fresh, void *out,
                          pm_stream_t stream) {
  if (!plan || !s_coarse || !fresh || !out) {
    pm::set_error("NULL plan / s_coarse / fresh / out");
    return PM_ERR_INVALID_ARG;
  }
  const int n = plan->f32 ? plan->f32->n : plan->f64->n;
  if (n_coarse < 2 || n_coarse >= n || (n_coarse & (n_coarse - 1))) {
    pm::set_error("n_coarse must be a power of two in [2, n)");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.refine_noise((const T *)s_coarse, n_coarse, (const T *)fresh, (T *)out));
}

pm_status pm_coarsen(int32_t n, int32_t factor, int32_t precision, int32_t mean, const void *in, void *out,
                     pm_stream_t stream) {
  if (!in || !out || n < 2 || n > 1024 || (n & (n - 1)) || factor < 2 || factor > n || (factor & (factor - 1)) ||
      (precision != PM_PREC_F32 && precision != PM_PREC_F64) || (mean != 0 && mean != 1)) {
    pm::set_error("invalid coarsen arguments");
    return PM_ERR_INVALID_ARG;
  }
  int logn = 0, logr = 0;
  while ((1 << logn) < n) ++logn;
  while ((1 << logr) < factor) ++logr;
  const int logc = logn - logr;
  const int64_t mc = (int64_t)1 << (3 * logc);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ::pm::note_launch();
  if (precision == PM_PREC_F32)
    pm::pw::k_block_reduce<float><<<pm::grid_for(mc, 256), 256, 0, s>>>((const float *)in, logc, logr, mean != 0,
                                                                       (float *)out);
  else
    pm::pw::k_block_reduce<double><<<pm::grid_for(mc, 256), 256, 0, s>>>((const double *)in, logc, logr,
                                                                        mean != 0, (double *)out);
  PM_LAUNCH_CHECK();
  return PM_OK;
}

pm_status pm_power_spectra(pm_plan *plan, const void *a, const void *b, int32_t n_bins, double k_min, double k_max,
                           double *p_aa, double *p_bb, double *p_ab, double *counts, double *r_c,
                           pm_stream_t stream) {
  if (!plan || !a || !p_aa || !counts || n_bins < 1 || n_bins > 1024 || !std::isfinite(k_min) ||
      !std::isfinite(k_max) || !(k_max > k_min)) {
    pm::set_error("invalid power spectrum arguments (n_bins in [1, 1024], k_max > k_min, outputs)");
    return PM_ERR_INVALID_ARG;
  }
  std::vector<double> h(4 * (size_t)n_bins);
  pm_status s;
  if (plan->f32) {
    auto &E = *plan->f32;
    E.st = reinterpret_cast<cudaStream_t>(stream);
    s = E.power_spectra((const float *)a, (const float *)b, n_bins, k_min, k_max, h.data());
  } else {
    auto &E = *plan->f64;
    E.st = reinterpret_cast<cudaStream_t>(stream);
    s = E.power_spectra((const double *)a, (const double *)b, n_bins, k_min, k_max, h.data());
  }
  if (s != PM_OK) return s;
  for (int j = 0; j < n_bins; ++j) {
    p_aa[j] = h[j];
    if (p_bb) p_bb[j] = h[n_bins + j];
    if (p_ab) p_ab[j] = h[2 * n_bins + j];
    counts[j] = h[3 * n_bins + j];
    // cross-correlation coefficient r_c = P_ab / sqrt(P_aa P_bb) (Sec. 3.2)
    if (r_c) r_c[j] = b ? h[2 * n_bins + j] / std::sqrt(h[j] * h[n_bins + j]) : NAN;
  }
  return PM_OK;
}

pm_status pm_smooth(pm_plan *plan, const void *in, double r_sm, void *out, pm_stream_t stream) {
  if (!plan || !in || !out || !(r_sm >= 0) || !std::isfinite(r_sm)) {
    pm::set_error("NULL in / out or invalid smoothing radius");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.smooth((const T *)in, r_sm, (T *)out));
}

pm_status pm_tweb(pm_plan *plan, const void *delta, double r_sm, double lambda_th, int32_t *labels, void *eig,
                  void *evec, pm_stream_t stream) {
  if (!plan || !delta || !labels || !(r_sm >= 0) || !std::isfinite(r_sm) || !std::isfinite(lambda_th)) {
    pm::set_error("NULL delta / labels or invalid smoothing radius / threshold");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH(E.tweb((const T *)delta, r_sm, lambda_th, (int *)labels, (T *)eig, (T *)evec));
}

pm_status pm_eigvec_cosines(int64_t n_cells, int32_t precision, const void *va, const void *vb, void *out,
                            pm_stream_t stream) {
  if (n_cells < 0 || !va || !vb || !out || (precision != PM_PREC_F32 && precision != PM_PREC_F64)) {
    pm::set_error("invalid eigenvector cosine arguments");
    return PM_ERR_INVALID_ARG;
  }
  if (n_cells == 0) return PM_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ::pm::note_launch();
  if (precision == PM_PREC_F32)
    pm::an::k_eig_cosines<float><<<pm::grid_for(n_cells, 256), 256, 0, s>>>((const float *)va, (const float *)vb,
                                                                            n_cells, (float *)out);
  else
    pm::an::k_eig_cosines<double><<<pm::grid_for(n_cells, 256), 256, 0, s>>>(
        (const double *)va, (const double *)vb, n_cells, (double *)out);
  PM_LAUNCH_CHECK();
  return PM_OK;
}

pm_status pm_confusion(int64_t n_cells, int32_t precision, const int32_t *labels_truth, const int32_t *labels_rec,
                       const void *R, int64_t *counts_out, pm_stream_t stream) {
  if (n_cells < 0 || !labels_truth || !labels_rec || !counts_out ||
      (precision != PM_PREC_F32 && precision != PM_PREC_F64)) {
    pm::set_error("invalid confusion arguments");
    return PM_ERR_INVALID_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  PM_CUDA_TRY(cudaMemsetAsync(counts_out, 0, 16 * sizeof(int64_t), s));
  if (n_cells == 0) return PM_OK;
  const int grid = (int)std::min<int64_t>(pm::grid_for(n_cells, 256), 152 * 8);
  auto *o = reinterpret_cast<unsigned long long *>(counts_out);
  ::pm::note_launch();
  if (precision == PM_PREC_F32)
    pm::an::k_confusion<float><<<grid, 256, 0, s>>>(labels_truth, labels_rec, (const float *)R, n_cells, o);
  else
    pm::an::k_confusion<double><<<grid, 256, 0, s>>>(labels_truth, labels_rec, (const double *)R, n_cells, o);
  PM_LAUNCH_CHECK();
  return PM_OK;
}

pm_status pm_profile(pm_plan *plan, int32_t enable, int32_t capacity) {
  if (!plan || (enable && capacity < 1)) {
    pm::set_error("invalid profiler arguments");
    return PM_ERR_INVALID_ARG;
  }
  pm::Profiler &p = plan->f32 ? plan->f32->prof : plan->f64->prof;
  if (!enable) {
    p.on = false;
    return PM_OK;
  }
  const cudaError_t e = p.enable(capacity);
  if (e != cudaSuccess) {
    pm::set_error(cudaGetErrorString(e));
    return PM_ERR_CUDA;
  }
  return PM_OK;
}

pm_status pm_profile_read(pm_plan *plan, int32_t kernel_class, double *ms_total, int64_t *launches,
                          double *bytes_total, double *impl_bytes_total, double *flops_total) {
  if (!plan || kernel_class < 0 || kernel_class >= pm::P_NCLASS || !ms_total || !launches || !bytes_total) {
    pm::set_error("invalid profiler read arguments");
    return PM_ERR_INVALID_ARG;
  }
  pm::Profiler &p = plan->f32 ? plan->f32->prof : plan->f64->prof;
  const cudaError_t e = p.read(kernel_class, ms_total, launches, bytes_total, impl_bytes_total, flops_total);
  if (e != cudaSuccess) {
    pm::set_error(cudaGetErrorString(e));
    return PM_ERR_CUDA;
  }
  return PM_OK;
}

pm_status pm_rom_fourier_counts(const pm_plan *plan, int64_t *counts_out) {
  if (!plan || !counts_out) {
    pm::set_error("NULL plan / counts_out");
    return PM_ERR_INVALID_ARG;
  }
  const std::vector<int64_t> &c = plan->f32 ? pm::rom::Rom<float>{*plan->f32}.counts()
                                            : pm::rom::Rom<double>{*plan->f64}.counts();
  for (int b = 0; b < 100; ++b) counts_out[b] = c[b];
  return PM_OK;
}

pm_status pm_count_positive(pm_plan *plan, const void *R, int64_t *count_out, pm_stream_t stream) {
  if (!R || !count_out) {
    pm::set_error("NULL R / count_out");
    return PM_ERR_INVALID_ARG;
  }
  PM_BOTH((pm::rom::Rom<T>{E}.count_positive((const T *)R, count_out)));
}

pm_status project_rank_match(pm_plan *plan, void *s_inout, uint32_t mode, const void *R, const void *targets_real,
                             const void *targets_fourier, uint64_t rng_seed, uint64_t rng_counter,
                             int64_t *n_reset_out, int32_t *rank_out, pm_stream_t stream) {
  if (!s_inout || (mode & ~7u) || ((mode & PM_ROM_REAL) && (!R || !targets_real)) ||
      ((mode & PM_ROM_FOURIER) && !targets_fourier)) {
    pm::set_error("invalid project_rank_match arguments");
    return PM_ERR_INVALID_ARG;
  }
  if (n_reset_out) *n_reset_out = 0;
  PM_BOTH(([&]() -> pm_status {
    pm::rom::Rom<T> r{E};
    pm_status st = PM_OK;
    if (mode & PM_ROM_FOURIER) st = r.fourier((T *)s_inout, (const T *)targets_fourier);
    if (!st && (mode & PM_ROM_REAL))
      st = r.real((T *)s_inout, (const T *)R, (const T *)targets_real, reinterpret_cast<int *>(rank_out));
    if (!st && (mode & PM_PROJECT)) st = r.project((T *)s_inout, rng_seed, rng_counter, n_reset_out);
    if (!st && !(mode & PM_PROJECT)) {
      const cudaError_t e = cudaStreamSynchronize(E.st);
      if (e != cudaSuccess) {
        pm::set_error(cudaGetErrorString(e));
        st = PM_ERR_CUDA;
      }
    }
    return st;
  }()));
}

}  // extern "C"

