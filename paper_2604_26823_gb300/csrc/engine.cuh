// Host orchestration of the particle-mesh forward model and its adjoint on
// one GPU: workspace layout, FFT pass launches, the leapfrog loop, the
// likelihood, the reverse sweep and the 2LPT / IC adjoints.
//
// Stage order follows the paper's forward model (Sec. 2.2.1 items 1-5 and
// Sec. 2.2.2); the reverse sweep applies the transpose of each stage in the
// opposite order (spectral transposes = conjugate multipliers, CIC transpose
// = weight-derivative gathers, reverse kick / drift).
#pragma once
#include <cstring>
#include <vector>

#include "../../include/mujica_pm.h"
#include "analysis.cuh"
#include "common.cuh"
#include "fft.cuh"
#include "host_cosmo.h"
#include "particles.cuh"
#include "pointwise.cuh"

namespace pm {

template <typename T> struct FftCfg {
  static constexpr int B = sizeof(T) == 4 ? 16 : 8;
};
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
// z-pass tiles.  SMALL (used by the c2r pass): FP32 meshes up to 256^3 take
// tiles of 8 rows on 128 threads (up to six CTAs per SM; measured 5% faster
// for the 3-input c2r at 256^3).  Otherwise, and for the r2c pass (whose
// fixed-point loader measured faster on the wide tile), FftCfg rows on 256
// (512 at N = 512) threads.
template <typename T, int N, bool SMALL = false> struct ZCfg {
  static constexpr bool kSmall = SMALL && sizeof(T) == 4 && N <= 256;
  static constexpr int B = kSmall ? 8 : FftCfg<T>::B;
  static constexpr int LEN = N / 2;
  static constexpr int NT = kSmall ? cmin(128, B * LEN) : cmin(N == 512 ? 512 : 256, B * LEN);
  static constexpr size_t SMEM = (size_t)LEN * (B + 1) * sizeof(cx<T>);
  // CTAs per SM the c2r pass with NIN inputs can hold by shared memory (up
  // to 6); its register budget is capped to match, so registers do not set a
  // lower occupancy than shared memory does.  The FP64 and N = 512 variants
  // keep the full budget (they would spill).
  template <int NIN> static constexpr int minb() {
    return kSmall ? cmax(1, cmin(6, (int)((227u * 1024u) / (NIN * SMEM)))) : 1;
  }
};
template <typename T, int N> struct CCfg {
  static constexpr int B = FftCfg<T>::B;
  static constexpr int NT = cmin(N == 512 ? 512 : 256, B * N);
  static constexpr size_t SMEM = (size_t)N * B * sizeof(cx<T>);
  static constexpr size_t SMEM2 = 2 * SMEM;  // fused x pass: two tiles
  // FP32, 256-thread tiles: CTAs per SM of the fused x pass by shared
  // memory (up to 3), as a floor for the register budget
  static constexpr int MINB_X = (sizeof(T) == 4 && NT <= 256) ? cmax(1, cmin(3, (int)((227u * 1024u) / SMEM2))) : 1;
};

#define PM_DISPATCH_N(nval, ...)             \
  switch (nval) {                            \
    case 16: { constexpr int NN = 16; __VA_ARGS__; } break;   \
    case 32: { constexpr int NN = 32; __VA_ARGS__; } break;   \
    case 64: { constexpr int NN = 64; __VA_ARGS__; } break;   \
    case 128: { constexpr int NN = 128; __VA_ARGS__; } break; \
    case 256: { constexpr int NN = 256; __VA_ARGS__; } break; \
    case 512: { constexpr int NN = 512; __VA_ARGS__; } break; \
    default: break;                          \
  }

template <class K> inline void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---- output functors of the c2r z pass ----------------------------------
template <typename T> struct OutPlanar {
  static constexpr double kWriteBytes = sizeof(T), kAlgWriteBytes = sizeof(T);
  T *out;
  int n;
  T scale = T(1);
  __device__ __forceinline__ void put(int64_t row, int m, const cx<T> *v) const {
    reinterpret_cast<cx<T> *>(out + row * n)[m] = mkc<cx<T>>(scale * v[0].x, scale * v[0].y);
  }
};
template <typename T> struct OutForce {
  static constexpr double kWriteBytes = 4 * sizeof(T), kAlgWriteBytes = 3 * sizeof(T);
  V4<T> *phi;
  int n;
  __device__ __forceinline__ void put(int64_t row, int m, const cx<T> *v) const {
    V4<T> *p = phi + row * n + 2 * m;
    p[0] = V4<T>{v[0].x, v[1].x, v[2].x, T(0)};
    p[1] = V4<T>{v[0].y, v[1].y, v[2].y, T(0)};
  }
};
template <typename T> struct OutLptSource {  // phi_ij (slots 00,11,22,01,02,12) -> S, phi stored
  static constexpr double kWriteBytes = 7 * sizeof(T), kAlgWriteBytes = 7 * sizeof(T);
  T *phi6;
  T *src;
  int64_t mcells;
  int n;
  __device__ __forceinline__ void put(int64_t row, int m, const cx<T> *v) const {
    const int64_t i = row * n + 2 * m;
    const T a[2][6] = {{v[0].x, v[1].x, v[2].x, v[3].x, v[4].x, v[5].x},
                       {v[0].y, v[1].y, v[2].y, v[3].y, v[4].y, v[5].y}};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const T *f = a[h];
      src[i + h] = f[0] * f[1] + f[0] * f[2] + f[1] * f[2] - f[3] * f[3] - f[4] * f[4] - f[5] * f[5];
      if (phi6) {
#pragma unroll
        for (int c = 0; c < 6; ++c) phi6[c * mcells + i + h] = f[c];
      }
    }
  }
};
template <typename T> struct OutGrad {  // out = v + w * s
  static constexpr double kWriteBytes = 2 * sizeof(T), kAlgWriteBytes = 2 * sizeof(T);
  T *out;
  const T *s;
  T w;
  int n;
  __device__ __forceinline__ void put(int64_t row, int m, const cx<T> *v) const {
    const int64_t i = row * n + 2 * m;
    const cx<T> sv = reinterpret_cast<const cx<T> *>(s)[i / 2];
    reinterpret_cast<cx<T> *>(out)[i / 2] = mkc<cx<T>>(v[0].x + w * sv.x, v[0].y + w * sv.y);
  }
};

static __global__ void k_set_int(int *p, int v) { *p = v; }

// ---- workspace layout -----------------------------------------------------
// Leapfrog states holding the lightcone snapshots at a = 0.8 and 0.9 (the
// one at a = 1 is the final state n_steps); false when the uniform grid
// a_k = a_init + k (1 - a_init) / n_steps has no state there after the
// initial one (a_init < 0.8 is required).
constexpr int kLcTable = 2049;  // distance table points, a uniform on [0.5, 1]
inline bool lightcone_states(const pm_config &c, int (&ks)[2]) {
  const double h = (1.0 - c.a_init) / c.n_steps;
  const double sa[2] = {0.8, 0.9};
  for (int j = 0; j < 2; ++j) {
    const double kf = std::nearbyint((sa[j] - c.a_init) / h);
    if (!(kf >= 1.0 && kf < c.n_steps)) return false;
    ks[j] = (int)kf;
    if (std::fabs(c.a_init + h * ks[j] - sa[j]) > 1e-9) return false;
  }
  return true;
}

struct Layout {
  size_t tw, amp, spec, fx, psi, psi2, src, dbar, mom, xbar, pbar, disp, phi, ckd, ckm, dwork, snap, lct, scal,
      total;
  int nck, seglen;
};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

inline Layout make_layout(const pm_config &c) {
  const size_t es = c.precision == PM_PREC_F64 ? 8 : 4;
  const size_t n = (size_t)c.n, m = n * n * n, h = n / 2 + 1, sp = n * n * h;
  const int steps = c.n_steps;
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L.tw = take(n * 2 * es);
  L.amp = take(sp * es);
  L.spec = take(9 * sp * 2 * es);
  L.fx = take(3 * m * 8);
  L.psi = take(9 * m * es);  // psi1 (3) followed by phi_ij (6)
  L.psi2 = take(3 * m * es);
  L.src = take(m * es);
  L.dbar = take(m * es);
  L.mom = take(3 * m * es);
  L.xbar = take(3 * m * es);
  L.pbar = take(3 * m * es);
  if (c.checkpoint_every <= 0) {
    L.nck = 0;
    L.seglen = steps + 1;
    L.disp = take((size_t)(steps + 1) * 3 * m * es);
    L.phi = take((size_t)(steps + 1) * m * 4 * es);
    L.ckd = L.ckm = L.dwork = 0;
  } else {
    const int ce = c.checkpoint_every;
    L.nck = steps / ce + 1;
    L.seglen = ce;
    L.disp = take((size_t)ce * 3 * m * es);       // segment states
    L.phi = take((size_t)ce * m * 4 * es);        // segment force meshes
    L.ckd = take((size_t)L.nck * 3 * m * es);
    L.ckm = take((size_t)L.nck * 3 * m * es);
    L.dwork = take(3 * m * es);
  }
  L.snap = L.lct = 0;
  if (c.lightcone) {
    L.snap = take(12 * m * es);             // X_0, X_1, P_0, P_1 (then their cotangents)
    L.lct = take(3 * kLcTable * es);        // a_j, chi_j, slope_j
  }
  L.scal = take(64 * 1024);
  L.total = off;
  return L;
}

// ---- the engine -------------------------------------------------------------
template <typename T> struct Engine {
  using C = cx<T>;
  pm_config cfg{};
  Layout lay{};
  int n = 0, logn = 0, H = 0;
  int64_t M = 0, S = 0;
  double cell = 0, kf = 0;
  std::vector<double> ck, dr;  // merged kick factors c_0..c_n and drifts
  std::vector<double> kbv;     // kbv[k] = Kb_{k-1}: second half-kick of the step into state k
  bool lc_on = false, lc_write = true;
  int lc_k[2] = {-1, -1};      // states of the snapshots at a = 0.8, 0.9
  T *snap = nullptr, *lct = nullptr;
  double d1 = 0, d2 = 0, gp1 = 0, gp2 = 0, rsd = 0;
  int rho_exp = 0;
  std::vector<int64_t> rom_counts;
  double last_lik = 0, last_prior = 0;
  cudaStream_t st = 0;

  char *base = nullptr;
  C *tw = nullptr, *spec = nullptr;
  T *amp = nullptr, *psi = nullptr, *phi6 = nullptr, *psi2 = nullptr, *src = nullptr, *dbar = nullptr;
  T *mom = nullptr, *xbar = nullptr, *pbar = nullptr, *disp = nullptr, *ckd = nullptr, *ckm = nullptr,
    *dwork = nullptr;
  long long *fx = nullptr;
  V4<T> *phi = nullptr;
  double *partial = nullptr, *results = nullptr;
  int *fx_exp = nullptr;
  unsigned long long *maxslot = nullptr;
  unsigned long long *maxslots = nullptr;  // part::kMaxSlots partial maxima (zero between uses)
  void *sort_ws = nullptr;
  Profiler prof;

  T obs_cell(int a) const { return (T)(cfg.observer[a] / cell); }  // observer in cell units
  part::LightCone<T> lightcone() const {
    part::LightCone<T> l{};
    l.snap = snap;
    l.ta = lct;
    l.tchi = lct + kLcTable;
    l.tsl = lct + 2 * kLcTable;
    l.ntab = kLcTable;
    l.om = (T)cfg.omega_m;
    l.cell = (T)cell;
    for (int a = 0; a < 3; ++a) l.o[a] = obs_cell(a);
    return l;
  }
  part::Geo geo() const {
    part::Geo g;
    g.L.logn = logn;
    g.L.mask = n - 1;
    g.np = M;
    g.log2np = 3 * logn;
    return g;
  }
  C *slot(int i) const { return spec + (int64_t)i * S; }
  bool keep_all() const { return cfg.checkpoint_every <= 0; }

  // ---- setup ----
  pm_status init(const pm_config &c, const double *lnk, const double *lnp, int npk, void *ws) {
    cfg = c;
    lay = make_layout(c);
    n = c.n;
    logn = 0;
    while ((1 << logn) < n) ++logn;
    H = n / 2 + 1;
    M = (int64_t)n * n * n;
    S = (int64_t)n * n * H;
    cell = c.box / n;
    kf = 2.0 * M_PI / c.box;
    base = reinterpret_cast<char *>(ws);
    tw = reinterpret_cast<C *>(base + lay.tw);
    amp = reinterpret_cast<T *>(base + lay.amp);
    spec = reinterpret_cast<C *>(base + lay.spec);
    fx = reinterpret_cast<long long *>(base + lay.fx);
    psi = reinterpret_cast<T *>(base + lay.psi);
    phi6 = psi + 3 * M;
    psi2 = reinterpret_cast<T *>(base + lay.psi2);
    src = reinterpret_cast<T *>(base + lay.src);
    dbar = reinterpret_cast<T *>(base + lay.dbar);
    mom = reinterpret_cast<T *>(base + lay.mom);
    xbar = reinterpret_cast<T *>(base + lay.xbar);
    pbar = reinterpret_cast<T *>(base + lay.pbar);
    disp = reinterpret_cast<T *>(base + lay.disp);
    phi = reinterpret_cast<V4<T> *>(base + lay.phi);
    if (!keep_all()) {
      ckd = reinterpret_cast<T *>(base + lay.ckd);
      ckm = reinterpret_cast<T *>(base + lay.ckm);
      dwork = reinterpret_cast<T *>(base + lay.dwork);
    }
    lc_on = c.lightcone != 0;
    if (lc_on) {
      snap = reinterpret_cast<T *>(base + lay.snap);
      lct = reinterpret_cast<T *>(base + lay.lct);
      if (!lightcone_states(c, lc_k)) {
        set_error("lightcone: the uniform step grid has no state at a = 0.8 or a = 0.9");
        return PM_ERR_UNSUPPORTED;
      }
    }
    char *sc = base + lay.scal;
    partial = reinterpret_cast<double *>(sc);
    results = partial + pw::kRedBlocks;
    fx_exp = reinterpret_cast<int *>(results + 16);
    maxslot = reinterpret_cast<unsigned long long *>(fx_exp + 8);
    maxslots = maxslot + 8;

    // coefficients (host FP64)
    const pmhost::Schedule sch = pmhost::leapfrog(c.omega_m, c.a_init, c.n_steps);
    const int ns = c.n_steps;
    ck.assign(ns + 1, 0.0);
    dr.assign(ns, 0.0);
    for (int k = 0; k <= ns; ++k) {
      double v = 0.0;
      if (k < ns) v += sch.Ka[k];
      if (k > 0) v += sch.Kb[k - 1];
      ck[k] = v;
    }
    for (int k = 0; k < ns; ++k) dr[k] = sch.Dr[k];
    kbv.assign(ns + 1, 0.0);
    for (int k = 1; k <= ns; ++k) kbv[k] = sch.Kb[k - 1];
    d1 = sch.lpt.D1;
    d2 = c.lpt_order == 2 ? sch.lpt.D2 : 0.0;
    gp1 = sch.lpt.Gp1;
    gp2 = c.lpt_order == 2 ? sch.lpt.Gp2 : 0.0;
    rsd = 1.0 / (1.0 * 1.0 * sch.e_final);
    rho_exp = 61 - 3 * logn - 1;  // unit weights: max sum n^3 < 2^(3 logn + 1)

    // twiddles e^{-2 pi i m / n}
    std::vector<C> h_tw(n);
    for (int m = 0; m < n; ++m) {
      const double ang = -2.0 * M_PI * m / n;
      h_tw[m] = mkc<C>((T)std::cos(ang), (T)std::sin(ang));
    }
    PM_CUDA_TRY(cudaMemcpy(tw, h_tw.data(), n * sizeof(C), cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemset(maxslots, 0, part::kMaxSlots * sizeof(unsigned long long)));
    if (lc_on) {
      // distance table (host FP64), with the slope of each interval taken in FP64
      std::vector<double> ta(kLcTable), tc(kLcTable);
      pmhost::distance_table(c.omega_m, 0.5, kLcTable, ta.data(), tc.data());
      std::vector<T> h(3 * kLcTable, T(0));
      for (int j = 0; j < kLcTable; ++j) {
        h[j] = (T)ta[j];
        h[kLcTable + j] = (T)tc[j];
        if (j + 1 < kLcTable) h[2 * kLcTable + j] = (T)((ta[j] - ta[j + 1]) / (tc[j] - tc[j + 1]));
      }
      PM_CUDA_TRY(cudaMemcpy(lct, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    // IC amplitude (table staged in the spectrum buffer)
    if ((size_t)npk * 16 > (size_t)S * sizeof(C)) {
      set_error("power table too large for this mesh");
      return PM_ERR_INVALID_ARG;
    }
    double *dtab = reinterpret_cast<double *>(spec);
    PM_CUDA_TRY(cudaMemcpy(dtab, lnk, npk * sizeof(double), cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(dtab + npk, lnp, npk * sizeof(double), cudaMemcpyHostToDevice));
    ::pm::note_launch();
    pw::k_amplitude<T><<<grid_for(S, 256), 256>>>(amp, n, kf, 1.0 / (cell * cell * cell), dtab, dtab + npk, npk);
    PM_LAUNCH_CHECK();
    PM_CUDA_TRY(cudaDeviceSynchronize());
    return PM_OK;
  }

  // ---- FFT passes ----
  pm_status r2c_real(const T *in, int nb, C *out) {
    ProfScope ps(prof, P_Z_R2C, st, (double)nb * (M * sizeof(T) + S * sizeof(C)), -1.0,
                 0.5 * fft_flops((double)nb * n * n, n));
    PM_DISPATCH_N(n, {
      using Z = ZCfg<T, NN>;
      auto kern = fft::k_z_r2c<T, NN, Z::B, Z::NT, fft::LoadReal<T>>;
      set_smem(kern, Z::SMEM);
      ::pm::note_launch();
      kern<<<(int)((int64_t)nb * n * n / Z::B), Z::NT, Z::SMEM, st>>>(fft::LoadReal<T>{in}, out, tw);
    });
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  pm_status r2c_fixed(const long long *in, const int *e, int nb, C *out, bool sub_unit = false) {
    // the method reads an FP32 / FP64 mesh; the implementation its 64-bit fixed-point paint
    ProfScope ps(prof, P_Z_R2C, st, (double)nb * (M * sizeof(T) + S * sizeof(C)), (double)nb * (M * 8.0 + S * sizeof(C)),
                 0.5 * fft_flops((double)nb * n * n, n));
    PM_DISPATCH_N(n, {
      using Z = ZCfg<T, NN>;
      auto kern = fft::k_z_r2c<T, NN, Z::B, Z::NT, fft::LoadFixed<T>>;
      set_smem(kern, Z::SMEM);
      ::pm::note_launch();
      kern<<<(int)((int64_t)nb * n * n / Z::B), Z::NT, Z::SMEM, st>>>(fft::LoadFixed<T>{in, e, sub_unit}, out, tw);
    });
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  pm_status ypass(C *buf, int nslots, int sign) {
    ProfScope ps(prof, P_COL, st, 2.0 * nslots * S * sizeof(C), -1.0, fft_flops((double)nslots * n * H, n));
    PM_DISPATCH_N(n, {
      using CC = CCfg<T, NN>;
      const int tiles = (H + CC::B - 1) / CC::B;
      const int grid = nslots * n * tiles;
      if (sign < 0) {
        auto kern = fft::k_col<T, NN, CC::B, CC::NT, -1>;
        set_smem(kern, CC::SMEM);
        ::pm::note_launch();
        kern<<<grid, CC::NT, CC::SMEM, st>>>(buf, buf, H, (int64_t)n * H, H, tiles, tw);
      } else {
        auto kern = fft::k_col<T, NN, CC::B, CC::NT, +1>;
        set_smem(kern, CC::SMEM);
        ::pm::note_launch();
        kern<<<grid, CC::NT, CC::SMEM, st>>>(buf, buf, H, (int64_t)n * H, H, tiles, tw);
      }
    });
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  pm_status x1toM(const C *in, const int *out_slots, const fft::MultDesc *m, int count) {
    fft::XArgs1 a{};
    a.in = in;
    for (int i = 0; i < count; ++i) a.out[i] = slot(out_slots[i]);
    a.plan = fft::make_xplan(m, count);
    a.amp = amp;
    a.kf = kf;
    ProfScope ps(prof, P_X_FUSED, st, (double)(1 + count) * S * sizeof(C), -1.0,
                 fft_flops((double)(1 + a.plan.nparts) * n * H, n));
    PM_DISPATCH_N(n, {
      using CC = CCfg<T, NN>;
      auto kern = fft::k_x_1toM<T, NN, CC::B, CC::NT, CC::MINB_X>;
      set_smem(kern, CC::SMEM2);
      ::pm::note_launch();
      kern<<<(int)(S / n / CC::B), CC::NT, CC::SMEM2, st>>>(a, tw);
    });
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  pm_status xMto1(const int *in_slots, int out_slot, const fft::MultDesc *m, int count) {
    fft::XArgsN a{};
    for (int i = 0; i < count; ++i) a.in[i] = slot(in_slots[i]);
    a.plan = fft::make_xplan(m, count);
    a.out = slot(out_slot);
    a.amp = amp;
    a.kf = kf;
    ProfScope ps(prof, P_X_FUSED, st, (double)(1 + count) * S * sizeof(C), -1.0,
                 fft_flops((double)(1 + a.plan.nparts) * n * H, n));
    PM_DISPATCH_N(n, {
      using CC = CCfg<T, NN>;
      auto kern = fft::k_x_Mto1<T, NN, CC::B, CC::NT, CC::MINB_X>;
      set_smem(kern, CC::SMEM2);
      ::pm::note_launch();
      kern<<<(int)(S / n / CC::B), CC::NT, CC::SMEM2, st>>>(a, tw);
    });
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  template <int NIN, class Out> pm_status c2r(int first_slot, int nb, Out out) {
    fft::Ins ins{};
    for (int i = 0; i < NIN; ++i) ins.p[i] = slot(first_slot + i);
    ProfScope ps(prof, P_Z_C2R, st, (double)nb * NIN * S * sizeof(C) + (double)nb * M * Out::kAlgWriteBytes,
                 (double)nb * NIN * S * sizeof(C) + (double)nb * M * Out::kWriteBytes,
                 0.5 * fft_flops((double)nb * NIN * n * n, n));
    PM_DISPATCH_N(n, {
      using Z = ZCfg<T, NN, true>;
      auto kern = fft::k_z_c2r<T, NN, Z::B, Z::NT, NIN, Out, Z::template minb<NIN>()>;
      set_smem(kern, NIN * Z::SMEM);
      ::pm::note_launch();
      kern<<<(int)((int64_t)nb * n * n / Z::B), Z::NT, NIN * Z::SMEM, st>>>(ins, out, tw);
    });
    PM_LAUNCH_CHECK();
    return PM_OK;
  }

  static fft::MultDesc md(double scale, int d1, int d2, int flags) {
    fft::MultDesc m{};
    m.scale = scale;
    m.d1 = d1;
    m.d2 = d2;
    m.flags = flags;
    return m;
  }
  double inv_n3() const { return 1.0 / (double)M; }
  // phi_ij slot order 00, 11, 22, 01, 02, 12
  static void pair_of(int c, int &i, int &j) {
    static const int P[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    i = P[c][0];
    j = P[c][1];
  }

#define PM_TRY(x)                  \
  do {                             \
    pm_status s__ = (x);           \
    if (s__ != PM_OK) return s__;  \
  } while (0)

  pm_status set_exp(int slot_i, int v) {
    ::pm::note_launch();
    k_set_int<<<1, 1, 0, st>>>(fx_exp + slot_i, v);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  // maxslot = max of the partial maxima a running-max kernel left in maxslots
  pm_status fold_max() {
    ::pm::note_launch();
    part::k_fold_max<T><<<1, part::kMaxSlots, 0, st>>>(maxslots, maxslot);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  pm_status memset_fx(int channels) {
    PM_CUDA_TRY(cudaMemsetAsync(fx, 0, (size_t)channels * M * sizeof(long long), st));
    return PM_OK;
  }
  // One deposition launch of a particle source into the fixed-point
  // channels of fx (Src::NCH planes of M cells).
  template <class Src> pm_status deposit(Src s) {
    ::pm::note_launch();
    part::k_deposit<T, Src><<<grid_for(M, 256), 256, 0, st>>>(geo(), s, reinterpret_cast<unsigned long long *>(fx), M);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }

  // ---- forward stages ----
  // 2LPT: fills disp0 / mom (cell units), phi_ij (when keep), paints density.
  pm_status lpt(const T *s, T *disp0, bool paint) {
    PM_TRY(r2c_real(s, 1, slot(0)));
    PM_TRY(ypass(slot(0), 1, -1));
    fft::MultDesc m[9];
    int outs[9];
    const double sc = inv_n3();
    for (int i = 0; i < 3; ++i) {
      m[i] = md(sc, i, -1, fft::M_INVK2 | fft::M_AMP);  // Psi1_i = D_i A / k^2
      outs[i] = i;
    }
    int cnt = 3;
    if (cfg.lpt_order == 2) {
      for (int c = 0; c < 6; ++c) {
        int i, j;
        pair_of(c, i, j);
        m[3 + c] = md(-sc, i, j, fft::M_INVK2 | fft::M_AMP);  // phi_ij = -D_i D_j A / k^2
        outs[3 + c] = 3 + c;
      }
      cnt = 9;
    }
    PM_TRY(x1toM(slot(0), outs, m, cnt));
    PM_TRY(ypass(slot(0), cnt, +1));
    PM_TRY((c2r<1>(0, 3, OutPlanar<T>{psi, n})));
    if (cfg.lpt_order == 2) {
      PM_TRY((c2r<6>(3, 1, OutLptSource<T>{phi6, src, M, n})));
      PM_TRY(r2c_real(src, 1, slot(0)));
      PM_TRY(ypass(slot(0), 1, -1));
      fft::MultDesc m2[3];
      int o2[3] = {0, 1, 2};
      for (int i = 0; i < 3; ++i) m2[i] = md(-sc, i, -1, fft::M_INVK2);  // Psi2_i = -D_i / k^2 S
      PM_TRY(x1toM(slot(0), o2, m2, 3));
      PM_TRY(ypass(slot(0), 3, +1));
      PM_TRY((c2r<1>(0, 3, OutPlanar<T>{psi2, n})));
    }
    if (paint) {
      PM_TRY(memset_fx(1));
      PM_TRY(set_exp(0, rho_exp));
    }
    const double ic = 1.0 / cell;
    const part::Geo g = geo();
    return deposit(part::SrcLpt<T>{g.L, M, psi, cfg.lpt_order == 2 ? psi2 : nullptr, (T)(d1 * ic), (T)(d2 * ic),
                                   (T)(gp1 * ic), (T)(gp2 * ic), disp0, mom, paint ? fx_exp : nullptr, T(0)});
  }

  // PM force mesh (cell units) of stored state `si` from the painted density
  // in fx channel 0 (transformed as delta = rho - 1, N_mesh = N_part).
  pm_status force_mesh(int si) {
    V4<T> *out = pstate(si);
    PM_TRY(r2c_fixed(fx, fx_exp, 1, slot(0), true));
    PM_TRY(ypass(slot(0), 1, -1));
    fft::MultDesc m[3];
    int outs[3] = {0, 1, 2};
    const double sc = 1.5 * cfg.omega_m / cell * inv_n3();
    for (int i = 0; i < 3; ++i) m[i] = md(sc, i, -1, fft::M_INVK2);  // F_i = 1.5 Om D_i / k^2 delta
    PM_TRY(x1toM(slot(0), outs, m, 3));
    PM_TRY(ypass(slot(0), 3, +1));
    PM_TRY((c2r<3>(0, 1, OutForce<T>{out, n})));
    return PM_OK;
  }

  T *dstate(int k) const { return disp + (int64_t)k * 3 * M; }
  V4<T> *pstate(int k) const { return phi + (int64_t)k * M; }

  // Leapfrog steps [k0, k1) from disp_k0 (in slot k0 - base) with force
  // meshes; when store, every state k in (k0, k1] gets its own slot.
  // After the loop the force mesh of state k1 is in its slot.
  pm_status run_steps(int k0, int k1, int base_slot, bool store, T *momb) {
    const part::Geo g = geo();
    for (int k = k0; k < k1; ++k) {
      const int si = store ? k - base_slot : 0;
      const int so = store ? k + 1 - base_slot : 0;
      PM_TRY(memset_fx(1));
      {
        // method: x, p read and written, 3 force components read, density written;
        // implementation: float4 force mesh, 64-bit fixed-point density
        ProfScope ps(prof, P_KDK, st, (double)M * 16 * sizeof(T), (double)M * (16 * sizeof(T) + 8));
        part::SrcKdk<T> src_k{g.L, M, pstate(si), dstate(si), dstate(so), momb, (T)ck[k], (T)dr[k], fx_exp, T(0)};
        if (lc_on && lc_write && (k == lc_k[0] || k == lc_k[1])) {
          const int j = k == lc_k[0] ? 0 : 1;
          src_k.snap_x = snap + (int64_t)j * 3 * M;
          src_k.snap_p = snap + (int64_t)(2 + j) * 3 * M;
          src_k.kb = (T)kbv[k];
        }
        PM_TRY(deposit(src_k));
      }
      PM_TRY(force_mesh(so));
    }
    return PM_OK;
  }

  // Full forward to the painted final density (fx channel 0).  keep: store
  // states for the adjoint.
  pm_status forward_to_density(const T *s, bool keep) {
    const int ns = cfg.n_steps;
    PM_TRY(lpt(s, dstate(0), true));
    PM_TRY(force_mesh(0));
    if (keep_all() || !keep) {
      PM_TRY(run_steps(0, ns, 0, keep && keep_all(), mom));
    } else {
      // checkpoint mode: states 0, c, 2c, ... kept in the checkpoint arrays
      const int ce = cfg.checkpoint_every;
      for (int k = 0; k < ns; ++k) {
        if (k % ce == 0) {
          PM_CUDA_TRY(cudaMemcpyAsync(ckd + (int64_t)(k / ce) * 3 * M, dstate(0), 3 * M * sizeof(T),
                                      cudaMemcpyDeviceToDevice, st));
          PM_CUDA_TRY(cudaMemcpyAsync(ckm + (int64_t)(k / ce) * 3 * M, mom, 3 * M * sizeof(T),
                                      cudaMemcpyDeviceToDevice, st));
        }
        PM_TRY(run_steps(k, k + 1, 0, false, mom));
      }
      if (ns % ce == 0) {
        PM_CUDA_TRY(cudaMemcpyAsync(ckd + (int64_t)(ns / ce) * 3 * M, dstate(0), 3 * M * sizeof(T),
                                    cudaMemcpyDeviceToDevice, st));
        PM_CUDA_TRY(cudaMemcpyAsync(ckm + (int64_t)(ns / ce) * 3 * M, mom, 3 * M * sizeof(T),
                                    cudaMemcpyDeviceToDevice, st));
      }
      PM_CUDA_TRY(cudaMemcpyAsync(dwork, dstate(0), 3 * M * sizeof(T), cudaMemcpyDeviceToDevice, st));
    }
    const int fin = (keep && keep_all()) ? ns : 0;
    PM_TRY(memset_fx(1));
    part::SrcFinal<T> fsrc{geo().L, M, pstate(fin), dstate(fin), mom, (T)ck[ns], cfg.rsd_axis, (T)rsd,
                           fx_exp, T(0), {obs_cell(0), obs_cell(1), obs_cell(2)}};
    if (lc_on) {
      fsrc.lightcone = true;
      fsrc.lc = lightcone();
    }
    return deposit(fsrc);
  }

  // likelihood and bias parameters of the kernels, the bias model resolved
  pw::LossParams loss_params() const {
    pw::LossParams lp{};
    lp.lik = cfg.likelihood;
    lp.bias = cfg.bias == PM_BIAS_LINEAR || (cfg.bias == PM_BIAS_AUTO && cfg.likelihood == PM_LIK_GAUSSIAN) ? 0 : 1;
    lp.b = cfg.bias_b;
    lp.inv_s2 = cfg.likelihood == PM_LIK_GAUSSIAN ? 1.0 / (cfg.sigma * cfg.sigma) : 0.0;
    lp.alpha = cfg.alpha;
    lp.delta_th = cfg.delta_th;
    lp.K = cfg.K;
    lp.nbar = cfg.nbar_cell;
    lp.rho_floor = cfg.rho_floor;
    lp.lw = 1.0;
    return lp;
  }

  pm_status loss_terms(const T *s, const T *data, const T *R, const T *cot, double lw, bool want_dbar,
                       T *delta_out) {
    pw::LossParams lp = loss_params();
    lp.lw = lw;
    const double lw_io = (2 + (want_dbar ? 1 : 0) + (delta_out ? 1 : 0)) * sizeof(T);
    ProfScope ps(prof, P_LOSS, st, (double)M * (sizeof(T) + lw_io), (double)M * (8 + lw_io));
    ::pm::note_launch();
    pw::k_loss<T><<<pw::kRedBlocks, pw::kRedThreads, 0, st>>>(lp, fx, fx_exp, data, R, cot,
                                                               want_dbar ? dbar : nullptr, delta_out, M, partial);
    PM_LAUNCH_CHECK();
    ::pm::note_launch();
    pw::k_sum_partials<<<1, pw::kRedThreads, 0, st>>>(partial, pw::kRedBlocks, results + 0);
    PM_LAUNCH_CHECK();
    ::pm::note_launch();
    pw::k_sumsq<T><<<pw::kRedBlocks, pw::kRedThreads, 0, st>>>(s, M, partial);
    PM_LAUNCH_CHECK();
    ::pm::note_launch();
    pw::k_sum_partials<<<1, pw::kRedThreads, 0, st>>>(partial, pw::kRedBlocks, results + 1);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }

  pm_status read_loss(double *loss_out) {
    double h[2];
    PM_CUDA_TRY(cudaMemcpyAsync(h, results, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    last_lik = h[0];
    last_prior = 0.5 * cfg.prior_weight * h[1];
    const double tot = last_lik + last_prior;
    if (loss_out) *loss_out = tot;
    if (!std::isfinite(tot)) {
      set_error("loss is not finite");
      return PM_ERR_NONFINITE;
    }
    return PM_OK;
  }

  pm_status forward(const T *s, const T *data, const T *R, double *loss_out, T *delta_out) {
    PM_TRY(forward_to_density(s, false));
    PM_TRY(loss_terms(s, data, R, nullptr, 1.0, false, delta_out));
    return read_loss(loss_out);
  }

  // ---- adjoint ----
  // rhobar = sum_i G_i^T m_i from the 3-channel fixed-point paint in fx.
  pm_status adjoint_force(T *rhobar) {
    PM_TRY(r2c_fixed(fx, fx_exp + 1, 3, slot(0)));
    PM_TRY(ypass(slot(0), 3, -1));
    fft::MultDesc m[3];
    int ins[3] = {0, 1, 2};
    const double sc = 1.5 * cfg.omega_m / cell * inv_n3();
    for (int i = 0; i < 3; ++i) m[i] = md(sc, i, -1, fft::M_INVK2 | fft::M_CONJ);
    PM_TRY(xMto1(ins, 0, m, 3));
    PM_TRY(ypass(slot(0), 1, +1));
    PM_TRY((c2r<1>(0, 1, OutPlanar<T>{rhobar, n})));
    return PM_OK;
  }

  // reverse of the kick at state k (x_k in xk, force mesh phik), then the
  // reverse of the drift into state k (when k > 0)
  pm_status reverse_step(int k, const T *xk, const V4<T> *phik, int slot) {
    const part::Geo g = geo();
    const int nb = grid_for(M, 256);
    if (k == cfg.n_steps && cfg.rsd_axis < 0) {
      // Without a redshift-space shift the final state's momentum cotangent is
      // exactly zero, so the last kick's adjoint (cotangent paint, adjoint
      // force, gather) adds exact zeros: only the reverse drift remains.
      const T drift = k > 0 ? (T)dr[k - 1] : T(0);
      const T cnext = k > 0 ? (T)ck[k - 1] : T(0);
      ::pm::note_launch();
      part::k_reverse_drift<T><<<nb, 256, 0, st>>>(g, xbar, pbar, drift, cnext, k > 0 ? maxslots : nullptr);
      PM_LAUNCH_CHECK();
      return k > 0 ? fold_max() : PM_OK;
    }
    PM_TRY(memset_fx(3));
    {
      // method (the 3-channel paint's 24 B / particle in FP32): positions read,
      // three mesh channels written; implementation: positions and cotangent
      // read, 64-bit fixed-point channels
      ProfScope ps(prof, P_ADJ_PAINT, st, (double)M * 6 * sizeof(T), (double)M * (6 * sizeof(T) + 24));
      PM_TRY(deposit(part::SrcAdj3<T>{g.L, M, g.log2np, xk, pbar, (T)ck[k], maxslot, fx_exp + 1, 0}));
    }
    PM_TRY(adjoint_force(src));
    const T drift = k > 0 ? (T)dr[k - 1] : T(0);
    const T cnext = k > 0 ? (T)ck[k - 1] : T(0);
    {
      // method: x, xbar, pbar read, xbar, pbar written, 3 force components and
      // rhobar read (the implementation's force mesh is float4)
      ProfScope ps(prof, P_ADJ_GATHER, st, (double)M * 19 * sizeof(T), (double)M * 20 * sizeof(T));
      ::pm::note_launch();
      part::k_adj_gather<T><<<nb, 256, 0, st>>>(g, xk, phik, src, (T)ck[k], xbar, pbar, drift, cnext,
                                                 k > 0 ? maxslots : nullptr);
    }
    PM_LAUNCH_CHECK();
    return k > 0 ? fold_max() : PM_OK;
  }

  // reverse_step, with the cotangents (Xbar_j, Pbar_j) of a lightcone snapshot
  // held at state k joined in.  The snapshot momentum mom + kb F(x_k) shares
  // the force F(x_k) with the merged kick c_k, so before the step
  // pbar += (kb / c_k) Pbar_j makes its cotangent paint c_k pbar + kb Pbar_j,
  // and after it pbar += (1 - kb / c_k) Pbar_j completes the cotangent of the
  // momentum before the kick (then the running max is taken again).
  pm_status reverse_step_lc(int k, const T *xk, const V4<T> *phik, int slot) {
    const int j = !lc_on ? -1 : (k == lc_k[0] ? 0 : (k == lc_k[1] ? 1 : -1));
    if (j < 0) return reverse_step(k, xk, phik, slot);
    const part::Geo g = geo();
    const int nb = grid_for(M, 256);
    const T *xb = snap + (int64_t)j * 3 * M, *pb = snap + (int64_t)(2 + j) * 3 * M;
    const double f = kbv[k] / ck[k];
    ::pm::note_launch();
    part::k_lc_join<T><<<nb, 256, 0, st>>>(g, xbar, pbar, xb, pb, (T)f, (T)ck[k], maxslots);
    PM_LAUNCH_CHECK();
    PM_TRY(fold_max());
    PM_TRY(reverse_step(k, xk, phik, slot));
    ::pm::note_launch();
    part::k_lc_join<T><<<nb, 256, 0, st>>>(g, nullptr, pbar, nullptr, pb, (T)(1.0 - f),
                                            k > 0 ? (T)ck[k - 1] : T(0), maxslots);
    PM_LAUNCH_CHECK();
    return fold_max();
  }

  pm_status adjoint(const T *s, const T *data, const T *R, double lw, const T *cot, double *loss_out,
                    T *grad) {
    const int ns = cfg.n_steps;
    PM_TRY(forward_to_density(s, true));
    PM_TRY(loss_terms(s, data, R, cot, lw, true, nullptr));
    const part::Geo g = geo();
    const int nb = grid_for(M, 256);
    // final paint + RSD
    const T *xn = keep_all() ? dstate(ns) : dwork;
    ::pm::note_launch();
    if (lc_on) {
      // cotangents of the final state into (xbar, pbar), of the other two
      // snapshots over the snapshot buffer
      part::k_adj_final_lc<T><<<nb, 256, 0, st>>>(g, lightcone(), snap, xn, mom, dbar, xbar, pbar, (T)ck[ns],
                                                   maxslots);
    } else {
      part::k_adj_final<T><<<nb, 256, 0, st>>>(g, xn, mom, cfg.rsd_axis, (T)rsd, obs_cell(0), obs_cell(1),
                                                obs_cell(2), dbar, xbar, pbar, (T)ck[ns], maxslots);
    }
    PM_LAUNCH_CHECK();
    PM_TRY(fold_max());
    if (keep_all()) {
      for (int k = ns; k >= 0; --k) PM_TRY(reverse_step_lc(k, dstate(k), pstate(k), k));
    } else {
      const int ce = cfg.checkpoint_every;
      for (int j = ns / ce; j >= 0; --j) {
        const int lo = j * ce, hi = std::min(lo + ce - 1, ns);
        // restore checkpoint j and recompute states lo..hi with their force meshes
        PM_CUDA_TRY(cudaMemcpyAsync(dstate(0), ckd + (int64_t)j * 3 * M, 3 * M * sizeof(T),
                                    cudaMemcpyDeviceToDevice, st));
        PM_CUDA_TRY(cudaMemcpyAsync(psi2, ckm + (int64_t)j * 3 * M, 3 * M * sizeof(T),
                                    cudaMemcpyDeviceToDevice, st));
        PM_TRY(memset_fx(1));
        PM_TRY(set_exp(0, rho_exp));
        PM_TRY(deposit(part::SrcPaint<T>{g.L, M, dstate(0), psi2, -1, T(0), fx_exp, T(0)}));
        PM_TRY(force_mesh(0));
        lc_write = false;  // the snapshot buffer holds their cotangents now
        const pm_status rs = run_steps(lo, hi, lo, true, psi2);
        lc_write = true;
        PM_TRY(rs);
        for (int k = hi; k >= lo; --k) PM_TRY(reverse_step_lc(k, dstate(k - lo), pstate(k - lo), k - lo));
      }
    }
    PM_TRY(lpt_adjoint(s, lw, grad));
    return read_loss(loss_out);
  }

  // 2LPT + IC adjoint from (xbar, pbar) at state 0, plus the prior gradient.
  pm_status lpt_adjoint(const T *s, double lw, T *grad) {
    const double ic = 1.0 / cell;
    ::pm::note_launch();
    part::k_lpt_adj<T><<<grid_for(3 * M, 256), 256, 0, st>>>(M, xbar, pbar, (T)d1, (T)d2, (T)gp1, (T)gp2, (T)ic,
                                                             psi, cfg.lpt_order == 2 ? psi2 : nullptr);
    PM_LAUNCH_CHECK();
    const double sc = inv_n3();
    fft::MultDesc m[9];
    int ins[9];
    int cnt = 3;
    for (int i = 0; i < 3; ++i) {
      m[i] = md(sc, i, -1, fft::M_INVK2 | fft::M_AMP | fft::M_CONJ);
      ins[i] = i;
    }
    if (cfg.lpt_order == 2) {
      // Sbar = sum_i conj(-D_i / k^2) FFT(psi2bar_i)
      PM_TRY(r2c_real(psi2, 3, slot(0)));
      PM_TRY(ypass(slot(0), 3, -1));
      fft::MultDesc m2[3];
      int in2[3] = {0, 1, 2};
      for (int i = 0; i < 3; ++i) m2[i] = md(-sc, i, -1, fft::M_INVK2 | fft::M_CONJ);
      PM_TRY(xMto1(in2, 0, m2, 3));
      PM_TRY(ypass(slot(0), 1, +1));
      PM_TRY((c2r<1>(0, 1, OutPlanar<T>{src, n})));
      ::pm::note_launch();
      pw::k_phibar<T><<<grid_for(M, 256), 256, 0, st>>>(phi6, src, M);
      PM_LAUNCH_CHECK();
      for (int c = 0; c < 6; ++c) {
        int i, j;
        pair_of(c, i, j);
        m[3 + c] = md(-sc, i, j, fft::M_INVK2 | fft::M_AMP | fft::M_CONJ);
        ins[3 + c] = 3 + c;
      }
      cnt = 9;
    }
    PM_TRY(r2c_real(psi, cnt, slot(0)));
    PM_TRY(ypass(slot(0), cnt, -1));
    PM_TRY(xMto1(ins, 0, m, cnt));
    PM_TRY(ypass(slot(0), 1, +1));
    PM_TRY((c2r<1>(0, 1, OutGrad<T>{grad, s, (T)(lw * cfg.prior_weight), n})));
    return PM_OK;
  }

  // model mean per cell: Poisson lambda = R nbar g(delta), Gaussian f(delta)
  pm_status expected_counts(const T *s, const T *R, T *out) {
    PM_TRY(forward_to_density(s, false));
    const pw::LossParams lp = loss_params();
    ::pm::note_launch();
    pw::k_expected<T><<<grid_for(M, 256), 256, 0, st>>>(lp, fx, fx_exp, R, out, M);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }

  // ---- resolution transfer of the white noise (annealing) ----
  // s_fine(k) = r^{3/2} s_c(k) on the coarse modes with every |n_i| < n_c / 2,
  // fresh(k) on all other modes (r = n / n_c): the fine field keeps the coarse
  // field's linear density (the IC amplitude scales as Delta^{-3/2}) and stays
  // unit white noise.  The coarse spectrum comes from the fine FFT of the
  // zero-stuffed coarse field; psi (rebuilt by every forward) is the scratch.
  pm_status refine_noise(const T *sc, int n_c, const T *fresh, T *out) {
    int logc = 0;
    while ((1 << logc) < n_c) ++logc;
    const int logr = logn - logc;
    ::pm::note_launch();
    pw::k_zero_stuff<T><<<grid_for(M, 256), 256, 0, st>>>(sc, logn, logr, psi);
    PM_LAUNCH_CHECK();
    PM_CUDA_TRY(cudaMemcpyAsync(psi + M, fresh, M * sizeof(T), cudaMemcpyDeviceToDevice, st));
    PM_TRY(r2c_real(psi, 2, slot(0)));
    PM_TRY(ypass(slot(0), 2, -1));
    const double r3 = std::ldexp(1.0, 3 * logr);
    fft::MultDesc m[2] = {md(std::sqrt(r3) * inv_n3(), -1, -1, fft::M_INCUBE),
                          md(inv_n3(), -1, -1, fft::M_OUTCUBE)};
    m[0].cube = m[1].cube = n_c / 2;
    int ins[2] = {0, 1};
    PM_TRY(xMto1(ins, 0, m, 2));
    PM_TRY(ypass(slot(0), 1, +1));
    PM_TRY((c2r<1>(0, 1, OutPlanar<T>{out, n})));
    return PM_OK;
  }

  // ---- analysis of fields (Sec. 3.2, 3.3) ----
  // Binned P_aa, P_bb, P_ab and mode counts (host[4][nbins]); b may be null.
  // P = (V / n^6) sum w |X|^2 / sum w over the bin's half-spectrum modes.
  pm_status power_spectra(const T *a, const T *b, int nbins, double kmin, double kmax, double *host) {
    double *bins = reinterpret_cast<double *>(fx);  // the paint meshes are free between model calls
    PM_CUDA_TRY(cudaMemsetAsync(bins, 0, 4 * (size_t)nbins * sizeof(double), st));
    PM_TRY(r2c_real(a, 1, slot(0)));
    if (b) PM_TRY(r2c_real(b, 1, slot(1)));
    PM_TRY(ypass(slot(0), b ? 2 : 1, -1));
    const double dk = (kmax - kmin) / nbins;
    PM_DISPATCH_N(n, {
      using CC = CCfg<T, NN>;
      auto kern = an::k_x_power<T, NN, CC::B, CC::NT>;
      const size_t sm = CC::SMEM2 + 4 * (size_t)nbins * sizeof(double);
      set_smem(kern, sm);
      ::pm::note_launch();
      kern<<<(int)(S / n / CC::B), CC::NT, sm, st>>>(slot(0), b ? slot(1) : nullptr, tw, kf, kmin, dk, nbins,
                                                    bins);
    });
    PM_LAUNCH_CHECK();
    PM_CUDA_TRY(cudaMemcpyAsync(host, bins, 4 * (size_t)nbins * sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    const double norm = cfg.box * cfg.box * cfg.box / ((double)M * (double)M);
    for (int j = 0; j < nbins; ++j) {
      const double cnt = host[3 * nbins + j];
      for (int q = 0; q < 3; ++q) host[q * nbins + j] = cnt > 0 ? host[q * nbins + j] * norm / cnt : NAN;
    }
    return PM_OK;
  }
  // out = IFFT[exp(-|k|^2 r^2 / 2) FFT(in)]
  pm_status smooth(const T *in, double r, T *out) {
    PM_TRY(r2c_real(in, 1, slot(0)));
    PM_TRY(ypass(slot(0), 1, -1));
    fft::MultDesc m = md(inv_n3(), -1, -1, fft::M_GAUSS);
    m.gauss = 0.5 * r * r;
    int o = 0;
    PM_TRY(x1toM(slot(0), &o, &m, 1));
    PM_TRY(ypass(slot(0), 1, +1));
    PM_TRY((c2r<1>(0, 1, OutPlanar<T>{out, n})));
    return PM_OK;
  }
  // T-web: psi_ij = IFFT[k_i k_j / k^2 G(k) FFT(delta)] (into the 2LPT scratch),
  // then the per-cell eigen-decomposition and label.
  pm_status tweb(const T *delta, double r, double th, int *labels, T *eig, T *evec) {
    PM_TRY(r2c_real(delta, 1, slot(0)));
    PM_TRY(ypass(slot(0), 1, -1));
    fft::MultDesc m[6];
    int outs[6];
    for (int c = 0; c < 6; ++c) {
      int i, j;
      pair_of(c, i, j);
      m[c] = md(-inv_n3(), i, j, fft::M_INVK2 | fft::M_GAUSS);  // -(i k_i)(i k_j) / k^2 G
      m[c].gauss = 0.5 * r * r;
      outs[c] = c;
    }
    PM_TRY(x1toM(slot(0), outs, m, 6));
    PM_TRY(ypass(slot(0), 6, +1));
    PM_TRY((c2r<1>(0, 6, OutPlanar<T>{psi, n})));
    ::pm::note_launch();
    an::k_tweb_eigen<T><<<grid_for(M, 256), 256, 0, st>>>(psi, M, th, labels, eig, evec);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }

  // ---- probes ----
  pm_status linear_field(const T *s, T *out) {
    PM_TRY(r2c_real(s, 1, slot(0)));
    PM_TRY(ypass(slot(0), 1, -1));
    fft::MultDesc m = md(inv_n3(), -1, -1, fft::M_AMP);
    int o = 0;
    PM_TRY(x1toM(slot(0), &o, &m, 1));
    PM_TRY(ypass(slot(0), 1, +1));
    PM_TRY((c2r<1>(0, 1, OutPlanar<T>{out, n})));
    return PM_OK;
  }
  pm_status probe_lpt(const T *s, T *disp_out, T *mom_out) {
    PM_TRY(lpt(s, dstate(0), false));
    const int nb = grid_for(3 * M, 256);
    ::pm::note_launch();
    pw::k_scale<T><<<nb, 256, 0, st>>>(dstate(0), (T)cell, disp_out, 3 * M);
    ::pm::note_launch();
    pw::k_scale<T><<<nb, 256, 0, st>>>(mom, (T)cell, mom_out, 3 * M);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  pm_status probe_force(const T *disp_in, T *force_out, T *density_out) {
    const int nb3 = grid_for(3 * M, 256);
    ::pm::note_launch();
    pw::k_scale<T><<<nb3, 256, 0, st>>>(disp_in, (T)(1.0 / cell), dstate(0), 3 * M);
    PM_LAUNCH_CHECK();
    PM_TRY(memset_fx(1));
    PM_TRY(set_exp(0, rho_exp));
    PM_TRY(deposit(part::SrcPaint<T>{geo().L, M, dstate(0), mom, -1, T(0), fx_exp, T(0)}));
    if (density_out) {
      ::pm::note_launch();
      pw::k_fixed_to_delta<T><<<grid_for(M, 256), 256, 0, st>>>(fx, fx_exp, density_out, M);
      PM_LAUNCH_CHECK();
    }
    PM_TRY(force_mesh(0));
    ::pm::note_launch();
    part::k_readout<T><<<grid_for(M, 256), 256, 0, st>>>(geo(), pstate(0), dstate(0), (T)cell, force_out);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  pm_status probe_evolve(const T *s, T *disp_out, T *mom_out) {
    PM_TRY(lpt(s, dstate(0), true));
    PM_TRY(force_mesh(0));
    PM_TRY(run_steps(0, cfg.n_steps, 0, false, mom));
    PM_TRY(deposit(part::SrcFinal<T>{geo().L, M, pstate(0), dstate(0), mom, (T)ck[cfg.n_steps], -1, T(0),
                                         nullptr, T(0)}));
    const int nb = grid_for(3 * M, 256);
    ::pm::note_launch();
    pw::k_scale<T><<<nb, 256, 0, st>>>(dstate(0), (T)cell, disp_out, 3 * M);
    ::pm::note_launch();
    pw::k_scale<T><<<nb, 256, 0, st>>>(mom, (T)cell, mom_out, 3 * M);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
#undef PM_TRY
};

}  // namespace pm
