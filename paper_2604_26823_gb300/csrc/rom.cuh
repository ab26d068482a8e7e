// Projection operator P and rank-order matching R on the GPU
// (Sec. 2.3.1: z-score then reset of |s_hat| > s_th = 10 to fresh N(0,1)
// draws; Sec. 2.3.2: rank-order matching in real space over R > 0 and in
// Fourier space in 100 equal-width |k| bins, k < 0.1 h/Mpc untouched).
//
// Reset draws: counter-based SplitMix64 stream (Steele, Lea & Flood 2014)
// keyed by (seed, counter, element index), Box-Muller in FP64:
//   key = mix(seed + counter*G + G),  h_j = mix(key + (2 i + 1 + j) G),
//   u1 = ((h_0 >> 11) + 1) 2^-53,  u2 = (h_1 >> 11) 2^-53,
//   z = sqrt(-2 ln u1) cos(2 pi u2),  G = 0x9E3779B97F4A7C15.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "engine.cuh"
#include "sort.cuh"

namespace pm {
namespace rom {

constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double counter_normal(unsigned long long key, unsigned long long idx) {
  const unsigned long long h0 = mix64(key + (2ull * idx + 1ull) * kGolden);
  const unsigned long long h1 = mix64(key + (2ull * idx + 2ull) * kGolden);
  const double u1 = ((double)(h0 >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(h1 >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// Block partials of the sum, or (mean from results[slot_mu] given) of the
// sum of squared deviations; FP64 partials.
template <typename T>
__global__ void k_moment(const T *__restrict__ x, int64_t n, const double *mean_sum, double *partial) {
  // FP32 data: the deviation is formed in FP32 from the rounded mean (its
  // rounding is ~1e-7 of the deviation, far inside the FP32 path's 1e-6
  // projection tolerance) and both sums are compensated (pw::DotAcc/SumAcc)
  const T mu = mean_sum ? (T)(*mean_sum / (double)n) : T(0);
  pw::SumAcc<T> s1;
  pw::DotAcc<T> s2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (mean_sum) {
      const T v = x[i] - mu;
      s2.add(v, v);
    } else {
      s1.add(x[i]);
    }
  }
  pw::block_sum_store(mean_sum ? s2.value() : s1.value(), partial);
}

// Projection scalars once: mu, sd, 1/sd (FP64) from the two FP64 sums, and
// a flag (1 or 0) telling whether they define a projection at all (finite
// moments, sd > 0).
static __global__ void k_project_scalars(int64_t n, const double *sum, const double *sumsq_dev, double *out4) {
  const double mu = *sum / (double)n;
  const double sd = sqrt(*sumsq_dev / (double)n);
  out4[0] = mu;
  out4[1] = sd;
  out4[2] = 1.0 / sd;
  out4[3] = (isfinite(mu) && isfinite(sd) && sd > 0.0) ? 1.0 : 0.0;
}

// s_hat = (s - mu)/sd; |s_hat| > s_th -> counter-based N(0,1).  The value is
// formed as (s - mu) * (1/sd) in T (within an ulp of T of the FP64 quotient,
// without an FP64 division per element on the narrow FP64 unit); the reset
// decision is taken on the FP64 quotient itself, evaluated for the elements
// whose fast value lies within 1e-4 of the threshold, so the set of reset
// elements is the FP64 rule's.  When the scalars' flag is 0 (NaN / Inf in s,
// or zero variance) nothing is written: s keeps its values and the host
// reports the error.
template <typename T>
__global__ void k_project(T *s, int64_t n, const double *scal, double s_th, unsigned long long key,
                          unsigned long long *nreset) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || scal[3] == 0.0) return;
  const T mu = (T)scal[0], inv = (T)scal[2];
  const T near_th = (T)(s_th * (1.0 - 1e-4));
  const T v = s[i];
  T z = (v - mu) * inv;
  if (fabs(z) > near_th) {
    const double zd = ((double)v - scal[0]) / scal[1];
    if (fabs(zd) > s_th) {
      z = (T)counter_normal(key, (unsigned long long)i);
      atomicAdd(nreset, 1ull);
    }
  }
  s[i] = z;
}

template <typename T> __global__ void k_count_pos(const T *__restrict__ R, int64_t n, double *partial) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += R[i] > T(0) ? 1.0 : 0.0;
  pw::block_sum_store(acc, partial);
}

// Real-space matching keys: cells with R > 0 sort first, descending by s.
template <typename T, typename K>
__global__ void k_real_keys(const T *__restrict__ s, const T *__restrict__ R, int64_t n, K *keys,
                            unsigned int *vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = R[i] > T(0) ? sortk::desc_key(s[i]) : ~K(0);
  vals[i] = (unsigned int)i;
}

// s[cell of the j-th sorted entry] = targets[j] for the R > 0 entries, and
// that cell's rank j (when rank is given; the other cells keep -1).
template <typename T, typename K>
__global__ void k_real_assign(const K *__restrict__ keys, const unsigned int *__restrict__ vals, int64_t n,
                              const T *__restrict__ targets, T *s, int *rank) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || keys[j] == ~K(0)) return;
  const unsigned int c = vals[j];
  s[c] = targets[j];
  if (rank) rank[c] = (int)j;
}

// Fourier mode selection: canonical member of its conjugate pair, not its
// own conjugate, |k| >= k_min; bin = floor(|k| / (sqrt(3) k_Nyq) * nbins).
// Integer arithmetic only per mode (the FP64 unit of this GPU is narrow): the
// test |k| >= k_min is n2 >= n2_min, the first |n|^2 at which the FP64
// expression kf sqrt(n2) >= kmin holds (it is monotone in n2), found once on
// the host by that same expression.
struct ModeSel {
  int n, h, nbins;
  double kf, kmin;
  long long n2_min;
  void init_threshold() {
    long long lo = 0, hi = 3ll * n * n + 1;  // kf sqrt(hi) exceeds any k_min the plan uses
    while (lo < hi) {
      const long long mid = (lo + hi) / 2;
      if (kf * std::sqrt((double)mid) < kmin) lo = mid + 1;
      else hi = mid;
    }
    n2_min = lo;
  }
  __host__ __device__ int bin_of(int ix, int iy, int iz) const {
    const int nx = ix < n / 2 ? ix : ix - n;
    const int ny = iy < n / 2 ? iy : iy - n;
    if ((long long)nx * nx + (long long)ny * ny + (long long)iz * iz < n2_min) return -1;
    if (iz == 0 || iz == n / 2) {
      const int px = (n - ix) % n, py = (n - iy) % n;
      const long long self = (long long)ix * n + iy, part = (long long)px * n + py;
      if (self >= part) return -1;  // self-conjugate or the partner is canonical
    }
    // bin = floor(|k| / (sqrt(3) k_Nyq) * nbins), evaluated exactly in
    // integers: the largest b with 3 n^2 b^2 <= 4 nbins^2 |n|^2
    const long long n2 = (long long)nx * nx + (long long)ny * ny + (long long)iz * iz;
    const long long lhs = 4ll * nbins * nbins * n2, c = 3ll * n * n;
    long long b = (long long)sqrtf((float)lhs / (float)c);  // estimate, corrected below
    while (b > 0 && c * b * b > lhs) --b;
    while (c * (b + 1) * (b + 1) <= lhs) ++b;
    return b < nbins - 1 ? (int)b : nbins - 1;
  }
};

// keys over all 2 S real components: value = sqrt(2/N^3) Re / Im
template <typename T, typename K>
__global__ void k_fourier_keys(const cx<T> *__restrict__ sk, ModeSel ms, T scale, int64_t nmodes, K *keys,
                               unsigned int *vals) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * nmodes) return;
  const cx<T> v = sk[e >> 1];
  keys[e] = sortk::desc_key((e & 1) ? scale * v.y : scale * v.x);
  vals[e] = (unsigned int)e;
}

// second pass key: the bin of each (sorted) element, 255 when not matched
template <typename K>
__global__ void k_fourier_binkeys(const unsigned int *__restrict__ vals, ModeSel ms, int64_t ne, K *keys) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ne) return;
  const int64_t mode = vals[j] >> 1;
  const int iz = (int)(mode % ms.h);
  const int iy = (int)((mode / ms.h) % ms.n);
  const int ix = (int)(mode / ((int64_t)ms.h * ms.n));
  const int b = ms.bin_of(ix, iy, iz);
  keys[j] = (K)(b < 0 ? 255 : b);
}

template <typename T>
__global__ void k_fourier_assign(const unsigned int *__restrict__ vals, int64_t total, const T *__restrict__ targets,
                                 T inv_scale, T *sk_components) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= total) return;
  sk_components[vals[j]] = inv_scale * targets[j];
}

// Hermitian partners on the kz = 0 and kz = N/2 planes: copy the conjugate
// of each matched canonical mode to its partner.
template <typename T>
__global__ void k_fourier_partners(cx<T> *sk, ModeSel ms) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t plane = (int64_t)ms.n * ms.n;
  if (t >= 2 * plane) return;
  const int iz = t < plane ? 0 : ms.n / 2;
  const int64_t q = t % plane;
  const int ix = (int)(q / ms.n), iy = (int)(q % ms.n);
  if (ms.bin_of(ix, iy, iz) < 0) return;
  const int px = (ms.n - ix) % ms.n, py = (ms.n - iy) % ms.n;
  const cx<T> v = sk[((int64_t)ix * ms.n + iy) * ms.h + iz];
  sk[((int64_t)px * ms.n + py) * ms.h + iz] = cconj(v);
}

template <typename T> struct Rom {
  using K = typename sortk::KeyOf<T>::type;
  Engine<T> &E;

  ModeSel sel() const {
    ModeSel m;
    m.n = E.n;
    m.h = E.H;
    m.nbins = 100;
    m.kf = E.kf;
    m.kmin = 0.1;
    m.init_threshold();
    return m;
  }

  // host enumeration of the per-bin counts (2 values per matched mode)
  const std::vector<int64_t> &counts() {
    if (E.rom_counts.empty()) {
      const ModeSel m = sel();
      E.rom_counts.assign(100, 0);
      for (int ix = 0; ix < E.n; ++ix)
        for (int iy = 0; iy < E.n; ++iy)
          for (int iz = 0; iz < E.H; ++iz) {
            const int b = m.bin_of(ix, iy, iz);
            if (b >= 0) E.rom_counts[b] += 2;
          }
    }
    return E.rom_counts;
  }

  struct SortWs {
    K *k1, *k2;
    unsigned int *v1, *v2, *hist, *totals;
  };
  SortWs ws(int64_t nmax) const {
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char *p = reinterpret_cast<char *>(E.sort_ws);
    SortWs w;
    w.k1 = reinterpret_cast<K *>(p);
    p += al(nmax * sizeof(K));
    w.k2 = reinterpret_cast<K *>(p);
    p += al(nmax * sizeof(K));
    w.v1 = reinterpret_cast<unsigned int *>(p);
    p += al(nmax * 4);
    w.v2 = reinterpret_cast<unsigned int *>(p);
    p += al(nmax * 4);
    w.hist = reinterpret_cast<unsigned int *>(p);
    p += al((size_t)256 * sortk::tiles_for(nmax) * 4);
    w.totals = reinterpret_cast<unsigned int *>(p);
    return w;
  }
  int64_t nmax() const { return 2 * E.S; }

  pm_status real(T *s, const T *R, const T *targets, int *rank) {
    const int64_t n = E.M;
    if (rank) PM_CUDA_TRY(cudaMemsetAsync(rank, 0xff, (size_t)n * sizeof(int), E.st));  // -1 everywhere
    SortWs w = ws(nmax());
    ::pm::note_launch();
    k_real_keys<T, K><<<grid_for(n, 256), 256, 0, E.st>>>(s, R, n, w.k1, w.v1);
    PM_LAUNCH_CHECK();
    K *kr;
    unsigned int *vr;
    PM_CUDA_TRY(sortk::radix_sort<K>(w.k1, w.v1, w.k2, w.v2, n, 8 * (int)sizeof(K), w.hist, w.totals, E.st, &kr, &vr));
    ::pm::note_launch();
    k_real_assign<T, K><<<grid_for(n, 256), 256, 0, E.st>>>(kr, vr, n, targets, s, rank);
    PM_LAUNCH_CHECK();
    return PM_OK;
  }

  pm_status fourier(T *s, const T *targets) {
    const ModeSel m = sel();
    const int64_t nm = E.S, ne = 2 * E.S;
    int64_t total = 0;
    for (int64_t c : counts()) total += c;
    // full 3-D spectrum of s in slot 0
    pm_status st = E.r2c_real(s, 1, E.slot(0));
    if (st) return st;
    st = E.ypass(E.slot(0), 1, -1);
    if (st) return st;
    st = xpass(-1);
    if (st) return st;
    SortWs w = ws(nmax());
    const T scale = (T)std::sqrt(2.0 / (double)E.M);
    ::pm::note_launch();
    k_fourier_keys<T, K><<<grid_for(ne, 256), 256, 0, E.st>>>(E.slot(0), m, scale, nm, w.k1, w.v1);
    PM_LAUNCH_CHECK();
    K *kr;
    unsigned int *vr;
    PM_CUDA_TRY(sortk::radix_sort<K>(w.k1, w.v1, w.k2, w.v2, ne, 8 * (int)sizeof(K), w.hist, w.totals, E.st, &kr, &vr));
    K *kb = (kr == w.k1) ? w.k2 : w.k1;
    unsigned int *vb = (vr == w.v1) ? w.v2 : w.v1;
    ::pm::note_launch();
    k_fourier_binkeys<K><<<grid_for(ne, 256), 256, 0, E.st>>>(vr, m, ne, kr);
    PM_LAUNCH_CHECK();
    K *kr2;
    unsigned int *vr2;
    PM_CUDA_TRY(sortk::radix_sort<K>(kr, vr, kb, vb, ne, 8, w.hist, w.totals, E.st, &kr2, &vr2));
    ::pm::note_launch();
    k_fourier_assign<T><<<grid_for(total, 256), 256, 0, E.st>>>(vr2, total, targets, (T)(1.0 / (double)scale),
                                                                 reinterpret_cast<T *>(E.slot(0)));
    PM_LAUNCH_CHECK();
    ::pm::note_launch();
    k_fourier_partners<T><<<grid_for(2 * (int64_t)E.n * E.n, 256), 256, 0, E.st>>>(E.slot(0), m);
    PM_LAUNCH_CHECK();
    st = xpass(+1);
    if (st) return st;
    st = E.ypass(E.slot(0), 1, +1);
    if (st) return st;
    return E.template c2r<1>(0, 1, OutPlanar<T>{s, E.n, (T)(1.0 / (double)E.M)});
  }

  // plain complex FFT along x over the whole spectrum in slot 0
  pm_status xpass(int sign) {
    PM_DISPATCH_N(E.n, {
      using CC = CCfg<T, NN>;
      const int64_t ncols = (int64_t)E.n * E.H;
      const int tiles = (int)(ncols / CC::B);
      if (sign < 0) {
        auto kern = fft::k_col<T, NN, CC::B, CC::NT, -1>;
        set_smem(kern, CC::SMEM);
        ::pm::note_launch();
        kern<<<tiles, CC::NT, CC::SMEM, E.st>>>(E.slot(0), E.slot(0), ncols, 0, (int)ncols, tiles, E.tw);
      } else {
        auto kern = fft::k_col<T, NN, CC::B, CC::NT, +1>;
        set_smem(kern, CC::SMEM);
        ::pm::note_launch();
        kern<<<tiles, CC::NT, CC::SMEM, E.st>>>(E.slot(0), E.slot(0), ncols, 0, (int)ncols, tiles, E.tw);
      }
    });
    PM_LAUNCH_CHECK();
    return PM_OK;
  }
  pm_status count_positive(const T *R, int64_t *out) {
    ::pm::note_launch();
    k_count_pos<T><<<pw::kRedBlocks, pw::kRedThreads, 0, E.st>>>(R, E.M, E.partial);
    ::pm::note_launch();
    pw::k_sum_partials<<<1, pw::kRedThreads, 0, E.st>>>(E.partial, pw::kRedBlocks, E.results + 5);
    PM_LAUNCH_CHECK();
    double h;
    PM_CUDA_TRY(cudaMemcpyAsync(&h, E.results + 5, sizeof(double), cudaMemcpyDeviceToHost, E.st));
    PM_CUDA_TRY(cudaStreamSynchronize(E.st));
    *out = (int64_t)h;
    return PM_OK;
  }

  pm_status project(T *s, unsigned long long seed, unsigned long long counter, int64_t *nreset_out) {
    const int64_t n = E.M;
    double *res = E.results;
    ::pm::note_launch();
    k_moment<T><<<pw::kRedBlocks, pw::kRedThreads, 0, E.st>>>(s, n, nullptr, E.partial);
    ::pm::note_launch();
    pw::k_sum_partials<<<1, pw::kRedThreads, 0, E.st>>>(E.partial, pw::kRedBlocks, res + 2);
    ::pm::note_launch();
    k_moment<T><<<pw::kRedBlocks, pw::kRedThreads, 0, E.st>>>(s, n, res + 2, E.partial);
    ::pm::note_launch();
    pw::k_sum_partials<<<1, pw::kRedThreads, 0, E.st>>>(E.partial, pw::kRedBlocks, res + 3);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(res + 4);
    PM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), E.st));
    const unsigned long long key = mix64(seed + counter * kGolden + kGolden);
    ::pm::note_launch();
    k_project_scalars<<<1, 1, 0, E.st>>>(n, res + 2, res + 3, res + 6);
    ::pm::note_launch();
    k_project<T><<<grid_for(n, 256), 256, 0, E.st>>>(s, n, res + 6, 10.0, key, cnt);
    PM_LAUNCH_CHECK();
    double h[3];
    PM_CUDA_TRY(cudaMemcpyAsync(h, res + 2, 3 * sizeof(double), cudaMemcpyDeviceToHost, E.st));
    PM_CUDA_TRY(cudaStreamSynchronize(E.st));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1]) || !(h[1] > 0)) {
      set_error("projection input has NaN / Inf or zero variance");
      return PM_ERR_NONFINITE;
    }
    unsigned long long c;
    std::memcpy(&c, &h[2], sizeof(c));
    if (nreset_out) *nreset_out = (int64_t)c;
    return PM_OK;
  }
};

}  // namespace rom
}  // namespace pm
