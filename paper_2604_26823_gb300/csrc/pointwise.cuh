// Mesh-wise kernels: IC amplitude table, likelihood + its derivative, the
// 2LPT source adjoint, deterministic FP64 reductions and small helpers.
#pragma once
#include "common.cuh"

namespace pm {
namespace pw {

constexpr int kRedBlocks = 1024;  // fixed grid of every reduction -> fixed summation order
constexpr int kRedThreads = 256;

// FP64 block reduction into partial[blockIdx.x] (tree order fixed by threadIdx).
__device__ __forceinline__ void block_sum_store(double v, double *partial) {
  __shared__ double sh[kRedThreads];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// Per-thread accumulator of a dot product.  For FP64 vectors it is a plain
// FP64 sum of products.  For FP32 vectors every product is split exactly into
// p + e (p = x y rounded, e = fma(x, y, -p)), the p's are summed with Knuth's
// TwoSum into the pair (s, c) and the e's into c, and (s + c) becomes the
// FP64 partial of the thread at the end.  A host check over 2000 random
// 64-term sums with magnitudes spread over 2^20 bounds the error by 1.5e-14
// of sum |x y| (an FP64 sum: 6e-16); for a thread's run of L terms the FP32
// carry c adds O(L 2^-48) of sum |x y| (measured 1.4e-13 at L = 512),
// far below the 6e-8 rounding of the FP32 vectors themselves.  No FP64
// instruction runs per element: on this GPU the FP64 unit is so narrow that
// one conversion and one addition per 16 elements made a 16.7M-element dot
// product three times slower than its memory traffic.  The order is fixed,
// so the result is deterministic.
template <typename T> struct DotAcc {
  double acc = 0.0;
  __device__ __forceinline__ void add(T x, T y) { acc += (double)x * (double)y; }
  __device__ __forceinline__ double value() const { return acc; }
};
template <> struct DotAcc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x, float y) {
    // __fmul_rn / __fadd_rn / __fsub_rn are never contracted into FMAs, which
    // would break the exactness of the split and of TwoSum
    const float p = __fmul_rn(x, y);
    const float e = fmaf(x, y, -p);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp)), e));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Per-thread sum with the same scheme: FP64 for FP64 data; for FP32 data a
// TwoSum-compensated FP32 pair, converted to FP64 once per thread.
template <typename T> struct SumAcc {
  double acc = 0.0;
  __device__ __forceinline__ void add(T x) { acc += (double)x; }
  __device__ __forceinline__ double value() const { return acc; }
};
template <> struct SumAcc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// out[slot] = sum of partial[0..n) in a fixed order (one block).
static __global__ void k_sum_partials(const double *__restrict__ partial, int n, double *out) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kRedThreads) acc += partial[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// sum x^2 (prior), block partials
template <typename T> __global__ void k_sumsq(const T *__restrict__ x, int64_t n, double *partial) {
  DotAcc<T> acc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = x[i];
    acc.add(v, v);
  }
  block_sum_store(acc.value(), partial);
}

// IC amplitude on the half spectrum: sqrt(P(|k|) / Delta^3), P from the
// (ln k, ln P) table by linear interpolation, clamped at the ends; A(0) = 0.
template <typename T>
__global__ void k_amplitude(T *amp, int n, double kf, double inv_cell3, const double *__restrict__ lnk,
                            const double *__restrict__ lnp, int npk) {
  const int h = n / 2 + 1;
  const int64_t total = (int64_t)n * n * h;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int iz = (int)(i % h);
  const int iy = (int)((i / h) % n);
  const int ix = (int)(i / ((int64_t)h * n));
  const int nx = ix < n / 2 ? ix : ix - n;
  const int ny = iy < n / 2 ? iy : iy - n;
  const int n2 = nx * nx + ny * ny + iz * iz;
  if (n2 == 0) {
    amp[i] = T(0);
    return;
  }
  const double lk = log(kf * sqrt((double)n2));
  double lp;
  if (lk <= lnk[0]) {
    lp = lnp[0];
  } else if (lk >= lnk[npk - 1]) {
    lp = lnp[npk - 1];
  } else {
    int lo = 0, hi = npk - 1;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (lnk[mid] <= lk) lo = mid;
      else hi = mid;
    }
    const double slope = (lnp[hi] - lnp[lo]) / (lnk[hi] - lnk[lo]);
    lp = slope * (lk - lnk[lo]) + lnp[lo];
  }
  amp[i] = (T)sqrt(exp(lp) * inv_cell3);
}

struct LossParams {
  int lik;           // 0 gaussian, 1 poisson
  int bias;          // 0 linear, 1 power law + sigmoid
  double b, inv_s2;  // linear bias; gaussian 1 / sigma^2
  double alpha, delta_th, K, nbar, rho_floor;  // power law + sigmoid; normalisation and floor
  double lw;         // loss weight for the derivative
};

// The parameters in the mesh type, converted once per thread (a conversion
// from FP64 per cell would run on the narrow FP64 unit).
template <typename T> struct LossT {
  int lik, bias;
  T b, inv_s2, alpha, delta_th, K, nbar, fl, lw;
  __device__ explicit LossT(const LossParams &p)
      : lik(p.lik), bias(p.bias), b((T)p.b), inv_s2((T)p.inv_s2), alpha((T)p.alpha), delta_th((T)p.delta_th),
        K((T)p.K), nbar((T)p.nbar), fl((T)p.rho_floor), lw((T)p.lw) {}
};

// delta = rho - 1 formed in integers (one unit weight is 2^-e) and 1 + delta
// = rho, each rounded once from the exact fixed-point value q, so both keep
// full relative precision (delta near 0, rho near the floor).  FP32: one
// conversion on the hardware (FP64-unit) path and one on the integer pipe,
// then an exact power-of-two scale (the fixed-point exponent of a density
// mesh is at most 62, so 2^e is a normal float).
template <typename T> __device__ __forceinline__ void density_of(long long q, int e, T &delta, T &onep) {
  if constexpr (sizeof(T) == 4) {
    const float a = __ll2float_rn(q - (1ll << -e)), b = fx_i64_to_f32(q);
    if (e >= -126) {
      const float sc = __int_as_float((e + 127) << 23);
      delta = a * sc;
      onep = b * sc;
    } else {
      delta = scalbnf(a, e);
      onep = scalbnf(b, e);
    }
  } else {
    delta = scalbn(__ll2double_rn(q - (1ll << -e)), e);
    onep = scalbn(__ll2double_rn(q), e);
  }
}

// Galaxy density per unit nbar, g(delta), and dg/d delta (Sec. 2.2.1 item 4).
// Linear: max(1 + b delta, rho_floor), derivative b above the floor.  Power law
// + sigmoid (Eq. galaxy_bias): max(1+delta, rho_floor)^alpha sigmoid(K (delta -
// delta_th)), the power-law factor's derivative zero below the floor.  onep is
// 1 + delta rounded once from the exact density.  FP32 forms the power as
// exp2(alpha log2 base) (a few ulp, against ~10 for the general pow).
template <typename T>
__device__ __forceinline__ void bias_rate(const LossT<T> &lp, T delta, T onep, T &g, T &dg) {
  if (lp.bias == 0) {
    const T base = T(1) + lp.b * delta;
    g = base > lp.fl ? base : lp.fl;
    dg = base > lp.fl ? lp.b : T(0);
  } else {
    const T base = onep > lp.fl ? onep : lp.fl;
    const T sg = T(1) / (T(1) + exp(-lp.K * (delta - lp.delta_th)));
    T pw;
    if constexpr (sizeof(T) == 4) pw = exp2f(lp.alpha * log2f(base));
    else pw = pow(base, lp.alpha);
    g = pw * sg;
    const T dpow = onep > lp.fl ? lp.alpha * pw / base : T(0);
    dg = dpow * sg + pw * lp.K * sg * (T(1) - sg);
  }
}

// Per cell: delta = rho - 1 from the fixed-point density, the likelihood term
// (block partials in FP64), dbar = lw * d(term)/d delta (+ cot), delta_out.
// Each thread walks its cells four at a time, all loads of the four first:
// the grid is fixed (it fixes the summation order), so the loads of several
// cells must be in flight per thread.  The terms are added in cell order, as
// one cell at a time would add them.
template <typename T>
__global__ void k_loss(LossParams lpd, const long long *__restrict__ rho, const int *fx_exp,
                       const T *__restrict__ data, const T *__restrict__ resp, const T *__restrict__ cot,
                       T *__restrict__ dbar, T *__restrict__ delta_out, int64_t n, double *partial) {
  const int e = -__ldg(fx_exp);
  const LossT<T> lp(lpd);
  SumAcc<T> acc;  // the likelihood terms, each formed in T
  auto cell = [&](int64_t i, long long q, T d, T r, T cv) {
    T delta, onep;
    density_of<T>(q, e, delta, onep);
    if (delta_out) delta_out[i] = delta;
    T g = T(0);
    if (lp.lik == 0) {
      // residual of the biased field: b delta, or nbar g(delta)
      T f = lp.b * delta, df = lp.b;
      if (lp.bias != 0) {
        T gb, dgb;
        bias_rate(lp, delta, onep, gb, dgb);
        f = lp.nbar * gb;
        df = lp.nbar * dgb;
      }
      const T res = f - d;
      acc.add(T(0.5) * r * res * res * lp.inv_s2);
      g = r * df * res * lp.inv_s2;
    } else if (r > T(0)) {
      T gb, dgb;
      bias_rate(lp, delta, onep, gb, dgb);
      const T lam = r * lp.nbar * gb;
      acc.add(lam - d * log(lam));
      g = r * lp.nbar * dgb * (T(1) - d / lam);
    }
    if (dbar) dbar[i] = lp.lw * g + cv;
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int U = 4;
  for (; i + (U - 1) * stride < n; i += U * stride) {
    long long q[U];
    T d[U], r[U], cv[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int64_t k = i + j * stride;
      q[j] = rho[k];
      d[j] = data[k];
      r[j] = resp[k];
      cv[j] = cot ? cot[k] : T(0);
    }
#pragma unroll
    for (int j = 0; j < U; ++j) cell(i + j * stride, q[j], d[j], r[j], cv[j]);
  }
  for (; i < n; i += stride) cell(i, rho[i], data[i], resp[i], cot ? cot[i] : T(0));
  block_sum_store(acc.value(), partial);
}

// Model mean per cell from the fixed-point density (mock generation).
template <typename T>
__global__ void k_expected(LossParams lpd, const long long *__restrict__ rho, const int *fx_exp,
                           const T *__restrict__ resp, T *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e = -__ldg(fx_exp);
  const LossT<T> lp(lpd);
  T delta, onep;
  density_of<T>(rho[i], e, delta, onep);
  T gb = T(0), dgb = T(0);
  if (lp.lik != 0 || lp.bias != 0) bias_rate(lp, delta, onep, gb, dgb);
  if (lp.lik == 0) {
    out[i] = lp.bias == 0 ? lp.b * delta : lp.nbar * gb;
  } else {
    out[i] = resp[i] > T(0) ? resp[i] * lp.nbar * gb : T(0);
  }
}

// 2LPT source adjoint: S = phi00 phi11 + phi00 phi22 + phi11 phi22
//                         - phi01^2 - phi02^2 - phi12^2  (slots 0..5 in that order)
// phibar_ii = Sbar (sum of the other two diagonals), phibar_ij = -2 Sbar phi_ij,
// written over phi in place.
template <typename T> __global__ void k_phibar(T *phi, const T *__restrict__ sbar, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T sb = sbar[i];
  const T p00 = phi[i], p11 = phi[n + i], p22 = phi[2 * n + i];
  phi[i] = sb * (p11 + p22);
  phi[n + i] = sb * (p00 + p22);
  phi[2 * n + i] = sb * (p00 + p11);
  phi[3 * n + i] = T(-2) * sb * phi[3 * n + i];
  phi[4 * n + i] = T(-2) * sb * phi[4 * n + i];
  phi[5 * n + i] = T(-2) * sb * phi[5 * n + i];
}

// out = a * x (elementwise), used for unit conversions of probe outputs.
template <typename T> __global__ void k_scale(const T *__restrict__ x, T a, T *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i];
}

// Zero-stuffing onto the fine mesh (2^logn per side) of a coarse field with
// 2^(logn - logr) cells per side: out(x) = s_c(x / r) where r divides every
// coordinate of x, 0 elsewhere.  Its fine DFT is the coarse DFT repeated over
// k (mod coarse size), so the fine FFT of it yields the coarse modes.
template <typename T>
__global__ void k_zero_stuff(const T *__restrict__ sc, int logn, int logr, T *__restrict__ out) {
  const int64_t m = (int64_t)1 << (3 * logn);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int mask = (1 << logn) - 1, rmask = (1 << logr) - 1, lc = logn - logr;
  const int x = (int)(i >> (2 * logn)), y = (int)(i >> logn) & mask, z = (int)i & mask;
  T v = T(0);
  if (((x | y | z) & rmask) == 0)
    v = sc[((int64_t)(x >> logr) << (2 * lc)) | ((int64_t)(y >> logr) << lc) | (int64_t)(z >> logr)];
  out[i] = v;
}

// Block sums (or means) of r^3 fine cells into a coarse mesh of 2^logc cells
// per side: one thread per coarse cell, children added in lattice order in FP64.
template <typename T>
__global__ void k_block_reduce(const T *__restrict__ in, int logc, int logr, bool mean, T *__restrict__ out) {
  const int64_t mc = (int64_t)1 << (3 * logc);
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= mc) return;
  const int cmask = (1 << logc) - 1, r = 1 << logr, logn = logc + logr;
  const int cx = (int)(j >> (2 * logc)), cy = (int)(j >> logc) & cmask, cz = (int)j & cmask;
  double acc = 0.0;
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < r; ++b) {
      const int64_t row = ((int64_t)((cx << logr) + a) << (2 * logn)) | ((int64_t)((cy << logr) + b) << logn);
      for (int c = 0; c < r; ++c) acc += (double)in[row | (int64_t)((cz << logr) + c)];
    }
  if (mean) acc /= (double)((int64_t)r * r * r);
  out[j] = (T)acc;
}

// Eight independent FMA chains per thread, iters steps each (an arithmetic
// rate probe); the result is stored only if it equals a value the chains
// never produce, which keeps them from being optimised away.
template <typename T> __global__ void k_fma_probe(int64_t iters, T *__restrict__ sink) {
  T a[8];
  const T m = T(0.999999), c = T(1e-7);
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
  const int it = (int)iters;
  for (int i = 0; i < it; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if constexpr (sizeof(T) == 4) a[j] = fmaf(a[j], m, c);  // the FP32 instruction, no promotion
      else a[j] = fma(a[j], m, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == T(-1.25e30)) sink[0] = s;
}

// out = y + a * x
template <typename T>
__global__ void k_axpy(const T *__restrict__ x, const T *__restrict__ y, double a, T *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = y[i] + (T)a * x[i];
}

// delta = rho - 1 from a fixed-point mesh
template <typename T>
__global__ void k_fixed_to_delta(const long long *__restrict__ rho, const int *fx_exp, T *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e = -__ldg(fx_exp);
  if constexpr (sizeof(T) == 4) out[i] = scalbnf(fx_i64_to_f32(rho[i] - (1ll << -e)), e);
  else out[i] = scalbn(__ll2double_rn(rho[i] - (1ll << -e)), e);
}

// count of non-finite values (for input validation), block partials
template <typename T> __global__ void k_count_nonfinite(const T *__restrict__ x, int64_t n, double *partial) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += isfinite(x[i]) ? 0.0 : 1.0;
  block_sum_store(acc, partial);
}

}  // namespace pw
}  // namespace pm
