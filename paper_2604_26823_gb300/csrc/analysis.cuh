// Analysis of reconstructed fields (Sec. 3.2, the correlation coefficient
// r_c(k); Sec. 3.3, the T-web): binned auto / cross power spectra, the
// per-cell eigen-decomposition of the smoothed deformation tensor with its
// classification, eigenvector cosine similarity and the confusion matrix of
// two classifications.  Spectral steps reuse the pencil FFT passes; these
// kernels are the parts that differ.
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace pm {
namespace an {

// x pass that ends in the spectrum: forward x FFT of one or two spectra
// (already transformed along z and y), then each mode (nx, ny, nz) of the
// half spectrum adds w |A|^2, w |B|^2, w Re(A conj B) and w to its |k| bin,
// floor((kf |n| - k_min) / dk), w = 1 on the nz = 0 and Nyquist planes and 2
// elsewhere (the conjugate partner).  Shared-memory bins per CTA, then one
// global FP64 atomic per bin (sums exact up to FP64 rounding order).
template <typename T, int N, int B, int NT>
__global__ void __launch_bounds__(NT) k_x_power(const cx<T> *__restrict__ a, const cx<T> *__restrict__ b,
                                                const cx<T> *__restrict__ tw, double kf, double kmin, double dk,
                                                int nbins, double *__restrict__ bins) {
  using C = cx<T>;
  constexpr int H = N / 2 + 1;
  static_assert(N * B % NT == 0 && NT % B == 0, "tile must split evenly over threads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *ta = reinterpret_cast<C *>(smem_raw);
  C *tb = ta + N * B;
  double *sb = reinterpret_cast<double *>(tb + N * B);
  const int col0 = blockIdx.x * B;
  const int64_t astride = (int64_t)N * H;
  for (int i = threadIdx.x; i < 4 * nbins; i += NT) sb[i] = 0.0;
  const C *sa = a + col0;
  fft::gather_tile<N * B / NT, NT, C>([&](int e) { return sa[(e / B) * astride + e % B]; },
                                      [&](int e, C v) { ta[e] = v; });
  if (b) {
    const C *sbb = b + col0;
    fft::gather_tile<N * B / NT, NT, C>([&](int e) { return sbb[(e / B) * astride + e % B]; },
                                        [&](int e, C v) { tb[e] = v; });
  }
  __syncthreads();
  fft::smem_fft<C, N, B, B, NT, -1>(ta, tw, 1);
  if (b) fft::smem_fft<C, N, B, B, NT, -1>(tb, tw, 1);
  const int c = threadIdx.x % B, colg = col0 + c;
  const int iy = colg / H, iz = colg % H;
  const int ny = iy < N / 2 ? iy : iy - N;
  const double w = (iz == 0 || iz == N / 2) ? 1.0 : 2.0;
  for (int ix = threadIdx.x / B; ix < N; ix += NT / B) {
    const int nx = ix < N / 2 ? ix : ix - N;
    const int n2 = nx * nx + ny * ny + iz * iz;
    const double fb = floor((kf * sqrt((double)n2) - kmin) / dk);
    if (fb >= 0.0 && fb < (double)nbins) {
      const int bi = (int)fb;
      const C va = ta[ix * B + c];
      atomicAdd(&sb[bi], w * ((double)va.x * va.x + (double)va.y * va.y));
      if (b) {
        const C vb = tb[ix * B + c];
        atomicAdd(&sb[nbins + bi], w * ((double)vb.x * vb.x + (double)vb.y * vb.y));
        atomicAdd(&sb[2 * nbins + bi], w * ((double)va.x * vb.x + (double)va.y * vb.y));
      }
      atomicAdd(&sb[3 * nbins + bi], w);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * nbins; i += NT)
    if (sb[i] != 0.0) atomicAdd(&bins[i], sb[i]);
}

// ---- symmetric 3 x 3 eigen-decomposition (FP64) ----------------------------
__device__ __forceinline__ void cross3(const double *u, const double *v, double *o) {
  o[0] = u[1] * v[2] - u[2] * v[1];
  o[1] = u[2] * v[0] - u[0] * v[2];
  o[2] = u[0] * v[1] - u[1] * v[0];
}
__device__ __forceinline__ double dot3(const double *u, const double *v) {
  return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}

// Unit vector spanning the null space of A - lam I (a symmetric, entries
// 00 11 22 01 02 12) from the largest cross product of two of its rows;
// false when every cross product vanishes.
__device__ __forceinline__ bool null_vector(const double *a, double lam, double *v) {
  const double r0[3] = {a[0] - lam, a[3], a[4]};
  const double r1[3] = {a[3], a[1] - lam, a[5]};
  const double r2[3] = {a[4], a[5], a[2] - lam};
  double c[3][3];
  cross3(r0, r1, c[0]);
  cross3(r0, r2, c[1]);
  cross3(r1, r2, c[2]);
  int best = 0;
  double bn = dot3(c[0], c[0]);
  for (int i = 1; i < 3; ++i) {
    const double nn = dot3(c[i], c[i]);
    if (nn > bn) {
      bn = nn;
      best = i;
    }
  }
  if (!(bn > 0.0)) return false;
  const double inv = 1.0 / sqrt(bn);
  for (int k = 0; k < 3; ++k) v[k] = c[best][k] * inv;
  return true;
}

// Eigen-decomposition, eigenvalues lam[0] <= lam[1] <= lam[2] with unit
// eigenvectors vec[i][*]: the trigonometric solution of the characteristic
// cubic (A = q I + p C, tr C = 0, det C = 2 cos 3phi) locates the eigenvalues;
// the better separated of the two extreme ones is polished by two Newton steps
// on det(A - lam I) and its eigenvector taken as the null vector of
// A - lam I; the other two come from the closed-form 2 x 2 problem of A in
// that vector's orthogonal complement (rotation angle
// theta = atan2(2 r, p - s) / 2), which stays accurate when they coincide.
__device__ __forceinline__ void sym3_eigen(const double *a, double *lam, double (*vec)[3]) {
  const double q = (a[0] + a[1] + a[2]) / 3.0;
  const double b0 = a[0] - q, b1 = a[1] - q, b2 = a[2] - q;
  const double p2 = b0 * b0 + b1 * b1 + b2 * b2 + 2.0 * (a[3] * a[3] + a[4] * a[4] + a[5] * a[5]);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) vec[i][k] = i == k ? 1.0 : 0.0;
  if (!(p2 > 0.0)) {
    lam[0] = lam[1] = lam[2] = q;
    return;
  }
  const double p = sqrt(p2 / 6.0);
  const double det = b0 * (b1 * b2 - a[5] * a[5]) - a[3] * (a[3] * b2 - a[5] * a[4]) + a[4] * (a[3] * a[5] - b1 * a[4]);
  double r = det / (2.0 * p * p * p);
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  const double two_pi_3 = 2.0943951023931954923;  // 2 pi / 3
  lam[2] = q + 2.0 * p * cos(phi);
  lam[0] = q + 2.0 * p * cos(phi + two_pi_3);
  lam[1] = 3.0 * q - lam[0] - lam[2];
  const int first = (lam[1] - lam[0]) >= (lam[2] - lam[1]) ? 0 : 2;
  double lf = lam[first];
  for (int it = 0; it < 2; ++it) {
    const double d0 = a[0] - lf, d1 = a[1] - lf, d2 = a[2] - lf;
    const double c = d0 * (d1 * d2 - a[5] * a[5]) - a[3] * (a[3] * d2 - a[5] * a[4]) + a[4] * (a[3] * a[5] - d1 * a[4]);
    const double dc = -((d1 * d2 - a[5] * a[5]) + (d0 * d2 - a[4] * a[4]) + (d0 * d1 - a[3] * a[3]));
    if (dc != 0.0) lf -= c / dc;
  }
  double v0[3];
  if (!null_vector(a, lf, v0)) return;
  // orthonormal basis (u, w) of the complement of v0
  const double ax[3] = {fabs(v0[0]) <= fabs(v0[1]) && fabs(v0[0]) <= fabs(v0[2]) ? 1.0 : 0.0,
                        fabs(v0[1]) < fabs(v0[0]) && fabs(v0[1]) <= fabs(v0[2]) ? 1.0 : 0.0,
                        fabs(v0[2]) < fabs(v0[0]) && fabs(v0[2]) < fabs(v0[1]) ? 1.0 : 0.0};
  double u[3], w[3];
  cross3(v0, ax, u);
  const double un = 1.0 / sqrt(dot3(u, u));
  for (int k = 0; k < 3; ++k) u[k] *= un;
  cross3(v0, u, w);
  auto av = [&](const double *x, double *y) {
    y[0] = a[0] * x[0] + a[3] * x[1] + a[4] * x[2];
    y[1] = a[3] * x[0] + a[1] * x[1] + a[5] * x[2];
    y[2] = a[4] * x[0] + a[5] * x[1] + a[2] * x[2];
  };
  double t0[3], tu[3], tw[3];
  av(v0, t0);
  av(u, tu);
  av(w, tw);
  const double pu = dot3(u, tu), ru = dot3(u, tw), su = dot3(w, tw);
  const double th = 0.5 * atan2(2.0 * ru, pu - su);
  const double ct = cos(th), st = sin(th);
  const double h = hypot(0.5 * (pu - su), ru), mean = 0.5 * (pu + su);
  double eb[3], es[3];
  for (int k = 0; k < 3; ++k) {
    eb[k] = ct * u[k] + st * w[k];   // eigenvalue mean + h
    es[k] = -st * u[k] + ct * w[k];  // eigenvalue mean - h
  }
  lam[first] = dot3(v0, t0);
  const int lo = first == 0 ? 1 : 0;  // the pair takes the two other slots in order
  lam[lo] = mean - h;
  lam[lo + 1] = mean + h;
  for (int k = 0; k < 3; ++k) {
    vec[first][k] = v0[k];
    vec[lo][k] = es[k];
    vec[lo + 1][k] = eb[k];
  }
}

// Per cell: eigen-decomposition of psi (6 planar fields 00 11 22 01 02 12),
// label = number of eigenvalues above lambda_th; eigenvalues [3][n] and
// eigenvectors [3 (which) x 3 (component)][n] when requested.
template <typename T>
__global__ void k_tweb_eigen(const T *__restrict__ psi, int64_t n, double lambda_th, int *__restrict__ labels,
                             T *__restrict__ eig, T *__restrict__ evec) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double a[6];
  for (int i = 0; i < 6; ++i) a[i] = (double)psi[i * n + c];
  double lam[3], vec[3][3];
  sym3_eigen(a, lam, vec);
  labels[c] = (lam[0] > lambda_th) + (lam[1] > lambda_th) + (lam[2] > lambda_th);
  if (eig)
    for (int i = 0; i < 3; ++i) eig[i * n + c] = (T)lam[i];
  if (evec)
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) evec[(3 * i + k) * n + c] = (T)vec[i][k];
}

// |cos theta_i| = |e_i,a . e_i,b| per cell, eigenvector layout [3 x 3][n].
template <typename T>
__global__ void k_eig_cosines(const T *__restrict__ va, const T *__restrict__ vb, int64_t n, T *__restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < 3; ++i) {
    T s = T(0);
    for (int k = 0; k < 3; ++k) s += va[(3 * i + k) * n + c] * vb[(3 * i + k) * n + c];
    out[i * n + c] = fabs(s);
  }
}

// 4 x 4 counts of (truth label, reconstructed label) over the cells with
// R > 0 (all cells when R is null); labels outside 0..3 are not counted.
template <typename T>
__global__ void k_confusion(const int *__restrict__ lt, const int *__restrict__ lr, const T *__restrict__ R,
                            int64_t n, unsigned long long *__restrict__ out) {
  __shared__ unsigned long long sh[16];
  if (threadIdx.x < 16) sh[threadIdx.x] = 0ull;
  __syncthreads();
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const int t = lt[c], r = lr[c];
    if ((R == nullptr || R[c] > T(0)) && t >= 0 && t < 4 && r >= 0 && r < 4) atomicAdd(&sh[4 * t + r], 1ull);
  }
  __syncthreads();
  if (threadIdx.x < 16 && sh[threadIdx.x]) atomicAdd(&out[threadIdx.x], sh[threadIdx.x]);
}

}  // namespace an
}  // namespace pm
