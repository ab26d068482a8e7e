// L-BFGS two-loop recursion on the GPU (Sec. 2.3.1: the projected L-BFGS
// step of MujicΛ).  Vectors in the plan precision, every dot product with
// FP64-quality accumulation (pw::DotAcc) and a fixed reduction order; the
// scalars alpha_i stay on the device so the two loops run without host round
// trips.
#include <cmath>
#include <new>
#include <vector>

#include "../../include/mujica_pm.h"
#include "common.cuh"
#include "pointwise.cuh"

namespace pm {
namespace lb {

using pw::kRedBlocks;
using pw::kRedThreads;

// The vector kernels below walk their elements in a grid-stride loop and
// issue the loads of four strides before using them (the kernels are short
// and otherwise wait on one load at a time); each thread still visits its
// elements in increasing order, so every sum is accumulated in the same order
// as a plain grid-stride loop.
constexpr int kU = 4;

// s = x_new - x_prev, y = g_new - g_prev into the history slot; x_prev, g_prev
// updated; block partials of s.y, s.s, y.y.
template <typename T>
__global__ void k_pair(const T *__restrict__ xn, const T *__restrict__ gn, T *xp, T *gp, T *__restrict__ sv,
                       T *__restrict__ yv, int64_t n, double *partial) {
  pw::DotAcc<T> a, b, c;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kU - 1) * st < n; i += kU * st) {
    T x1[kU], g1[kU], x0[kU], g0[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      x1[u] = xn[i + u * st];
      g1[u] = gn[i + u * st];
      x0[u] = xp[i + u * st];
      g0[u] = gp[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const T s = x1[u] - x0[u], y = g1[u] - g0[u];
      sv[i + u * st] = s;
      yv[i + u * st] = y;
      xp[i + u * st] = x1[u];
      gp[i + u * st] = g1[u];
      a.add(s, y);
      b.add(s, s);
      c.add(y, y);
    }
  }
  for (; i < n; i += st) {
    const T s = xn[i] - xp[i];
    const T y = gn[i] - gp[i];
    sv[i] = s;
    yv[i] = y;
    xp[i] = xn[i];
    gp[i] = gn[i];
    a.add(s, y);
    b.add(s, s);
    c.add(y, y);
  }
  pw::block_sum_store(a.value(), partial);
  __syncthreads();
  pw::block_sum_store(b.value(), partial + kRedBlocks);
  __syncthreads();
  pw::block_sum_store(c.value(), partial + 2 * kRedBlocks);
}

template <typename T> __global__ void k_dot(const T *__restrict__ a, const T *__restrict__ b, int64_t n, double *partial) {
  pw::DotAcc<T> acc;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kU - 1) * st < n; i += kU * st) {
    T av[kU], bv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      av[u] = a[i + u * st];
      bv[u] = b[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) acc.add(av[u], bv[u]);
  }
  for (; i < n; i += st) acc.add(a[i], b[i]);
  pw::block_sum_store(acc.value(), partial);
}

// coefficient on the device: c = c0 * (*p1) + c1 * (*p2) (pointers may be null)
struct Coef {
  double c0, c1;
  const double *p1, *p2;
  __device__ double eval() const { return (p1 ? c0 * *p1 : c0) + (p2 ? c1 * *p2 : 0.0); }
};

// v += c * x, then (if dotv) block partials of dotv . v
template <typename T>
__global__ void k_axpy_dot(T *v, const T *__restrict__ x, Coef cf, int64_t n, const T *__restrict__ dotv,
                           double *partial) {
  const T c = (T)cf.eval();
  pw::DotAcc<T> acc;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kU - 1) * st < n; i += kU * st) {
    T vv[kU], xv[kU], dv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      vv[u] = v[i + u * st];
      xv[u] = x[i + u * st];
      dv[u] = dotv ? dotv[i + u * st] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const T nv = vv[u] + c * xv[u];
      v[i + u * st] = nv;
      if (dotv) acc.add(dv[u], nv);
    }
  }
  for (; i < n; i += st) {
    const T nv = v[i] + c * x[i];
    v[i] = nv;
    if (dotv) acc.add(dotv[i], nv);
  }
  if (dotv) pw::block_sum_store(acc.value(), partial);
}

template <typename T> __global__ void k_scale_copy(const T *__restrict__ x, double a, T *__restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)a * x[i];
}

__global__ void k_mul(double *dst, const double *src, double f) { *dst = f * *src; }

}  // namespace lb
}  // namespace pm

// The history holds m + 1 physical (s, y) slots: phys[0..m) maps the ring
// positions to slots and `spare` is the free one.  A new pair is written into
// the spare slot and enters the ring only when it passes the curvature test
// (the slot of the pair it displaces becomes the spare), so a rejected pair
// never overwrites a stored one.
struct lbfgs_state {
  int64_t n = 0;
  int m = 0;
  int prec = 0;
  size_t es = 4;
  char *ws = nullptr;
  void *S = nullptr, *Y = nullptr, *xprev = nullptr, *gprev = nullptr;
  double *partial = nullptr, *dres = nullptr;  // dres: alpha[m + 1], dots[m + 8]
  std::vector<double> rho;                     // per physical slot
  std::vector<int> phys;                       // ring position -> physical slot
  int spare = 0;
  int count = 0, head = 0;
  bool has_prev = false;
  double gamma = 1.0;
};

namespace {

size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

size_t lb_bytes(int64_t n, int m, size_t es) {
  return 2 * (size_t)(m + 1) * al(n * es) + 2 * al(n * es) + al(3 * pm::pw::kRedBlocks * 8) + al((2 * m + 16) * 8);
}

template <typename T> void *vec(lbfgs_state *s, void *base, int i) {
  return static_cast<char *>(base) + (size_t)i * al(s->n * sizeof(T));
}

double sum_to_host(double *partial, double *slot, cudaStream_t st, cudaError_t &err) {
  ::pm::note_launch();
  pm::pw::k_sum_partials<<<1, pm::pw::kRedThreads, 0, st>>>(partial, pm::pw::kRedBlocks, slot);
  double h = 0;
  err = cudaMemcpyAsync(&h, slot, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  return h;
}

template <typename T>
pm_status step_impl(lbfgs_state *s, const T *xn, const T *gn, T *d, double *gdotd, double *dnorm, int *pushed,
                    cudaStream_t st) {
  using namespace pm::lb;
  const int64_t n = s->n;
  const int nb = kRedBlocks, nt = kRedThreads;
  cudaError_t err = cudaSuccess;
  double *alpha = s->dres;            // alpha per physical slot, m + 1
  double *dots = s->dres + s->m + 1;  // scratch scalars
  int did_push = 0;
  if (s->has_prev) {
    const int slot = s->spare;
    T *sv = static_cast<T *>(vec<T>(s, s->S, slot));
    T *yv = static_cast<T *>(vec<T>(s, s->Y, slot));
    ::pm::note_launch();
    k_pair<T><<<nb, nt, 0, st>>>(xn, gn, static_cast<T *>(s->xprev), static_cast<T *>(s->gprev), sv, yv, n, s->partial);
    ::pm::note_launch();
    pm::pw::k_sum_partials<<<1, nt, 0, st>>>(s->partial, nb, dots + 0);
    ::pm::note_launch();
    pm::pw::k_sum_partials<<<1, nt, 0, st>>>(s->partial + nb, nb, dots + 1);
    ::pm::note_launch();
    pm::pw::k_sum_partials<<<1, nt, 0, st>>>(s->partial + 2 * nb, nb, dots + 2);
    double h[3];
    PM_CUDA_TRY(cudaMemcpyAsync(h, dots, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    const double sy = h[0], ss = h[1], yy = h[2];
    if (std::isfinite(sy) && sy > 1e-10 * std::sqrt(ss) * std::sqrt(yy) && yy > 0) {
      s->rho[slot] = 1.0 / sy;
      s->gamma = sy / yy;
      // ring position `head` receives the new pair; the slot it held (free,
      // or the oldest pair when the ring is full) becomes the spare
      s->spare = s->phys[s->head];
      s->phys[s->head] = slot;
      s->head = (s->head + 1) % s->m;
      if (s->count < s->m) ++s->count;
      did_push = 1;
    }
  } else {
    PM_CUDA_TRY(cudaMemcpyAsync(s->xprev, xn, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    PM_CUDA_TRY(cudaMemcpyAsync(s->gprev, gn, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    s->has_prev = true;
  }
  // two-loop recursion, q in d
  const int k = s->count;
  // physical slot of the pair of the given age (0 = newest)
  auto idx = [&](int age) { return s->phys[((s->head - 1 - age) % s->m + s->m) % s->m]; };
  PM_CUDA_TRY(cudaMemcpyAsync(d, gn, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  if (k > 0) {
    // alpha_newest = rho * s_newest . q
    ::pm::note_launch();
    k_dot<T><<<nb, nt, 0, st>>>(static_cast<const T *>(vec<T>(s, s->S, idx(0))), d, n, s->partial);
    ::pm::note_launch();
    pm::pw::k_sum_partials<<<1, nt, 0, st>>>(s->partial, nb, dots + 3);
    ::pm::note_launch();
    k_mul<<<1, 1, 0, st>>>(alpha + idx(0), dots + 3, s->rho[idx(0)]);
    for (int a = 0; a < k; ++a) {
      const int i = idx(a);
      const T *next_s = a + 1 < k ? static_cast<const T *>(vec<T>(s, s->S, idx(a + 1))) : nullptr;
      Coef cf{-1.0, 0.0, alpha + i, nullptr};
      ::pm::note_launch();
      k_axpy_dot<T><<<nb, nt, 0, st>>>(d, static_cast<const T *>(vec<T>(s, s->Y, i)), cf, n, next_s, s->partial);
      if (next_s) {
        ::pm::note_launch();
        pm::pw::k_sum_partials<<<1, nt, 0, st>>>(s->partial, nb, dots + 3);
        ::pm::note_launch();
        k_mul<<<1, 1, 0, st>>>(alpha + idx(a + 1), dots + 3, s->rho[idx(a + 1)]);
      }
    }
  }
  const double gam = k > 0 ? s->gamma : 1.0;
  if (gam != 1.0) {
    ::pm::note_launch();
    k_scale_copy<T><<<nb, nt, 0, st>>>(d, gam, d, n);
  }
  if (k > 0) {  // y_oldest . r
    ::pm::note_launch();
    k_dot<T><<<nb, nt, 0, st>>>(static_cast<const T *>(vec<T>(s, s->Y, idx(k - 1))), d, n, s->partial);
    ::pm::note_launch();
    pm::pw::k_sum_partials<<<1, nt, 0, st>>>(s->partial, nb, dots + 4);
  }
  for (int a = k - 1; a >= 0; --a) {  // oldest -> newest
    const int i = idx(a);
    // r += (alpha_i - rho_i y_i.r) s_i, fused with y_next . r of the next pair
    const T *next_y = a > 0 ? static_cast<const T *>(vec<T>(s, s->Y, idx(a - 1))) : nullptr;
    Coef cf{1.0, -s->rho[i], alpha + i, dots + 4};
    ::pm::note_launch();
    k_axpy_dot<T><<<nb, nt, 0, st>>>(d, static_cast<const T *>(vec<T>(s, s->S, i)), cf, n, next_y, s->partial);
    if (next_y) {
      ::pm::note_launch();
      pm::pw::k_sum_partials<<<1, nt, 0, st>>>(s->partial, nb, dots + 4);
    }
  }
  // d = -r
  ::pm::note_launch();
  k_scale_copy<T><<<nb, nt, 0, st>>>(d, -1.0, d, n);
  PM_LAUNCH_CHECK();
  ::pm::note_launch();
  k_dot<T><<<nb, nt, 0, st>>>(gn, d, n, s->partial);
  double gd = sum_to_host(s->partial, dots + 5, st, err);
  if (err != cudaSuccess) {
    pm::set_error(cudaGetErrorString(err));
    return PM_ERR_CUDA;
  }
  if (!(gd < 0.0)) {  // not a descent direction: drop the pairs, d = -g
    s->count = 0;
    s->head = 0;
    ::pm::note_launch();
    k_scale_copy<T><<<nb, nt, 0, st>>>(gn, -1.0, d, n);
    ::pm::note_launch();
    k_dot<T><<<nb, nt, 0, st>>>(gn, d, n, s->partial);
    gd = sum_to_host(s->partial, dots + 5, st, err);
  }
  ::pm::note_launch();
  k_dot<T><<<nb, nt, 0, st>>>(d, d, n, s->partial);
  const double dd = sum_to_host(s->partial, dots + 6, st, err);
  if (err != cudaSuccess) {
    pm::set_error(cudaGetErrorString(err));
    return PM_ERR_CUDA;
  }
  PM_LAUNCH_CHECK();
  if (gdotd) *gdotd = gd;
  if (dnorm) *dnorm = std::sqrt(dd);
  if (pushed) *pushed = did_push;
  if (!std::isfinite(gd) || !std::isfinite(dd)) {
    pm::set_error("L-BFGS direction is not finite");
    return PM_ERR_NONFINITE;
  }
  return PM_OK;
}

}  // namespace

extern "C" {

pm_status lbfgs_workspace_bytes(int64_t n_elems, int32_t m, int32_t precision, size_t *bytes) {
  if (n_elems < 1 || m < 1 || m > 64 || (precision != PM_PREC_F32 && precision != PM_PREC_F64) || !bytes) {
    pm::set_error("invalid L-BFGS size / memory / precision");
    return PM_ERR_INVALID_ARG;
  }
  *bytes = lb_bytes(n_elems, m, precision == PM_PREC_F64 ? 8 : 4);
  return PM_OK;
}

pm_status lbfgs_create(int64_t n_elems, int32_t m, int32_t precision, void *workspace, size_t bytes,
                       lbfgs_state **out) {
  size_t need = 0;
  const pm_status s = lbfgs_workspace_bytes(n_elems, m, precision, &need);
  if (s) return s;
  if (!workspace || !out) {
    pm::set_error("NULL workspace / out");
    return PM_ERR_INVALID_ARG;
  }
  if (bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    pm::set_error("L-BFGS workspace too small or not 256-byte aligned");
    return PM_ERR_WORKSPACE;
  }
  lbfgs_state *st = new (std::nothrow) lbfgs_state;
  if (!st) return PM_ERR_INVALID_ARG;
  st->n = n_elems;
  st->m = m;
  st->prec = precision;
  st->es = precision == PM_PREC_F64 ? 8 : 4;
  st->rho.assign(m + 1, 0.0);
  st->phys.resize(m);
  for (int i = 0; i < m; ++i) st->phys[i] = i;
  st->spare = m;
  char *p = static_cast<char *>(workspace);
  const size_t v = al(n_elems * st->es);
  st->S = p;
  p += (m + 1) * v;
  st->Y = p;
  p += (m + 1) * v;
  st->xprev = p;
  p += v;
  st->gprev = p;
  p += v;
  st->partial = reinterpret_cast<double *>(p);
  p += al(3 * pm::pw::kRedBlocks * 8);
  st->dres = reinterpret_cast<double *>(p);
  *out = st;
  return PM_OK;
}

pm_status lbfgs_destroy(lbfgs_state *st) {
  delete st;
  return PM_OK;
}

pm_status lbfgs_reset(lbfgs_state *st) {
  if (!st) {
    pm::set_error("state is NULL");
    return PM_ERR_INVALID_ARG;
  }
  st->count = 0;
  st->head = 0;
  st->has_prev = false;
  st->gamma = 1.0;
  return PM_OK;
}

pm_status lbfgs_step(lbfgs_state *st, const void *x_new, const void *g_new, void *d_out, double *gdotd_out,
                     double *dnorm_out, int32_t *pushed_out, pm_stream_t stream) {
  if (!st || !x_new || !g_new || !d_out) {
    pm::set_error("NULL state / x_new / g_new / d_out");
    return PM_ERR_INVALID_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (st->prec == PM_PREC_F32)
    return step_impl<float>(st, (const float *)x_new, (const float *)g_new, (float *)d_out, gdotd_out, dnorm_out,
                            pushed_out, s);
  return step_impl<double>(st, (const double *)x_new, (const double *)g_new, (double *)d_out, gdotd_out, dnorm_out,
                           pushed_out, s);
}

pm_status pm_axpy(int64_t n, int32_t precision, double alpha, const void *x, const void *y, void *out,
                  pm_stream_t stream) {
  if (n < 0 || !x || !y || !out || (precision != PM_PREC_F32 && precision != PM_PREC_F64)) {
    pm::set_error("invalid axpy arguments");
    return PM_ERR_INVALID_ARG;
  }
  if (n == 0) return PM_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ::pm::note_launch();
  if (precision == PM_PREC_F32)
    pm::pw::k_axpy<float><<<pm::grid_for(n, 256), 256, 0, s>>>((const float *)x, (const float *)y, alpha,
                                                               (float *)out, n);
  else
    pm::pw::k_axpy<double><<<pm::grid_for(n, 256), 256, 0, s>>>((const double *)x, (const double *)y, alpha,
                                                                (double *)out, n);
  PM_LAUNCH_CHECK();
  return PM_OK;
}

}  // extern "C"
