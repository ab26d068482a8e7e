// Per-particle kernels of the PM model: cloud-in-cell deposition (paint),
// interpolation (readout), the leapfrog kick / drift, the redshift-space
// shift, and the adjoint gathers with CIC weight derivatives.
//
// Particle p = (i*N + j)*N + l carries its displacement d from the Lagrangian
// node (i, j, l) in cell units (FP32 or FP64).  The cell of a particle is
// formed in integers, c = (node + floor(d)) mod N, with the FP offset
// f = d - floor(d) in [0, 1), so large boxes keep sub-cell accuracy.
// CIC: node c + o (o in {0,1}^3) gets prod_a (o_a ? f_a : 1 - f_a); the weight
// derivative is prod over the other axes times (o_a ? +1 : -1).
// Sec. 2.2.1 item 2 (PM steps), item 3 (RSD), Sec. 2.2.2 (CiC binning).
#pragma once
#include "common.cuh"

namespace pm {
namespace part {

struct Lattice {
  int logn;
  int mask;
  __device__ __forceinline__ void node(int64_t p, int &i, int &j, int &l) const {
    i = (int)(p >> (2 * logn));
    j = (int)(p >> logn) & mask;
    l = (int)p & mask;
  }
};

template <typename T> struct Cell {
  int c[3];   // base node (periodic)
  T f[3];     // fractional offset in [0, 1)
};

template <typename T>
__device__ __forceinline__ Cell<T> locate(const Lattice &L, int64_t p, T dx, T dy, T dz) {
  int nd[3];
  L.node(p, nd[0], nd[1], nd[2]);
  const T d[3] = {dx, dy, dz};
  Cell<T> c;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T fl = floor(d[a]);
    c.f[a] = d[a] - fl;
    c.c[a] = (nd[a] + (int)fl) & L.mask;
  }
  return c;
}

__device__ __forceinline__ int64_t mesh_index(const Lattice &L, int x, int y, int z) {
  return ((((int64_t)x) << L.logn | y) << L.logn) | z;
}

// 2^e for the unit-weight deposit scale (e = 61 - log2(np) - 1 lies in
// [33, 48] for 512^3 .. 16^3 particles, inside the float exponent range);
// built from the exponent bits, since a double ldexp would issue on the
// narrow FP64 unit.
template <typename T> __device__ __forceinline__ T pow2(int e) {
  if constexpr (sizeof(T) == 4) return __int_as_float((e + 127) << 23);
  else return ldexp(1.0, e);
}

// A deposit rint(w) of a weight already scaled by 2^E, as an integer: FP32
// through one FP32 -> int32 conversion and a shift (exact, fx_f32_to_i64_split),
// FP64 through the hardware conversion.
template <typename T> __device__ __forceinline__ long long fx_round(T w) {
  if constexpr (sizeof(T) == 4) return fx_f32_to_i64_split(w);
  else return __double2ll_rn(w);
}

// F = sum_c W(u - c) Phi(c) over a 4-component mesh (x, y, z used).
template <typename T>
__device__ __forceinline__ void readout3(const Lattice &L, const V4<T> *__restrict__ phi, const Cell<T> &c,
                                         T &fx, T &fy, T &fz) {
  const int x1 = (c.c[0] + 1) & L.mask, y1 = (c.c[1] + 1) & L.mask, z1 = (c.c[2] + 1) & L.mask;
  const T wx[2] = {T(1) - c.f[0], c.f[0]};
  const T wy[2] = {T(1) - c.f[1], c.f[1]};
  const T wz[2] = {T(1) - c.f[2], c.f[2]};
  const int xs[2] = {c.c[0], x1}, ys[2] = {c.c[1], y1}, zs[2] = {c.c[2], z1};
  fx = fy = fz = T(0);
#pragma unroll
  for (int ox = 0; ox < 2; ++ox)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
      const T wxy = wx[ox] * wy[oy];
#pragma unroll
      for (int oz = 0; oz < 2; ++oz) {
        const V4<T> m = phi[mesh_index(L, xs[ox], ys[oy], zs[oz])];
        const T w = wxy * wz[oz];
        fx += w * m.x;
        fy += w * m.y;
        fz += w * m.z;
      }
    }
}

// Gradient wrt u of sum_c W(u - c) [a . Phi(c) + s(c)] (adjoint gather);
// phi may be null (then only the scalar mesh s contributes).
template <typename T>
__device__ __forceinline__ void grad_gather(const Lattice &L, const V4<T> *__restrict__ phi,
                                            const T *__restrict__ smesh, const Cell<T> &c, T ax, T ay,
                                            T az, T &gx, T &gy, T &gz) {
  const int x1 = (c.c[0] + 1) & L.mask, y1 = (c.c[1] + 1) & L.mask, z1 = (c.c[2] + 1) & L.mask;
  const T wx[2] = {T(1) - c.f[0], c.f[0]};
  const T wy[2] = {T(1) - c.f[1], c.f[1]};
  const T wz[2] = {T(1) - c.f[2], c.f[2]};
  const T sg[2] = {T(-1), T(1)};
  const int xs[2] = {c.c[0], x1}, ys[2] = {c.c[1], y1}, zs[2] = {c.c[2], z1};
  gx = gy = gz = T(0);
#pragma unroll
  for (int ox = 0; ox < 2; ++ox)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int oz = 0; oz < 2; ++oz) {
        const int64_t idx = mesh_index(L, xs[ox], ys[oy], zs[oz]);
        T val = smesh ? smesh[idx] : T(0);
        if (phi) {
          const V4<T> m = phi[idx];
          val += ax * m.x + ay * m.y + az * m.z;
        }
        gx += sg[ox] * wy[oy] * wz[oz] * val;
        gy += wx[ox] * sg[oy] * wz[oz] * val;
        gz += wx[ox] * wy[oy] * sg[oz] * val;
      }
}

template <typename T> __device__ __forceinline__ void atomic_max_abs(unsigned long long *slot, T v) {
  // |v| of a float / double orders like its bit pattern (non-negative)
  if constexpr (sizeof(T) == 4) {
    atomicMax(reinterpret_cast<unsigned int *>(slot), __float_as_uint(fabsf(v)));
  } else {
    atomicMax(slot, (unsigned long long)__double_as_longlong(fabs(v)));
  }
}

template <typename T> __device__ __forceinline__ T read_max_abs(const unsigned long long *slot) {
  if constexpr (sizeof(T) == 4) return __uint_as_float(*reinterpret_cast<const unsigned int *>(slot));
  else return __longlong_as_double((long long)*slot);
}

// Running max of |v| over a launch.  One atomic per warp on a single word
// serialises at the L2 (524k same-address atomics at 256^3 cost ~0.25 ms), so
// each block reduces to one value, which goes to one of kMaxSlots words
// (chosen by block index, so the atomics spread over the L2); k_fold_max then
// folds the words into the single slot the next paint reads.  Every thread of
// the block must call this (it synchronises the block).
constexpr int kMaxSlots = 256;
template <typename T> __device__ __forceinline__ void block_max_to_slots(T mx, unsigned long long *slots) {
  __shared__ T wmax[32];
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) wmax[w] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    T m = wmax[0];
    for (int i = 1; i < nw; ++i) m = max(m, wmax[i]);
    atomic_max_abs<T>(slots + (blockIdx.x & (kMaxSlots - 1)), m);
  }
}

// maxslot = max over the kMaxSlots words; the words are cleared for the next
// launch.  One block of kMaxSlots threads.
template <typename T> __global__ void k_fold_max(unsigned long long *slots, unsigned long long *maxslot) {
  __shared__ T sh[kMaxSlots];
  sh[threadIdx.x] = read_max_abs<T>(slots + threadIdx.x);
  slots[threadIdx.x] = 0ull;
  __syncthreads();
  for (int st = kMaxSlots / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] = max(sh[threadIdx.x], sh[threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *maxslot = 0ull;
    atomic_max_abs<T>(maxslot, sh[0]);
  }
}

// Exponent E with 2^E * maxabs * n_particles < 2^61 (no overflow of the
// int64 accumulators); deposits are rint(w * 2^E).
__device__ __forceinline__ int fixed_exponent(double maxabs, int log2_particles) {
  if (!(maxabs > 0.0)) return 0;
  int e;
  frexp(maxabs, &e);  // maxabs < 2^e
  return 61 - log2_particles - e;
}
// The same from the running max held as the bits of a non-negative float
// (read_max_abs<float>), without FP64 arithmetic for normal numbers.
__device__ __forceinline__ int fixed_exponent_f32(unsigned bits, int log2_particles) {
  const int be = (int)(bits >> 23);
  if (bits == 0u || be == 0) return fixed_exponent((double)__uint_as_float(bits), log2_particles);
  return 61 - log2_particles - (be - 126);  // maxabs = m 2^(be - 126), m in [0.5, 1)
}

// ---- kernels ------------------------------------------------------------

struct Geo {
  Lattice L;
  int64_t np;        // particles
  int log2np;
};

// ---- particle sources of the deposition kernel ---------------------------
// A source is called once per particle p: it performs the particle update
// (if any), fills the particle's cell and its NCH deposit values (scaled by
// 2^E), and returns whether the particle deposits at all.

// 2LPT initial conditions: disp = (D1 psi1 + D2 psi2)/Delta,
// mom = (Gp1 psi1 + Gp2 psi2)/Delta (cell units); deposit unit weight.
template <typename T> struct SrcLpt {
  static constexpr int kMinBlocks = 5;  // FP32 blocks of 256 per SM (register cap)
  static constexpr int NCH = 1;
  Lattice L;
  int64_t np;
  const T *psi1, *psi2;
  T d1, d2, gp1, gp2;
  T *disp, *mom;
  const int *fx_exp;  // null: no deposit
  T scale;
  __device__ void setup() { scale = fx_exp ? pow2<T>(__ldg(fx_exp)) : T(0); }
  __device__ bool operator()(int64_t p, Cell<T> &c, T (&v)[1]) const {
    T d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T a1 = psi1[a * np + p];
      const T a2 = psi2 ? psi2[a * np + p] : T(0);
      d[a] = d1 * a1 + d2 * a2;
      disp[a * np + p] = d[a];
      mom[a * np + p] = gp1 * a1 + gp2 * a2;
    }
    c = locate<T>(L, p, d[0], d[1], d[2]);
    v[0] = scale;
    return fx_exp != nullptr;
  }
};

// Positions disp + rsd * mom along rsd_axis (rsd_axis < 0: none), unit weight.
template <typename T> struct SrcPaint {
  static constexpr int kMinBlocks = 5;
  static constexpr int NCH = 1;
  Lattice L;
  int64_t np;
  const T *disp, *mom;
  int rsd_axis;
  T rsd;
  const int *fx_exp;
  T scale;
  __device__ void setup() { scale = pow2<T>(__ldg(fx_exp)); }
  __device__ bool operator()(int64_t p, Cell<T> &c, T (&v)[1]) const {
    T d[3] = {disp[p], disp[np + p], disp[2 * np + p]};
    if (rsd_axis >= 0) d[rsd_axis] += rsd * mom[rsd_axis * np + p];
    c = locate<T>(L, p, d[0], d[1], d[2]);
    v[0] = scale;
    return true;
  }
};

// One fused leapfrog update: F = readout(Phi, x); p += kick F; x' = x + drift p;
// deposit x'.  x and x' may alias.
template <typename T> struct SrcKdk {
  static constexpr int kMinBlocks = 6;  // 40 registers: more warps hide the readout's corner loads
  static constexpr int NCH = 1;
  Lattice L;
  int64_t np;
  const V4<T> *phi;
  const T *x;
  T *xn, *mom;
  T kick, drift;
  const int *fx_exp;
  T scale;
  // lightcone snapshot of this state (null: none): position, and the momentum
  // synchronised with it, mom + kb F (kb: second half-kick of the previous step)
  T *snap_x = nullptr, *snap_p = nullptr;
  T kb = T(0);
  __device__ void setup() { scale = pow2<T>(__ldg(fx_exp)); }
  __device__ bool operator()(int64_t p, Cell<T> &c, T (&v)[1]) const {
    const T x0 = x[p], x1 = x[np + p], x2 = x[2 * np + p];
    c = locate<T>(L, p, x0, x1, x2);
    T f0, f1, f2;
    readout3<T>(L, phi, c, f0, f1, f2);
    if (snap_x) {
      snap_x[p] = x0;
      snap_x[np + p] = x1;
      snap_x[2 * np + p] = x2;
      snap_p[p] = mom[p] + kb * f0;
      snap_p[np + p] = mom[np + p] + kb * f1;
      snap_p[2 * np + p] = mom[2 * np + p] + kb * f2;
    }
    const T p0 = mom[p] + kick * f0, p1 = mom[np + p] + kick * f1, p2 = mom[2 * np + p] + kick * f2;
    mom[p] = p0;
    mom[np + p] = p1;
    mom[2 * np + p] = p2;
    const T y0 = x0 + drift * p0, y1 = x1 + drift * p1, y2 = x2 + drift * p2;
    xn[p] = y0;
    xn[np + p] = y1;
    xn[2 * np + p] = y2;
    c = locate<T>(L, p, y0, y1, y2);
    v[0] = scale;
    return true;
  }
};

// Last half kick p += kick F(x), then deposit x + rsd * p along rsd_axis
// (fx_exp null: kick only).
// Line of sight of particle p (radial redshift-space shift, Sec. 2.2.1 item
// 3): r = node + d - o in cell units (the unwrapped position seen from the
// observer o), unit vector u = r/|r| and 1/|r|.
template <typename T>
__device__ __forceinline__ void line_of_sight(const Lattice &L, int64_t p, const T (&d)[3], const T (&o)[3],
                                              T (&u)[3], T &inv_r) {
  int nd[3];
  L.node(p, nd[0], nd[1], nd[2]);
  T r[3], r2 = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[a] = ((T)nd[a] + d[a]) - o[a];
    r2 += r[a] * r[a];
  }
  inv_r = T(1) / sqrt(r2);
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = r[a] * inv_r;
}

// Shifted displacement along a box axis (0..2) or the line of sight (3).
template <typename T>
__device__ __forceinline__ void rsd_shift(const Lattice &L, int64_t p, int rsd_axis, T rsd, const T (&o)[3],
                                          const T (&m)[3], T (&d)[3]) {
  if (rsd_axis >= 0 && rsd_axis <= 2) {
    d[rsd_axis] += rsd * m[rsd_axis];
  } else if (rsd_axis == 3) {
    T u[3], inv_r;
    line_of_sight<T>(L, p, d, o, u, inv_r);
    const T pu = m[0] * u[0] + m[1] * u[1] + m[2] * u[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] += rsd * pu * u[a];
  }
}

// ---- lightcone (Sec. 2.2.1 item 3, Appendix A) ---------------------------
// Snapshots at a = 0.8, 0.9, 1: positions X_j and synchronised momenta P_j
// (cell units; X_2, P_2 are the final state).  Each particle's scale factor on
// the observer's past light cone comes from three fixed-point iterations
// a <- DistToScaleFactor(Delta |node + x(a) - o|) from a = 1, x(a) linear in a
// between the bracketing snapshots (a clamped to [0.8, 1]); its observed
// displacement is x(a) + (p(a) . u) u / (a^2 E(a)), u the unit line of sight.
// DistToScaleFactor interpolates the table (a_j, chi_j) linearly in chi.
constexpr int kLcIter = 3;
template <typename T> struct LightCone {
  const T *snap;        // X_0, X_1, P_0, P_1, each [3][np]
  const T *ta, *tchi;   // table, a increasing, chi (Mpc/h) decreasing
  const T *tsl;         // slope of each interval, da / dchi
  int ntab;
  T om, cell;           // Omega_m, cell size (Mpc/h)
  T o[3];               // observer, cell units

  __device__ __forceinline__ T snapv(int which, int a, int64_t np, int64_t p) const {
    return snap[((int64_t)which * 3 + a) * np + p];
  }
  // a(d) and da/dd of the table interpolant, linear in chi between nodes and
  // clamped to the table's ends (slope 0 outside)
  __device__ __forceinline__ T d2s(T d, T &slope) const {
    if (!(d < tchi[0])) {
      slope = T(0);
      return ta[0];
    }
    if (!(d > tchi[ntab - 1])) {
      slope = T(0);
      return ta[ntab - 1];
    }
    int lo = 0, hi = ntab - 1;  // chi decreases: chi[lo] > d > chi[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tchi[mid] > d) lo = mid; else hi = mid;
    }
    slope = tsl[lo];  // (a_lo - a_hi) / (chi_lo - chi_hi), taken in FP64 on the host
    return ta[hi] + slope * (d - tchi[hi]);
  }
  // y(a) between the snapshots (Y2 passed in), weights w[3] and dy/da
  __device__ __forceinline__ void interp(T a, const T (&y0)[3], const T (&y1)[3], const T (&y2)[3], T (&y)[3],
                                         T (&w)[3], T (&dy)[3]) const {
    const T s0 = T(0.8), s1 = T(0.9), s2 = T(1.0);
    const T ac = a < s0 ? s0 : (a > s2 ? s2 : a);
    const bool first = ac <= s1;
    const T lo = first ? s0 : s1, hi = first ? s1 : s2;
    const T t = (ac - lo) / (hi - lo);
    w[0] = first ? T(1) - t : T(0);
    w[1] = first ? t : T(1) - t;
    w[2] = first ? T(0) : t;
    const bool inside = a >= s0 && a <= s2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      y[c] = w[0] * y0[c] + w[1] * y1[c] + w[2] * y2[c];
      const T ya = first ? y0[c] : y1[c], yb = first ? y1[c] : y2[c];
      dy[c] = inside ? (yb - ya) / (hi - lo) : T(0);
    }
  }
};

// Observed displacement of particle p on the light cone from the final state
// (x2, p2) and the stored snapshots.
template <typename T>
__device__ __forceinline__ void lightcone_observed(const Lattice &L, const LightCone<T> &lc, int64_t np, int64_t p,
                                                   const T (&x2)[3], const T (&p2)[3], T (&out)[3]) {
  T x0[3], x1[3], q0[3], q1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x0[c] = lc.snapv(0, c, np, p);
    x1[c] = lc.snapv(1, c, np, p);
    q0[c] = lc.snapv(2, c, np, p);
    q1[c] = lc.snapv(3, c, np, p);
  }
  int nd[3];
  L.node(p, nd[0], nd[1], nd[2]);
  T a = T(1), x[3], w[3], dx[3], slope;
  for (int it = 0; it < kLcIter; ++it) {
    lc.interp(a, x0, x1, x2, x, w, dx);
    T r2 = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T r = ((T)nd[c] + x[c]) - lc.o[c];
      r2 += r * r;
    }
    a = lc.d2s(lc.cell * sqrt(r2), slope);
  }
  T pp[3], dp[3];
  lc.interp(a, x0, x1, x2, x, w, dx);
  lc.interp(a, q0, q1, p2, pp, w, dp);
  T r[3], r2 = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    r[c] = ((T)nd[c] + x[c]) - lc.o[c];
    r2 += r[c] * r[c];
  }
  const T inv = T(1) / sqrt(r2);
  const T e = sqrt(lc.om / (a * a * a) + (T(1) - lc.om));
  const T sh = T(1) / (a * a * e);
  const T pu = (pp[0] * r[0] + pp[1] * r[1] + pp[2] * r[2]) * inv;
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = x[c] + sh * pu * (r[c] * inv);
}

template <typename T> struct SrcFinal {
  static constexpr int kMinBlocks = 5;
  static constexpr int NCH = 1;
  Lattice L;
  int64_t np;
  const V4<T> *phi;
  const T *x;
  T *mom;
  T kick;
  int rsd_axis;
  T rsd;
  const int *fx_exp;
  T scale;
  T obs[3];  // observer, cell units (rsd_axis = 3)
  bool lightcone = false;
  LightCone<T> lc{};
  __device__ void setup() { scale = fx_exp ? pow2<T>(__ldg(fx_exp)) : T(0); }
  __device__ bool operator()(int64_t p, Cell<T> &c, T (&v)[1]) const {
    T d[3] = {x[p], x[np + p], x[2 * np + p]};
    c = locate<T>(L, p, d[0], d[1], d[2]);
    T f[3];
    readout3<T>(L, phi, c, f[0], f[1], f[2]);
    T m[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      m[a] = mom[a * np + p] + kick * f[a];
      mom[a * np + p] = m[a];
    }
    if (lightcone) {
      lightcone_observed<T>(L, lc, np, p, d, m, d);
    } else {
      rsd_shift<T>(L, p, rsd_axis, rsd, obs, m, d);
    }
    c = locate<T>(L, p, d[0], d[1], d[2]);
    v[0] = scale;
    return fx_exp != nullptr;
  }
};

// 3-channel force cotangent c_k * pbar at x_k, fixed point with the exponent
// chosen from the running max of |c_k pbar| (written to fx_exp_out).

template <typename T> struct SrcAdj3 {
  static constexpr int kMinBlocks = 5;
  static constexpr int NCH = 3;
  Lattice L;
  int64_t np;
  int log2np;
  const T *x, *pbar;
  T ck;
  const unsigned long long *maxslot;
  int *fx_exp_out;
  int e;
  __device__ void setup() {
    if constexpr (sizeof(T) == 4) e = fixed_exponent_f32(*reinterpret_cast<const unsigned *>(maxslot), log2np);
    else e = fixed_exponent((double)read_max_abs<T>(maxslot), log2np);
    if (blockIdx.x == 0 && threadIdx.x == 0) *fx_exp_out = e;
  }
  __device__ bool operator()(int64_t p, Cell<T> &c, T (&v)[3]) const {
    c = locate<T>(L, p, x[p], x[np + p], x[2 * np + p]);
    bool any = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T w = ck * pbar[a * np + p];
      if constexpr (sizeof(T) == 4) w = scalbnf(w, e);
      else w = scalbn(w, e);
      v[a] = w;
      any |= (w != T(0));
    }
    return any;
  }
};

// ---- deposition launch ----------------------------------------------------
// One thread per particle, in lattice order: a warp covers 32 consecutive
// particles along the fastest lattice axis (z), so its loads are coalesced.
// Each particle's 8 CIC deposits are integers q = rint(w v) added with
// integer atomics, so the mesh is the same for every schedule.
//
// Warp merge along z: when the next lane's particle has the same (x, y) cell
// and the z cell above (the usual case away from shell crossing), its four
// lower-z deposits land on this lane's four upper-z nodes; they are passed
// down by a shuffle and added here, so that lane issues only its upper-z
// atomics.  Same-cell merge: in each run of consecutive lanes whose particles
// share a cell (clustered states), the lanes at even positions of the run add
// all eight deposits of the next lane, which issues none (pairs only, so no
// lane waits on a chain).  The merged sums are sums of the same integers, so
// the mesh is unchanged bit for bit, with fewer atomics: the L2's reductions,
// not their width, bound the paint.

template <typename T, class Src>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? Src::kMinBlocks : 1) k_deposit(Geo g, Src src, unsigned long long *mesh, int64_t plane) {
  constexpr int NCH = Src::NCH;
  constexpr unsigned kFull = 0xffffffffu;
  Src s = src;
  s.setup();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Cell<T> c{};
  T v[NCH] = {};
  bool live = false;
  if (p < g.np) live = s(p, c, v);
  const int mask = g.L.mask, lane = threadIdx.x & 31;
  const int cx = live ? c.c[0] : -1, cy = live ? c.c[1] : -1, cz = live ? c.c[2] : -1;
  const int ux = __shfl_down_sync(kFull, cx, 1), uy = __shfl_down_sync(kFull, cy, 1);
  const int uz = __shfl_down_sync(kFull, cz, 1);
  const bool merge_up = live && lane < 31 && ux == cx && uy == cy && uz == ((cz + 1) & mask);
  const bool merged_down = __shfl_up_sync(kFull, merge_up ? 1 : 0, 1) != 0 && lane > 0;
  // same-cell pairs: in each run of lanes with one cell, the lanes at even
  // positions take over all deposits of the next lane (no chains)
  const bool same_next = live && lane < 31 && ux == cx && uy == cy && uz == cz;
  const bool same_prev = __shfl_up_sync(kFull, same_next ? 1 : 0, 1) != 0 && lane > 0;
  const unsigned starts = __ballot_sync(kFull, live && !same_prev);
  const int run0 = 31 - __clz(starts & ((2u << lane) - 1u));
  const bool absorber = same_next && !((lane - run0) & 1);
  const bool absorbed = __shfl_up_sync(kFull, absorber ? 1 : 0, 1) != 0 && lane > 0;
  const T wx[2] = {T(1) - c.f[0], c.f[0]};
  const T wy[2] = {T(1) - c.f[1], c.f[1]};
  const T wz[2] = {T(1) - c.f[2], c.f[2]};
  const int xs[2] = {cx, (cx + 1) & mask}, ys[2] = {cy, (cy + 1) & mask};
  const int z1 = (cz + 1) & mask;
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
#pragma unroll
    for (int ox = 0; ox < 2; ++ox)
#pragma unroll
      for (int oy = 0; oy < 2; ++oy) {
        const T wxy = wx[ox] * wy[oy] * v[ch];
        long long q0 = live ? fx_round<T>(wxy * wz[0]) : 0;
        long long q1 = live ? fx_round<T>(wxy * wz[1]) : 0;
        const long long up0 = __shfl_down_sync(kFull, q0, 1);
        if (merge_up) q1 += up0;
        const long long up1 = __shfl_down_sync(kFull, q1, 1);
        long long qz0 = merged_down ? 0 : q0;
        if (absorber) {
          qz0 += up0;
          q1 += up1;
        }
        if (live && !absorbed) {
          unsigned long long *col = mesh + ch * plane + ((((int64_t)xs[ox]) << g.L.logn | ys[oy]) << g.L.logn);
          if (qz0) fx_add(col + cz, qz0);
          if (q1) fx_add(col + z1, q1);
        }
      }
  }
}

// Plain readout of the force (probe): out = Delta * F at x.
template <typename T>
__global__ void k_readout(Geo g, const V4<T> *__restrict__ phi, const T *__restrict__ x, T scale,
                          T *__restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.np) return;
  const Cell<T> c = locate<T>(g.L, p, x[p], x[g.np + p], x[2 * g.np + p]);
  T f0, f1, f2;
  readout3<T>(g.L, phi, c, f0, f1, f2);
  out[p] = scale * f0;
  out[g.np + p] = scale * f1;
  out[2 * g.np + p] = scale * f2;
}

// Adjoint of the final paint (and RSD): xbar = grad_u sum W(u_s - c) dbar(c);
// pbar = rsd * xbar along the RSD axis; then the running max of |cn * pbar|.
template <typename T>
__global__ void k_adj_final(Geo g, const T *__restrict__ x, const T *__restrict__ mom, int rsd_axis, T rsd,
                            T ox, T oy, T oz, const T *__restrict__ dbar, T *__restrict__ xbar,
                            T *__restrict__ pbar, T cn, unsigned long long *maxslot) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T mx = T(0);
  if (p < g.np) {
    const T x0[3] = {x[p], x[g.np + p], x[2 * g.np + p]};
    const T m[3] = {mom[p], mom[g.np + p], mom[2 * g.np + p]};
    const T o[3] = {ox, oy, oz};
    T d[3] = {x0[0], x0[1], x0[2]};
    rsd_shift<T>(g.L, p, rsd_axis, rsd, o, m, d);
    const Cell<T> c = locate<T>(g.L, p, d[0], d[1], d[2]);
    T gx, gy, gz;
    grad_gather<T>(g.L, nullptr, dbar, c, T(0), T(0), T(0), gx, gy, gz);
    T pb[3] = {T(0), T(0), T(0)};
    T xb[3] = {gx, gy, gz};
    if (rsd_axis >= 0 && rsd_axis <= 2) {
      pb[rsd_axis] = rsd * xb[rsd_axis];
    } else if (rsd_axis == 3) {
      // x_s = x + c (p.u) u:  pbar = c u (u.g),
      // xbar = g + (c/|r|) [P p (u.g) + (p.u) P g],  P = I - u u^T
      T u[3], inv_r;
      line_of_sight<T>(g.L, p, x0, o, u, inv_r);
      const T ug = u[0] * gx + u[1] * gy + u[2] * gz;
      const T pu = m[0] * u[0] + m[1] * u[1] + m[2] * u[2];
      const T gg[3] = {gx, gy, gz};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pb[a] = rsd * u[a] * ug;
        xb[a] = gg[a] + rsd * inv_r * ((m[a] - u[a] * pu) * ug + pu * (gg[a] - u[a] * ug));
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xbar[a * g.np + p] = xb[a];
      pbar[a * g.np + p] = pb[a];
      mx = max(mx, fabs(cn * pb[a]));
    }
  }
  block_max_to_slots<T>(mx, maxslot);
}

// Adjoint of the final paint on the light cone (the transpose of
// lightcone_observed): per particle, the forward iterations are repeated
// (their inputs a and slopes kept), the paint's gradient g is gathered at the
// observed position, then
//   pbar(a) = s (u.g) u,   xbar(a) = g + (s/|r|) [P p (u.g) + (p.u) P g],
//   abar = s'(a) (p.u)(u.g) + xbar . dx/da + pbar . dp/da,
// Xbar_j = w_j xbar, Pbar_j = w_j pbar, and back through the iterations
// rbar = abar (da/dd) Delta r/|r|, Xbar_j += w_j rbar, abar = rbar . dx/da.
// Writes (Xbar_2, Pbar_2) to (xbar, pbar) and (Xbar_0, Xbar_1, Pbar_0,
// Pbar_1) over the snapshots in snapbar (= lc.snap), and the running max of
// |cn pbar|.
template <typename T>
__global__ void k_adj_final_lc(Geo g, LightCone<T> lc, T *snapbar, const T *__restrict__ x,
                               const T *__restrict__ mom, const T *__restrict__ dbar, T *__restrict__ xbar,
                               T *__restrict__ pbar, T cn, unsigned long long *maxslot) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t np = g.np;
  T mx = T(0);
  if (p < np) {
    T x0[3], x1[3], x2[3], q0[3], q1[3], q2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x0[c] = lc.snapv(0, c, np, p);
      x1[c] = lc.snapv(1, c, np, p);
      q0[c] = lc.snapv(2, c, np, p);
      q1[c] = lc.snapv(3, c, np, p);
      x2[c] = x[c * np + p];
      q2[c] = mom[c * np + p];
    }
    int nd[3];
    g.L.node(p, nd[0], nd[1], nd[2]);
    T ain[kLcIter], sl[kLcIter];
    T a = T(1), xx[3], w[3], dx[3];
    for (int it = 0; it < kLcIter; ++it) {
      ain[it] = a;
      lc.interp(a, x0, x1, x2, xx, w, dx);
      T r2 = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T r = ((T)nd[c] + xx[c]) - lc.o[c];
        r2 += r * r;
      }
      a = lc.d2s(lc.cell * sqrt(r2), sl[it]);
    }
    T pp[3], dp[3], wf[3];
    lc.interp(a, x0, x1, x2, xx, wf, dx);
    lc.interp(a, q0, q1, q2, pp, w, dp);
    T r[3], r2 = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r[c] = ((T)nd[c] + xx[c]) - lc.o[c];
      r2 += r[c] * r[c];
    }
    const T inv = T(1) / sqrt(r2);
    T u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = r[c] * inv;
    const T e = sqrt(lc.om / (a * a * a) + (T(1) - lc.om));
    const T s = T(1) / (a * a * e);
    const T pu = pp[0] * u[0] + pp[1] * u[1] + pp[2] * u[2];
    T ob[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ob[c] = xx[c] + s * pu * u[c];
    const Cell<T> cl = locate<T>(g.L, p, ob[0], ob[1], ob[2]);
    T gg[3];
    grad_gather<T>(g.L, nullptr, dbar, cl, T(0), T(0), T(0), gg[0], gg[1], gg[2]);
    const T ug = u[0] * gg[0] + u[1] * gg[1] + u[2] * gg[2];
    T xb[3], pb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pb[c] = s * u[c] * ug;
      xb[c] = gg[c] + s * inv * ((pp[c] - u[c] * pu) * ug + pu * (gg[c] - u[c] * ug));
    }
    // s = 1/(a^2 E), dE/da = -1.5 Omega_m a^-4 / E
    const T de = T(-1.5) * lc.om / (a * a * a * a * e);
    const T ds = T(-2) / (a * a * a * e) - de / (a * a * e * e);
    T abar = ds * pu * ug;
#pragma unroll
    for (int c = 0; c < 3; ++c) abar += xb[c] * dx[c] + pb[c] * dp[c];
    T X0[3], X1[3], X2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X0[c] = wf[0] * xb[c];
      X1[c] = wf[1] * xb[c];
      X2[c] = wf[2] * xb[c];
    }
    for (int it = kLcIter - 1; it >= 0; --it) {
      lc.interp(ain[it], x0, x1, x2, xx, w, dx);
      T rr[3], q2s = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        rr[c] = ((T)nd[c] + xx[c]) - lc.o[c];
        q2s += rr[c] * rr[c];
      }
      const T f = abar * sl[it] * lc.cell / sqrt(q2s);
      T nb = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T rb = f * rr[c];
        X0[c] += w[0] * rb;
        X1[c] += w[1] * rb;
        X2[c] += w[2] * rb;
        nb += rb * dx[c];
      }
      abar = nb;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      snapbar[(0 * 3 + c) * np + p] = X0[c];
      snapbar[(1 * 3 + c) * np + p] = X1[c];
      snapbar[(2 * 3 + c) * np + p] = wf[0] * pb[c];
      snapbar[(3 * 3 + c) * np + p] = wf[1] * pb[c];
      xbar[c * np + p] = X2[c];
      const T p2b = wf[2] * pb[c];
      pbar[c * np + p] = p2b;
      mx = max(mx, fabs(cn * p2b));
    }
  }
  block_max_to_slots<T>(mx, maxslot);
}

// Joins a snapshot's cotangents into the reverse sweep: xbar += xb (when
// given), pbar += f pb; then the running max of |cmax pbar|.
template <typename T>
__global__ void k_lc_join(Geo g, T *__restrict__ xbar, T *__restrict__ pbar, const T *__restrict__ xb,
                          const T *__restrict__ pb, T f, T cmax, unsigned long long *maxslot) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T mx = T(0);
  if (p < g.np) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t i = c * g.np + p;
      if (xbar) xbar[i] += xb[i];
      const T v = pbar[i] + f * pb[i];
      pbar[i] = v;
      mx = max(mx, fabs(cmax * v));
    }
  }
  block_max_to_slots<T>(mx, maxslot);
}

// Adjoint gather at x_k: xbar += grad_u sum W (c_k pbar . Phi_k + rhobar);
// then (if drift != 0) pbar += drift * xbar and the running max of |cnext pbar|.
// The FP32 kernel is capped at 40 registers (6 blocks of 256 per SM): it is
// bound by the latency of its dependent corner loads, and more resident warps
// keep more of them in flight.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 1) k_adj_gather(Geo g, const T *__restrict__ x, const V4<T> *__restrict__ phi,
                             const T *__restrict__ rhobar, T ck, T *__restrict__ xbar, T *__restrict__ pbar,
                             T drift, T cnext, unsigned long long *maxslot) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T mx = T(0);
  if (p < g.np) {
    const Cell<T> c = locate<T>(g.L, p, x[p], x[g.np + p], x[2 * g.np + p]);
    T pb[3] = {pbar[p], pbar[g.np + p], pbar[2 * g.np + p]};
    T gx, gy, gz;
    grad_gather<T>(g.L, phi, rhobar, c, ck * pb[0], ck * pb[1], ck * pb[2], gx, gy, gz);
    const T xb[3] = {xbar[p] + gx, xbar[g.np + p] + gy, xbar[2 * g.np + p] + gz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xbar[a * g.np + p] = xb[a];
      if (drift != T(0)) {
        pb[a] += drift * xb[a];
        pbar[a * g.np + p] = pb[a];
      }
      mx = max(mx, fabs(cnext * pb[a]));
    }
  }
  if (maxslot) block_max_to_slots<T>(mx, maxslot);
}

// Reverse drift alone (a reverse step whose kick cotangent is zero):
// pbar += drift * xbar, then the running max of |cnext pbar|; the same
// arithmetic as k_adj_gather with a zero gather.
template <typename T>
__global__ void k_reverse_drift(Geo g, const T *__restrict__ xbar, T *__restrict__ pbar, T drift, T cnext,
                                unsigned long long *maxslot) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T mx = T(0);
  if (p < g.np) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T pb = pbar[a * g.np + p];
      if (drift != T(0)) {
        pb += drift * xbar[a * g.np + p];
        pbar[a * g.np + p] = pb;
      }
      mx = max(mx, fabs(cnext * pb));
    }
  }
  if (maxslot) block_max_to_slots<T>(mx, maxslot);
}

// 2LPT adjoint, per particle (= per Lagrangian node): psi1bar, psi2bar.
template <typename T>
__global__ void k_lpt_adj(int64_t np, const T *__restrict__ xbar, const T *__restrict__ pbar, T d1, T d2,
                          T gp1, T gp2, T inv_cell, T *__restrict__ psi1bar, T *__restrict__ psi2bar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * np) return;
  const T xb = xbar[i] * inv_cell, pb = pbar[i] * inv_cell;
  psi1bar[i] = d1 * xb + gp1 * pb;
  if (psi2bar) psi2bar[i] = d2 * xb + gp2 * pb;
}

}  // namespace part
}  // namespace pm
