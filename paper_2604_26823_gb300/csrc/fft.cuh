// Batched pencil FFTs over power-of-two meshes (16..512 per side) for the
// spectral steps of the particle-mesh model (linear field, 2LPT, Poisson
// force and their adjoints).
//
// A 3-D real transform is three passes over HBM:
//   z pass   contiguous rows, real <-> half complex (length-N/2 complex FFT
//            plus the even/odd split), tiles of B rows per CTA;
//   y pass   complex FFT along a strided axis, tiles of B contiguous columns;
//   x pass   complex FFT along the slowest axis; the spectral multipliers
//            (IC amplitude, 1/k^2, i k_i) are applied between the forward
//            and the inverse x FFT inside one kernel, so a real -> real
//            spectral operator never writes its spectrum back to HBM.
// Inside a CTA the FFT runs in shared memory as mixed-radix Stockham passes
// (radix 4/8/16 butterflies in registers, one barrier pair per pass).
// Convention: forward X(k) = sum_x x e^{-ikx}; the inverse passes are
// unnormalised (1/N^3 is folded into the multipliers).
#pragma once
#include "common.cuh"

namespace pm {
namespace fft {

// ---- radix plans --------------------------------------------------------
template <int LEN> struct Plan;
template <> struct Plan<8> { static constexpr int NP = 1, R0 = 8, R1 = 1, R2 = 1; };
template <> struct Plan<16> { static constexpr int NP = 1, R0 = 16, R1 = 1, R2 = 1; };
template <> struct Plan<32> { static constexpr int NP = 2, R0 = 8, R1 = 4, R2 = 1; };
template <> struct Plan<64> { static constexpr int NP = 2, R0 = 8, R1 = 8, R2 = 1; };
template <> struct Plan<128> { static constexpr int NP = 2, R0 = 16, R1 = 8, R2 = 1; };
template <> struct Plan<256> { static constexpr int NP = 2, R0 = 16, R1 = 16, R2 = 1; };
template <> struct Plan<512> { static constexpr int NP = 3, R0 = 8, R1 = 8, R2 = 8; };

// cos(2 pi j / 16) for j mod 16, as exact decimal constants of the unit circle
__host__ __device__ constexpr double cos16(int j) {
  switch (j & 15) {
    case 0: return 1.0;
    case 1: return 0.92387953251128675613;
    case 2: return 0.70710678118654752440;
    case 3: return 0.38268343236508977173;
    case 4: return 0.0;
    case 5: return -0.38268343236508977173;
    case 6: return -0.70710678118654752440;
    case 7: return -0.92387953251128675613;
    case 8: return -1.0;
    case 9: return -0.92387953251128675613;
    case 10: return -0.70710678118654752440;
    case 11: return -0.38268343236508977173;
    case 12: return 0.0;
    case 13: return 0.38268343236508977173;
    case 14: return 0.70710678118654752440;
    default: return 0.92387953251128675613;
  }
}
__host__ __device__ constexpr double sin16(int j) { return cos16(j + 12); }

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// In-register DFT of length R (2..16), X_k = sum_n x_n e^{SIGN 2 pi i n k / R}:
// iterative radix-2 decimation in time with constant twiddles.
template <int R, int SIGN, typename C>
__device__ __forceinline__ void dft(C *v) {
  using T = decltype(C::x);
  constexpr int L = ilog2(R);
  C t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[bitrev(i, L)] = v[i];
#pragma unroll
  for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
    for (int i = 0; i < R; i += len) {
#pragma unroll
      for (int j = 0; j < len / 2; ++j) {
        const int m = j * (16 / len);  // twiddle e^{SIGN 2 pi i j / len} = e^{SIGN 2 pi i m / 16}
        C b = t[i + j + len / 2];
        if (m == 4) {
          b = cmul_i<SIGN>(b);
        } else if (m != 0) {
          b = cmul(b, mkc<C>((T)cos16(m), (T)(SIGN * sin16(m))));
        }
        const C a = t[i + j];
        t[i + j] = cadd(a, b);
        t[i + j + len / 2] = csub(a, b);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = t[i];
}

// One Stockham pass of radix R (span P) over B sequences of length LEN held
// in shared memory as buf[pos * SB + col].  tw[m] = e^{-2 pi i m / (LEN*twmul)}.
template <typename C, int LEN, int R, int P, int B, int SB, int NT, int SIGN>
__device__ __forceinline__ void stockham_pass(C *buf, const C *__restrict__ tw, int twmul) {
  constexpr int NBF = B * (LEN / R);
  constexpr int PER = (NBF + NT - 1) / NT;
  C v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int id = threadIdx.x + q * NT;
    if (NBF % NT == 0 || id < NBF) {
      const int col = id % B, j = id / B;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[(j + r * (LEN / R)) * SB + col];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int id = threadIdx.x + q * NT;
    if (NBF % NT == 0 || id < NBF) {
      const int col = id % B, j = id / B;
      const int k = j & (P - 1);
      if (P > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = __ldg(&tw[r * k * (LEN / (P * R)) * twmul]);
          if (SIGN > 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft<R, SIGN>(v[q]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(base + r * P) * SB + col] = v[q][r];
    }
  }
  __syncthreads();
}

// Full length-LEN FFT of the B sequences in buf (caller syncs before).
template <typename C, int LEN, int B, int SB, int NT, int SIGN>
__device__ __forceinline__ void smem_fft(C *buf, const C *__restrict__ tw, int twmul) {
  using PL = Plan<LEN>;
  stockham_pass<C, LEN, PL::R0, 1, B, SB, NT, SIGN>(buf, tw, twmul);
  if constexpr (PL::NP > 1) stockham_pass<C, LEN, PL::R1, PL::R0, B, SB, NT, SIGN>(buf, tw, twmul);
  if constexpr (PL::NP > 2)
    stockham_pass<C, LEN, PL::R2, PL::R0 * PL::R1, B, SB, NT, SIGN>(buf, tw, twmul);
}

// ---- spectral multipliers -----------------------------------------------
enum : int { M_INVK2 = 1, M_AMP = 2, M_CONJ = 4, M_INCUBE = 8, M_OUTCUBE = 16, M_GAUSS = 32 };

// h(k) = scale * [A(k)] * [1/k^2 (0 at k = 0)] * D_d1(k) * D_d2(k), with
// D_i = i k_i (0 at the Nyquist index of axis i); conjugated on M_CONJ.
// M_INCUBE keeps only the modes with every |n_i| < cube (integer wave
// numbers), M_OUTCUBE only the others; M_GAUSS multiplies by
// exp(-gauss |k|^2) (gauss = R^2 / 2 for a Gaussian of width R).
struct MultDesc {
  double scale;
  int d1, d2, flags, cube;
  double gauss;
};
// The x pass sees one column (k_y, k_z fixed) at a time, so each multiplier
// factors as h_o(k) = X_p(k) C_o(k_y, k_z): a part X_p that varies along the
// column (amplitude, 1/k^2, Gaussian, cube masks, derivatives along x) and a
// per-column constant C_o (scale, derivatives along y and z; with nd
// derivatives in all, (i)^nd = (i)^nx (i)^nc).  Multipliers with the same X_p
// share one transform: IFFT_x(h_o X) = C_o IFFT_x(X_p X), and
// sum_i h_i FFT_x(in_i) = sum_p X_p FFT_x(sum_{i in p} C_i in_i).
struct XPlan {
  MultDesc xpart[9];  // distinct column-varying parts (scale 1, x derivatives only)
  MultDesc col[9];    // per spectrum: scale and y / z derivatives (no other flag but M_CONJ)
  int part_of[9];     // spectrum -> its part
  int nparts, count;
};

inline XPlan make_xplan(const MultDesc *m, int count) {
  XPlan p{};
  p.count = count;
  for (int o = 0; o < count; ++o) {
    const int ds[2] = {m[o].d1, m[o].d2};
    int nx = 0, dc[2] = {-1, -1}, nc = 0;
    for (int d : ds) {
      if (d == 0) ++nx;
      else if (d > 0) dc[nc++] = d;
    }
    MultDesc x = m[o];
    x.scale = 1.0;
    x.d1 = nx >= 1 ? 0 : -1;
    x.d2 = nx >= 2 ? 0 : -1;
    if (nx != 1) x.flags &= ~M_CONJ;  // the sign only enters with one imaginary unit
    MultDesc c{};
    c.scale = m[o].scale;
    c.d1 = dc[0];
    c.d2 = dc[1];
    c.flags = nc == 1 ? (m[o].flags & M_CONJ) : 0;
    c.cube = 0;
    c.gauss = 0.0;
    int q = 0;
    for (; q < p.nparts; ++q) {
      const MultDesc &y = p.xpart[q];
      if (y.flags == x.flags && y.d1 == x.d1 && y.d2 == x.d2 && y.cube == x.cube && y.gauss == x.gauss) break;
    }
    if (q == p.nparts) p.xpart[p.nparts++] = x;
    p.part_of[o] = q;
    p.col[o] = c;
  }
  return p;
}

template <typename T> struct ModeK {
  T k[3];   // k_i, zero at that axis' Nyquist index
  T ik2;    // 1/|k|^2, zero at k = 0
  T k2;     // |k|^2 (Nyquist components included)
  int amax; // max_i |n_i|
};

template <typename T>
__device__ __forceinline__ ModeK<T> mode_k(int ix, int iy, int iz, int n, T kf) {
  ModeK<T> m;
  const int h = n >> 1;
  const int nx = ix < h ? ix : ix - n;
  const int ny = iy < h ? iy : iy - n;
  const int nz = iz;
  m.k[0] = (ix == h) ? T(0) : kf * (T)nx;
  m.k[1] = (iy == h) ? T(0) : kf * (T)ny;
  m.k[2] = (iz == h) ? T(0) : kf * (T)nz;
  const int n2 = nx * nx + ny * ny + nz * nz;
  m.ik2 = n2 > 0 ? T(1) / (kf * kf * (T)n2) : T(0);
  m.k2 = kf * kf * (T)n2;
  m.amax = max(abs(nx), max(abs(ny), nz));
  return m;
}

// The x pass gives each thread one fixed column (iy, iz) of its tile, so the
// column part of the mode is formed once per thread and only the x part per
// element (same arithmetic as mode_k).
template <typename T> struct ColMode {
  T ky, kz, kf;
  int nyz2, ayz, h, n;
  __device__ __forceinline__ void init(int iy, int iz, int n_, T kf_) {
    n = n_;
    h = n >> 1;
    kf = kf_;
    const int ny = iy < h ? iy : iy - n;
    ky = (iy == h) ? T(0) : kf * (T)ny;
    kz = (iz == h) ? T(0) : kf * (T)iz;
    nyz2 = ny * ny + iz * iz;
    ayz = max(abs(ny), iz);
  }
  __device__ __forceinline__ ModeK<T> at(int ix) const {
    ModeK<T> m;
    const int nx = ix < h ? ix : ix - n;
    m.k[0] = (ix == h) ? T(0) : kf * (T)nx;
    m.k[1] = ky;
    m.k[2] = kz;
    const int n2 = nx * nx + nyz2;
    m.ik2 = n2 > 0 ? T(1) / (kf * kf * (T)n2) : T(0);
    m.k2 = kf * kf * (T)n2;
    m.amax = max(abs(nx), ayz);
    return m;
  }
};

template <typename T, typename C>
__device__ __forceinline__ C apply_mult(const MultDesc &d, C x, const ModeK<T> &mk, T amp) {
  T f = (T)d.scale;
  if (d.flags & M_AMP) f *= amp;
  if (d.flags & M_INVK2) f *= mk.ik2;
  if (d.flags & M_GAUSS) f *= exp(-(T)d.gauss * mk.k2);
  if (d.flags & (M_INCUBE | M_OUTCUBE)) {
    const bool in = mk.amax < d.cube;
    if ((d.flags & M_INCUBE) ? !in : in) f = T(0);
  }
  int nd = 0;
  if (d.d1 >= 0) {
    f *= mk.k[d.d1];
    ++nd;
  }
  if (d.d2 >= 0) {
    f *= mk.k[d.d2];
    ++nd;
  }
  C r;
  if (nd == 0) {
    r = mkc<C>(f * x.x, f * x.y);
  } else if (nd == 1) {  // (i f) x, conj: (-i f) x
    const T g = (d.flags & M_CONJ) ? -f : f;
    r = mkc<C>(-g * x.y, g * x.x);
  } else {  // (i f1)(i f2) = -f
    r = mkc<C>(-f * x.x, -f * x.y);
  }
  return r;
}

// ---- kernels ------------------------------------------------------------

// Tile gather into shared memory: every thread issues all PER of its loads
// before its first shared store, so PER independent loads per thread are in
// flight (the passes are bound by HBM latency, not by arithmetic).
template <int PER, int NT, typename V, class Ld, class St>
__device__ __forceinline__ void gather_tile(Ld ld, St st) {
  V r[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) r[q] = ld(threadIdx.x + q * NT);
#pragma unroll
  for (int q = 0; q < PER; ++q) st(threadIdx.x + q * NT, r[q]);
}

// Input loaders of the real z pass: a real mesh of type T, or a fixed-point
// (int64, value * 2^E) mesh converted on the fly.
template <typename T> struct LoadReal {
  const T *p;
  __device__ __forceinline__ void pair(int64_t i, T &a, T &b) const {
    const cx<T> v = reinterpret_cast<const cx<T> *>(p)[i];
    a = v.x;
    b = v.y;
  }
};
template <typename T> struct LoadFixed {
  const long long *p;
  const int *exp;  // value = q * 2^-exp (device scalar written by the paint)
  // subtract one unit weight (q = 2^exp) before the conversion: a painted
  // density rho (mean 1 particle per cell) becomes delta = rho - 1 exactly, in
  // integers, so the FP32 FFT's rounding scales with delta, not with rho
  bool sub_unit = false;
  __device__ __forceinline__ void pair(int64_t i, T &a, T &b) const {
    longlong2 v = reinterpret_cast<const longlong2 *>(p)[i];
    if (sub_unit) {
      const long long unit = 1ll << __ldg(exp);
      v.x -= unit;
      v.y -= unit;
    }
    const int e = -__ldg(exp);
    if constexpr (sizeof(T) == 4) {
      // the two exact int64 -> float conversions run on different units (the
      // hardware one on the FP64 unit, the other on the integer pipe); the
      // power-of-two scale is exact for normal results
      const float fa = __ll2float_rn(v.x), fb = fx_i64_to_f32(v.y);
      if (e >= -126) {
        const float sc = __int_as_float((e + 127) << 23);
        a = fa * sc;
        b = fb * sc;
      } else {
        a = scalbnf(fa, e);
        b = scalbnf(fb, e);
      }
    } else {
      a = scalbn(__ll2double_rn(v.x), e);
      b = scalbn(__ll2double_rn(v.y), e);
    }
  }
};

// z pass, real -> half complex: rows of N reals -> rows of N/2+1 complex.
// Row r of the batch reads in[r*N ...] and writes out[r*(N/2+1) ...].
template <typename T, int N, int B, int NT, class Load>
__global__ void __launch_bounds__(NT) k_z_r2c(Load in, cx<T> *__restrict__ out,
                                              const cx<T> *__restrict__ tw) {
  using C = cx<T>;
  constexpr int LEN = N / 2;
  constexpr int SB = B + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *buf = reinterpret_cast<C *>(smem_raw);
  static_assert(B * LEN % NT == 0, "tile must split evenly over threads");
  const int64_t row0 = (int64_t)blockIdx.x * B;
  gather_tile<B * LEN / NT, NT, C>(
      [&](int e) {
        T a, b;
        in.pair(row0 * LEN + e, a, b);
        return mkc<C>(a, b);
      },
      [&](int e, C v) { buf[(e % LEN) * SB + e / LEN] = v; });
  __syncthreads();
  smem_fft<C, LEN, B, SB, NT, -1>(buf, tw, 2);
  for (int e = threadIdx.x; e < B * (LEN + 1); e += NT) {
    const int row = e / (LEN + 1), k = e % (LEN + 1);
    const C zk = buf[(k % LEN) * SB + row];
    const C zc = cconj(buf[((LEN - k) % LEN) * SB + row]);
    const C ev = mkc<C>(T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y + zc.y));
    const C od = mkc<C>(T(0.5) * (zk.y - zc.y), -T(0.5) * (zk.x - zc.x));  // -i (zk - zc) / 2
    out[(row0 + row) * (LEN + 1) + k] = cadd(ev, cmul(__ldg(&tw[k]), od));
  }
}

// Complex FFT along a strided axis: element (b, pos, col) at
// base + b*bstride + pos*astride + col, cols [0, ncols); in place allowed.
template <typename T, int LEN, int B, int NT, int SIGN>
__global__ void __launch_bounds__(NT) k_col(const cx<T> *in, cx<T> *out, int64_t astride,
                                            int64_t bstride, int ncols, int tiles,
                                            const cx<T> *__restrict__ tw) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *buf = reinterpret_cast<C *>(smem_raw);
  const int tile = blockIdx.x % tiles;
  const int64_t b = blockIdx.x / tiles;
  const int col0 = tile * B;
  const int ncol = min(B, ncols - col0);
  const C *src = in + b * bstride + col0;
  C *dst = out + b * bstride + col0;
  static_assert(LEN * B % NT == 0, "tile must split evenly over threads");
  gather_tile<LEN * B / NT, NT, C>(
      [&](int e) {
        const int pos = e / B, c = e % B;
        return (c < ncol) ? src[pos * astride + c] : mkc<C>(T(0), T(0));
      },
      [&](int e, C v) { buf[e] = v; });
  __syncthreads();
  smem_fft<C, LEN, B, B, NT, SIGN>(buf, tw, 1);
  for (int e = threadIdx.x; e < LEN * B; e += NT) {
    const int pos = e / B, c = e % B;
    if (c < ncol) dst[pos * astride + c] = buf[e];
  }
}

struct XArgs1 {  // one input spectrum -> up to 9 output spectra
  const void *in;
  void *out[9];
  XPlan plan;
  const void *amp;  // IC amplitude on the half spectrum (or null)
  double kf;        // 2 pi / L
  int64_t bstride;  // batch stride of the input (and outputs) in complex elements
};
struct XArgsN {  // up to 9 input spectra -> one output spectrum
  const void *in[9];
  void *out;
  XPlan plan;
  const void *amp;
  double kf;
};

// x pass, case "one to many": X = FFT_x(in); out_o = IFFT_x(h_o X), o < count,
// one inverse transform per part X_p (out_o = C_o IFFT_x(X_p X)).
// Shared memory holds the transformed input (kept) and one work tile.
template <typename T, int N, int B, int NT, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) k_x_1toM(XArgs1 a, const cx<T> *__restrict__ tw) {
  using C = cx<T>;
  constexpr int H = N / 2 + 1;
  static_assert(N * B % NT == 0, "tile must split evenly over threads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *xin = reinterpret_cast<C *>(smem_raw);
  C *buf = xin + N * B;
  const int col0 = blockIdx.x * B;
  const int64_t astride = (int64_t)N * H;
  const C *src = reinterpret_cast<const C *>(a.in) + col0;
  gather_tile<N * B / NT, NT, C>([&](int e) { return src[(e / B) * astride + e % B]; },
                                 [&](int e, C v) { xin[e] = v; });
  __syncthreads();
  smem_fft<C, N, B, B, NT, -1>(xin, tw, 1);
  static_assert(NT % B == 0, "a thread keeps one column of the tile");
  const int c = threadIdx.x % B, colg = col0 + c;
  ColMode<T> cm;
  cm.init(colg / H, colg % H, N, (T)a.kf);
  const ModeK<T> mcol = cm.at(0);  // k_y, k_z of this thread's column
  for (int p = 0; p < a.plan.nparts; ++p) {
    const MultDesc &xm = a.plan.xpart[p];
    const bool use_amp = (xm.flags & M_AMP) != 0;
    for (int ix = threadIdx.x / B; ix < N; ix += NT / B) {
      const int e = ix * B + c;
      const T amp = use_amp ? reinterpret_cast<const T *>(a.amp)[(int64_t)ix * astride + colg] : T(0);
      buf[e] = apply_mult<T, C>(xm, xin[e], cm.at(ix), amp);
    }
    __syncthreads();
    smem_fft<C, N, B, B, NT, +1>(buf, tw, 1);
    for (int o = 0; o < a.plan.count; ++o) {
      if (a.plan.part_of[o] != p) continue;
      const C f = apply_mult<T, C>(a.plan.col[o], mkc<C>(T(1), T(0)), mcol, T(0));
      C *dst = reinterpret_cast<C *>(a.out[o]) + col0;
      for (int e = threadIdx.x; e < N * B; e += NT) dst[(e / B) * astride + e % B] = cmul(f, buf[e]);
    }
    __syncthreads();
  }
}

// x pass, case "many to one": out = IFFT_x( sum_i h_i FFT_x(in_i) ), one
// forward transform per part: sum_p X_p FFT_x(sum_{i in p} C_i in_i).
// Shared memory holds one work tile and the accumulator.
template <typename T, int N, int B, int NT, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) k_x_Mto1(XArgsN a, const cx<T> *__restrict__ tw) {
  using C = cx<T>;
  constexpr int H = N / 2 + 1;
  static_assert(N * B % NT == 0, "tile must split evenly over threads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *buf = reinterpret_cast<C *>(smem_raw);
  C *acc = buf + N * B;
  const int col0 = blockIdx.x * B;
  const int64_t astride = (int64_t)N * H;
  static_assert(NT % B == 0, "a thread keeps one column of the tile");
  const int c = threadIdx.x % B, colg = col0 + c;
  ColMode<T> cm;
  cm.init(colg / H, colg % H, N, (T)a.kf);
  const ModeK<T> mcol = cm.at(0);  // k_y, k_z of this thread's column
  for (int p = 0; p < a.plan.nparts; ++p) {
    // the tile loads of one input are the thread's own elements (column c),
    // so the part's inputs accumulate without a barrier between them
    bool first = true;
    for (int i = 0; i < a.plan.count; ++i) {
      if (a.plan.part_of[i] != p) continue;
      const C f = apply_mult<T, C>(a.plan.col[i], mkc<C>(T(1), T(0)), mcol, T(0));
      const C *src = reinterpret_cast<const C *>(a.in[i]) + col0;
      if (first)
        gather_tile<N * B / NT, NT, C>([&](int e) { return src[(e / B) * astride + e % B]; },
                                       [&](int e, C v) { buf[e] = cmul(f, v); });
      else
        gather_tile<N * B / NT, NT, C>([&](int e) { return src[(e / B) * astride + e % B]; },
                                       [&](int e, C v) { buf[e] = cadd(buf[e], cmul(f, v)); });
      first = false;
    }
    __syncthreads();
    smem_fft<C, N, B, B, NT, -1>(buf, tw, 1);
    const MultDesc &xm = a.plan.xpart[p];
    const bool use_amp = (xm.flags & M_AMP) != 0;
    for (int ix = threadIdx.x / B; ix < N; ix += NT / B) {
      const int e = ix * B + c;
      const T amp = use_amp ? reinterpret_cast<const T *>(a.amp)[(int64_t)ix * astride + colg] : T(0);
      const C h = apply_mult<T, C>(xm, buf[e], cm.at(ix), amp);
      acc[e] = p ? cadd(acc[e], h) : h;
    }
    __syncthreads();
  }
  smem_fft<C, N, B, B, NT, +1>(acc, tw, 1);
  C *dst = reinterpret_cast<C *>(a.out) + col0;
  for (int e = threadIdx.x; e < N * B; e += NT) dst[(e / B) * astride + e % B] = acc[e];
}

struct Ins {
  const void *p[9];
};

// z pass, half complex -> real (unnormalised) for NIN spectra sharing rows;
// Out::put(row, m, v[NIN]) receives the real pair (x_{2m}, x_{2m+1}) of each.
// Each input is transformed in its own shared-memory tile.
template <typename T, int N, int B, int NT, int NIN, class Out, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) k_z_c2r(Ins ins, Out out, const cx<T> *__restrict__ tw) {
  using C = cx<T>;
  constexpr int LEN = N / 2;
  constexpr int SB = B + 1;
  static_assert(B * LEN % NT == 0, "tile must split evenly over threads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *bufs = reinterpret_cast<C *>(smem_raw);
  const int64_t row0 = (int64_t)blockIdx.x * B;
#pragma unroll 1
  for (int i = 0; i < NIN; ++i) {
    C *buf = bufs + i * LEN * SB;
    const C *src = reinterpret_cast<const C *>(ins.p[i]);
    struct Pair {
      C k, c;
    };
    gather_tile<B * LEN / NT, NT, Pair>(
        [&](int e) {
          const C *rp = src + (row0 + e / LEN) * (LEN + 1);
          const int k = e % LEN;
          return Pair{rp[k], rp[LEN - k]};
        },
        [&](int e, Pair pr) {
          const int row = e / LEN, k = e % LEN;
          C xk = pr.k, xc = cconj(pr.c);
          if (k == 0) {
            xk.y = T(0);
            xc.y = T(0);
          }
          const C ev = cadd(xk, xc);
          const C od = cmul(csub(xk, xc), cconj(__ldg(&tw[k])));
          buf[k * SB + row] = mkc<C>(ev.x - od.y, ev.y + od.x);  // ev + i od
        });
    __syncthreads();
    smem_fft<C, LEN, B, SB, NT, +1>(buf, tw, 2);
  }
#pragma unroll 2
  for (int e = threadIdx.x; e < B * LEN; e += NT) {
    C w[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) w[i] = bufs[i * LEN * SB + (e % LEN) * SB + e / LEN];
    out.put(row0 + e / LEN, e % LEN, w);
  }
}

}  // namespace fft
}  // namespace pm
