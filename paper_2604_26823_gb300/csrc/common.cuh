// Shared device types and helpers of the particle-mesh library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <string>

namespace pm {

// ---- complex / vector types per precision -------------------------------
template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx = typename Cx<T>::type;

// four-component force mesh element (F_x, F_y, F_z, unused)
template <typename T> struct alignas(4 * sizeof(T)) V4 { T x, y, z, w; };

template <typename C> __host__ __device__ __forceinline__ C mkc(decltype(C::x) r, decltype(C::x) i) {
  C c;
  c.x = r;
  c.y = i;
  return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mkc<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mkc<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mkc<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mkc<C>(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return mkc<C>(a.x * s, a.y * s); }
// multiply by +i (SIGN > 0) or -i (SIGN < 0)
template <int SIGN, typename C> __device__ __forceinline__ C cmul_i(C a) {
  return SIGN > 0 ? mkc<C>(-a.y, a.x) : mkc<C>(a.y, -a.x);
}

// ---- fixed-point deposition ---------------------------------------------
// CIC deposits are accumulated as 64-bit integers, q = rint(w * 2^E), with
// integer atomics: integer addition is associative, so the painted mesh is
// identical for every thread schedule (deterministic deposition).
__device__ __forceinline__ void fx_add(unsigned long long *p, long long q) {
  atomicAdd(p, (unsigned long long)q);
}

// FP32 <-> int64 conversions (round to nearest, ties to even) that avoid the
// hardware conversions between FP32 and 64-bit integers, which issue on the
// FP64 unit -- narrow on this GPU, it limited the fixed-point paint.  Both are
// host-callable so they can be checked exhaustively on the CPU.
__host__ __device__ __forceinline__ unsigned fx_f32_bits(float w) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(w);
#else
  unsigned b;
  __builtin_memcpy(&b, &w, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float fx_bits_f32(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float w;
  __builtin_memcpy(&w, &b, 4);
  return w;
#endif
}
__host__ __device__ __forceinline__ int fx_clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

// rint(w) as int64 for |w| < 2^61 with one FP32 -> int32 conversion: below
// 2^31 the conversion itself is exact; above, w is an integer (its 24
// significant bits sit at 2^(e-23) and higher), so w 2^-s with
// s = exponent - 30 is still an integer below 2^31, converted exactly, and
// shifted back.  The FP32 -> int32 conversion issues on the FP32 side of the
// SM, not on the narrow FP64 unit that the FP32 -> int64 conversion uses.
__host__ __device__ __forceinline__ long long fx_f32_to_i64_split(float w) {
  const unsigned b = fx_f32_bits(w);
  const int be = (int)((b >> 23) & 0xffu);
  const int s = be > 157 ? be - 157 : 0;                 // |w| < 2^(be - 126)
  const float y = w * fx_bits_f32((unsigned)(127 - s) << 23);  // exact power-of-two scale
#ifdef __CUDA_ARCH__
  const int i = __float2int_rn(y);
#else
  const int i = (int)std::nearbyint(y);
#endif
  return (long long)((unsigned long long)(long long)i << s);
}

// Nearest float to the int64 q.
__host__ __device__ __forceinline__ float fx_i64_to_f32(long long q) {
  if (q == 0) return 0.0f;
  const unsigned long long mag = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
  int ex = 63 - fx_clz64(mag);  // position of the leading bit
  unsigned long long mm;
  if (ex <= 23) {
    mm = mag << (23 - ex);
  } else {
    const int sh = ex - 23;  // 1 .. 40
    mm = mag >> sh;
    const unsigned long long rem = mag & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    mm += (rem > half || (rem == half && (mm & 1ull))) ? 1ull : 0ull;
    if (mm >> 24) {  // rounding carried into a new leading bit
      mm >>= 1;
      ++ex;
    }
  }
  const unsigned bits = ((unsigned)(ex + 127) << 23) | ((unsigned)mm & 0x7fffffu);
  return fx_bits_f32(bits | (q < 0 ? 0x80000000u : 0u));
}

// ---- launch geometry ----------------------------------------------------
constexpr int kSMs = 152;

inline int grid_for(int64_t n, int threads, int max_blocks = 1 << 30) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// Number of kernel launches the library has issued since it was loaded
// (every launch site calls note_launch() right before its launch).
inline std::atomic<long long> g_launches{0};
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// thread-local error string of the C ABI
void set_error(const std::string &msg);

// Optional CUDA-event timing of kernel classes (off by default): every
// launch of a profiled class is bracketed by two events on its stream.
enum ProfClass : int {
  P_KDK = 0,       // fused readout + kick + drift + paint
  P_Z_R2C = 1,     // z pass real -> half complex
  P_COL = 2,       // strided complex column pass (y, or plain x)
  P_X_FUSED = 3,   // x pass with spectral multipliers
  P_Z_C2R = 4,     // z pass half complex -> real
  P_ADJ_PAINT = 5, // 3-channel cotangent paint
  P_ADJ_GATHER = 6,// adjoint weight-derivative gather
  P_LOSS = 7,      // likelihood / reductions
  P_OTHER = 8,     // 2LPT pointwise, memsets, ROM, projection
  P_NCLASS = 9
};

struct Profiler {
  bool on = false;
  int used = 0, cap = 0;
  cudaEvent_t *ev = nullptr;  // 2 per launch
  int *cls = nullptr;
  double *bytes = nullptr;    // algorithmic bytes of each launch (the method's arrays, FP32 / FP64 words)
  double *ibytes = nullptr;   // bytes of the implementation's own arrays (fixed-point meshes, padded vectors)
  double *flops = nullptr;    // floating-point operations of each launch (FFT passes; 0 elsewhere)
  ~Profiler() { release(); }
  void release() {
    for (int i = 0; i < 2 * cap; ++i) cudaEventDestroy(ev[i]);
    delete[] ev;
    delete[] cls;
    delete[] bytes;
    delete[] ibytes;
    delete[] flops;
    ev = nullptr;
    cls = nullptr;
    bytes = nullptr;
    ibytes = nullptr;
    flops = nullptr;
    cap = used = 0;
    on = false;
  }
  cudaError_t enable(int capacity) {
    release();
    ev = new cudaEvent_t[2 * capacity];
    cls = new int[capacity];
    bytes = new double[capacity];
    ibytes = new double[capacity];
    flops = new double[capacity];
    for (int i = 0; i < 2 * capacity; ++i) {
      const cudaError_t e = cudaEventCreate(&ev[i]);
      if (e != cudaSuccess) {
        cap = i / 2;
        return e;
      }
    }
    cap = capacity;
    on = true;
    return cudaSuccess;
  }
  int begin(int c, cudaStream_t st, double nbytes, double impl_bytes, double nflops) {
    if (!on || used >= cap) return -1;
    cls[used] = c;
    bytes[used] = nbytes;
    ibytes[used] = impl_bytes;
    flops[used] = nflops;
    cudaEventRecord(ev[2 * used], st);
    return used++;
  }
  void end(int slot, cudaStream_t st) {
    if (slot >= 0) cudaEventRecord(ev[2 * slot + 1], st);
  }
  // total milliseconds, launch count, algorithmic and implementation bytes
  // and flops of one class (synchronises)
  cudaError_t read(int c, double *ms, int64_t *count, double *nbytes, double *impl_bytes, double *nflops) {
    double t = 0.0, b = 0.0, ib = 0.0, fl = 0.0;
    int64_t k = 0;
    for (int i = 0; i < used; ++i) {
      if (cls[i] != c) continue;
      cudaError_t e = cudaEventSynchronize(ev[2 * i + 1]);
      if (e != cudaSuccess) return e;
      float f = 0.f;
      e = cudaEventElapsedTime(&f, ev[2 * i], ev[2 * i + 1]);
      if (e != cudaSuccess) return e;
      t += f;
      b += bytes[i];
      ib += ibytes[i];
      fl += flops[i];
      ++k;
    }
    *ms = t;
    *count = k;
    *nbytes = b;
    if (impl_bytes) *impl_bytes = ib;
    if (nflops) *nflops = fl;
    return cudaSuccess;
  }
};

// RAII bracket of one profiled launch: the method's algorithmic bytes, (when
// they differ) the implementation's bytes, and the launch's flops
struct ProfScope {
  Profiler &p;
  cudaStream_t st;
  int slot;
  ProfScope(Profiler &pr, int c, cudaStream_t s, double nbytes, double impl_bytes = -1.0, double nflops = 0.0)
      : p(pr), st(s), slot(pr.begin(c, s, nbytes, impl_bytes < 0 ? nbytes : impl_bytes, nflops)) {}
  ~ProfScope() { p.end(slot, st); }
};

// Flops of n_ffts complex FFTs of length len (the customary 5 len log2 len);
// a real FFT of length len counts half of that.
inline double fft_flops(double n_ffts, int len) {
  int lg = 0;
  while ((1 << lg) < len) ++lg;
  return 5.0 * n_ffts * len * lg;
}

}  // namespace pm

#define PM_CUDA_TRY(expr)                                                              \
  do {                                                                                 \
    cudaError_t e__ = (expr);                                                          \
    if (e__ != cudaSuccess) {                                                          \
      ::pm::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));            \
      return PM_ERR_CUDA;                                                              \
    }                                                                                  \
  } while (0)

#define PM_LAUNCH_CHECK()                                                              \
  do {                                                                                 \
    cudaError_t e__ = cudaGetLastError();                                              \
    if (e__ != cudaSuccess) {                                                          \
      ::pm::set_error(std::string("kernel launch: ") + cudaGetErrorString(e__));      \
      return PM_ERR_CUDA;                                                              \
    }                                                                                  \
  } while (0)
