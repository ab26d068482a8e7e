// Stable LSD radix sort of (key, value) pairs, 8-bit digits, for the
// rank-order-matching step (Sec. 2.3.2).  Stability makes ties keep their
// input (index) order, so the matched permutation is unique and bit-exact.
//
// One digit pass = three kernels:
//   k_digit_hist    per-tile 256-bin histograms, stored digit-major [256][tiles]
//   k_digit_scan    exclusive scan of each digit row, then of the digit totals
//   k_digit_scatter stable in-tile ranking (warp match + per-warp counts, in
//                   element order) and scatter to the global position
#pragma once
#include "common.cuh"

namespace pm {
namespace sortk {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // elements per tile
constexpr int kWarps = kThreads / 32;

inline int64_t tiles_for(int64_t n) { return (n + kTile - 1) / kTile; }

// Bytes of scratch for sorting up to n pairs with keys of kbytes bytes.
inline size_t scratch_bytes(int64_t n, int kbytes) {
  const int64_t t = tiles_for(n);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return 2 * al((size_t)n * kbytes) + 2 * al((size_t)n * 4) + al((size_t)256 * t * 4) + al(256 * 4);
}

template <typename K> __device__ __forceinline__ int digit_of(K k, int shift) { return (int)((k >> shift) & 0xFF); }

template <typename K>
__global__ void __launch_bounds__(kThreads) k_digit_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                          unsigned int *__restrict__ hist, int64_t tiles) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += kThreads) {
    const int64_t g = t0 + i;
    if (g < n) atomicAdd(&h[digit_of(keys[g], shift)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of hist[d][0..tiles) in place; the row
// total goes to totals[d].
static __global__ void __launch_bounds__(kThreads) k_digit_scan_rows(unsigned int *hist, int64_t tiles,
                                                               unsigned int *totals) {
  __shared__ unsigned int sh[kThreads];
  unsigned int *row = hist + (int64_t)blockIdx.x * tiles;
  unsigned int carry = 0;
  for (int64_t base = 0; base < tiles; base += kThreads) {
    const int64_t i = base + threadIdx.x;
    const unsigned int v = i < tiles ? row[i] : 0u;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {  // inclusive Hillis-Steele scan
      const unsigned int a = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
      __syncthreads();
      sh[threadIdx.x] += a;
      __syncthreads();
    }
    if (i < tiles) row[i] = carry + sh[threadIdx.x] - v;
    carry += sh[kThreads - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Exclusive scan of the 256 digit totals (one block of 256 threads).
static __global__ void k_digit_scan_totals(unsigned int *totals) {
  __shared__ unsigned int sh[256];
  const unsigned int v = totals[threadIdx.x];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const unsigned int a = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
    __syncthreads();
    sh[threadIdx.x] += a;
    __syncthreads();
  }
  totals[threadIdx.x] = sh[threadIdx.x] - v;
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_digit_scatter(const K *__restrict__ kin, const unsigned int *__restrict__ vin,
                                                             K *__restrict__ kout, unsigned int *__restrict__ vout,
                                                             int64_t n, int shift, const unsigned int *__restrict__ hist,
                                                             const unsigned int *__restrict__ totals, int64_t tiles) {
  __shared__ unsigned int base[256];
  __shared__ unsigned int wcnt[kWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  base[threadIdx.x] = totals[threadIdx.x] + hist[(int64_t)threadIdx.x * tiles + blockIdx.x];
  const int64_t t0 = (int64_t)blockIdx.x * kTile;
  for (int r = 0; r < kItems; ++r) {
    for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t g = t0 + (int64_t)r * kThreads + threadIdx.x;
    const bool valid = g < n;
    K key = valid ? kin[g] : K(0);
    const int d = valid ? digit_of(key, shift) : 256 + lane;  // invalid lanes match nobody valid
    const unsigned int peers = __match_any_sync(0xffffffffu, d);
    const unsigned int below = peers & ((1u << lane) - 1u);
    if (valid && below == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned int pos = base[d] + __popc(below);
      for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
      kout[pos] = key;
      vout[pos] = vin[g];
    }
    __syncthreads();
    unsigned int add = 0;
    for (int w = 0; w < kWarps; ++w) add += wcnt[w][threadIdx.x];
    base[threadIdx.x] += add;
    __syncthreads();
  }
}

// Sorts (keys, vals) of length n by the bits [0, nbits) of the key, stably.
// Ping-pongs with (k2, v2); the result pointers are returned through kres/vres.
template <typename K>
inline cudaError_t radix_sort(K *k1, unsigned int *v1, K *k2, unsigned int *v2, int64_t n, int nbits,
                              unsigned int *hist, unsigned int *totals, cudaStream_t st, K **kres,
                              unsigned int **vres) {
  const int64_t tiles = tiles_for(n);
  K *ka = k1, *kb = k2;
  unsigned int *va = v1, *vb = v2;
  for (int shift = 0; shift < nbits; shift += 8) {
    ::pm::note_launch();
    k_digit_hist<K><<<(int)tiles, kThreads, 0, st>>>(ka, n, shift, hist, tiles);
    ::pm::note_launch();
    k_digit_scan_rows<<<256, kThreads, 0, st>>>(hist, tiles, totals);
    ::pm::note_launch();
    k_digit_scan_totals<<<1, 256, 0, st>>>(totals);
    ::pm::note_launch();
    k_digit_scatter<K><<<(int)tiles, kThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, totals, tiles);
    K *tk = ka;
    ka = kb;
    kb = tk;
    unsigned int *tv = va;
    va = vb;
    vb = tv;
  }
  *kres = ka;
  *vres = va;
  return cudaGetLastError();
}

// Keys that sort a float / double in DESCENDING order (ascending key), with
// -0 folded onto +0 so equal values tie and fall back to index order.
__device__ __forceinline__ unsigned int desc_key(float x) {
  if (x == 0.0f) x = 0.0f;
  const unsigned int b = __float_as_uint(x);
  const unsigned int asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return ~asc;
}
__device__ __forceinline__ unsigned long long desc_key(double x) {
  if (x == 0.0) x = 0.0;
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long asc = (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
  return ~asc;
}

template <typename T> struct KeyOf;
template <> struct KeyOf<float> { using type = unsigned int; };
template <> struct KeyOf<double> { using type = unsigned long long; };

}  // namespace sortk
}  // namespace pm
