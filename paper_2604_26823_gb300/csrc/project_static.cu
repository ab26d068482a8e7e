// pm_project_noalloc: the projection step (z-score + reset of |s_hat| > 10)
// for callers that cannot give the library any device memory -- for example
// a host application whose GPU memory is entirely owned by another allocator
// (a framework's caching allocator or a fixed pool), or code that must not call
// cudaMalloc mid-run because an allocation can synchronise the device.  Such a
// caller passes only its input / output vector; the reduction scratch this
// step needs lives in a file-scope device array of the library instead.
//
// Scratch: one FP64 partial sum per 4096 elements (at most kMaxBlocks), plus
// the sum, the sum of squared deviations, the reset counter and mu, sd, 1/sd
// with the flag that lets the projection kernel leave s untouched when the
// moments are not finite or the variance is zero.  Every GPU
// that loads the library holds this array (about 512 KB) until the process
// exits.  Every call shares it and it keeps the last call's contents; the
// reset counter is cleared at the start of each call.  Calls that overlap on
// the GPU (different streams, or different host threads on one device) race
// on the shared array: serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/mujica_pm.h"
#include "common.cuh"
#include "pointwise.cuh"
#include "rom.cuh"

namespace {

constexpr int kItems = 4096;                                  // elements per partial sum
constexpr int64_t kMaxBlocks = 65536;                         // partial sums in the array
constexpr int64_t kMaxElems = kMaxBlocks * (int64_t)kItems;   // 2^28 elements
constexpr int kTail = 8;                                      // sums, counter, mu / sd / 1/sd / valid flag, spare

static __device__ __align__(256) double g_project_scratch[kMaxBlocks + kTail];

// Host-side address of g_project_scratch on each device, looked up once per
// device (with that device current) by the first call made on it.
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

pm_status scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    pm::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return PM_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    pm::set_error("device index beyond the supported range of pm_project_noalloc");
    return PM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_project_scratch);
    if (e != cudaSuccess) {
      pm::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return PM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return PM_OK;
}

// One FP64 partial per block of kItems elements: sum of x, or (when mean_sum
// is given) sum of (x - mean)^2.
template <typename T>
__global__ void k_partials(const T *__restrict__ x, int64_t n, const double *mean_sum, double *partial) {
  const double mu = mean_sum ? *mean_sum / (double)n : 0.0;
  const int64_t base = (int64_t)blockIdx.x * kItems;
  double acc = 0.0;
  for (int i = threadIdx.x; i < kItems; i += blockDim.x) {
    const int64_t g = base + i;
    if (g < n) {
      const double v = (double)x[g] - mu;
      acc += mean_sum ? v * v : (double)x[g];
    }
  }
  pm::pw::block_sum_store(acc, partial);
}

template <typename T>
pm_status run(int64_t n, T *s, uint64_t seed, uint64_t counter, int64_t *n_reset_out, cudaStream_t st) {
  double *scr = nullptr;
  pm_status ps = scratch_for_current_device(&scr);
  if (ps) return ps;
  double *partial = scr, *res = scr + kMaxBlocks;
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(res + 2);
  const int blocks = (int)((n + kItems - 1) / kItems);
  PM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
  ::pm::note_launch();
  k_partials<T><<<blocks, pm::pw::kRedThreads, 0, st>>>(s, n, nullptr, partial);
  ::pm::note_launch();
  pm::pw::k_sum_partials<<<1, pm::pw::kRedThreads, 0, st>>>(partial, blocks, res + 0);
  ::pm::note_launch();
  k_partials<T><<<blocks, pm::pw::kRedThreads, 0, st>>>(s, n, res + 0, partial);
  ::pm::note_launch();
  pm::pw::k_sum_partials<<<1, pm::pw::kRedThreads, 0, st>>>(partial, blocks, res + 1);
  const unsigned long long key = pm::rom::mix64(seed + counter * pm::rom::kGolden + pm::rom::kGolden);
  ::pm::note_launch();
  pm::rom::k_project_scalars<<<1, 1, 0, st>>>(n, res + 0, res + 1, res + 3);
  ::pm::note_launch();
  pm::rom::k_project<T><<<pm::grid_for(n, 256), 256, 0, st>>>(s, n, res + 3, 10.0, key, cnt);
  PM_LAUNCH_CHECK();
  double h[3];
  PM_CUDA_TRY(cudaMemcpyAsync(h, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  PM_CUDA_TRY(cudaStreamSynchronize(st));
  if (!std::isfinite(h[0]) || !std::isfinite(h[1]) || !(h[1] > 0)) {
    pm::set_error("projection input has NaN / Inf or zero variance");
    return PM_ERR_NONFINITE;
  }
  unsigned long long c;
  std::memcpy(&c, &h[2], sizeof(c));
  if (n_reset_out) *n_reset_out = (int64_t)c;
  return PM_OK;
}

}  // namespace

extern "C" pm_status pm_project_noalloc(int64_t n, int32_t precision, void *s_inout, uint64_t rng_seed,
                                        uint64_t rng_counter, int64_t *n_reset_out, pm_stream_t stream) {
  if (!s_inout || n < 2 || (precision != PM_PREC_F32 && precision != PM_PREC_F64)) {
    pm::set_error("pm_project_noalloc: NULL s, fewer than 2 elements, or bad precision");
    return PM_ERR_INVALID_ARG;
  }
  if (n > kMaxElems) {
    pm::set_error("pm_project_noalloc: n = " + std::to_string(n) + " exceeds the maximum of " +
                  std::to_string(kMaxElems) + " elements (2^28) its static scratch supports");
    return PM_ERR_UNSUPPORTED;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (precision == PM_PREC_F32)
    return run<float>(n, static_cast<float *>(s_inout), rng_seed, rng_counter, n_reset_out, st);
  return run<double>(n, static_cast<double *>(s_inout), rng_seed, rng_counter, n_reset_out, st);
}
