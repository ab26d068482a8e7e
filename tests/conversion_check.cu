// Host check of the library's FP32 <-> int64 conversions (common.cuh:
// fx_f32_to_i64_split, fx_i64_to_f32), which the FP32
// deposits and the fixed-point loader use on the GPU.  Both must equal
// round-to-nearest-even conversions, here the C library's llrintf and the
// compiler's int64 -> float cast.  Prints the number of mismatches of each;
// exit code 0 when both are 0.
#include <cfenv>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "../paper_2604_26823_gb300/csrc/common.cuh"

int main() {
  std::fesetround(FE_TONEAREST);
  long long bad_f2i = 0, n_f2i = 0, bad_i2f = 0, n_i2f = 0;
  // float -> int64: every 97th bit pattern with |w| < 2^61 (finite), plus the halves
  for (uint64_t b = 0; b <= 0xffffffffull; b += 97) {
    const uint32_t bits = (uint32_t)b;
    if (((bits >> 23) & 0xffu) >= 0xbcu) continue;  // |w| >= 2^61
    float w;
    std::memcpy(&w, &bits, 4);
    ++n_f2i;
    const long long r = llrintf(w);
    if (pm::fx_f32_to_i64_split(w) != r) ++bad_f2i;
  }
  for (int k = -30; k <= 30; ++k) {
    const float w = (float)k + 0.5f;  // ties to even
    ++n_f2i;
    const long long r = llrintf(w);
    if (pm::fx_f32_to_i64_split(w) != r) ++bad_f2i;
  }
  // the split conversion's boundaries: every float within 2^12 ulps of 2^30,
  // 2^31 and the powers of two up to 2^60, both signs
  for (int ex = 30; ex <= 60; ++ex)
    for (int sgn = 0; sgn < 2; ++sgn)
      for (int d = -4096; d <= 4096; ++d) {
        float w = std::ldexp(1.0f, ex);
        uint32_t bits;
        std::memcpy(&bits, &w, 4);
        bits = (uint32_t)((int64_t)bits + d) | (sgn ? 0x80000000u : 0u);
        std::memcpy(&w, &bits, 4);
        if (!(std::fabs(w) < std::ldexp(1.0f, 61))) continue;
        ++n_f2i;
        if (pm::fx_f32_to_i64_split(w) != llrintf(w)) ++bad_f2i;
      }
  // int64 -> float: random magnitudes over the whole range, ties, extremes
  std::mt19937_64 g(12345);
  for (int i = 0; i < 20000000; ++i) {
    long long q = (long long)(g() >> (g() % 64));
    if (g() & 1) q = -q;
    const float a = pm::fx_i64_to_f32(q), r = (float)q;
    ++n_i2f;
    if (std::memcmp(&a, &r, 4)) ++bad_i2f;
  }
  for (int sh = 1; sh < 40; ++sh)
    for (long long k = 0; k < 2000; ++k) {
      const long long q = (((1ll << 23) + k) << sh) + (1ll << (sh - 1));  // exactly halfway
      for (int sgn = 0; sgn < 2; ++sgn) {
        const long long qq = sgn ? -q : q;
        const float a = pm::fx_i64_to_f32(qq), r = (float)qq;
        ++n_i2f;
        if (std::memcmp(&a, &r, 4)) ++bad_i2f;
      }
    }
  const long long edge[] = {0, 1, -1, (1ll << 24) - 1, 1ll << 24, (1ll << 24) + 1, (1ll << 25) + 3, INT64_MAX,
                            INT64_MIN, INT64_MIN + 1};
  for (long long q : edge) {
    const float a = pm::fx_i64_to_f32(q), r = (float)q;
    ++n_i2f;
    if (std::memcmp(&a, &r, 4)) ++bad_i2f;
  }
  std::printf("f2i %lld checked %lld mismatches; i2f %lld checked %lld mismatches\n", n_f2i, bad_f2i, n_i2f,
              bad_i2f);
  return (bad_f2i || bad_i2f) ? 1 : 0;
}
