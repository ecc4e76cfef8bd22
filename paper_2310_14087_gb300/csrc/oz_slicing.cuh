// Slicing arithmetic of the emulated-FP64 product (oz_gemm.cu): the fixed-point digit extraction
// and the rule that closes exact accumulation groups.  Plain integer code, compiled for the
// device by the kernels and for the host by the tests that pin its exactness without a GPU.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define KOT_HD __host__ __device__ __forceinline__
#define KOT_UNROLL _Pragma("unroll")
#else
#define KOT_HD inline
#define KOT_UNROLL
#endif

namespace kot {
namespace oz {

constexpr int kExactLevels = 4;    // slice levels t = i + j below this are summed exactly
constexpr int kExactTiles = 8;     // 8 x 64 products of |.| <= 2^14 per exact group: |sum| <= 2^23
constexpr int kMaxSlices = 8;

KOT_HD unsigned long long bits_of(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  std::memcpy(&b, &v, sizeof(b));
  return b;
#endif
}

KOT_HD int biased_exp(double v) { return (int)((bits_of(v) >> 52) & 0x7FFu); }

// Does the tile of level lv (following a tile of level prev; gt tiles already in the current
// group) start a new accumulation group?  Levels below kExactLevels are never mixed and close
// after kExactTiles tiles; the higher levels share one group.
KOT_HD bool new_group(int prev, int lv, int gt) {
  if (gt == 0) return true;
  if (lv != prev && (lv < kExactLevels || prev < kExactLevels)) return true;
  return lv < kExactLevels && gt >= kExactTiles;
}

// Balanced base-256 digits of v relative to the row exponent er (max |v| < 2^er):
// |v| 2^(7 + 8 (s-1) - er) rounded (half up) to the integer X = sum_i d_i 256^(s-1-i),
// |d_i| <= 128, signs following v.  Integer arithmetic only (FP64 issue is scarce on the GPU).
KOT_HD void digits(double v, int er, int s, int (&d)[kMaxSlices]) {
  const unsigned long long b = bits_of(v);
  int E = (int)((b >> 52) & 0x7FFu);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (E == 0) E = 1;             // subnormal: no implicit bit
  else m |= 1ull << 52;          // |v| = m 2^(E - 1075)
  const int sh = 1075 - E - 7 - 8 * (s - 1) + er;
  unsigned long long X;
  if (sh >= 64) X = 0;
  else if (sh > 0) X = (m >> sh) + ((m >> (sh - 1)) & 1ull);
  else X = m << (-sh);
  KOT_UNROLL
  for (int i = kMaxSlices - 1; i >= 1; --i) {
    d[i] = 0;
    if (i < s) {
      int dd = (int)(X & 0xFFu);
      X >>= 8;
      if (dd >= 128) {
        dd -= 256;
        ++X;
      }
      d[i] = dd;
    }
  }
  d[0] = (int)X;
  if (b >> 63) {
    KOT_UNROLL
    for (int i = 0; i < kMaxSlices; ++i) d[i] = -d[i];
  }
}

}  // namespace oz
}  // namespace kot
