// Division of a cell index by an invariant grid extent as a multiply and a shift
// (Granlund and Montgomery 1994, Theorem 4.2, with N = 31).  For 1 <= d < 2^31 let
// l = ceil(log2 d) and m = ceil(2^(31 + l) / d).  Then 0 <= m d - 2^(31 + l) < d <= 2^l,
// and for every 0 <= n < 2^31, floor(n / d) = floor(n m / 2^(31 + l)).  m < 2^32, so the
// product of n and m fits in 64 bits (below 2^63).  Host and device code include this
// file; tests/native/divmagic_check.cpp checks it against the division operator.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define IDX_HD __host__ __device__ __forceinline__
#else
#define IDX_HD inline
#endif

namespace idx {

// m and the shift 31 + l for divisor d (1 <= d < 2^31)
inline void div_magic(uint32_t d, uint32_t& m, int& shift) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  const uint64_t p = 1ull << (31 + l);
  m = (uint32_t)((p + d - 1) / d);
  shift = 31 + l;
}

// floor(n / d) for 0 <= n < 2^31, from d's m and shift
IDX_HD uint32_t div_by_magic(uint32_t n, uint32_t m, int shift) {
  return (uint32_t)(((uint64_t)n * m) >> shift);
}

}  // namespace idx
