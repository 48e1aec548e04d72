// Bitwise check of the integer-pipe float <-> double conversions of mhd_math.cuh against
// the IEEE round-to-nearest-even conversions: on the host (the bit recipes, compared
// with the CPU's converters) or on the GPU (the device functions, fast and slow paths,
// compared with the hardware converters).  Prints "mismatches <n> checked <m>".
//   conv_check host <count>     conv_check device <count>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../paper_2304_13746_b300/csrc/mhd_math.cuh"

using namespace idx;

// splitmix64: a counter-based generator of test bit patterns
__host__ __device__ inline uint64_t mix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// double patterns concentrated on the float range, plus ties and specials
__host__ __device__ inline uint64_t double_case(uint64_t i) {
  const uint64_t r = mix(i);
  switch (i % 8) {
    case 0: return r;                                               // any pattern
    case 1: {                                                       // exponent near float range
      const uint64_t e = 0x360 + (r >> 52) % 0x120;                 // 2^-159 .. 2^128
      return (r & 0x800fffffffffffffull) | (e << 52);
    }
    case 2: return (r & 0xfffffffff0000000ull) | 0x10000000ull;     // exact tie
    case 3: return (r & 0xffffffffe0000000ull) | 0x0fffffffull;     // just below a tie
    case 4: return (r & 0x800fffffffffffffull) | (0x47eull << 52);  // near the float maximum
    case 5: return (r & 0x800fffffffffffffull) | (0x380ull << 52);  // near the float minimum
    case 6: return (r & 0x8000000000000000ull) | ((r & 7) << 60);   // zeros and a few others
    default: return (r & 0x800fffffffffffffull) | ((0x3ff + ((r >> 52) % 64) - 32) << 52);
  }
}

__host__ __device__ inline uint32_t float_case(uint64_t i) {
  const uint64_t r = mix(i ^ 0x5bd1e995ull);
  if (i % 4 == 0) return (uint32_t)(r & 0x807fffffu);               // subnormals and zeros
  return (uint32_t)r;
}

__global__ void k_check(uint64_t n, unsigned long long* bad) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t db = double_case(i);
    const double d = __longlong_as_double((long long)db);
    const float f1 = d2f(d), f2 = (float)d;
    const bool nan1 = f1 != f1, nan2 = f2 != f2;
    if (nan1 != nan2 || (!nan1 && __float_as_uint(f1) != __float_as_uint(f2))) atomicAdd(bad, 1ull);
    const uint32_t fb = float_case(i);
    const float f = __uint_as_float(fb);
    const double e1 = f2d(f), e2 = (double)f;
    const bool n1 = e1 != e1, n2 = e2 != e2;
    if (n1 != n2 || (!n1 && __double_as_longlong(e1) != __double_as_longlong(e2))) atomicAdd(bad, 1ull);
  }
}

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  const uint64_t n = strtoull(argv[2], nullptr, 10);
  unsigned long long bad = 0, checked = 0;
  if (!strcmp(argv[1], "host")) {
    for (uint64_t i = 0; i < n; ++i) {
      const uint64_t db = double_case(i);
      double d;
      memcpy(&d, &db, 8);
      bool slow;
      const uint32_t q = d2f_bits((uint32_t)(db >> 32), (uint32_t)db, &slow);
      if (!slow) {
        const float ref = (float)d;
        uint32_t rb;
        memcpy(&rb, &ref, 4);
        bad += rb != q;
        ++checked;
      }
      const uint32_t fb = float_case(i);
      const uint64_t e = f2d_bits(fb, &slow);
      if (!slow) {
        float f;
        memcpy(&f, &fb, 4);
        const double ref = (double)f;
        uint64_t rb;
        memcpy(&rb, &ref, 8);
        bad += rb != e;
        ++checked;
      }
    }
  } else {
    unsigned long long* dbad;
    if (cudaMalloc(&dbad, sizeof(*dbad)) != cudaSuccess) return 3;
    cudaMemset(dbad, 0, sizeof(*dbad));
    k_check<<<1184, 256>>>(n, dbad);
    if (cudaMemcpy(&bad, dbad, sizeof(bad), cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
    cudaFree(dbad);
    checked = 2 * n;
  }
  printf("mismatches %llu checked %llu\n", bad, checked);
  return bad == 0 ? 0 : 1;
}
