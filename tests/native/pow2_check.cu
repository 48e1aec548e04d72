// Check of the exponent-field scalings of mhd_math.cuh on the GPU: pow2_fp64<K>(x) for
// K = -2, -1, 2 must equal the product x * 2^K bit for bit (NaN for NaN), whatever the other
// lanes of the warp hold.  Arguments: warps of normal values well inside the range (the
// integer path), warps with values at the ends of the exponent range, zeros of both signs,
// subnormals, infinities and NaNs (the product path), and warps that mix both.  Prints
// "mismatches <n> checked <m> fast_warps <f>" (warps whose lanes all take the integer path
// for every K).
//   pow2_check <count>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../paper_2304_13746_b300/csrc/mhd_math.cuh"

using namespace idx;

__host__ __device__ inline uint64_t mix(uint64_t z) {  // splitmix64
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// warp w of kind w % 4: 0, 1 normal values with exponent fields 3 .. 0x7fc (the integer path
// for every K); 2 exponent fields 0, 1, 2, 0x7fc .. 0x7ff and zeros; 3 any bit pattern
__host__ __device__ inline uint64_t arg_case(uint64_t i) {
  const uint64_t r = mix(i);
  const uint64_t kind = (i >> 5) % 4;
  const uint64_t sign = r & 0x8000000000000000ull, frac = r & 0x000fffffffffffffull;
  if (kind <= 1) return sign | ((3 + (r >> 52) % (0x7fc - 3 + 1)) << 52) | frac;
  if (kind == 2) {
    const uint64_t ends[8] = {0, 1, 2, 0x7fc, 0x7fd, 0x7fe, 0x7ff, 0};
    const uint64_t e = ends[(r >> 52) % 8];
    const uint64_t f = (r >> 60) % 4 == 0 ? 0 : frac;  // exact zeros and infinities too
    return sign | (e << 52) | f;
  }
  return r;
}

__global__ void k_pow2(uint64_t n, uint64_t* out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const double x = __longlong_as_double((long long)arg_case(i));
    out[6 * i + 0] = (uint64_t)__double_as_longlong(pow2_fp64<-2>(x));
    out[6 * i + 1] = (uint64_t)__double_as_longlong(x * 0.25);
    out[6 * i + 2] = (uint64_t)__double_as_longlong(pow2_fp64<-1>(x));
    out[6 * i + 3] = (uint64_t)__double_as_longlong(x * 0.5);
    out[6 * i + 4] = (uint64_t)__double_as_longlong(pow2_fp64<2>(x));
    out[6 * i + 5] = (uint64_t)__double_as_longlong(x * 4.0);
  }
}

static bool is_nan(uint64_t b) { return (b & 0x7ff0000000000000ull) == 0x7ff0000000000000ull && (b & 0x000fffffffffffffull); }

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const uint64_t n = (strtoull(argv[1], nullptr, 10) + 31) / 32 * 32;  // whole warps
  uint64_t* dout;
  if (cudaMalloc(&dout, 6 * n * sizeof(uint64_t)) != cudaSuccess) return 3;
  k_pow2<<<1184, 256>>>(n, dout);
  std::vector<uint64_t> out(6 * n);
  if (cudaMemcpy(out.data(), dout, 6 * n * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return 4;
  cudaFree(dout);
  unsigned long long bad = 0, checked = 0, fast_warps = 0;
  for (uint64_t w = 0; w < n; w += 32) {
    bool fast = true;
    for (uint64_t i = w; i < w + 32; ++i) {
      const unsigned e = (unsigned)((arg_case(i) >> 52) & 0x7ff);
      fast = fast && e >= 3 && e <= 0x7fc;
    }
    fast_warps += fast;
    for (uint64_t i = w; i < w + 32; ++i)
      for (int k = 0; k < 3; ++k) {
        const uint64_t a = out[6 * i + 2 * k], b = out[6 * i + 2 * k + 1];
        ++checked;
        if (!(a == b || (is_nan(a) && is_nan(b)))) {
          if (bad < 5) printf("x %016llx K-case %d: %016llx != %016llx\n",
                              (unsigned long long)arg_case(i), k, (unsigned long long)a,
                              (unsigned long long)b);
          ++bad;
        }
      }
  }
  printf("mismatches %llu checked %llu fast_warps %llu\n", bad, checked, fast_warps);
  return bad == 0 ? 0 : 1;
}
