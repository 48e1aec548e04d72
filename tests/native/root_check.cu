// Accuracy check of the FP64 square root and reciprocal square root of mhd_math.cuh
// (sqrt_nr, rsqrt_nr: FP32 estimate + two Newton-Raphson steps) on the GPU.  Arguments
// inside the fast range must lie within 1 ulp of the exact root (a long-double reference
// on the host); a warp with any argument outside it takes the library function, so there
// every lane must equal the library result bit for bit.  Prints
// "mismatches <n> checked <m> maxulp_sqrt <a> maxulp_rsqrt <b> rounded_sqrt <fraction>".
//   root_check <count>
#include <cmath>
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

// arguments: mostly positive values spread over the fast range and just beyond it; one
// warp in 16 gets any bit pattern (zeros, negatives, subnormals, infinities, NaNs)
__host__ __device__ inline uint64_t arg_case(uint64_t i) {
  const uint64_t r = mix(i);
  if ((i >> 5) % 16 == 0) return r;
  const uint64_t e = 1023 - 126 + (r >> 52) % 253;  // 2^-126 .. 2^126
  return (r & 0x000fffffffffffffull) | (e << 52);
}

__global__ void k_roots(uint64_t n, double* out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const double x = __longlong_as_double((long long)arg_case(i));
    out[4 * i + 0] = sqrt_nr(x);
    out[4 * i + 1] = rsqrt_nr(x);
    out[4 * i + 2] = sqrt(x);
    out[4 * i + 3] = rsqrt(x);
  }
}

static uint64_t bits(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
}
static bool same(double a, double b) { return (a != a && b != b) || bits(a) == bits(b); }
static double ulps(double got, long double ref) {
  int e;
  frexpl(ref, &e);
  return (double)(fabsl((long double)got - ref) / ldexpl(1.0L, e - 53));
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const uint64_t n = (strtoull(argv[1], nullptr, 10) + 31) / 32 * 32;  // whole warps
  double* dout;
  if (cudaMalloc(&dout, 4 * n * sizeof(double)) != cudaSuccess) return 3;
  k_roots<<<1184, 256>>>(n, dout);
  std::vector<double> out(4 * n);
  if (cudaMemcpy(out.data(), dout, 4 * n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return 4;
  cudaFree(dout);
  unsigned long long bad = 0, checked = 0, rounded = 0, fast = 0;
  double max_s = 0, max_r = 0;
  for (uint64_t w = 0; w < n; w += 32) {
    bool warp_fast = true;
    for (uint64_t i = w; i < w + 32; ++i) {
      const uint64_t b = arg_case(i);
      const unsigned e = (unsigned)(b >> 52);  // sign and exponent
      warp_fast = warp_fast && e - (1023u - 120u) <= 240u;
    }
    for (uint64_t i = w; i < w + 32; ++i) {
      const double x = [&] { double v; const uint64_t b = arg_case(i); memcpy(&v, &b, 8); return v; }();
      const double* o = &out[4 * i];
      ++checked;
      if (!warp_fast) {
        bad += !(same(o[0], o[2]) && same(o[1], o[3]));
        continue;
      }
      const long double rs = sqrtl((long double)x), rr = 1.0L / rs;
      const double us = ulps(o[0], rs), ur = ulps(o[1], rr);
      max_s = us > max_s ? us : max_s;
      max_r = ur > max_r ? ur : max_r;
      bad += !(us <= 1.0 && ur <= 1.0);
      rounded += same(o[0], o[2]);
      ++fast;
    }
  }
  printf("mismatches %llu checked %llu maxulp_sqrt %.3f maxulp_rsqrt %.3f rounded_sqrt %.6f\n",
         bad, checked, max_s, max_r, fast ? (double)rounded / fast : 0.0);
  return bad == 0 ? 0 : 1;
}
