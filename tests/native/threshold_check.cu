// Check of the FP64 HLLD threshold tests of mhd_math.cuh on the GPU: degenerate_fp64 and
// hllc_limit_fp64 decide from the binary exponents where those settle the question and by
// the FP64 comparison otherwise; every decision must equal the plain comparison's,
//   |D| <= 1e-12 (|q e| + Bx^2)      and      Bx^2 / 2 < 1e-12 p_T*,
// whatever the other lanes of the warp hold.  Arguments: magnitudes over the whole exponent
// range, ratios near the thresholds (within a few powers of two of 1e-12), exact zeros,
// subnormals, negative values, and lanes of every kind mixed in one warp.  Prints
// "mismatches <n> checked <m> exact_deg <a> exact_hllc <b>" (how many went to the comparison).
//   threshold_check <count>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../paper_2304_13746_b300/csrc/mhd_math.cuh"

using namespace idx;

__host__ __device__ inline uint64_t mix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// a double from a random word: kind 0 any exponent, 1 near `ref` times 2^(-40 +- 6), 2 zero,
// 3 subnormal, 4 negative of kind 0/1
__host__ __device__ inline double make(uint64_t r, double ref) {
  const int kind = (int)((r >> 59) % 8);
  uint64_t frac = r & 0x000fffffffffffffull;
  double v;
  if (kind <= 2) {
    const uint64_t e = 1 + (r >> 52) % 2046;
    uint64_t b = (e << 52) | frac;
    memcpy(&v, &b, 8);
  } else if (kind <= 5) {
    const int sh = -46 + (int)((r >> 52) % 13);  // 2^-46 .. 2^-34 of ref
    v = ldexp(1.0 + (double)(frac >> 20) / 4294967296.0, sh) * ref;
  } else if (kind == 6) {
    v = 0.0;
  } else {
    uint64_t b = frac >> ((r >> 40) % 52);  // subnormal (or zero)
    memcpy(&v, &b, 8);
  }
  if (((r >> 32) & 15) == 0) v = -v;
  return v;
}

__global__ void k_check(uint64_t n, unsigned long long* bad, unsigned long long* exact_d,
                        unsigned long long* exact_h) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r0 = mix(4 * i), r1 = mix(4 * i + 1), r2 = mix(4 * i + 2), r3 = mix(4 * i + 3);
    const double qe = make(r0, 1.0);
    const double bx2 = fabs(make(r1, fabs(qe) + 1e-300));
    const double D = make(r2, fabs(qe) + bx2);
    // p_T* near 5e11 Bx^2 * 2^(+-6), where Bx^2 / 2 meets 1e-12 p_T*, or anywhere
    const double pTs = make(r3, bx2 > 0.0 ? bx2 * 5.5e23 : 1.0);
    const bool d_fast = degenerate_fp64(D, qe, bx2);
    const bool d_plain = le_nn(fabs(D), Eps<double>::degen * (fabs(qe) + bx2));
    const bool h_fast = hllc_limit_fp64(bx2, pTs);
    const bool h_plain = lt_nn(0.5 * bx2, Eps<double>::hllc * pTs);
    if (d_fast != d_plain || h_fast != h_plain) atomicAdd(bad, 1ull);
    // how many lanes the exponents left to the comparison
    const int eq = bexp(qe), eb = bexp(bx2), eD = bexp(D), ep = bexp(pTs);
    if (eD == 0 || eD < (eq > eb ? eq : eb) - 37) atomicAdd(exact_d, 1ull);
    const bool quick = ep > 0 && !(pTs < 0.0);
    if (!quick || (!(eb < ep - 41) && (eb == 0 || eb < ep - 37))) atomicAdd(exact_h, 1ull);
  }
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const uint64_t n = (strtoull(argv[1], nullptr, 10) + 31) / 32 * 32;
  unsigned long long* d;
  if (cudaMalloc(&d, 3 * sizeof(unsigned long long)) != cudaSuccess) return 3;
  cudaMemset(d, 0, 3 * sizeof(unsigned long long));
  k_check<<<1184, 256>>>(n, d, d + 1, d + 2);
  unsigned long long h[3];
  if (cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
  cudaFree(d);
  printf("mismatches %llu checked %llu exact_deg %llu exact_hllc %llu\n", h[0],
         (unsigned long long)n, h[1], h[2]);
  return h[0] == 0 ? 0 : 1;
}
