// Check of the multiply-and-shift division of csrc/divmagic.cuh against the division
// operator, on the host: every divisor 1 .. 70000 and random divisors up to 2^31 - 1, each
// with the dividends 0, 1, d - 1, d, d + 1, the last multiples of d below 2^31 and next to
// them, 2^31 - 1, and random ones.  Prints "mismatches <n> checked <m>".
//   divmagic_check <random divisors>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "../../paper_2304_13746_b300/csrc/divmagic.cuh"

static uint64_t mix(uint64_t z) {  // splitmix64
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

int main(int argc, char** argv) {
  const uint64_t nrand = argc > 1 ? strtoull(argv[1], nullptr, 10) : 100000;
  const uint32_t top = 0x7fffffffu;  // 2^31 - 1
  unsigned long long bad = 0, checked = 0;
  uint64_t seed = 1;
  auto check_divisor = [&](uint32_t d) {
    uint32_t m;
    int sh;
    idx::div_magic(d, m, sh);
    const uint32_t last = top / d * d;
    uint32_t ns[16] = {0, 1, d - 1, d, d + 1 <= top ? d + 1 : top, last, last - 1 <= top ? last - 1 : 0,
                       last >= d ? last - d : 0, last >= d + 1 ? last - d - 1 : 0, top, top - 1};
    int cnt = 11;
    for (int q = 0; q < 5; ++q) ns[cnt++] = (uint32_t)(mix(seed++) & top);
    for (int q = 0; q < cnt; ++q) {
      const uint32_t n = ns[q];
      ++checked;
      if (idx::div_by_magic(n, m, sh) != n / d) {
        if (bad < 5) printf("d %u n %u: %u != %u\n", d, n, idx::div_by_magic(n, m, sh), n / d);
        ++bad;
      }
    }
  };
  for (uint32_t d = 1; d <= 70000; ++d) check_divisor(d);
  for (uint64_t i = 0; i < nrand; ++i) check_divisor(1u + (uint32_t)(mix(seed++) % top));
  for (int l = 0; l < 31; ++l) {  // powers of two and their neighbours
    const uint32_t p = 1u << l;
    check_divisor(p);
    if (p > 1) check_divisor(p - 1);
    if (p + 1 <= top) check_divisor(p + 1);
  }
  printf("mismatches %llu checked %llu\n", bad, checked);
  return bad == 0 ? 0 : 1;
}
