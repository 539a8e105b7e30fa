// Library reference for the Philox4x32-10 pin: runs PyTorch's ATen Philox4_32
// engine (a library routine, header-only) on counters/keys read from stdin.
// Input lines: c0 c1 c2 c3 k0 k1 (decimal); output lines: four hex words.
// at::Philox4_32(seed, subsequence, offset) draws from counter
// (offset_lo, offset_hi, subsequence_lo, subsequence_hi) with key (seed_lo, seed_hi).
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>

int main() {
  unsigned long long c0, c1, c2, c3, k0, k1;
  while (std::scanf("%llu %llu %llu %llu %llu %llu", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    const uint64_t seed = (k1 << 32) | k0;
    const uint64_t subsequence = (c3 << 32) | c2;
    const uint64_t offset = (c1 << 32) | c0;
    at::Philox4_32 eng(seed, subsequence, offset);
    const uint32_t a = eng(), b = eng(), c = eng(), d = eng();
    std::printf("%08x %08x %08x %08x\n", a, b, c, d);
  }
  return 0;
}
