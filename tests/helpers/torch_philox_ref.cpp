// Prints Philox4x32-10 output words computed by PyTorch's header-only engine
// (ATen/core/PhiloxRNGEngine.h), an implementation independent of this
// repository's.  Input lines: "seed c0 c1 c2 c3" (decimal); output lines: the
// four 32-bit words.  The engine keys on the seed and places `offset` in
// counter words (0,1) and `subsequence` in counter words (2,3).
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>

int main() {
  unsigned long long seed, c0, c1, c2, c3;
  while (std::scanf("%llu %llu %llu %llu %llu", &seed, &c0, &c1, &c2, &c3) == 5) {
    uint64_t offset = (uint64_t)c0 | ((uint64_t)c1 << 32);
    uint64_t subseq = (uint64_t)c2 | ((uint64_t)c3 << 32);
    at::philox_engine eng(seed, subseq, offset);
    uint32_t a = eng(), b = eng(), c = eng(), d = eng();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
