// Test helper: prints Philox4x32-10 outputs computed by PyTorch's header-only
// ATen engine (at::Philox4_32), an implementation independent of the oracle.
// stdin: lines "k0 k1 c0 c1 c2 c3" (decimal uint32); stdout: "x0 x1 x2 x3".
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>

int main() {
    unsigned long long k0, k1, c0, c1, c2, c3;
    while (std::scanf("%llu %llu %llu %llu %llu %llu", &k0, &k1, &c0, &c1, &c2, &c3) == 6) {
        uint64_t seed = k0 | (k1 << 32);
        uint64_t subsequence = c2 | (c3 << 32);
        uint64_t offset = c0 | (c1 << 32);
        at::Philox4_32 eng(seed, subsequence, offset);
        uint32_t a = eng(), b = eng(), c = eng(), d = eng();
        std::printf("%u %u %u %u\n", a, b, c, d);
    }
    return 0;
}
