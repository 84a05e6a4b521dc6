// Test helper: prints Philox4x32-10 blocks computed by PyTorch's host-side
// at::Philox4_32 engine, an implementation independent of the oracle's.
// Input lines on stdin: "seed subsequence offset"; output: four words in hex.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cinttypes>

int main() {
    unsigned long long seed, subseq, offset;
    while (std::scanf("%llu %llu %llu", &seed, &subseq, &offset) == 3) {
        at::Philox4_32 eng(seed, subseq, offset);
        uint32_t r0 = eng(), r1 = eng(), r2 = eng(), r3 = eng();
        std::printf("%08" PRIx32 " %08" PRIx32 " %08" PRIx32 " %08" PRIx32 "\n", r0, r1, r2, r3);
    }
    return 0;
}
