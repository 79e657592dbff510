// Radix-sort scratch of the tree build (the workspace's `hist` section): the
// digit counts of every pass over all particles (kSortMaxPasses x 256 words,
// cleared by the tree build's first launch), then per pass a ticket word and
// one look-back status word per (sort tile, digit), cleared by the keys
// kernel.
#pragma once

#include "common.cuh"

namespace p2p {

constexpr int kSortMaxPasses = 4;   // 3 * P2P_MAX_LEVEL key bits in digits of <= 8 bits
static_assert(3 * P2P_MAX_LEVEL <= 8 * kSortMaxPasses, "key bits beyond the reserved radix passes");
static_assert(P2P_MAX_N < (1LL << 30), "look-back counts hold 30 bits");
constexpr int64_t kSortCountWords = (int64_t)kSortMaxPasses * 256;
inline int64_t sort_pass_words(int radix, int tiles) { return 1 + (int64_t)radix * tiles; }
inline size_t sort_scratch_bytes(int tiles) {
    return (size_t)(kSortCountWords + kSortMaxPasses * sort_pass_words(256, tiles)) * 4;
}

// zero two 32-bit ranges in one launch
int clear2(void* a, int64_t na, void* b, int64_t nb, cudaStream_t s);

}  // namespace p2p
