// Record copies of the restructuring (the redundant gather and the pair-task
// stream): 16-byte words, streamed stores (the data is read later by the bulk
// copies of the P2P kernels).  A periodic image code other than 13 moves the
// positions (word 0: x, y, z) by the image offset times the domain edge.
#pragma once

#include "common.cuh"

namespace p2p {

// A record's first word (x, y, z) moved to the periodic image `code`
// ((ox+1) + 3(oy+1) + 9(oz+1); 13: no move) of a domain of edge `edge`.
__device__ __forceinline__ float4 image_shifted(float4 v, int32_t code, float edge) {
    if (code != 13) {
        v.x += (float)(code % 3 - 1) * edge;
        v.y += (float)((code / 3) % 3 - 1) * edge;
        v.z += (float)(code / 9 - 1) * edge;
    }
    return v;
}

// One warp copies cnt records of `words` 16-byte words from src to dst
// (coalesced, eight loads in flight per lane).
__device__ __forceinline__ void warp_copy_records(const float4* __restrict__ src, float4* __restrict__ dst,
                                                  int32_t cnt, int words, int lane, int32_t code, float edge) {
    if (code != 13) {
        for (int32_t l = lane; l < cnt; l += 32) {
            __stcs(dst + (int64_t)l * words, image_shifted(__ldg(src + (int64_t)l * words), code, edge));
            for (int w = 1; w < words; ++w) __stcs(dst + (int64_t)l * words + w, __ldg(src + (int64_t)l * words + w));
        }
        return;
    }
    const int64_t nw = (int64_t)cnt * words;
    int64_t w = lane;
    for (; w + 224 < nw; w += 256) {  // eight independent 16-byte loads in flight per lane
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(src + w + 32 * u);
#pragma unroll
        for (int u = 0; u < 8; ++u) __stcs(dst + w + 32 * u, v[u]);
    }
    // the last (up to seven) rounds: their loads issued together, then the stores
    float4 v[7];
#pragma unroll
    for (int u = 0; u < 7; ++u)
        if (w + 32 * u < nw) v[u] = __ldg(src + w + 32 * u);
#pragma unroll
    for (int u = 0; u < 7; ++u)
        if (w + 32 * u < nw) __stcs(dst + w + 32 * u, v[u]);
}

}  // namespace p2p
