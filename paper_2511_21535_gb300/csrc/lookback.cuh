// Single-pass chained scan across the blocks of one launch (decoupled
// look-back, Merrill & Garland, "Single-pass Parallel Prefix Scan with
// Decoupled Look-back", 2016).
//
// Each block takes a ticket as its tile index, so a tile only ever waits on
// tiles whose blocks are already running.  A tile publishes its aggregate,
// walks back over its predecessors' published values until it meets one that
// holds an inclusive prefix, then publishes its own inclusive prefix.  One
// status word per tile: (state << 32) | value, state 0 = nothing yet,
// 1 = aggregate, 2 = inclusive prefix.  Values are non-negative int32.
//
// Scratch: word 0 = ticket counter, word 1 + t = status of tile t; all zero
// before the launch.  Every wait is bounded: after kLookbackLimitNs the tile
// records P2P_FLAG_TIMEOUT and continues with what it has (the result is then
// wrong but flagged, and the launch ends).
#pragma once

#include "common.cuh"
#include "device.cuh"

namespace p2p {

constexpr unsigned long long kLbAggregate = 1ull << 32;
constexpr unsigned long long kLbPrefix = 2ull << 32;
constexpr uint64_t kLookbackLimitNs = 1000000000ull;

__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}
__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ int32_t warp_sum(int32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Thread 0 of the block: the tile index of this block.
__device__ __forceinline__ int lb_ticket(unsigned long long* lb) { return (int)atomicAdd(lb, 1ull); }

// Called by all 32 lanes of one warp of tile `tile` with the tile's aggregate
// `agg`: returns the sum of all earlier tiles' aggregates (in every lane).
__device__ __forceinline__ int32_t lb_exclusive(unsigned long long* lb, int tile, int32_t agg, Header* hdr) {
    unsigned long long* st = lb + 1;
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) lb_store(&st[0], kLbPrefix | (uint32_t)agg);
        return 0;
    }
    if (lane == 0) lb_store(&st[tile], kLbAggregate | (uint32_t)agg);
    int32_t excl = 0;
    int pred = tile - 1;
    const uint64_t t0 = global_ns();
    for (;;) {
        const int idx = pred - lane;
        unsigned long long v = kLbPrefix;            // before tile 0: an empty prefix
        bool expired = false;
        for (;;) {
            v = idx >= 0 ? lb_load(&st[idx]) : kLbPrefix;
            if (!__any_sync(FULL, (v >> 32) == 0ull)) break;
            expired = __shfl_sync(FULL, (lane == 0) && (global_ns() - t0 > kLookbackLimitNs), 0);
            if (expired) break;
        }
        if (expired) {
            if (lane == 0) atomicOr(&hdr->flags, P2P_FLAG_TIMEOUT);
            break;
        }
        const unsigned pm = __ballot_sync(FULL, (v >> 32) == 2ull);
        if (pm) {
            const int k = __ffs(pm) - 1;             // nearest predecessor holding a prefix
            excl += warp_sum(lane <= k ? (int32_t)(uint32_t)v : 0);
            break;
        }
        excl += warp_sum((int32_t)(uint32_t)v);
        pred -= 32;
    }
    if (lane == 0) lb_store(&st[tile], kLbPrefix | (uint32_t)(excl + agg));
    return excl;
}

}  // namespace p2p
