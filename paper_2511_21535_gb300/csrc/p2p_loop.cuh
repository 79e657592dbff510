// The P2P compute loop shared by the gravity and Helmholtz kernels.
//
// Work unit: one warp owns one item = (target box b, up to 32*K of its
// targets), K targets per lane held in registers.  The warp streams the
// item's sources through a two-stage shared-memory ring filled by 1-D bulk
// asynchronous copies (cp.async.bulk, the TMA engine) that one lane issues
// while the warp computes the previous stage; an mbarrier per stage signals
// arrival.  Sources are read as ranges of 16-byte records:
//   redundant layout: one range, the box's contiguous stream (Section 5.2.1);
//   indirect layout:  one range per neighbour box in the box-ordered array.
// Items are taken from a global counter (persistent grid, longest-first
// order prepared by the restructuring pass).  Outputs are owned by exactly
// one warp, so no atomics touch results and the result does not depend on
// the schedule.
//
// The self pair is excluded by identity: each target knows the record index
// of its own copy inside the stream; only tiles that overlap the item's own
// window run the checking variant of the tile body.
#pragma once

#include "common.cuh"
#include "device.cuh"

namespace p2p {

constexpr int kLoopWarps = 4;          // warps per CTA
constexpr int kLoopThreads = 32 * kLoopWarps;
constexpr int kBarBytes = 64;          // per-warp slot for the two mbarriers

struct LoopArgs {
    const float4* rec;         // box-ordered records [n * words]
    const float4* red;         // redundant streams, or nullptr for the indirect layout
    int words;                 // 16-byte words per record
    int tile;                  // records per stage
    const int32_t* box_start;
    const int32_t* nbr_start;
    const int32_t* nbr_idx;
    const int32_t* red_start;
    const int32_t* red_self;
    const int2* items;
    Header* hdr;
};

inline size_t loop_smem_bytes(int tile, int words) {
    return (size_t)kLoopWarps * (2 * (size_t)tile * words * 16 + kBarBytes);
}

template <int K, class Op>
__device__ __forceinline__ void warp_item_loop(const LoopArgs& a, Op& op) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t stage_bytes = (uint32_t)a.tile * a.words * 16u;
    unsigned char* wb = smem_raw + (size_t)warp * (2 * stage_bytes + kBarBytes);
    float4* stage0 = reinterpret_cast<float4*>(wb);
    float4* stage1 = reinterpret_cast<float4*>(wb + stage_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(wb + 2 * stage_bytes);
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();

    if (a.hdr->flags & P2P_FLAG_CAPACITY) return;  // restructuring was skipped
    const int32_t n_items = a.hdr->n_items;
    const bool redundant = a.red != nullptr;
    const float4* base = redundant ? a.red : a.rec;
    uint32_t pseq = 0, cseq = 0;       // tiles issued / consumed by this warp

    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(&a.hdr->work_ctr, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= n_items) break;
        const int2 it = a.items[item];
        const int b = it.x, t0 = it.y;
        const int bs = a.box_start[b];
        const int nt = min(32 * K, a.box_start[b + 1] - bs - t0);

        // source ranges: lane r holds range r
        int nr, rs = 0, rc = 0, self_base;
        if (redundant) {
            nr = 1;
            rs = a.red_start[b];
            rc = a.red_start[b + 1] - rs;
            self_base = rs + a.red_self[b];
        } else {
            const int e0 = a.nbr_start[b];
            nr = a.nbr_start[b + 1] - e0;
            if (lane < nr) {
                const int c = a.nbr_idx[e0 + lane];
                rs = a.box_start[c];
                rc = a.box_start[c + 1] - rs;
            }
            self_base = bs;
        }
        const int sw_lo = self_base + t0, sw_hi = sw_lo + nt;
        op.begin(bs + t0, nt, sw_lo, lane);

        // producer and consumer cursors over (range, offset); empty ranges skipped
        int p_r = 0, p_o = 0, p_s = 0, p_c = 0;
        int c_r = 0, c_o = 0, c_s = 0, c_c = 0;
        while (p_r < nr) {
            p_s = __shfl_sync(FULL, rs, p_r);
            p_c = __shfl_sync(FULL, rc, p_r);
            if (p_c > 0) break;
            ++p_r;
        }
        c_r = p_r; c_s = p_s; c_c = p_c;

        auto issue = [&]() {
            const int cnt = min(a.tile, p_c - p_o);
            const uint32_t bytes = (uint32_t)cnt * (uint32_t)a.words * 16u;
            const int st = pseq & 1;
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect_tx(&bar[st], bytes);
                bulk_g2s(st ? stage1 : stage0, base + (int64_t)(p_s + p_o) * a.words, bytes, &bar[st]);
            }
            ++pseq;
            p_o += a.tile;
            if (p_o >= p_c) {
                p_o = 0;
                for (++p_r; p_r < nr; ++p_r) {
                    p_s = __shfl_sync(FULL, rs, p_r);
                    p_c = __shfl_sync(FULL, rc, p_r);
                    if (p_c > 0) break;
                }
            }
        };

        if (p_r < nr) issue();
        while (c_r < nr) {
            if (p_r < nr) issue();
            const int st = cseq & 1;
            if (!warp_wait(&bar[st], (cseq >> 1) & 1)) {
                // give up: flag, let copies in flight land (bounded), leave
                if (lane == 0) atomicOr(&a.hdr->flags, P2P_FLAG_TIMEOUT);
                for (uint32_t q = cseq; q < pseq; ++q) warp_wait(&bar[q & 1], (q >> 1) & 1);
                return;
            }
            const int cnt = min(a.tile, c_c - c_o);
            const int rec0 = c_s + c_o;
            const bool chk = rec0 < sw_hi && rec0 + cnt > sw_lo;
            op.tile(st ? stage1 : stage0, cnt, rec0, chk);
            __syncwarp();
            ++cseq;
            c_o += a.tile;
            if (c_o >= c_c) {
                c_o = 0;
                for (++c_r; c_r < nr; ++c_r) {
                    c_s = __shfl_sync(FULL, rs, c_r);
                    c_c = __shfl_sync(FULL, rc, c_r);
                    if (c_c > 0) break;
                }
            }
        }
        op.end(lane);
    }
}

// Kahan (compensated) summation step: add partial p into (s, c).
__device__ __forceinline__ void kahan_add(float& s, float& c, float p) {
    const float y = p - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

}  // namespace p2p
