// The P2P compute loop shared by the gravity and Helmholtz kernels.
//
// Work unit: one item = (target box b, up to 32*K of its targets), K targets
// per lane held in registers, processed by a group of G warps (G = 1, 2 or
// 4).  Every warp of the group holds the same targets; the item's source
// tiles are dealt round-robin to the group's warps, and at the end the warps'
// partial sums are added in warp order through shared memory (deterministic).
// Several warps per item give the persistent grid several items per worker,
// which is what keeps the SMs evenly loaded when items are few and equal.
//
// Each warp streams its tiles through a two-stage shared-memory ring filled
// by 1-D bulk asynchronous copies (cp.async.bulk, the TMA engine) that one
// lane issues while the warp computes the previous stage; an mbarrier per
// stage signals arrival.  Sources are read as ranges of 16-byte records:
//   redundant layout: one range, the box's contiguous stream (Section 5.2.1);
//   indirect layout:  one range per neighbour box in the box-ordered array;
//   pair tasks:       an item is (task e = (b, c), targets); its targets and
//                     its one source range both come from the task's block
//                     [records of b | records of c], and its results go to
//                     the task's own partial-result slots (reduced later);
//   symmetric tasks:  as pair tasks, but a mutual task evaluates each pair of
//                     its unordered box pair once and also credits the
//                     sources (the op's B-side sums, written per source to
//                     the slots after the targets'); a self task's block is
//                     the box alone.
// Items are taken from a global counter (persistent grid, longest-first
// order prepared by the restructuring pass).  Outputs are owned by exactly
// one group, so no atomics touch results and the result does not depend on
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
    const int32_t* nbr_img;    // periodic indirect layout: image code per neighbour entry, else nullptr
    float edge;                // domain edge (periodic image shifts)
    const int32_t* ent_box;    // pair tasks: target box of each task (entry), else nullptr
    const int32_t* pt_start;   // pair tasks: record block of each task in the task stream (red)
    const int32_t* part_start; // pair tasks: first partial-result slot of each task
    void* part;                // pair tasks: partial results
    int64_t part_cap;          // pair tasks: slots per right-hand side
    const int32_t* task_kind;  // symmetric tasks: 0 none, 1 self, 2 mutual, 3 one-sided; else nullptr
    const int32_t* bslot;      // symmetric plans (target-owned layouts): source-sum slots per entry
    // capacities (checked builds verify every item against them)
    int64_t rec_cap;           // records in rec
    int64_t red_cap;           // records in red
    int64_t items_cap;         // work items
    int64_t box_cap;           // boxes
    int64_t n;                 // particles (output indices)
};


// dynamic shared memory: per warp two stages + mbarriers, then (G > 1) the
// partial-sum exchange area of `outs` floats per lane, then (ops with
// mutual tasks) per warp the B-side sums of one tile, `mut` floats a source
inline size_t loop_smem_bytes(int tile, int words, int outs, int group, int mut = 0) {
    size_t b = (size_t)kLoopWarps * (2 * (size_t)tile * words * 16 + kBarBytes);
    if (group > 1) b += (size_t)kLoopWarps * 32 * outs * sizeof(float);
    b += (size_t)kLoopWarps * tile * mut * sizeof(float);
    return b;
}

// position in the item's tile sequence: range r, offset o; (s, c) = range start/count
struct TileCursor {
    int r, o, s, c;
    __device__ __forceinline__ void settle(int nr, int rs, int rc) {  // first non-empty range from r on
        for (; r < nr; ++r) {
            s = __shfl_sync(FULL, rs, r);
            c = __shfl_sync(FULL, rc, r);
            if (c > 0) break;
        }
    }
    __device__ __forceinline__ void next(int nr, int rs, int rc, int tile) {
        o += tile;
        if (o >= c) {
            o = 0;
            ++r;
            settle(nr, rs, rc);
        }
    }
};

template <int G>
__device__ __forceinline__ void group_sync(int group) {
    if (G == 1) __syncwarp();
    else if (G == kLoopWarps) __syncthreads();
    else named_bar_sync(1 + group, 32 * G);
}

template <int K, int G, class Op>
__device__ __forceinline__ void warp_item_loop(const LoopArgs& a, Op& op) {
    static_assert(G == 1 || G == 2 || G == 4, "group size");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int item_slot[kLoopWarps];
    __shared__ volatile int abort_flag[kLoopWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int group = warp / G, gw = warp % G;
    const uint32_t stage_bytes = (uint32_t)a.tile * a.words * 16u;
    unsigned char* wb = smem_raw + (size_t)warp * (2 * stage_bytes + kBarBytes);
    float4* stage0 = reinterpret_cast<float4*>(wb);
    float4* stage1 = reinterpret_cast<float4*>(wb + stage_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(wb + 2 * stage_bytes);
    float* partial = reinterpret_cast<float*>(smem_raw + (size_t)kLoopWarps * (2 * stage_bytes + kBarBytes));
    if constexpr (Op::kMutFloats > 0) {
        float* mut_area = partial + (G > 1 ? (size_t)kLoopWarps * 32 * Op::kOuts : 0);
        op.set_scratch(mut_area + (size_t)warp * a.tile * Op::kMutFloats);
    }
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        if (gw == 0) abort_flag[group] = 0;
    }
    __syncwarp();

    if (a.hdr->flags & (P2P_FLAG_CAPACITY | P2P_FLAG_LATTICE)) return;  // inputs rejected (uniform)
    const int32_t n_items = a.hdr->n_items;
    const bool pairtask = a.ent_box != nullptr;
    const bool redundant = a.red != nullptr;   // also the pair-task stream
    const float4* base = redundant ? a.red : a.rec;
    uint32_t pseq = 0, cseq = 0;       // tiles issued / consumed by this warp

    for (;;) {
        int item = 0;
        if (G == 1) {
            if (lane == 0) item = (int)atomicAdd(&a.hdr->work_ctr, 1u);
            item = __shfl_sync(FULL, item, 0);
        } else {
            if (gw == 0 && lane == 0) item_slot[group] = (int)atomicAdd(&a.hdr->work_ctr, 1u);
            group_sync<G>(group);
            item = item_slot[group];
            if (abort_flag[group]) item = n_items;
        }
        if (item >= n_items) break;
        if constexpr (kChecked) {
            if (!dcheck(item < a.items_cap, a.hdr)) break;   // item is the same in every warp of the group
        }
        const int2 it = a.items[item];
        const int t0 = it.y;
        if constexpr (kChecked) {
            if (!dcheck(it.x >= 0 && it.x < (pairtask ? a.hdr->n_nbr : a.hdr->n_boxes), a.hdr)) continue;
        }
        const int b = pairtask ? a.ent_box[it.x] : it.x;
        if constexpr (kChecked) {
            if (!dcheck(b >= 0 && b < a.hdr->n_boxes, a.hdr)) continue;
        }
        const int bs = a.box_start[b];
        const int nbox = a.box_start[b + 1] - bs;
        const int nt = min(32 * K, nbox - t0);

        // source ranges: lane r holds range r (and its image code, periodic indirect;
        // its task kind and source-sum slots, symmetric plans)
        int nr, rs = 0, rc = 0, ri = 13, rk = kTaskOneSided, rb = 0, self_base, tgt = bs + t0;
        const bool sym = a.task_kind != nullptr && !pairtask;
        int64_t slot = 0;
        bool mutual = false;
        if (pairtask) {
            const int e = it.x, tb = a.pt_start[e];
            const int kind = a.task_kind ? a.task_kind[e] : kTaskOneSided;
            nr = 1;
            if (kind == kTaskSelf) {   // the block is the box itself: sources = targets
                rs = tb;
                rc = nbox;
                self_base = tb;
            } else {
                rs = tb + nbox;
                rc = a.pt_start[e + 1] - rs;
                // plain pair tasks: only the task of the box with itself holds the targets' own copies
                self_base = (kind == kTaskOneSided && a.nbr_idx[e] == b) ? rs : -(1 << 30);
            }
            mutual = kind == kTaskMutual;   // a single item (t0 = 0): the B-side slots follow the targets'
            tgt = tb + t0;
            slot = (int64_t)a.part_start[e] + t0;
        } else if (redundant && !sym) {
            nr = 1;
            rs = a.red_start[b];
            rc = a.red_start[b + 1] - rs;
            self_base = rs + a.red_self[b];
        } else {
            // one range per neighbour entry (symmetric: entries without a task are empty)
            const int e0 = a.nbr_start[b];
            nr = a.nbr_start[b + 1] - e0;
            if (lane < nr) {
                const int c = a.nbr_idx[e0 + lane];
                rs = a.box_start[c];
                rc = a.box_start[c + 1] - rs;
                if (a.nbr_img) ri = a.nbr_img[e0 + lane];
                if (sym) {
                    rk = a.task_kind[e0 + lane];
                    rb = a.bslot[e0 + lane];
                    if (rk == kTaskNone) rc = 0;
                }
            }
            self_base = bs;
            if (redundant) {   // symmetric streams hold the streamed entries back to back
                const int inc = warp_incl_scan(rc);
                rs = a.red_start[b] + inc - rc;
                self_base = a.red_start[b] + a.red_self[b];
            }
        }
        if constexpr (kChecked) {
            // every range inside the buffer it is copied from, the targets and slots inside theirs
            const int64_t bufcap = redundant ? a.red_cap : a.rec_cap;
            bool good = b < a.box_cap && t0 >= 0 && nt > 0 &&
                        tgt >= 0 && (int64_t)tgt + nt <= (pairtask ? a.red_cap : a.rec_cap);
            const bool range_ok = lane >= nr || rc == 0 || (rs >= 0 && (int64_t)rs + rc <= bufcap);
            const bool slot_ok = !sym || lane >= nr || rk != kTaskMutual || (rb >= 0 && (int64_t)rb + rc <= a.part_cap);
            good = __all_sync(FULL, range_ok && slot_ok) && good;
            if (pairtask) good = good && slot + nt <= a.part_cap && (!mutual || slot + nbox + rc <= a.part_cap);
            if (!dcheck(good, a.hdr)) continue;   // the same decision in every warp of the group
        }
        const int sw_lo = self_base + t0, sw_hi = sw_lo + nt;

        // this warp's tiles: gw, gw + G, gw + 2G, ... of the item's tile sequence
        TileCursor pc{0, 0, 0, 0};
        pc.settle(nr, rs, rc);
        for (int g = 0; g < gw && pc.r < nr; ++g) pc.next(nr, rs, rc, a.tile);
        TileCursor cc = pc;

        auto issue = [&]() {
            const int cnt = min(a.tile, pc.c - pc.o);
            const uint32_t bytes = (uint32_t)cnt * (uint32_t)a.words * 16u;
            const int st = pseq & 1;
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect_tx(&bar[st], bytes);
                bulk_g2s(st ? stage1 : stage0, base + (int64_t)(pc.s + pc.o) * a.words, bytes, &bar[st]);
            }
            ++pseq;
            for (int g = 0; g < G && pc.r < nr; ++g) pc.next(nr, rs, rc, a.tile);
        };

        // the item's first tile is in flight while the op loads its targets (both
        // stages are free between items: every issued tile has been consumed)
        if (pc.r < nr) issue();
        op.begin(tgt, nt, sw_lo, lane);
        if constexpr (Op::kMutFloats > 0) {
            if (pairtask) op.set_range(mutual, slot + nbox, rs);
        }
        bool failed = false;
        int cur_r = -1;   // range whose per-range state (image shift, task kind) the op holds
        const bool per_range = a.nbr_img != nullptr || (Op::kMutFloats > 0 && sym);
        while (cc.r < nr) {
            if (pc.r < nr) issue();
            if (per_range && cc.r != cur_r) {
                cur_r = cc.r;
                if (a.nbr_img) {
                    // periodic: meet this neighbour's image by moving the targets the other way
                    const int code = __shfl_sync(FULL, ri, cc.r);
                    op.set_shift((float)(code % 3 - 1) * a.edge, (float)((code / 3) % 3 - 1) * a.edge,
                                 (float)(code / 9 - 1) * a.edge);
                }
                if constexpr (Op::kMutFloats > 0) {
                    if (sym) {
                        const int k = __shfl_sync(FULL, rk, cc.r);
                        const int slot_b = __shfl_sync(FULL, rb, cc.r);
                        op.set_range(k == kTaskMutual, slot_b, cc.s);
                    }
                }
            }
            const int st = cseq & 1;
            if (!warp_wait(&bar[st], (cseq >> 1) & 1)) {
                failed = true;
                break;
            }
            const int cnt = min(a.tile, cc.c - cc.o);
            const int rec0 = cc.s + cc.o;
            const bool chk = rec0 < sw_hi && rec0 + cnt > sw_lo;
            op.tile(st ? stage1 : stage0, cnt, rec0, chk);
            __syncwarp();
            ++cseq;
            for (int g = 0; g < G && cc.r < nr; ++g) cc.next(nr, rs, rc, a.tile);
        }
        if (failed) {
            // give up: flag, let copies in flight land (bounded), leave after this item
            if (lane == 0) atomicOr(&a.hdr->flags, P2P_FLAG_TIMEOUT);
            for (uint32_t q = cseq; q < pseq; ++q) warp_wait(&bar[q & 1], (q >> 1) & 1);
            if (G == 1) return;
            if (lane == 0) abort_flag[group] = 1;
        }
        auto finish = [&]() {
            if constexpr (Op::kPartial) {
                if (pairtask) {
                    op.end_partial(lane, a.part, a.part_cap, slot);
                    return;
                }
            }
            op.end(lane);
        };
        if (G == 1) {
            finish();
        } else {
            float* mine = partial + (size_t)warp * Op::kOuts * 32;
            if (gw != 0) op.store_partial(mine, lane);
            group_sync<G>(group);
            if (gw == 0) {
                op.fold();
                for (int w = 1; w < G; ++w) op.add_partial(mine + (size_t)w * Op::kOuts * 32, lane);
                finish();
            }
            group_sync<G>(group);
            if (abort_flag[group]) return;
        }
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
