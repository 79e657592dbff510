// Pair-task layout: the thread-level form of the redundant design
// (Section 5.2.1) with results duplicated and reduced afterwards (Section
// 1.1).
//
// One task per neighbour-list entry e = (b, c), target box b, source box c.
// The task stream holds, per task, the block [records of b | records of c]
// (both attributes of the interaction in one contiguous block: array of
// structures); pt_start[e] is the block's first record.  The P2P kernel
// computes task e's sums for b's targets over c's sources only and writes
// them to the task's partial-result slots part_start[e] + t (t = target in
// b).  The update step then adds, per target, the partials of b's tasks in
// neighbour-list order: a fixed order, so the result is deterministic and
// no two workers ever write the same output.
//
// Symmetric tasks (P2P_LAYOUT_SYMMETRIC) keep one task per unordered box
// pair where one of the two boxes fits a work item: that "mutual" task sits
// in the list of the lane box (the smaller index, else the other one), its
// block is [lane box | other box], and its slots are the lane box's targets
// followed by the other box's particles.  The mirror entry holds no task; the
// reduction reads the other box's slots of the mutual task there.  Pairs of
// two large boxes keep one one-sided task per direction; every box has a
// self task whose block is the box alone.
#include <algorithm>

#include "common.cuh"
#include "copy.cuh"
#include "device.cuh"

namespace p2p {

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// per entry: its target box, the block length and the slot count (plain
// pair tasks: n_b + n_c and n_b); symmetric tasks also get their kind and,
// for entries without a task, the mirror entry (c -> b) in c's list
__global__ void __launch_bounds__(256) k_pt_entries(const int32_t* __restrict__ box_start,
                                                   const int32_t* __restrict__ nbr_start,
                                                   const int32_t* __restrict__ nbr_idx, Header* hdr,
                                                   int32_t* __restrict__ ent_box, int32_t* __restrict__ blk_len,
                                                   int32_t* __restrict__ slot_len, int32_t* __restrict__ task_kind,
                                                   int32_t* __restrict__ mirror) {
    pdl_wait();
    pdl_release();
    if (hdr->flags & P2P_FLAG_CAPACITY) return;   // an inconsistent imported structure
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = hdr->n_boxes;
    for (int64_t b = warp; b < nb; b += nwarps) {
        const int32_t occ = box_start[b + 1] - box_start[b];
        for (int32_t e = nbr_start[b] + lane; e < nbr_start[b + 1]; e += 32) {
            const int32_t c = nbr_idx[e];
            const int32_t nc = box_start[c + 1] - box_start[c];
            ent_box[e] = (int32_t)b;
            if (!task_kind) {
                blk_len[e] = occ + nc;
                slot_len[e] = occ;
                continue;
            }
            int32_t kind, mir = -1;
            if (c == b) {
                kind = kTaskSelf;
            } else {
                const int32_t lo = min((int32_t)b, c), hi = max((int32_t)b, c);
                const int32_t nlo = (lo == b) ? occ : nc, nhi = (hi == b) ? occ : nc;
                const int32_t lane_box = nlo <= kMutualMax ? lo : (nhi <= kMutualMax ? hi : -1);
                kind = lane_box < 0 ? kTaskOneSided : (lane_box == b ? kTaskMutual : kTaskNone);
                if (kind == kTaskNone) {   // find b in c's ascending list
                    int32_t l = nbr_start[c], h = nbr_start[c + 1];
                    while (l < h) {
                        const int32_t m = (l + h) >> 1;
                        if (nbr_idx[m] < b) l = m + 1;
                        else h = m;
                    }
                    if (l < nbr_start[c + 1] && nbr_idx[l] == b) mir = l;
                    else atomicOr(&hdr->flags, P2P_FLAG_CAPACITY);   // an inconsistent (imported) relation
                }
            }
            task_kind[e] = kind;
            mirror[e] = mir;
            // the statistics counted every entry's work; a mirror entry's pairs are evaluated by its mutual task
            if (kind == kTaskNone) atomicAdd(&hdr->evals_nS, 0ull - (unsigned long long)occ * (unsigned long long)nc);
            blk_len[e] = kind == kTaskNone ? 0 : (kind == kTaskSelf ? occ : occ + nc);
            slot_len[e] = kind == kTaskNone ? 0 : (kind == kTaskMutual ? occ + nc : occ);
        }
    }
}

// The task stream: per task [records of b | records of c (at its periodic
// image)] (symmetric self tasks: [records of b]; entries without a task:
// nothing).  The copies wait on dependent loads (the entry, its boxes'
// bounds, the records), so a warp takes 32 consecutive tasks at once, lane i
// task i: their blocks are contiguous in the stream, and the blocks of at
// most kPtFlatMax records are copied flat (in each round lane l takes
// position 32 r + l of the small blocks, finds its task by a binary search
// over the blocks' offsets held in the lanes, and the round's loads are
// issued before its stores, which are coalesced); larger blocks are copied
// afterwards, one at a time by the whole warp (eight loads in flight per
// lane), the warps taking the tasks strided.
// W: words per record when known at compile time (1, 2), else 0.
constexpr int32_t kPtFlatMax = 64;

// task e's block: b's records (sb, nb) then c's (sc, nc, image code), at out
struct PtBlock {
    int32_t sb, nb, sc, nc, code, out;
};

__device__ __forceinline__ PtBlock pt_block(int64_t e, int32_t ne, const int32_t* __restrict__ box_start,
                                            const int32_t* __restrict__ nbr_idx, const int32_t* __restrict__ ent_box,
                                            const int32_t* __restrict__ nbr_img, const int32_t* __restrict__ pt_start,
                                            const int32_t* __restrict__ task_kind) {
    PtBlock t{0, 0, 0, 0, 13, 0};
    if (e < ne) {
        const int32_t kind = task_kind ? task_kind[e] : kTaskOneSided;
        t.out = pt_start[e];
        if (kind != kTaskNone) {
            const int32_t b = ent_box[e], c = nbr_idx[e];
            t.sb = box_start[b];
            t.nb = box_start[b + 1] - t.sb;
            if (kind != kTaskSelf) {
                t.sc = box_start[c];
                t.nc = box_start[c + 1] - t.sc;
            }
            if (nbr_img) t.code = nbr_img[e];
        }
    }
    return t;
}

template <int W>
__global__ void __launch_bounds__(256) k_pt_gather(const float4* __restrict__ rec, int words,
                                                  const int32_t* __restrict__ box_start,
                                                  const int32_t* __restrict__ nbr_idx,
                                                  const int32_t* __restrict__ ent_box,
                                                  const int32_t* __restrict__ nbr_img, float edge,
                                                  const int32_t* __restrict__ pt_start, Header* hdr, int64_t cap,
                                                  int64_t part_cap, float4* __restrict__ pt,
                                                  uint32_t* __restrict__ gather, const int32_t* __restrict__ task_kind) {
    pdl_wait();
    pdl_release();
    const int lane = threadIdx.x & 31;
    // an imported, inconsistent neighbour relation can exceed the capacities
    if ((hdr->flags & P2P_FLAG_CAPACITY) || hdr->total_src < 0 || (int64_t)hdr->total_src > cap || hdr->part_total < 0 ||
        (int64_t)hdr->part_total > part_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&hdr->flags, P2P_FLAG_CAPACITY);
        return;
    }
    const int wd = W > 0 ? W : words;
    constexpr int WV = W > 0 ? W : 1;      // words loaded before the stores
    constexpr int RU = W == 1 ? 4 : 2;     // rounds per step
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t ne = hdr->n_nbr;
    for (int64_t e0 = warp * 32; e0 < ne; e0 += nwarps * 32) {
        const PtBlock t = pt_block(e0 + lane, ne, box_start, nbr_idx, ent_box, nbr_img, pt_start, task_kind);
        const int32_t sb = t.sb, nbk = t.nb, sc = t.sc, code = t.code, out = t.out;
        const int32_t blk = t.nb + t.nc;
        const bool big = blk > kPtFlatMax;
        const int32_t fl = big ? 0 : blk;
        const int32_t inc = warp_incl_scan(fl), excl = inc - fl;
        const int32_t total = __shfl_sync(FULL, inc, 31);
        // the small blocks, flat
        for (int32_t p0 = 0; p0 < total; p0 += 32 * RU) {
            float4 v[RU][WV];
            int32_t src[RU], dst[RU], cd[RU];
#pragma unroll
            for (int q = 0; q < RU; ++q) {
                const int32_t p = p0 + 32 * q + lane;
                int j = 0;   // the last task whose small block starts at or before p
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int cand = j + st;   // <= 31
                    if (__shfl_sync(FULL, excl, cand) <= p) j = cand;
                }
                const int32_t o = p - __shfl_sync(FULL, excl, j), nbj = __shfl_sync(FULL, nbk, j);
                const int32_t sbj = __shfl_sync(FULL, sb, j), scj = __shfl_sync(FULL, sc, j);
                const int32_t cdj = __shfl_sync(FULL, code, j);
                const bool second = o >= nbj;   // c's part of the block
                src[q] = second ? scj + (o - nbj) : sbj + o;
                dst[q] = __shfl_sync(FULL, out, j) + o;
                cd[q] = second ? cdj : 13;
                if (p < total) {
#pragma unroll
                    for (int w = 0; w < WV; ++w) v[q][w] = __ldg(rec + (int64_t)src[q] * wd + w);
                }
            }
#pragma unroll
            for (int q = 0; q < RU; ++q) {
                if (p0 + 32 * q + lane >= total) continue;
                float4* o = pt + (int64_t)dst[q] * wd;
                __stcs(o, image_shifted(v[q][0], cd[q], edge));
#pragma unroll
                for (int w = 1; w < WV; ++w) __stcs(o + w, v[q][w]);
                if (W == 0)
                    for (int w = 1; w < wd; ++w) __stcs(o + w, __ldg(rec + (int64_t)src[q] * wd + w));
                if (gather) gather[dst[q]] = (uint32_t)src[q];
            }
        }
    }
    // the large blocks, one at a time with the whole warp: tasks warp + nwarps k,
    // examined 32 at a time (lane l: k = 32 i + l), so that the large tasks of a
    // region of big boxes are spread over the warps
    for (int64_t base = warp; base < ne; base += 32 * nwarps) {
        const PtBlock t = pt_block(base + (int64_t)lane * nwarps, ne, box_start, nbr_idx, ent_box, nbr_img, pt_start,
                                   task_kind);
        unsigned bm = __ballot_sync(FULL, t.nb + t.nc > kPtFlatMax);
        while (bm) {
            const int j = __ffs(bm) - 1;
            bm &= bm - 1;
            const int32_t sbj = __shfl_sync(FULL, t.sb, j), nbj = __shfl_sync(FULL, t.nb, j);
            const int32_t scj = __shfl_sync(FULL, t.sc, j), ncj = __shfl_sync(FULL, t.nc, j);
            const int32_t cdj = __shfl_sync(FULL, t.code, j);
            const int64_t oj = __shfl_sync(FULL, t.out, j);
            warp_copy_records(rec + (int64_t)sbj * wd, pt + oj * wd, nbj, wd, lane, 13, edge);
            warp_copy_records(rec + (int64_t)scj * wd, pt + (oj + nbj) * wd, ncj, wd, lane, cdj, edge);
            if (gather) {
                for (int32_t l = lane; l < nbj; l += 32) gather[oj + l] = (uint32_t)(sbj + l);
                for (int32_t l = lane; l < ncj; l += 32) gather[oj + nbj + l] = (uint32_t)(scj + l);
            }
        }
    }
}

int pairtask_restructure(Plan* p, void* ws, int words, cudaStream_t s) {
    const Layout& L = p->L;
    Header* hdr = at<Header>(ws, L.header);
    const int64_t ecap = 27 * p->box_cap;
    int32_t* ent_box = at<int32_t>(ws, L.ent_box);
    int32_t* pt_start = at<int32_t>(ws, L.pt_start);
    int32_t* part_start = at<int32_t>(ws, L.part_start);
    const unsigned wb = (unsigned)std::min<int64_t>(blocks_for(p->box_cap * 32, 256), (int64_t)num_sms() * 16);
    const bool sym = p->layout == P2P_LAYOUT_SYMMETRIC;
    int32_t* kind = sym ? at<int32_t>(ws, L.task_kind) : nullptr;
    P2P_CUDA_TRY(launch_pdl(k_pt_entries, wb, 256, 0, s, at<int32_t>(ws, L.box_start), at<int32_t>(ws, L.nbr_start),
                            at<int32_t>(ws, L.nbr_idx), hdr, ent_box, pt_start, part_start, kind,
                            sym ? at<int32_t>(ws, L.mirror) : nullptr));
    P2P_LAUNCH_CHECK();
    int st = scan_exclusive(pt_start, pt_start, ecap, &hdr->n_nbr, &hdr->total_src, at<int32_t>(ws, L.scan_tmp), s);
    if (st) return st;
    st = scan_exclusive(part_start, part_start, ecap, &hdr->n_nbr, &hdr->part_total, at<int32_t>(ws, L.scan_tmp), s);
    if (st) return st;
    auto gk = words == 1 ? k_pt_gather<1> : words == 2 ? k_pt_gather<2> : k_pt_gather<0>;
    P2P_CUDA_TRY(launch_pdl(gk, num_sms() * 8, 256, 0, s, at<float4>(ws, L.src), words, at<int32_t>(ws, L.box_start),
                                            at<int32_t>(ws, L.nbr_idx), ent_box,
                                            p->periodic ? at<int32_t>(ws, L.nbr_img) : nullptr, p->edge, pt_start,
                                            hdr, p->red_cap, p->part_cap, at<float4>(ws, L.red_src),
                                            (p->flags & P2P_PLAN_GATHER_MAP) ? at<uint32_t>(ws, L.gather) : nullptr,
                                            kind));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

// First partial slot of box b's contribution from its neighbour entry e: the
// entry's own task, or (symmetric, no task there) the other-box slots of the
// mirror entry's mutual task, which follow that task's lane-box slots.
__device__ __forceinline__ int64_t contrib_slot(int32_t e, const int32_t* __restrict__ part_start,
                                                const int32_t* __restrict__ task_kind,
                                                const int32_t* __restrict__ mirror,
                                                const int32_t* __restrict__ nbr_idx,
                                                const int32_t* __restrict__ box_start) {
    if (!task_kind || task_kind[e] != kTaskNone) return part_start[e];
    const int32_t c = nbr_idx[e];
    return (int64_t)part_start[mirror[e]] + (box_start[c + 1] - box_start[c]);
}

// Update: per target, the partials of its box's tasks in neighbour order,
// compensated, then scattered to original order.  One warp per box.
__global__ void __launch_bounds__(256) k_pt_reduce_gravity(const int32_t* __restrict__ box_start,
                                                          const int32_t* __restrict__ nbr_start,
                                                          const int32_t* __restrict__ part_start,
                                                          const int32_t* __restrict__ perm, const Header* hdr,
                                                          const float4* __restrict__ part, float* __restrict__ phi,
                                                          float* __restrict__ acc,
                                                          const int32_t* __restrict__ task_kind,
                                                          const int32_t* __restrict__ mirror,
                                                          const int32_t* __restrict__ nbr_idx) {
    pdl_wait();
    pdl_release();
    if (hdr->flags & (P2P_FLAG_CAPACITY | P2P_FLAG_TIMEOUT)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = hdr->n_boxes;
    for (int64_t b = warp; b < nb; b += nwarps) {
        const int32_t bs = box_start[b], occ = box_start[b + 1] - bs;
        const int32_t e0 = nbr_start[b], e1 = nbr_start[b + 1];
        for (int32_t l = lane; l < occ; l += 32) {
            float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
            for (int32_t e = e0; e < e1; ++e) {
                const float4 v = part[contrib_slot(e, part_start, task_kind, mirror, nbr_idx, box_start) + l];
                const float in[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const float y = in[o] - c[o];
                    const float t = s[o] + y;
                    c[o] = (t - s[o]) - y;
                    s[o] = t;
                }
            }
            const int64_t o = perm[bs + l];
            phi[o] = -(s[0] - c[0]);
            acc[3 * o + 0] = s[1] - c[1];
            acc[3 * o + 1] = s[2] - c[2];
            acc[3 * o + 2] = s[3] - c[3];
        }
    }
}

__global__ void __launch_bounds__(256) k_pt_reduce_helmholtz(const int32_t* __restrict__ box_start,
                                                            const int32_t* __restrict__ nbr_start,
                                                            const int32_t* __restrict__ part_start,
                                                            const int32_t* __restrict__ perm, const Header* hdr,
                                                            const float2* __restrict__ part, int64_t cap, int nrhs,
                                                            int64_t n, float2* __restrict__ u,
                                                            const int32_t* __restrict__ task_kind,
                                                            const int32_t* __restrict__ mirror,
                                                            const int32_t* __restrict__ nbr_idx) {
    pdl_wait();
    pdl_release();
    if (hdr->flags & (P2P_FLAG_CAPACITY | P2P_FLAG_TIMEOUT)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = hdr->n_boxes;
    for (int64_t b = warp; b < nb; b += nwarps) {
        const int32_t bs = box_start[b], occ = box_start[b + 1] - bs;
        const int32_t e0 = nbr_start[b], e1 = nbr_start[b + 1];
        for (int r = 0; r < nrhs; ++r) {
            const float2* pr = part + (int64_t)r * cap;
            for (int32_t l = lane; l < occ; l += 32) {
                float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
                for (int32_t e = e0; e < e1; ++e) {
                    const float2 v = pr[contrib_slot(e, part_start, task_kind, mirror, nbr_idx, box_start) + l];
                    const float yr = v.x - cr, tr = sr + yr;
                    cr = (tr - sr) - yr;
                    sr = tr;
                    const float yi = v.y - ci, ti = si + yi;
                    ci = (ti - si) - yi;
                    si = ti;
                }
                u[(int64_t)r * n + perm[bs + l]] = make_float2(sr - cr, si - ci);
            }
        }
    }
}

// Symmetric plans on target-owned layouts: the kernel wrote every target's
// own-item sums to the outputs; add, in neighbour order, the source sums
// other boxes' mutual ranges left for it (entries without a task: the slots
// of the mirror entry, one per particle of this box in box order).
__global__ void __launch_bounds__(256) k_sym_fixup_gravity(const int32_t* __restrict__ box_start,
                                                          const int32_t* __restrict__ nbr_start,
                                                          const int32_t* __restrict__ task_kind,
                                                          const int32_t* __restrict__ mirror,
                                                          const int32_t* __restrict__ bslot,
                                                          const int32_t* __restrict__ perm, const Header* hdr,
                                                          const float4* __restrict__ part, float* __restrict__ phi,
                                                          float* __restrict__ acc) {
    pdl_wait();
    pdl_release();
    if (hdr->flags & (P2P_FLAG_CAPACITY | P2P_FLAG_TIMEOUT)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = hdr->n_boxes;
    for (int64_t b = warp; b < nb; b += nwarps) {
        const int32_t bs = box_start[b], occ = box_start[b + 1] - bs;
        const int32_t e0 = nbr_start[b], ne = nbr_start[b + 1] - e0;
        // lane e: the first slot of this box's sums in entry e's mirror task, if e holds no task
        int32_t my_slot = -1;
        if (lane < ne && task_kind[e0 + lane] == kTaskNone) my_slot = bslot[mirror[e0 + lane]];
        const unsigned none = __ballot_sync(FULL, my_slot >= 0);
        if (!none) continue;
        for (int32_t l0 = 0; l0 < occ; l0 += 32) {   // whole warp in step: the shuffles need every lane
            const int32_t l = l0 + lane;
            const bool act = l < occ;
            float sm[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
            for (unsigned m = none; m; m &= m - 1) {
                const int32_t slot = __shfl_sync(FULL, my_slot, __ffs(m) - 1);
                if (!act) continue;
                const float4 v = part[(int64_t)slot + l];
                const float in[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const float y = in[o] - c[o];
                    const float t = sm[o] + y;
                    c[o] = (t - sm[o]) - y;
                    sm[o] = t;
                }
            }
            if (!act) continue;
            const int64_t o = perm[bs + l];
            phi[o] -= sm[0] - c[0];
            acc[3 * o + 0] += sm[1] - c[1];
            acc[3 * o + 1] += sm[2] - c[2];
            acc[3 * o + 2] += sm[3] - c[3];
        }
    }
}

__global__ void __launch_bounds__(256) k_sym_fixup_helmholtz(const int32_t* __restrict__ box_start,
                                                            const int32_t* __restrict__ nbr_start,
                                                            const int32_t* __restrict__ task_kind,
                                                            const int32_t* __restrict__ mirror,
                                                            const int32_t* __restrict__ bslot,
                                                            const int32_t* __restrict__ perm, const Header* hdr,
                                                            const float2* __restrict__ part, int64_t cap, int nrhs,
                                                            int64_t n, float2* __restrict__ u) {
    pdl_wait();
    pdl_release();
    if (hdr->flags & (P2P_FLAG_CAPACITY | P2P_FLAG_TIMEOUT)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = hdr->n_boxes;
    for (int64_t b = warp; b < nb; b += nwarps) {
        const int32_t bs = box_start[b], occ = box_start[b + 1] - bs;
        const int32_t e0 = nbr_start[b], e1 = nbr_start[b + 1];
        int32_t my_slot = -1;
        if (lane < e1 - e0 && task_kind[e0 + lane] == kTaskNone) my_slot = bslot[mirror[e0 + lane]];
        const unsigned none = __ballot_sync(FULL, my_slot >= 0);
        if (!none) continue;
        for (int r = 0; r < nrhs; ++r) {
            const float2* pr = part + (int64_t)r * cap;
            for (int32_t l0 = 0; l0 < occ; l0 += 32) {   // whole warp in step: the shuffles need every lane
                const int32_t l = l0 + lane;
                const bool act = l < occ;
                float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
                for (unsigned m = none; m; m &= m - 1) {
                    const int32_t slot = __shfl_sync(FULL, my_slot, __ffs(m) - 1);
                    if (!act) continue;
                    const float2 v = pr[(int64_t)slot + l];
                    const float yr = v.x - cr, tr = sr + yr;
                    cr = (tr - sr) - yr;
                    sr = tr;
                    const float yi = v.y - ci, ti = si + yi;
                    ci = (ti - si) - yi;
                    si = ti;
                }
                if (!act) continue;
                float2& out = u[(int64_t)r * n + perm[bs + l]];
                out = make_float2(out.x + (sr - cr), out.y + (si - ci));
            }
        }
    }
}

int sym_fixup_gravity(const Plan* p, void* ws, float* phi, float* acc, cudaStream_t s) {
    const Layout& L = p->L;
    const unsigned wb = (unsigned)std::min<int64_t>(blocks_for(p->box_cap * 32, 256), (int64_t)num_sms() * 16);
    P2P_CUDA_TRY(launch_pdl(k_sym_fixup_gravity, wb, 256, 0, s, at<int32_t>(ws, L.box_start),
                            at<int32_t>(ws, L.nbr_start), at<int32_t>(ws, L.task_kind), at<int32_t>(ws, L.mirror),
                            at<int32_t>(ws, L.bslot), at<int32_t>(ws, L.perm), at<Header>(ws, L.header),
                            at<float4>(ws, L.part), phi, acc));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

int sym_fixup_helmholtz(const Plan* p, void* ws, float2* u, cudaStream_t s) {
    const Layout& L = p->L;
    const unsigned wb = (unsigned)std::min<int64_t>(blocks_for(p->box_cap * 32, 256), (int64_t)num_sms() * 16);
    P2P_CUDA_TRY(launch_pdl(k_sym_fixup_helmholtz, wb, 256, 0, s, at<int32_t>(ws, L.box_start),
                            at<int32_t>(ws, L.nbr_start), at<int32_t>(ws, L.task_kind), at<int32_t>(ws, L.mirror),
                            at<int32_t>(ws, L.bslot), at<int32_t>(ws, L.perm), at<Header>(ws, L.header),
                            at<float2>(ws, L.part), p->part_cap, p->nrhs, p->n, u));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

int pairtask_reduce_gravity(const Plan* p, void* ws, float* phi, float* acc, cudaStream_t s) {
    const Layout& L = p->L;
    const bool sym = p->layout == P2P_LAYOUT_SYMMETRIC;
    const unsigned wb = (unsigned)std::min<int64_t>(blocks_for(p->box_cap * 32, 256), (int64_t)num_sms() * 16);
    P2P_CUDA_TRY(launch_pdl(k_pt_reduce_gravity, wb, 256, 0, s, at<int32_t>(ws, L.box_start), at<int32_t>(ws, L.nbr_start),
                                           at<int32_t>(ws, L.part_start), at<int32_t>(ws, L.perm),
                                           at<Header>(ws, L.header), at<float4>(ws, L.part), phi, acc,
                                           sym ? at<int32_t>(ws, L.task_kind) : nullptr,
                                           sym ? at<int32_t>(ws, L.mirror) : nullptr, at<int32_t>(ws, L.nbr_idx)));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

int pairtask_reduce_helmholtz(const Plan* p, void* ws, float2* u, cudaStream_t s) {
    const Layout& L = p->L;
    const bool sym = p->layout == P2P_LAYOUT_SYMMETRIC;
    const unsigned wb = (unsigned)std::min<int64_t>(blocks_for(p->box_cap * 32, 256), (int64_t)num_sms() * 16);
    P2P_CUDA_TRY(launch_pdl(k_pt_reduce_helmholtz, wb, 256, 0, s, at<int32_t>(ws, L.box_start), at<int32_t>(ws, L.nbr_start),
                                             at<int32_t>(ws, L.part_start), at<int32_t>(ws, L.perm),
                                             at<Header>(ws, L.header), at<float2>(ws, L.part), p->part_cap, p->nrhs,
                                             p->n, u, sym ? at<int32_t>(ws, L.task_kind) : nullptr,
                                             sym ? at<int32_t>(ws, L.mirror) : nullptr, at<int32_t>(ws, L.nbr_idx)));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

}  // namespace p2p
