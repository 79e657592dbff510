// Collect, part 2: restructuring (Section 5.2.1) and the work list.
//
//  - box-ordered source records (both layouts): record s holds the position
//    and strength of particle perm[s];
//  - per-box statistics: S_b (sources in the E2 neighbourhood), the offset of
//    the box's own particles in its stream, the pair count sum_b n_b S_b;
//  - the redundant gather: for each target box, its neighbours' records
//    copied into one contiguous stream (data duplicated per box so that a
//    warp reads a single contiguous block), plus the optional gather map;
//  - the work list: (box, first target) items of up to 32*targets_per_lane
//    targets, ordered by descending cost class (longest-first scheduling).
//
// Source record formats (16-byte words):
//   gravity    [x, y, z, m]
//   Helmholtz  [x, y, z, 0] then nrhs complex q values packed two per word
#include "common.cuh"
#include "device.cuh"

namespace p2p {

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__global__ void k_records_gravity(const float* __restrict__ pos, const float* __restrict__ mass,
                                  const int32_t* __restrict__ perm, int64_t n, float4* __restrict__ rec) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
    rec[s] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], mass[i]);
}

__global__ void k_records_helmholtz(const float* __restrict__ pos, const float2* __restrict__ q,
                                    const int32_t* __restrict__ perm, int64_t n, int nrhs, int words,
                                    float4* __restrict__ rec) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
    float4* r = rec + s * words;
    r[0] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], 0.0f);
    for (int w = 1; w < words; ++w) {
        const int r0 = 2 * (w - 1), r1 = r0 + 1;
        const float2 a = q[(int64_t)r0 * n + i];
        const float2 b = (r1 < nrhs) ? q[(int64_t)r1 * n + i] : make_float2(0.0f, 0.0f);
        r[w] = make_float4(a.x, a.y, b.x, b.y);
    }
}

// Per-box statistics and the cost-class histogram of the work items.
// S[b] = sum of occupancies of b's neighbours; self[b] = offset of b's own
// particles in its stream (neighbours are ascending, so it is the sum over
// neighbours with a smaller index).
__global__ void __launch_bounds__(256) k_box_stats(const int32_t* __restrict__ box_start,
                                                  const int32_t* __restrict__ nbr_start,
                                                  const int32_t* __restrict__ nbr_idx, Header* hdr,
                                                  int64_t box_cap, int tt, int32_t* __restrict__ S,
                                                  int32_t* __restrict__ self_off) {
    __shared__ int32_t cls[kCostClasses];
    __shared__ unsigned long long pairs_s;
    __shared__ int32_t items_s;
    for (int c = threadIdx.x; c < kCostClasses; c += blockDim.x) cls[c] = 0;
    if (threadIdx.x == 0) {
        pairs_s = 0ull;
        items_s = 0;
    }
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t nb = hdr->n_boxes;
    if (b < box_cap) {
        if (b >= nb) {
            S[b] = 0;
        } else {
            int32_t sb = 0, so = 0;
            for (int32_t e = nbr_start[b]; e < nbr_start[b + 1]; ++e) {
                const int32_t c = nbr_idx[e];
                const int32_t cnt = box_start[c + 1] - box_start[c];
                if (c < b) so += cnt;
                sb += cnt;
            }
            S[b] = sb;
            if (self_off) self_off[b] = so;
            const int32_t occ = box_start[b + 1] - box_start[b];
            atomicAdd(&pairs_s, (unsigned long long)occ * (unsigned long long)sb);
            int32_t ni = 0;
            for (int32_t t0 = 0; t0 < occ; t0 += tt, ++ni) {
                const int32_t nt = min(tt, occ - t0);
                const unsigned long long cost = (unsigned long long)nt * (unsigned long long)max(sb, 1);
                atomicAdd(&cls[63 - __clzll(cost)], 1);
            }
            atomicAdd(&items_s, ni);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kCostClasses; c += blockDim.x)
        if (cls[c]) atomicAdd(&hdr->cls_cnt[c], cls[c]);
    if (threadIdx.x == 0) {
        if (pairs_s) atomicAdd(&hdr->pairs_nS, pairs_s);
        if (items_s) atomicAdd(&hdr->n_items, items_s);
    }
}

// Place each item in its cost class, heaviest class first.  Blocks reserve a
// range per class with one atomic, then fill it through shared counters.
__global__ void __launch_bounds__(256) k_items_fill(const int32_t* __restrict__ box_start,
                                                   const int32_t* __restrict__ S, Header* hdr, int64_t box_cap,
                                                   int tt, int2* __restrict__ items) {
    __shared__ int32_t cls_base[kCostClasses];
    __shared__ int32_t local_cnt[kCostClasses];
    __shared__ int32_t local_cur[kCostClasses];
    if (threadIdx.x < kCostClasses) {
        // descending order: items of class c start after all heavier classes
        int32_t off = 0;
        for (int c2 = kCostClasses - 1; c2 > (int)threadIdx.x; --c2) off += hdr->cls_cnt[c2];
        cls_base[threadIdx.x] = off;
        local_cnt[threadIdx.x] = 0;
        local_cur[threadIdx.x] = 0;
    }
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = b < box_cap && b < hdr->n_boxes;
    int32_t occ = 0, sb = 0;
    if (active) {
        occ = box_start[b + 1] - box_start[b];
        sb = max(S[b], 1);
        for (int32_t t0 = 0; t0 < occ; t0 += tt) {
            const unsigned long long cost = (unsigned long long)min(tt, occ - t0) * (unsigned long long)sb;
            atomicAdd(&local_cnt[63 - __clzll(cost)], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < kCostClasses && local_cnt[threadIdx.x])
        cls_base[threadIdx.x] += atomicAdd(&hdr->cls_cursor[threadIdx.x], local_cnt[threadIdx.x]);
    __syncthreads();
    if (active) {
        for (int32_t t0 = 0; t0 < occ; t0 += tt) {
            const unsigned long long cost = (unsigned long long)min(tt, occ - t0) * (unsigned long long)sb;
            const int c = 63 - __clzll(cost);
            const int32_t pos = cls_base[c] + atomicAdd(&local_cur[c], 1);
            items[pos] = make_int2((int32_t)b, t0);
        }
    }
}

// Redundant gather: one warp per target box copies the records of each
// neighbour box, in neighbour order, into the box's stream (16-byte words,
// coalesced), and optionally the sorted index of every copied record.
__global__ void __launch_bounds__(256) k_red_gather(const float4* __restrict__ rec, int words,
                                                   const int32_t* __restrict__ box_start,
                                                   const int32_t* __restrict__ nbr_start,
                                                   const int32_t* __restrict__ nbr_idx,
                                                   const int32_t* __restrict__ red_start, Header* hdr,
                                                   int64_t red_cap, float4* __restrict__ red,
                                                   uint32_t* __restrict__ gather) {
    const int lane = threadIdx.x & 31;
    // an imported, inconsistent neighbour relation can exceed the stream capacity
    if (hdr->total_src < 0 || (int64_t)hdr->total_src > red_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&hdr->flags, P2P_FLAG_CAPACITY);
        return;
    }
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = hdr->n_boxes;
    for (int64_t b = warp; b < nb; b += nwarps) {
        int64_t out = red_start[b];
        for (int32_t e = nbr_start[b]; e < nbr_start[b + 1]; ++e) {
            const int32_t c = nbr_idx[e];
            const int32_t s0 = box_start[c];
            const int32_t cnt = box_start[c + 1] - s0;
            const int64_t nw = (int64_t)cnt * words;
            const float4* src = rec + (int64_t)s0 * words;
            float4* dst = red + out * words;
            for (int64_t w = lane; w < nw; w += 32) dst[w] = src[w];
            if (gather)
                for (int32_t l = lane; l < cnt; l += 32) gather[out + l] = (uint32_t)(s0 + l);
            out += cnt;
        }
    }
}

int restructure(Plan* p, const float* pos, const void* strength, void* ws, cudaStream_t s) {
    const Layout& L = p->L;
    Header* hdr = at<Header>(ws, L.header);
    const int64_t n = p->n;
    const int32_t* perm = at<int32_t>(ws, L.perm);
    float4* rec = at<float4>(ws, L.src);
    if (p->kind == P2P_GRAVITY) {
        k_records_gravity<<<blocks_for(n, 256), 256, 0, s>>>(pos, static_cast<const float*>(strength), perm, n, rec);
    } else {
        k_records_helmholtz<<<blocks_for(n, 256), 256, 0, s>>>(pos, static_cast<const float2*>(strength), perm, n,
                                                              p->nrhs, p->rec_words, rec);
    }
    P2P_LAUNCH_CHECK();
    if (p->layout == P2P_LAYOUT_REDUNDANT) {
        const int64_t bc = p->box_cap;
        int32_t* S = at<int32_t>(ws, L.box_S);
        int32_t* red_start = at<int32_t>(ws, L.red_start);
        int32_t* red_self = at<int32_t>(ws, L.red_self);
        // box statistics also fill the operator section; it is cleared again by the operator call
        P2P_CUDA_TRY(cudaMemsetAsync(reinterpret_cast<char*>(hdr) + kOpSectionOffset, 0,
                                     sizeof(Header) - kOpSectionOffset, s));
        k_box_stats<<<blocks_for(bc, 256), 256, 0, s>>>(at<int32_t>(ws, L.box_start), at<int32_t>(ws, L.nbr_start),
                                                       at<int32_t>(ws, L.nbr_idx), hdr, bc, 32 * p->tpl, S,
                                                       red_self);
        P2P_LAUNCH_CHECK();
        int st = scan_exclusive(S, red_start, bc, &hdr->n_boxes, &hdr->total_src, at<int32_t>(ws, L.scan_tmp), s);
        if (st) return st;
        const int sms = num_sms();
        k_red_gather<<<sms * 8, 256, 0, s>>>(rec, p->rec_words, at<int32_t>(ws, L.box_start),
                                            at<int32_t>(ws, L.nbr_start), at<int32_t>(ws, L.nbr_idx), red_start,
                                            hdr, p->red_cap, at<float4>(ws, L.red_src),
                                            (p->flags & P2P_PLAN_GATHER_MAP) ? at<uint32_t>(ws, L.gather) : nullptr);
        P2P_LAUNCH_CHECK();
    }
    p->src_ready = 1;
    return P2P_OK;
}

int build_items(Plan* p, void* ws, int tt, cudaStream_t s) {
    const Layout& L = p->L;
    Header* hdr = at<Header>(ws, L.header);
    const int64_t bc = p->box_cap;
    int32_t* S = at<int32_t>(ws, L.box_S);
    P2P_CUDA_TRY(cudaMemsetAsync(reinterpret_cast<char*>(hdr) + kOpSectionOffset, 0,
                                 sizeof(Header) - kOpSectionOffset, s));
    k_box_stats<<<blocks_for(bc, 256), 256, 0, s>>>(at<int32_t>(ws, L.box_start), at<int32_t>(ws, L.nbr_start),
                                                   at<int32_t>(ws, L.nbr_idx), hdr, bc, tt, S, nullptr);
    P2P_LAUNCH_CHECK();
    k_items_fill<<<blocks_for(bc, 256), 256, 0, s>>>(at<int32_t>(ws, L.box_start), S, hdr, bc, tt,
                                                    at<int2>(ws, L.items));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

}  // namespace p2p
