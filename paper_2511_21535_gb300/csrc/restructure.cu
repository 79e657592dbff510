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
//   Helmholtz  [x, y, z, 0] then nrhs complex q values packed two per word,
//              [Re q_a, Im q_a, Re q_b, Im q_b]; plans of four or more
//              right-hand sides (direct evaluation) hold each pair planar,
//              [Re q_a, Re q_b, Im q_a, Im q_b]
#include <algorithm>
#include <climits>
#include <cstdint>

#include "common.cuh"
#include "copy.cuh"
#include "device.cuh"
#include "lookback.cuh"

namespace p2p {

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__global__ void k_records_gravity(const float* __restrict__ pos, const float* __restrict__ mass,
                                  const int32_t* __restrict__ perm, int64_t n, float4* __restrict__ rec,
                                  unsigned long long* __restrict__ lb, int64_t lb_words, Header* __restrict__ hdr) {
    pdl_wait();
    pdl_release();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < lb_words) lb[s] = 0ull;   // chained-scan scratch of the box statistics
    if (s < (int64_t)(kOpSectionOffset - kRestrSectionOffset) / 4)   // the restructuring's header counts
        reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(hdr) + kRestrSectionOffset)[s] = 0u;
    if (s >= n || (hdr->flags & P2P_FLAG_CAPACITY)) return;   // an inconsistent imported structure
    const int64_t i = perm[s];
    rec[s] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], mass[i]);
}

// right-hand side r of particle i: q[r] for r < split, conj(q2[r - split]) after
// (a forward+adjoint pair runs as one operator: conj(P) y = conj(P conj(y)))
__device__ __forceinline__ float2 rhs_value(const float2* __restrict__ q, const float2* __restrict__ q2, int split,
                                            int64_t n, int r, int64_t i) {
    if (r < split) return q[(int64_t)r * n + i];
    const float2 v = q2[(int64_t)(r - split) * n + i];
    return make_float2(v.x, -v.y);
}

__global__ void k_clear_flag(Header* hdr, uint32_t bit) {
    pdl_wait();
    pdl_release();
    atomicAnd(&hdr->flags, ~bit);
}

// Pattern mode: lattice code of a point, ix*1 + iy*sy + iz*sz with
// ix = rint((x - lo)/h - 1/2); the point must be within 1 % of h of the
// lattice and in the leaf box (ix div t) the tree put it in.
struct LatticeArgs {
    int on;
    float lo[3];
    float inv_h;
    int t, sy, sz;
    float scale;      // the tree's (float)2^level / edge
    int cmax;         // 2^level - 1
};

__device__ __forceinline__ bool lattice_code(const float* x, const LatticeArgs& g, int* code) {
    int c = 0;
    const int stride[3] = {1, g.sy, g.sz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float f = (x[a] - g.lo[a]) * g.inv_h - 0.5f;
        const float r = rintf(f);
        if (!(fabsf(f - r) <= 0.01f)) return false;
        const int ix = (int)r;
        int cell = (int)floorf(__fmul_rn(__fsub_rn(x[a], g.lo[a]), g.scale));
        cell = cell > g.cmax ? g.cmax : cell;
        if (ix < 0 || ix / g.t != cell) return false;
        c += ix * stride[a];
    }
    *code = c;
    return true;
}

__global__ void k_records_helmholtz(const float* __restrict__ pos, const float2* __restrict__ q,
                                    const float2* __restrict__ q2, int split, const int32_t* __restrict__ perm,
                                    int64_t n, int nrhs, int words, int planar, LatticeArgs lat, Header* hdr,
                                    float4* __restrict__ rec,
                                  unsigned long long* __restrict__ lb, int64_t lb_words) {
    pdl_wait();
    pdl_release();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < lb_words) lb[s] = 0ull;   // chained-scan scratch of the box statistics
    if (s < (int64_t)(kOpSectionOffset - kRestrSectionOffset) / 4)   // the restructuring's header counts
        reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(hdr) + kRestrSectionOffset)[s] = 0u;
    if (s >= n || (hdr->flags & P2P_FLAG_CAPACITY)) return;   // an inconsistent imported structure
    const int64_t i = perm[s];
    float4* r = rec + s * words;
    float w = 0.0f;
    if (lat.on) {
        int code = 0;
        if (!lattice_code(pos + 3 * i, lat, &code)) atomicOr(&hdr->flags, P2P_FLAG_LATTICE);
        w = __int_as_float(code);
        if (words == 1) {   // compact pattern record [code, Re q, Im q, 0] (one right-hand side)
            const float2 a = rhs_value(q, q2, split, n, 0, i);
            r[0] = make_float4(w, a.x, a.y, 0.0f);
            return;
        }
    }
    r[0] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], w);
    for (int w = 1; w < words; ++w) {
        const int r0 = 2 * (w - 1), r1 = r0 + 1;
        const float2 a = rhs_value(q, q2, split, n, r0, i);
        const float2 b = (r1 < nrhs) ? rhs_value(q, q2, split, n, r1, i) : make_float2(0.0f, 0.0f);
        r[w] = planar ? make_float4(a.x, b.x, a.y, b.y) : make_float4(a.x, a.y, b.x, b.y);
    }
}

__global__ void k_records_helm_adjoint(const float* __restrict__ pos, const float2* __restrict__ q,
                                       const float2* __restrict__ gbar, const int32_t* __restrict__ perm, int64_t n,
                                       int nrhs, int words, float4* __restrict__ rec,
                                  unsigned long long* __restrict__ lb, int64_t lb_words, Header* __restrict__ hdr) {
    pdl_wait();
    pdl_release();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < lb_words) lb[s] = 0ull;   // chained-scan scratch of the box statistics
    if (s < (int64_t)(kOpSectionOffset - kRestrSectionOffset) / 4)   // the restructuring's header counts
        reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(hdr) + kRestrSectionOffset)[s] = 0u;
    if (s >= n || (hdr->flags & P2P_FLAG_CAPACITY)) return;   // an inconsistent imported structure
    const int64_t i = perm[s];
    float4* r = rec + s * words;
    const int half = (nrhs + 1) / 2;
    r[0] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], 0.0f);
    for (int w = 0; w < half; ++w) {
        const int r0 = 2 * w, r1 = r0 + 1;
        const float2 a = q[(int64_t)r0 * n + i];
        const float2 b = (r1 < nrhs) ? q[(int64_t)r1 * n + i] : make_float2(0.0f, 0.0f);
        r[1 + w] = make_float4(a.x, a.y, b.x, b.y);
        const float2 c = gbar[(int64_t)r0 * n + i];
        const float2 d = (r1 < nrhs) ? gbar[(int64_t)r1 * n + i] : make_float2(0.0f, 0.0f);
        r[1 + half + w] = make_float4(c.x, c.y, d.x, d.y);
    }
}

__global__ void k_records_grav_adjoint(const float* __restrict__ pos, const float* __restrict__ mass,
                                       const float* __restrict__ gphi, const float* __restrict__ gacc,
                                       const int32_t* __restrict__ perm, int64_t n, float4* __restrict__ rec,
                                  unsigned long long* __restrict__ lb, int64_t lb_words, Header* __restrict__ hdr) {
    pdl_wait();
    pdl_release();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < lb_words) lb[s] = 0ull;   // chained-scan scratch of the box statistics
    if (s < (int64_t)(kOpSectionOffset - kRestrSectionOffset) / 4)   // the restructuring's header counts
        reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(hdr) + kRestrSectionOffset)[s] = 0u;
    if (s >= n || (hdr->flags & P2P_FLAG_CAPACITY)) return;   // an inconsistent imported structure
    const int64_t i = perm[s];
    rec[2 * s] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], mass[i]);
    rec[2 * s + 1] = make_float4(gphi[i], gacc[3 * i], gacc[3 * i + 1], gacc[3 * i + 2]);
}

// Per-box statistics, a tile of kBoxTile boxes per block, four per warp
// (lane e reads neighbour e): S[b] = sum of the occupancies of the
// neighbours in b's stream; self[b] = offset of b's own particles in it
// (neighbours are ascending, so it is the sum over streamed neighbours with a
// smaller index); the pair count sum_b n_b S_b over all neighbours.  For the
// redundant layout the stream bounds red_start = exclusive scan of S are
// chained across tiles in the same pass (lookback.cuh), and the tile holding
// the last box closes them.
//
// Symmetric plans (task_kind != nullptr) also classify each entry (b -> c):
// self; mutual when b is the pair's lane box (the smaller index if it holds
// <= kMutualMax particles, else the other one if that one does); none for
// the other entry of such a pair (its mirror entry is found in c's list);
// one-sided when neither box fits.  Only self, mutual and one-sided entries
// are streamed, and the mutual entries' source-sum slots (one per source
// particle) are a second chained scan.
constexpr int kStatsPerWarp = kBoxTile / 8;

__device__ __forceinline__ int32_t entry_kind(int32_t b, int32_t c, int32_t nb_occ, int32_t nc) {
    if (c == b) return kTaskSelf;
    const int32_t lo = min(b, c), hi = max(b, c);
    const int32_t nlo = (lo == b) ? nb_occ : nc, nhi = (hi == b) ? nb_occ : nc;
    const int32_t lane_box = nlo <= kMutualMax ? lo : (nhi <= kMutualMax ? hi : -1);
    return lane_box < 0 ? kTaskOneSided : (lane_box == b ? kTaskMutual : kTaskNone);
}

__global__ void __launch_bounds__(256) k_box_stats(const int32_t* __restrict__ box_start,
                                                  const int32_t* __restrict__ nbr_start,
                                                  const int32_t* __restrict__ nbr_idx, Header* hdr,
                                                  int32_t* __restrict__ S, int32_t* __restrict__ self_off,
                                                  int32_t* __restrict__ red_start, unsigned long long* lb,
                                                  int32_t* __restrict__ task_kind, int32_t* __restrict__ mirror,
                                                  int32_t* __restrict__ bslot, unsigned long long* lb2,
                                                  int64_t part_cap, int32_t* __restrict__ heavy) {
    pdl_wait();
    pdl_release();
    __shared__ int tile_s;
    __shared__ int32_t s_s[kBoxTile], b_s[kBoxTile];
    __shared__ int32_t pre_s[kBoxTile + 1], bpre_s[kBoxTile + 1];
    __shared__ unsigned long long pairs_s, evals_s;
    if (threadIdx.x == 0) {
        pairs_s = 0ull;
        evals_s = 0ull;
    }
    const int32_t nb = hdr->n_boxes;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long pairs = 0ull, evals = 0ull;   // this warp's share over all its tiles
    // a few blocks per SM take tiles of kBoxTile boxes by ticket until the boxes run out
    for (;;) {
        if (threadIdx.x == 0) {
            // a rejected structure: the block takes no tile (later tiles wait only on taken ones);
            // one thread reads the flag, which other blocks of this launch may be setting
            tile_s = (hdr->flags & P2P_FLAG_CAPACITY) ? -1 : lb_ticket(lb);
        }
        __syncthreads();
        const int tile = tile_s;
        if (tile < 0) break;
        const int64_t b0 = (int64_t)tile * kBoxTile;
        if (b0 >= nb) break;   // past the last box (whole block): no later tile waits on it
        int32_t cbx[kStatsPerWarp];   // symmetric: this lane's offset among its box's mutual source slots
#pragma unroll
        for (int q = 0; q < kStatsPerWarp; ++q) {
            const int64_t b = b0 + warp * kStatsPerWarp + q;
            int32_t all = 0, cnt = 0, lower = 0, cb = 0;
            if (b < nb) {
                const int32_t e0 = nbr_start[b], ne = nbr_start[b + 1] - e0;
                if (lane < ne) {
                    const int32_t e = e0 + lane;
                    const int32_t c = nbr_idx[e];
                    const int32_t nc = box_start[c + 1] - box_start[c];
                    all = nc;
                    int32_t kind = kTaskOneSided;
                    if (task_kind) {
                        kind = entry_kind((int32_t)b, c, box_start[b + 1] - box_start[b], nc);
                        int32_t mir = -1;
                        if (kind == kTaskNone) {
                            // b's position in c's ascending list: independent loads, one latency
                            const int32_t c0 = nbr_start[c], cn = nbr_start[c + 1] - c0;
                            int32_t below = 0;
                            bool found = false;
#pragma unroll
                            for (int i = 0; i < 27; ++i) {
                                const int32_t v = i < cn ? nbr_idx[c0 + i] : INT32_MAX;
                                below += v < b ? 1 : 0;
                                found |= v == b;
                            }
                            if (found && cn <= 27) mir = c0 + below;
                            else atomicOr(&hdr->flags, P2P_FLAG_CAPACITY);   // inconsistent (imported) relation
                        }
                        task_kind[e] = kind;
                        mirror[e] = mir;
                    }
                    cnt = kind == kTaskNone ? 0 : nc;
                    lower = (c < b) ? cnt : 0;
                    cb = kind == kTaskMutual ? nc : 0;
                }
            }
            const int32_t cbi = warp_incl_scan(cb);
            cbx[q] = cbi - cb;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                all += __shfl_xor_sync(FULL, all, o);
                cnt += __shfl_xor_sync(FULL, cnt, o);
                lower += __shfl_xor_sync(FULL, lower, o);
            }
            const int32_t cbt = __shfl_sync(FULL, cbi, 31);
            if (lane == 0) {
                s_s[warp * kStatsPerWarp + q] = cnt;
                b_s[warp * kStatsPerWarp + q] = cbt;
                if (b < nb) {
                    S[b] = cnt;
                    if (heavy && cnt > kGatherLight) heavy[atomicAdd(&hdr->n_heavy, 1)] = (int32_t)b;
                    if (self_off) self_off[b] = lower;
                    pairs += (unsigned long long)(box_start[b + 1] - box_start[b]) * (unsigned long long)all;
                    evals += (unsigned long long)(box_start[b + 1] - box_start[b]) * (unsigned long long)cnt;
                }
            }
        }
        __syncthreads();
        const bool last = nb - 1 >= b0 && nb - 1 < b0 + kBoxTile;
        if (red_start) {
            if (warp == 0) {
                const int32_t v = s_s[lane];
                const int32_t inc = warp_incl_scan(v);
                const int32_t agg = __shfl_sync(FULL, inc, 31);
                const int32_t ex = lb_exclusive(lb, tile, agg, hdr);
                pre_s[lane] = ex + inc - v;
                if (lane == 31) pre_s[kBoxTile] = ex + inc;
            }
            __syncthreads();
            if (threadIdx.x < kBoxTile && b0 + threadIdx.x < nb) red_start[b0 + threadIdx.x] = pre_s[threadIdx.x];
            if (threadIdx.x == 0 && last) {
                red_start[nb] = pre_s[kBoxTile];
                hdr->total_src = pre_s[kBoxTile];
            }
        }
        if (bslot) {
            if (warp == 0) {
                const int32_t v = b_s[lane];
                const int32_t inc = warp_incl_scan(v);
                const int32_t agg = __shfl_sync(FULL, inc, 31);
                const int32_t ex = lb_exclusive(lb2, tile, agg, hdr);
                bpre_s[lane] = ex + inc - v;
                if (lane == 31) bpre_s[kBoxTile] = ex + inc;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kStatsPerWarp; ++q) {
                const int64_t b = b0 + warp * kStatsPerWarp + q;
                if (b < nb) {
                    const int32_t e0 = nbr_start[b], ne = nbr_start[b + 1] - e0;
                    if (lane < ne) bslot[e0 + lane] = bpre_s[warp * kStatsPerWarp + q] + cbx[q];
                }
            }
            if (threadIdx.x == 0 && last) {
                hdr->part_total = bpre_s[kBoxTile];
                if ((int64_t)bpre_s[kBoxTile] > part_cap) atomicOr(&hdr->flags, P2P_FLAG_CAPACITY);
            }
        }
        __syncthreads();   // the shared tile state is reused by the next tile
    }
    // the pair counts of this block's tiles
    if (lane == 0 && pairs) atomicAdd(&pairs_s, pairs);
    if (lane == 0 && evals) atomicAdd(&evals_s, evals);
    __syncthreads();
    if (threadIdx.x == 0 && pairs_s) atomicAdd(&hdr->pairs_nS, pairs_s);
    if (threadIdx.x == 0 && evals_s) atomicAdd(&hdr->evals_nS, evals_s);
}

__device__ __forceinline__ int cost_class(int32_t nt, int32_t sb) {
    const unsigned long long cost = (unsigned long long)nt * (unsigned long long)max(sb, 1);
    return 63 - __clzll(cost);
}

// Work units: target boxes (unit u = box b: occupancy n_b, sources S_b), or
// for pair tasks neighbour entries (u = e = (b, c): n_b targets, n_c sources).
struct Units {
    const int32_t* box_start;
    const int32_t* S;          // per box S_b (box units)
    const int32_t* ent_box;    // pair tasks: target box per entry, else nullptr
    const int32_t* nbr_idx;    // pair tasks: source box per entry
    int64_t cap;               // units the grid covers
    const int32_t* task_kind;  // symmetric tasks: entries without a task have no items; self tasks read the box
};

__device__ __forceinline__ int32_t unit_count(const Units& U, const Header* hdr) {
    return U.ent_box ? hdr->n_nbr : hdr->n_boxes;
}
__device__ __forceinline__ void unit_shape(const Units& U, int64_t u, int32_t& occ, int32_t& sb) {
    if (U.ent_box) {
        const int32_t b = U.ent_box[u], c = U.nbr_idx[u];
        occ = U.box_start[b + 1] - U.box_start[b];
        sb = U.box_start[c + 1] - U.box_start[c];
        if (U.task_kind && U.task_kind[u] == kTaskNone) occ = 0;
    } else {
        occ = U.box_start[u + 1] - U.box_start[u];
        sb = U.S[u];
    }
}

// Cost-class histogram of the work items (items of up to tt targets).
__global__ void __launch_bounds__(256) k_items_count(Units U, Header* hdr, int tt) {
    pdl_wait();
    pdl_release();
    if (hdr->flags & P2P_FLAG_CAPACITY) return;   // no items: the operator does nothing
    __shared__ int32_t cls[kCostClasses];
    __shared__ int32_t items_s;
    for (int c = threadIdx.x; c < kCostClasses; c += blockDim.x) cls[c] = 0;
    if (threadIdx.x == 0) items_s = 0;
    __syncthreads();
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < U.cap && u < unit_count(U, hdr)) {
        int32_t occ, sb;
        unit_shape(U, u, occ, sb);
        int32_t ni = 0;
        for (int32_t t0 = 0; t0 < occ; t0 += tt, ++ni) atomicAdd(&cls[cost_class(min(tt, occ - t0), sb)], 1);
        atomicAdd(&items_s, ni);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kCostClasses; c += blockDim.x)
        if (cls[c]) atomicAdd(&hdr->cls_cnt[c], cls[c]);
    if (threadIdx.x == 0 && items_s) atomicAdd(&hdr->n_items, items_s);
}

// Place each item in its cost class, heaviest class first.  Blocks reserve a
// range per class with one atomic, then fill it through shared counters.
__global__ void __launch_bounds__(256) k_items_fill(Units U, Header* hdr, int tt, int2* __restrict__ items) {
    pdl_wait();
    pdl_release();
    if (hdr->flags & P2P_FLAG_CAPACITY) return;
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
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = u < U.cap && u < unit_count(U, hdr);
    int32_t occ = 0, sb = 0;
    if (active) {
        unit_shape(U, u, occ, sb);
        for (int32_t t0 = 0; t0 < occ; t0 += tt) atomicAdd(&local_cnt[cost_class(min(tt, occ - t0), sb)], 1);
    }
    __syncthreads();
    if (threadIdx.x < kCostClasses && local_cnt[threadIdx.x])
        cls_base[threadIdx.x] += atomicAdd(&hdr->cls_cursor[threadIdx.x], local_cnt[threadIdx.x]);
    __syncthreads();
    if (active) {
        for (int32_t t0 = 0; t0 < occ; t0 += tt) {
            const int c = cost_class(min(tt, occ - t0), sb);
            const int32_t pos = cls_base[c] + atomicAdd(&local_cur[c], 1);
            items[pos] = make_int2((int32_t)u, t0);
        }
    }
}

// Redundant gather: each target box's stream is the records of its neighbour
// boxes, in neighbour order (16-byte words), optionally with the sorted index
// of every copied record.  The kernel waits on chains of dependent loads
// (stream bounds, neighbour list, neighbour occupancies, records), so it is
// organised to keep many chains in flight per warp:
//  - a light stream (<= kGatherLight records: the sparse boxes of a
//    clustered distribution, most of its boxes) is copied flat, LB boxes per
//    warp at once: each level of their loads is issued for all LB boxes
//    together; lane e reads the box's neighbour entry e, a warp scan of the
//    entries' counts gives each entry's offset in the stream, and in each
//    round lane l takes position 32 r + l of every box's stream, finds its
//    entry by a binary search over the offsets held in the lanes (shuffles)
//    and issues the loads of all LB boxes before their stores (coalesced);
//  - a heavy stream (listed by the box statistics) is copied in
//    kGatherParts parts of its entries, one warp per part copying one entry
//    at a time with the whole warp (coalesced, eight loads in flight per
//    lane).
// With periodic boundaries a wrapped neighbour's records are copied with
// their positions moved to the image the box meets (word 0 holds x, y, z),
// so the kernel needs no image logic.
// The light streams of boxes bx[0 .. LB) (bx[u] < 0: none).  W: words per
// record when known at compile time (1, 2), else 0 (`words`).
template <int W, int LB>
__device__ __forceinline__ void gather_light(const int64_t (&bx)[LB], const float4* __restrict__ rec, int words,
                                             const int32_t* __restrict__ box_start,
                                             const int32_t* __restrict__ nbr_start,
                                             const int32_t* __restrict__ nbr_idx,
                                             const int32_t* __restrict__ nbr_img, float edge,
                                             const int32_t* __restrict__ red_start, float4* __restrict__ red,
                                             uint32_t* __restrict__ gather, const int32_t* __restrict__ task_kind,
                                             int lane) {
    const int wd = W > 0 ? W : words;
    // level 1: the boxes' entry ranges and stream starts
    int32_t e0[LB], ne[LB], rs[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
        e0[u] = 0;
        ne[u] = 0;
        rs[u] = 0;
        if (bx[u] >= 0) {
            e0[u] = nbr_start[bx[u]];
            ne[u] = nbr_start[bx[u] + 1] - e0[u];
            rs[u] = red_start[bx[u]];
        }
    }
    // level 2: lane e's neighbour entry (symmetric plans: entries of kind none stream nothing)
    int32_t cb[LB], code[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
        cb[u] = -1;
        code[u] = 13;
        if (lane < ne[u] && !(task_kind && task_kind[e0[u] + lane] == kTaskNone)) {
            cb[u] = nbr_idx[e0[u] + lane];
            if (nbr_img) code[u] = nbr_img[e0[u] + lane];
        }
    }
    // level 3: the neighbours' source runs, and each entry's offset in the stream
    int32_t s0[LB], excl[LB], len[LB];
    int32_t rounds = 0;
#pragma unroll
    for (int u = 0; u < LB; ++u) {
        s0[u] = 0;
        int32_t cnt = 0;
        if (cb[u] >= 0) {
            s0[u] = box_start[cb[u]];
            cnt = box_start[cb[u] + 1] - s0[u];
        }
        const int32_t inc = warp_incl_scan(cnt);
        excl[u] = inc - cnt;
        len[u] = __shfl_sync(FULL, inc, 31);
        rounds = max(rounds, (len[u] + 31) >> 5);
    }
    constexpr int WV = W > 0 ? W : 1;   // words loaded before the stores
    for (int32_t r = 0; r < rounds; ++r) {
        const int32_t p = 32 * r + lane;   // position in each stream
        float4 v[LB][WV];
        int32_t src[LB], cd[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            int j = 0;   // the last entry that starts at or before p
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int cand = j + st;   // <= 31
                const int32_t ex = __shfl_sync(FULL, excl[u], cand);
                if (cand < ne[u] && ex <= p) j = cand;
            }
            src[u] = __shfl_sync(FULL, s0[u], j) + (p - __shfl_sync(FULL, excl[u], j));
            cd[u] = nbr_img ? __shfl_sync(FULL, code[u], j) : 13;
            if (p < len[u]) {
#pragma unroll
                for (int w = 0; w < WV; ++w) v[u][w] = __ldg(rec + (int64_t)src[u] * wd + w);
            }
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            if (p >= len[u]) continue;
            const int64_t d = (int64_t)rs[u] + p;
            float4* o = red + d * wd;
            __stcs(o, image_shifted(v[u][0], cd[u], edge));
#pragma unroll
            for (int w = 1; w < WV; ++w) __stcs(o + w, v[u][w]);
            if (W == 0)
                for (int w = 1; w < wd; ++w) __stcs(o + w, __ldg(rec + (int64_t)src[u] * wd + w));
            if (gather) gather[d] = (uint32_t)src[u];
        }
    }
}

__device__ __forceinline__ void gather_part(int64_t b, int part, const float4* __restrict__ rec, int words,
                                            const int32_t* __restrict__ box_start,
                                            const int32_t* __restrict__ nbr_start,
                                            const int32_t* __restrict__ nbr_idx,
                                            const int32_t* __restrict__ nbr_img, float edge, int32_t rs0,
                                            float4* __restrict__ red, uint32_t* __restrict__ gather,
                                            const int32_t* __restrict__ task_kind, int lane) {
    const int32_t e0 = nbr_start[b], ne = nbr_start[b + 1] - e0;
    const int32_t lo = part * ne / kGatherParts, hi = (part + 1) * ne / kGatherParts;
    // the chunk's offset in the stream: the streamed counts of the entries before it
    int32_t before = 0;
    if (lane < lo && !(task_kind && task_kind[e0 + lane] == kTaskNone)) {
        const int32_t c = nbr_idx[e0 + lane];
        before = box_start[c + 1] - box_start[c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(FULL, before, o);
    int64_t out = (int64_t)rs0 + before;
    for (int32_t e = e0 + lo; e < e0 + hi; ++e) {
        if (task_kind && task_kind[e] == kTaskNone) continue;   // symmetric: the mirror's mutual item covers it
        const int32_t c = nbr_idx[e];
        const int32_t s0 = box_start[c];
        const int32_t cnt = box_start[c + 1] - s0;
        const float4* src = rec + (int64_t)s0 * words;
        float4* dst = red + out * words;
        warp_copy_records(src, dst, cnt, words, lane, nbr_img ? nbr_img[e] : 13, edge);
        if (gather)
            for (int32_t l = lane; l < cnt; l += 32) gather[out + l] = (uint32_t)(s0 + l);
        out += cnt;
    }
}

// Six blocks of four warps per SM (registers capped to 80, a few bytes spilled):
// the kernel is latency bound, and 24 resident warps measured faster than 20
// with no spill (the 4.2 M-particle Plummer sphere and the 128^3 grid).  The
// grid is 32 blocks per SM (about five waves): the boxes and heavy parts are
// dealt to warps by a fixed stride, and smaller shares per warp even out the
// waves (measured faster than 16 and than one resident wave on the clustered
// sphere, equal on grids).
template <int W>
__global__ void __launch_bounds__(128, 6) k_red_gather(const float4* __restrict__ rec, int words,
                                                   const int32_t* __restrict__ box_start,
                                                   const int32_t* __restrict__ nbr_start,
                                                   const int32_t* __restrict__ nbr_idx,
                                                   const int32_t* __restrict__ nbr_img, float edge,
                                                   const int32_t* __restrict__ red_start, Header* hdr,
                                                   int64_t red_cap, float4* __restrict__ red,
                                                   uint32_t* __restrict__ gather,
                                                   const int32_t* __restrict__ task_kind,
                                                   const int32_t* __restrict__ heavy, int64_t heavy_cap) {
    pdl_wait();
    pdl_release();
    const int lane = threadIdx.x & 31;
    // an imported, inconsistent neighbour relation can exceed the stream capacity
    if ((hdr->flags & P2P_FLAG_CAPACITY) || hdr->total_src < 0 || (int64_t)hdr->total_src > red_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&hdr->flags, P2P_FLAG_CAPACITY);
        return;
    }
    constexpr int LB = W == 1 ? 4 : 2;   // light boxes per warp at once (registers: LB x W loads in flight)
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = hdr->n_boxes;
    // light streams: boxes warp, warp + nwarps, ..., LB at a time
    for (int64_t b = warp; b < nb; b += LB * nwarps) {
        int64_t bx[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int64_t c = b + u * nwarps;
            bx[u] = (c < nb && red_start[c + 1] - red_start[c] <= kGatherLight) ? c : -1;
        }
        gather_light<W, LB>(bx, rec, words, box_start, nbr_start, nbr_idx, nbr_img, edge, red_start, red, gather,
                            task_kind, lane);
    }
    // heavy streams, kGatherParts parts each
    const int64_t nh = min((int64_t)hdr->n_heavy, heavy_cap);
    for (int64_t w = warp; w < nh * kGatherParts; w += nwarps) {
        const int32_t b = heavy[w / kGatherParts];
        gather_part(b, (int)(w % kGatherParts), rec, words, box_start, nbr_start, nbr_idx, nbr_img, edge, red_start[b],
                    red, gather, task_kind, lane);
    }
}

// box statistics, and for the redundant layout the per-box streams of the
// records already written in box order (words per record)
static int restructure_tail(Plan* p, void* ws, int words, cudaStream_t s) {
    const Layout& L = p->L;
    Header* hdr = at<Header>(ws, L.header);
    const int64_t bc = p->box_cap;
    float4* rec = at<float4>(ws, L.src);
    const bool red = p->layout == P2P_LAYOUT_REDUNDANT;
    int32_t* S = at<int32_t>(ws, L.box_S);
    // (the restructuring section of the header was zeroed by the records kernel)
    int32_t* red_start = red ? at<int32_t>(ws, L.red_start) : nullptr;
    unsigned long long* lb = at<unsigned long long>(ws, L.lookback) + lb_regions(p->n, bc).stats;   // stream bounds
    const LbRegions lr = lb_regions(p->n, bc);
    unsigned long long* lb2 = at<unsigned long long>(ws, L.lookback) + lr.stats2;
    int32_t* kinds = p->sym ? at<int32_t>(ws, L.task_kind) : nullptr;
    const unsigned stats_blocks = (unsigned)std::min<int64_t>(blocks_for(bc, kBoxTile), (int64_t)num_sms() * 8);
    P2P_CUDA_TRY(launch_pdl(k_box_stats, stats_blocks, 256, 0, s, at<int32_t>(ws, L.box_start),
                            at<int32_t>(ws, L.nbr_start), at<int32_t>(ws, L.nbr_idx), hdr, S,
                            red ? at<int32_t>(ws, L.red_self) : nullptr, red_start, lb, kinds,
                            p->sym ? at<int32_t>(ws, L.mirror) : nullptr, p->sym ? at<int32_t>(ws, L.bslot) : nullptr,
                            lb2, p->part_cap, red ? at<int32_t>(ws, L.heavy) : nullptr));
    P2P_LAUNCH_CHECK();
    if (red) {
        const int sms = num_sms();
        auto kern = words == 1 ? k_red_gather<1> : words == 2 ? k_red_gather<2> : k_red_gather<0>;
        P2P_CUDA_TRY(launch_pdl(kern, sms * 32, 128, 0, s, rec, words, at<int32_t>(ws, L.box_start), at<int32_t>(ws, L.nbr_start),
                                            at<int32_t>(ws, L.nbr_idx),
                                            p->periodic ? at<int32_t>(ws, L.nbr_img) : nullptr, p->edge, red_start,
                                            hdr, p->red_cap,
                                            at<float4>(ws, L.red_src),
                                            (p->flags & P2P_PLAN_GATHER_MAP) ? at<uint32_t>(ws, L.gather) : nullptr,
                                            kinds, at<int32_t>(ws, L.heavy), bc));
        P2P_LAUNCH_CHECK();
    } else if (is_pairtask(p->layout)) {
        return pairtask_restructure(p, ws, words, s);
    }
    return P2P_OK;
}

int restructure(Plan* p, const float* pos, const void* strength, void* ws, cudaStream_t s, const void* strength2) {
    const Layout& L = p->L;
    const int64_t n = p->n;
    const int32_t* perm = at<int32_t>(ws, L.perm);
    float4* rec = at<float4>(ws, L.src);
    const LbRegions lr = lb_regions(n, p->box_cap);
    unsigned long long* lbc = at<unsigned long long>(ws, L.lookback) + lr.stats;
    const int64_t lbc_words = lr.words - lr.stats;
    if (p->kind == P2P_GRAVITY) {
        P2P_CUDA_TRY(launch_pdl(k_records_gravity, blocks_for(n, 256), 256, 0, s, pos, static_cast<const float*>(strength),
                                perm, n, rec, lbc, lbc_words, at<Header>(ws, L.header)));
    } else {
        const int split = strength2 ? p->split : p->nrhs;
        LatticeArgs lat{};
        lat.on = p->pattern;
        if (p->pattern) {
            for (int a = 0; a < 3; ++a) lat.lo[a] = p->lo[a];
            lat.inv_h = 1.0f / p->grid_h;
            lat.t = p->grid_t;
            lat.sy = p->pat_sy;
            lat.sz = p->pat_sz;
            lat.scale = p->scale;
            lat.cmax = (1 << p->level) - 1;
            // the lattice flag belongs to this restructuring
            P2P_CUDA_TRY(launch_pdl(k_clear_flag, 1, 1, 0, s, at<Header>(ws, L.header), P2P_FLAG_LATTICE));
            P2P_LAUNCH_CHECK();
        }
        P2P_CUDA_TRY(launch_pdl(k_records_helmholtz, blocks_for(n, 256), 256, 0, s, pos, static_cast<const float2*>(strength),
                                                              static_cast<const float2*>(strength2), split, perm, n,
                                                              p->nrhs, p->rec_words, helmholtz_planar(p) ? 1 : 0, lat,
                                                              at<Header>(ws, L.header),
                                                              rec, lbc, lbc_words));
    }
    P2P_LAUNCH_CHECK();
    int st = restructure_tail(p, ws, p->rec_words, s);
    if (st) return st;
    p->src_ready = 1;
    return P2P_OK;
}

int restructure_adjoint(Plan* p, const float* pos, const void* a, const void* b, const void* c, void* ws, int* words,
                        cudaStream_t s) {
    const Layout& L = p->L;
    const int64_t n = p->n;
    const int32_t* perm = at<int32_t>(ws, L.perm);
    float4* rec = at<float4>(ws, L.src);
    const LbRegions lr = lb_regions(n, p->box_cap);
    unsigned long long* lbc = at<unsigned long long>(ws, L.lookback) + lr.stats;
    const int64_t lbc_words = lr.words - lr.stats;
    int w;
    if (p->kind == P2P_GRAVITY) {
        w = kGravityAdjointWords;
        if (w > p->rec_alloc_words) return P2P_ERR_UNSUPPORTED;
        P2P_CUDA_TRY(launch_pdl(k_records_grav_adjoint, blocks_for(n, 256), 256, 0, s, pos, static_cast<const float*>(a),
                                                                 static_cast<const float*>(b),
                                                                 static_cast<const float*>(c), perm, n, rec, lbc,
                                                                 lbc_words, at<Header>(ws, L.header)));
    } else {
        w = helmholtz_adjoint_words(p->nrhs);
        if (w > p->rec_alloc_words) return P2P_ERR_UNSUPPORTED;
        P2P_CUDA_TRY(launch_pdl(k_records_helm_adjoint, blocks_for(n, 256), 256, 0, s, pos, static_cast<const float2*>(a),
                                                                 static_cast<const float2*>(b), perm, n, p->nrhs, w,
                                                                 rec, lbc, lbc_words, at<Header>(ws, L.header)));
    }
    P2P_LAUNCH_CHECK();
    p->src_ready = 0;   // the forward records are overwritten
    *words = w;
    return restructure_tail(p, ws, w, s);
}

int build_items(Plan* p, void* ws, int tt, cudaStream_t s) {
    const Layout& L = p->L;
    Header* hdr = at<Header>(ws, L.header);
    const int64_t bc = p->box_cap;
    const int32_t* S = at<int32_t>(ws, L.box_S);
    int st0 = fill32(reinterpret_cast<char*>(hdr) + kOpSectionOffset, 0u, (sizeof(Header) - kOpSectionOffset) / 4, s);
    if (st0) return st0;
    Units U{at<int32_t>(ws, L.box_start), S, nullptr, nullptr, bc, nullptr};
    if (is_pairtask(p->layout)) {
        U.ent_box = at<int32_t>(ws, L.ent_box);
        U.nbr_idx = at<int32_t>(ws, L.nbr_idx);
        U.cap = 27 * bc;
        if (p->layout == P2P_LAYOUT_SYMMETRIC) U.task_kind = at<int32_t>(ws, L.task_kind);
    }
    P2P_CUDA_TRY(launch_pdl(k_items_count, blocks_for(U.cap, 256), 256, 0, s, U, hdr, tt));
    P2P_LAUNCH_CHECK();
    P2P_CUDA_TRY(launch_pdl(k_items_fill, blocks_for(U.cap, 256), 256, 0, s, U, hdr, tt, at<int2>(ws, L.items)));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

}  // namespace p2p
