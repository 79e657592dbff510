// Collect, part 1: the leaf-box structure, built on the device.
//
//  1. box key of every particle (float32 boxing rule, Morton interleave);
//  2. stable LSD radix sort of (key, original index) -> perm;
//  3. box CSR over the sorted particles (non-empty boxes, ascending key);
//  4. E2 neighbour lists (Section 5.1 / Table 5: the same-level boxes at
//     Chebyshev distance <= 1, self included), ascending key, as CSR.
//
// Everything runs on the caller's stream with device-side counts: no host
// synchronisation, so the build can be captured in a CUDA graph.
#include <algorithm>

#include "common.cuh"
#include "device.cuh"

namespace p2p {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

// ---------------------------------------------------------------------------
// 1. keys
// ---------------------------------------------------------------------------
__global__ void k_keys(const float* __restrict__ pos, int64_t n, float lo0, float lo1, float lo2,
                       float scale, int level, uint32_t* __restrict__ keys, Header* hdr) {
    pdl_wait();
    pdl_release();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float side = (float)(1 << level);
    const int32_t cmax = (1 << level) - 1;
    const float lo[3] = {lo0, lo1, lo2};
    uint32_t c[3];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // exactly one float32 subtraction and one float32 product, no contraction
        float u = __fmul_rn(__fsub_rn(pos[3 * i + a], lo[a]), scale);
        if (!(u >= 0.0f && u <= side)) {
            bad = true;
            u = 0.0f;
        }
        int32_t ci = (int32_t)floorf(u);
        c[a] = (uint32_t)(ci > cmax ? cmax : ci);
    }
    if (bad) atomicOr(&hdr->flags, P2P_FLAG_DOMAIN);
    keys[i] = morton3(c[0], c[1], c[2]);
}

// ---------------------------------------------------------------------------
// 2. stable radix sort
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys, int64_t n,
                                                            int shift, uint32_t mask, int32_t* hist, int tiles) {
    pdl_wait();
    pdl_release();
    __shared__ int32_t cnt[256];
    const int radix = (int)mask + 1;
    for (int d = threadIdx.x; d < radix; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & mask], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += kSortThreads) hist[(int64_t)d * tiles + blockIdx.x] = cnt[d];
}

// Stable scatter.  Within a tile, keys are taken in index order: round-major,
// then warp, then lane.  A key's rank among equal digits is its rank inside
// its warp (match + popcount) plus the counts of earlier warps of the same
// round plus the counts of earlier rounds.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                               const int32_t* __restrict__ vin, int64_t n,
                                                               int shift, uint32_t mask,
                                                               const int32_t* __restrict__ hist, int tiles,
                                                               uint32_t* __restrict__ kout,
                                                               int32_t* __restrict__ vout) {
    pdl_wait();
    pdl_release();
    constexpr int W = kSortThreads / 32;
    __shared__ int32_t base[256];
    __shared__ int32_t wcnt[W][256];
    __shared__ int32_t woff[W][256];
    const int radix = (int)mask + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < radix; d += kSortThreads) {
        base[d] = hist[(int64_t)d * tiles + blockIdx.x];
#pragma unroll
        for (int w = 0; w < W; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = tbase + r * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        uint32_t key = 0;
        int32_t val = 0;
        if (valid) {
            key = kin[i];
            val = vin ? vin[i] : (int32_t)i;
        }
        const uint32_t d = valid ? ((key >> shift) & mask) : (uint32_t)radix;
        const uint32_t m = __match_any_sync(FULL, d);
        const int rank = __popc(m & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(m);
        __syncthreads();
        for (int dd = threadIdx.x; dd < radix; dd += kSortThreads) {
            int32_t run = base[dd];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                int32_t c = wcnt[w][dd];
                woff[w][dd] = run;
                run += c;
                wcnt[w][dd] = 0;
            }
            base[dd] = run;
        }
        __syncthreads();
        if (valid) {
            const int32_t p = woff[warp][d] + rank;
            kout[p] = key;
            vout[p] = val;
        }
    }
}

// ---------------------------------------------------------------------------
// 3. box CSR
// ---------------------------------------------------------------------------
__global__ void k_box_flags(const uint32_t* __restrict__ skey, int64_t n, int32_t* __restrict__ flag) {
    pdl_wait();
    pdl_release();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || skey[i] != skey[i - 1]) ? 1 : 0;
}

// flag_scan[i] = number of boxes starting before i; n_boxes already in hdr
__global__ void k_box_emit(const uint32_t* __restrict__ skey, int64_t n, const int32_t* __restrict__ flag_scan,
                           uint32_t* __restrict__ box_key, int32_t* __restrict__ box_start) {
    pdl_wait();
    pdl_release();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0 || skey[i] != skey[i - 1]) {
        const int32_t b = flag_scan[i];
        box_key[b] = skey[i];
        box_start[b] = (int32_t)i;
    }
    if (i == n - 1) box_start[flag_scan[n]] = (int32_t)n;
}

// ---------------------------------------------------------------------------
// 4. neighbour lists
// ---------------------------------------------------------------------------
__global__ void k_table_fill(const uint32_t* __restrict__ box_key, const Header* hdr, int32_t* __restrict__ table) {
    pdl_wait();
    pdl_release();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hdr->n_boxes) return;
    table[box_key[b]] = (int32_t)b;
}

__device__ __forceinline__ int32_t find_box(uint32_t key, const uint32_t* __restrict__ box_key, int32_t nb,
                                            const int32_t* __restrict__ table) {
    if (table) return table[key];
    int32_t lo = 0, hi = nb;  // first index with box_key >= key
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (box_key[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < nb && box_key[lo] == key) ? lo : -1;
}

// One warp per box: lane l < 27 examines the neighbour cell at offset
// (l % 3 - 1, l / 3 % 3 - 1, l / 9 - 1) and looks it up; the found box
// indices are ranked across the warp so the list is written ascending.
// count mode (nbr_start == nullptr): cnt[b] = |N(b)|; write mode: fill nbr_idx.
// Periodic: cells wrap and the image code (ox+1) + 3(oy+1) + 9(oz+1) records
// which domain image of the neighbour's sources the box meets.
__device__ __forceinline__ void neighbours_of(int64_t b, const uint32_t* __restrict__ box_key, int32_t nb, int level,
                                             const int32_t* __restrict__ table, int32_t* __restrict__ cnt,
                                             const int32_t* __restrict__ nbr_start, int32_t* __restrict__ nbr_idx,
                                             int32_t* __restrict__ nbr_img, int periodic, int lane) {
    const uint32_t key = box_key[b];
    const int32_t cx = (int32_t)compact3(key), cy = (int32_t)compact3(key >> 1), cz = (int32_t)compact3(key >> 2);
    const int32_t side = 1 << level;
    int32_t c = -1, code = 13;
    if (lane < 27) {
        int32_t x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
        if (periodic) {
            int32_t ox = 0, oy = 0, oz = 0;
            if (x < 0) { x += side; ox = -1; } else if (x >= side) { x -= side; ox = 1; }
            if (y < 0) { y += side; oy = -1; } else if (y >= side) { y -= side; oy = 1; }
            if (z < 0) { z += side; oz = -1; } else if (z >= side) { z -= side; oz = 1; }
            code = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
            c = find_box(morton3(x, y, z), box_key, nb, table);
        } else if (x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
            c = find_box(morton3(x, y, z), box_key, nb, table);
        }
    }
    const unsigned found = __ballot_sync(FULL, c >= 0);
    if (!nbr_start) {
        if (lane == 0) cnt[b] = __popc(found);
        return;
    }
    int rank = 0;  // found indices are distinct: rank = how many are smaller
#pragma unroll
    for (int j = 0; j < 27; ++j) {
        const int32_t v = __shfl_sync(FULL, c, j);
        rank += (v >= 0 && v < c) ? 1 : 0;
    }
    if (c >= 0) {
        nbr_idx[nbr_start[b] + rank] = c;
        if (nbr_img) nbr_img[nbr_start[b] + rank] = code;
    }
}

// Grid-stride over the boxes that exist (the count is on the device); the
// count array needs no zeros beyond it because its scan reads only n_boxes.
__global__ void __launch_bounds__(256) k_neighbours(const uint32_t* __restrict__ box_key, const Header* hdr,
                                                   int level, const int32_t* __restrict__ table,
                                                   int32_t* __restrict__ cnt, const int32_t* __restrict__ nbr_start,
                                                   int32_t* __restrict__ nbr_idx, int32_t* __restrict__ nbr_img,
                                                   int periodic) {
    pdl_wait();
    pdl_release();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = hdr->n_boxes;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += nwarps)
        neighbours_of(b, box_key, nb, level, table, cnt, nbr_start, nbr_idx, nbr_img, periodic, lane);
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

int tree_build(Plan* p, const float* pos, void* ws, cudaStream_t s) {
    const Layout& L = p->L;
    Header* hdr = at<Header>(ws, L.header);
    const int64_t n = p->n;
    // clear the tree and restructuring sections of the header (counts and flags)
    int st0 = fill32(hdr, 0u, kOpSectionOffset / 4, s);
    if (st0) return st0;

    uint32_t* ka = at<uint32_t>(ws, L.keys_a);
    uint32_t* kb = at<uint32_t>(ws, L.keys_b);
    int32_t* va = at<int32_t>(ws, L.vals_a);
    int32_t* perm = at<int32_t>(ws, L.perm);
    uint32_t* skey = at<uint32_t>(ws, L.sorted_key);
    int32_t* hist = at<int32_t>(ws, L.hist);
    int32_t* scratch = at<int32_t>(ws, L.scan_tmp);

    P2P_CUDA_TRY(launch_pdl(k_keys, blocks_for(n, 256), 256, 0, s, pos, n, p->lo[0], p->lo[1], p->lo[2], p->scale, p->level, ka, hdr));
    P2P_LAUNCH_CHECK();

    // radix passes over 3*level key bits, equal digit widths <= 8 bits
    const int bits = 3 * p->level;
    const int passes = (bits + 7) / 8;
    const int dbits = (bits + passes - 1) / passes;
    const uint32_t mask = (1u << dbits) - 1u;
    const int tiles = p->sort_tiles;
    // ping-pong so that the last pass lands in (skey, perm)
    const uint32_t* kin = ka;
    const int32_t* vin = nullptr;  // first pass: values are the original indices
    for (int ps = 0; ps < passes; ++ps) {
        const int remaining = passes - 1 - ps;
        uint32_t* kout = (remaining % 2 == 0) ? skey : kb;
        int32_t* vout = (remaining % 2 == 0) ? perm : va;
        if (kout == kin) kout = (kout == skey) ? kb : skey;  // never in place
        const int shift = ps * dbits;
        P2P_CUDA_TRY(launch_pdl(k_radix_hist, tiles, kSortThreads, 0, s, kin, n, shift, mask, hist, tiles));
        P2P_LAUNCH_CHECK();
        int st = scan_exclusive(hist, hist, (int64_t)(mask + 1) * tiles, nullptr, nullptr, scratch, s);
        if (st) return st;
        P2P_CUDA_TRY(launch_pdl(k_radix_scatter, tiles, kSortThreads, 0, s, kin, vin, n, shift, mask, hist, tiles, kout, vout));
        P2P_LAUNCH_CHECK();
        kin = kout;
        vin = vout;
    }
    if (kin != skey) {  // cannot happen with the parity above; kept as a guard
        P2P_CUDA_TRY(cudaMemcpyAsync(skey, kin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        P2P_CUDA_TRY(cudaMemcpyAsync(perm, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }

    // box CSR
    int32_t* flag = at<int32_t>(ws, L.flags);
    uint32_t* box_key = at<uint32_t>(ws, L.box_key);
    int32_t* box_start = at<int32_t>(ws, L.box_start);
    P2P_CUDA_TRY(launch_pdl(k_box_flags, blocks_for(n, 256), 256, 0, s, skey, n, flag));
    P2P_LAUNCH_CHECK();
    int st = scan_exclusive(flag, flag, n, nullptr, &hdr->n_boxes, scratch, s);
    if (st) return st;
    P2P_CUDA_TRY(launch_pdl(k_box_emit, blocks_for(n, 256), 256, 0, s, skey, n, flag, box_key, box_start));
    P2P_LAUNCH_CHECK();

    // neighbour lists
    const int64_t bc = p->box_cap;
    int32_t* table = nullptr;
    if (p->use_table) {
        table = at<int32_t>(ws, L.table);
        st = fill32(table, 0xffffffffu, (int64_t)1 << (3 * p->level), s);
        if (st) return st;
        P2P_CUDA_TRY(launch_pdl(k_table_fill, blocks_for(bc, 256), 256, 0, s, box_key, hdr, table));
        P2P_LAUNCH_CHECK();
    }
    int32_t* ncnt = at<int32_t>(ws, L.nbr_cnt);
    int32_t* nstart = at<int32_t>(ws, L.nbr_start);
    int32_t* nidx = at<int32_t>(ws, L.nbr_idx);
    const unsigned nbl = (unsigned)std::min<int64_t>(blocks_for(bc * 32, 256), (int64_t)num_sms() * 16);
    int32_t* nimg = p->periodic ? at<int32_t>(ws, L.nbr_img) : nullptr;
    P2P_CUDA_TRY(launch_pdl(k_neighbours, nbl, 256, 0, s, box_key, hdr, p->level, table, ncnt, nullptr, nullptr, nullptr, p->periodic));
    P2P_LAUNCH_CHECK();
    st = scan_exclusive(ncnt, nstart, bc, &hdr->n_boxes, &hdr->n_nbr, scratch, s);
    if (st) return st;
    P2P_CUDA_TRY(launch_pdl(k_neighbours, nbl, 256, 0, s, box_key, hdr, p->level, table, ncnt, nstart, nidx, nimg, p->periodic));
    P2P_LAUNCH_CHECK();
    p->tree_ready = 1;
    p->src_ready = 0;
    return P2P_OK;
}

// ---------------------------------------------------------------------------
// import of a caller-built structure
// ---------------------------------------------------------------------------
__global__ void k_set_counts(Header* hdr, int32_t n_boxes, int32_t n_nbr) {
    pdl_wait();
    pdl_release();
    hdr->n_boxes = n_boxes;
    hdr->n_nbr = n_nbr;
}

int tree_import(Plan* p, const int32_t* perm, const int32_t* box_start, int32_t n_boxes, const int32_t* nbr_start,
                const int32_t* nbr_idx, int32_t n_nbr, void* ws, cudaStream_t s) {
    const Layout& L = p->L;
    Header* hdr = at<Header>(ws, L.header);
    if (n_boxes < 1 || n_boxes > p->n || n_nbr < n_boxes || (int64_t)n_nbr > 27 * (int64_t)n_boxes)
        return P2P_ERR_INVALID_ARG;
    P2P_CUDA_TRY(cudaMemsetAsync(hdr, 0, kOpSectionOffset, s));
    P2P_CUDA_TRY(cudaMemcpyAsync(at<int32_t>(ws, L.perm), perm, p->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    P2P_CUDA_TRY(cudaMemcpyAsync(at<int32_t>(ws, L.box_start), box_start, (n_boxes + 1) * sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, s));
    P2P_CUDA_TRY(cudaMemcpyAsync(at<int32_t>(ws, L.nbr_start), nbr_start, (n_boxes + 1) * sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, s));
    P2P_CUDA_TRY(cudaMemcpyAsync(at<int32_t>(ws, L.nbr_idx), nbr_idx, (size_t)n_nbr * sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, s));
    P2P_CUDA_TRY(launch_pdl(k_set_counts, 1, 1, 0, s, hdr, n_boxes, n_nbr));
    P2P_LAUNCH_CHECK();
    p->tree_ready = 1;
    p->src_ready = 0;
    return P2P_OK;
}

}  // namespace p2p
