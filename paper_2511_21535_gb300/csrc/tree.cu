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
#include "lookback.cuh"
#include "sort_scratch.cuh"

namespace p2p {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

// ---------------------------------------------------------------------------
// 1. keys (with every radix pass's digit counts)
// ---------------------------------------------------------------------------
// One sort tile per block: the box key of each particle, and the counts of
// each pass's digits over the tile, added to the global counts (gcount[pass *
// 256 + digit], zeroed before the launch).  Also clears the chained-scan
// scratch of the radix passes (sort_words words) and of the box and neighbour
// CSR kernels (lb_words words) that follow, and the dense key -> box table (-1).
__global__ void __launch_bounds__(kSortThreads) k_keys(const float* __restrict__ pos, int64_t n, float lo0,
                                                      float lo1, float lo2, float scale, int level,
                                                      uint32_t* __restrict__ keys, Header* hdr,
                                                      unsigned long long* __restrict__ lb, int64_t lb_words,
                                                      uint32_t* __restrict__ sort_st, int64_t sort_words,
                                                      int32_t* __restrict__ table, int64_t table_words,
                                                      int passes, int dbits, uint32_t* __restrict__ gcount) {
    pdl_wait();
    pdl_release();
    __shared__ int32_t cnt[kSortMaxPasses][256];
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = gid; t < lb_words; t += gstride) lb[t] = 0ull;
    for (int64_t t = gid; t < sort_words; t += gstride) sort_st[t] = 0u;
    // the dense key -> box table starts empty (-1); the box CSR kernel fills it
    for (int64_t t = gid; t < table_words; t += gstride) table[t] = -1;
    const uint32_t mask = (1u << dbits) - 1u;
    const int radix = (int)mask + 1;
    for (int t = threadIdx.x; t < kSortMaxPasses * 256; t += kSortThreads) (&cnt[0][0])[t] = 0;
    __syncthreads();
    const float side = (float)(1 << level);
    const int32_t cmax = (1 << level) - 1;
    const float lo[3] = {lo0, lo1, lo2};
    bool bad = false;
    // all of the thread's positions are loaded before any is used (independent loads in flight)
    float x[kSortItems][3];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = (int64_t)blockIdx.x * kSortTile + r * kSortThreads + threadIdx.x;
#pragma unroll
        for (int a = 0; a < 3; ++a) x[r][a] = i < n ? pos[3 * i + a] : lo[a];
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = (int64_t)blockIdx.x * kSortTile + r * kSortThreads + threadIdx.x;
        if (i < n) {
            uint32_t c[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // exactly one float32 subtraction and one float32 product, no contraction
                float u = __fmul_rn(__fsub_rn(x[r][a], lo[a]), scale);
                if (!(u >= 0.0f && u <= side)) {
                    bad = true;
                    u = 0.0f;
                }
                int32_t ci = (int32_t)floorf(u);
                c[a] = (uint32_t)(ci > cmax ? cmax : ci);
            }
            const uint32_t key = morton3(c[0], c[1], c[2]);
            keys[i] = key;
            for (int ps = 0; ps < passes; ++ps) atomicAdd(&cnt[ps][(key >> (ps * dbits)) & mask], 1);
        }
    }
    if (bad) atomicOr(&hdr->flags, P2P_FLAG_DOMAIN);
    __syncthreads();
    for (int t = threadIdx.x; t < passes * radix; t += kSortThreads) {
        const int ps = t / radix, d = t - ps * radix;
        const int32_t c = cnt[ps][d];
        if (c) atomicAdd(&gcount[ps * 256 + d], (uint32_t)c);
    }
}

// ---------------------------------------------------------------------------
// 2. stable radix sort, one launch per pass
// ---------------------------------------------------------------------------
// Each pass is a single-pass scatter with a decoupled look-back per digit
// (the scheme of Merrill & Garland's chained scan, lookback.cuh, run for all
// digits at once, as in Adinets & Merrill, "Onesweep", 2022): a block takes a
// ticket as its sort tile, counts the tile's digits, publishes the counts,
// and thread d walks back over the earlier tiles' status words of digit d,
// kLookWindow tiles per step, until it meets an inclusive prefix.  The destination of the tile's first
// key of digit d is then
//   (keys of smaller digits, all tiles) + (keys of digit d in earlier tiles).
// Status word of (tile, digit): (state << 30) | count; state 1 = the tile's
// own count, 2 = the inclusive prefix over tiles 0..tile (counts < 2^30).
// Word 0 of the pass's status region is the ticket counter.  Every wait is
// bounded: past kLookbackLimitNs the digit records P2P_FLAG_TIMEOUT and goes
// on with what it has (the order is then wrong but flagged).
constexpr uint32_t kStOwn = 1u << 30;
constexpr uint32_t kStPrefix = 2u << 30;
constexpr uint32_t kStValue = (1u << 30) - 1u;
constexpr int kLookWindow = 8;

__device__ __forceinline__ void st_store(uint32_t* p, uint32_t v) { *reinterpret_cast<volatile uint32_t*>(p) = v; }
__device__ __forceinline__ uint32_t st_load(const uint32_t* p) { return *reinterpret_cast<const volatile uint32_t*>(p); }

// Within a tile, keys are taken in index order: round-major, then warp, then
// lane.  A key's rank among equal digits is its rank inside its warp (match +
// popcount) plus the counts of earlier warps of the same round plus the
// counts of earlier rounds.
__global__ void __launch_bounds__(kSortThreads) k_radix_pass(const uint32_t* __restrict__ kin,
                                                            const int32_t* __restrict__ vin, int64_t n,
                                                            int shift, uint32_t mask,
                                                            const uint32_t* __restrict__ gcount,
                                                            uint32_t* st, uint32_t* __restrict__ kout,
                                                            int32_t* __restrict__ vout, Header* hdr) {
    pdl_wait();
    pdl_release();
    constexpr int W = kSortThreads / 32;
    __shared__ int32_t base[256];
    __shared__ int32_t wcnt[W][256];
    __shared__ int32_t woff[W][256];
    __shared__ int tile_s;
    const int radix = (int)mask + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) tile_s = (int)atomicAdd(st, 1u);
    for (int d = threadIdx.x; d < radix; d += kSortThreads) {
        base[d] = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    const int tile = tile_s;
    const int64_t tbase = (int64_t)tile * kSortTile;
    uint32_t key[kSortItems];
    int32_t val[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = tbase + r * kSortThreads + threadIdx.x;
        key[r] = 0;
        val[r] = 0;
        if (i < n) {
            key[r] = kin[i];
            val[r] = vin ? vin[i] : (int32_t)i;
        }
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r)
        if (tbase + r * kSortThreads + threadIdx.x < n) atomicAdd(&base[(key[r] >> shift) & mask], 1);
    __syncthreads();

    // look-back: thread d finds the keys of digit d in the earlier tiles
    int32_t excl = 0;
    if (threadIdx.x < radix) {
        uint32_t* sd = st + 1 + threadIdx.x;          // status of (t, d) at sd[t * radix]
        const int32_t own = base[threadIdx.x];
        if (tile == 0) {
            st_store(sd, kStPrefix | (uint32_t)own);
        } else {
            st_store(sd + (int64_t)tile * radix, kStOwn | (uint32_t)own);
            const uint64_t t0 = global_ns();
            int t = tile - 1;   // nearest tile not yet added
            for (;;) {
                // kLookWindow predecessors per round trip (independent loads)
                uint32_t v[kLookWindow];
#pragma unroll
                for (int j = 0; j < kLookWindow; ++j)
                    v[j] = t - j >= 0 ? st_load(sd + (int64_t)(t - j) * radix) : kStPrefix;   // before tile 0: 0
                bool done = false;
                int j = 0;
                for (; j < kLookWindow; ++j) {
                    const uint32_t state = v[j] >> 30;
                    if (state == 0u) break;           // not published yet: read again from here
                    excl += (int32_t)(v[j] & kStValue);
                    if (state == 2u) {
                        done = true;
                        break;
                    }
                }
                if (done) break;
                t -= j;
                if (j < kLookWindow && global_ns() - t0 > kLookbackLimitNs) {
                    atomicOr(&hdr->flags, P2P_FLAG_TIMEOUT);
                    break;
                }
            }
            st_store(sd + (int64_t)tile * radix, kStPrefix | (uint32_t)(excl + own));
        }
    }
    // keys of smaller digits over all tiles (exclusive scan of the global counts)
    const int32_t g = threadIdx.x < radix ? (int32_t)gcount[threadIdx.x] : 0;
    int32_t gtotal;
    const int32_t gex = block_excl_scan<kSortThreads>(g, &gtotal);
    if (threadIdx.x < radix) base[threadIdx.x] = gex + excl;
    __syncthreads();

    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const bool valid = tbase + r * kSortThreads + threadIdx.x < n;
        const uint32_t d = valid ? ((key[r] >> shift) & mask) : (uint32_t)radix;
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
            kout[p] = key[r];
            vout[p] = val[r];
        }
    }
}

// ---------------------------------------------------------------------------
// 3. box CSR: one pass over the sorted keys.  A box starts where the key
// changes; box indices are a chained scan of those starts across tiles
// (lookback.cuh).  The kernel also fills the dense key -> box table and
// closes the CSR (box_start[n_boxes] = n, the box count in the header).
// ---------------------------------------------------------------------------
constexpr int kCsrThreads = 256;
constexpr int kCsrItems = 8;
constexpr int kCsrTile = kCsrThreads * kCsrItems;
static_assert(kCsrTile == kCsrTileElems, "box CSR tile");

__global__ void __launch_bounds__(kCsrThreads) k_box_csr(const uint32_t* __restrict__ skey, int64_t n,
                                                        uint32_t* __restrict__ box_key,
                                                        int32_t* __restrict__ box_start,
                                                        int32_t* __restrict__ table, unsigned long long* lb,
                                                        Header* hdr) {
    pdl_wait();
    pdl_release();
    __shared__ int tile_s;
    __shared__ int32_t prefix_s;
    if (threadIdx.x == 0) tile_s = lb_ticket(lb);
    __syncthreads();
    const int tile = tile_s;
    const int64_t base = (int64_t)tile * kCsrTile + (int64_t)threadIdx.x * kCsrItems;
    uint32_t k[kCsrItems];
    int32_t cnt = 0;
    unsigned starts = 0;
    uint32_t prev = (base > 0 && base <= n) ? skey[base - 1] : 0xffffffffu;   // keys have <= 30 bits
#pragma unroll
    for (int j = 0; j < kCsrItems; ++j) {
        const int64_t i = base + j;
        k[j] = 0;
        if (i < n) {
            k[j] = skey[i];
            if (k[j] != prev) {
                starts |= 1u << j;
                ++cnt;
            }
            prev = k[j];
        }
    }
    int32_t agg;
    const int32_t off = block_excl_scan<kCsrThreads>(cnt, &agg);
    if (threadIdx.x < 32) {
        const int32_t ex = lb_exclusive(lb, tile, agg, hdr);
        if (threadIdx.x == 0) prefix_s = ex;
    }
    __syncthreads();
    int32_t b = prefix_s + off;
#pragma unroll
    for (int j = 0; j < kCsrItems; ++j) {
        if (starts & (1u << j)) {
            box_key[b] = k[j];
            box_start[b] = (int32_t)(base + j);
            if (table) table[k[j]] = b;
            ++b;
        }
    }
    if (n - 1 >= base && n - 1 < base + kCsrItems) {   // the thread holding the last particle
        box_start[b] = (int32_t)n;
        hdr->n_boxes = b;
    }
}

// ---------------------------------------------------------------------------
// 4. neighbour lists
// ---------------------------------------------------------------------------
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

// Lane l < 27 of a warp examines the neighbour cell of box b at offset
// (l % 3 - 1, l / 3 % 3 - 1, l / 9 - 1) and returns the box found there (or
// -1).  Periodic: cells wrap and *code receives the image code
// (ox+1) + 3(oy+1) + 9(oz+1) of the domain copy of that box which b meets.
__device__ __forceinline__ int32_t neighbour_cell(int64_t b, const uint32_t* __restrict__ box_key, int32_t nb,
                                                  int level, const int32_t* __restrict__ table, int periodic,
                                                  int lane, int32_t* code) {
    const uint32_t key = box_key[b];
    const int32_t cx = (int32_t)compact3(key), cy = (int32_t)compact3(key >> 1), cz = (int32_t)compact3(key >> 2);
    const int32_t side = 1 << level;
    int32_t c = -1;
    *code = 13;
    if (lane < 27) {
        int32_t x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
        if (periodic) {
            int32_t ox = 0, oy = 0, oz = 0;
            if (x < 0) { x += side; ox = -1; } else if (x >= side) { x -= side; ox = 1; }
            if (y < 0) { y += side; oy = -1; } else if (y >= side) { y -= side; oy = 1; }
            if (z < 0) { z += side; oz = -1; } else if (z >= side) { z -= side; oz = 1; }
            *code = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
            c = find_box(morton3(x, y, z), box_key, nb, table);
        } else if (x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
            c = find_box(morton3(x, y, z), box_key, nb, table);
        }
    }
    return c;
}

// Neighbour CSR in one pass: a tile of kNbrTile boxes, four per warp; the list
// lengths are scanned across tiles (lookback.cuh) and each list is written
// ascending (a found box's rank = how many found indices are smaller; they
// are distinct).  The tile holding the last box closes the CSR.  A grid of a
// few blocks per SM takes tiles by ticket until the boxes run out (the box
// count is known on the device only; a grid sized for the capacity would
// launch mostly empty blocks on sparse distributions).
constexpr int kNbrPerWarp = 4;
constexpr int kNbrTile = 8 * kNbrPerWarp;
static_assert(kNbrTile == kBoxTile, "neighbour CSR tile");

__global__ void __launch_bounds__(256) k_nbr_csr(const uint32_t* __restrict__ box_key, Header* hdr, int level,
                                                const int32_t* __restrict__ table, int32_t* __restrict__ nbr_start,
                                                int32_t* __restrict__ nbr_idx, int32_t* __restrict__ nbr_img,
                                                int periodic, unsigned long long* lb) {
    pdl_wait();
    pdl_release();
    __shared__ int tile_s;
    __shared__ int32_t cnt_s[kNbrTile];
    __shared__ int32_t pre_s[kNbrTile + 1];
    const int32_t nb = hdr->n_boxes;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) tile_s = lb_ticket(lb);
        __syncthreads();
        const int tile = tile_s;
        const int64_t b0 = (int64_t)tile * kNbrTile;
        if (b0 >= nb) return;   // past the last box (whole block): no later tile waits on it
        int32_t c[kNbrPerWarp], code[kNbrPerWarp];
#pragma unroll
        for (int q = 0; q < kNbrPerWarp; ++q) {
            const int64_t b = b0 + warp * kNbrPerWarp + q;
            c[q] = -1;
            code[q] = 13;
            if (b < nb) c[q] = neighbour_cell(b, box_key, nb, level, table, periodic, lane, &code[q]);
            const int32_t found = __popc(__ballot_sync(FULL, c[q] >= 0));
            if (lane == 0) cnt_s[warp * kNbrPerWarp + q] = found;
        }
        __syncthreads();
        if (warp == 0) {
            const int32_t v = cnt_s[lane];
            const int32_t inc = warp_incl_scan(v);
            const int32_t agg = __shfl_sync(FULL, inc, 31);
            const int32_t ex = lb_exclusive(lb, tile, agg, hdr);
            pre_s[lane] = ex + inc - v;
            if (lane == 31) pre_s[kNbrTile] = ex + inc;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kNbrPerWarp; ++q) {
            const int64_t b = b0 + warp * kNbrPerWarp + q;
            if (b >= nb) break;
            const int32_t start = pre_s[warp * kNbrPerWarp + q];
            if (lane == 0) nbr_start[b] = start;
            int rank = 0;
#pragma unroll
            for (int j = 0; j < 27; ++j) {
                const int32_t v = __shfl_sync(FULL, c[q], j);
                rank += (v >= 0 && v < c[q]) ? 1 : 0;
            }
            if (c[q] >= 0) {
                nbr_idx[start + rank] = c[q];
                if (nbr_img) nbr_img[start + rank] = code[q];
            }
        }
        if (threadIdx.x == 0 && nb - 1 >= b0 && nb - 1 < b0 + kNbrTile) {
            nbr_start[nb] = pre_s[kNbrTile];
            hdr->n_nbr = pre_s[kNbrTile];
        }
        __syncthreads();   // the shared tile state is reused by the next tile
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

int tree_build(Plan* p, const float* pos, void* ws, cudaStream_t s) {
    const Layout& L = p->L;
    Header* hdr = at<Header>(ws, L.header);
    const int64_t n = p->n;
    uint32_t* ka = at<uint32_t>(ws, L.keys_a);
    uint32_t* kb = at<uint32_t>(ws, L.keys_b);
    int32_t* va = at<int32_t>(ws, L.vals_a);
    int32_t* perm = at<int32_t>(ws, L.perm);
    uint32_t* skey = at<uint32_t>(ws, L.sorted_key);

    // radix passes over 3*level key bits, equal digit widths <= 8 bits
    int passes = 0, dbits = 0;
    sort_digits(p->level, &passes, &dbits);
    const uint32_t mask = (1u << dbits) - 1u;
    const int tiles = p->sort_tiles;
    uint32_t* gcount = at<uint32_t>(ws, L.hist);
    uint32_t* sort_st = gcount + kSortCountWords;
    const int64_t pass_words = sort_pass_words((int)mask + 1, tiles);

    // clear the tree and restructuring sections of the header (counts and flags) and the digit counts
    int st0 = clear2(hdr, kOpSectionOffset / 4, gcount, kSortCountWords, s);
    if (st0) return st0;

    const LbRegions lr = lb_regions(n, p->box_cap);
    unsigned long long* lb = at<unsigned long long>(ws, L.lookback);
    int32_t* table = p->use_table ? at<int32_t>(ws, L.table) : nullptr;
    const int64_t table_words = p->use_table ? ((int64_t)1 << (3 * p->level)) : 0;
    P2P_CUDA_TRY(launch_pdl(k_keys, tiles, kSortThreads, 0, s, pos, n, p->lo[0], p->lo[1], p->lo[2], p->scale,
                            p->level, ka, hdr, lb, lr.tree_words, sort_st, passes * pass_words, table, table_words,
                            passes, dbits, gcount));
    P2P_LAUNCH_CHECK();

    // ping-pong so that the last pass lands in (skey, perm)
    const uint32_t* kin = ka;
    const int32_t* vin = nullptr;  // first pass: values are the original indices
    for (int ps = 0; ps < passes; ++ps) {
        const int remaining = passes - 1 - ps;
        uint32_t* kout = (remaining % 2 == 0) ? skey : kb;
        int32_t* vout = (remaining % 2 == 0) ? perm : va;
        if (kout == kin) kout = (kout == skey) ? kb : skey;  // never in place
        P2P_CUDA_TRY(launch_pdl(k_radix_pass, tiles, kSortThreads, 0, s, kin, vin, n, ps * dbits, mask,
                                (const uint32_t*)(gcount + ps * 256), sort_st + ps * pass_words, kout, vout, hdr));
        P2P_LAUNCH_CHECK();
        kin = kout;
        vin = vout;
    }
    if (kin != skey) {  // cannot happen with the parity above; kept as a guard
        P2P_CUDA_TRY(cudaMemcpyAsync(skey, kin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        P2P_CUDA_TRY(cudaMemcpyAsync(perm, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }

    // box CSR (and the dense key -> box table, cleared by k_keys)
    uint32_t* box_key = at<uint32_t>(ws, L.box_key);
    int32_t* box_start = at<int32_t>(ws, L.box_start);
    P2P_CUDA_TRY(launch_pdl(k_box_csr, blocks_for(n, kCsrTile), kCsrThreads, 0, s, skey, n, box_key, box_start,
                            table, lb + lr.csr, hdr));
    P2P_LAUNCH_CHECK();

    // neighbour lists
    const int64_t bc = p->box_cap;
    int32_t* nimg = p->periodic ? at<int32_t>(ws, L.nbr_img) : nullptr;
    const unsigned nbr_blocks = (unsigned)std::min<int64_t>(blocks_for(bc, kNbrTile), (int64_t)num_sms() * 8);
    P2P_CUDA_TRY(launch_pdl(k_nbr_csr, nbr_blocks, 256, 0, s, box_key, hdr, p->level, table,
                            at<int32_t>(ws, L.nbr_start), at<int32_t>(ws, L.nbr_idx), nimg, p->periodic,
                            lb + lr.nbr));
    P2P_LAUNCH_CHECK();
    p->tree_ready = 1;
    p->src_ready = 0;
    return P2P_OK;
}

// ---------------------------------------------------------------------------
// import of a caller-built structure
// ---------------------------------------------------------------------------
// An imported structure is checked before anything indexes through it:
// perm in [0, n), box bounds strictly increasing from 0 to n, neighbour
// bounds non-decreasing from 0 to n_nbr with at most 27 entries a box, and
// neighbour indices in [0, n_boxes).  A violation sets P2P_FLAG_CAPACITY;
// every later kernel of the plan then skips its work.
__global__ void __launch_bounds__(256) k_validate_import(const int32_t* __restrict__ perm, int64_t n,
                                                        const int32_t* __restrict__ box_start, int32_t nb,
                                                        const int32_t* __restrict__ nbr_start,
                                                        const int32_t* __restrict__ nbr_idx, int32_t ne,
                                                        Header* hdr) {
    pdl_wait();
    pdl_release();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t i = t0; i < n; i += stride) bad |= perm[i] < 0 || perm[i] >= n;
    for (int64_t b = t0; b <= nb; b += stride) {
        if (b == 0) bad |= box_start[0] != 0 || nbr_start[0] != 0;
        if (b == nb) bad |= box_start[nb] != n || nbr_start[nb] != ne;
        if (b < nb) {
            bad |= box_start[b + 1] <= box_start[b];
            const int32_t d = nbr_start[b + 1] - nbr_start[b];
            bad |= d < 0 || d > 27;
        }
    }
    for (int64_t e = t0; e < ne; e += stride) bad |= nbr_idx[e] < 0 || nbr_idx[e] >= nb;
    if (bad) atomicOr(&hdr->flags, P2P_FLAG_CAPACITY);
}

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
    P2P_CUDA_TRY(launch_pdl(k_validate_import, (unsigned)num_sms() * 4, 256, 0, s, at<int32_t>(ws, L.perm), p->n,
                            at<int32_t>(ws, L.box_start), n_boxes, at<int32_t>(ws, L.nbr_start),
                            at<int32_t>(ws, L.nbr_idx), n_nbr, hdr));
    P2P_LAUNCH_CHECK();
    p->tree_ready = 1;
    p->src_ready = 0;
    return P2P_OK;
}

}  // namespace p2p
