// Device-wide exclusive scan of int32 counts (CSR offsets of boxes, neighbour
// lists, redundant streams and radix-sort digit histograms).
//
// Three phases (block reduce -> scan of block sums -> block scan + offset),
// no inter-block waiting.  Lengths may be given on the device so that the
// whole tree build runs without a host round trip.
#include <algorithm>

#include "common.cuh"
#include "device.cuh"
#include "sort_scratch.cuh"

namespace p2p {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;   // elements per block
constexpr int64_t kSingleBlockMax = 1 << 16;              // one-kernel path up to this size

__device__ __forceinline__ int64_t eff_len(int64_t n_cap, const int32_t* d_len) {
    if (!d_len) return n_cap;
    int64_t l = *d_len;
    return l < n_cap ? (l < 0 ? 0 : l) : n_cap;
}

// one block scans everything, chunk by chunk, carrying the running total
__global__ void __launch_bounds__(kScanThreads) k_scan_single(const int32_t* in, int32_t* out, int64_t n_cap,
                                                             const int32_t* d_len, int32_t* d_total) {
    pdl_wait();
    pdl_release();
    const int64_t len = eff_len(n_cap, d_len);
    int32_t carry = 0;
    for (int64_t base = 0; base < n_cap; base += kScanChunk) {
        int32_t v[kScanItems];
        int32_t s = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
            v[j] = (i < len) ? in[i] : 0;
            s += v[j];
        }
        int32_t tot;
        int32_t ex = block_excl_scan<kScanThreads>(s, &tot) + carry;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
            if (i < n_cap) out[i] = ex;
            ex += v[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        out[n_cap] = carry;
        if (d_total) *d_total = carry;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* in, int64_t n_cap,
                                                             const int32_t* d_len, int32_t* block_sums) {
    pdl_wait();
    pdl_release();
    const int64_t len = eff_len(n_cap, d_len);
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    int32_t s = 0;
    if (base < len) {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
            if (i < len) s += in[i];
        }
    }
    int32_t tot;
    block_excl_scan<kScanThreads>(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const int32_t* in, int32_t* out, int64_t n_cap,
                                                            const int32_t* d_len, const int32_t* block_off,
                                                            int32_t* d_total, int nblocks) {
    pdl_wait();
    pdl_release();
    const int64_t len = eff_len(n_cap, d_len);
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
        v[j] = (i < len) ? in[i] : 0;
        s += v[j];
    }
    int32_t tot;
    int32_t ex = block_excl_scan<kScanThreads>(s, &tot) + block_off[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
        if (i < n_cap) out[i] = ex;
        ex += v[j];
    }
    if (blockIdx.x == nblocks - 1 && threadIdx.x == 0) {
        int32_t total = block_off[nblocks];
        out[n_cap] = total;
        if (d_total) *d_total = total;
    }
}

__global__ void __launch_bounds__(256) k_fill32(uint32_t* __restrict__ dst, uint32_t value, int64_t count) {
    pdl_wait();
    pdl_release();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) dst[i] = value;
}

// two ranges in one launch (value 0)
__global__ void __launch_bounds__(256) k_clear2(uint32_t* __restrict__ a, int64_t na, uint32_t* __restrict__ b,
                                               int64_t nb) {
    pdl_wait();
    pdl_release();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride) {
        if (i < na) a[i] = 0u;
        else b[i - na] = 0u;
    }
}

int clear2(void* a, int64_t na, void* b, int64_t nb, cudaStream_t s) {
    if (na + nb <= 0) return P2P_OK;
    const int64_t blocks = std::min<int64_t>((na + nb + 255) / 256, (int64_t)num_sms() * 8);
    P2P_CUDA_TRY(launch_pdl(k_clear2, (unsigned)blocks, 256, 0, s, static_cast<uint32_t*>(a), na,
                            static_cast<uint32_t*>(b), nb));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

int fill32(void* dst, uint32_t value, int64_t count, cudaStream_t s) {
    if (count <= 0) return P2P_OK;
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)num_sms() * 8);
    P2P_CUDA_TRY(launch_pdl(k_fill32, (unsigned)blocks, 256, 0, s, static_cast<uint32_t*>(dst), value, count));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

size_t scan_scratch_bytes(int64_t n_cap) {
    int64_t nb = (n_cap + kScanChunk - 1) / kScanChunk;
    return (size_t)(nb + 1) * 2 * sizeof(int32_t) + 256;
}

int scan_exclusive(const int32_t* in, int32_t* out, int64_t n_cap, const int32_t* d_len,
                   int32_t* d_total, int32_t* scratch, cudaStream_t s) {
    if (n_cap <= 0) return P2P_ERR_INVALID_ARG;
    if (n_cap <= kSingleBlockMax) {
        P2P_CUDA_TRY(launch_pdl(k_scan_single, 1, kScanThreads, 0, s, in, out, n_cap, d_len, d_total));
        P2P_LAUNCH_CHECK();
        return P2P_OK;
    }
    int nblocks = (int)((n_cap + kScanChunk - 1) / kScanChunk);
    int32_t* sums = scratch;
    int32_t* offs = scratch + (nblocks + 1);
    P2P_CUDA_TRY(launch_pdl(k_scan_reduce, nblocks, kScanThreads, 0, s, in, n_cap, d_len, sums));
    P2P_LAUNCH_CHECK();
    P2P_CUDA_TRY(launch_pdl(k_scan_single, 1, kScanThreads, 0, s, sums, offs, nblocks, nullptr, nullptr));
    P2P_LAUNCH_CHECK();
    P2P_CUDA_TRY(launch_pdl(k_scan_final, nblocks, kScanThreads, 0, s, in, out, n_cap, d_len, offs, d_total, nblocks));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

}  // namespace p2p
