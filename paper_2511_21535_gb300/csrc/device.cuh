// Device-side helpers: warp/block scans, Morton keys, mbarrier and 1-D bulk
// copy (TMA) wrappers written as inline PTX for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace p2p {

// ---------------------------------------------------------------------------
// Morton (Z-order) keys: bit b of x, y, z -> key bits 3b, 3b+1, 3b+2
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spread3(uint32_t v) {   // 10 bits -> every third bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t compact3(uint32_t v) {  // inverse of spread3
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x000003ffu;
    return v;
}
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan for blockDim.x == NT (multiple of 32, <= 1024).
// Returns the exclusive prefix; *total receives the block total.
template <int NT>
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* total) {
    __shared__ int32_t warp_off[32];
    __shared__ int32_t block_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = warp_incl_scan(v);
    if (lane == 31) warp_off[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = (lane < NT / 32) ? warp_off[lane] : 0;
        int32_t wi = warp_incl_scan(w);
        warp_off[lane] = wi - w;
        if (lane == 31) block_total = wi;
    }
    __syncthreads();
    int32_t res = warp_off[warp] + inc - v;
    int32_t tot = block_total;
    __syncthreads();  // the shared slots may be reused by the next call
    *total = tot;
    return res;
}

// Sums of four per-lane values v0..v3 over the warp in one transposed
// reduction (6 shuffles instead of 20): the halves exchange so that lanes
// 0-15 keep sources {0,1} and 16-31 keep {2,3}, then octets split those, then
// three butterfly steps; lanes 8u..8u+7 end with the total of v_u.
__device__ __forceinline__ float warp_reduce4(float v0, float v1, float v2, float v3, int lane) {
    const bool h16 = (lane & 16) != 0;
    float k0 = h16 ? v2 : v0, k1 = h16 ? v3 : v1;
    const float s0 = h16 ? v0 : v2, s1 = h16 ? v1 : v3;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    const bool h8 = (lane & 8) != 0;
    float kk = h8 ? k1 : k0;
    const float ss = h8 ? k0 : k1;
    kk += __shfl_xor_sync(0xffffffffu, ss, 8);
    kk += __shfl_xor_sync(0xffffffffu, kk, 4);
    kk += __shfl_xor_sync(0xffffffffu, kk, 2);
    kk += __shfl_xor_sync(0xffffffffu, kk, 1);
    return kk;
}

// ---------------------------------------------------------------------------
// MUFU approximations, flush-to-zero forms (the kernels' arguments are normal
// numbers: r^2 >= eps^2 or the squared distance of distinct points, and the
// phase k r); the non-FTZ forms add denormal handling around each MUFU op
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// named barrier over `threads` threads (id 1..15; id 0 is __syncthreads)
__device__ __forceinline__ void named_bar_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// ---------------------------------------------------------------------------
// mbarrier + 1-D bulk async copy (global -> shared)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// make mbarrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bytes must be a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Warp-uniform bounded wait on an mbarrier phase: gives up after limit_ns of
// global time (checked every 64 polls).  Returns false if the limit expired
// (the caller records P2P_FLAG_TIMEOUT).
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        const bool done = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        if ((it & 63u) == 0) {
            const bool late = (global_ns() - t0) > limit_ns;
            if (__any_sync(0xffffffffu, late)) return false;
        }
    }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream drains.
// pdl_wait() blocks until the predecessor grid has completed and its memory
// is visible (a no-op for an ordinary launch), so every kernel calls it before
// touching memory; pdl_release() lets the successor be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace p2p
