// Double-precision reductions on the device for the operator's check
// quantities: the momentum invariant of the gravity near field (sum_i m_i a_i
// is zero in exact arithmetic, because the neighbour relation is symmetric
// and the softened kernel's gradient is odd) and the inner products of the
// adjoint identity Re<P x, y> = Re<x, P^H y>.  The operator itself computes
// in FP32; only these global sums accumulate in FP64.
//
// One block of 1024 threads reads the whole array (a check, not a hot path):
// each thread accumulates in double, then the block adds the threads' sums
// in a fixed order, so the result is deterministic.
#include "common.cuh"
#include "device.cuh"
#include "nvtx_range.cuh"

namespace p2p {

constexpr int kCheckThreads = 1024;

// fixed-order block sum of one double per thread (all threads get the total)
__device__ __forceinline__ double block_sum_f64(double v) {
    __shared__ double part[kCheckThreads / 32];
    __shared__ double total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kCheckThreads / 32; ++w) t += part[w];
        total = t;
    }
    __syncthreads();
    const double t = total;
    __syncthreads();   // the shared slots may be reused by the next call
    return t;
}

__global__ void __launch_bounds__(kCheckThreads) k_momentum_f64(const float* __restrict__ mass,
                                                               const float* __restrict__ acc, int64_t n,
                                                               double* __restrict__ out) {
    pdl_wait();
    pdl_release();
    double s[3] = {0.0, 0.0, 0.0}, a[3] = {0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < n; i += kCheckThreads) {
        const double m = (double)mass[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double f = m * (double)acc[3 * i + c];
            s[c] += f;
            a[c] += fabs(f);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double ts = block_sum_f64(s[c]);
        const double ta = block_sum_f64(a[c]);
        if (threadIdx.x == 0) {
            out[c] = ts;
            out[3 + c] = ta;
        }
    }
}

__global__ void __launch_bounds__(kCheckThreads) k_dot_f64(const float* __restrict__ x, const float* __restrict__ y,
                                                          int64_t count, double* __restrict__ out) {
    pdl_wait();
    pdl_release();
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += kCheckThreads) s += (double)x[i] * (double)y[i];
    const double t = block_sum_f64(s);
    if (threadIdx.x == 0) out[0] = t;
}

}  // namespace p2p

using namespace p2p;

extern "C" int p2p_momentum_fp64(const float* mass, const float* acc, int64_t n, double* out, void* stream) {
    NvtxRange nvtx_range("p2p_momentum_fp64");
    if (!mass || !acc || !out || n < 0 ||
        ((reinterpret_cast<uintptr_t>(mass) | reinterpret_cast<uintptr_t>(acc)) & 3u) ||
        (reinterpret_cast<uintptr_t>(out) & 7u))
        return P2P_ERR_INVALID_ARG;
    P2P_CUDA_TRY(launch_pdl(k_momentum_f64, 1, kCheckThreads, 0, static_cast<cudaStream_t>(stream), mass, acc, n, out));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

extern "C" int p2p_dot_fp64(const float* x, const float* y, int64_t count, double* out, void* stream) {
    NvtxRange nvtx_range("p2p_dot_fp64");
    if (!x || !y || !out || count < 0 || ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 3u) ||
        (reinterpret_cast<uintptr_t>(out) & 7u))
        return P2P_ERR_INVALID_ARG;
    P2P_CUDA_TRY(launch_pdl(k_dot_f64, 1, kCheckThreads, 0, static_cast<cudaStream_t>(stream), x, y, count, out));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}
