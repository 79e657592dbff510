// Pipe-throughput microbenchmark: the peaks the P2P kernels are measured
// against.  One CTA of 1024 threads per SM runs independent dependency
// chains of one instruction kind; the CTA's own clock64() span gives
// lane-operations per SM per clock, independent of the clock frequency, and
// the CUDA-event time of the launch gives the SM clock during the run.
#include "common.cuh"
#include "device.cuh"

namespace p2p {

constexpr int kMbThreads = 1024;
constexpr int kMbChains = 8;

__global__ void __launch_bounds__(kMbThreads) k_mb_ffma(float b, float c, int iters, float* sink,
                                                        long long* cycles) {
    float a[kMbChains];
#pragma unroll
    for (int i = 0; i < kMbChains; ++i) a[i] = threadIdx.x * 1e-3f + i;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kMbChains; ++i) a[i] = fmaf(a[i], b, c);
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kMbChains; ++i) s += a[i];
    if (s == 12345.f) sink[threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// packed two-wide FFMA (fma.rn.f32x2): each instruction does two lane-operations
__global__ void __launch_bounds__(kMbThreads) k_mb_ffma2(float b, float c, int iters, float* sink,
                                                         long long* cycles) {
    float2 a[kMbChains];
#pragma unroll
    for (int i = 0; i < kMbChains; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, threadIdx.x * 2e-3f - i);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kMbChains; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kMbChains; ++i) s += a[i].x + a[i].y;
    if (s == 12345.f) sink[threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
__global__ void __launch_bounds__(kMbThreads) k_mb_mufu(int iters, float* sink, long long* cycles) {
    float a[kMbChains];
#pragma unroll
    for (int i = 0; i < kMbChains; ++i) a[i] = 0.5f + threadIdx.x * 1e-4f + i * 0.01f;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kMbChains; ++i) {
            if (OP == 0) asm volatile("rsqrt.approx.f32 %0, %0;" : "+f"(a[i]));
            else asm volatile("sin.approx.f32 %0, %0;" : "+f"(a[i]));
        }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kMbChains; ++i) s += a[i];
    if (s == 12345.f) sink[threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// One warp initialises an mbarrier that expects one arrival and never gets
// it, then waits on it with a limit of limit_ns: the wait must run out and
// the kernel must record P2P_FLAG_TIMEOUT and return.  No copy is in flight.
__global__ void k_selftest_wait(uint64_t limit_ns, uint32_t* flags) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (!warp_wait(&bar, 0, limit_ns)) {
        if (threadIdx.x == 0) atomicOr(flags, P2P_FLAG_TIMEOUT);
    }
}

}  // namespace p2p

using namespace p2p;

extern "C" int p2p_selftest_bounded_wait(uint64_t limit_ns, uint32_t* flags_dev, void* stream) {
    if (!flags_dev || limit_ns == 0 || limit_ns > 10000000000ull) return P2P_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    P2P_CUDA_TRY(cudaMemsetAsync(flags_dev, 0, sizeof(uint32_t), s));
    k_selftest_wait<<<1, 32, 0, s>>>(limit_ns, flags_dev);
    P2P_LAUNCH_CHECK();
    uint32_t h = 0;
    P2P_CUDA_TRY(cudaMemcpyAsync(&h, flags_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    P2P_CUDA_TRY(cudaStreamSynchronize(s));
    return (h & P2P_FLAG_TIMEOUT) ? P2P_ERR_TIMEOUT : P2P_OK;
}

extern "C" int p2p_measure_pipes(double* out, void* stream) {
    if (!out) return P2P_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = num_sms();
    // scratch: per-CTA cycle counts and a sink (allocated here: a measurement
    // utility, not part of the operator path)
    long long* cyc = nullptr;
    float* sink = nullptr;
    if (cudaMalloc(&cyc, sizeof(long long) * sms) != cudaSuccess) return P2P_ERR_CUDA;
    if (cudaMalloc(&sink, sizeof(float) * kMbThreads) != cudaSuccess) {
        cudaFree(cyc);
        return P2P_ERR_CUDA;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = P2P_OK;
    long long* host = new long long[sms];
    for (int which = 0; which < 4 && rc == P2P_OK; ++which) {
        const int iters = (which == 0 || which == 3) ? 40000 : 4000;
        double best = 0.0, mhz = 0.0;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, s);
            if (which == 0) k_mb_ffma<<<sms, kMbThreads, 0, s>>>(1.0000001f, 1e-7f, iters, sink, cyc);
            else if (which == 1) k_mb_mufu<0><<<sms, kMbThreads, 0, s>>>(iters, sink, cyc);
            else if (which == 2) k_mb_mufu<1><<<sms, kMbThreads, 0, s>>>(iters, sink, cyc);
            else k_mb_ffma2<<<sms, kMbThreads, 0, s>>>(1.0000001f, 1e-7f, iters, sink, cyc);
            count_launch();
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = P2P_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaMemcpy(host, cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
            long long mx = 0;
            double mean = 0.0;
            for (int b = 0; b < sms; ++b) {
                mx = host[b] > mx ? host[b] : mx;
                mean += (double)host[b] / sms;
            }
            const double ops = (double)kMbThreads * kMbChains * iters * (which == 3 ? 2 : 1);
            const double rate = ops / mean;           // lane-ops per SM per clock
            if (rate > best) {
                best = rate;
                mhz = ms > 0.f ? (double)mx / (ms * 1e3) : 0.0;
            }
        }
        out[which == 3 ? 4 : which] = best;
        if (which == 0) out[3] = mhz;
    }
    delete[] host;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(cyc);
    cudaFree(sink);
    return rc;
}
