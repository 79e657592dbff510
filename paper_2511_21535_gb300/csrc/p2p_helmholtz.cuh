// Helmholtz P2P kernel (Green's function of the Helmholtz equation,
// Section 5.1, taken in 3-D):
//   u_i^(r) = sum_{j in near(i), j != i} q_j^(r) exp(i k r_ij) / (4 pi r_ij)
// The 1/(4 pi) factor is applied once per output.  Per pair: 3 FADD, 3
// FMUL/FFMA for r^2, MUFU rsqrt, r = r^2 * rsqrt, k r, sine and cosine
// (MUFU), 2 FMUL for G, then 4 FFMA per right-hand side.  With one RHS the
// three MUFU operations bind; with 8 RHS the FP32 pipe does.
//
// Several right-hand sides are processed in passes of R in {1, 2, 4, 8}
// values sharing one evaluation of G per pair.
#pragma once

#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {

// W: record stride in 16-byte words when known at compile time (0 = runtime)
template <int K, int R, bool COMP, bool PRECISE, int W = 0>
struct HelmOp {
    static constexpr int kOuts = 2 * R * K;
    static constexpr bool kPartial = true;    // can write pair-task partial results
    static constexpr int kMutFloats = 0;      // one-sided (symmetric plans use HelmSymOp)

    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float kk;
    int words;          // record stride in 16-byte words
    int qw0;            // first q word of this pass inside a record
    int64_t n;
    int r0;             // first right-hand side of this pass
    HelmOut out;

    float tx[K], ty[K], tz[K];
    int self[K];
    float sr[K][R], si[K][R], cr[K][R], ci[K][R], pr[K][R], pi_[K][R];
    int tbase, nt;

    __device__ __forceinline__ void begin(int tb, int ntg, int sw_lo, int lane) {
        tbase = tb;
        nt = ntg;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            // idle lanes sit on the first target: finite distances to every other particle
            const float4 r = rec[(int64_t)(tb + (l < nt ? l : 0)) * words];
            tx[k] = r.x;
            ty[k] = r.y;
            tz[k] = r.z;
            self[k] = (l < nt) ? sw_lo + l : -1;
#pragma unroll
            for (int q = 0; q < R; ++q) sr[k][q] = si[k][q] = cr[k][q] = ci[k][q] = pr[k][q] = pi_[k][q] = 0.f;
        }
    }

    // periodic image of the current neighbour range: targets move by -shift
    __device__ __forceinline__ void set_shift(float sx, float sy, float sz) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            const float4 r = rec[(int64_t)(tbase + (l < nt ? l : 0)) * words];
            tx[k] = r.x - sx;
            ty[k] = r.y - sy;
            tz[k] = r.z - sz;
        }
    }

    template <bool CHECK>
    __device__ __forceinline__ void body(const float4* __restrict__ sm, int cnt, int rec0) {
        const int stride = W ? W : words;
        const float4* rj = sm;
#pragma unroll 4
        for (int j = 0; j < cnt; ++j, rj += stride) {
            const float4 ps = rj[0];
            float qr[R], qi[R];
#pragma unroll
            for (int w = 0; w < (R + 1) / 2; ++w) {
                const float4 v = rj[qw0 + w];
                qr[2 * w] = v.x;
                qi[2 * w] = v.y;
                if (2 * w + 1 < R) {
                    qr[2 * w + 1] = v.z;
                    qi[2 * w + 1] = v.w;
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float dx = ps.x - tx[k];
                const float dy = ps.y - ty[k];
                const float dz = ps.z - tz[k];
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                bool me = false;
                if (CHECK) {
                    me = (rec0 + j) == self[k];
                    r2 = me ? 1.f : r2;
                }
                const float inv = rsqrt_approx(r2);
                const float th = kk * (r2 * inv);
                float sn, cs;
                if (PRECISE) {
                    sincosf(th, &sn, &cs);
                } else {
                    sn = sin_approx(th);
                    cs = cos_approx(th);
                }
                float gr = inv * cs, gi = inv * sn;
                if (CHECK) {
                    gr = me ? 0.f : gr;
                    gi = me ? 0.f : gi;
                }
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    float& ar = COMP ? pr[k][q] : sr[k][q];
                    float& ai = COMP ? pi_[k][q] : si[k][q];
                    ar = fmaf(gr, qr[q], fmaf(-gi, qi[q], ar));
                    ai = fmaf(gr, qi[q], fmaf(gi, qr[q], ai));
                }
            }
        }
    }

    __device__ __forceinline__ void tile(const float4* sm, int cnt, int rec0, bool chk) {
        if (chk) body<true>(sm, cnt, rec0);
        else body<false>(sm, cnt, rec0);
        if (COMP) {
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    kahan_add(sr[k][q], cr[k][q], pr[k][q]);
                    kahan_add(si[k][q], ci[k][q], pi_[k][q]);
                    pr[k][q] = 0.f;
                    pi_[k][q] = 0.f;
                }
        }
    }

    __device__ __forceinline__ void store_partial(float* dst, int lane) const {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                dst[((k * R + q) * 2 + 0) * 32 + lane] = sr[k][q] - cr[k][q];
                dst[((k * R + q) * 2 + 1) * 32 + lane] = si[k][q] - ci[k][q];
            }
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                sr[k][q] -= cr[k][q];
                si[k][q] -= ci[k][q];
                cr[k][q] = ci[k][q] = 0.f;
            }
    }
    __device__ __forceinline__ void add_partial(const float* src, int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                sr[k][q] += src[((k * R + q) * 2 + 0) * 32 + lane];
                si[k][q] += src[((k * R + q) * 2 + 1) * 32 + lane];
            }
    }

    // pair task: this task's contribution, scaled, to slot `slot` of each RHS row
    __device__ __forceinline__ void end_partial(int lane, void* part, int64_t cap, int64_t slot) {
        const float inv4pi = 0.0795774715459476678844418816862571882f;  // 1 / (4 pi)
        float2* o = static_cast<float2*>(part) + slot;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt) {
#pragma unroll
                for (int q = 0; q < R; ++q)
                    o[(int64_t)(r0 + q) * cap + l] =
                        make_float2((sr[k][q] - cr[k][q]) * inv4pi, (si[k][q] - ci[k][q]) * inv4pi);
            }
        }
    }

    __device__ __forceinline__ void end(int lane) {
        const float inv4pi = 0.0795774715459476678844418816862571882f;  // 1 / (4 pi)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt) {
                const int64_t o = perm[tbase + l];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float re = (sr[k][q] - cr[k][q]) * inv4pi, im = (si[k][q] - ci[k][q]) * inv4pi;
                    const int r = r0 + q;
                    if (r < out.split) out.u[(int64_t)r * n + o] = make_float2(re, im);
                    else out.u2[(int64_t)(r - out.split) * n + o] = make_float2(re, -im);
                }
            }
        }
    }
};

// register bound by the accumulators' size: four or eight right-hand sides
// per pass with two targets per lane need 123 / 168 registers (no spills)
template <int K, int G, int R, bool COMP, bool PRECISE, int W = 0>
__global__ void __launch_bounds__(kLoopThreads, R >= 8 ? (K >= 2 ? 3 : 4) : R == 4 ? (K >= 2 ? 4 : 5) : 6)
    k_helmholtz(LoopArgs a, const int32_t* __restrict__ perm, float kk, int qw0, int64_t n, int r0, HelmOut out) {
    pdl_wait();
    HelmOp<K, R, COMP, PRECISE, W> op;
    op.rec = a.rec;
    op.perm = perm;
    op.kk = kk;
    op.words = a.words;
    op.qw0 = qw0;
    op.n = n;
    op.r0 = r0;
    op.out = out;
    warp_item_loop<K, G>(a, op);
}

template <int K, int G, int R, bool COMP, bool PRECISE, int W = 0>
int launch_helm(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, HelmOut u, cudaStream_t s) {
    auto kern = k_helmholtz<K, G, R, COMP, PRECISE, W>;
    using Op = HelmOp<K, R, COMP, PRECISE, W>;
    const size_t smem = loop_smem_bytes(a.tile, a.words, Op::kOuts, G, Op::kMutFloats);
    P2P_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0) {
        P2P_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
        if (per_sm < 1) per_sm = 1;
    }
    const int qw0 = 1 + r0 / 2;
    P2P_CUDA_TRY(launch_pdl(kern, num_sms() * per_sm, kLoopThreads, smem, s, a, perm, kk, qw0, p->n, r0, u));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

// per-variant dispatchers (each in its own translation unit)
int launch_helm_fast(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                     cudaStream_t s);
int launch_helm_plain(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                      cudaStream_t s);
int launch_helm_precise(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                        cudaStream_t s);
// records with the right-hand sides planar per word (plans of four or more): passes of 2, 4 or 8 values,
// nval of them valid
int launch_helm_planar(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, int nval,
                       bool comp, bool precise, HelmOut u, cudaStream_t s);

}  // namespace p2p
