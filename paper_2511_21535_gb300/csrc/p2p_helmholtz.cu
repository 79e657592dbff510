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
#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {

template <int K, int R, bool COMP, bool PRECISE>
struct HelmOp {
    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float kk;
    int words;          // record stride in 16-byte words
    int qw0;            // first q word of this pass inside a record
    int64_t n;
    int r0;             // first right-hand side of this pass
    float2* __restrict__ u;

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
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
            if (l < nt) r = rec[(int64_t)(tb + l) * words];
            tx[k] = r.x;
            ty[k] = r.y;
            tz[k] = r.z;
            self[k] = (l < nt) ? sw_lo + l : -1;
#pragma unroll
            for (int q = 0; q < R; ++q) sr[k][q] = si[k][q] = cr[k][q] = ci[k][q] = pr[k][q] = pi_[k][q] = 0.f;
        }
    }

    template <bool CHECK>
    __device__ __forceinline__ void body(const float4* __restrict__ sm, int cnt, int rec0) {
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const float4* rj = sm + j * words;
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
                const float inv = rsqrtf(r2);
                const float th = kk * (r2 * inv);
                float sn, cs;
                if (PRECISE) sincosf(th, &sn, &cs);
                else __sincosf(th, &sn, &cs);
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

    __device__ __forceinline__ void end(int lane) {
        const float inv4pi = 0.0795774715459476678844418816862571882f;  // 1 / (4 pi)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt) {
                const int64_t o = perm[tbase + l];
#pragma unroll
                for (int q = 0; q < R; ++q)
                    u[(int64_t)(r0 + q) * n + o] =
                        make_float2((sr[k][q] - cr[k][q]) * inv4pi, (si[k][q] - ci[k][q]) * inv4pi);
            }
        }
    }
};

template <int K, int R, bool COMP, bool PRECISE>
__global__ void __launch_bounds__(kLoopThreads, 4)
    k_helmholtz(LoopArgs a, const int32_t* __restrict__ perm, float kk, int qw0, int64_t n, int r0,
                float2* __restrict__ u) {
    HelmOp<K, R, COMP, PRECISE> op;
    op.rec = a.rec;
    op.perm = perm;
    op.kk = kk;
    op.words = a.words;
    op.qw0 = qw0;
    op.n = n;
    op.r0 = r0;
    op.u = u;
    warp_item_loop<K>(a, op);
}

template <int K, int R, bool COMP, bool PRECISE>
static int launch_helm(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, float2* u,
                       cudaStream_t s) {
    auto kern = k_helmholtz<K, R, COMP, PRECISE>;
    const size_t smem = loop_smem_bytes(a.tile, a.words);
    P2P_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0) {
        P2P_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
        if (per_sm < 1) per_sm = 1;
    }
    const int qw0 = 1 + r0 / 2;
    kern<<<num_sms() * per_sm, kLoopThreads, smem, s>>>(a, perm, kk, qw0, p->n, r0, u);
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

template <int K, int R>
static int launch_helm_kr(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, float2* u,
                          bool comp, bool precise, cudaStream_t s) {
    if (precise) return comp ? launch_helm<K, R, true, true>(p, a, perm, kk, r0, u, s)
                             : launch_helm<K, R, false, true>(p, a, perm, kk, r0, u, s);
    return comp ? launch_helm<K, R, true, false>(p, a, perm, kk, r0, u, s)
                : launch_helm<K, R, false, false>(p, a, perm, kk, r0, u, s);
}

template <int K>
static int launch_helm_k(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, float2* u,
                         bool comp, bool precise, cudaStream_t s) {
    switch (R) {
        case 1: return launch_helm_kr<K, 1>(p, a, perm, kk, r0, u, comp, precise, s);
        case 2: return launch_helm_kr<K, 2>(p, a, perm, kk, r0, u, comp, precise, s);
        case 4: return launch_helm_kr<K, 4>(p, a, perm, kk, r0, u, comp, precise, s);
        case 8: return launch_helm_kr<K, 8>(p, a, perm, kk, r0, u, comp, precise, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

// Largest k * r over any pair of neighbouring boxes below which the hardware
// sine/cosine approximation is used (its argument reduction keeps the
// absolute error near 1e-6 over this range; the parity tests measure it).
constexpr float kFastPhaseMax = 32.0f;

int launch_helmholtz_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float k, float2* u,
                            cudaStream_t s) {
    const bool comp = !(p->flags & P2P_PLAN_PLAIN_FP32);
    const float box = p->edge / (float)(1 << p->level);
    const float rmax = 2.0f * box * 1.7320508f;
    const bool precise = fabsf(k) * rmax > kFastPhaseMax;
    // passes of 8, 4, 2, 1 right-hand sides; every pass but the last starts at an even index
    int r0 = 0;
    while (r0 < p->nrhs) {
        const int left = p->nrhs - r0;
        const int R = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        P2P_CUDA_TRY(cudaMemsetAsync(&a.hdr->work_ctr, 0, sizeof(uint32_t), s));
        int st = (p->tpl == 2) ? launch_helm_k<2>(p, a, perm, k, r0, R, u, comp, precise, s)
                               : launch_helm_k<1>(p, a, perm, k, r0, R, u, comp, precise, s);
        if (st) return st;
        r0 += R;
    }
    return P2P_OK;
}

}  // namespace p2p
