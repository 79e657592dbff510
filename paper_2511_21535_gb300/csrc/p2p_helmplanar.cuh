// Helmholtz P2P for plans of four or more right-hand sides (the Green's
// function of Section 5.1, 3-D):
//   u_i^(r) = sum_{j in near(i), j != i} q_j^(r) exp(i k r_ij) / (4 pi r_ij)
//
// With many right-hand sides the complex products dominate: after G is
// evaluated once per pair (3 FADD, 3 for r^2, MUFU rsqrt, r, k r, MUFU sine
// and cosine, 2 FMUL), each right-hand side costs 4 FMAs.  The records of
// these plans hold the right-hand sides planar per 16-byte word,
//   word 1 + w = [Re q_a, Re q_b, Im q_a, Im q_b],  (a, b) = (2w, 2w + 1),
// so that each half of the word is a (right-hand side a, right-hand side b)
// pair in two adjacent registers, and one packed two-wide FMA
// (fma.rn.f32x2) does one step of both right-hand sides:
//   (ar_a, ar_b) += (g_r, g_r)(Re q_a, Re q_b) + (-g_i, -g_i)(Im q_a, Im q_b)
//   (ai_a, ai_b) += (g_r, g_r)(Im q_a, Im q_b) + ( g_i,  g_i)(Re q_a, Re q_b)
// which halves the issue slots of the products (2 packed FMAs per right-hand
// side) and needs no register moves for the sources' values.  Each half is
// rounded exactly as the scalar kernel's FMA in the same order, so every
// right-hand side gives the same bits as a plan of one right-hand side.
//
// Passes of R in {2, 4, 8} right-hand sides (R / 2 words); the last pass of
// an odd count reads one word whose second half is zero and writes only the
// valid right-hand sides.
#pragma once

#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {

template <int K, int R, bool COMP, bool PRECISE>
struct HelmPlanarOp {
    static_assert(R == 2 || R == 4 || R == 8, "planar passes hold pairs of right-hand sides");
    static constexpr int RP = R / 2;               // right-hand-side pairs (words) per pass
    static constexpr int kOuts = 2 * R * K;        // floats per lane exchanged between cooperating warps
    static constexpr bool kPartial = true;         // can write pair-task partial results
    static constexpr int kMutFloats = 0;           // one-sided

    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float kk;
    int words;          // record stride in 16-byte words
    int qw0;            // first q word of this pass inside a record
    int64_t n;
    int r0;             // first right-hand side of this pass
    int nval;           // right-hand sides of this pass that exist (R, or R - 1 for the last of an odd count)
    HelmOut out;

    float tx[K], ty[K], tz[K];
    int self[K];
    float2 pr[K][RP], pi_[K][RP];                  // the current tile's partial sums (compensated mode)
    float2 sr[K][RP], si[K][RP], cr[K][RP], ci[K][RP];
    int tbase, nt;

    __device__ __forceinline__ void begin(int tb, int ntg, int sw_lo, int lane) {
        tbase = tb;
        nt = ntg;
        const float2 z = make_float2(0.f, 0.f);
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
            for (int w = 0; w < RP; ++w) sr[k][w] = si[k][w] = cr[k][w] = ci[k][w] = pr[k][w] = pi_[k][w] = z;
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
        const float4* rj = sm;
#pragma unroll 8
        for (int j = 0; j < cnt; ++j, rj += words) {
            const float4 ps = rj[0];
            float2 qr[RP], qi[RP];
#pragma unroll
            for (int w = 0; w < RP; ++w) {
                const float4 v = rj[qw0 + w];
                qr[w] = make_float2(v.x, v.y);
                qi[w] = make_float2(v.z, v.w);
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
                const float2 g_r = make_float2(gr, gr), g_i = make_float2(gi, gi), g_n = make_float2(-gi, -gi);
#pragma unroll
                for (int w = 0; w < RP; ++w) {
                    float2& ar = COMP ? pr[k][w] : sr[k][w];
                    float2& ai = COMP ? pi_[k][w] : si[k][w];
                    ar = __ffma2_rn(g_r, qr[w], __ffma2_rn(g_n, qi[w], ar));
                    ai = __ffma2_rn(g_r, qi[w], __ffma2_rn(g_i, qr[w], ai));
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
                for (int w = 0; w < RP; ++w) {
                    kahan_add(sr[k][w].x, cr[k][w].x, pr[k][w].x);
                    kahan_add(sr[k][w].y, cr[k][w].y, pr[k][w].y);
                    kahan_add(si[k][w].x, ci[k][w].x, pi_[k][w].x);
                    kahan_add(si[k][w].y, ci[k][w].y, pi_[k][w].y);
                    pr[k][w] = make_float2(0.f, 0.f);
                    pi_[k][w] = make_float2(0.f, 0.f);
                }
        }
    }

    // value h (0: right-hand side 2w, 1: 2w + 1) of a packed pair
    static __device__ __forceinline__ float half(const float2& v, int h) { return h ? v.y : v.x; }

    __device__ __forceinline__ void store_partial(float* dst, int lane) const {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int w = 0; w < RP; ++w)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = 2 * w + h;
                    dst[((k * R + q) * 2 + 0) * 32 + lane] = half(sr[k][w], h) - half(cr[k][w], h);
                    dst[((k * R + q) * 2 + 1) * 32 + lane] = half(si[k][w], h) - half(ci[k][w], h);
                }
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int w = 0; w < RP; ++w) {
                sr[k][w].x -= cr[k][w].x;
                sr[k][w].y -= cr[k][w].y;
                si[k][w].x -= ci[k][w].x;
                si[k][w].y -= ci[k][w].y;
                cr[k][w] = ci[k][w] = make_float2(0.f, 0.f);
            }
    }
    __device__ __forceinline__ void add_partial(const float* src, int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int w = 0; w < RP; ++w) {
                sr[k][w].x += src[((k * R + 2 * w) * 2 + 0) * 32 + lane];
                si[k][w].x += src[((k * R + 2 * w) * 2 + 1) * 32 + lane];
                sr[k][w].y += src[((k * R + 2 * w + 1) * 2 + 0) * 32 + lane];
                si[k][w].y += src[((k * R + 2 * w + 1) * 2 + 1) * 32 + lane];
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
                for (int w = 0; w < RP; ++w)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q = 2 * w + h;
                        if (q < nval)
                            o[(int64_t)(r0 + q) * cap + l] =
                                make_float2((half(sr[k][w], h) - half(cr[k][w], h)) * inv4pi,
                                            (half(si[k][w], h) - half(ci[k][w], h)) * inv4pi);
                    }
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
                for (int w = 0; w < RP; ++w)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q = 2 * w + h;
                        if (q >= nval) continue;
                        const float re = (half(sr[k][w], h) - half(cr[k][w], h)) * inv4pi;
                        const float im = (half(si[k][w], h) - half(ci[k][w], h)) * inv4pi;
                        const int r = r0 + q;
                        if (r < out.split) out.u[(int64_t)r * n + o] = make_float2(re, im);
                        else out.u2[(int64_t)(r - out.split) * n + o] = make_float2(re, -im);
                    }
            }
        }
    }
};

// register bound by the accumulators' size (as the interleaved-record kernel)
template <int K, int G, int R, bool COMP, bool PRECISE>
__global__ void __launch_bounds__(kLoopThreads, R >= 8 ? (K >= 2 ? 3 : 4) : R == 4 ? (K >= 2 ? 4 : 5) : 6)
    k_helmplanar(LoopArgs a, const int32_t* __restrict__ perm, float kk, int qw0, int64_t n, int r0, int nval,
                 HelmOut out) {
    pdl_wait();
    HelmPlanarOp<K, R, COMP, PRECISE> op;
    op.rec = a.rec;
    op.perm = perm;
    op.kk = kk;
    op.words = a.words;
    op.qw0 = qw0;
    op.n = n;
    op.r0 = r0;
    op.nval = nval;
    op.out = out;
    warp_item_loop<K, G>(a, op);
}

template <int K, int G, int R, bool COMP, bool PRECISE>
int launch_helmplanar(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int nval, HelmOut u,
                      cudaStream_t s) {
    auto kern = k_helmplanar<K, G, R, COMP, PRECISE>;
    using Op = HelmPlanarOp<K, R, COMP, PRECISE>;
    const size_t smem = loop_smem_bytes(a.tile, a.words, Op::kOuts, G, Op::kMutFloats);
    P2P_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0) {
        P2P_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
        if (per_sm < 1) per_sm = 1;
    }
    const int qw0 = 1 + r0 / 2;
    P2P_CUDA_TRY(launch_pdl(kern, num_sms() * per_sm, kLoopThreads, smem, s, a, perm, kk, qw0, p->n, r0, nval, u));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

}  // namespace p2p
