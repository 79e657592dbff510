// One-sided Helmholtz P2P kernel with the pairs of a tile laid out over the
// warp in two dimensions (the Green's function of Section 5.1, 3-D):
//   u_i^(r) = sum_{j in near(i), j != i} q_j^(r) exp(i k r_ij) / (4 pi r_ij)
//
// The item's 64 targets are spread as four per lane over 16 target groups,
// and the tile's sources over two source groups: lane = 2 tg + sg holds
// targets 4 tg .. 4 tg + 3 and takes sources j = sg, sg + 2, ...  Each source
// record read from shared memory then serves four evaluations instead of two,
// which halves the shared-memory loads per pair; those loads and the three
// MUFU operations per pair (rsqrt, sine, cosine) share one issue queue, so
// fewer loads leave more of it to the MUFU pipe.  At the end of an item the
// two source groups' sums of each target are added across the lane pair.
//
// Arithmetic on target pairs: a lane's four targets form two pairs, and the
// per-pair FP32 work (differences, r^2, k r, G, the complex products) runs
// as packed two-wide instructions (add/mul/fma .f32x2, sm_100 and later), so
// one issue slot does the work of two; only the MUFU operations stay scalar.
// Each packed operation rounds each half exactly as the scalar one would.
//
// Summation: per lane, a tile's partial (up to tile / 2 sources) is added to
// the running sum with a compensated (Kahan) step.
#pragma once

#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {

template <int R, int W>
struct HelmTileOp {
    static constexpr int KT = 4;                  // targets per lane
    static constexpr int SP = 2;                  // source groups (64 targets per warp)
    static constexpr int kOuts = 2 * R * KT;      // floats per lane exchanged between cooperating warps
    static constexpr bool kPartial = true;        // can write pair-task partial results
    static constexpr int kMutFloats = 0;          // one-sided

    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float kk;
    int qw0;
    int64_t n;
    int r0;
    HelmOut out;

    static constexpr int KP = KT / 2;             // target pairs per lane
    float2 ntx[KP], nty[KP], ntz[KP];             // negated target coordinates, packed in pairs
    float2 pr[KP][R], pi_[KP][R];                 // the current tile's partial sums, packed
    float sr[KT][R], si[KT][R], cr[KT][R], ci[KT][R];
    int tbase, nt, self0;

    __device__ __forceinline__ void load_positions(int lane, float sx, float sy, float sz) {
        const int t0 = (lane / SP) * KT;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int t = t0 + k;
            // idle targets sit on the first target: finite distances to every other particle
            const float4 r = rec[(int64_t)(tbase + (t < nt ? t : 0)) * W];
            const float x = sx - r.x, y = sy - r.y, z = sz - r.z;
            if (k & 1) {
                ntx[k / 2].y = x;
                nty[k / 2].y = y;
                ntz[k / 2].y = z;
            } else {
                ntx[k / 2].x = x;
                nty[k / 2].x = y;
                ntz[k / 2].x = z;
            }
        }
    }

    __device__ __forceinline__ void begin(int tb, int ntg, int sw_lo, int lane) {
        tbase = tb;
        nt = ntg;
        self0 = sw_lo;
        load_positions(lane, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) sr[k][q] = si[k][q] = cr[k][q] = ci[k][q] = 0.f;
#pragma unroll
        for (int h = 0; h < KP; ++h)
#pragma unroll
            for (int q = 0; q < R; ++q) pr[h][q] = pi_[h][q] = make_float2(0.f, 0.f);
    }

    // periodic image of the current neighbour range: targets move by -shift
    __device__ __forceinline__ void set_shift(float sx, float sy, float sz) {
        load_positions(threadIdx.x & 31, sx, sy, sz);
    }

    template <bool CHECK>
    __device__ __forceinline__ void body(const float4* __restrict__ sm, int cnt, int rec0) {
        const int lane = threadIdx.x & 31, sg = lane % SP, t0 = (lane / SP) * KT;
        const float2 kk2 = make_float2(kk, kk);
        const float4* rj = sm + (int64_t)sg * W;
#pragma unroll 8
        for (int j = sg; j < cnt; j += SP, rj += SP * W) {
            const float4 ps = rj[0];
            const float2 sx = make_float2(ps.x, ps.x), sy = make_float2(ps.y, ps.y), sz = make_float2(ps.z, ps.z);
            float2 qr[R], qi[R], nqi[R];
#pragma unroll
            for (int w = 0; w < (R + 1) / 2; ++w) {
                const float4 v = rj[qw0 + w];
                qr[2 * w] = make_float2(v.x, v.x);
                qi[2 * w] = make_float2(v.y, v.y);
                nqi[2 * w] = make_float2(-v.y, -v.y);
                if (2 * w + 1 < R) {
                    qr[2 * w + 1] = make_float2(v.z, v.z);
                    qi[2 * w + 1] = make_float2(v.w, v.w);
                    nqi[2 * w + 1] = make_float2(-v.w, -v.w);
                }
            }
#pragma unroll
            for (int h = 0; h < KP; ++h) {
                const float2 dx = __fadd2_rn(sx, ntx[h]), dy = __fadd2_rn(sy, nty[h]), dz = __fadd2_rn(sz, ntz[h]);
                float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                bool me0 = false, me1 = false;
                if (CHECK) {
                    const int t = t0 + 2 * h;
                    me0 = (rec0 + j) == self0 + t && t < nt;
                    me1 = (rec0 + j) == self0 + t + 1 && t + 1 < nt;
                    r2.x = me0 ? 1.f : r2.x;
                    r2.y = me1 ? 1.f : r2.y;
                }
                const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                const float2 th = __fmul2_rn(kk2, __fmul2_rn(r2, inv));
                float2 gr = __fmul2_rn(inv, make_float2(cos_approx(th.x), cos_approx(th.y)));
                float2 gi = __fmul2_rn(inv, make_float2(sin_approx(th.x), sin_approx(th.y)));
                if (CHECK) {
                    gr.x = me0 ? 0.f : gr.x;
                    gi.x = me0 ? 0.f : gi.x;
                    gr.y = me1 ? 0.f : gr.y;
                    gi.y = me1 ? 0.f : gi.y;
                }
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    pr[h][q] = __ffma2_rn(gr, qr[q], __ffma2_rn(gi, nqi[q], pr[h][q]));
                    pi_[h][q] = __ffma2_rn(gr, qi[q], __ffma2_rn(gi, qr[q], pi_[h][q]));
                }
            }
        }
    }

    __device__ __forceinline__ void tile(const float4* sm, int cnt, int rec0, bool chk) {
        if (chk) body<true>(sm, cnt, rec0);
        else body<false>(sm, cnt, rec0);
#pragma unroll
        for (int h = 0; h < KP; ++h)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                kahan_add(sr[2 * h][q], cr[2 * h][q], pr[h][q].x);
                kahan_add(si[2 * h][q], ci[2 * h][q], pi_[h][q].x);
                kahan_add(sr[2 * h + 1][q], cr[2 * h + 1][q], pr[h][q].y);
                kahan_add(si[2 * h + 1][q], ci[2 * h + 1][q], pi_[h][q].y);
                pr[h][q] = pi_[h][q] = make_float2(0.f, 0.f);
            }
    }

    // partial exchange between the warps of a group: layout [value][lane]
    __device__ __forceinline__ void store_partial(float* dst, int lane) const {
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                dst[((k * R + q) * 2 + 0) * 32 + lane] = sr[k][q] - cr[k][q];
                dst[((k * R + q) * 2 + 1) * 32 + lane] = si[k][q] - ci[k][q];
            }
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                sr[k][q] -= cr[k][q];
                si[k][q] -= ci[k][q];
                cr[k][q] = ci[k][q] = 0.f;
            }
    }
    __device__ __forceinline__ void add_partial(const float* src, int lane) {
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                sr[k][q] += src[((k * R + q) * 2 + 0) * 32 + lane];
                si[k][q] += src[((k * R + q) * 2 + 1) * 32 + lane];
            }
    }

    // each target's total: the compensated sums of the two source groups added
    // across the lane pair (both lanes get it)
    __device__ __forceinline__ void reduce_groups() {
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                sr[k][q] -= cr[k][q];
                si[k][q] -= ci[k][q];
                cr[k][q] = ci[k][q] = 0.f;
                sr[k][q] += __shfl_xor_sync(FULL, sr[k][q], 1);
                si[k][q] += __shfl_xor_sync(FULL, si[k][q], 1);
            }
    }

    // lane sg writes its group's targets k with k % 2 = sg
    __device__ __forceinline__ void end(int lane) {
        reduce_groups();
        const float inv4pi = 0.0795774715459476678844418816862571882f;  // 1 / (4 pi)
        const int t0 = (lane / SP) * KT, sg = lane % SP;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int t = t0 + k;
            if (k % SP == sg && t < nt) {
                const int64_t o = perm[tbase + t];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float re = sr[k][q] * inv4pi, im = si[k][q] * inv4pi;
                    const int r = r0 + q;
                    if (r < out.split) out.u[(int64_t)r * n + o] = make_float2(re, im);
                    else out.u2[(int64_t)(r - out.split) * n + o] = make_float2(re, -im);
                }
            }
        }
    }

    // pair task: this task's contribution, scaled, to slot `slot` of each RHS row
    __device__ __forceinline__ void end_partial(int lane, void* part, int64_t cap, int64_t slot) {
        reduce_groups();
        const float inv4pi = 0.0795774715459476678844418816862571882f;  // 1 / (4 pi)
        float2* o = static_cast<float2*>(part) + slot;
        const int t0 = (lane / SP) * KT, sg = lane % SP;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int t = t0 + k;
            if (k % SP == sg && t < nt) {
#pragma unroll
                for (int q = 0; q < R; ++q)
                    o[(int64_t)(r0 + q) * cap + t] = make_float2(sr[k][q] * inv4pi, si[k][q] * inv4pi);
            }
        }
    }
};

template <int G, int R>
__global__ void __launch_bounds__(kLoopThreads, R == 1 ? 5 : 4)
    k_helmtile(LoopArgs a, const int32_t* __restrict__ perm, float kk, int qw0, int64_t n, int r0, HelmOut out) {
    pdl_wait();
    HelmTileOp<R, 2> op;
    op.rec = a.rec;
    op.perm = perm;
    op.kk = kk;
    op.qw0 = qw0;
    op.n = n;
    op.r0 = r0;
    op.out = out;
    warp_item_loop<2, G>(a, op);   // items of 64 targets
}

// records of one or two right-hand sides (two 16-byte words)
template <int G, int R>
int launch_helmtile(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, HelmOut u,
                    cudaStream_t s) {
    auto kern = k_helmtile<G, R>;
    using Op = HelmTileOp<R, 2>;
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

}  // namespace p2p
