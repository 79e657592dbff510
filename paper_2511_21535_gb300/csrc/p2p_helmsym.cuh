// Symmetric Helmholtz kernel: the work item's 64 targets and a tile's
// sources form a 64 x tile block of pairs laid out over the warp in two
// dimensions.  With KT targets per lane and SP = KT / 2 source groups, lane
// = SP tg + sg holds targets KT tg .. KT tg + KT - 1 in registers and takes
// the tile's sources j = sg, sg + SP, ...; each source read from shared
// memory serves KT evaluations, and for a mutual range the source sums (the
// pair credited to the source) are reduced over only the 32 / SP lanes that
// share sg.  At the end of the item the target sums of the SP source groups
// are added across lanes.
//
//   A side (target i):  u_i += G(r_ij) q_j,   B side (source j):  u_j += G(r_ij) q_i
//   G = exp(i k r) / r, the 1/(4 pi) applied when written.
//
// Summation is blocked: per lane a tile's partial (<= 16 sources) is added
// to the lane's running sum, the four lanes' sums are added at the end, and
// the update step adds the items' and tasks' partials compensated.
#pragma once

#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {

// Sums of four per-lane values over the lanes that share lane % SP (lane
// bits log2 SP .. 4), transposed: lanes with bits (4, 3) = u end with the
// total of v_u (SP = 4: 4 shuffles instead of 12; SP = 2: 5 instead of 16).
template <int SP>
__device__ __forceinline__ float group_reduce4(float v0, float v1, float v2, float v3, int lane) {
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
    if (SP == 2) kk += __shfl_xor_sync(0xffffffffu, kk, 2);
    return kk;
}

template <int R, int KT>
struct HelmSymOp {
    static_assert(KT == 4 || KT == 8, "targets per lane");
    static constexpr int SP = KT / 2;             // source groups (64 targets per warp)
    static constexpr int kOuts = 2 * R * KT;      // floats per lane exchanged between cooperating warps
    static constexpr bool kPartial = true;        // can write pair-task partial results
    static constexpr int kMutFloats = 2 * R;      // source sums per source in the tile scratch
    static constexpr int W = 2;                   // record stride: [x y z code | q pairs]

    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float kk;
    int qw0;
    int64_t n;
    int r0;
    HelmOut out;
    float2* mpart;
    int64_t mcap;

    float tx[KT], ty[KT], tz[KT];
    float tqr[KT][R], tqi[KT][R];
    float sr[KT][R], si[KT][R], pr[KT][R], pi_[KT][R];
    int tbase, nt, self0;
    float2* bsum;
    bool mut;
    int64_t mslot;
    int msrc0;

    __device__ __forceinline__ void set_scratch(float* p) { bsum = reinterpret_cast<float2*>(p); }
    __device__ __forceinline__ void set_range(bool on, int64_t slot_b, int src0) {
        mut = on;
        mslot = slot_b;
        msrc0 = src0;
    }

    __device__ __forceinline__ void load_positions(int lane, float sx, float sy, float sz) {
        const int t0 = (lane / SP) * KT;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int t = t0 + k;
            // idle targets sit on the first target: finite distances to every other particle
            const float4 r = rec[(int64_t)(tbase + (t < nt ? t : 0)) * W];
            tx[k] = r.x - sx;
            ty[k] = r.y - sy;
            tz[k] = r.z - sz;
        }
    }

    __device__ __forceinline__ void begin(int tb, int ntg, int sw_lo, int lane) {
        tbase = tb;
        nt = ntg;
        self0 = sw_lo;
        mut = false;
        load_positions(lane, 0.f, 0.f, 0.f);
        const int t0 = (lane / SP) * KT;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int t = t0 + k;
            const float4* rq = rec + (int64_t)(tb + (t < nt ? t : 0)) * W;
#pragma unroll
            for (int w = 0; w < (R + 1) / 2; ++w) {
                const float4 v = (t < nt) ? rq[qw0 + w] : make_float4(0.f, 0.f, 0.f, 0.f);
                tqr[k][2 * w] = v.x;
                tqi[k][2 * w] = v.y;
                if (2 * w + 1 < R) {
                    tqr[k][2 * w + 1] = v.z;
                    tqi[k][2 * w + 1] = v.w;
                }
            }
#pragma unroll
            for (int q = 0; q < R; ++q) sr[k][q] = si[k][q] = pr[k][q] = pi_[k][q] = 0.f;
        }
    }

    // periodic image of the current neighbour range: targets move by -shift
    __device__ __forceinline__ void set_shift(float sx, float sy, float sz) {
        load_positions(threadIdx.x & 31, sx, sy, sz);
    }

    __device__ __forceinline__ void source(const float4* __restrict__ sm, int j, bool valid, float4& ps, float (&qr)[R],
                                           float (&qi)[R]) const {
        const float4* rj = sm + (int64_t)j * W;
        ps = rj[0];
#pragma unroll
        for (int w = 0; w < (R + 1) / 2; ++w) {
            const float4 v = rj[qw0 + w];
            qr[2 * w] = valid ? v.x : 0.f;
            qi[2 * w] = valid ? v.y : 0.f;
            if (2 * w + 1 < R) {
                qr[2 * w + 1] = valid ? v.z : 0.f;
                qi[2 * w + 1] = valid ? v.w : 0.f;
            }
        }
    }

    // one-sided ranges (self and large boxes): A side only
    template <bool CHECK>
    __device__ __forceinline__ void body(const float4* __restrict__ sm, int cnt, int rec0) {
        const int lane = threadIdx.x & 31, sg = lane % SP, t0 = (lane / SP) * KT;
#pragma unroll 2
        for (int j = sg; j < cnt; j += SP) {
            float4 ps;
            float qr[R], qi[R];
            source(sm, j, true, ps, qr, qi);
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                const float dx = ps.x - tx[k], dy = ps.y - ty[k], dz = ps.z - tz[k];
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                bool me = false;
                if (CHECK) {
                    me = (rec0 + j) == self0 + t0 + k && t0 + k < nt;
                    r2 = me ? 1.f : r2;
                }
                const float inv = rsqrt_approx(r2);
                const float th = kk * (r2 * inv);
                float gr = inv * cos_approx(th), gi = inv * sin_approx(th);
                if (CHECK) {
                    gr = me ? 0.f : gr;
                    gi = me ? 0.f : gi;
                }
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    pr[k][q] = fmaf(gr, qr[q], fmaf(-gi, qi[q], pr[k][q]));
                    pi_[k][q] = fmaf(gr, qi[q], fmaf(gi, qr[q], pi_[k][q]));
                }
            }
        }
    }

    // mutual ranges: both sides; sources in steps of 4 SP (four per lane)
    template <bool ALLV>
    __device__ __forceinline__ void body_mut(const float4* __restrict__ sm, int cnt) {
        const int lane = threadIdx.x & 31, sg = lane % SP;
        const int u_me = ((lane >> 4) << 1) | ((lane >> 3) & 1);
#pragma unroll 2
        for (int g = 0; g < cnt; g += 4 * SP) {
            float vr[4][R], vi[4][R];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = g + SP * u + sg;
                const bool valid = ALLV || j < cnt;
                float4 ps;
                float qr[R], qi[R];
                source(sm, ALLV ? j : min(j, cnt - 1), valid, ps, qr, qi);
#pragma unroll
                for (int q = 0; q < R; ++q) vr[u][q] = vi[u][q] = 0.f;
#pragma unroll
                for (int k = 0; k < KT; ++k) {
                    const float dx = ps.x - tx[k], dy = ps.y - ty[k], dz = ps.z - tz[k];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float inv = rsqrt_approx(r2);
                    const float th = kk * (r2 * inv);
                    const float gr = inv * cos_approx(th), gi = inv * sin_approx(th);
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        pr[k][q] = fmaf(gr, qr[q], fmaf(-gi, qi[q], pr[k][q]));
                        pi_[k][q] = fmaf(gr, qi[q], fmaf(gi, qr[q], pi_[k][q]));
                        vr[u][q] = fmaf(gr, tqr[k][q], fmaf(-gi, tqi[k][q], vr[u][q]));
                        vi[u][q] = fmaf(gr, tqi[k][q], fmaf(gi, tqr[k][q], vi[u][q]));
                    }
                }
            }
            const int j_me = g + SP * u_me + sg;
            const bool writer = (lane & (SP == 4 ? 4 : 6)) == 0;   // one lane per (u, sg)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const float br = group_reduce4<SP>(vr[0][q], vr[1][q], vr[2][q], vr[3][q], lane);
                const float bi = group_reduce4<SP>(vi[0][q], vi[1][q], vi[2][q], vi[3][q], lane);
                if (writer && (ALLV || j_me < cnt)) bsum[j_me * R + q] = make_float2(br, bi);
            }
        }
    }

    __device__ __forceinline__ void tile(const float4* sm, int cnt, int rec0, bool chk) {
        if (mut) {
            // a mutual range never holds the targets' own copies
            if ((cnt & (4 * SP - 1)) == 0) body_mut<true>(sm, cnt);
            else body_mut<false>(sm, cnt);
            __syncwarp();
            const float inv4pi = 0.0795774715459476678844418816862571882f;  // 1 / (4 pi)
            const int lane = threadIdx.x & 31;
            const int64_t o = mslot + (rec0 - msrc0);
            for (int l = lane; l < cnt; l += 32)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float2 v = bsum[l * R + q];
                    mpart[(int64_t)(r0 + q) * mcap + o + l] = make_float2(v.x * inv4pi, v.y * inv4pi);
                }
            __syncwarp();
        } else if (chk) {
            body<true>(sm, cnt, rec0);
        } else {
            body<false>(sm, cnt, rec0);
        }
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                sr[k][q] += pr[k][q];
                si[k][q] += pi_[k][q];
                pr[k][q] = pi_[k][q] = 0.f;
            }
    }

    // partial exchange between the warps of a group: layout [value][lane]
    __device__ __forceinline__ void store_partial(float* dst, int lane) const {
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                dst[((k * R + q) * 2 + 0) * 32 + lane] = sr[k][q];
                dst[((k * R + q) * 2 + 1) * 32 + lane] = si[k][q];
            }
    }
    __device__ __forceinline__ void fold() {}
    __device__ __forceinline__ void add_partial(const float* src, int lane) {
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                sr[k][q] += src[((k * R + q) * 2 + 0) * 32 + lane];
                si[k][q] += src[((k * R + q) * 2 + 1) * 32 + lane];
            }
    }

    // the source groups' sums of each target, added across lanes (every lane gets the totals)
    __device__ __forceinline__ void reduce_groups() {
#pragma unroll
        for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
#pragma unroll
                for (int o = 1; o < SP; o <<= 1) {
                    sr[k][q] += __shfl_xor_sync(FULL, sr[k][q], o);
                    si[k][q] += __shfl_xor_sync(FULL, si[k][q], o);
                }
            }
    }

    // lane sg writes its group's targets k with k % SP = sg
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

template <int G, int R, int KT>
__global__ void __launch_bounds__(kLoopThreads, KT == 4 ? 4 : 3)
    k_helmsym(LoopArgs a, const int32_t* __restrict__ perm, float kk, int qw0, int64_t n, int r0, HelmOut out) {
    pdl_wait();
    HelmSymOp<R, KT> op;
    op.mpart = static_cast<float2*>(a.part);
    op.mcap = a.part_cap;
    op.rec = a.rec;
    op.perm = perm;
    op.kk = kk;
    op.qw0 = qw0;
    op.n = n;
    op.r0 = r0;
    op.out = out;
    warp_item_loop<2, G>(a, op);   // items of 64 targets
}

template <int G, int R, int KT>
int launch_helmsym(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, HelmOut u, cudaStream_t s) {
    auto kern = k_helmsym<G, R, KT>;
    using Op = HelmSymOp<R, KT>;
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
