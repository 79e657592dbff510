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
// The FP32 work of each pair of a lane's targets (differences, r^2, k r, G,
// the complex products of both sides) runs as packed two-wide instructions
// (add/mul/fma.rn.f32x2); a source's sums over the lane's targets are kept as
// an (even, odd) pair and added before the cross-lane reduction.
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

    static constexpr int KP = KT / 2;             // target pairs per lane (packed two-wide arithmetic)
    float2 ntx[KP], nty[KP], ntz[KP];             // negated target coordinates, packed in pairs
    float2 tqr[KP][R], tqi[KP][R], ntqi[KP][R];   // the targets' charges (zero for idle targets), packed
    float2 pr[KP][R], pi_[KP][R];                 // the current tile's target partial sums, packed
    float sr[KT][R], si[KT][R];
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
#pragma unroll
                for (int e = 0; e < 2 && 2 * w + e < R; ++e) {
                    const float re = e ? v.z : v.x, im = e ? v.w : v.y;
                    float2& a = tqr[k / 2][2 * w + e];
                    float2& b = tqi[k / 2][2 * w + e];
                    float2& c = ntqi[k / 2][2 * w + e];
                    if (k & 1) {
                        a.y = re;
                        b.y = im;
                        c.y = -im;
                    } else {
                        a.x = re;
                        b.x = im;
                        c.x = -im;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < R; ++q) sr[k][q] = si[k][q] = 0.f;
        }
#pragma unroll
        for (int h = 0; h < KP; ++h)
#pragma unroll
            for (int q = 0; q < R; ++q) pr[h][q] = pi_[h][q] = make_float2(0.f, 0.f);
    }

    // periodic image of the current neighbour range: targets move by -shift
    __device__ __forceinline__ void set_shift(float sx, float sy, float sz) {
        load_positions(threadIdx.x & 31, sx, sy, sz);
    }

    // source j of the tile: position and charges duplicated into both halves
    // (zero charges for an invalid source)
    __device__ __forceinline__ void source(const float4* __restrict__ sm, int j, bool valid, float2& sx, float2& sy,
                                           float2& sz, float2 (&qr)[R], float2 (&qi)[R], float2 (&nqi)[R]) const {
        const float4* rj = sm + (int64_t)j * W;
        const float4 ps = rj[0];
        sx = make_float2(ps.x, ps.x);
        sy = make_float2(ps.y, ps.y);
        sz = make_float2(ps.z, ps.z);
#pragma unroll
        for (int w = 0; w < (R + 1) / 2; ++w) {
            const float4 v = rj[qw0 + w];
#pragma unroll
            for (int e = 0; e < 2 && 2 * w + e < R; ++e) {
                const float re = valid ? (e ? v.z : v.x) : 0.f, im = valid ? (e ? v.w : v.y) : 0.f;
                qr[2 * w + e] = make_float2(re, re);
                qi[2 * w + e] = make_float2(im, im);
                nqi[2 * w + e] = make_float2(-im, -im);
            }
        }
    }

    // G = exp(i k r) / r for a source and the target pair h, packed (self pairs: 0)
    template <bool CHECK>
    __device__ __forceinline__ void kernel_g(float2 sx, float2 sy, float2 sz, int h, bool me0, bool me1,
                                             float2& gr, float2& gi, float2& dr2) const {
        const float2 dx = __fadd2_rn(sx, ntx[h]), dy = __fadd2_rn(sy, nty[h]), dz = __fadd2_rn(sz, ntz[h]);
        float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        if (CHECK) {
            r2.x = me0 ? 1.f : r2.x;
            r2.y = me1 ? 1.f : r2.y;
        }
        const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        const float2 th = __fmul2_rn(make_float2(kk, kk), __fmul2_rn(r2, inv));
        gr = __fmul2_rn(inv, make_float2(cos_approx(th.x), cos_approx(th.y)));
        gi = __fmul2_rn(inv, make_float2(sin_approx(th.x), sin_approx(th.y)));
        if (CHECK) {
            gr.x = me0 ? 0.f : gr.x;
            gi.x = me0 ? 0.f : gi.x;
            gr.y = me1 ? 0.f : gr.y;
            gi.y = me1 ? 0.f : gi.y;
        }
        dr2 = r2;
    }

    // one-sided ranges (self and large boxes): A side only
    template <bool CHECK>
    __device__ __forceinline__ void body(const float4* __restrict__ sm, int cnt, int rec0) {
        const int lane = threadIdx.x & 31, sg = lane % SP, t0 = (lane / SP) * KT;
#pragma unroll 2
        for (int j = sg; j < cnt; j += SP) {
            float2 sx, sy, sz, qr[R], qi[R], nqi[R];
            source(sm, j, true, sx, sy, sz, qr, qi, nqi);
#pragma unroll
            for (int h = 0; h < KP; ++h) {
                const int t = t0 + 2 * h;
                const bool me0 = CHECK && (rec0 + j) == self0 + t && t < nt;
                const bool me1 = CHECK && (rec0 + j) == self0 + t + 1 && t + 1 < nt;
                float2 gr, gi, r2;
                kernel_g<CHECK>(sx, sy, sz, h, me0, me1, gr, gi, r2);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    pr[h][q] = __ffma2_rn(gr, qr[q], __ffma2_rn(gi, nqi[q], pr[h][q]));
                    pi_[h][q] = __ffma2_rn(gr, qi[q], __ffma2_rn(gi, qr[q], pi_[h][q]));
                }
            }
        }
    }

    // mutual ranges: both sides; sources in steps of 4 SP (four per lane)
    template <bool ALLV>
    __device__ __forceinline__ void body_mut(const float4* __restrict__ sm, int cnt) {
        const int lane = threadIdx.x & 31, sg = lane % SP;
        const int u_me = ((lane >> 4) << 1) | ((lane >> 3) & 1);
#pragma unroll 1
        for (int g = 0; g < cnt; g += 4 * SP) {
            float vr[4][R], vi[4][R];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = g + SP * u + sg;
                const bool valid = ALLV || j < cnt;
                float2 sx, sy, sz, qr[R], qi[R], nqi[R];
                source(sm, ALLV ? j : min(j, cnt - 1), valid, sx, sy, sz, qr, qi, nqi);
                float2 br[R], bi[R];   // the source's sums over the lane's target pairs (even, odd)
#pragma unroll
                for (int q = 0; q < R; ++q) br[q] = bi[q] = make_float2(0.f, 0.f);
#pragma unroll
                for (int h = 0; h < KP; ++h) {
                    float2 gr, gi, r2;
                    kernel_g<false>(sx, sy, sz, h, false, false, gr, gi, r2);
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        pr[h][q] = __ffma2_rn(gr, qr[q], __ffma2_rn(gi, nqi[q], pr[h][q]));
                        pi_[h][q] = __ffma2_rn(gr, qi[q], __ffma2_rn(gi, qr[q], pi_[h][q]));
                        br[q] = __ffma2_rn(gr, tqr[h][q], __ffma2_rn(gi, ntqi[h][q], br[q]));
                        bi[q] = __ffma2_rn(gr, tqi[h][q], __ffma2_rn(gi, tqr[h][q], bi[q]));
                    }
                }
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    vr[u][q] = br[q].x + br[q].y;
                    vi[u][q] = bi[q].x + bi[q].y;
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
        for (int h = 0; h < KP; ++h)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                sr[2 * h][q] += pr[h][q].x;
                si[2 * h][q] += pi_[h][q].x;
                sr[2 * h + 1][q] += pr[h][q].y;
                si[2 * h + 1][q] += pi_[h][q].y;
                pr[h][q] = pi_[h][q] = make_float2(0.f, 0.f);
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
