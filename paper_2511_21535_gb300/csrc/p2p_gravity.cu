// Softened-gravity P2P kernel (stellar dynamics, Section 5.2):
//   phi_i = - sum_{j in near(i), j != i} m_j (r^2 + eps^2)^(-1/2)
//   a_i   =   sum_{j in near(i), j != i} m_j (x_j - x_i) (r^2 + eps^2)^(-3/2)
// Per pair: 3 FADD, 3 FFMA, 1 MUFU rsqrt, 3 FMUL, 1 FADD, 3 FFMA -> the
// kernel is bound by the FP32 pipe.  Each tile's partial sums are folded into
// compensated (Kahan) accumulators unless the plan asks for plain FP32.
#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {

// MUT: mutual (symmetric) pair tasks: each pair is evaluated once and
// credited to both particles; a tile's B-side (source) sums [phi, a] are
// reduced across the warp four sources at a time and written per source.
template <int K, bool COMP, bool MUT = false>
struct GravityOp {
    static constexpr int kOuts = 4 * K;   // floats per lane exchanged between cooperating warps
    static constexpr bool kPartial = true; // can write pair-task partial results
    static constexpr int kMutFloats = MUT ? 4 : 0;

    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float eps2;
    float* __restrict__ phi;
    float* __restrict__ acc;

    float tx[K], ty[K], tz[K];
    int self[K];
    float s[K][4], c[K][4], p[K][4];
    int tbase, nt;
    // mutual tasks: the targets' masses (zero on idle lanes), the per-warp
    // B-side scratch of one tile, and where the B-side sums go
    float tm[K];
    float4* bsum;
    bool mut;
    float4* mpart;
    int64_t mslot;
    int msrc0;

    __device__ __forceinline__ void set_scratch(float* q) { bsum = reinterpret_cast<float4*>(q); }

    // the current source range: mutual or not, its first source-sum slot and first record
    __device__ __forceinline__ void set_range(bool on, int64_t slot_b, int src0) {
        mut = MUT && on;
        mslot = slot_b;
        msrc0 = src0;
    }

    __device__ __forceinline__ void begin(int tb, int ntg, int sw_lo, int lane) {
        tbase = tb;
        nt = ntg;
        mut = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            // idle lanes sit on the first target: finite distances to every other particle
            const float4 r = rec[tb + (l < nt ? l : 0)];
            tx[k] = r.x;
            ty[k] = r.y;
            tz[k] = r.z;
            tm[k] = (MUT && l < nt) ? r.w : 0.f;   // mutual ranges: the targets' masses (zero on idle lanes)
            self[k] = (l < nt) ? sw_lo + l : -1;
#pragma unroll
            for (int o = 0; o < 4; ++o) s[k][o] = c[k][o] = p[k][o] = 0.f;
        }
    }

    // periodic image of the current neighbour range: targets move by -shift
    // (reloaded from the records, so no extra registers hold the originals)
    __device__ __forceinline__ void set_shift(float sx, float sy, float sz) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            const float4 r = rec[tbase + (l < nt ? l : 0)];
            tx[k] = r.x - sx;
            ty[k] = r.y - sy;
            tz[k] = r.z - sz;
        }
    }

    template <bool CHECK>
    __device__ __forceinline__ void body(const float4* __restrict__ sm, int cnt, int rec0) {
#pragma unroll 8
        for (int j = 0; j < cnt; ++j) {
            const float4 src = sm[j];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float dx = src.x - tx[k];
                const float dy = src.y - ty[k];
                const float dz = src.z - tz[k];
                float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                float m = src.w;
                if (CHECK) {
                    const bool me = (rec0 + j) == self[k];
                    m = me ? 0.f : m;
                    r2 = me ? 1.f : r2;
                }
                const float inv = rsqrt_approx(r2);
                const float mi = m * inv;
                const float mi3 = mi * (inv * inv);
                float (&acc_k)[4] = COMP ? p[k] : s[k];
                acc_k[0] += mi;
                acc_k[1] = fmaf(mi3, dx, acc_k[1]);
                acc_k[2] = fmaf(mi3, dy, acc_k[2]);
                acc_k[3] = fmaf(mi3, dz, acc_k[3]);
            }
        }
    }

    // Mutual body: four sources per step (see the Helmholtz op); the source
    // receives m_i (x_i - x_j) h^-3 = -m_i d h^-3 and m_i / h from target i.
    template <bool ALLV>
    __device__ __forceinline__ void body_mut(const float4* __restrict__ sm, int cnt) {
        const int lane = threadIdx.x & 31;
        for (int j0 = 0; j0 < cnt; j0 += 4) {
            float v[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool valid = ALLV || (j0 + u < cnt);
                const float4 src = sm[ALLV ? j0 + u : min(j0 + u, cnt - 1)];
                const float m = valid ? src.w : 0.f;
#pragma unroll
                for (int o = 0; o < 4; ++o) v[u][o] = 0.f;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float dx = src.x - tx[k];
                    const float dy = src.y - ty[k];
                    const float dz = src.z - tz[k];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    const float inv = rsqrt_approx(r2);
                    const float inv2 = inv * inv;
                    const float mi = m * inv;
                    const float mi3 = mi * inv2;
                    float (&acc_k)[4] = COMP ? p[k] : s[k];
                    acc_k[0] += mi;
                    acc_k[1] = fmaf(mi3, dx, acc_k[1]);
                    acc_k[2] = fmaf(mi3, dy, acc_k[2]);
                    acc_k[3] = fmaf(mi3, dz, acc_k[3]);
                    const float ti = tm[k] * inv;
                    const float ti3 = ti * inv2;
                    v[u][0] += ti;
                    v[u][1] = fmaf(-ti3, dx, v[u][1]);
                    v[u][2] = fmaf(-ti3, dy, v[u][2]);
                    v[u][3] = fmaf(-ti3, dz, v[u][3]);
                }
            }
            const int u_me = lane >> 3;
            float t[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) t[o] = warp_reduce4(v[0][o], v[1][o], v[2][o], v[3][o], lane);
            if ((lane & 7) == 0 && (ALLV || j0 + u_me < cnt)) bsum[j0 + u_me] = make_float4(t[0], t[1], t[2], t[3]);
        }
    }

    __device__ __forceinline__ void tile(const float4* sm, int cnt, int rec0, bool chk) {
        if (MUT && mut) {
            // a mutual task never holds the targets' own copies
            if ((cnt & 3) == 0) body_mut<true>(sm, cnt);
            else body_mut<false>(sm, cnt);
            __syncwarp();
            const int lane = threadIdx.x & 31;
            const int64_t o = mslot + (rec0 - msrc0);
            for (int l = lane; l < cnt; l += 32) mpart[o + l] = bsum[l];
            __syncwarp();
        } else if (chk) {
            body<true>(sm, cnt, rec0);
        } else {
            body<false>(sm, cnt, rec0);
        }
        if (COMP) {
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    kahan_add(s[k][o], c[k][o], p[k][o]);
                    p[k][o] = 0.f;
                }
        }
    }

    // partial exchange between the warps of a group: layout [value][lane]
    __device__ __forceinline__ void store_partial(float* dst, int lane) const {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < 4; ++o) dst[(k * 4 + o) * 32 + lane] = s[k][o] - c[k][o];
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                s[k][o] -= c[k][o];
                c[k][o] = 0.f;
            }
    }
    __device__ __forceinline__ void add_partial(const float* src, int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < 4; ++o) s[k][o] += src[(k * 4 + o) * 32 + lane];
    }

    // pair task: raw sums (phi not yet negated) to the task's slots
    __device__ __forceinline__ void end_partial(int lane, void* part, int64_t, int64_t slot) {
        float4* o = static_cast<float4*>(part) + slot;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt)
                o[l] = make_float4(s[k][0] - c[k][0], s[k][1] - c[k][1], s[k][2] - c[k][2], s[k][3] - c[k][3]);
        }
    }

    __device__ __forceinline__ void end(int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt) {
                const int64_t o = perm[tbase + l];
                phi[o] = -(s[k][0] - c[k][0]);
                acc[3 * o + 0] = s[k][1] - c[k][1];
                acc[3 * o + 1] = s[k][2] - c[k][2];
                acc[3 * o + 2] = s[k][3] - c[k][3];
            }
        }
    }
};

// One-sided, compensated, K in {2, 4}: the same arithmetic as GravityOp with
// the FP32 work of each pair of targets in packed two-wide instructions
// (add/mul/fma.rn.f32x2: two lane-operations per issue slot, each half rounded
// as the scalar operation would be, so the sums are bitwise those of the
// scalar kernel); rsqrt stays scalar on the MUFU pipe.  The scalar kernel
// issues about as many instructions per pair as the FP32 pipe has cycles.
//
// Items of at most 32 targets with two targets per lane (a box of <= 32
// particles, or the last part of a larger box) would leave the second half
// of every packed operation idle; such an item runs source-split instead:
// each lane holds its one target in both halves, the halves take the even and
// the odd sources of the tile, and the two halves' compensated sums are added
// when the item is written.  (On the 4.2 M Plummer sphere 5.5 % of the
// evaluated slots of 64-target items are idle; source-split halves that.)
template <int K>
struct GravityPackOp {
    static_assert(K == 2 || K == 4, "target pairs");
    static constexpr int KP = K / 2;
    static constexpr int kOuts = 4 * K;
    static constexpr bool kPartial = true;
    static constexpr int kMutFloats = 0;

    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float eps2;
    float* __restrict__ phi;
    float* __restrict__ acc;

    float2 ntx[KP], nty[KP], ntz[KP];   // negated target coordinates of lanes' targets (2h, 2h+1)
    float2 pp[KP][4];                   // the current tile's partial sums, packed
    float s[K][4], c[K][4];             // source-split items: [0] even, [1] odd sources of the one target
    int self[K];
    int tbase, nt;
    bool split;                         // K == 2 and the item holds <= 32 targets

    __device__ __forceinline__ void load_positions(int lane, float sx, float sy, float sz) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = split ? lane : lane + 32 * k;
            // idle lanes sit on the first target: finite distances to every other particle
            const float4 r = rec[tbase + (l < nt ? l : 0)];
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
        split = K == 2 && ntg <= 32;
        load_positions(lane, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = split ? lane : lane + 32 * k;
            self[k] = (l < nt) ? sw_lo + l : -1;
#pragma unroll
            for (int o = 0; o < 4; ++o) s[k][o] = c[k][o] = 0.f;
        }
#pragma unroll
        for (int h = 0; h < KP; ++h)
#pragma unroll
            for (int o = 0; o < 4; ++o) pp[h][o] = make_float2(0.f, 0.f);
    }

    // periodic image of the current neighbour range: targets move by -shift
    __device__ __forceinline__ void set_shift(float sx, float sy, float sz) {
        load_positions(threadIdx.x & 31, sx, sy, sz);
    }

    template <bool CHECK>
    __device__ __forceinline__ void body(const float4* __restrict__ sm, int cnt, int rec0) {
        const float2 e2 = make_float2(eps2, eps2);
#pragma unroll 4
        for (int j = 0; j < cnt; ++j) {
            const float4 src = sm[j];
            const float2 sx = make_float2(src.x, src.x), sy = make_float2(src.y, src.y),
                         sz = make_float2(src.z, src.z);
#pragma unroll
            for (int h = 0; h < KP; ++h) {
                const float2 dx = __fadd2_rn(sx, ntx[h]), dy = __fadd2_rn(sy, nty[h]), dz = __fadd2_rn(sz, ntz[h]);
                float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
                float2 m = make_float2(src.w, src.w);
                if (CHECK) {
                    const bool me0 = (rec0 + j) == self[2 * h], me1 = (rec0 + j) == self[2 * h + 1];
                    m.x = me0 ? 0.f : m.x;
                    m.y = me1 ? 0.f : m.y;
                    r2.x = me0 ? 1.f : r2.x;
                    r2.y = me1 ? 1.f : r2.y;
                }
                const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                const float2 mi = __fmul2_rn(m, inv);
                const float2 mi3 = __fmul2_rn(mi, __fmul2_rn(inv, inv));
                pp[h][0] = __fadd2_rn(pp[h][0], mi);
                pp[h][1] = __ffma2_rn(mi3, dx, pp[h][1]);
                pp[h][2] = __ffma2_rn(mi3, dy, pp[h][2]);
                pp[h][3] = __ffma2_rn(mi3, dz, pp[h][3]);
            }
        }
    }

    // source-split pair step: sources a (half 0) and b (half 1) against the lane's one target;
    // a lone last source leaves half 1 with no mass and a unit distance
    template <bool CHECK>
    __device__ __forceinline__ void split_pair(const float4& a, const float4& b, bool lone, int ja, float2 e2) {
        const float2 sx = make_float2(a.x, b.x), sy = make_float2(a.y, b.y), sz = make_float2(a.z, b.z);
        const float2 dx = __fadd2_rn(sx, ntx[0]), dy = __fadd2_rn(sy, nty[0]), dz = __fadd2_rn(sz, ntz[0]);
        float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
        float2 m = make_float2(a.w, lone ? 0.f : b.w);
        if (lone) r2.y = 1.f;
        if (CHECK) {
            const bool me0 = ja == self[0], me1 = !lone && ja + 1 == self[0];
            m.x = me0 ? 0.f : m.x;
            m.y = me1 ? 0.f : m.y;
            r2.x = me0 ? 1.f : r2.x;
            r2.y = me1 ? 1.f : r2.y;
        }
        const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        const float2 mi = __fmul2_rn(m, inv);
        const float2 mi3 = __fmul2_rn(mi, __fmul2_rn(inv, inv));
        pp[0][0] = __fadd2_rn(pp[0][0], mi);
        pp[0][1] = __ffma2_rn(mi3, dx, pp[0][1]);
        pp[0][2] = __ffma2_rn(mi3, dy, pp[0][2]);
        pp[0][3] = __ffma2_rn(mi3, dz, pp[0][3]);
    }

    template <bool CHECK>
    __device__ __forceinline__ void body_split(const float4* __restrict__ sm, int cnt, int rec0) {
        const float2 e2 = make_float2(eps2, eps2);
        const int cpair = cnt & ~1;
#pragma unroll 4
        for (int j = 0; j < cpair; j += 2) split_pair<CHECK>(sm[j], sm[j + 1], false, rec0 + j, e2);
        if (cnt & 1) {
            const float4 a = sm[cpair];
            split_pair<CHECK>(a, a, true, rec0 + cpair, e2);
        }
    }

    __device__ __forceinline__ void tile(const float4* sm, int cnt, int rec0, bool chk) {
        if (K == 2 && split) {
            if (chk) body_split<true>(sm, cnt, rec0);
            else body_split<false>(sm, cnt, rec0);
        } else if (chk) {
            body<true>(sm, cnt, rec0);
        } else {
            body<false>(sm, cnt, rec0);
        }
#pragma unroll
        for (int h = 0; h < KP; ++h)
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                kahan_add(s[2 * h][o], c[2 * h][o], pp[h][o].x);
                kahan_add(s[2 * h + 1][o], c[2 * h + 1][o], pp[h][o].y);
                pp[h][o] = make_float2(0.f, 0.f);
            }
    }

    __device__ __forceinline__ void store_partial(float* dst, int lane) const {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < 4; ++o) dst[(k * 4 + o) * 32 + lane] = s[k][o] - c[k][o];
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                s[k][o] -= c[k][o];
                c[k][o] = 0.f;
            }
    }
    __device__ __forceinline__ void add_partial(const float* src, int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < 4; ++o) s[k][o] += src[(k * 4 + o) * 32 + lane];
    }
    // source-split items: the one target's sums, even plus odd sources
    __device__ __forceinline__ float4 split_total() const {
        return make_float4((s[0][0] - c[0][0]) + (s[1][0] - c[1][0]), (s[0][1] - c[0][1]) + (s[1][1] - c[1][1]),
                           (s[0][2] - c[0][2]) + (s[1][2] - c[1][2]), (s[0][3] - c[0][3]) + (s[1][3] - c[1][3]));
    }
    __device__ __forceinline__ void end_partial(int lane, void* part, int64_t, int64_t slot) {
        float4* o = static_cast<float4*>(part) + slot;
        if (K == 2 && split) {
            if (lane < nt) o[lane] = split_total();
            return;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt)
                o[l] = make_float4(s[k][0] - c[k][0], s[k][1] - c[k][1], s[k][2] - c[k][2], s[k][3] - c[k][3]);
        }
    }
    __device__ __forceinline__ void end(int lane) {
        if (K == 2 && split) {
            if (lane < nt) {
                const int64_t o = perm[tbase + lane];
                const float4 v = split_total();
                phi[o] = -v.x;
                acc[3 * o + 0] = v.y;
                acc[3 * o + 1] = v.z;
                acc[3 * o + 2] = v.w;
            }
            return;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt) {
                const int64_t o = perm[tbase + l];
                phi[o] = -(s[k][0] - c[k][0]);
                acc[3 * o + 0] = s[k][1] - c[k][1];
                acc[3 * o + 1] = s[k][2] - c[k][2];
                acc[3 * o + 2] = s[k][3] - c[k][3];
            }
        }
    }
};

template <int K, int G>
__global__ void __launch_bounds__(kLoopThreads, 4)
    k_gravity_pk(LoopArgs a, const int32_t* __restrict__ perm, float eps2, float* __restrict__ phi,
                 float* __restrict__ acc) {
    pdl_wait();
    GravityPackOp<K> op;
    op.rec = a.rec;
    op.perm = perm;
    op.eps2 = eps2;
    op.phi = phi;
    op.acc = acc;
    warp_item_loop<K, G>(a, op);
}

template <int K, int G>
static int launch_gravity_pk(const Plan* p, const LoopArgs& a, const int32_t* perm, float eps2, float* phi,
                             float* acc, cudaStream_t s) {
    auto kern = k_gravity_pk<K, G>;
    using Op = GravityPackOp<K>;
    const size_t smem = loop_smem_bytes(a.tile, a.words, Op::kOuts, G, Op::kMutFloats);
    P2P_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0) {
        P2P_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
        if (per_sm < 1) per_sm = 1;
    }
    P2P_CUDA_TRY(launch_pdl(kern, num_sms() * per_sm, kLoopThreads, smem, s, a, perm, eps2, phi, acc));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

template <int K, int G, bool COMP, bool MUT = false>
__global__ void __launch_bounds__(kLoopThreads, MUT ? 3 : 4)
    k_gravity(LoopArgs a, const int32_t* __restrict__ perm, float eps2, float* __restrict__ phi,
              float* __restrict__ acc) {
    pdl_wait();
    GravityOp<K, COMP, MUT> op;
    if constexpr (MUT) op.mpart = static_cast<float4*>(a.part);
    op.rec = a.rec;
    op.perm = perm;
    op.eps2 = eps2;
    op.phi = phi;
    op.acc = acc;
    warp_item_loop<K, G>(a, op);
}

template <int K, int G, bool COMP, bool MUT = false>
static int launch_gravity(const Plan* p, const LoopArgs& a, const int32_t* perm, float eps2, float* phi, float* acc,
                          cudaStream_t s) {
    auto kern = k_gravity<K, G, COMP, MUT>;
    using Op = GravityOp<K, COMP, MUT>;
    const size_t smem = loop_smem_bytes(a.tile, a.words, Op::kOuts, G, Op::kMutFloats);
    P2P_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0) {
        P2P_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
        if (per_sm < 1) per_sm = 1;
    }
    P2P_CUDA_TRY(launch_pdl(kern, num_sms() * per_sm, kLoopThreads, smem, s, a, perm, eps2, phi, acc));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

template <int G>
static int launch_gravity_g(const Plan* p, const LoopArgs& a, const int32_t* perm, float eps2, float* phi, float* acc,
                            bool comp, cudaStream_t s) {
    if (a.task_kind) {   // symmetric tasks or plans: two targets per lane, compensated
        if (p->tpl != 2 || !comp) return P2P_ERR_UNSUPPORTED;
        return launch_gravity<2, G, true, true>(p, a, perm, eps2, phi, acc, s);
    }
    switch (p->tpl) {
        case 1: return comp ? launch_gravity<1, G, true>(p, a, perm, eps2, phi, acc, s)
                            : launch_gravity<1, G, false>(p, a, perm, eps2, phi, acc, s);
        case 2: return comp ? launch_gravity_pk<2, G>(p, a, perm, eps2, phi, acc, s)
                            : launch_gravity<2, G, false>(p, a, perm, eps2, phi, acc, s);
        case 4: return comp ? launch_gravity_pk<4, G>(p, a, perm, eps2, phi, acc, s)
                            : launch_gravity<4, G, false>(p, a, perm, eps2, phi, acc, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

int launch_gravity_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float eps, float* phi, float* acc,
                          cudaStream_t s) {
    const float eps2 = eps * eps;
    const bool comp = !(p->flags & P2P_PLAN_PLAIN_FP32);
    switch (p->group) {
        case 1: return launch_gravity_g<1>(p, a, perm, eps2, phi, acc, comp, s);
        case 2: return launch_gravity_g<2>(p, a, perm, eps2, phi, acc, comp, s);
        case 4: return launch_gravity_g<4>(p, a, perm, eps2, phi, acc, comp, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

}  // namespace p2p
