// Pattern mode for regular grids: the precomputed-pattern P2P of the DBIM
// solver (Section 5.1), where all interaction patterns between neighbouring
// boxes are computed once and read from shared memory.
//
// On a lattice of spacing h with t points per leaf-box edge, the lattice
// displacement between a target and a source in a neighbouring box lies in
// [-(2t-1), 2t-1]^3, so G takes at most (4t-1)^3 values.  The table holds
// 4 pi G(h |D|) = exp(i k h |D|) / (h |D|) (0 at D = 0, which excludes the
// self pair) in double precision rounded to float, at index
//   (Dx + m) + (Dy + m) sy + (Dz + m) sz,   m = 2t - 1,
// and each record carries its lattice code ix + iy sy + iz sz in the w slot,
// so a pair's entry is table[code_j - code_i + bias].  sy = 20 (= 4 mod 16)
// makes the 16 lanes of a half-warp, which hold the 4 x 4 targets of one
// box layer, read 16 distinct 8-byte slots: no shared-memory bank conflicts.
#include <cmath>

#include "common.cuh"
#include "p2p_helmholtz.cuh"

namespace p2p {

int pattern_setup(Plan* p, float h, int t) {
    const int D = 4 * t - 1;
    int sy = D;
    while (sy % 16 != 4) ++sy;
    const int sz = sy * D;
    const int m = 2 * t - 1;
    const int size = (D - 1) * (1 + sy + sz) + 1;
    if (size > kPatternMaxEntries) return P2P_ERR_UNSUPPORTED;
    p->pattern = 1;
    p->grid_h = h;
    p->grid_t = t;
    p->pat_sy = sy;
    p->pat_sz = sz;
    p->pat_size = size;
    p->pat_bias = m * (1 + sy + sz);
    return P2P_OK;
}

__global__ void k_pattern_table(double h, double k, int t, int sy, int sz, int size, float2* __restrict__ table) {
    pdl_wait();
    pdl_release();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= size) return;
    const int D = 4 * t - 1, m = 2 * t - 1;
    const int iz = idx / sz, rem = idx % sz, iy = rem / sy, ix = rem % sy;
    float2 v = make_float2(0.f, 0.f);
    if (ix < D && iy < D && iz < D) {
        const double dx = ix - m, dy = iy - m, dz = iz - m;
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > 0.0) {
            const double r = h * sqrt(d2);
            double sn, cs;
            sincos(k * r, &sn, &cs);
            v = make_float2((float)(cs / r), (float)(sn / r));
        }
    }
    table[idx] = v;
}

// COMPACT: one right-hand side, records [code, Re q, Im q, 0]
template <int K, int R, bool COMPACT = false>
struct HelmPatternOp : HelmOp<K, R, true, false, 0> {
    using Base = HelmOp<K, R, true, false, 0>;
    static constexpr bool kPartial = false;   // pattern plans are target-owned
    static constexpr int kMutFloats = 0;
    const float2* tab;   // shared-memory table, already offset by the bias
    int tcode[K];

    __device__ __forceinline__ void begin(int tb, int ntg, int sw_lo, int lane) {
        Base::begin(tb, ntg, sw_lo, lane);
        // idle lanes borrow the first target's code so every lookup stays inside the table
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            const float4 r = this->rec[(int64_t)(tb + (l < ntg ? l : 0)) * this->words];
            tcode[k] = __float_as_int(COMPACT ? r.x : r.w);
        }
    }

    __device__ __forceinline__ void tile(const float4* sm, int cnt, int, bool) {
        const float4* rj = sm;
#pragma unroll 4
        for (int j = 0; j < cnt; ++j, rj += (COMPACT ? 1 : this->words)) {
            const float4 ps = rj[0];
            const int cj = __float_as_int(COMPACT ? ps.x : ps.w);
            float qr[R], qi[R];
            if (COMPACT) {
                qr[0] = ps.y;
                qi[0] = ps.z;
            } else {
#pragma unroll
                for (int w = 0; w < (R + 1) / 2; ++w) {
                    const float4 v = rj[this->qw0 + w];
                    qr[2 * w] = v.x;
                    qi[2 * w] = v.y;
                    if (2 * w + 1 < R) {
                        qr[2 * w + 1] = v.z;
                        qi[2 * w + 1] = v.w;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float2 g = tab[cj - tcode[k]];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    this->pr[k][q] = fmaf(g.x, qr[q], fmaf(-g.y, qi[q], this->pr[k][q]));
                    this->pi_[k][q] = fmaf(g.x, qi[q], fmaf(g.y, qr[q], this->pi_[k][q]));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                kahan_add(this->sr[k][q], this->cr[k][q], this->pr[k][q]);
                kahan_add(this->si[k][q], this->ci[k][q], this->pi_[k][q]);
                this->pr[k][q] = 0.f;
                this->pi_[k][q] = 0.f;
            }
    }
};

template <int K, int G, int R, bool COMPACT>
__global__ void __launch_bounds__(kLoopThreads, 4)
    k_helmholtz_pattern(LoopArgs a, const int32_t* __restrict__ perm, const float2* __restrict__ table, int size,
                        int bias, size_t table_off, int qw0, int64_t n, int r0, HelmOut out) {
    pdl_wait();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* tab = reinterpret_cast<float2*>(smem_raw + table_off);
    for (int i = threadIdx.x; i < size; i += blockDim.x) tab[i] = table[i];
    __syncthreads();
    HelmPatternOp<K, R, COMPACT> op;
    op.rec = a.rec;
    op.perm = perm;
    op.kk = 0.f;
    op.words = a.words;
    op.qw0 = qw0;
    op.n = n;
    op.r0 = r0;
    op.out = out;
    op.tab = tab + bias;
    warp_item_loop<K, G>(a, op);
}

template <int K, int G, int R, bool COMPACT = false>
static int launch_pat(const Plan* p, const LoopArgs& a, const int32_t* perm, const float2* table, int r0, HelmOut out,
                      cudaStream_t s) {
    auto kern = k_helmholtz_pattern<K, G, R, COMPACT>;
    const size_t loop = loop_smem_bytes(a.tile, a.words, HelmPatternOp<K, R, COMPACT>::kOuts, G);
    const size_t table_off = (loop + 15) / 16 * 16;
    const size_t smem = table_off + (size_t)p->pat_size * sizeof(float2);
    P2P_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0) {
        P2P_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
        if (per_sm < 1) per_sm = 1;
    }
    P2P_CUDA_TRY(launch_pdl(kern, num_sms() * per_sm, kLoopThreads, smem, s, a, perm, table, p->pat_size, p->pat_bias, table_off,
                                                        1 + r0 / 2, p->n, r0, out));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

template <int K, int G>
static int pat_r(const Plan* p, const LoopArgs& a, const int32_t* perm, const float2* table, int r0, int R,
                 HelmOut out, cudaStream_t s) {
    switch (R) {
        case 1: return a.words == 1 ? launch_pat<K, G, 1, true>(p, a, perm, table, r0, out, s)
                                    : launch_pat<K, G, 1>(p, a, perm, table, r0, out, s);
        case 2: return launch_pat<K, G, 2>(p, a, perm, table, r0, out, s);
        case 4: return launch_pat<K, G, 4>(p, a, perm, table, r0, out, s);
        case 8: return launch_pat<K, G, 8>(p, a, perm, table, r0, out, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

int launch_helmholtz_pattern(const Plan* p, const LoopArgs& a, const int32_t* perm, float k, float2* table,
                             HelmOut out, cudaStream_t s) {
    P2P_CUDA_TRY(launch_pdl(k_pattern_table, (p->pat_size + 255) / 256, 256, 0, s, (double)p->grid_h, (double)k, p->grid_t, p->pat_sy,
                                                              p->pat_sz, p->pat_size, table));
    P2P_LAUNCH_CHECK();
    const int K = p->tpl >= 2 ? 2 : 1;
    int r0 = 0;
    while (r0 < p->nrhs) {
        const int left = p->nrhs - r0;
        const int R = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        if (r0 > 0) {   // the first pass follows build_items, which zeroed the operator section
            const int st0 = fill32(&a.hdr->work_ctr, 0u, 1, s);
            if (st0) return st0;
        }
        int st;
        if (p->group >= 2)
            st = K == 2 ? pat_r<2, 4>(p, a, perm, table, r0, R, out, s) : pat_r<1, 4>(p, a, perm, table, r0, R, out, s);
        else
            st = K == 2 ? pat_r<2, 1>(p, a, perm, table, r0, R, out, s) : pat_r<1, 1>(p, a, perm, table, r0, R, out, s);
        if (st) return st;
        r0 += R;
    }
    return P2P_OK;
}

}  // namespace p2p
