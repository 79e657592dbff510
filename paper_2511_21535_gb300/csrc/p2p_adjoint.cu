// Adjoint P2P kernels: gradients of a real loss L through the near-field sums
// (the gradient loop of the DBIM inverse solver, Section 5.1, needs them).
// Convention for complex values: grad = dL/dRe + i dL/dIm.  Pair terms are
// recomputed, never stored.
//
// Helmholtz, given gbar = dL/du, records [x y z 0 | q pairs | gbar pairs]:
//   grad_q_k = sum_j conj(G_kj) gbar_j
//   grad_x_k = Re sum_j sum_r (conj(gbar_k) q_j + conj(gbar_j) q_k) dG/dr (x_k - x_j)/r
//   dG/dr    = G (i k - 1/r)
// Gravity, given gphi = dL/dphi and gacc = dL/da, records [x y z m | gphi gacc]:
//   grad_m_k = sum_j [ -gphi_j h^-1 - (gacc_j . d) h^-3 ]
//   grad_x_k = sum_j [ -h^-3 d (gphi_k m_j + gphi_j m_k) + J(d)(m_k gacc_j - m_j gacc_k) ]
//   with d = x_j - x_k, h^2 = r^2 + eps^2, J(d) v = h^-3 v - 3 h^-5 d (d . v).
#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {

// ---------------------------------------------------------------------------
// Helmholtz: grad_q and grad_x together
// ---------------------------------------------------------------------------
template <int K, int R, bool PRECISE>
struct HelmAdjOp {
    static constexpr int NO = 2 * R + 3;        // outputs per target: grad_q (R complex), grad_x (3)
    static constexpr int kOuts = NO * K;
    static constexpr bool kPartial = false;   // adjoints are target-owned only
    static constexpr int kMutFloats = 0;

    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float kk;
    int words, qw0, gw0;
    int64_t n;
    int r0;
    bool accumulate_x;                           // a later RHS pass adds to grad_x
    float2* __restrict__ grad_q;
    float* __restrict__ grad_x;

    float tx[K], ty[K], tz[K];
    float tqr[K][R], tqi[K][R], tbr[K][R], tbi[K][R];
    int self[K];
    float s[K][NO], c[K][NO], p[K][NO];
    int tbase, nt;

    __device__ __forceinline__ void begin(int tb, int ntg, int sw_lo, int lane) {
        tbase = tb;
        nt = ntg;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            const bool v = l < nt;
            const float4* r = rec + (int64_t)(tb + (v ? l : 0)) * words;
            const float4 ps = v ? r[0] : make_float4(0.f, 0.f, 0.f, 0.f);
            tx[k] = ps.x;
            ty[k] = ps.y;
            tz[k] = ps.z;
#pragma unroll
            for (int w = 0; w < (R + 1) / 2; ++w) {
                const float4 a = v ? r[qw0 + w] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 g = v ? r[gw0 + w] : make_float4(0.f, 0.f, 0.f, 0.f);
                tqr[k][2 * w] = a.x;
                tqi[k][2 * w] = a.y;
                tbr[k][2 * w] = g.x;
                tbi[k][2 * w] = g.y;
                if (2 * w + 1 < R) {
                    tqr[k][2 * w + 1] = a.z;
                    tqi[k][2 * w + 1] = a.w;
                    tbr[k][2 * w + 1] = g.z;
                    tbi[k][2 * w + 1] = g.w;
                }
            }
            self[k] = v ? sw_lo + l : -1;
#pragma unroll
            for (int o = 0; o < NO; ++o) s[k][o] = c[k][o] = p[k][o] = 0.f;
        }
    }

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
        for (int j = 0; j < cnt; ++j, rj += words) {
            const float4 ps = rj[0];
            float qr[R], qi[R], br[R], bi[R];
#pragma unroll
            for (int w = 0; w < (R + 1) / 2; ++w) {
                const float4 a = rj[qw0 + w];
                const float4 g = rj[gw0 + w];
                qr[2 * w] = a.x;
                qi[2 * w] = a.y;
                br[2 * w] = g.x;
                bi[2 * w] = g.y;
                if (2 * w + 1 < R) {
                    qr[2 * w + 1] = a.z;
                    qi[2 * w + 1] = a.w;
                    br[2 * w + 1] = g.z;
                    bi[2 * w + 1] = g.w;
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float dx = ps.x - tx[k], dy = ps.y - ty[k], dz = ps.z - tz[k];
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
                float gr = inv * cs, gi = inv * sn;      // 4 pi G
                if (CHECK) {
                    gr = me ? 0.f : gr;
                    gi = me ? 0.f : gi;
                }
                // B = 4 pi dG/dr = G (i k - 1/r)
                const float Br = fmaf(-gr, inv, -kk * gi);
                const float Bi = fmaf(-gi, inv, kk * gr);
                float ar = 0.f, ai = 0.f;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    // grad_q += conj(G) gbar_j
                    p[k][2 * q] = fmaf(gr, br[q], fmaf(gi, bi[q], p[k][2 * q]));
                    p[k][2 * q + 1] = fmaf(gr, bi[q], fmaf(-gi, br[q], p[k][2 * q + 1]));
                    // A = conj(gbar_k) q_j + conj(gbar_j) q_k
                    ar = fmaf(tbr[k][q], qr[q], fmaf(tbi[k][q], qi[q], fmaf(br[q], tqr[k][q], fmaf(bi[q], tqi[k][q], ar))));
                    ai = fmaf(tbr[k][q], qi[q], fmaf(-tbi[k][q], qr[q], fmaf(br[q], tqi[k][q], fmaf(-bi[q], tqr[k][q], ai))));
                }
                // grad_x += Re(A B) (x_k - x_j)/r = -Re(A B) inv d
                const float cf = -(ar * Br - ai * Bi) * inv;
                p[k][2 * R + 0] = fmaf(cf, dx, p[k][2 * R + 0]);
                p[k][2 * R + 1] = fmaf(cf, dy, p[k][2 * R + 1]);
                p[k][2 * R + 2] = fmaf(cf, dz, p[k][2 * R + 2]);
            }
        }
    }

    __device__ __forceinline__ void tile(const float4* sm, int cnt, int rec0, bool chk) {
        if (chk) body<true>(sm, cnt, rec0);
        else body<false>(sm, cnt, rec0);
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                kahan_add(s[k][o], c[k][o], p[k][o]);
                p[k][o] = 0.f;
            }
    }

    __device__ __forceinline__ void store_partial(float* dst, int lane) const {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < NO; ++o) dst[(k * NO + o) * 32 + lane] = s[k][o] - c[k][o];
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                s[k][o] -= c[k][o];
                c[k][o] = 0.f;
            }
    }
    __device__ __forceinline__ void add_partial(const float* src, int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < NO; ++o) s[k][o] += src[(k * NO + o) * 32 + lane];
    }

    __device__ __forceinline__ void end(int lane) {
        const float inv4pi = 0.0795774715459476678844418816862571882f;  // 1 / (4 pi)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt) {
                const int64_t o = perm[tbase + l];
                if (grad_q)
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        grad_q[(int64_t)(r0 + q) * n + o] = make_float2((s[k][2 * q] - c[k][2 * q]) * inv4pi,
                                                                        (s[k][2 * q + 1] - c[k][2 * q + 1]) * inv4pi);
                if (grad_x)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float v = (s[k][2 * R + a] - c[k][2 * R + a]) * inv4pi;
                        grad_x[3 * o + a] = accumulate_x ? grad_x[3 * o + a] + v : v;
                    }
            }
        }
    }
};

template <int K, int G, int R, bool PRECISE>
__global__ void __launch_bounds__(kLoopThreads, 2)
    k_helmholtz_adjoint(LoopArgs a, const int32_t* __restrict__ perm, float kk, int qw0, int gw0, int64_t n, int r0,
                        int accumulate_x, float2* __restrict__ grad_q, float* __restrict__ grad_x) {
    pdl_wait();
    HelmAdjOp<K, R, PRECISE> op;
    op.rec = a.rec;
    op.perm = perm;
    op.kk = kk;
    op.words = a.words;
    op.qw0 = qw0;
    op.gw0 = gw0;
    op.n = n;
    op.r0 = r0;
    op.accumulate_x = accumulate_x != 0;
    op.grad_q = grad_q;
    op.grad_x = grad_x;
    warp_item_loop<K, G>(a, op);
}

template <int G, int R, bool PRECISE>
static int launch_hadj(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, bool accumulate,
                       float2* grad_q, float* grad_x, cudaStream_t s) {
    auto kern = k_helmholtz_adjoint<1, G, R, PRECISE>;
    const size_t smem = loop_smem_bytes(a.tile, a.words, HelmAdjOp<1, R, PRECISE>::kOuts, G);
    P2P_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0) {
        P2P_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
        if (per_sm < 1) per_sm = 1;
    }
    const int qw0 = 1 + r0 / 2;
    const int gw0 = 1 + (p->nrhs + 1) / 2 + r0 / 2;
    P2P_CUDA_TRY(launch_pdl(kern, num_sms() * per_sm, kLoopThreads, smem, s, a, perm, kk, qw0, gw0, p->n, r0, accumulate ? 1 : 0, grad_q,
                                                        grad_x));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

template <int G, bool PRECISE>
static int hadj_r(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, bool acc,
                  float2* gq, float* gx, cudaStream_t s) {
    switch (R) {
        case 1: return launch_hadj<G, 1, PRECISE>(p, a, perm, kk, r0, acc, gq, gx, s);
        case 2: return launch_hadj<G, 2, PRECISE>(p, a, perm, kk, r0, acc, gq, gx, s);
        case 4: return launch_hadj<G, 4, PRECISE>(p, a, perm, kk, r0, acc, gq, gx, s);
        case 8: return launch_hadj<G, 8, PRECISE>(p, a, perm, kk, r0, acc, gq, gx, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

int launch_helmholtz_adjoint_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float k, bool precise,
                                    float2* grad_q, float* grad_x, cudaStream_t s) {
    int r0 = 0;
    while (r0 < p->nrhs) {
        const int left = p->nrhs - r0;
        const int R = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        int st0 = fill32(&a.hdr->work_ctr, 0u, 1, s);
        if (st0) return st0;
        const bool acc = r0 > 0;
        int st;
        if (p->group >= 2)
            st = precise ? hadj_r<4, true>(p, a, perm, k, r0, R, acc, grad_q, grad_x, s)
                         : hadj_r<4, false>(p, a, perm, k, r0, R, acc, grad_q, grad_x, s);
        else
            st = precise ? hadj_r<1, true>(p, a, perm, k, r0, R, acc, grad_q, grad_x, s)
                         : hadj_r<1, false>(p, a, perm, k, r0, R, acc, grad_q, grad_x, s);
        if (st) return st;
        r0 += R;
    }
    return P2P_OK;
}

// ---------------------------------------------------------------------------
// gravity: grad_m and grad_x together
// ---------------------------------------------------------------------------
template <int K>
struct GravAdjOp {
    static constexpr int NO = 4;                 // grad_m, grad_x (3)
    static constexpr int kOuts = NO * K;
    static constexpr bool kPartial = false;   // adjoints are target-owned only
    static constexpr int kMutFloats = 0;

    const float4* __restrict__ rec;
    const int32_t* __restrict__ perm;
    float eps2;
    float* __restrict__ grad_m;
    float* __restrict__ grad_x;

    float tx[K], ty[K], tz[K], tm[K], tgp[K], tga[K][3];
    int self[K];
    float s[K][NO], c[K][NO], p[K][NO];
    int tbase, nt;

    __device__ __forceinline__ void begin(int tb, int ntg, int sw_lo, int lane) {
        tbase = tb;
        nt = ntg;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            const bool v = l < nt;
            const float4 a = v ? rec[2 * (int64_t)(tb + l)] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 g = v ? rec[2 * (int64_t)(tb + l) + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            tx[k] = a.x;
            ty[k] = a.y;
            tz[k] = a.z;
            tm[k] = a.w;
            tgp[k] = g.x;
            tga[k][0] = g.y;
            tga[k][1] = g.z;
            tga[k][2] = g.w;
            self[k] = v ? sw_lo + l : -1;
#pragma unroll
            for (int o = 0; o < NO; ++o) s[k][o] = c[k][o] = p[k][o] = 0.f;
        }
    }

    __device__ __forceinline__ void set_shift(float sx, float sy, float sz) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            const float4 r = rec[2 * (int64_t)(tbase + (l < nt ? l : 0))];
            tx[k] = r.x - sx;
            ty[k] = r.y - sy;
            tz[k] = r.z - sz;
        }
    }

    template <bool CHECK>
    __device__ __forceinline__ void body(const float4* __restrict__ sm, int cnt, int rec0) {
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const float4 a = sm[2 * j];
            const float4 g = sm[2 * j + 1];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float dx = a.x - tx[k], dy = a.y - ty[k], dz = a.z - tz[k];
                float h2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                float mj = a.w, gpj = g.x, gax = g.y, gay = g.z, gaz = g.w;
                if (CHECK) {
                    const bool me = (rec0 + j) == self[k];
                    h2 = me ? 1.f : h2;
                    mj = me ? 0.f : mj;
                    gpj = me ? 0.f : gpj;
                    gax = me ? 0.f : gax;
                    gay = me ? 0.f : gay;
                    gaz = me ? 0.f : gaz;
                }
                const float h1 = rsqrt_approx(h2);
                const float hi2 = h1 * h1;
                const float h3 = h1 * hi2;
                const float h5 = h3 * hi2;
                const float gad = fmaf(gax, dx, fmaf(gay, dy, gaz * dz));
                p[k][0] = fmaf(-gpj, h1, fmaf(-gad, h3, p[k][0]));
                const float s1 = fmaf(tgp[k], mj, gpj * tm[k]);
                const float vx = fmaf(tm[k], gax, -mj * tga[k][0]);
                const float vy = fmaf(tm[k], gay, -mj * tga[k][1]);
                const float vz = fmaf(tm[k], gaz, -mj * tga[k][2]);
                const float dv = fmaf(dx, vx, fmaf(dy, vy, dz * vz));
                const float t = fmaf(h3, s1, 3.f * h5 * dv);
                p[k][1] = fmaf(h3, vx, fmaf(-t, dx, p[k][1]));
                p[k][2] = fmaf(h3, vy, fmaf(-t, dy, p[k][2]));
                p[k][3] = fmaf(h3, vz, fmaf(-t, dz, p[k][3]));
            }
        }
    }

    __device__ __forceinline__ void tile(const float4* sm, int cnt, int rec0, bool chk) {
        if (chk) body<true>(sm, cnt, rec0);
        else body<false>(sm, cnt, rec0);
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                kahan_add(s[k][o], c[k][o], p[k][o]);
                p[k][o] = 0.f;
            }
    }
    __device__ __forceinline__ void store_partial(float* dst, int lane) const {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < NO; ++o) dst[(k * NO + o) * 32 + lane] = s[k][o] - c[k][o];
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                s[k][o] -= c[k][o];
                c[k][o] = 0.f;
            }
    }
    __device__ __forceinline__ void add_partial(const float* src, int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 0; o < NO; ++o) s[k][o] += src[(k * NO + o) * 32 + lane];
    }
    __device__ __forceinline__ void end(int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            if (l < nt) {
                const int64_t o = perm[tbase + l];
                if (grad_m) grad_m[o] = s[k][0] - c[k][0];
                if (grad_x)
#pragma unroll
                    for (int a = 0; a < 3; ++a) grad_x[3 * o + a] = s[k][1 + a] - c[k][1 + a];
            }
        }
    }
};

template <int K, int G>
__global__ void __launch_bounds__(kLoopThreads, 4)
    k_gravity_adjoint(LoopArgs a, const int32_t* __restrict__ perm, float eps2, float* __restrict__ grad_m,
                      float* __restrict__ grad_x) {
    pdl_wait();
    GravAdjOp<K> op;
    op.rec = a.rec;
    op.perm = perm;
    op.eps2 = eps2;
    op.grad_m = grad_m;
    op.grad_x = grad_x;
    warp_item_loop<K, G>(a, op);
}

template <int K, int G>
static int launch_gadj(const Plan* p, const LoopArgs& a, const int32_t* perm, float eps2, float* gm, float* gx,
                       cudaStream_t s) {
    auto kern = k_gravity_adjoint<K, G>;
    const size_t smem = loop_smem_bytes(a.tile, a.words, GravAdjOp<K>::kOuts, G);
    P2P_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0) {
        P2P_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
        if (per_sm < 1) per_sm = 1;
    }
    P2P_CUDA_TRY(launch_pdl(kern, num_sms() * per_sm, kLoopThreads, smem, s, a, perm, eps2, gm, gx));
    P2P_LAUNCH_CHECK();
    return P2P_OK;
}

int gravity_adjoint_targets_per_lane(const Plan* p) { return p->tpl >= 2 ? 2 : 1; }

int launch_gravity_adjoint_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float eps, float* grad_m,
                                  float* grad_x, cudaStream_t s) {
    const float eps2 = eps * eps;
    const int K = gravity_adjoint_targets_per_lane(p);
    if (p->group >= 2)
        return K == 2 ? launch_gadj<2, 4>(p, a, perm, eps2, grad_m, grad_x, s)
                      : launch_gadj<1, 4>(p, a, perm, eps2, grad_m, grad_x, s);
    return K == 2 ? launch_gadj<2, 1>(p, a, perm, eps2, grad_m, grad_x, s)
                  : launch_gadj<1, 1>(p, a, perm, eps2, grad_m, grad_x, s);
}

}  // namespace p2p
