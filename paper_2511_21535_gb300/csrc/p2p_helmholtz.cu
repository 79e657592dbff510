// Helmholtz P2P: dispatch over right-hand-side passes, and the fast
// (hardware sine/cosine, compensated) kernel variants.
#include "p2p_helm2d.cuh"
#include "p2p_helmholtz.cuh"
#include "p2p_helmsym.cuh"

namespace p2p {

template <int K, int G>
static int fast_kg(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                   cudaStream_t s) {
    const bool w2 = a.words == 2;   // records of one or two right-hand sides
    if (K == 2 && p->tpl == 4 && w2) {
        // four targets per lane in two source groups (items of 64 targets, as with two per lane)
        if (R == 1) return launch_helmtile<G, 1>(p, a, perm, kk, r0, u, s);
        if (R == 2) return launch_helmtile<G, 2>(p, a, perm, kk, r0, u, s);
    }
    switch (R) {
        case 1: return w2 ? launch_helm<K, G, 1, true, false, 2>(p, a, perm, kk, r0, u, s)
                          : launch_helm<K, G, 1, true, false>(p, a, perm, kk, r0, u, s);
        case 2: return w2 ? launch_helm<K, G, 2, true, false, 2>(p, a, perm, kk, r0, u, s)
                          : launch_helm<K, G, 2, true, false>(p, a, perm, kk, r0, u, s);
        case 4: return launch_helm<K, G, 4, true, false>(p, a, perm, kk, r0, u, s);
        case 8: return launch_helm<K, G, 8, true, false>(p, a, perm, kk, r0, u, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

// symmetric tasks and plans: items of 64 targets (a mutual task or box is one
// work item), one or two right-hand sides in two-word records
template <int G>
static int mutual_g(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                    cudaStream_t s) {
    if (p->tpl != 2 || a.words != 2) return P2P_ERR_UNSUPPORTED;
    switch (R) {   // four targets per lane, two source groups (measured best on GB300)
        case 1: return launch_helmsym<G, 1, 4>(p, a, perm, kk, r0, u, s);
        case 2: return launch_helmsym<G, 2, 4>(p, a, perm, kk, r0, u, s);
        default: return P2P_ERR_UNSUPPORTED;
    }
}

int launch_helm_fast(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                     cudaStream_t s) {
    if (a.task_kind) {
        switch (p->group) {
            case 1: return mutual_g<1>(p, a, perm, kk, r0, R, u, s);
            case 2: return mutual_g<2>(p, a, perm, kk, r0, R, u, s);
            case 4: return mutual_g<4>(p, a, perm, kk, r0, R, u, s);
            default: return P2P_ERR_INVALID_ARG;
        }
    }
    const int K = p->tpl >= 2 ? 2 : 1;
    switch (p->group) {
        case 1: return K == 2 ? fast_kg<2, 1>(p, a, perm, kk, r0, R, u, s) : fast_kg<1, 1>(p, a, perm, kk, r0, R, u, s);
        case 2: return K == 2 ? fast_kg<2, 2>(p, a, perm, kk, r0, R, u, s) : fast_kg<1, 2>(p, a, perm, kk, r0, R, u, s);
        case 4: return K == 2 ? fast_kg<2, 4>(p, a, perm, kk, r0, R, u, s) : fast_kg<1, 4>(p, a, perm, kk, r0, R, u, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

// Largest k * r over any pair of neighbouring boxes below which the hardware
// sine/cosine approximation is used (the parity tests measure its error over
// this range); beyond it the accurate library routine is used.
constexpr float kFastPhaseMax = 32.0f;

bool helmholtz_needs_precise(const Plan* p, float k) { return fabsf(k) * p->rmax > kFastPhaseMax; }

int helmholtz_targets_per_lane(const Plan* p, float k) {
    const bool comp = !(p->flags & P2P_PLAN_PLAIN_FP32);
    if (helmholtz_needs_precise(p, k) || !comp) return 1;   // the variant kernels hold one target per lane
    return p->tpl >= 2 ? 2 : 1;
}

int launch_helmholtz_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float k, HelmOut u,
                            cudaStream_t s) {
    const bool comp = !(p->flags & P2P_PLAN_PLAIN_FP32);
    const bool precise = helmholtz_needs_precise(p, k);
    const bool planar = helmholtz_planar(p);
    // passes of 8, 4, 2, 1 right-hand sides; every pass but the last starts at an even index
    // (planar records: 8, 4 or 2, the last pair of an odd count half empty)
    int r0 = 0;
    while (r0 < p->nrhs) {
        const int left = p->nrhs - r0;
        const int R = left >= 8 ? 8 : left >= 4 ? 4 : (left >= 2 || planar) ? 2 : 1;
        if (r0 > 0) {   // the first pass follows build_items, which zeroed the operator section
            const int st0 = fill32(&a.hdr->work_ctr, 0u, 1, s);
            if (st0) return st0;
        }
        // symmetric tasks run only in the compensated hardware-sin/cos kernel
        if (a.task_kind && (precise || !comp)) return P2P_ERR_UNSUPPORTED;
        int st = planar  ? launch_helm_planar(p, a, perm, k, r0, R, left < R ? left : R, comp, precise, u, s)
                 : precise ? launch_helm_precise(p, a, perm, k, r0, R, u, s)
                 : comp    ? launch_helm_fast(p, a, perm, k, r0, R, u, s)
                           : launch_helm_plain(p, a, perm, k, r0, R, u, s);
        if (st) return st;
        r0 += R;
    }
    return P2P_OK;
}

}  // namespace p2p
