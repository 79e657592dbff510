// Helmholtz P2P kernel variants used outside the default path: plain FP32
// accumulation (for the compensated-vs-plain error comparison) and the
// accurate sine/cosine (large k r).  One target per lane.
#include "p2p_helmholtz.cuh"

namespace p2p {

template <int G, bool COMP, bool PRECISE>
static int var_g(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                 cudaStream_t s) {
    switch (R) {
        case 1: return launch_helm<1, G, 1, COMP, PRECISE>(p, a, perm, kk, r0, u, s);
        case 2: return launch_helm<1, G, 2, COMP, PRECISE>(p, a, perm, kk, r0, u, s);
        case 4: return launch_helm<1, G, 4, COMP, PRECISE>(p, a, perm, kk, r0, u, s);
        case 8: return launch_helm<1, G, 8, COMP, PRECISE>(p, a, perm, kk, r0, u, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

int launch_helm_plain(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                      cudaStream_t s) {
    return p->group >= 2 ? var_g<4, false, false>(p, a, perm, kk, r0, R, u, s)
                         : var_g<1, false, false>(p, a, perm, kk, r0, R, u, s);
}

int launch_helm_precise(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, HelmOut u,
                        cudaStream_t s) {
    const bool comp = !(p->flags & P2P_PLAN_PLAIN_FP32);
    if (p->group >= 2)
        return comp ? var_g<4, true, true>(p, a, perm, kk, r0, R, u, s) : var_g<4, false, true>(p, a, perm, kk, r0, R, u, s);
    return comp ? var_g<1, true, true>(p, a, perm, kk, r0, R, u, s) : var_g<1, false, true>(p, a, perm, kk, r0, R, u, s);
}

}  // namespace p2p
