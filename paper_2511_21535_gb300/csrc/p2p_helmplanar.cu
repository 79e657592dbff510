// Helmholtz P2P for plans of four or more right-hand sides (records with the
// right-hand sides planar per word): dispatch over targets per lane, warps
// per item, passes of 2, 4 or 8 right-hand sides and the kernel variants
// (compensated hardware sine/cosine; plain FP32 or the accurate sine/cosine
// with one target per lane, as for the other records).
#include "p2p_helmplanar.cuh"

namespace p2p {

template <int K, int G, bool COMP, bool PRECISE>
static int planar_r(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, int nval,
                    HelmOut u, cudaStream_t s) {
    switch (R) {
        case 2: return launch_helmplanar<K, G, 2, COMP, PRECISE>(p, a, perm, kk, r0, nval, u, s);
        case 4: return launch_helmplanar<K, G, 4, COMP, PRECISE>(p, a, perm, kk, r0, nval, u, s);
        case 8: return launch_helmplanar<K, G, 8, COMP, PRECISE>(p, a, perm, kk, r0, nval, u, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

int launch_helm_planar(const Plan* p, const LoopArgs& a, const int32_t* perm, float kk, int r0, int R, int nval,
                       bool comp, bool precise, HelmOut u, cudaStream_t s) {
    if (a.task_kind) return P2P_ERR_UNSUPPORTED;   // symmetric plans hold at most two right-hand sides
    if (!comp || precise) {   // one target per lane; one or four warps per item
        const bool g4 = p->group >= 2;
        if (!comp && precise)
            return g4 ? planar_r<1, 4, false, true>(p, a, perm, kk, r0, R, nval, u, s)
                      : planar_r<1, 1, false, true>(p, a, perm, kk, r0, R, nval, u, s);
        if (!comp)
            return g4 ? planar_r<1, 4, false, false>(p, a, perm, kk, r0, R, nval, u, s)
                      : planar_r<1, 1, false, false>(p, a, perm, kk, r0, R, nval, u, s);
        return g4 ? planar_r<1, 4, true, true>(p, a, perm, kk, r0, R, nval, u, s)
                  : planar_r<1, 1, true, true>(p, a, perm, kk, r0, R, nval, u, s);
    }
    const bool k2 = p->tpl >= 2;
    switch (p->group) {
        case 1: return k2 ? planar_r<2, 1, true, false>(p, a, perm, kk, r0, R, nval, u, s)
                          : planar_r<1, 1, true, false>(p, a, perm, kk, r0, R, nval, u, s);
        case 2: return k2 ? planar_r<2, 2, true, false>(p, a, perm, kk, r0, R, nval, u, s)
                          : planar_r<1, 2, true, false>(p, a, perm, kk, r0, R, nval, u, s);
        case 4: return k2 ? planar_r<2, 4, true, false>(p, a, perm, kk, r0, R, nval, u, s)
                          : planar_r<1, 4, true, false>(p, a, perm, kk, r0, R, nval, u, s);
        default: return P2P_ERR_INVALID_ARG;
    }
}

}  // namespace p2p
