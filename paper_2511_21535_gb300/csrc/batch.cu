// Batched near field: many independent instances (uneven grid sizes and box
// occupancies) and several right-hand sides per instance in ONE persistent
// kernel launch, captured in a CUDA graph.
//
// The paper's PhotoNs port suffers from many small launches (Section 5.2:
// one local, >= 1 remote and 27 periodic launches per iteration; batches of
// ~20,000 tasks, Section 5.2.3 item 4).  Here each instance's tree is built
// once (the geometry is fixed across solver iterations, as in the DBIM loop of
// Section 5.1) and merged on the device into one combined box structure with
// offsets; one work list ordered longest-first across all instances then
// drives one persistent kernel.
//
// A forward + adjoint pair (u = P q and g = conj(P) y, the two products of a
// BiCG-type iteration) runs as one operator with 2R right-hand sides
// [q ; conj(y)], since conj(P) y = conj(P conj(y)); the epilogue writes the
// second half conjugated.
#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"
#include "nvtx_range.cuh"
#include "p2p_loop.cuh"

namespace p2p {

struct Batch {
    int kind;
    int nrhs_in;                      // RHS per instance given by the caller
    int pair;                         // forward + adjoint
    int I;
    std::vector<int64_t> n, off;      // particles per instance and prefix offsets (off[I] = N)
    std::vector<int> level;
    std::vector<float> lo, edge;
    int64_t N;
    Plan tmp;                         // one instance's tree, sized for the largest instance
    Plan comb;                        // all instances
    bool red_alloc;                   // the combined workspace holds redundant streams
    size_t tmp_off, comb_off, total;
    int built;
    cudaStream_t cap_stream;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int64_t graph_launches;
};

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__global__ void k_batch_merge(const int32_t* __restrict__ perm_i, const int32_t* __restrict__ bs_i,
                              const int32_t* __restrict__ ns_i, const int32_t* __restrict__ ni_i, int64_t n_i,
                              int32_t B_i, int32_t E_i, int32_t P, int32_t Boff, int32_t Eoff,
                              int32_t* __restrict__ perm, int32_t* __restrict__ bs, int32_t* __restrict__ ns,
                              int32_t* __restrict__ ni) {
    pdl_wait();
    pdl_release();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t m = std::max<int64_t>(n_i, std::max<int64_t>(B_i, E_i));
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += stride) {
        if (t < n_i) perm[P + t] = P + perm_i[t];
        if (t < B_i) {
            bs[Boff + t] = P + bs_i[t];
            ns[Boff + t] = Eoff + ns_i[t];
        }
        if (t < E_i) ni[Eoff + t] = Boff + ni_i[t];
    }
}

__global__ void k_batch_finish(Header* hdr, int32_t* bs, int32_t* ns, int32_t B, int32_t E, int32_t N) {
    pdl_wait();
    pdl_release();
    bs[B] = N;
    ns[B] = E;
    hdr->n_boxes = B;
    hdr->n_nbr = E;
}

}  // namespace p2p

using namespace p2p;

struct p2p_batch {
    Batch b;
};

static int batch_ws(const Batch& b, void* ws, size_t bytes) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || bytes < b.total) return P2P_ERR_WORKSPACE;
    return P2P_OK;
}

static int batch_run(Batch& b, float k, const float* pos, const void* q, const void* y, void* u, void* g, void* ws,
                     cudaStream_t s) {
    void* cws = static_cast<char*>(ws) + b.comb_off;
    Plan* p = &b.comb;
    ev_begin(p, P2P_PHASE_RESTRUCTURE, s);
    int st = restructure(p, pos, q, cws, s, b.pair ? y : nullptr);
    if (st) return st;
    ev_end(p, P2P_PHASE_RESTRUCTURE, s);
    ev_begin(p, P2P_PHASE_OPERATOR, s);
    st = build_items(p, cws, 32 * helmholtz_targets_per_lane(p, k), s);
    if (st) return st;
    ev_begin(p, P2P_PHASE_KERNEL, s);
    st = launch_helmholtz_kernel(p, loop_args(p, cws, p->rec_words), at<int32_t>(cws, p->L.perm), k,
                                 HelmOut{static_cast<float2*>(u), static_cast<float2*>(g), p->split}, s);
    if (st) return st;
    ev_end(p, P2P_PHASE_KERNEL, s);
    ev_end(p, P2P_PHASE_OPERATOR, s);
    return P2P_OK;
}

static void batch_events_destroy(Batch& b) {
    for (int ph = 0; ph < P2P_PHASE_COUNT; ++ph)
        for (int e = 0; e < 2; ++e)
            if (b.comb.ev[ph][e]) {
                cudaEventDestroy(b.comb.ev[ph][e]);
                b.comb.ev[ph][e] = nullptr;
            }
}

extern "C" {

int p2p_batch_create(p2p_batch** out, int kind, int n_instances, const int64_t* n, const int* level, const float* lo,
                     const float* edge, int nrhs, int pair, int layout, unsigned flags) {
    if (!out) return P2P_ERR_INVALID_ARG;
    *out = nullptr;
    if (kind != P2P_HELMHOLTZ) return P2P_ERR_UNSUPPORTED;
    if (n_instances < 1 || !n || !level || !lo || !edge) return P2P_ERR_INVALID_ARG;
    if (layout != P2P_LAYOUT_INDIRECT && layout != P2P_LAYOUT_REDUNDANT && layout != P2P_LAYOUT_AUTO)
        return P2P_ERR_INVALID_ARG;
    if (flags & ~(P2P_PLAN_PLAIN_FP32 | P2P_PLAN_TIMING)) return P2P_ERR_INVALID_ARG;
    const int total_rhs = pair ? 2 * nrhs : nrhs;
    if (nrhs < 1 || total_rhs > P2P_MAX_NRHS) return P2P_ERR_INVALID_ARG;
    p2p_batch* h = host_alloc_should_fail() ? nullptr : new (std::nothrow) p2p_batch;
    if (!h) return P2P_ERR_OOM;
    Batch& b = h->b;
    b.kind = kind;
    b.nrhs_in = nrhs;
    b.pair = pair ? 1 : 0;
    b.I = n_instances;
    b.n.assign(n, n + n_instances);
    b.level.assign(level, level + n_instances);
    b.lo.assign(lo, lo + 3 * n_instances);
    b.edge.assign(edge, edge + n_instances);
    b.off.resize(n_instances + 1);
    b.off[0] = 0;
    int64_t nmax = 0;
    int lmax = 1, imax = 0;
    float rmax = 0.f;
    for (int i = 0; i < n_instances; ++i) {
        if (b.n[i] < 1 || b.level[i] < 1 || b.level[i] > P2P_MAX_LEVEL || !(b.edge[i] > 0.f)) {
            delete h;
            return P2P_ERR_INVALID_ARG;
        }
        b.off[i + 1] = b.off[i] + b.n[i];
        if (b.n[i] > nmax) {
            nmax = b.n[i];
            imax = i;
        }
        lmax = std::max(lmax, b.level[i]);
        rmax = std::max(rmax, 2.0f * (b.edge[i] / (float)(1 << b.level[i])) * 1.7320508f);
    }
    b.N = b.off[n_instances];
    if (b.N > P2P_MAX_N) {
        delete h;
        return P2P_ERR_INVALID_ARG;
    }
    int st = plan_init(&b.tmp, kind, nmax, lmax, &b.lo[3 * imax], b.edge[imax], 1, P2P_LAYOUT_INDIRECT, 0);
    if (st) {
        delete h;
        return st;
    }
    const float zero[3] = {0.f, 0.f, 0.f};
    b.red_alloc = layout != P2P_LAYOUT_INDIRECT;
    st = plan_init(&b.comb, kind, b.N, P2P_MAX_LEVEL, zero, 1.0f, total_rhs,
                   b.red_alloc ? P2P_LAYOUT_REDUNDANT : P2P_LAYOUT_INDIRECT, flags);
    if (st) {
        delete h;
        return st;
    }
    b.comb.split = nrhs;
    b.comb.rmax = rmax;
    b.comb.timing = (flags & P2P_PLAN_TIMING) ? 1 : 0;
    for (int ph = 0; ph < P2P_PHASE_COUNT; ++ph) {
        b.comb.ev_valid[ph] = 0;
        b.comb.ev[ph][0] = b.comb.ev[ph][1] = nullptr;
    }
    if (b.comb.timing)
        for (int ph = 0; ph < P2P_PHASE_COUNT; ++ph)
            for (int e = 0; e < 2; ++e)
                if (cudaEventCreate(&b.comb.ev[ph][e]) != cudaSuccess) {
                    batch_events_destroy(b);
                    delete h;
                    return P2P_ERR_CUDA;
                }
    if (layout == P2P_LAYOUT_AUTO) b.comb.layout = P2P_LAYOUT_INDIRECT;  // until the autotuner decides
    b.tmp_off = 0;
    b.comb_off = (b.tmp.L.total + 255) / 256 * 256;
    b.total = b.comb_off + b.comb.L.total;
    b.built = 0;
    b.cap_stream = nullptr;
    b.graph = nullptr;
    b.exec = nullptr;
    b.graph_launches = 0;
    *out = h;
    return P2P_OK;
}

int p2p_batch_destroy(p2p_batch* h) {
    if (!h) return P2P_OK;
    Batch& b = h->b;
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    if (b.cap_stream) cudaStreamDestroy(b.cap_stream);
    batch_events_destroy(b);
    delete h;
    return P2P_OK;
}

int p2p_batch_workspace_bytes(const p2p_batch* h, size_t* bytes) {
    if (!h || !bytes) return P2P_ERR_INVALID_ARG;
    *bytes = h->b.total;
    return P2P_OK;
}

int p2p_batch_build(p2p_batch* h, const float* pos, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("p2p_batch_build");
    if (!h || !pos || (reinterpret_cast<uintptr_t>(pos) & 3u)) return P2P_ERR_INVALID_ARG;
    Batch& b = h->b;
    int st = batch_ws(b, ws, ws_bytes);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* tws = static_cast<char*>(ws) + b.tmp_off;
    void* cws = static_cast<char*>(ws) + b.comb_off;
    int32_t Boff = 0, Eoff = 0;
    for (int i = 0; i < b.I; ++i) {
        Plan pi = b.tmp;   // same workspace layout, this instance's shape
        pi.n = b.n[i];
        pi.level = b.level[i];
        for (int a = 0; a < 3; ++a) pi.lo[a] = b.lo[3 * i + a];
        pi.edge = b.edge[i];
        pi.scale = (float)(1 << pi.level) / pi.edge;
        pi.sort_tiles = (int)((pi.n + 2047) / 2048);
        const int64_t boxes = (int64_t)1 << (3 * pi.level);
        pi.box_cap = pi.n < boxes ? pi.n : boxes;
        pi.use_table = b.tmp.use_table && pi.level <= 8;
        st = tree_build(&pi, pos + 3 * b.off[i], tws, s);
        if (st) return st;
        Header hdr;
        P2P_CUDA_TRY(cudaMemcpyAsync(&hdr, static_cast<char*>(tws) + pi.L.header, sizeof(Header),
                                     cudaMemcpyDeviceToHost, s));
        P2P_CUDA_TRY(cudaStreamSynchronize(s));
        if (hdr.flags & P2P_FLAG_DOMAIN) return P2P_ERR_DOMAIN;
        const int64_t m = std::max<int64_t>(pi.n, std::max<int64_t>(hdr.n_boxes, hdr.n_nbr));
        P2P_CUDA_TRY(launch_pdl(k_batch_merge, std::min<unsigned>(blocks_for(m, 256), (unsigned)num_sms() * 8), 256, 0, s, 
            at<int32_t>(tws, pi.L.perm), at<int32_t>(tws, pi.L.box_start), at<int32_t>(tws, pi.L.nbr_start),
            at<int32_t>(tws, pi.L.nbr_idx), pi.n, hdr.n_boxes, hdr.n_nbr, (int32_t)b.off[i], Boff, Eoff,
            at<int32_t>(cws, b.comb.L.perm), at<int32_t>(cws, b.comb.L.box_start), at<int32_t>(cws, b.comb.L.nbr_start),
            at<int32_t>(cws, b.comb.L.nbr_idx)));
        P2P_LAUNCH_CHECK();
        Boff += hdr.n_boxes;
        Eoff += hdr.n_nbr;
    }
    {
        int st0 = fill32(at<Header>(cws, b.comb.L.header), 0u, kOpSectionOffset / 4, s);
        if (st0) return st0;
    }
    P2P_CUDA_TRY(launch_pdl(k_batch_finish, 1, 1, 0, s, at<Header>(cws, b.comb.L.header), at<int32_t>(cws, b.comb.L.box_start),
                                   at<int32_t>(cws, b.comb.L.nbr_start), Boff, Eoff, (int32_t)b.N));
    P2P_LAUNCH_CHECK();
    P2P_CUDA_TRY(cudaStreamSynchronize(s));
    b.comb.tree_ready = 1;
    b.built = 1;
    return P2P_OK;
}

int p2p_batch_set_tuning(p2p_batch* h, int layout, int targets_per_lane, int tile, int ctas_per_sm,
                         int warps_per_item) {
    if (!h) return P2P_ERR_INVALID_ARG;
    Batch& b = h->b;
    if (layout != P2P_LAYOUT_INDIRECT && layout != P2P_LAYOUT_REDUNDANT) return P2P_ERR_INVALID_ARG;
    if (layout == P2P_LAYOUT_REDUNDANT && !b.red_alloc) return P2P_ERR_UNSUPPORTED;
    const bool g_ok = warps_per_item == 1 || warps_per_item == 2 || warps_per_item == 4;
    if ((targets_per_lane != 1 && targets_per_lane != 2) || !g_ok || (tile != 32 && tile != 64) ||
        ctas_per_sm < 0 || ctas_per_sm > 32)
        return P2P_ERR_INVALID_ARG;
    b.comb.layout = layout;
    b.comb.tpl = targets_per_lane;
    b.comb.tile = tile;
    b.comb.ctas_per_sm = ctas_per_sm;
    b.comb.group = warps_per_item;
    return P2P_OK;
}

int p2p_batch_run(p2p_batch* h, float k, const float* pos, const void* q, const void* y, void* u, void* g, void* ws,
                  size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("p2p_batch_run");
    if (!h || !pos || !q || !u) return P2P_ERR_INVALID_ARG;
    Batch& b = h->b;
    if (b.pair && (!y || !g)) return P2P_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(y) |
         reinterpret_cast<uintptr_t>(g)) & 7u)
        return P2P_ERR_INVALID_ARG;
    if (!(k == k) || !(fabsf(k) < 1.0e30f)) return P2P_ERR_INVALID_ARG;
    int st = batch_ws(b, ws, ws_bytes);
    if (st) return st;
    if (!b.built) return P2P_ERR_STATE;
    return batch_run(b, k, pos, q, y, u, g, ws, static_cast<cudaStream_t>(stream));
}

int p2p_batch_autotune(p2p_batch* h, float k, const float* pos, const void* q, const void* y, void* u, void* g,
                       void* ws, size_t ws_bytes, void* stream, int* best, float* best_ms) {
    NvtxRange nvtx_range("p2p_batch_autotune");
    if (!h || !best || !best_ms) return P2P_ERR_INVALID_ARG;
    Batch& b = h->b;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    P2P_CUDA_TRY(cudaEventCreate(&e0));
    P2P_CUDA_TRY(cudaEventCreate(&e1));
    float bms = 1e30f;
    int bl = b.comb.layout, bt = b.comb.tpl, bs = b.comb.tile, bg = b.comb.group;
    int rc = P2P_OK;
    const int layouts[2] = {P2P_LAYOUT_INDIRECT, P2P_LAYOUT_REDUNDANT};
    for (int li = 0; li < (b.red_alloc ? 2 : 1) && rc == P2P_OK; ++li)
        for (int tpl = 1; tpl <= 2 && rc == P2P_OK; ++tpl)
            for (int tile = 32; tile <= 64 && rc == P2P_OK; tile *= 2)
                for (int grp = 1; grp <= 4 && rc == P2P_OK; grp *= 2) {
                    p2p_batch_set_tuning(h, layouts[li], tpl, tile, 0, grp);
                    rc = p2p_batch_run(h, k, pos, q, y, u, g, ws, ws_bytes, stream);  // warm-up
                    if (rc) break;
                    float tot = 0.f;
                    for (int rep = 0; rep < 2 && rc == P2P_OK; ++rep) {
                        cudaEventRecord(e0, s);
                        rc = p2p_batch_run(h, k, pos, q, y, u, g, ws, ws_bytes, stream);
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) rc = P2P_ERR_CUDA;
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        tot += ms;
                    }
                    if (rc == P2P_OK && tot / 2 < bms) {
                        bms = tot / 2;
                        bl = layouts[li];
                        bt = tpl;
                        bs = tile;
                        bg = grp;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    p2p_batch_set_tuning(h, bl, bt, bs, 0, bg);
    best[0] = bl;
    best[1] = bt;
    best[2] = bs;
    best[3] = 0;
    best[4] = bg;
    *best_ms = bms;
    return P2P_OK;
}

int p2p_batch_capture(p2p_batch* h, float k, const float* pos, const void* q, const void* y, void* u, void* g, void* ws,
                      size_t ws_bytes) {
    NvtxRange nvtx_range("p2p_batch_capture");
    if (!h || !pos || !q || !u) return P2P_ERR_INVALID_ARG;
    Batch& b = h->b;
    if (b.pair && (!y || !g)) return P2P_ERR_INVALID_ARG;
    int st = batch_ws(b, ws, ws_bytes);
    if (st) return st;
    if (!b.built) return P2P_ERR_STATE;
    if (!b.cap_stream) P2P_CUDA_TRY(cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking));
    if (b.exec) {
        cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
    }
    if (b.graph) {
        cudaGraphDestroy(b.graph);
        b.graph = nullptr;
    }
    // one eager run on the capture stream sets kernel attributes before capture
    st = batch_run(b, k, pos, q, y, u, g, ws, b.cap_stream);
    if (st) return st;
    P2P_CUDA_TRY(cudaStreamSynchronize(b.cap_stream));
    const long long l0 = p2p_launch_count();
    P2P_CUDA_TRY(cudaStreamBeginCapture(b.cap_stream, cudaStreamCaptureModeThreadLocal));
    st = batch_run(b, k, pos, q, y, u, g, ws, b.cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b.cap_stream, &graph);
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess || !graph) return P2P_ERR_CUDA;
    b.graph_launches = p2p_launch_count() - l0;
    b.graph = graph;
    P2P_CUDA_TRY(cudaGraphInstantiate(&b.exec, b.graph, 0));
    return P2P_OK;
}

int p2p_batch_launch(p2p_batch* h, void* stream) {
    NvtxRange nvtx_range("p2p_batch_launch");
    if (!h) return P2P_ERR_INVALID_ARG;
    Batch& b = h->b;
    if (!b.exec) return P2P_ERR_STATE;
    P2P_CUDA_TRY(cudaGraphLaunch(b.exec, static_cast<cudaStream_t>(stream)));
    count_launch((int)b.graph_launches);
    return P2P_OK;
}

int p2p_batch_timing(p2p_batch* h, float* ms_out) {
    if (!h || !ms_out) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->b.comb;
    for (int ph = 0; ph < P2P_PHASE_COUNT; ++ph) {
        ms_out[ph] = -1.0f;
        if (!p->timing || !p->ev_valid[ph]) continue;
        if (cudaEventSynchronize(p->ev[ph][1]) != cudaSuccess) return P2P_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev[ph][0], p->ev[ph][1]) != cudaSuccess) return P2P_ERR_CUDA;
        ms_out[ph] = ms;
    }
    return P2P_OK;
}

int p2p_batch_counters(const p2p_batch* h, const void* ws, int64_t* out, void* stream) {
    if (!h || !ws || !out) return P2P_ERR_INVALID_ARG;
    const Batch& b = h->b;
    Header hdr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&hdr, static_cast<const char*>(ws) + b.comb_off + b.comb.L.header, sizeof(Header),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return P2P_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return P2P_ERR_CUDA;
    out[P2P_CTR_N_BOXES] = hdr.n_boxes;
    out[P2P_CTR_N_NBR] = hdr.n_nbr;
    out[P2P_CTR_FLAGS] = hdr.flags;
    out[P2P_CTR_TOTAL_SRC] = hdr.total_src;
    out[P2P_CTR_PAIRS] = (int64_t)hdr.pairs_nS - b.N;
    out[P2P_CTR_N_ITEMS] = hdr.n_items;
    out[P2P_CTR_EVALS] = (int64_t)hdr.evals_nS - b.N;
    if (hdr.flags & P2P_FLAG_BOUNDS) return P2P_ERR_BOUNDS;
    if (hdr.flags & P2P_FLAG_TIMEOUT) return P2P_ERR_TIMEOUT;
    return P2P_OK;
}

}  // extern "C"
