// C ABI: plans, workspace layout, argument checks, phase timing.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <new>

#include "common.cuh"
#include "nvtx_range.cuh"
#include "p2p_loop.cuh"
#include "sort_scratch.cuh"

struct p2p_plan {
    p2p::Plan p;
};

namespace p2p {

static std::atomic<long long> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static std::atomic<int> g_fail_allocs{0};
bool host_alloc_should_fail() {
    int v = g_fail_allocs.load();
    while (v > 0) {
        if (g_fail_allocs.compare_exchange_weak(v, v - 1)) return true;
    }
    return false;
}

bool pdl_enabled() {
    static const bool on = [] {
        const char* v = getenv("P2P_NO_PDL");
        return !(v && v[0] == '1');
    }();
    return on;
}

static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void compute_layout(Plan* p) {
    Layout& L = p->L;
    const int64_t n = p->n;
    const int64_t bc = p->box_cap;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + (bytes ? bytes : 16), 256);
        return o;
    };
    L.header = take(kHeaderBytes);
    L.keys_a = take(n * 4);
    L.keys_b = take(n * 4);
    L.vals_a = take(n * 4);
    L.perm = take(n * 4);
    L.sorted_key = take(n * 4);
    L.hist = take(sort_scratch_bytes(p->sort_tiles));
    int64_t scan_max = n;
    const bool pt = is_pairtask(p->layout);
    if (pt && 27 * bc > scan_max) scan_max = 27 * bc;   // scans over neighbour entries
    L.scan_tmp = take(scan_scratch_bytes(scan_max));
    L.lookback = take((size_t)lb_regions(n, bc).words * 8);
    L.box_key = take(bc * 4);
    L.box_start = take((bc + 1) * 4);
    L.table = p->use_table ? take(((size_t)1 << (3 * p->level)) * 4) : 0;
    L.nbr_start = take((bc + 1) * 4);
    L.nbr_idx = take((size_t)27 * bc * 4);
    L.nbr_img = p->periodic ? take((size_t)27 * bc * 4) : 0;
    L.src = take((size_t)n * p->rec_alloc_words * 16);
    L.box_S = take((bc + 1) * 4);
    L.items = take((size_t)p->items_cap * 8);
    L.pattern = (p->kind == P2P_HELMHOLTZ) ? take((size_t)kPatternMaxEntries * 8) : 0;
    L.red_start = L.red_self = L.red_src = L.gather = L.heavy = 0;
    L.ent_box = L.pt_start = L.part_start = L.part = 0;
    L.task_kind = L.mirror = L.bslot = 0;
    if (p->layout == P2P_LAYOUT_REDUNDANT) {
        L.red_start = take((bc + 1) * 4);
        L.red_self = take(bc * 4);
        L.heavy = take(bc * 4);
    } else if (pt) {
        L.ent_box = take((size_t)27 * bc * 4);
        L.pt_start = take(((size_t)27 * bc + 1) * 4);
        L.part_start = take(((size_t)27 * bc + 1) * 4);
        L.part = take((size_t)p->part_cap * pairtask_part_floats(p->kind, p->nrhs) * 4);
        if (p->layout == P2P_LAYOUT_SYMMETRIC) {
            L.task_kind = take((size_t)27 * bc * 4);
            L.mirror = take((size_t)27 * bc * 4);
        }
    }
    if (p->sym) {   // symmetric evaluation on a target-owned layout
        L.task_kind = take((size_t)27 * bc * 4);
        L.mirror = take((size_t)27 * bc * 4);
        L.bslot = take(((size_t)27 * bc + 1) * 4);
        L.part = take((size_t)p->part_cap * pairtask_part_floats(p->kind, p->nrhs) * 4);
    }
    if (p->layout == P2P_LAYOUT_REDUNDANT || pt) {   // the per-box streams, or the task stream
        L.red_src = take((size_t)p->red_cap * p->rec_alloc_words * 16);
        L.gather = (p->flags & P2P_PLAN_GATHER_MAP) ? take((size_t)p->red_cap * 4) : 0;
    }
    L.io_pos = L.io_str = L.io_out = 0;
    if (p->flags & P2P_PLAN_HOST_IO) {
        const size_t per = (p->kind == P2P_GRAVITY) ? 4 : (size_t)8 * p->nrhs;   // strength bytes per particle
        L.io_pos = take((size_t)n * 12);
        L.io_str = take((size_t)n * per);
        L.io_out = take((size_t)n * ((p->kind == P2P_GRAVITY) ? 16 : per));   // gravity: phi, then acc
    }
    L.total = off;
}

int check_ws(const Plan* p, const void* ws, size_t ws_bytes) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < p->L.total) return P2P_ERR_WORKSPACE;
    return P2P_OK;
}

// Inside a stream capture the events become external event-record nodes, so
// a replayed graph still records them and their elapsed time can be read.
static void ev_record(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, s);
}
void ev_begin(Plan* p, int ph, cudaStream_t s) {
    if (p->timing) ev_record(p->ev[ph][0], s);
}
void ev_end(Plan* p, int ph, cudaStream_t s) {
    if (p->timing) {
        ev_record(p->ev[ph][1], s);
        p->ev_valid[ph] = 1;
    }
}

LoopArgs loop_args(const Plan* p, void* ws, int words) {
    const Layout& L = p->L;
    LoopArgs a{};   // every field not set below is null
    a.rec = at<float4>(ws, L.src);
    a.red = (p->layout == P2P_LAYOUT_REDUNDANT) ? at<float4>(ws, L.red_src) : nullptr;
    a.words = words;
    // wide records: halve the tile until a stage stays within ~2.5 KB (32 at least)
    int tile = p->tile;
    while (tile > 32 && words * tile > 160) tile = tile > 64 ? tile / 2 : 32;
    a.tile = tile;
    a.box_start = at<int32_t>(ws, L.box_start);
    a.nbr_start = at<int32_t>(ws, L.nbr_start);
    a.nbr_idx = at<int32_t>(ws, L.nbr_idx);
    a.red_start = (p->layout == P2P_LAYOUT_REDUNDANT) ? at<int32_t>(ws, L.red_start) : nullptr;
    a.red_self = (p->layout == P2P_LAYOUT_REDUNDANT) ? at<int32_t>(ws, L.red_self) : nullptr;
    a.items = at<int2>(ws, L.items);
    a.hdr = at<Header>(ws, L.header);
    // periodic images: the redundant and task streams carry shifted sources;
    // the indirect layout shifts the targets per neighbour range
    a.nbr_img = (p->periodic && p->layout == P2P_LAYOUT_INDIRECT) ? at<int32_t>(ws, L.nbr_img) : nullptr;
    a.edge = p->edge;
    a.rec_cap = p->n;
    a.red_cap = p->red_cap;
    a.items_cap = p->items_cap;
    a.box_cap = p->box_cap;
    a.n = p->n;
    a.ent_box = a.pt_start = a.part_start = a.task_kind = nullptr;
    a.part = nullptr;
    a.part_cap = 0;
    if (is_pairtask(p->layout)) {
        // targets and sources both come from the task stream
        a.rec = a.red = at<float4>(ws, L.red_src);
        a.rec_cap = p->red_cap;
        a.ent_box = at<int32_t>(ws, L.ent_box);
        a.pt_start = at<int32_t>(ws, L.pt_start);
        a.part_start = at<int32_t>(ws, L.part_start);
        a.part = at<float>(ws, L.part);
        a.part_cap = p->part_cap;
        if (p->layout == P2P_LAYOUT_SYMMETRIC) a.task_kind = at<int32_t>(ws, L.task_kind);
    }
    if (p->sym) {
        a.task_kind = at<int32_t>(ws, L.task_kind);
        a.bslot = at<int32_t>(ws, L.bslot);
        a.part = at<float>(ws, L.part);
        a.part_cap = p->part_cap;
    }
    return a;
}


int plan_init(Plan* p, int kind, int64_t n, int level, const float* lo, float edge, int nrhs, int layout,
              unsigned flags) {
    if (kind != P2P_GRAVITY && kind != P2P_HELMHOLTZ) return P2P_ERR_INVALID_ARG;
    if (n < 1 || n > P2P_MAX_N) return P2P_ERR_INVALID_ARG;
    if (level < 1 || level > P2P_MAX_LEVEL) return P2P_ERR_INVALID_ARG;
    if (!lo || !(edge > 0.0f) || !(edge < 3.0e38f)) return P2P_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(lo[a] == lo[a]) || lo[a] > 3.0e38f || lo[a] < -3.0e38f) return P2P_ERR_INVALID_ARG;
    if (layout != P2P_LAYOUT_INDIRECT && layout != P2P_LAYOUT_REDUNDANT && !is_pairtask(layout))
        return P2P_ERR_INVALID_ARG;
    if (is_pairtask(layout) && (n > P2P_MAX_N_PAIRTASK || (flags & P2P_PLAN_ADJOINT))) return P2P_ERR_INVALID_ARG;
    if (layout == P2P_LAYOUT_SYMMETRIC && kind == P2P_HELMHOLTZ && nrhs > 2) return P2P_ERR_INVALID_ARG;
    if (kind == P2P_GRAVITY && nrhs != 1) return P2P_ERR_INVALID_ARG;
    if (nrhs < 1 || nrhs > P2P_MAX_NRHS) return P2P_ERR_INVALID_ARG;
    if (flags & ~(P2P_PLAN_GATHER_MAP | P2P_PLAN_PLAIN_FP32 | P2P_PLAN_TIMING | P2P_PLAN_ADJOINT |
                  P2P_PLAN_PERIODIC | P2P_PLAN_SYMMETRIC | P2P_PLAN_HOST_IO))
        return P2P_ERR_INVALID_ARG;
    if ((flags & P2P_PLAN_SYMMETRIC) &&
        (is_pairtask(layout) || (flags & P2P_PLAN_ADJOINT) || (kind == P2P_HELMHOLTZ && nrhs > 2)))
        return P2P_ERR_INVALID_ARG;
    if ((flags & P2P_PLAN_PERIODIC) && level < 2) return P2P_ERR_INVALID_ARG;
    *p = Plan{};
    p->periodic = (flags & P2P_PLAN_PERIODIC) ? 1 : 0;
    p->sym = (flags & P2P_PLAN_SYMMETRIC) ? 1 : 0;
    p->kind = kind;
    p->n = n;
    p->level = level;
    for (int a = 0; a < 3; ++a) p->lo[a] = lo[a];
    p->edge = edge;
    p->scale = (float)(1 << level) / edge;
    p->nrhs = nrhs;
    p->layout = layout;
    p->flags = flags;
    const int64_t boxes = (int64_t)1 << (3 * level);
    p->box_cap = n < boxes ? n : boxes;
    p->red_cap = (is_pairtask(layout) ? 54 : 27) * n;
    // partial slots: one per (task, target); mutual tasks add one per source
    p->part_cap = (layout == P2P_LAYOUT_PAIRTASK || (flags & P2P_PLAN_SYMMETRIC)) ? 27 * n
                  : (layout == P2P_LAYOUT_SYMMETRIC) ? 54 * n : 0;
    p->rec_words = (kind == P2P_GRAVITY) ? 1 : helmholtz_rec_words(nrhs);
    p->rec_alloc_words = p->rec_words;
    if (flags & P2P_PLAN_ADJOINT)
        p->rec_alloc_words = (kind == P2P_GRAVITY) ? kGravityAdjointWords : helmholtz_adjoint_words(nrhs);
    p->sort_tiles = (int)((n + 2047) / 2048);
    p->use_table = level <= 8;
    // defaults; p2p_plan_set_tuning / the autotuner may change them
    if (kind == P2P_GRAVITY) {
        p->tpl = 2;
        p->tile = 128;   // 2 KB stages of 16-byte records: half the per-tile overhead of 64 (measured)
    } else {
        // one or two right-hand sides, one-sided: four targets per lane in two source groups;
        // otherwise two per lane
        const bool sym = (flags & P2P_PLAN_SYMMETRIC) || layout == P2P_LAYOUT_SYMMETRIC;
        p->tpl = (nrhs <= 2 && !sym) ? 4 : 2;
        p->tile = nrhs > 8 ? 32 : 64;
    }
    p->ctas_per_sm = 0;
    // Warps per work item.  A pair task holds one box's sources, usually a
    // single tile: one warp per task.  Otherwise, when the work items far
    // outnumber the resident warps (upper bound: every box non-empty) one warp
    // per item balances well and saves the group's exchange; few, heavy items
    // need cooperating warps.  Crossover measured on GB300 between the 2^20-point
    // (level 6) and 2^22-point (level 7) Plummer spheres.
    const int item_lanes = (kind == P2P_GRAVITY || p->tpl < 2) ? p->tpl : 2;   // Helmholtz items: <= 64 targets
    const double items_est = (double)p->box_cap + (double)n / (32.0 * item_lanes);
    const double resident_warps = (double)num_sms() * 16.0;
    p->group = (is_pairtask(layout) || items_est > 256.0 * resident_warps) ? 1 : 4;
    // symmetric Helmholtz items (self plus about half the neighbours as mutual
    // ranges) are uneven: two warps per item measured best on the 64^3 grid
    if (p->group == 4 && kind == P2P_HELMHOLTZ && (flags & P2P_PLAN_SYMMETRIC)) p->group = 2;
    p->split = nrhs;
    p->rmax = 2.0f * (edge / (float)(1 << level)) * 1.7320508f;
    p->items_cap = is_pairtask(layout) ? 27 * p->box_cap + (27 * n + 31) / 32 + 1
                                                   : p->box_cap + (n + 31) / 32 + 1;
    compute_layout(p);
    return P2P_OK;
}

}  // namespace p2p

using namespace p2p;

extern "C" {

const char* p2p_status_string(int status) {
    switch (status) {
        case P2P_OK: return "ok";
        case P2P_ERR_INVALID_ARG: return "invalid argument";
        case P2P_ERR_CUDA: return "CUDA runtime error";
        case P2P_ERR_OOM: return "out of host memory";
        case P2P_ERR_TIMEOUT: return "bounded device wait expired";
        case P2P_ERR_UNSUPPORTED: return "unsupported request";
        case P2P_ERR_DOMAIN: return "position outside the boxing domain";
        case P2P_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case P2P_ERR_STATE: return "call out of order";
        case P2P_ERR_BOUNDS: return "index check failed (checked build)";
        default: return "unknown status";
    }
}

int p2p_abi_version(void) { return P2P_ABI_VERSION; }

int p2p_build_checked(void) { return kChecked ? 1 : 0; }

int p2p_fail_host_allocs(int count) {
    g_fail_allocs.store(count > 0 ? count : 0);
    return P2P_OK;
}

int64_t p2p_launch_count(void) { return (int64_t)g_launches.load(); }

int p2p_plan_create(p2p_plan** out, int kind, int64_t n, int level, const float* lo, float edge, int nrhs,
                    int layout, unsigned flags) {
    if (!out) return P2P_ERR_INVALID_ARG;
    *out = nullptr;
    Plan tmp{};
    int st = plan_init(&tmp, kind, n, level, lo, edge, nrhs, layout, flags);
    if (st) return st;
    p2p_plan* h = host_alloc_should_fail() ? nullptr : new (std::nothrow) p2p_plan;
    if (!h) return P2P_ERR_OOM;
    h->p = tmp;
    Plan* p = &h->p;
    p->timing = (flags & P2P_PLAN_TIMING) ? 1 : 0;
    if (p->timing) {
        for (int ph = 0; ph < P2P_PHASE_COUNT; ++ph)
            for (int e = 0; e < 2; ++e)
                if (cudaEventCreate(&p->ev[ph][e]) != cudaSuccess) {
                    for (int q = 0; q <= ph; ++q)
                        for (int f = 0; f < 2; ++f)
                            if (p->ev[q][f]) cudaEventDestroy(p->ev[q][f]);
                    delete h;
                    return P2P_ERR_CUDA;
                }
    }
    *out = h;
    return P2P_OK;
}

int p2p_plan_destroy(p2p_plan* h) {
    if (!h) return P2P_OK;
    Plan* p = &h->p;
    if (p->timing)
        for (int ph = 0; ph < P2P_PHASE_COUNT; ++ph)
            for (int e = 0; e < 2; ++e)
                if (p->ev[ph][e]) cudaEventDestroy(p->ev[ph][e]);
    if (p->io_fork) cudaEventDestroy(p->io_fork);
    if (p->io_join) cudaEventDestroy(p->io_join);
    if (p->io_stream) cudaStreamDestroy(p->io_stream);
    delete h;
    return P2P_OK;
}

int p2p_plan_workspace_bytes(const p2p_plan* h, size_t* bytes) {
    if (!h || !bytes) return P2P_ERR_INVALID_ARG;
    *bytes = h->p.L.total;
    return P2P_OK;
}

int p2p_plan_set_tuning(p2p_plan* h, int targets_per_lane, int tile, int ctas_per_sm, int warps_per_item) {
    if (!h) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    const bool tpl_ok = targets_per_lane == 1 || targets_per_lane == 2 || targets_per_lane == 4;
    const bool g_ok = warps_per_item == 1 || warps_per_item == 2 || warps_per_item == 4;
    if (!tpl_ok || !g_ok || (tile != 32 && tile != 48 && tile != 64 && tile != 128) || ctas_per_sm < 0 ||
        ctas_per_sm > 32)
        return P2P_ERR_INVALID_ARG;
    p->tpl = targets_per_lane;
    p->tile = tile;
    p->ctas_per_sm = ctas_per_sm;
    p->group = warps_per_item;
    return P2P_OK;
}

int p2p_plan_set_grid(p2p_plan* h, float grid_h, int points_per_box) {
    if (!h) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    if (p->kind != P2P_HELMHOLTZ) return P2P_ERR_UNSUPPORTED;
    if ((is_pairtask(p->layout) || p->sym) && points_per_box != 0) return P2P_ERR_UNSUPPORTED;
    if (points_per_box == 0) {
        p->pattern = 0;
        p->rec_words = helmholtz_rec_words(p->nrhs);
        p->src_ready = 0;
        return P2P_OK;
    }
    if (!(grid_h > 0.0f) || points_per_box < 1 || points_per_box > 4) return P2P_ERR_INVALID_ARG;
    if (p->periodic) return P2P_ERR_UNSUPPORTED;   // the tabulated lattice displacements are not wrapped
    // the leaf box must hold points_per_box lattice points per edge
    const double box = (double)p->edge / (double)(1 << p->level);
    if (std::fabs(box / ((double)grid_h * points_per_box) - 1.0) > 1e-5) return P2P_ERR_INVALID_ARG;
    int st = pattern_setup(p, grid_h, points_per_box);
    if (st) return st;
    // one right-hand side: compact records [code, Re q, Im q, 0] (positions are not read)
    p->rec_words = (p->nrhs == 1) ? 1 : helmholtz_rec_words(p->nrhs);
    p->src_ready = 0;
    return P2P_OK;
}

int p2p_tree_build(p2p_plan* h, const float* pos, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("p2p_tree_build");
    if (!h || !pos || (reinterpret_cast<uintptr_t>(pos) & 3u)) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    int st = check_ws(p, ws, ws_bytes);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ev_begin(p, P2P_PHASE_TREE, s);
    st = tree_build(p, pos, ws, s);
    ev_end(p, P2P_PHASE_TREE, s);
    return st;
}

int p2p_tree_import(p2p_plan* h, const int32_t* perm, const int32_t* box_start, int32_t n_boxes,
                    const int32_t* nbr_start, const int32_t* nbr_idx, int32_t n_nbr, void* ws, size_t ws_bytes,
                    void* stream) {
    NvtxRange nvtx_range("p2p_tree_import");
    if (!h || !perm || !box_start || !nbr_start || !nbr_idx) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    int st = check_ws(p, ws, ws_bytes);
    if (st) return st;
    if ((int64_t)n_boxes > p->box_cap) return P2P_ERR_INVALID_ARG;
    if (p->periodic) return P2P_ERR_UNSUPPORTED;   // imported lists carry no image codes
    return tree_import(p, perm, box_start, n_boxes, nbr_start, nbr_idx, n_nbr, ws, static_cast<cudaStream_t>(stream));
}

int p2p_restructure(p2p_plan* h, const float* pos, const void* strength, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("p2p_restructure");
    if (!h || !pos || !strength || (reinterpret_cast<uintptr_t>(pos) & 3u)) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    if ((reinterpret_cast<uintptr_t>(strength) & (p->kind == P2P_GRAVITY ? 3u : 7u)) != 0) return P2P_ERR_INVALID_ARG;
    int st = check_ws(p, ws, ws_bytes);
    if (st) return st;
    if (!p->tree_ready) return P2P_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ev_begin(p, P2P_PHASE_RESTRUCTURE, s);
    st = restructure(p, pos, strength, ws, s);
    ev_end(p, P2P_PHASE_RESTRUCTURE, s);
    return st;
}

int p2p_gravity(p2p_plan* h, float eps, float* phi, float* acc, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("p2p_gravity");
    if (!h || !phi || !acc) return P2P_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(phi) & 3u) || (reinterpret_cast<uintptr_t>(acc) & 3u)) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    if (p->kind != P2P_GRAVITY || !(eps >= 0.0f) || !(eps < 1.0e19f)) return P2P_ERR_INVALID_ARG;
    int st = check_ws(p, ws, ws_bytes);
    if (st) return st;
    if (!p->tree_ready || !p->src_ready) return P2P_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ev_begin(p, P2P_PHASE_OPERATOR, s);
    st = build_items(p, ws, 32 * p->tpl, s);
    if (st) return st;
    ev_begin(p, P2P_PHASE_KERNEL, s);
    st = launch_gravity_kernel(p, loop_args(p, ws, p->rec_words), at<int32_t>(ws, p->L.perm), eps, phi, acc, s);
    if (st) return st;
    ev_end(p, P2P_PHASE_KERNEL, s);
    if (is_pairtask(p->layout)) {
        st = pairtask_reduce_gravity(p, ws, phi, acc, s);
        if (st) return st;
    } else if (p->sym) {
        st = sym_fixup_gravity(p, ws, phi, acc, s);
        if (st) return st;
    }
    ev_end(p, P2P_PHASE_OPERATOR, s);
    return P2P_OK;
}

int p2p_helmholtz(p2p_plan* h, float k, void* u, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("p2p_helmholtz");
    if (!h || !u || (reinterpret_cast<uintptr_t>(u) & 7u)) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    if (p->kind != P2P_HELMHOLTZ || !(k == k) || !(fabsf(k) < 1.0e30f)) return P2P_ERR_INVALID_ARG;
    int st = check_ws(p, ws, ws_bytes);
    if (st) return st;
    if (!p->tree_ready || !p->src_ready) return P2P_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ev_begin(p, P2P_PHASE_OPERATOR, s);
    st = build_items(p, ws, 32 * (p->pattern ? (p->tpl >= 2 ? 2 : 1) : helmholtz_targets_per_lane(p, k)), s);
    if (st) return st;
    if (p->pattern) {
        ev_begin(p, P2P_PHASE_KERNEL, s);
        st = launch_helmholtz_pattern(p, loop_args(p, ws, p->rec_words), at<int32_t>(ws, p->L.perm), k,
                                      at<float2>(ws, p->L.pattern), HelmOut{static_cast<float2*>(u), nullptr, p->nrhs},
                                      s);
        if (st) return st;
        ev_end(p, P2P_PHASE_KERNEL, s);
        ev_end(p, P2P_PHASE_OPERATOR, s);
        return P2P_OK;
    }
    ev_begin(p, P2P_PHASE_KERNEL, s);
    st = launch_helmholtz_kernel(p, loop_args(p, ws, p->rec_words), at<int32_t>(ws, p->L.perm), k,
                                 HelmOut{static_cast<float2*>(u), nullptr, p->nrhs}, s);
    if (st) return st;
    ev_end(p, P2P_PHASE_KERNEL, s);
    if (is_pairtask(p->layout)) {
        st = pairtask_reduce_helmholtz(p, ws, static_cast<float2*>(u), s);
        if (st) return st;
    } else if (p->sym) {
        st = sym_fixup_helmholtz(p, ws, static_cast<float2*>(u), s);
        if (st) return st;
    }
    ev_end(p, P2P_PHASE_OPERATOR, s);
    return P2P_OK;
}

// The transfer phase and the collect phase of a host-buffer step: the
// strengths' copy is forked onto the plan's own stream (after the work already
// queued on `s`) and joined before the restructuring, so it overlaps the
// position copy and the tree build.
static int host_inputs(p2p_plan* h, const float* pos, const void* str, size_t str_bytes, void* ws, size_t ws_bytes,
                       cudaStream_t s) {
    Plan* p = &h->p;
    const Layout& L = p->L;
    float* dpos = at<float>(ws, L.io_pos);
    void* dstr = at<unsigned char>(ws, L.io_str);
    if (!p->io_stream) {   // created on first use (on the current device)
        P2P_CUDA_TRY(cudaStreamCreateWithFlags(&p->io_stream, cudaStreamNonBlocking));
        P2P_CUDA_TRY(cudaEventCreateWithFlags(&p->io_fork, cudaEventDisableTiming));
        P2P_CUDA_TRY(cudaEventCreateWithFlags(&p->io_join, cudaEventDisableTiming));
    }
    P2P_CUDA_TRY(cudaEventRecord(p->io_fork, s));
    P2P_CUDA_TRY(cudaStreamWaitEvent(p->io_stream, p->io_fork, 0));
    P2P_CUDA_TRY(cudaMemcpyAsync(dstr, str, str_bytes, cudaMemcpyHostToDevice, p->io_stream));
    P2P_CUDA_TRY(cudaEventRecord(p->io_join, p->io_stream));
    P2P_CUDA_TRY(cudaMemcpyAsync(dpos, pos, (size_t)p->n * 12, cudaMemcpyHostToDevice, s));
    int st = p2p_tree_build(h, dpos, ws, ws_bytes, s);
    // join the side stream even when the build failed, so it never outlives the call
    const cudaError_t e = cudaStreamWaitEvent(s, p->io_join, 0);
    if (st) return st;
    if (e != cudaSuccess) return P2P_ERR_CUDA;
    return p2p_restructure(h, dpos, dstr, ws, ws_bytes, s);
}

static int host_check(p2p_plan* h, int kind, const void* a, const void* b, const void* c, void* ws, size_t ws_bytes) {
    if (!h || !a || !b || !c) return P2P_ERR_INVALID_ARG;
    const Plan* p = &h->p;
    if (p->kind != kind) return P2P_ERR_INVALID_ARG;
    if (!(p->flags & P2P_PLAN_HOST_IO)) return P2P_ERR_UNSUPPORTED;
    return check_ws(p, ws, ws_bytes);
}

int p2p_gravity_host(p2p_plan* h, float eps, const float* pos, const float* mass, float* phi, float* acc, void* ws,
                     size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("p2p_gravity_host");
    int st = host_check(h, P2P_GRAVITY, pos, mass, phi, ws, ws_bytes);
    if (st) return st;
    if (!acc) return P2P_ERR_INVALID_ARG;
    const Plan* p = &h->p;
    const int64_t n = p->n;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = host_inputs(h, pos, mass, (size_t)n * 4, ws, ws_bytes, s);
    if (st) return st;
    float* dphi = at<float>(ws, p->L.io_out);
    float* dacc = dphi + n;
    st = p2p_gravity(h, eps, dphi, dacc, ws, ws_bytes, stream);
    if (st) return st;
    P2P_CUDA_TRY(cudaMemcpyAsync(phi, dphi, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    P2P_CUDA_TRY(cudaMemcpyAsync(acc, dacc, (size_t)n * 12, cudaMemcpyDeviceToHost, s));
    return P2P_OK;
}

int p2p_helmholtz_host(p2p_plan* h, float k, const float* pos, const void* q, void* u, void* ws, size_t ws_bytes,
                       void* stream) {
    NvtxRange nvtx_range("p2p_helmholtz_host");
    int st = host_check(h, P2P_HELMHOLTZ, pos, q, u, ws, ws_bytes);
    if (st) return st;
    const Plan* p = &h->p;
    const size_t bytes = (size_t)p->n * 8 * p->nrhs;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = host_inputs(h, pos, q, bytes, ws, ws_bytes, s);
    if (st) return st;
    void* du = at<unsigned char>(ws, p->L.io_out);
    st = p2p_helmholtz(h, k, du, ws, ws_bytes, stream);
    if (st) return st;
    P2P_CUDA_TRY(cudaMemcpyAsync(u, du, bytes, cudaMemcpyDeviceToHost, s));
    return P2P_OK;
}

int p2p_helmholtz_adjoint(p2p_plan* h, float k, const float* pos, const void* q, const void* gbar, void* grad_q,
                          float* grad_pos, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("p2p_helmholtz_adjoint");
    if (!h || !pos || !gbar || (!grad_q && !grad_pos)) return P2P_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(gbar) & 7u) || (reinterpret_cast<uintptr_t>(grad_q) & 7u) ||
        (reinterpret_cast<uintptr_t>(grad_pos) & 3u) || (reinterpret_cast<uintptr_t>(pos) & 3u))
        return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    if (p->kind != P2P_HELMHOLTZ || !(k == k) || !(fabsf(k) < 1.0e30f)) return P2P_ERR_INVALID_ARG;
    if (is_pairtask(p->layout) || p->sym) return P2P_ERR_UNSUPPORTED;
    int st = check_ws(p, ws, ws_bytes);
    if (st) return st;
    if (!p->tree_ready) return P2P_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!grad_pos) {
        // grad_q = conj(P) gbar = P(-k) gbar: the forward operator on gbar
        ev_begin(p, P2P_PHASE_RESTRUCTURE, s);
        st = restructure(p, pos, gbar, ws, s);
        if (st) return st;
        ev_end(p, P2P_PHASE_RESTRUCTURE, s);
        ev_begin(p, P2P_PHASE_OPERATOR, s);
        if (p->pattern) {
            st = build_items(p, ws, 32 * (p->tpl >= 2 ? 2 : 1), s);
            if (st) return st;
            ev_begin(p, P2P_PHASE_KERNEL, s);
            st = launch_helmholtz_pattern(p, loop_args(p, ws, p->rec_words), at<int32_t>(ws, p->L.perm), -k,
                                          at<float2>(ws, p->L.pattern),
                                          HelmOut{static_cast<float2*>(grad_q), nullptr, p->nrhs}, s);
            p->src_ready = 0;
            if (st) return st;
            ev_end(p, P2P_PHASE_KERNEL, s);
            ev_end(p, P2P_PHASE_OPERATOR, s);
            return P2P_OK;
        }
        st = build_items(p, ws, 32 * helmholtz_targets_per_lane(p, -k), s);
        if (st) return st;
        ev_begin(p, P2P_PHASE_KERNEL, s);
        st = launch_helmholtz_kernel(p, loop_args(p, ws, p->rec_words), at<int32_t>(ws, p->L.perm), -k,
                                     HelmOut{static_cast<float2*>(grad_q), nullptr, p->nrhs}, s);
        p->src_ready = 0;   // the records hold gbar, not the forward sources
        if (st) return st;
        ev_end(p, P2P_PHASE_KERNEL, s);
        ev_end(p, P2P_PHASE_OPERATOR, s);
        return P2P_OK;
    }
    if (!q || (reinterpret_cast<uintptr_t>(q) & 7u)) return P2P_ERR_INVALID_ARG;
    int words = 0;
    ev_begin(p, P2P_PHASE_RESTRUCTURE, s);
    st = restructure_adjoint(p, pos, q, gbar, nullptr, ws, &words, s);
    if (st) return st;
    ev_end(p, P2P_PHASE_RESTRUCTURE, s);
    ev_begin(p, P2P_PHASE_OPERATOR, s);
    st = build_items(p, ws, 32, s);
    if (st) return st;
    ev_begin(p, P2P_PHASE_KERNEL, s);
    st = launch_helmholtz_adjoint_kernel(p, loop_args(p, ws, words), at<int32_t>(ws, p->L.perm), k,
                                         helmholtz_needs_precise(p, k), static_cast<float2*>(grad_q), grad_pos, s);
    if (st) return st;
    ev_end(p, P2P_PHASE_KERNEL, s);
    ev_end(p, P2P_PHASE_OPERATOR, s);
    return P2P_OK;
}

int p2p_gravity_adjoint(p2p_plan* h, float eps, const float* pos, const float* mass, const float* grad_phi,
                        const float* grad_acc, float* grad_mass, float* grad_pos, void* ws, size_t ws_bytes,
                        void* stream) {
    NvtxRange nvtx_range("p2p_gravity_adjoint");
    if (!h || !pos || !mass || !grad_phi || !grad_acc || (!grad_mass && !grad_pos)) return P2P_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(pos) | reinterpret_cast<uintptr_t>(mass) | reinterpret_cast<uintptr_t>(grad_phi) |
         reinterpret_cast<uintptr_t>(grad_acc) | reinterpret_cast<uintptr_t>(grad_mass) |
         reinterpret_cast<uintptr_t>(grad_pos)) & 3u)
        return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
    if (p->kind != P2P_GRAVITY || !(eps >= 0.0f) || !(eps < 1.0e19f)) return P2P_ERR_INVALID_ARG;
    if (is_pairtask(p->layout) || p->sym) return P2P_ERR_UNSUPPORTED;
    int st = check_ws(p, ws, ws_bytes);
    if (st) return st;
    if (!p->tree_ready) return P2P_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int words = 0;
    ev_begin(p, P2P_PHASE_RESTRUCTURE, s);
    st = restructure_adjoint(p, pos, mass, grad_phi, grad_acc, ws, &words, s);
    if (st) return st;
    ev_end(p, P2P_PHASE_RESTRUCTURE, s);
    ev_begin(p, P2P_PHASE_OPERATOR, s);
    st = build_items(p, ws, 32 * gravity_adjoint_targets_per_lane(p), s);
    if (st) return st;
    ev_begin(p, P2P_PHASE_KERNEL, s);
    st = launch_gravity_adjoint_kernel(p, loop_args(p, ws, words), at<int32_t>(ws, p->L.perm), eps, grad_mass,
                                       grad_pos, s);
    if (st) return st;
    ev_end(p, P2P_PHASE_KERNEL, s);
    ev_end(p, P2P_PHASE_OPERATOR, s);
    return P2P_OK;
}

int p2p_plan_array(const p2p_plan* h, int which, int64_t* offset_bytes, int64_t* capacity) {
    if (!h || !offset_bytes || !capacity) return P2P_ERR_INVALID_ARG;
    const Plan* p = &h->p;
    const Layout& L = p->L;
    const bool red = p->layout == P2P_LAYOUT_REDUNDANT;
    const bool pt = is_pairtask(p->layout);
    const bool sym = p->layout == P2P_LAYOUT_SYMMETRIC || p->sym;
    switch (which) {
        case P2P_ARR_PERM: *offset_bytes = L.perm; *capacity = p->n; break;
        case P2P_ARR_BOX_KEY: *offset_bytes = L.box_key; *capacity = p->box_cap; break;
        case P2P_ARR_BOX_START: *offset_bytes = L.box_start; *capacity = p->box_cap + 1; break;
        case P2P_ARR_NBR_START: *offset_bytes = L.nbr_start; *capacity = p->box_cap + 1; break;
        case P2P_ARR_NBR_IDX: *offset_bytes = L.nbr_idx; *capacity = 27 * p->box_cap; break;
        case P2P_ARR_RED_START:
            if (!red) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.red_start; *capacity = p->box_cap + 1; break;
        case P2P_ARR_RED_SELF:
            if (!red) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.red_self; *capacity = p->box_cap; break;
        case P2P_ARR_GATHER_IDX:
            if (!(red || pt) || !(p->flags & P2P_PLAN_GATHER_MAP)) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.gather; *capacity = p->red_cap; break;
        case P2P_ARR_SORTED_KEY: *offset_bytes = L.sorted_key; *capacity = p->n; break;
        case P2P_ARR_NBR_IMG:
            if (!p->periodic) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.nbr_img; *capacity = 27 * p->box_cap; break;
        case P2P_ARR_ENT_BOX:
            if (!pt) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.ent_box; *capacity = 27 * p->box_cap; break;
        case P2P_ARR_PT_START:
            if (!pt) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.pt_start; *capacity = 27 * p->box_cap + 1; break;
        case P2P_ARR_PART_START:
            if (!pt) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.part_start; *capacity = 27 * p->box_cap + 1; break;
        case P2P_ARR_TASK_KIND:
            if (!sym) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.task_kind; *capacity = 27 * p->box_cap; break;
        case P2P_ARR_MIRROR:
            if (!sym) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.mirror; *capacity = 27 * p->box_cap; break;
        case P2P_ARR_BSLOT:
            if (!p->sym) return P2P_ERR_UNSUPPORTED;
            *offset_bytes = L.bslot; *capacity = 27 * p->box_cap + 1; break;
        default: return P2P_ERR_INVALID_ARG;
    }
    return P2P_OK;
}

int p2p_read_counters(const p2p_plan* h, const void* ws, int64_t* out, void* stream) {
    if (!h || !ws || !out) return P2P_ERR_INVALID_ARG;
    Header hdr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&hdr, static_cast<const char*>(ws) + h->p.L.header, sizeof(Header), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess)
        return P2P_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return P2P_ERR_CUDA;
    out[P2P_CTR_N_BOXES] = hdr.n_boxes;
    out[P2P_CTR_N_NBR] = hdr.n_nbr;
    out[P2P_CTR_FLAGS] = hdr.flags;
    out[P2P_CTR_TOTAL_SRC] = hdr.total_src;
    out[P2P_CTR_PAIRS] = (int64_t)hdr.pairs_nS - h->p.n;
    out[P2P_CTR_N_ITEMS] = hdr.n_items;
    out[P2P_CTR_EVALS] = (int64_t)hdr.evals_nS - h->p.n;
    if (hdr.flags & P2P_FLAG_BOUNDS) return P2P_ERR_BOUNDS;
    if (hdr.flags & P2P_FLAG_TIMEOUT) return P2P_ERR_TIMEOUT;
    if (hdr.flags & P2P_FLAG_DOMAIN) return P2P_ERR_DOMAIN;
    if (hdr.flags & (P2P_FLAG_CAPACITY | P2P_FLAG_LATTICE)) return P2P_ERR_INVALID_ARG;
    return P2P_OK;
}

int p2p_plan_timing(p2p_plan* h, float* ms_out) {
    if (!h || !ms_out) return P2P_ERR_INVALID_ARG;
    Plan* p = &h->p;
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

}  // extern "C"
