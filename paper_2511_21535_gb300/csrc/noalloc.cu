// Gravity near field without a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need
// the operator: code running under an allocator that forbids new device
// allocations (a fixed memory pool or budget), plugins handed only their
// input and output buffers by a host framework, or code paths that must not
// add allocation calls to an otherwise pre-planned sequence.  For them,
// p2p_gravity_noalloc runs the same pipeline as p2p_tree_build +
// p2p_restructure + p2p_gravity (same kernels, same results) with its scratch
// in one file-scope device array of fixed size, so it allocates nothing.
//
// Limits: n <= P2P_NOALLOC_MAX_N particles and level <= P2P_NOALLOC_MAX_LEVEL
// (scratch of P2P_NOALLOC_SCRATCH_BYTES, held on every GPU that loads the
// library until the process exits).  Every call shares the array, so calls
// whose work overlaps on the GPU (other streams, other host threads) race.
#include <mutex>

#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {
namespace {

static_assert(P2P_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");
static __device__ __align__(256) unsigned char g_noalloc_scratch[P2P_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

inline size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// The scratch layout: the same arrays as a plan's workspace (capi.cu), sized
// for this call.
void noalloc_layout(Plan* p) {
    Layout& L = p->L;
    const int64_t n = p->n, bc = p->box_cap;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = up256(off + (bytes ? bytes : 16));
        return o;
    };
    L.header = take(kHeaderBytes);
    L.keys_a = take(n * 4);
    L.keys_b = take(n * 4);
    L.vals_a = take(n * 4);
    L.perm = take(n * 4);
    L.sorted_key = take(n * 4);
    L.hist = take(((size_t)256 * p->sort_tiles + 1) * 4);
    int64_t scan_max = (int64_t)256 * p->sort_tiles;
    if (n > scan_max) scan_max = n;
    L.scan_tmp = take(scan_scratch_bytes(scan_max));
    L.lookback = take((size_t)lb_regions(n, bc).words * 8);
    L.box_key = take(bc * 4);
    L.box_start = take((bc + 1) * 4);
    L.table = take(((size_t)1 << (3 * p->level)) * 4);
    L.nbr_start = take((bc + 1) * 4);
    L.nbr_idx = take((size_t)27 * bc * 4);
    L.src = take((size_t)n * 16);
    L.box_S = take((bc + 1) * 4);
    L.items = take((size_t)p->items_cap * 8);
    if (p->layout == P2P_LAYOUT_REDUNDANT) {
        L.red_start = take((bc + 1) * 4);
        L.red_self = take(bc * 4);
        L.red_src = take((size_t)p->red_cap * 16);
    } else {
        L.red_start = L.red_self = L.red_src = 0;
    }
    L.gather = 0;
    L.pattern = 0;
    L.nbr_img = 0;
    L.ent_box = L.pt_start = L.part_start = L.part = 0;
    L.task_kind = L.mirror = L.bslot = 0;
    L.total = off;
}

// Device address of the scratch array for the current device, looked up
// once per device (the host-side name of the array is not a device address).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return P2P_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return P2P_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return P2P_ERR_CUDA;
        g_addr[dev] = ptr;
    }
    *out = g_addr[dev];
    return P2P_OK;
}

}  // namespace
}  // namespace p2p

using namespace p2p;

extern "C" int p2p_gravity_noalloc(const float* pos, const float* mass, int64_t n, int level, const float* lo,
                                   float edge, float eps, int layout, float* phi, float* acc, void* stream) {
    if (!pos || !mass || !phi || !acc || !lo) return P2P_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(pos) | reinterpret_cast<uintptr_t>(mass) | reinterpret_cast<uintptr_t>(phi) |
         reinterpret_cast<uintptr_t>(acc)) & 3u)
        return P2P_ERR_INVALID_ARG;
    if (n < 1 || level < 1 || !(edge > 0.0f) || !(edge < 3.0e38f) || !(eps >= 0.0f) || !(eps < 1.0e19f))
        return P2P_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(lo[a] == lo[a]) || lo[a] > 3.0e38f || lo[a] < -3.0e38f) return P2P_ERR_INVALID_ARG;
    if (layout != P2P_LAYOUT_INDIRECT && layout != P2P_LAYOUT_REDUNDANT) return P2P_ERR_INVALID_ARG;
    if (n > P2P_NOALLOC_MAX_N || level > P2P_NOALLOC_MAX_LEVEL) return P2P_ERR_UNSUPPORTED;

    Plan p{};
    p.kind = P2P_GRAVITY;
    p.n = n;
    p.level = level;
    for (int a = 0; a < 3; ++a) p.lo[a] = lo[a];
    p.edge = edge;
    p.scale = (float)(1 << level) / edge;
    p.nrhs = 1;
    p.layout = layout;
    p.flags = 0;
    const int64_t boxes = (int64_t)1 << (3 * level);
    p.box_cap = n < boxes ? n : boxes;
    p.red_cap = 27 * n;
    p.rec_words = 1;
    p.rec_alloc_words = 1;
    p.sort_tiles = (int)((n + 2047) / 2048);
    p.use_table = 1;
    p.tpl = 2;
    p.tile = 64;
    p.ctas_per_sm = 0;
    p.group = 4;
    p.split = 1;
    p.rmax = 2.0f * (edge / (float)(1 << level)) * 1.7320508f;
    p.items_cap = p.box_cap + (n + 31) / 32 + 1;
    noalloc_layout(&p);
    if (p.L.total > (size_t)P2P_NOALLOC_SCRATCH_BYTES) return P2P_ERR_UNSUPPORTED;

    void* ws = nullptr;
    int st = scratch_address(&ws);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = tree_build(&p, pos, ws, s);
    if (st) return st;
    st = restructure(&p, pos, mass, ws, s);
    if (st) return st;
    st = build_items(&p, ws, 32 * p.tpl, s);
    if (st) return st;
    LoopArgs a{};   // every field not set below is null
    a.rec = at<float4>(ws, p.L.src);
    a.red = (layout == P2P_LAYOUT_REDUNDANT) ? at<float4>(ws, p.L.red_src) : nullptr;
    a.words = 1;
    a.tile = p.tile;
    a.box_start = at<int32_t>(ws, p.L.box_start);
    a.nbr_start = at<int32_t>(ws, p.L.nbr_start);
    a.nbr_idx = at<int32_t>(ws, p.L.nbr_idx);
    a.red_start = (layout == P2P_LAYOUT_REDUNDANT) ? at<int32_t>(ws, p.L.red_start) : nullptr;
    a.red_self = (layout == P2P_LAYOUT_REDUNDANT) ? at<int32_t>(ws, p.L.red_self) : nullptr;
    a.items = at<int2>(ws, p.L.items);
    a.hdr = at<Header>(ws, p.L.header);
    a.nbr_img = nullptr;
    a.edge = p.edge;
    a.rec_cap = p.n;
    a.red_cap = p.red_cap;
    a.items_cap = p.items_cap;
    a.box_cap = p.box_cap;
    a.n = p.n;
    a.ent_box = a.pt_start = a.part_start = nullptr;
    a.part = nullptr;
    a.part_cap = 0;
    return launch_gravity_kernel(&p, a, at<int32_t>(ws, p.L.perm), eps, phi, acc, s);
}
