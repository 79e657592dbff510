// Gravity near field without a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need
// the operator: code running under an allocator that forbids new device
// allocations (a fixed memory pool or budget), plugins handed only their
// input and output buffers by a host framework, or code paths that must not
// add allocation calls to an otherwise pre-planned sequence.  For them,
// p2p_gravity_noalloc runs the same pipeline as p2p_tree_build +
// p2p_restructure + p2p_gravity on a plan with the default tuning (the same
// plan set-up, workspace layout and kernels, so the same results bit for
// bit) with its scratch in one file-scope device array of fixed size, so it
// allocates nothing.  p2p_gravity_noalloc_status reads the device flag word
// that the last call left in that array.
//
// Limits: n <= P2P_NOALLOC_MAX_N particles and level <= P2P_NOALLOC_MAX_LEVEL
// (scratch of P2P_NOALLOC_SCRATCH_BYTES, held on every GPU that loads the
// library until the process exits).  Every call shares the array, so calls
// whose work overlaps on the GPU (other streams, other host threads) race.
#include "common.cuh"
#include "p2p_loop.cuh"

namespace p2p {
namespace {

static_assert(P2P_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");
static __device__ __align__(256) unsigned char g_noalloc_scratch[P2P_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current context.  The host-side
// name of the array is not a device address; cudaGetSymbolAddress gives it.
// It is looked up on every call (after the first call on a device, which
// loads the library's module there, this is a host-side lookup), so the
// address is never stale, e.g. after a cudaDeviceReset.
int scratch_address(void** out) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return P2P_ERR_CUDA;
    *out = ptr;
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

    // the plan a workspace call with these arguments would use (host only)
    Plan p{};
    int st = plan_init(&p, P2P_GRAVITY, n, level, lo, edge, 1, layout, 0);
    if (st) return st;
    if (p.L.total > (size_t)P2P_NOALLOC_SCRATCH_BYTES) return P2P_ERR_UNSUPPORTED;

    void* ws = nullptr;
    st = scratch_address(&ws);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = tree_build(&p, pos, ws, s);
    if (st) return st;
    st = restructure(&p, pos, mass, ws, s);
    if (st) return st;
    st = build_items(&p, ws, 32 * p.tpl, s);
    if (st) return st;
    return launch_gravity_kernel(&p, loop_args(&p, ws, p.rec_words), at<int32_t>(ws, p.L.perm), eps, phi, acc, s);
}

extern "C" int p2p_gravity_noalloc_status(uint32_t* flags, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Header hdr;
    if (cudaMemcpyFromSymbolAsync(&hdr, g_noalloc_scratch, sizeof(Header), 0, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return P2P_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return P2P_ERR_CUDA;
    if (flags) *flags = hdr.flags;
    if (hdr.flags & P2P_FLAG_BOUNDS) return P2P_ERR_BOUNDS;
    if (hdr.flags & P2P_FLAG_TIMEOUT) return P2P_ERR_TIMEOUT;
    if (hdr.flags & P2P_FLAG_DOMAIN) return P2P_ERR_DOMAIN;
    if (hdr.flags & (P2P_FLAG_CAPACITY | P2P_FLAG_LATTICE)) return P2P_ERR_INVALID_ARG;
    return P2P_OK;
}
