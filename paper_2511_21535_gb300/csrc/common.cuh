// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "p2p_gb300.h"

namespace p2p {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// workspace header (first 1 KiB of the workspace)
// ---------------------------------------------------------------------------
constexpr int kCostClasses = 64;

struct Header {
    // tree section (written by the tree build / import), offset 0
    int32_t n_boxes;
    int32_t n_nbr;
    uint32_t flags;
    int32_t tree_pad[13];
    // restructuring section (zeroed at the start of each restructuring), offset 64
    unsigned long long pairs_nS;       // sum_b n_b S_b
    int32_t total_src;                 // sum_b S_b (redundant records; pair tasks: task-stream records)
    int32_t part_total;                // pair tasks: partial-result slots, sum_e n_b(e)
    unsigned long long evals_nS;       // sum over streamed pairs (symmetric: mutual pairs once), self included
    int32_t n_heavy;                   // redundant gather: boxes whose streams exceed kGatherLight records
    int32_t restr_pad[9];
    // operator section (zeroed at the start of each operator call), offset 128
    int32_t n_items;
    uint32_t work_ctr;
    int32_t cls_cnt[kCostClasses];
    int32_t cls_cursor[kCostClasses];
};
constexpr size_t kHeaderBytes = 1024;
constexpr size_t kRestrSectionOffset = 64;
constexpr size_t kOpSectionOffset = 128;
static_assert(sizeof(Header) <= kHeaderBytes, "header too large");
static_assert(offsetof(Header, pairs_nS) == kRestrSectionOffset, "header layout");
static_assert(offsetof(Header, n_items) == kOpSectionOffset, "header layout");

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
struct Layout {                        // byte offsets inside the workspace
    size_t header, keys_a, keys_b, vals_a, perm, sorted_key, hist, scan_tmp, lookback,
        box_key, box_start, table, nbr_start, nbr_idx, src, box_S, red_start,
        red_self, red_src, gather, items, pattern, nbr_img, heavy,
        ent_box, pt_start, part_start, part,   // pair tasks (red_src/gather hold the task stream)
        task_kind, mirror,                      // symmetric tasks (layout or plan flag)
        bslot,                                  // plan flag: source-sum slots of mutual entries
        io_pos, io_str, io_out,                 // P2P_PLAN_HOST_IO: device copies of inputs and outputs
        total;
};

struct Plan {
    int kind;
    int64_t n;
    int level;
    float lo[3];
    float edge;
    float scale;                       // (float)2^level / edge
    int nrhs;
    int layout;
    unsigned flags;
    int64_t box_cap;                   // min(n, 8^level)
    int64_t items_cap;
    int64_t red_cap;                   // 27 n records (pair tasks: 54 n)
    int64_t part_cap;                  // pair tasks: 27 n partial-result slots (symmetric: 54 n)
    int rec_words;                     // 16-byte words per source record (forward)
    int rec_alloc_words;               // words per record the workspace holds (>= adjoint records)
    int sort_tiles;
    int use_table;                     // dense key -> box table (level <= 8)
    // tuning
    int tpl;                           // targets per lane
    int tile;                          // source records per stage
    int ctas_per_sm;
    int group;                         // warps cooperating on one work item
    int split;                         // Helmholtz RHS from here on form a conjugated second output
    // pattern mode (regular grids): lattice spacing, points per box edge, table strides
    int periodic;
    int sym;                           // P2P_PLAN_SYMMETRIC on a target-owned layout
    int pattern;
    float grid_h;
    int grid_t;
    int pat_sy, pat_sz, pat_size, pat_bias;
    float rmax;                        // largest distance between points of neighbouring boxes
    Layout L;
    // state
    int tree_ready;
    int src_ready;
    // timing
    cudaEvent_t ev[P2P_PHASE_COUNT][2];
    int ev_valid[P2P_PHASE_COUNT];
    int timing;
    // P2P_PLAN_HOST_IO: the stream that copies the strengths, and its fork / join events
    cudaStream_t io_stream;
    cudaEvent_t io_fork, io_join;
};

// launch accounting
void count_launch(int k = 1);

// phase timing of plans with P2P_PLAN_TIMING: CUDA events on the launching
// stream (external event nodes while the stream is being captured)
void ev_begin(Plan* p, int phase, cudaStream_t s);
void ev_end(Plan* p, int phase, cudaStream_t s);

// host allocation failure injection (testing): true while failures are pending
bool host_alloc_should_fail();

// Checked builds (P2P_CHECKED): index checks that record P2P_FLAG_BOUNDS and
// let the caller skip the access instead of faulting.
#ifdef P2P_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
__device__ __forceinline__ bool dcheck(bool cond, Header* hdr) {
    if (!kChecked || cond) return true;
    atomicOr(&hdr->flags, P2P_FLAG_BOUNDS);
    return false;
}

// error helper
#define P2P_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return P2P_ERR_CUDA;         \
    } while (0)

#define P2P_LAUNCH_CHECK()                                  \
    do {                                                    \
        ::p2p::count_launch();                              \
        cudaError_t _e = cudaGetLastError();                \
        if (_e != cudaSuccess) return P2P_ERR_CUDA;         \
    } while (0)

template <typename T>
inline T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

// Launches with programmatic stream serialisation, so that a kernel's launch
// overlaps the end of its predecessor in the stream (the kernels wait on the
// predecessor's completion themselves, see pdl_wait); disabled when the
// environment sets P2P_NO_PDL=1.
bool pdl_enabled();
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Chained-scan scratch (lookback.cuh), regions of 1 + tiles words: the box
// CSR (tiles of kCsrTileElems sorted particles), the neighbour CSR and two
// chains of the box statistics (tiles of kBoxTile boxes).  The key kernel
// clears the first two, the record kernels of the restructuring the others.
constexpr int kCsrTileElems = 2048;
constexpr int kBoxTile = 32;
// redundant gather: a stream of at most kGatherLight records is copied flat by
// one warp (with other light streams); longer ones by kGatherParts warps
constexpr int kGatherLight = 512;
constexpr int kGatherParts = 4;
// Radix sort of 3 * level key bits: equal digit widths of at most 8 bits.
inline void sort_digits(int level, int* passes, int* dbits) {
    const int bits = 3 * level;
    *passes = (bits + 7) / 8;
    *dbits = (bits + *passes - 1) / *passes;
}

struct LbRegions {
    int64_t csr, nbr, stats, stats2, tree_words, words;   // offsets and sizes in 8-byte words
};
inline LbRegions lb_regions(int64_t n, int64_t box_cap) {
    LbRegions r;
    const int64_t a = 1 + (n + kCsrTileElems - 1) / kCsrTileElems;
    const int64_t b = 1 + (box_cap + kBoxTile - 1) / kBoxTile;
    r.csr = 0;
    r.nbr = a;
    r.stats = a + b;                   // stream bounds
    r.stats2 = a + 2 * b;              // source-sum slots (symmetric plans)
    r.tree_words = a + b;
    r.words = a + 3 * b;
    return r;
}

// 32-bit fill of a device range as a kernel (a memset node would break the
// chain of programmatic launches)
int fill32(void* dst, uint32_t value, int64_t count, cudaStream_t s);

inline int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ---------------------------------------------------------------------------
// phases implemented in the other translation units
// ---------------------------------------------------------------------------

// exclusive scan of int32 in[0..n_cap) (elements at index >= *d_len read as 0
// when d_len != nullptr) into out[0..n_cap]; out[n_cap] (and out[len]) is the
// total, also stored to *d_total when non-null.  in may alias out.
size_t scan_scratch_bytes(int64_t n_cap);
int scan_exclusive(const int32_t* in, int32_t* out, int64_t n_cap, const int32_t* d_len,
                   int32_t* d_total, int32_t* scratch, cudaStream_t s);

struct LoopArgs;
int plan_init(Plan* p, int kind, int64_t n, int level, const float* lo, float edge, int nrhs, int layout,
              unsigned flags);
void compute_layout(Plan* p);
int check_ws(const Plan* p, const void* ws, size_t ws_bytes);
LoopArgs loop_args(const Plan* p, void* ws, int words);
int tree_build(Plan* p, const float* pos, void* ws, cudaStream_t s);
int tree_import(Plan* p, const int32_t* perm, const int32_t* box_start, int32_t n_boxes,
                const int32_t* nbr_start, const int32_t* nbr_idx, int32_t n_nbr, void* ws,
                cudaStream_t s);
// strength2 (Helmholtz, optional): right-hand sides from p->split on are conj(strength2)
int restructure(Plan* p, const float* pos, const void* strength, void* ws, cudaStream_t s,
                const void* strength2 = nullptr);
// adjoint records: Helmholtz [pos | q | gbar] (a = q, b = gbar), gravity [pos m | gphi gacc]
// (a = mass, b = grad_phi, c = grad_acc); returns the record width in words via *words
int restructure_adjoint(Plan* p, const float* pos, const void* a, const void* b, const void* c, void* ws,
                        int* words, cudaStream_t s);
int launch_helmholtz_adjoint_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float k, bool precise,
                                    float2* grad_q, float* grad_x, cudaStream_t s);
int launch_gravity_adjoint_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float eps, float* grad_m,
                                  float* grad_x, cudaStream_t s);
int gravity_adjoint_targets_per_lane(const Plan* p);
bool helmholtz_needs_precise(const Plan* p, float k);
inline int helmholtz_adjoint_words(int nrhs) { return 1 + 2 * ((nrhs + 1) / 2); }
constexpr int kGravityAdjointWords = 2;
// work items of up to tt targets (tt = 32 * the kernel's targets per lane)
int build_items(Plan* p, void* ws, int tt, cudaStream_t s);
// pair tasks: task list, task stream and the reductions of the partial results
int pairtask_restructure(Plan* p, void* ws, int words, cudaStream_t s);
int pairtask_reduce_gravity(const Plan* p, void* ws, float* phi, float* acc, cudaStream_t s);
int pairtask_reduce_helmholtz(const Plan* p, void* ws, float2* u, cudaStream_t s);
// symmetric plans on target-owned layouts: add the source sums of the mutual
// entries (written by other boxes' items) to the outputs
int sym_fixup_gravity(const Plan* p, void* ws, float* phi, float* acc, cudaStream_t s);
int sym_fixup_helmholtz(const Plan* p, void* ws, float2* u, cudaStream_t s);
// pair-task family: plain pair tasks or symmetric tasks
inline bool is_pairtask(int layout) { return layout == P2P_LAYOUT_PAIRTASK || layout == P2P_LAYOUT_SYMMETRIC; }
// the largest box a mutual task holds in one work item (two targets per lane)
constexpr int kMutualMax = 64;
// symmetric task kinds per neighbour entry (P2P_ARR_TASK_KIND)
constexpr int kTaskNone = 0, kTaskSelf = 1, kTaskMutual = 2, kTaskOneSided = 3;
// floats of partial result per (task, target)
inline int pairtask_part_floats(int kind, int nrhs) { return kind == P2P_GRAVITY ? 4 : 2 * nrhs; }
int helmholtz_targets_per_lane(const Plan* p, float k);
int launch_gravity_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float eps, float* phi, float* acc,
                          cudaStream_t s);
// u: RHS r < split -> u[r]; r >= split -> u2[r - split], conjugated
struct HelmOut {
    float2* u;
    float2* u2;
    int split;
};
int launch_helmholtz_kernel(const Plan* p, const LoopArgs& a, const int32_t* perm, float k, HelmOut out,
                            cudaStream_t s);
// pattern mode: table of 4 pi G(lattice displacement) and the table-lookup kernel
constexpr int kPatternMaxEntries = 4608;
int pattern_setup(Plan* p, float h, int t);
int launch_helmholtz_pattern(const Plan* p, const LoopArgs& a, const int32_t* perm, float k, float2* table,
                             HelmOut out, cudaStream_t s);

// records
inline int helmholtz_rec_words(int nrhs) { return 1 + (nrhs + 1) / 2; }
// Helmholtz records of plans with four or more right-hand sides (direct
// evaluation) hold each pair of right-hand sides planar in its word,
// [Re q_a, Re q_b, Im q_a, Im q_b]; otherwise interleaved, [Re q_a, Im q_a, Re q_b, Im q_b]
inline bool helmholtz_planar(const Plan* p) { return p->kind == P2P_HELMHOLTZ && p->nrhs >= 4 && !p->pattern; }

}  // namespace p2p
