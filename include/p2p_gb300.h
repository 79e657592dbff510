/*
 * p2p_gb300.h -- C ABI of the GB300 (sm_103a) near-field (P2P) library.
 *
 * The library computes the near-field operator of the Multilevel Fast
 * Multipole Algorithm (MLFMA): for every leaf box of a uniform octree, the
 * direct pairwise kernel is summed over the particles of the box's E2
 * neighbourhood (the <= 27 same-level boxes at Chebyshev distance <= 1,
 * itself included).  It follows the paper's P2P pipeline (Section 3.2,
 * Proposition 2, Eq. 2: collect -> transfer -> compute -> update), with the
 * collect step done on the device, and offers both data layouts the paper
 * compares (Section 5.2.1):
 *
 *   P2P_LAYOUT_INDIRECT   sources read through the box bounds and neighbour
 *                         lists from the box-ordered particle array
 *                         (the "Indexing" implementation);
 *   P2P_LAYOUT_REDUNDANT  a restructuring pass first copies every box's
 *                         neighbour sources into one contiguous per-box
 *                         stream (the "Redundant" implementation, data
 *                         duplicated so that each worker reads one
 *                         contiguous block);
 *   P2P_LAYOUT_PAIRTASK   the thread-level form of the redundant design: one
 *                         task per (target box, source box) interaction,
 *                         whose record block holds the target box's
 *                         particles followed by the source box's (array of
 *                         structures, both attributes per task, Section
 *                         5.2.1); every task writes its own partial results
 *                         and a deterministic reduction in neighbour order
 *                         adds them per target afterwards (results
 *                         duplicated, then reduced, Section 1.1);
 *   P2P_LAYOUT_SYMMETRIC  pair tasks over unordered box pairs: where one box
 *                         of a pair fits one work item (<= 64 particles), a
 *                         single "mutual" task evaluates each of its pairs
 *                         once and credits both particles (the kernel is
 *                         symmetric in the two particles), writing the
 *                         partials of both boxes; other pairs get one
 *                         one-sided task per direction, each box one self
 *                         task; the same ordered reduction follows.
 *
 * Kernels (the paper names the physics, Sections 5.1 and 5.2, not formulas;
 * these are the library's definitions):
 *   gravity    phi_i = - sum_{j in near(i), j != i} m_j (r_ij^2 + eps^2)^(-1/2)
 *              a_i   =   sum_{j in near(i), j != i} m_j (x_j - x_i)(r_ij^2 + eps^2)^(-3/2)
 *   Helmholtz  u_i   =   sum_{j in near(i), j != i} q_j exp(i k r_ij) / (4 pi r_ij)
 *              for each of nrhs right-hand sides.
 * The excluded term is the self pair; for Helmholtz on distinct points this
 * is exactly the r = 0 term.  Two distinct particles at the same position
 * are outside the Helmholtz operator's domain (and outside gravity's when
 * eps = 0).
 *
 * Conventions
 *  - Every array argument is a DEVICE pointer owned by the caller, unless
 *    the comment says "host".  The library allocates no device memory: it
 *    works inside one caller-provided workspace whose size
 *    p2p_plan_workspace_bytes() returns.  Workspace base must be 256-byte
 *    aligned; array arguments must be aligned to their element type (float2
 *    arrays to 8 bytes).
 *  - Inputs and outputs are in ORIGINAL particle order.  Positions are
 *    float32 [n][3] row-major; masses float32 [n]; complex data is complex64
 *    (interleaved re, im float32) laid out [nrhs][n].
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All work is enqueued asynchronously on it; no call
 *    synchronises with the host except p2p_read_counters() and
 *    p2p_plan_timing().  No call performs a host<->device copy on the hot
 *    path, so a sequence of calls can be captured into a CUDA graph.
 *  - Errors: argument checks are synchronous and return a status.  Errors the
 *    device detects (a position outside the boxing domain, an expired
 *    bounded wait) set bits in a flag word in the workspace header, read with
 *    p2p_read_counters().  No call aborts, traps or throws.
 *  - Thread-compatible: distinct plans may be used concurrently; one plan
 *    must not be used by two host threads at once.
 */
#ifndef P2P_GB300_H
#define P2P_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define P2P_ABI_VERSION 1

typedef enum {
    P2P_OK = 0,
    P2P_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment or option        */
    P2P_ERR_CUDA = 2,          /* a CUDA runtime call failed                     */
    P2P_ERR_OOM = 3,           /* host allocation failed                         */
    P2P_ERR_TIMEOUT = 4,       /* a bounded device wait expired                  */
    P2P_ERR_UNSUPPORTED = 5,   /* valid request this build does not handle       */
    P2P_ERR_DOMAIN = 6,        /* a position lies outside the boxing domain      */
    P2P_ERR_WORKSPACE = 7,     /* workspace missing, misaligned or too small     */
    P2P_ERR_STATE = 8,         /* call out of order (e.g. operator before tree)  */
    P2P_ERR_BOUNDS = 9         /* checked builds: an index check failed and the  */
                               /* access was skipped (results are incomplete)    */
} p2p_status;

typedef enum { P2P_GRAVITY = 0, P2P_HELMHOLTZ = 1 } p2p_kernel_kind;
typedef enum {
    P2P_LAYOUT_INDIRECT = 0,
    P2P_LAYOUT_REDUNDANT = 1,
    P2P_LAYOUT_AUTO = 2,       /* batches only: the autotuner picks indirect or redundant */
    P2P_LAYOUT_PAIRTASK = 3,   /* single plans only; forward operators only               */
    P2P_LAYOUT_SYMMETRIC = 4   /* as pair tasks; Helmholtz: nrhs <= 2, hardware sin/cos,
                                  compensated; 2 targets per lane                         */
} p2p_layout;

/* plan flags */
#define P2P_PLAN_GATHER_MAP  0x1u  /* restructuring also writes the gather map      */
#define P2P_PLAN_PLAIN_FP32  0x2u  /* plain FP32 accumulation (default: compensated) */
#define P2P_PLAN_TIMING      0x4u  /* record CUDA events around each phase           */
#define P2P_PLAN_ADJOINT     0x8u  /* size the workspace for the adjoint records     */
#define P2P_PLAN_PERIODIC    0x10u /* toroidal boundaries: neighbour cells wrap and  */
                                   /* a wrapped neighbour's sources interact through */
                                   /* their image one domain edge away (level >= 2)  */
#define P2P_PLAN_SYMMETRIC   0x20u /* indirect / redundant layouts: each pair of a   */
                                   /* box pair in which one box holds <= 64          */
                                   /* particles is evaluated once and credited to    */
                                   /* both particles (see P2P_ARR_TASK_KIND); forward */
                                   /* operators only; Helmholtz nrhs <= 2, hardware  */
                                   /* sine/cosine range, compensated; 2 targets/lane */
#define P2P_PLAN_HOST_IO     0x40u /* the workspace also holds device copies of the */
                                   /* inputs and outputs for p2p_*_host; the plan   */
                                   /* creates a second stream for input copies on   */
                                   /* the first such call (destroyed with the plan) */

/* device flag bits (p2p_read_counters: counters[P2P_CTR_FLAGS]) */
#define P2P_FLAG_DOMAIN   0x1u     /* a position was outside the domain             */
#define P2P_FLAG_TIMEOUT  0x2u     /* a bounded wait expired in a kernel             */
#define P2P_FLAG_CAPACITY 0x4u     /* an imported structure overflowed a workspace   */
                                   /* array; the affected step was skipped          */
#define P2P_FLAG_LATTICE  0x8u     /* pattern mode: a point is off the grid lattice */
                                   /* or its box; the operator call was skipped     */
#define P2P_FLAG_BOUNDS   0x10u    /* checked builds: an index was outside its array */

/* limits of this build */
#define P2P_MAX_N      (1LL << 26) /* particles per plan (27 n must fit in int32)   */
#define P2P_MAX_N_PAIRTASK (1LL << 25) /* pair-task and symmetric plans (54 n must fit in int32) */
#define P2P_MAX_LEVEL  10          /* octree levels (30-bit Morton keys)            */
#define P2P_MAX_NRHS   16

typedef struct p2p_plan p2p_plan;

/* Human-readable name of a status code (static storage). */
const char* p2p_status_string(int status);

/* ABI version (P2P_ABI_VERSION). */
int p2p_abi_version(void);

/*
 * Create a plan (host memory only).  The plan fixes the problem shape:
 *   kind    P2P_GRAVITY or P2P_HELMHOLTZ
 *   n       particles, 1 <= n <= P2P_MAX_N
 *   level   octree level, 1..P2P_MAX_LEVEL; 8^level leaf boxes
 *   lo      host float[3], lower corner of the boxing cube
 *   edge    edge length of the boxing cube (> 0); a point's box per axis is
 *           min(floor((x - lo) * s), 2^level - 1) with s = (float)2^level / edge,
 *           evaluated in float32 as written (one subtraction, one product);
 *           points with (x - lo) * s outside [0, 2^level] are out of domain
 *   nrhs    right-hand sides (Helmholtz, 1..P2P_MAX_NRHS; must be 1 for gravity)
 *   layout  P2P_LAYOUT_INDIRECT, P2P_LAYOUT_REDUNDANT, P2P_LAYOUT_PAIRTASK or
 *           P2P_LAYOUT_SYMMETRIC (pair-task and symmetric plans: n <=
 *           P2P_MAX_N_PAIRTASK, no P2P_PLAN_ADJOINT; symmetric Helmholtz
 *           plans: nrhs <= 2)
 *   flags   P2P_PLAN_* bits
 * Returns P2P_ERR_INVALID_ARG on a bad shape, P2P_ERR_OOM if the host
 * allocation fails.  *out is NULL on failure.
 */
int p2p_plan_create(p2p_plan** out, int kind, int64_t n, int level, const float* lo,
                    float edge, int nrhs, int layout, unsigned flags);

/* Release a plan (NULL is a no-op).  Does not touch device memory. */
int p2p_plan_destroy(p2p_plan* plan);

/* Bytes of device workspace the plan needs (host out-pointer). */
int p2p_plan_workspace_bytes(const p2p_plan* plan, size_t* bytes);

/*
 * Tuning knobs (the autotuner's search space, Section 3.5: threads per box
 * and redundancy grain).  targets_per_lane: 1, 2 or 4 targets held in
 * registers by each lane; a gravity work item is 32*targets_per_lane targets
 * of one box.  Helmholtz items hold at most 64 targets: with 4, a lane holds
 * four of them and takes every other source of a tile (two source groups per
 * warp; one-sided compensated passes of one or two right-hand sides, others
 * run as with 2; symmetric plans take 2).  tile: source records per shared-memory stage (32, 48,
 * 64 or 128; records wider than 16 bytes reduce it until a stage holds at
 * most 160 words, 32 at least).  ctas_per_sm: 0 = as many as fit.  warps_per_item: 1, 2 or 4 warps
 * share one item, splitting its source tiles and adding their partial sums
 * in warp order.  Returns P2P_ERR_INVALID_ARG on values outside these sets.
 */
int p2p_plan_set_tuning(p2p_plan* plan, int targets_per_lane, int tile, int ctas_per_sm,
                        int warps_per_item);

/*
 * Pattern mode for regular grids (Helmholtz): the precomputed-pattern P2P of
 * the DBIM solver (Section 5.1).  Every particle must sit on the lattice
 * lo + (i + 1/2) h (per axis, i integer) and every leaf box must hold
 * points_per_box lattice points per edge (edge / 2^level = points_per_box * h).
 * G is then tabulated once per wavenumber for the (4 points_per_box - 1)^3
 * lattice displacements between neighbouring boxes, in double precision at
 * the ideal lattice distances, and the kernel reads it from shared memory
 * instead of evaluating rsqrt/sin/cos per pair.  Particles off the lattice
 * (by more than 1 % of h) or outside their lattice box set P2P_FLAG_LATTICE
 * during p2p_restructure and the next operator call computes nothing.
 * points_per_box in 1..4 (the table must fit in shared memory); 0 disables.
 * Takes effect at the next p2p_restructure.
 */
int p2p_plan_set_grid(p2p_plan* plan, float h, int points_per_box);

/*
 * Collect, part 1 -- build the leaf-box structure from positions:
 * Morton keys, stable radix sort of (key, original index), box bounds (CSR
 * over the sorted particles, non-empty boxes in ascending key), and each
 * box's E2 neighbour list (ascending key).  pos: float32 [n][3] (device).
 * Clears the device flag word first.  Out-of-domain points set
 * P2P_FLAG_DOMAIN.  Results stay in the workspace; p2p_plan_array() locates
 * them.
 */
int p2p_tree_build(p2p_plan* plan, const float* pos, void* ws, size_t ws_bytes, void* stream);

/*
 * Collect, alternative -- import a caller-built leaf-box structure (the
 * paper's statement of the problem: leaf-box bounds and neighbour lists in).
 * All arrays device, int32:
 *   perm[n]                   sorted position -> original particle index
 *   box_start[n_boxes+1]      CSR bounds of each box in sorted order
 *   nbr_start[n_boxes+1]      CSR bounds of each box's neighbour list
 *   nbr_idx[nbr_start[n_boxes]] neighbour box indices
 * box_key may be NULL (it is only used by p2p_tree_build itself).  The
 * neighbour relation must be symmetric and each list must contain the box
 * itself and be ascending; the library does not verify this.
 */
int p2p_tree_import(p2p_plan* plan, const int32_t* perm, const int32_t* box_start,
                    int32_t n_boxes, const int32_t* nbr_start, const int32_t* nbr_idx,
                    int32_t n_nbr, void* ws, size_t ws_bytes, void* stream);

/*
 * Collect, part 2 -- restructuring.  Gathers positions and source strengths
 * into box order (every layout), and for P2P_LAYOUT_REDUNDANT copies each
 * box's neighbour sources into one contiguous stream (Section 5.2.1), plus
 * the gather map if P2P_PLAN_GATHER_MAP.  For P2P_LAYOUT_PAIRTASK it lists
 * the tasks (one per neighbour-list entry e = (b, c)), and copies task e's
 * block [records of b | records of c] to offset pt_start[e] of the task
 * stream; the gather map then holds the sorted index of every copied record.
 * P2P_LAYOUT_SYMMETRIC lists its tasks the same way, one per entry that holds
 * a task (P2P_ARR_TASK_KIND: 0 = none, the mirror entry's mutual task covers
 * the pair; 1 = self, block [records of b]; 2 = mutual; 3 = one-sided).
 *   pos        float32 [n][3]
 *   strength   gravity: float32 mass [n]; Helmholtz: complex64 q [nrhs][n]
 */
int p2p_restructure(p2p_plan* plan, const float* pos, const void* strength, void* ws,
                    size_t ws_bytes, void* stream);

/*
 * Compute + update -- softened gravity.  Needs p2p_tree_build (or import) and
 * p2p_restructure on this workspace first.  Writes phi float32 [n] and acc
 * float32 [n][3] in original particle order.  eps >= 0 (float32).
 * Pair-task plans: the kernel writes one partial result per (task, target)
 * and a reduction pass adds each target's partials in neighbour-list order
 * (symmetric plans: the same, with mutual tasks writing both boxes' partials).
 */
int p2p_gravity(p2p_plan* plan, float eps, float* phi, float* acc, void* ws, size_t ws_bytes,
                void* stream);

/*
 * Compute + update -- Helmholtz.  Writes u complex64 [nrhs][n] in original
 * order.  k is the float32 wavenumber.  When |k| * r_max <= 32, with
 * r_max = 2 sqrt(3) x box edge (the largest distance between points of
 * neighbouring boxes), the sine and cosine use the hardware approximation
 * (its error grows with the phase; the parity tests cover phases up to 31.6
 * at the complex64 tolerance); otherwise the accurate library routines.
 * Pair-task plans reduce partial results as p2p_gravity.
 * Symmetric plans need the hardware sine/cosine range and compensated
 * accumulation (otherwise P2P_ERR_UNSUPPORTED).
 */
int p2p_helmholtz(p2p_plan* plan, float k, void* u, void* ws, size_t ws_bytes, void* stream);

/*
 * Adjoint of p2p_helmholtz: gradients of a real loss L given gbar = dL/du
 * (complex convention: dL/dRe + i dL/dIm, as PyTorch).  Pair terms are
 * recomputed (nothing from the forward call is reused but the tree):
 *   grad_q_k   = sum_{j in near(k), j != k} conj(G(x_k - x_j)) gbar_j
 *   grad_pos_k = Re sum_{j in near(k), j != k} sum_r (conj(gbar_k) q_j + conj(gbar_j) q_k)
 *                   G (i k - 1/r) (x_k - x_j)/r,     r = |x_k - x_j|
 * This is the gradient the DBIM inverse solver (Section 5.1) needs.
 *   pos       float32 [n][3]; q complex64 [nrhs][n] (needed only for grad_pos)
 *   gbar      complex64 [nrhs][n]
 *   grad_q    complex64 [nrhs][n] or NULL;  grad_pos float32 [n][3] or NULL
 * With grad_pos == NULL this is the forward operator with k -> -k on gbar.
 * Pair-task and symmetric plans return P2P_ERR_UNSUPPORTED (as does
 * p2p_gravity_adjoint).
 * With grad_pos the plan must have P2P_PLAN_ADJOINT (else
 * P2P_ERR_UNSUPPORTED).  Needs the tree; overwrites the restructured
 * records, so run p2p_restructure again before the next p2p_helmholtz.
 */
int p2p_helmholtz_adjoint(p2p_plan* plan, float k, const float* pos, const void* q, const void* gbar,
                          void* grad_q, float* grad_pos, void* ws, size_t ws_bytes, void* stream);

/*
 * Adjoint of p2p_gravity, given grad_phi = dL/dphi [n] and grad_acc = dL/da
 * [n][3] (float32): with d = x_j - x_k, h^2 = r^2 + eps^2,
 *   grad_mass_k = sum_j [ -grad_phi_j h^-1 - (grad_acc_j . d) h^-3 ]
 *   grad_pos_k  = sum_j [ -h^-3 d (grad_phi_k m_j + grad_phi_j m_k)
 *                         + h^-3 v - 3 h^-5 d (d . v) ],  v = m_k grad_acc_j - m_j grad_acc_k
 * over j in near(k), j != k.  grad_mass [n] / grad_pos [n][3] may be NULL
 * (not both).  The plan must have P2P_PLAN_ADJOINT.  Needs the tree;
 * overwrites the restructured records.
 */
int p2p_gravity_adjoint(p2p_plan* plan, float eps, const float* pos, const float* mass,
                        const float* grad_phi, const float* grad_acc, float* grad_mass,
                        float* grad_pos, void* ws, size_t ws_bytes, void* stream);

/*
 * Batched near field: many independent Helmholtz instances (uneven sizes and
 * box occupancies) with nrhs right-hand sides each, run by ONE persistent
 * kernel over a work list spanning all instances, optionally captured in a
 * CUDA graph.  This answers the many small launches of the paper's PhotoNs
 * port (Section 5.2, Section 5.2.3 item 4); each instance's tree is built once
 * because the geometry is fixed across solver iterations (Section 5.1).
 *
 * Data of the batch is CONCATENATED: instance i owns particles
 * [off_i, off_i + n_i) of every array (off = prefix sums of n); positions are
 * float32 [N][3]; right-hand sides complex64 [nrhs][N].
 *
 *   p2p_batch_create   host only.  n/level/edge: host arrays [n_instances];
 *                      lo: host float [n_instances][3] (boxing domain of each
 *                      instance, as for p2p_plan_create).  pair != 0: every
 *                      run computes the forward product u = P q AND the
 *                      adjoint product g = conj(P) y (one operator of 2 nrhs
 *                      right-hand sides, since conj(P) y = conj(P conj y)).
 *                      layout: INDIRECT, REDUNDANT or AUTO (the workspace
 *                      holds redundant streams; p2p_batch_autotune chooses).
 *                      flags: 0, P2P_PLAN_PLAIN_FP32 and/or
 *                      P2P_PLAN_TIMING (phase events, p2p_batch_timing).
 *                      Helmholtz only (P2P_ERR_UNSUPPORTED otherwise).
 *   p2p_batch_build    builds every instance's tree and merges them into one
 *                      box structure; synchronises the stream once per
 *                      instance (set-up, not the hot path).
 *   p2p_batch_run      restructuring + one operator launch for all
 *                      instances: u [nrhs][N] (and g [nrhs][N] if pair).
 *   p2p_batch_set_tuning / p2p_batch_autotune
 *                      the tuning space (layout, targets per lane, tile,
 *                      warps per item); the autotuner times every candidate
 *                      with CUDA events on the given buffers, keeps the
 *                      fastest and returns best[5] = {layout, targets/lane,
 *                      tile, ctas/SM, warps/item} and its time; synchronises.
 *   p2p_batch_capture  captures p2p_batch_run on these buffers into a CUDA
 *                      graph (on an internal stream); p2p_batch_launch then
 *                      replays it on any stream.
 */
typedef struct p2p_batch p2p_batch;
int p2p_batch_create(p2p_batch** out, int kind, int n_instances, const int64_t* n, const int* level,
                     const float* lo, const float* edge, int nrhs, int pair, int layout, unsigned flags);
int p2p_batch_destroy(p2p_batch* batch);
int p2p_batch_workspace_bytes(const p2p_batch* batch, size_t* bytes);
int p2p_batch_build(p2p_batch* batch, const float* pos, void* ws, size_t ws_bytes, void* stream);
int p2p_batch_set_tuning(p2p_batch* batch, int layout, int targets_per_lane, int tile, int ctas_per_sm,
                         int warps_per_item);
int p2p_batch_run(p2p_batch* batch, float k, const float* pos, const void* q, const void* y, void* u,
                  void* g, void* ws, size_t ws_bytes, void* stream);
int p2p_batch_autotune(p2p_batch* batch, float k, const float* pos, const void* q, const void* y,
                       void* u, void* g, void* ws, size_t ws_bytes, void* stream, int* best,
                       float* best_ms);
int p2p_batch_capture(p2p_batch* batch, float k, const float* pos, const void* q, const void* y,
                      void* u, void* g, void* ws, size_t ws_bytes);
int p2p_batch_launch(p2p_batch* batch, void* stream);
/* counters of the combined structure (as p2p_read_counters; pairs are geometric) */
int p2p_batch_counters(const p2p_batch* batch, const void* ws, int64_t* out, void* stream);
/* Milliseconds of the last run's phases (batches created with
 * P2P_PLAN_TIMING), as p2p_plan_timing: RESTRUCTURE, KERNEL (every
 * right-hand-side pass of the P2P kernel) and OPERATOR (work list + kernel);
 * TREE is -1 (the trees are built once, by p2p_batch_build).  Inside a
 * captured graph the events are external event nodes, so a replay records
 * them.  Host float ms_out[P2P_PHASE_COUNT]; waits for the events. */
int p2p_batch_timing(p2p_batch* batch, float* ms_out);

/*
 * Self-test of the bounded device waits (a library check; the paper has no
 * counterpart).  Every wait of the P2P kernels on an mbarrier gives up after
 * ~2 s of global time, records P2P_FLAG_TIMEOUT and lets its copies land
 * before the warp leaves, so a lost signal can never hang the GPU.  This
 * call runs one warp waiting on an mbarrier that nothing completes, with a
 * limit of limit_ns (1 .. 1e10): it returns P2P_ERR_TIMEOUT when the wait
 * expired as designed (P2P_OK would mean the mechanism is broken).  flags_dev
 * is a caller-owned device uint32 (overwritten).  Synchronises the stream.
 */
int p2p_selftest_bounded_wait(uint64_t limit_ns, uint32_t* flags_dev, void* stream);

/*
 * Testing aids.
 * p2p_build_checked: 1 if this library was built with device index checks
 * (P2P_CHECKED: every work item's ranges, slots and output indices, the
 * stream and partial-slot writes are checked; a failed check sets
 * P2P_FLAG_BOUNDS and skips the access instead of faulting), else 0.
 * p2p_fail_host_allocs: the next `count` host allocations of plan and batch
 * creation fail (they return P2P_ERR_OOM); 0 clears.  Returns P2P_OK.
 */
int p2p_build_checked(void);
int p2p_fail_host_allocs(int count);

/*
 * One step from host buffers (plans created with P2P_PLAN_HOST_IO), the
 * paper's transfer phase included: copies the positions (float [n][3]) and
 * strengths (gravity: float [n]; Helmholtz: complex64 [nrhs][n]) from host
 * memory into the workspace, builds the tree, restructures, evaluates, and
 * copies the results back (gravity: phi float [n], acc float [n][3];
 * Helmholtz: u complex64 [nrhs][n]).  The strengths' copy runs on a stream
 * of the plan's own, overlapped with the tree build.  All host pointers are
 * caller-owned; page-locked buffers let the copies run asynchronously
 * (pageable ones work, with synchronous copies).  Asynchronous on `stream`:
 * the results are in host memory once the stream has passed this call.
 * Returns P2P_ERR_UNSUPPORTED for plans without P2P_PLAN_HOST_IO, and the
 * statuses of p2p_tree_build / p2p_restructure / the operator.
 */
int p2p_gravity_host(p2p_plan* plan, float eps, const float* pos, const float* mass, float* phi, float* acc,
                     void* ws, size_t ws_bytes, void* stream);
int p2p_helmholtz_host(p2p_plan* plan, float k, const float* pos, const void* q, void* u, void* ws,
                       size_t ws_bytes, void* stream);

/* identifiers of workspace arrays for p2p_plan_array */
typedef enum {
    P2P_ARR_PERM = 0,        /* int32 [n]               sorted -> original index    */
    P2P_ARR_BOX_KEY = 1,     /* uint32 [n_boxes]        Morton key of each box       */
    P2P_ARR_BOX_START = 2,   /* int32 [n_boxes+1]       box bounds                   */
    P2P_ARR_NBR_START = 3,   /* int32 [n_boxes+1]       neighbour-list bounds        */
    P2P_ARR_NBR_IDX = 4,     /* int32 [n_nbr]           neighbour box indices        */
    P2P_ARR_RED_START = 5,   /* int32 [n_boxes+1]       redundant stream bounds      */
    P2P_ARR_RED_SELF = 6,    /* int32 [n_boxes]         own particles' stream offset */
    P2P_ARR_GATHER_IDX = 7,  /* uint32 [red_start[n_boxes]] sorted source per record */
    P2P_ARR_SORTED_KEY = 8,  /* uint32 [n]              Morton key, sorted order     */
    P2P_ARR_NBR_IMG = 9,     /* int32 [n_nbr] periodic: image code (ox+1)+3(oy+1)+9(oz+1) */
                             /* of each neighbour entry, o = image offset in domain edges */
    P2P_ARR_ENT_BOX = 10,    /* int32 [n_nbr]   pair tasks: target box of entry e  */
    P2P_ARR_PT_START = 11,   /* int32 [n_nbr+1] pair tasks: record block bounds     */
    P2P_ARR_PART_START = 12, /* int32 [n_nbr+1] pair tasks: partial-result bounds   */
    P2P_ARR_TASK_KIND = 13,  /* int32 [n_nbr]   symmetric: kind of entry e (0 none, 1 self, 2 mutual, 3 one-sided) */
    P2P_ARR_MIRROR = 14,     /* int32 [n_nbr]   symmetric: entry (c -> b) of an entry (b -> c) without a task */
    P2P_ARR_BSLOT = 15,      /* int32 [n_nbr]   P2P_PLAN_SYMMETRIC: first slot of a mutual entry's source sums */
    P2P_ARR_COUNT = 16
} p2p_array_id;

/*
 * Where a workspace array lives: *offset_bytes from the workspace base and
 * *capacity elements reserved (the used length is given by the counters).
 * Returns P2P_ERR_UNSUPPORTED for an array the plan does not keep (the
 * gather map without P2P_PLAN_GATHER_MAP; redundant arrays for the indirect
 * layout; pair-task arrays for the other layouts).  For pair-task plans
 * P2P_ARR_GATHER_IDX covers the task stream (pt_start[n_nbr] records).
 */
int p2p_plan_array(const p2p_plan* plan, int which, int64_t* offset_bytes, int64_t* capacity);

/* counters of the workspace header (p2p_read_counters) */
typedef enum {
    P2P_CTR_N_BOXES = 0,     /* non-empty leaf boxes                        */
    P2P_CTR_N_NBR = 1,       /* neighbour-list entries E                    */
    P2P_CTR_FLAGS = 2,       /* P2P_FLAG_* bits                             */
    P2P_CTR_TOTAL_SRC = 3,   /* redundant records sum_b S_b (pair tasks: task-stream records) */
    P2P_CTR_PAIRS = 4,       /* ordered pairs sum_b n_b S_b - n (last op)   */
    P2P_CTR_N_ITEMS = 5,     /* work items of the last operator call        */
    P2P_CTR_EVALS = 6,       /* pair evaluations: P2P_CTR_PAIRS, but a mutual evaluation of a */
                             /* symmetric plan counts once for its two ordered pairs          */
    P2P_CTR_COUNT = 7
} p2p_counter_id;

/*
 * Copy the header counters to host int64 out[P2P_CTR_COUNT] and synchronise
 * the stream.  Returns P2P_ERR_DOMAIN / P2P_ERR_TIMEOUT if the flag word has
 * the matching bit set (the counters are still written).
 */
int p2p_read_counters(const p2p_plan* plan, const void* ws, int64_t* out, void* stream);

/* phases timed when the plan has P2P_PLAN_TIMING */
typedef enum {
    P2P_PHASE_TREE = 0,        /* p2p_tree_build                                 */
    P2P_PHASE_RESTRUCTURE = 1, /* p2p_restructure (adjoints: their records)      */
    P2P_PHASE_KERNEL = 2,      /* the P2P compute kernel alone (operator or      */
                               /* adjoint, whichever ran last)                   */
    P2P_PHASE_OPERATOR = 3,    /* p2p_gravity / p2p_helmholtz / an adjoint call  */
                               /* as a whole (work list + kernel + reduction)    */
    P2P_PHASE_COUNT = 4
} p2p_phase_id;

/*
 * Milliseconds of each phase's last run (host float out[P2P_PHASE_COUNT]),
 * measured with CUDA events on the launching stream; waits for the events.
 * A phase not run since the plan was created reports -1.
 */
int p2p_plan_timing(p2p_plan* plan, float* ms_out);

/* Number of kernels this library has launched in this process (all plans). */
int64_t p2p_launch_count(void);

/*
 * Measured peak rates of the pipes that bind the P2P kernels (a measurement
 * utility, not part of the operator; it allocates its own small scratch and
 * synchronises).  On the current device, one CTA of 1024 threads per SM runs
 * independent chains of one instruction kind; host double out[5]:
 *   out[0]  FP32 FFMA lane-operations per SM per clock
 *   out[1]  MUFU rsqrt.approx lane-operations per SM per clock
 *   out[2]  MUFU sin.approx lane-operations per SM per clock
 *   out[3]  SM clock in MHz during the FFMA run (clock64 span / event time)
 *   out[4]  packed fma.rn.f32x2: FP32 lane-operations (two per instruction
 *           and lane) per SM per clock
 */
int p2p_measure_pipes(double* out, void* stream);

/*
 * Double-precision check reductions on the device (the paper has no
 * counterpart; the operator computes in FP32 and only these global sums
 * accumulate in FP64).  One block reads the whole array; the sums are added
 * in a fixed order (deterministic).  Asynchronous on `stream`.
 *
 * p2p_momentum_fp64: the momentum invariant of the gravity near field.
 *   mass float32 [n], acc float32 [n][3] (device, e.g. the inputs and the
 *   output of p2p_gravity); out double [6] (device):
 *   out[c] = sum_i m_i a_i[c], out[3 + c] = sum_i |m_i a_i[c]|, c = x, y, z.
 *   The first three vanish in exact arithmetic (the neighbour relation is
 *   symmetric and the softened kernel's gradient is odd, also across
 *   periodic images).
 * p2p_dot_fp64: out double [1] (device) = sum_i x_i y_i over `count` float32
 *   values.  On complex64 arrays viewed as 2 count floats this is
 *   Re sum_i conj(x_i) y_i, the inner product of the adjoint identity
 *   Re<P q, y> = Re<q, P^H y> (p2p_helmholtz_adjoint gives P^H y).
 */
int p2p_momentum_fp64(const float* mass, const float* acc, int64_t n, double* out, void* stream);
int p2p_dot_fp64(const float* x, const float* y, int64_t count, double* out, void* stream);

/*
 * Gravity near field for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a library convenience.
 *
 * Some callers cannot call cudaMalloc where they need the operator (code
 * under an allocator that forbids new device allocations, a plugin given
 * only its input and output buffers, a pre-planned sequence that must not
 * gain allocation calls).  This entry point runs the same pipeline and
 * kernels as p2p_tree_build + p2p_restructure + p2p_gravity, with all scratch
 * in one fixed device array inside the library, and allocates nothing.
 *   pos float32 [n][3], mass float32 [n]   inputs (device, original order)
 *   phi float32 [n], acc float32 [n][3]    outputs (device, original order)
 *   level, lo (host float[3]), edge, eps, layout as for p2p_plan_create /
 *   p2p_gravity.
 * Limits: n <= P2P_NOALLOC_MAX_N, level <= P2P_NOALLOC_MAX_LEVEL; larger
 * requests return P2P_ERR_UNSUPPORTED without touching the device.  The
 * scratch (P2P_NOALLOC_SCRATCH_BYTES) exists on every GPU that loads the
 * library, until the process exits.
 * The set-up, workspace layout and kernels are those of a plan created
 * with the same arguments and flags 0 (default tuning), so the results equal
 * the workspace path's bit for bit; the scratch needed is that plan's
 * p2p_plan_workspace_bytes, which for every n, level and layout within the
 * limits is at most P2P_NOALLOC_SCRATCH_BYTES.
 * Every call looks up the scratch array's device address with
 * cudaGetSymbolAddress in the current context; the first call on a device
 * also loads the library's module there, so make that first call before any
 * stream capture.  Every call shares the one array and leaves its contents
 * behind; the call clears what it needs.  Calls whose GPU work overlaps
 * (different streams or host threads) race on the scratch.
 * Errors the device detects (a position outside the boxing domain or NaN, an
 * expired bounded wait) are not in the return value: the call only queues
 * the work.  Read them with p2p_gravity_noalloc_status.
 */
#define P2P_NOALLOC_MAX_N 8192
#define P2P_NOALLOC_MAX_LEVEL 4
#define P2P_NOALLOC_SCRATCH_BYTES (4718592)  /* 4.5 MiB */
int p2p_gravity_noalloc(const float* pos, const float* mass, int64_t n, int level, const float* lo,
                        float edge, float eps, int layout, float* phi, float* acc, void* stream);

/*
 * Status of the last p2p_gravity_noalloc call on the current device: waits
 * for `stream`, reads the device flag word that call left in the library's
 * scratch array (allocating nothing) and returns the status it maps to, as
 * p2p_read_counters does: P2P_ERR_DOMAIN for a position outside the boxing
 * domain (or NaN; phi and acc are then not meaningful), P2P_ERR_TIMEOUT for
 * an expired bounded wait, P2P_ERR_BOUNDS (checked builds), else P2P_OK.
 * flags: host uint32, nullable; receives the raw P2P_FLAG_* bits.
 * The paper has no counterpart.
 */
int p2p_gravity_noalloc_status(uint32_t* flags, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* P2P_GB300_H */
