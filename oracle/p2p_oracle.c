/*
 * FP64 CPU oracle for the MLFMA near-field (P2P) operator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or helper with the CUDA library, and the library never calls it.
 *
 * What it computes (readings of the paper are marked "reading"):
 *
 *  - Leaf boxes of a uniform octree of `level` levels over the cube
 *    [lo, lo+edge)^3, with boxes numbered by Morton (Z-order) key: the
 *    space-filling-curve ordering of Section 1 / Section 2.3.  Box of a point,
 *    per axis, with float32 operations exactly as written (reading):
 *        t = x - lo,  u = t * s,  s = (float)2^level / edge,
 *        cell = min(floor(u), 2^level - 1);  invalid unless 0 <= u <= 2^level.
 *    Morton key: bit b of the x, y, z cell goes to key bit 3b, 3b+1, 3b+2.
 *  - Stable sort of (key, original index) -> perm (sorted -> original).
 *  - Box CSR over the sorted particles (non-empty boxes only, ascending key).
 *  - Neighbour lists: the E2 neighbourhood of Section 5.1 / Table 5, i.e. the
 *    same-level boxes at Chebyshev cell distance <= 1 (self included), no
 *    periodic wrap, non-empty only, ascending key (reading).
 *  - The redundant layout of Section 5.2.1 (data duplicated per interaction
 *    so that a thread reads one contiguous block), restated per target box:
 *    red_start = exclusive scan of S_b = sum of the occupancies of b's
 *    neighbours, gather_idx = the sorted source indices in neighbour order.
 *  - The P2P sums (the near-field operator of Section 2.1; the paper names
 *    the physics only, the kernels are readings):
 *      gravity   (Section 5.2, stellar dynamics; G = 1, Plummer softening)
 *          phi_i = - sum_{j in near(i), j != i} m_j (r^2 + eps^2)^(-1/2)
 *          a_i   =   sum_{j in near(i), j != i} m_j (x_j - x_i) (r^2 + eps^2)^(-3/2)
 *      Helmholtz (Section 5.1, Green's function of the Helmholtz equation, 3-D)
 *          u_i   =   sum_{j in near(i), j != i} q_j exp(i k r) / (4 pi r)
 *    where near(i) = particles of the neighbour boxes of i's box.  The
 *    excluded term is the self pair (j = i), i.e. the r = 0 term (reading).
 *
 * Every sum is a plain double-precision loop over the definition; the inputs
 * are the float32 values widened exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_DOMAIN 6
#define ORC_ERR_NOMEM 3

static const double ORC_PI = 3.14159265358979323846264338327950288;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the sums' parallel loops started by the calling host thread from
 * now on (OpenMP); returns the previous count.  Used to time the oracle on one
 * core and on all cores. */
int orc_set_num_threads(int t) {
#ifdef _OPENMP
    const int old = omp_get_max_threads();
    if (t > 0) omp_set_num_threads(t);
    return old;
#else
    (void)t;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* boxing                                                                     */
/* ------------------------------------------------------------------------- */

/* One axis of the box rule (float32 ops, no contraction: built -ffp-contract=off). */
static int orc_axis_cell(float x, float lo, float s, int level, int32_t* cell) {
    float t = x - lo;
    float u = t * s;
    float side = (float)(1 << level);
    if (!(u >= 0.0f && u <= side)) return -1; /* also rejects NaN */
    int32_t c = (int32_t)floorf(u);
    if (c > (1 << level) - 1) c = (1 << level) - 1;
    *cell = c;
    return 0;
}

uint32_t orc_morton(int32_t cx, int32_t cy, int32_t cz, int level) {
    uint32_t key = 0;
    for (int b = 0; b < level; ++b) {
        key |= (uint32_t)((cx >> b) & 1) << (3 * b);
        key |= (uint32_t)((cy >> b) & 1) << (3 * b + 1);
        key |= (uint32_t)((cz >> b) & 1) << (3 * b + 2);
    }
    return key;
}

void orc_unmorton(uint32_t key, int level, int32_t* cx, int32_t* cy, int32_t* cz) {
    int32_t x = 0, y = 0, z = 0;
    for (int b = 0; b < level; ++b) {
        x |= (int32_t)((key >> (3 * b)) & 1) << b;
        y |= (int32_t)((key >> (3 * b + 1)) & 1) << b;
        z |= (int32_t)((key >> (3 * b + 2)) & 1) << b;
    }
    *cx = x; *cy = y; *cz = z;
}

/* Cells [n,3] and Morton keys [n] of every point (original order).  Returns
 * ORC_ERR_DOMAIN if any point lies outside the boxing domain. */
int orc_cells(const float* pos, int64_t n, int level, const float* lo, float edge,
              int32_t* cell, uint32_t* key) {
    if (n < 0 || level < 1 || level > 10 || !(edge > 0.0f)) return ORC_ERR_ARG;
    float s = (float)(1 << level) / edge;
    for (int64_t i = 0; i < n; ++i) {
        int32_t c[3];
        for (int a = 0; a < 3; ++a)
            if (orc_axis_cell(pos[3 * i + a], lo[a], s, level, &c[a]) != 0) return ORC_ERR_DOMAIN;
        if (cell) { cell[3 * i] = c[0]; cell[3 * i + 1] = c[1]; cell[3 * i + 2] = c[2]; }
        if (key) key[i] = orc_morton(c[0], c[1], c[2], level);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* tree: sort, box CSR, neighbour CSR                                         */
/* ------------------------------------------------------------------------- */

typedef struct { uint32_t key; int32_t idx; } orc_kv;

static int orc_kv_cmp(const void* a, const void* b) {
    const orc_kv* x = (const orc_kv*)a;
    const orc_kv* y = (const orc_kv*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static int orc_u32_cmp(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

static int orc_i32_cmp(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* index of `key` in the ascending array box_key[0..nb), or -1 */
static int32_t orc_find_box(const uint32_t* box_key, int32_t nb, uint32_t key) {
    const uint32_t* p = (const uint32_t*)bsearch(&key, box_key, (size_t)nb, sizeof(uint32_t), orc_u32_cmp);
    return p ? (int32_t)(p - box_key) : -1;
}

/*
 * Build the leaf-box structure.  Outputs (caller-allocated):
 *   perm[n]            sorted position -> original index
 *   box_key[n] (cap)   Morton key of each non-empty box, ascending
 *   box_start[n+1]     CSR bounds of each box in sorted order
 *   *n_boxes
 *   nbr_start[n+1]     CSR bounds of each box's neighbour list
 *   nbr_idx[27 n]      neighbour box indices, ascending
 *   *n_nbr             total neighbour entries E
 */
int orc_tree_ex(const float* pos, int64_t n, int level, const float* lo, float edge, int periodic,
                int32_t* perm, uint32_t* box_key, int32_t* box_start, int32_t* n_boxes,
                int32_t* nbr_start, int32_t* nbr_idx, int32_t* nbr_img, int64_t* n_nbr) {
    if (periodic && level < 2) return ORC_ERR_ARG;
    if (n <= 0) return ORC_ERR_ARG;
    uint32_t* key = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    orc_kv* kv = (orc_kv*)malloc((size_t)n * sizeof(orc_kv));
    if (!key || !kv) { free(key); free(kv); return ORC_ERR_NOMEM; }
    int st = orc_cells(pos, n, level, lo, edge, NULL, key);
    if (st != ORC_OK) { free(key); free(kv); return st; }
    for (int64_t i = 0; i < n; ++i) { kv[i].key = key[i]; kv[i].idx = (int32_t)i; }
    qsort(kv, (size_t)n, sizeof(orc_kv), orc_kv_cmp);

    int32_t nb = 0;
    for (int64_t s = 0; s < n; ++s) {
        perm[s] = kv[s].idx;
        if (s == 0 || kv[s].key != kv[s - 1].key) {
            box_key[nb] = kv[s].key;
            box_start[nb] = (int32_t)s;
            ++nb;
        }
    }
    box_start[nb] = (int32_t)n;
    *n_boxes = nb;

    int64_t e = 0;
    int32_t side = 1 << level;
    for (int32_t b = 0; b < nb; ++b) {
        int32_t cx, cy, cz;
        orc_unmorton(box_key[b], level, &cx, &cy, &cz);
        /* found[j] = box index * 32 + image code, so sorting by it orders by box */
        int32_t found[27];
        int nf = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int32_t x = cx + dx, y = cy + dy, z = cz + dz;
                    int32_t o[3] = {0, 0, 0};
                    if (periodic) {
                        /* toroidal wrap: the source image sits one domain edge away */
                        if (x < 0) { x += side; o[0] = -1; } else if (x >= side) { x -= side; o[0] = 1; }
                        if (y < 0) { y += side; o[1] = -1; } else if (y >= side) { y -= side; o[1] = 1; }
                        if (z < 0) { z += side; o[2] = -1; } else if (z >= side) { z -= side; o[2] = 1; }
                    } else if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) {
                        continue;
                    }
                    int32_t c = orc_find_box(box_key, nb, orc_morton(x, y, z, level));
                    int32_t code = (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);
                    if (c >= 0) found[nf++] = c * 32 + code;
                }
        qsort(found, (size_t)nf, sizeof(int32_t), orc_i32_cmp);
        nbr_start[b] = (int32_t)e;
        for (int j = 0; j < nf; ++j) {
            if (nbr_img) nbr_img[e] = found[j] % 32;
            nbr_idx[e++] = found[j] / 32;
        }
    }
    nbr_start[nb] = (int32_t)e;
    *n_nbr = e;
    free(key);
    free(kv);
    return ORC_OK;
}

int orc_tree(const float* pos, int64_t n, int level, const float* lo, float edge,
             int32_t* perm, uint32_t* box_key, int32_t* box_start, int32_t* n_boxes,
             int32_t* nbr_start, int32_t* nbr_idx, int64_t* n_nbr) {
    return orc_tree_ex(pos, n, level, lo, edge, 0, perm, box_key, box_start, n_boxes, nbr_start, nbr_idx,
                       NULL, n_nbr);
}

/*
 * Redundant layout (Section 5.2.1, restated per target box): for each box b,
 * its sources are the particles of its neighbour boxes, in neighbour order,
 * each box's particles in sorted order.
 *   red_start[nb+1]  exclusive scan of S_b
 *   red_self[nb]     offset of b's own particles inside its stream
 *   gather_idx[sum S_b] (optional) sorted source index of each record
 * Returns the total number of records in *total.
 */
int orc_redundant(const int32_t* box_start, int32_t nb, const int32_t* nbr_start,
                  const int32_t* nbr_idx, int32_t* red_start, int32_t* red_self,
                  uint32_t* gather_idx, int64_t* total) {
    int64_t off = 0;
    for (int32_t b = 0; b < nb; ++b) {
        red_start[b] = (int32_t)off;
        int64_t own = 0;
        for (int32_t e = nbr_start[b]; e < nbr_start[b + 1]; ++e) {
            int32_t c = nbr_idx[e];
            if (c == b && red_self) red_self[b] = (int32_t)own;
            for (int32_t s = box_start[c]; s < box_start[c + 1]; ++s) {
                if (gather_idx) gather_idx[off] = (uint32_t)s;
                ++off;
                ++own;
            }
        }
    }
    red_start[nb] = (int32_t)off;
    *total = off;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* P2P sums                                                                   */
/* ------------------------------------------------------------------------- */

/* Shared tree context used by the sums: built once per call by orc_tree. */
typedef struct {
    int64_t n;
    int32_t nb;
    int32_t* perm;
    uint32_t* box_key;
    int32_t* box_start;
    int32_t* nbr_start;
    int32_t* nbr_idx;
    int32_t* nbr_img;  /* periodic: image code of each neighbour entry, else NULL */
    int32_t* box_of;   /* original index -> box */
    double edge;
} orc_ctx;

/* shift of a neighbour entry's sources: image offset times the domain edge */
static void orc_img_shift(const orc_ctx* c, int32_t e, double* sh) {
    if (!c->nbr_img) { sh[0] = sh[1] = sh[2] = 0.0; return; }
    int32_t code = c->nbr_img[e];
    sh[0] = (double)(code % 3 - 1) * c->edge;
    sh[1] = (double)((code / 3) % 3 - 1) * c->edge;
    sh[2] = (double)(code / 9 - 1) * c->edge;
}

static void orc_ctx_free(orc_ctx* c) {
    free(c->perm); free(c->box_key); free(c->box_start);
    free(c->nbr_start); free(c->nbr_idx); free(c->nbr_img); free(c->box_of);
}

/* Tree context of one call; periodic != 0 wraps the neighbour cells and
 * records an image code per neighbour entry.  Every call builds its own
 * context, so concurrent calls (open or periodic) do not interact. */
static int orc_ctx_build(orc_ctx* c, const float* pos, int64_t n, int level, const float* lo, float edge,
                         int periodic) {
    memset(c, 0, sizeof(*c));
    c->n = n;
    c->edge = (double)edge;
    if (periodic) {
        c->nbr_img = (int32_t*)malloc((size_t)n * 27 * sizeof(int32_t));
        if (!c->nbr_img) return ORC_ERR_NOMEM;
    }
    c->perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    c->box_key = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    c->box_start = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    c->nbr_start = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    c->nbr_idx = (int32_t*)malloc((size_t)n * 27 * sizeof(int32_t));
    c->box_of = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!c->perm || !c->box_key || !c->box_start || !c->nbr_start || !c->nbr_idx || !c->box_of) {
        orc_ctx_free(c);
        return ORC_ERR_NOMEM;
    }
    int64_t e;
    int st = orc_tree_ex(pos, n, level, lo, edge, periodic, c->perm, c->box_key, c->box_start, &c->nb,
                         c->nbr_start, c->nbr_idx, c->nbr_img, &e);
    if (st != ORC_OK) { orc_ctx_free(c); return st; }
    for (int32_t b = 0; b < c->nb; ++b)
        for (int32_t s = c->box_start[b]; s < c->box_start[b + 1]; ++s) c->box_of[c->perm[s]] = b;
    return ORC_OK;
}

/*
 * Softened gravity at the listed targets (original indices; NULL = all n).
 * phi[nt], acc[nt*3] in double.  eps is the float32 softening widened.
 * Optionally counts the ordered pairs visited into *pairs.
 */
static void orc_gravity_sum(const orc_ctx* cp, const float* pos, const float* mass, float eps,
                            const int64_t* targets, int64_t nt, double* phi, double* acc, int64_t* pairs) {
    const orc_ctx c = *cp;
    if (!targets) nt = c.n;
    const double e2 = (double)eps * (double)eps;
    int64_t count = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : count)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        int32_t b = c.box_of[i];
        double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        double p = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
        for (int32_t e = c.nbr_start[b]; e < c.nbr_start[b + 1]; ++e) {
            int32_t nbox = c.nbr_idx[e];
            double sh[3];
            orc_img_shift(&c, e, sh);
            for (int32_t s = c.box_start[nbox]; s < c.box_start[nbox + 1]; ++s) {
                int64_t j = c.perm[s];
                if (j == i) continue;
                double dx = (double)pos[3 * j] + sh[0] - xi;
                double dy = (double)pos[3 * j + 1] + sh[1] - yi;
                double dz = (double)pos[3 * j + 2] + sh[2] - zi;
                double r2 = dx * dx + dy * dy + dz * dz + e2;
                double inv = 1.0 / sqrt(r2);
                double m = (double)mass[j];
                p -= m * inv;
                double w = m * inv * inv * inv;
                ax += w * dx; ay += w * dy; az += w * dz;
                ++count;
            }
        }
        phi[t] = p;
        acc[3 * t] = ax; acc[3 * t + 1] = ay; acc[3 * t + 2] = az;
    }
    if (pairs) *pairs = count;
}

static int orc_gravity_ex(const float* pos, const float* mass, int64_t n, int level, const float* lo,
                          float edge, float eps, const int64_t* targets, int64_t nt,
                          double* phi, double* acc, int64_t* pairs, int periodic) {
    orc_ctx c;
    int st = orc_ctx_build(&c, pos, n, level, lo, edge, periodic);
    if (st != ORC_OK) return st;
    orc_gravity_sum(&c, pos, mass, eps, targets, nt, phi, acc, pairs);
    orc_ctx_free(&c);
    return ORC_OK;
}

/*
 * Helmholtz near field at the listed targets (original indices; NULL = all).
 * q: complex64 sources laid out [nrhs][n][re,im] (float32); u: [nrhs][nt][re,im]
 * in double.  k is the float32 wavenumber widened.
 */
static void orc_helmholtz_sum(const orc_ctx* cp, const float* pos, const float* q, int nrhs, float k,
                              const int64_t* targets, int64_t nt, double* u, int64_t* pairs) {
    const orc_ctx c = *cp;
    const int64_t n = c.n;
    if (!targets) nt = n;
    const double kk = (double)k;
    const double inv4pi = 1.0 / (4.0 * ORC_PI);
    int64_t count = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : count)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        int32_t b = c.box_of[i];
        double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        for (int r = 0; r < nrhs; ++r) { u[2 * (r * nt + t)] = 0.0; u[2 * (r * nt + t) + 1] = 0.0; }
        for (int32_t e = c.nbr_start[b]; e < c.nbr_start[b + 1]; ++e) {
            int32_t nbox = c.nbr_idx[e];
            double sh[3];
            orc_img_shift(&c, e, sh);
            for (int32_t s = c.box_start[nbox]; s < c.box_start[nbox + 1]; ++s) {
                int64_t j = c.perm[s];
                if (j == i) continue;
                double dx = (double)pos[3 * j] + sh[0] - xi;
                double dy = (double)pos[3 * j + 1] + sh[1] - yi;
                double dz = (double)pos[3 * j + 2] + sh[2] - zi;
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                double gre = cos(kk * r) * inv4pi / r;
                double gim = sin(kk * r) * inv4pi / r;
                for (int rr = 0; rr < nrhs; ++rr) {
                    double qre = q[2 * (rr * n + j)], qim = q[2 * (rr * n + j) + 1];
                    u[2 * (rr * nt + t)] += gre * qre - gim * qim;
                    u[2 * (rr * nt + t) + 1] += gre * qim + gim * qre;
                }
                ++count;
            }
        }
    }
    if (pairs) *pairs = count;
}

static int orc_helmholtz_ex(const float* pos, const float* q, int nrhs, int64_t n, int level,
                            const float* lo, float edge, float k, const int64_t* targets, int64_t nt,
                            double* u, int64_t* pairs, int periodic) {
    if (nrhs < 1) return ORC_ERR_ARG;
    orc_ctx c;
    int st = orc_ctx_build(&c, pos, n, level, lo, edge, periodic);
    if (st != ORC_OK) return st;
    orc_helmholtz_sum(&c, pos, q, nrhs, k, targets, nt, u, pairs);
    orc_ctx_free(&c);
    return ORC_OK;
}

int orc_gravity(const float* pos, const float* mass, int64_t n, int level, const float* lo,
                float edge, float eps, const int64_t* targets, int64_t nt,
                double* phi, double* acc, int64_t* pairs) {
    return orc_gravity_ex(pos, mass, n, level, lo, edge, eps, targets, nt, phi, acc, pairs, 0);
}

int orc_helmholtz(const float* pos, const float* q, int nrhs, int64_t n, int level,
                  const float* lo, float edge, float k, const int64_t* targets, int64_t nt,
                  double* u, int64_t* pairs) {
    return orc_helmholtz_ex(pos, q, nrhs, n, level, lo, edge, k, targets, nt, u, pairs, 0);
}

/*
 * A tree context kept across calls: the same sums as orc_gravity /
 * orc_helmholtz (periodic != 0: as the *_periodic calls) at several target
 * samples on one tree, so that a caller can time the tree build and the sums
 * apart.  pos must be the positions the context was built from.
 * orc_context_new returns NULL on failure and the status in *status.
 */
void* orc_context_new(const float* pos, int64_t n, int level, const float* lo, float edge, int periodic,
                      int* status) {
    orc_ctx* c = (orc_ctx*)malloc(sizeof(orc_ctx));
    int st = c ? ORC_OK : ORC_ERR_NOMEM;
    if (c && periodic && level < 2) st = ORC_ERR_ARG;
    if (st == ORC_OK) st = orc_ctx_build(c, pos, n, level, lo, edge, periodic);
    if (status) *status = st;
    if (st != ORC_OK) { free(c); return NULL; }
    return c;
}

void orc_context_free(void* h) {
    if (!h) return;
    orc_ctx_free((orc_ctx*)h);
    free(h);
}

int orc_gravity_ctx(const void* h, const float* pos, const float* mass, float eps, const int64_t* targets,
                    int64_t nt, double* phi, double* acc, int64_t* pairs) {
    if (!h) return ORC_ERR_ARG;
    orc_gravity_sum((const orc_ctx*)h, pos, mass, eps, targets, nt, phi, acc, pairs);
    return ORC_OK;
}

int orc_helmholtz_ctx(const void* h, const float* pos, const float* q, int nrhs, float k, const int64_t* targets,
                      int64_t nt, double* u, int64_t* pairs) {
    if (!h || nrhs < 1) return ORC_ERR_ARG;
    orc_helmholtz_sum((const orc_ctx*)h, pos, q, nrhs, k, targets, nt, u, pairs);
    return ORC_OK;
}

/* Number of ordered pairs P = sum_b n_b S_b - n (self pairs excluded). */
int orc_pair_count(const float* pos, int64_t n, int level, const float* lo, float edge,
                   int64_t* pairs) {
    orc_ctx c;
    int st = orc_ctx_build(&c, pos, n, level, lo, edge, 0);
    if (st != ORC_OK) return st;
    int64_t p = 0;
    for (int32_t b = 0; b < c.nb; ++b) {
        int64_t sb = 0;
        for (int32_t e = c.nbr_start[b]; e < c.nbr_start[b + 1]; ++e) {
            int32_t nbox = c.nbr_idx[e];
            sb += c.box_start[nbox + 1] - c.box_start[nbox];
        }
        p += (int64_t)(c.box_start[b + 1] - c.box_start[b]) * sb;
    }
    *pairs = p - n;
    orc_ctx_free(&c);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* adjoints (gradients of a real loss L through the P2P sums)                */
/* ------------------------------------------------------------------------- */
/*
 * Convention: for a complex quantity z the gradient is dL/dRe z + i dL/dIm z.
 * The DBIM solver of Section 5.1 is a gradient-based inverse-scattering loop;
 * these are the gradients of the near-field operator it needs.
 *
 * Helmholtz, given gbar = dL/du ([nrhs][n] complex):
 *   grad_q_k   = sum_{j in near(k), j != k} conj(G(x_k - x_j)) gbar_j
 *   grad_x_k   = Re sum_{j in near(k), j != k} sum_r
 *                  (conj(gbar_k) q_j + conj(gbar_j) q_k) grad G(x_k - x_j)
 *   grad G(v)  = G(|v|) (i k - 1/|v|) v / |v|
 * (u_i depends on x_k through the pairs (k, j) and (i, k); G is even and
 *  grad G odd, so both pair orders collapse into one sum over k's neighbours.)
 */
int orc_helmholtz_adjoint(const float* pos, const float* q, const float* gbar, int nrhs, int64_t n,
                          int level, const float* lo, float edge, float k, double* grad_q,
                          double* grad_x) {
    if (nrhs < 1) return ORC_ERR_ARG;
    orc_ctx c;
    int st = orc_ctx_build(&c, pos, n, level, lo, edge, 0);
    if (st != ORC_OK) return st;
    const double kk = (double)k;
    const double inv4pi = 1.0 / (4.0 * ORC_PI);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < n; ++t) {
        const int64_t i = t;
        int32_t b = c.box_of[i];
        double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int r = 0; r < nrhs; ++r) { grad_q[2 * (r * n + i)] = 0.0; grad_q[2 * (r * n + i) + 1] = 0.0; }
        for (int32_t e = c.nbr_start[b]; e < c.nbr_start[b + 1]; ++e) {
            int32_t nbox = c.nbr_idx[e];
            for (int32_t s = c.box_start[nbox]; s < c.box_start[nbox + 1]; ++s) {
                int64_t j = c.perm[s];
                if (j == i) continue;
                /* v = x_i - x_j */
                double vx = xi - (double)pos[3 * j], vy = yi - (double)pos[3 * j + 1], vz = zi - (double)pos[3 * j + 2];
                double r = sqrt(vx * vx + vy * vy + vz * vz);
                double gre = cos(kk * r) * inv4pi / r, gim = sin(kk * r) * inv4pi / r;
                /* dG/dr = G (i k - 1/r) */
                double dre = -gre / r - kk * gim, dim = -gim / r + kk * gre;
                double coef = 0.0;
                for (int rr = 0; rr < nrhs; ++rr) {
                    double qjr = q[2 * (rr * n + j)], qji = q[2 * (rr * n + j) + 1];
                    double qir = q[2 * (rr * n + i)], qii = q[2 * (rr * n + i) + 1];
                    double bjr = gbar[2 * (rr * n + j)], bji = gbar[2 * (rr * n + j) + 1];
                    double bir = gbar[2 * (rr * n + i)], bii = gbar[2 * (rr * n + i) + 1];
                    /* grad_q_i += conj(G) gbar_j */
                    grad_q[2 * (rr * n + i)] += gre * bjr + gim * bji;
                    grad_q[2 * (rr * n + i) + 1] += gre * bji - gim * bjr;
                    /* A = conj(gbar_i) q_j + conj(gbar_j) q_i */
                    double ar = bir * qjr + bii * qji + bjr * qir + bji * qii;
                    double ai = bir * qji - bii * qjr + bjr * qii - bji * qir;
                    coef += ar * dre - ai * dim;           /* Re(A dG/dr) */
                }
                gx += coef * vx / r; gy += coef * vy / r; gz += coef * vz / r;
            }
        }
        grad_x[3 * i] = gx; grad_x[3 * i + 1] = gy; grad_x[3 * i + 2] = gz;
    }
    orc_ctx_free(&c);
    return ORC_OK;
}

/*
 * Softened gravity, given gphi = dL/dphi [n] and gacc = dL/da [n][3] (real):
 * with d = x_j - x_k and h^2 = r^2 + eps^2,
 *   grad_m_k = sum_{j in near(k), j != k} [ -gphi_j h^-1 - gacc_j . d h^-3 ]
 *   grad_x_k = sum_{j in near(k), j != k} [ -h^-3 d (gphi_k m_j + gphi_j m_k)
 *                                           + J(d) (m_k gacc_j - m_j gacc_k) ]
 *   J(d) v   = h^-3 v - 3 h^-5 d (d . v)   (Jacobian of d h^-3)
 */
int orc_gravity_adjoint(const float* pos, const float* mass, const float* gphi, const float* gacc,
                        int64_t n, int level, const float* lo, float edge, float eps,
                        double* grad_m, double* grad_x) {
    orc_ctx c;
    int st = orc_ctx_build(&c, pos, n, level, lo, edge, 0);
    if (st != ORC_OK) return st;
    const double e2 = (double)eps * (double)eps;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; ++k) {
        int32_t b = c.box_of[k];
        double xk = pos[3 * k], yk = pos[3 * k + 1], zk = pos[3 * k + 2];
        double mk = mass[k], gpk = gphi[k];
        double gak[3] = {gacc[3 * k], gacc[3 * k + 1], gacc[3 * k + 2]};
        double gm = 0.0, gx[3] = {0.0, 0.0, 0.0};
        for (int32_t e = c.nbr_start[b]; e < c.nbr_start[b + 1]; ++e) {
            int32_t nbox = c.nbr_idx[e];
            for (int32_t s = c.box_start[nbox]; s < c.box_start[nbox + 1]; ++s) {
                int64_t j = c.perm[s];
                if (j == k) continue;
                double d[3] = {(double)pos[3 * j] - xk, (double)pos[3 * j + 1] - yk, (double)pos[3 * j + 2] - zk};
                double h2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + e2;
                double h1 = 1.0 / sqrt(h2), h3 = h1 / h2, h5 = h3 / h2;
                double mj = mass[j], gpj = gphi[j];
                double gaj[3] = {gacc[3 * j], gacc[3 * j + 1], gacc[3 * j + 2]};
                gm += -gpj * h1 - (gaj[0] * d[0] + gaj[1] * d[1] + gaj[2] * d[2]) * h3;
                double s1 = gpk * mj + gpj * mk;
                double v[3] = {mk * gaj[0] - mj * gak[0], mk * gaj[1] - mj * gak[1], mk * gaj[2] - mj * gak[2]};
                double dv = d[0] * v[0] + d[1] * v[1] + d[2] * v[2];
                for (int a = 0; a < 3; ++a) gx[a] += -h3 * d[a] * s1 + h3 * v[a] - 3.0 * h5 * d[a] * dv;
            }
        }
        grad_m[k] = gm;
        grad_x[3 * k] = gx[0]; grad_x[3 * k + 1] = gx[1]; grad_x[3 * k + 2] = gx[2];
    }
    orc_ctx_free(&c);
    return ORC_OK;
}


/*
 * Periodic (toroidal) boundaries, the "periodic" interactions of the PhotoNs
 * case (Section 5.2): neighbour cells wrap around the domain and a wrapped
 * neighbour's sources interact through their image one domain edge away.
 * Needs level >= 2 so that a box meets each neighbour through one image.
 * Same outputs as the non-periodic calls.
 */
int orc_tree_periodic(const float* pos, int64_t n, int level, const float* lo, float edge,
                      int32_t* perm, uint32_t* box_key, int32_t* box_start, int32_t* n_boxes,
                      int32_t* nbr_start, int32_t* nbr_idx, int32_t* nbr_img, int64_t* n_nbr) {
    return orc_tree_ex(pos, n, level, lo, edge, 1, perm, box_key, box_start, n_boxes, nbr_start, nbr_idx,
                       nbr_img, n_nbr);
}

int orc_gravity_periodic(const float* pos, const float* mass, int64_t n, int level, const float* lo,
                         float edge, float eps, const int64_t* targets, int64_t nt,
                         double* phi, double* acc, int64_t* pairs) {
    if (level < 2) return ORC_ERR_ARG;
    return orc_gravity_ex(pos, mass, n, level, lo, edge, eps, targets, nt, phi, acc, pairs, 1);
}

int orc_helmholtz_periodic(const float* pos, const float* q, int nrhs, int64_t n, int level,
                           const float* lo, float edge, float k, const int64_t* targets, int64_t nt,
                           double* u, int64_t* pairs) {
    if (level < 2) return ORC_ERR_ARG;
    return orc_helmholtz_ex(pos, q, nrhs, n, level, lo, edge, k, targets, nt, u, pairs, 1);
}
