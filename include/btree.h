/*
 * btree.h -- C ABI of the GB300 b-tree neighbour search.
 *
 * The method is the b-tree of "Finding Neighbors in a Forest: A b-tree for
 * Smoothed Particle Hydrodynamics Simulations" (arXiv:1910.02639):
 *   BuildTree     (Algorithm 1; Eq. 1 branching factor, Eq. 2 sub-cell
 *                  coordinates, Eq. 3 sub-cell id, Eq. 4 distribution ratio)
 *   FindNeighbors (Algorithm 2; Eqs. 5-6 range of sub-cells to visit)
 * plus the SPH density sum with the M4 cubic spline as a consumer of the
 * neighbour lists (the SPH interpolation of Sec. 1).
 *
 * Conventions shared by every call:
 *  - Pointers marked "device" are CUDA device pointers (cudaMalloc, a
 *    PyTorch CUDA tensor's data_ptr, ...) owned by the caller; the library
 *    never frees them.  Pointers marked "host" are ordinary host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it.
 *  - Particle indices are int32: n must be < 2^31 and n * ngmax < 2^62.
 *  - k = 3 spatial dimensions (Table 1).
 *  - Every call returns a status (bt_status).  Negative values are errors and
 *    leave the outputs unspecified; positive values are warnings.
 *  - Arithmetic contract: the tree (branching factors, cell membership) is the
 *    one an IEEE binary64 evaluation of Eqs. 1-4 gives, with the readings
 *    listed beside btree_build; the neighbour predicate is the binary64
 *    D = ((dx*dx + dy*dy) + dz*dz) < (2 h_i)^2, no FMA contraction, with
 *    dx = x_j - x_i from the float inputs.  Results are therefore identical
 *    to a plain CPU evaluation of the same definitions.
 */
#ifndef BTREE_GB300_H
#define BTREE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct btree btree_t; /* opaque; owns its device buffers */

typedef enum {
    BT_OK = 0,
    BT_ERR_ARG = -1,        /* an argument is out of range or NULL          */
    BT_ERR_OOM = -2,        /* a device allocation failed                   */
    BT_ERR_CUDA = -3,       /* a CUDA call or kernel launch failed          */
    BT_ERR_TIMEOUT = -4,    /* a bounded device-side wait gave up           */
    BT_ERR_NONFINITE = -5,  /* a position or h is NaN/Inf, or h < 0         */
    BT_ERR_CAPACITY = -6,   /* a fixed-size buffer was too small            */
    BT_WARN_NGMAX = 1,      /* some particle has more than ngmax neighbours;
                               its row holds the ngmax smallest indices and
                               counts[i] holds the full count               */
    BT_WARN_OVERSIZED_LEAF = 2 /* some leaf holds more than s particles
                               (coincident particles or depth limit 32)     */
} bt_status;

/* Stream-ordered device allocator used for the tree's internal buffers.
 * alloc(ctx, bytes, stream) returns a device pointer aligned to at least 256
 * bytes (as cudaMalloc's are), or NULL (the call that
 * needed it then returns BT_ERR_OOM; the handle stays valid and freeable);
 * free(ctx, ptr, stream) releases it.  Pass NULL to use cudaMallocAsync /
 * cudaFreeAsync on the call's stream.  When a handle is rebuilt with a
 * different allocator (or none), its buffers first go back to the one that
 * gave them. */
typedef struct {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, void *stream);
} bt_allocator;

/* Summary of a built tree (host struct filled by btree_get_info). */
typedef struct {
    int64_t n;               /* particles                                      */
    int32_t bucket_size;     /* s                                              */
    int32_t max_depth;       /* deepest node (root = 0)                        */
    int64_t num_nodes;       /* internal nodes (the root counts if split)      */
    int64_t num_slots;       /* sub-cells of all internal nodes (sum of b^3)   */
    int64_t num_groups;      /* query groups of <= 32 particles used by find   */
    int32_t root_b;          /* branching factor chosen at the root (0: leaf)  */
    int32_t num_oversized;   /* leaves holding more than s particles           */
    double build_ms;         /* device time of the last build (0 if unknown)   */
} bt_info;

/*
 * btree_build -- BuildTree (Algorithm 1) over n particles.
 *
 * x, y, z, h : device, float32 [n], particle positions and smoothing lengths.
 *              Read by the build's work on `stream` (the tree keeps its own
 *              copy); keep them valid until that work has run.
 * n          : 0 <= n < 2^31.
 * bucket_size: s >= 1, the maximum number of particles in a leaf (Table 1).
 * alpha      : fraction of s below which a sub-cell counts as underfull
 *              (Table 1, Eq. 4); the paper's default is 0.5.
 * beta       : the largest accepted ratio of underfull sub-cells (Eq. 4);
 *              default 0.5.
 * alloc      : allocator for internal buffers, or NULL.
 * stream     : cudaStream_t.
 * out        : host, receives the tree.  If *out already holds a tree from
 *              an earlier btree_build, it is rebuilt in place and its device
 *              buffers are reused when large enough.
 *
 * Readings of the paper (Sec. 3.1):
 *  - b = smallest integer >= 2 with b^3 s >= count (Eq. 1 in integers);
 *  - a sub-cell coordinate is clamp(floor(((x - lo)/(hi - lo)) * b), 0, b-1)
 *    in binary64, 0 in a dimension with hi == lo (Eq. 2); id = c1 + c2 b +
 *    c3 b^2 (Eq. 3);
 *  - b is halved (b <- max(2, floor(b/2))) while #{j : n_j <= alpha s} >
 *    beta b^3 and b > 2 (Eq. 4, the prose's "r larger than beta");
 *  - sub-cell boxes: w = (hi-lo)/b, lo' = lo + c w, hi' = lo + (c+1) w
 *    (hi' = hi for c = b-1); the root box is the inputs' bounding box;
 *  - a cell with more than s particles stays a leaf at depth 32, or when
 *    all its particles fall into one sub-cell whose box equals its own.
 *
 * Synchronous and asynchronous builds.  The first build of a handle (and
 * any build whose sets or parameters differ from the handle's last
 * synchronous build) synchronises `stream` a few times (once per level of
 * cells with more than 256 particles) to size the next level, grows its
 * buffers if they fall short, and returns when the tree is complete.  A
 * rebuild of the same sets with the same parameters (new positions) is one
 * launch of a captured CUDA graph whose level and ratio loops run on the
 * device, and returns at once (BT_OK) without waiting for the device.  The
 * searches that follow on `stream` read the tree's work-unit counts on the
 * device.  The host-side summary of such a rebuild is read by the next call
 * that needs it (btree_get_info, btree_export, btree_status, the compressed
 * rows, the next build): a capacity overflow (BT_ERR_CAPACITY; the searches
 * then write nothing), non-finite input or an oversized leaf of that rebuild
 * is reported there, and the next build is synchronous again.
 * Errors: BT_ERR_ARG (NULL pointer, n < 0, s < 1, alpha/beta not finite),
 * BT_ERR_NONFINITE (a NaN/Inf coordinate or h, or h < 0), BT_ERR_OOM,
 * BT_ERR_CUDA.  Warning: BT_WARN_OVERSIZED_LEAF.
 */
int btree_build(const float *x, const float *y, const float *z, const float *h,
                int64_t n, int bucket_size, double alpha, double beta,
                const bt_allocator *alloc, void *stream, btree_t **out);

/* Per-set parameters of btree_build_batched. */
#define BT_SET_OCTREE 1       /* b fixed to 2, no Eq. 1 / Eq. 4: the classical octree */
#define BT_SET_FIND_COMPACT 2 /* search this set with 4 warps per work unit and a
                                 512-candidate window instead of 8 warps and 1024
                                 (often faster on near-uniform sets); same results */
#define BT_SET_2D 4           /* k = 2 (Table 1: the tree of a two-dimensional
                                 problem): Eqs. 1 and 4 with b^2, cells split in x
                                 and y only (b^2 sub-cells), z never split.  The
                                 neighbour lists are those of the 3-D distance, so
                                 a planar set (z = 0) gets the 2-D lists. */
#define BT_SET_PACK_LEAVES 8  /* sibling leaves adjacent in tree order share find
                                 work units (up to group_size particles): fewer,
                                 fuller units; same results */
typedef struct {
    int bucket_size; /* s >= 1                                  */
    int flags;       /* 0 or BT_SET_OCTREE | BT_SET_FIND_COMPACT | BT_SET_2D |
                        BT_SET_PACK_LEAVES */
    double alpha;    /* underfull fraction (Eq. 4), e.g. 0.5    */
    double beta;     /* empty-cell limit (Eq. 4), e.g. 0.5      */
    int group_size;  /* queries searched together (a find work
                        unit; leaves are split to fit), 1..32,
                        0 = 32.  Changes speed, never results.  */
    int reserved;    /* 0                                       */
} bt_set_params;

/*
 * btree_build_batched -- BuildTree for many independent particle sets at once
 * (one set of launches for all of them).
 *
 * x, y, z, h : device float32 [offsets[nsets]]: the sets concatenated;
 *              set i is particles [offsets[i], offsets[i+1]).
 * offsets    : host int64 [nsets+1], offsets[0] = 0, non-decreasing,
 *              offsets[nsets] < 2^31.
 * nsets      : 1 <= nsets <= 2^24.
 * params     : host [nsets] per-set parameters, or NULL for s = 16,
 *              alpha = beta = 0.5.
 * Every set gets its own tree (its root box is its own bounding box); the
 * result for a set is exactly what btree_build gives for that set alone.
 * With BT_SET_OCTREE the set is split into octants at every level (the
 * paper's octree comparison baseline; same neighbour lists).
 * The find and density calls accept a batched tree: row i of `neighbors` is
 * the i-th particle of the concatenation, its entries are indices WITHIN the
 * particle's own set (0 .. set size - 1), ascending.
 * Errors and synchronisation: as btree_build.
 */
int btree_build_batched(const float *x, const float *y, const float *z, const float *h,
                        const int64_t *offsets, int nsets, const bt_set_params *params,
                        const bt_allocator *alloc, void *stream, btree_t **out);

/*
 * btree_build_find_batched -- btree_build_batched followed by
 * btree_find_neighbors_density (m != NULL) or btree_find_neighbors (m ==
 * NULL), as ONE CUDA graph launch on `stream`.  Inside the graph the level
 * loop of BuildTree and the ratio-test loop of Eq. 4 are conditional
 * while-nodes whose conditions the level kernels set on the device, so the
 * host never waits between steps.  Results are those of the separate calls.
 * The captured graph is kept in the handle and relaunched without a new
 * capture while every pointer and size stays the same (the per-set
 * parameters may change).
 * m, rho : device float32 [n] or both NULL (no density).
 * Other arguments: as btree_build_batched and btree_find_neighbors_density.
 * Synchronises `stream` before returning (the device reports capacity
 * problems, and the call grows the handle's buffers and runs again).
 * Returns BT_WARN_NGMAX when some row was capped, else as btree_build.
 */
int btree_build_find_batched(const float *x, const float *y, const float *z, const float *h,
                             const float *m, const int64_t *offsets, int nsets,
                             const bt_set_params *params, int ngmax, int32_t *neighbors,
                             int32_t *counts, float *rho, const bt_allocator *alloc, void *stream,
                             btree_t **out);

/*
 * btree_find_neighbors -- FindNeighbors (Algorithm 2) for every particle.
 *
 * N(i) = { j != i : D(i,j) < (2 h_i)^2 } (strict, binary64, see above);
 * the paper's Algorithm 2 writes "<=", its prose "less than"; the strict form
 * is used.
 * ngmax     : >= 1, row length of `neighbors`.
 * neighbors : device, int32 [n * ngmax], row-major by ORIGINAL particle index:
 *             row i holds the min(|N(i)|, ngmax) smallest j of N(i) in
 *             ascending order; entries past that are not written.
 * counts    : device, int32 [n], counts[i] = |N(i)| (uncapped).
 * Asynchronous on `stream`.  Returns BT_OK on launch; device-detected
 * conditions (a count above ngmax) are reported by btree_status.
 */
int btree_find_neighbors(const btree_t *t, int ngmax, int32_t *neighbors,
                         int32_t *counts, void *stream);

/*
 * btree_find_neighbors_csr -- FindNeighbors (Algorithm 2) into compressed
 * rows: every neighbour of every particle, no ngmax cap.  The paper has no
 * output format of its own; this is the compacted form of the same lists.
 * flags     : 0, or BT_FIND_HALF: row i holds only {j in N(i) : j > i}
 *             (symmetric half lists; no density with this flag).
 *
 * Two passes over the tree: the first counts (and, when m != NULL, computes
 * rho exactly as btree_find_neighbors_density does), an exclusive scan turns
 * the counts into row offsets, and the second writes row i, ascending by
 * original index, at neighbors[offsets[i] .. offsets[i+1]).
 * m, rho    : device float32 [n] or both NULL (no density).
 * offsets   : device int64 [n + 1], written; offsets[n] = total pairs.
 * neighbors : device int32 [capacity], or NULL to stop after the offsets
 *             (e.g. to size the buffer: the total is returned in *total).
 * capacity  : entries available in neighbors.
 * total     : host int64 or NULL; receives offsets[n].
 * Returns BT_ERR_CAPACITY (neighbors untouched, offsets and total valid) when
 * the total exceeds capacity.  Synchronises `stream` once (to read the
 * total); the second pass is asynchronous.  Uses scratch owned by the tree
 * (counts and scan partials, allocated on first use).
 */
#define BT_FIND_HALF 1 /* rows hold only the neighbours j > i: with a uniform h the
                          relation is symmetric and every pair appears once */
int btree_find_neighbors_csr(const btree_t *t, int flags, const float *m, float *rho, int64_t *offsets,
                             int32_t *neighbors, int64_t capacity, int64_t *total, void *stream);

/*
 * btree_pack_rows -- pack fixed rows (from btree_find_neighbors or
 * btree_find_neighbors_density on this tree) into compressed rows: row i's
 * first min(counts[i], ngmax) entries go to csr[offsets[i] ..].  The paper
 * has no counterpart; this is a layout change of the same lists (for moving
 * only the neighbours, e.g. to the host).  When no count exceeds ngmax the
 * result equals btree_find_neighbors_csr, at the cost of one read and one
 * write of the lists instead of a second search.
 * rows      : device int32 [n * ngmax];  counts : device int32 [n].
 * offsets   : device int64 [n + 1], written (exclusive scan of the capped counts).
 * csr       : device int32 [capacity], or NULL to stop after the offsets.
 * total     : host int64 or NULL; receives offsets[n].
 * Returns BT_ERR_CAPACITY (csr untouched) when the total exceeds capacity.
 * Synchronises `stream` once (to read the total); the packing is asynchronous.
 */
int btree_pack_rows(const btree_t *t, const int32_t *rows, const int32_t *counts, int ngmax,
                    int64_t *offsets, int32_t *csr, int64_t capacity, int64_t *total, void *stream);

/*
 * btree_find_neighbors_density -- FindNeighbors fused with the SPH density.
 *
 * As btree_find_neighbors, and in the same pass
 *   rho[i] = m_i W(0, h_i) + sum_{j in N(i)} m_j W(r_ij, h_i)
 * over the UNCAPPED set N(i), with the M4 cubic spline
 *   W(r,h) = (1/(pi h^3)) {1 - 1.5 q^2 + 0.75 q^3 (0 <= q < 1);
 *                          0.25 (2-q)^3 (1 <= q < 2); 0 (q >= 2)},  q = r/h,
 * accumulated in float32 in a fixed order (deterministic).
 * m   : device, float32 [n] masses.   rho : device, float32 [n].
 */
int btree_find_neighbors_density(const btree_t *t, const float *m, int ngmax,
                                 int32_t *neighbors, int32_t *counts,
                                 float *rho, void *stream);

/*
 * btree_find_neighbors_density_noalloc -- btree_find_neighbors_density for
 * callers that cannot allocate device memory when they search (a real-time
 * loop that forbids allocation after set-up, a host framework that owns all
 * device memory).  The paper has no counterpart: this is a deployment form
 * of the same computation, with identical results.
 *
 * The fused search needs one scratch buffer (the masses in tree order,
 * n floats).  btree_find_neighbors_density allocates it on first use; this
 * entry point uses a fixed array compiled into the library instead and calls
 * no allocator (no cudaMalloc/cudaFree, no allocating library routine).
 *  - Limit: t's n must be <= btree_noalloc_max_particles() (2^21 = 2097152);
 *    larger trees are rejected with BT_ERR_CAPACITY before any GPU work.
 *  - The array (8 MB) lives on every GPU that loads the library until the
 *    process exits.
 *  - The first call on a device looks up the array's device address (once
 *    per device, with that device current); make that first call before any
 *    CUDA stream capture.  The device current at the call must be the one
 *    the tree was built on (else BT_ERR_ARG).  The address belongs to that
 *    device's primary context: after cudaDeviceReset it is stale, so do not
 *    use this entry point again in a process that reset the device.
 *  - All calls share the one array: calls whose GPU work overlaps in time
 *    (different streams, or different threads) race on it and may return
 *    wrong densities.  Serialise them (same stream, or events).
 * Arguments, outputs and the other errors are those of
 * btree_find_neighbors_density.  The tree itself must already be built
 * (btree_build allocates; do that during set-up).
 */
int btree_find_neighbors_density_noalloc(const btree_t *t, const float *m, int ngmax,
                                         int32_t *neighbors, int32_t *counts,
                                         float *rho, void *stream);

/* Largest n accepted by btree_find_neighbors_density_noalloc. */
int64_t btree_noalloc_max_particles(void);

/*
 * sph_density -- the density sum above, computed from existing lists.
 *
 * Uses the first min(counts[i], ngmax) entries of row i (so rows truncated
 * by ngmax give a partial sum) and the positions and h the tree was built
 * from.  m, neighbors, counts: device inputs; rho: device float32 [n].
 */
int sph_density(const btree_t *t, const float *m, const int32_t *neighbors,
                const int32_t *counts, int ngmax, float *rho, void *stream);

/* Reads (synchronising `stream`) and clears the tree's device status word:
 * *out receives the most severe pending condition (BT_OK if none). */
int btree_status(btree_t *t, void *stream, int *out);

/* Fills *info (host).  Cheap; no device work. */
int btree_get_info(const btree_t *t, bt_info *info);

/*
 * btree_export -- copy the tree to host memory (for inspection and tests).
 * Any pointer may be NULL to skip that array.  Sizes come from bt_info.
 *  node_lo, node_hi : host double [num_nodes*3] box of each internal node
 *  node_b           : host int32 [num_nodes]  branching factor (0 = a cell
 *                     with more than s particles that stayed a leaf)
 *  node_depth       : host int32 [num_nodes]
 *  node_start,count : host int32 [num_nodes]  particle range in tree order
 *  node_slot0       : host int32 [num_nodes]  first sub-cell in `slot_*`
 *  slot_start,count : host int32 [num_slots]  particle range of a sub-cell
 *  slot_child       : host int32 [num_slots]  internal node id, or -1 (leaf)
 *  order            : host int32 [n]          original index at each tree
 *                     position
 * Node 0 is the root.  Synchronises `stream`.
 */
int btree_export(const btree_t *t, void *stream, double *node_lo,
                 double *node_hi, int32_t *node_b, int32_t *node_depth,
                 int32_t *node_start, int32_t *node_count, int32_t *node_slot0,
                 int32_t *slot_start, int32_t *slot_count, int32_t *slot_child,
                 int32_t *order);

/* Stream-ordered release of the tree and its buffers.  NULL is ignored. */
void btree_free(btree_t *t);

/* Static text for a status code. */
const char *btree_strerror(int status);

/* Library version string. */
const char *btree_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all trees).  For instrumentation: the difference across a region
 * is the number of kernel launches the region made. */
uint64_t btree_kernel_launches(void);

/* Measured arithmetic rates of the current device, in GFLOP/s (an FMA counts
 * as 2): scalar FP32 FMA, packed FP32x2 FMA, and binary64 FMA, each from a
 * kernel of independent FMA chains on every SM, timed with events on
 * `stream` after a warm-up launch.  They justify the FP32 distance filter
 * with binary64 only in its uncertain band (the distance test of Algorithm 2
 * would be ALU-bound in binary64).  Any output pointer may be NULL.  Takes
 * a few milliseconds and synchronises `stream`.  BT_ERR_CUDA on a launch or
 * timing failure. */
int btree_arith_rates(void *stream, double *fp32_gflops, double *fp32x2_gflops,
                      double *fp64_gflops);

#ifdef __cplusplus
}
#endif

#endif /* BTREE_GB300_H */
