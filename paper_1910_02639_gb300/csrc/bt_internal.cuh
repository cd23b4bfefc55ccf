// bt_internal.cuh -- device data layout and geometry primitives shared by the
// build, find and density kernels of the b-tree (arXiv:1910.02639).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/btree.h"

namespace bt {

// Host-side count of kernel launches (defined in bt_api.cu).
void note_launch(int k = 1);

constexpr int kDepthMax = 32;   // a cell at depth 32 is never split
constexpr int kGroupMax = 32;   // most particles per find work unit (per set: 1..32)
constexpr int kWholeMax = 32;   // cells up to this size become one work unit
constexpr int kSmallCap = 256;  // cells up to this size are built by one warp in smem
constexpr int kTinyCap = 32;    // ... by a leaner instance of the warp builder up to this size
constexpr int kBigChunk = 4096; // particles per block in the per-level big-cell passes
constexpr int kRootChunk = 4096; // particles per block in the root passes (one set per block)

// Status bits accumulated on the device (reported by btree_status).
enum : uint32_t {
    kStNgmax = 1u << 0,
    kStOversized = 1u << 1,
    kStNonfinite = 1u << 2,
    kStCapNodes = 1u << 3,
    kStCapSlots = 1u << 4,
    kStCapGroups = 1u << 5,
    kStCapSmall = 1u << 6,
    kStCapBig = 1u << 7,
    kStWalk = 1u << 8,  // a find work unit fell back to a wider (still exact) path
};

// NodeWalk.flags
enum : int {
    kFlagWide = 2,         // FP32 fast path unusable: build uses FP64, walk visits all cells
    kFlagDegen0 = 4,       // zero width in dimension 0 (then 8, 16 for dims 1, 2)
};

// Exact binary64 box of an internal node plus its particle range (build side)
// and the particle set it belongs to.
struct __align__(16) NodeGeom {
    double lo[3];
    double hi[3];
    int start, count, depth, set;
};

// What the walk and the per-particle sub-cell computation read (48 B + range).
struct __align__(16) NodeWalk {
    float lo[3];     // fl32(lo)
    float scale[3];  // fl32(b / (hi - lo)); 0 in a zero-width dimension
    float cn[3];     // additive error bound of the FP32 sub-cell coordinate
    int b;           // branching factor (0: unsplit)
    int slot0;       // first sub-cell
    int flags;
    int start, count, pad0, pad1;
};

// One sub-cell: its particle range in tree order and the internal node it is,
// or -1 for a leaf.  Sub-cells of a node are contiguous in id order, and so
// are their particle ranges.
struct __align__(16) Slot {
    int start, count, child, pad;
};

// -------------------------------------------------------------------------
// Eq. 2 in binary64, exactly as the definition: floor(((x-lo)/(hi-lo))*b),
// clamped to [0, b-1].  Each operation is a correctly rounded intrinsic, so
// no contraction or reassociation can change it.
__device__ __forceinline__ int coord_fp64(float x, double lo, double hi, int b)
{
    double t = __ddiv_rn(__dsub_rn((double)x, lo), __dsub_rn(hi, lo));
    double v = __dmul_rn(t, (double)b);
    double f = floor(v);
    if (!(f >= 0.0)) return 0;
    if (f > (double)(b - 1)) return b - 1;
    return (int)f;
}

// Eq. 2 with an FP32 fast path.  v32 = fl32(fl32(x - lo32) * scale32) with
// scale32 = fl32(b / fl32(hi - lo)) differs from the binary64 value v by at
// most E = 2^-21 (|v32| + |lo| s) + 2^-146 (s + 1), s = b/(hi-lo): the scale
// carries two float roundings, the subtraction, the product and lo32 one
// each (relative 2^-24), binary64 adds 4 * 2^-53, underflow an absolute
// 2^-149 per step; cn holds the constant part rounded up.  If v32 is farther
// than E from every integer, floor(v32) = floor(v); otherwise the binary64
// definition decides.
__device__ __forceinline__ int coord_fast(float x, const NodeWalk &w, const NodeGeom &g,
                                          int l, int b)
{
    if (w.flags & (kFlagDegen0 << l)) return 0;
    if (!(w.flags & kFlagWide)) {
        float v = __fmul_rn(__fsub_rn(x, w.lo[l]), w.scale[l]);
        float av = fabsf(v);
        if (av < 4194304.0f) {  // 2^22: fractional part exact
            float e = __fmaf_ru(av, 0x1p-21f, w.cn[l]);
            float k = floorf(v);
            if (__fsub_rn(v, k) > e && __fsub_rn(k + 1.0f, v) > e) {
                int c = (int)k;
                return c < 0 ? 0 : (c > b - 1 ? b - 1 : c);
            }
        }
    }
    return coord_fp64(x, g.lo[l], g.hi[l], b);
}

// Conservative range of sub-cells [r0, r1] in one dimension whose cells may
// hold a particle with coordinate in [ql, qh] (Eqs. 5-6 on an interval).
// Rounded outward by the same error bound, so it always contains the exact
// binary64 range; clamped like Eq. 2.
__device__ __forceinline__ void walk_range(float ql, float qh, const NodeWalk &w, int l,
                                           int &r0, int &r1)
{
    int b = w.b;
    if (w.flags & (kFlagDegen0 << l)) { r0 = 0; r1 = 0; return; }
    if (w.flags & kFlagWide) { r0 = 0; r1 = b - 1; return; }
    // same operation sequence as coord_fast, so the same bound E applies
    float vl = __fmul_rn(__fsub_rn(ql, w.lo[l]), w.scale[l]);
    float vh = __fmul_rn(__fsub_rn(qh, w.lo[l]), w.scale[l]);
    float el = __fmaf_ru(fabsf(vl), 0x1p-21f, w.cn[l]);
    float eh = __fmaf_ru(fabsf(vh), 0x1p-21f, w.cn[l]);
    float fl = floorf(__fsub_rd(vl, el));
    float fh = floorf(__fadd_ru(vh, eh));
    // clamp in float first (also maps NaN to the full range)
    fl = fmaxf(fl, 0.0f);
    fh = fminf(fh, (float)(b - 1));
    if (!(fl <= (float)(b - 1))) fl = (float)(b - 1);
    if (!(fh >= 0.0f)) fh = 0.0f;
    r0 = (int)fl;
    r1 = (int)fh;
}

// Fill the walk/coordinate parameters of a node with branching factor b.
// k = 2: the z dimension is not split (treated like a zero-width dimension:
// sub-cell coordinate 0, walk range [0, 0]).
__device__ __forceinline__ void make_walk(const NodeGeom &g, int b, int slot0, NodeWalk &w, int k = 3)
{
    w.b = b;
    w.slot0 = slot0;
    w.flags = 0;
    w.start = g.start;
    w.count = g.count;
    w.pad0 = w.pad1 = 0;
    for (int l = 0; l < 3; l++) {
        double width = __dsub_rn(g.hi[l], g.lo[l]);
        w.lo[l] = __double2float_rn(g.lo[l]);
        if (width == 0.0 || (k == 2 && l == 2)) {
            w.flags |= (kFlagDegen0 << l);
            w.scale[l] = 0.0f;
            w.cn[l] = 0.0f;
            continue;
        }
        // FP32 scale (binary64 division is slow on this GPU); its rounding is
        // part of the bound documented at coord_fast.
        const float wid32 = __double2float_rn(width);
        const float alo = fabsf(w.lo[l]);
        if (!(wid32 > 0x1p-100f) || !(wid32 < 0x1p100f) || !(alo < 0x1p100f)) {
            w.flags |= kFlagWide;
            w.scale[l] = 0.0f;
            w.cn[l] = 0.0f;
            continue;
        }
        const float s32 = __fdiv_rn((float)b, wid32);
        w.scale[l] = s32;
        const float s_up = __fmul_ru(s32, 1.0f + 0x1p-20f);     // >= b/(hi-lo)
        const float alo_up = __fmul_ru(alo, 1.0f + 0x1p-22f);   // >= |lo|
        float c = __fmaf_ru(__fmul_ru(alo_up, s_up), 0x1p-21f, 0x1p-21f);
        c = __fmaf_ru(__fadd_ru(s_up, 1.0f), 0x1p-126f, c);     // covers 2^-146 (s + 1)
        w.cn[l] = c;
    }
}

// Sub-cell width w = (hi - lo)/b of one dimension, binary64.
__device__ __forceinline__ double cell_width(double lo, double hi, int b)
{
    return __ddiv_rn(__dsub_rn(hi, lo), (double)b);
}

// Child box of sub-cell coordinate c in one dimension (Sec. 3.1 step 2,
// equal-size sub-cells), binary64 in the oracle's operation order, given the
// cell width w from cell_width.
__device__ __forceinline__ void child_bounds_w(double lo, double hi, double w, int b, int c,
                                               double &clo, double &chi)
{
    clo = __dadd_rn(lo, __dmul_rn((double)c, w));
    chi = (c == b - 1) ? hi : __dadd_rn(lo, __dmul_rn((double)(c + 1), w));
}

// Eq. 1 in integers: smallest b >= 2 with b^3 s >= n.  A float cube root
// gives the starting point, exact integer tests settle it (no binary64 math:
// it is slow on this GPU).
__device__ __host__ __forceinline__ int branching_factor(long long n, long long s)
{
    long long b = (long long)cbrtf((float)n / (float)s);
    if (b < 2) b = 2;
    while (b > 2 && (b - 1) * (b - 1) * (b - 1) * s >= n) b--;
    while (b * b * b * s < n) b++;
    return (int)b;
}

// Eq. 1 for k = 2: smallest b >= 2 with b^2 s >= n.
__device__ __host__ __forceinline__ int branching_factor2(long long n, long long s)
{
    long long b = (long long)sqrtf((float)n / (float)s);
    if (b < 2) b = 2;
    while (b > 2 && (b - 1) * (b - 1) * s >= n) b--;
    while (b * b * s < n) b++;
    return (int)b;
}

// Sub-cells of a node: b^k.
__device__ __host__ __forceinline__ int ncells(int b, int k) { return k == 2 ? b * b : b * b * b; }

// Branching factor of dimension l of a node: b, except the unsplit z of k = 2.
__device__ __host__ __forceinline__ int dim_b(int b, int k, int l) { return (k == 2 && l == 2) ? 1 : b; }

// Order-preserving float <-> int map for atomicMin/atomicMax on floats.
__device__ __forceinline__ int float_to_ordered(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_to_float(int i)
{
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// Device-side counters of one build (one struct in device memory).
// The counters that every cell's builder updates sit on cache lines of their
// own, so that their atomics do not queue behind one another.
struct Counters {
    alignas(128) int nnodes;     // internal nodes allocated
    alignas(128) int nslots;     // sub-cells allocated
    alignas(128) int ngroups;    // find groups emitted
    alignas(128) int nsmall;     // cells queued for the warp builder
    alignas(128) int ngroups_c;  // work units of the compact-shape list (end of the groups array)
    alignas(128) int small_next; // dynamic work counter of the warp builder
    alignas(128) int ntiny;      // cells of <= kTinyCap particles queued for the warp builder
    alignas(128) int tiny_next;  // their dynamic work counter
    alignas(128) int nbig_next;  // big cells queued for the next level
    int again;         // some big cell halved b in the last ratio pass
    int max_depth;
    int noversized;
    int bbox[6];       // ordered-int min x,y,z then max x,y,z
    unsigned status;
    int hist_total;    // sum of b0^3 over this level's big cells
    int chunk_total;   // blocks of kBigChunk particles over this level's big cells
    int level;         // big-cell level being built (0 = the set roots)
    int nbig;          // big cells of this level
    int slot_base;     // first sub-cell of this level's big cells
    int ratio_it;      // ratio-test passes of this level
    int ratio_total;   // ratio-test passes over all levels
    int ratio_go;      // another ratio pass follows
    int level_go;      // another level follows
    int abort;         // capacity or input problem: the remaining kernels do nothing
    long long hist_need;  // histogram entries a level asked for (on abort)
    int nsplit;        // one-query work units made by the search from very wide units
};

// Per big cell of the current level.
struct BigCell {
    int node;
    int b0, b;
    int hist_n;        // b0^3 (histogram entries reserved)
    int chunk_n;       // kBigChunk blocks of the cell
    int hist_base;     // offset into the level histogram (prefix of hist_n)
    int chunk_base;    // first kBigChunk block of this cell (prefix of chunk_n)
    int state;         // 0 pending, 1 accepted, 2 stays a leaf
    int slot0;
    int u;             // sub-cells with n_j <= alpha s (current b)
    int ne;            // non-empty sub-cells
    int lastj;         // largest non-empty sub-cell id
    int halved;        // b was just halved: histogram to clear
    int set;           // particle set of the cell
    double w[3];       // sub-cell widths (hi - lo)/b of the accepted b
};

struct SmallItem {
    int node;
    int src;  // 0/1: working buffer holding its particles; 2: the input arrays
};

// One set's parameters as staged by the host (copied to the device once per
// build; k_init_sets derives the per-set tables from it).
struct SetRec {
    int start, end;  // particles [start, end)
    int s;           // bucket size
    int flags;       // kSetOctree
    int gmax;        // particles per find work unit, 1..kGroupMax
    int chunk0;      // first kRootChunk-particle block of the set (root passes)
    double alpha, beta;  // Eq. 4
};

// Per-set flags.
enum : int {
    kSetOctree = 1,    // b fixed to 2 (no Eq. 1 / Eq. 4): the classical octree
    kSetLeafRoot = 2,  // the whole set fits one leaf
    kSetFindCompact = 4,  // searched by the compact block shape (4 warps, 512 candidates)
    kSetTwoD = 8,         // k = 2: cells split in x and y only (b^2 sub-cells)
    kSetPackLeaves = 16,  // sibling leaves adjacent in tree order share work units
};

// Work units are (first tree position, set << 6 | count), count <= 32.
__device__ __host__ __forceinline__ int group_count(int v) { return v & 63; }
__device__ __host__ __forceinline__ int group_set(int v) { return v >> 6; }
__device__ __host__ __forceinline__ int group_pack(int set, int count) { return (set << 6) | count; }

// Everything the kernels need to see of one tree (one or more particle sets;
// node i < nsets is the root of set i).
struct TreeDev {
    int n;               // particles over all sets
    int nsets;
    const int *set_start;  // [nsets+1] first particle of each set
    const int *set_s;      // [nsets] bucket size s
    const int *set_na;     // [nsets] largest n_j counted as underfull (alpha s, Eq. 4)
    const double *set_beta;  // [nsets] beta of Eq. 4
    const int *set_gmax;   // [nsets] particles per find work unit
    const int *set_chunk0; // [nsets+1] first root-pass block of each set; [nsets] = all blocks
    int *set_flags;        // [nsets]
    int *set_bbox;         // [nsets][6] ordered-int min x,y,z, max x,y,z
    NodeGeom *geom;
    NodeWalk *walk;
    Slot *slots;
    int2 *groups;
    float4 *spos;   // tree order: x, y, z, orig index (bits)
    float *sh;      // tree order: h
    int *inv;       // inverse permutation: tree position of original index
    Counters *ctr;
    int cap_nodes, cap_slots, cap_groups, cap_small;
    int small_hist;  // histogram entries per warp of the small-cell builder (>= b0^k at kSmallCap)
    int tiny_hist;   // the same at kTinyCap
};

// Largest b^k that any cell of at most cap particles starts from, over
// sets whose bucket size is at least smin (Eq. 1 is monotone in n and in 1/s;
// the ratio test only lowers b).
__host__ __device__ __forceinline__ int small_hist_cells(int smin, int cap = kSmallCap)
{
    int c = ncells(branching_factor(cap, smin), 3);
    c = c > ncells(branching_factor2(cap, smin), 2) ? c : ncells(branching_factor2(cap, smin), 2);
    c = c > 8 ? c : 8;  // octree
    return (c + 3) & ~3;
}

// Ratio test of Eq. 4 for a cell of the given set: halve b iff
// u > beta * b^k, in binary64 (b^k is exact; u is an integer).
__device__ __forceinline__ int set_dim(const TreeDev &T, int set)
{
    return (T.set_flags[set] & kSetTwoD) ? 2 : 3;
}

__device__ __forceinline__ bool ratio_halves(const TreeDev &T, int set, int u, int b)
{
    const double bb = (double)ncells(b, set_dim(T, set));
    return (double)u > __dmul_rn(T.set_beta[set], bb);
}

// The set of root-pass block c: the last set whose first block is <= c
// (empty sets own no block and are skipped).
__device__ __forceinline__ int set_of_chunk(const int *chunk0, int nsets, int c)
{
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunk0[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The set holding particle p (binary search over the set offsets).
__device__ __forceinline__ int find_set(const int *set_start, int nsets, int p)
{
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (set_start[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Load particle p of the level's source: the input arrays (root level) or a
// working buffer.
struct Src {
    const float *x, *y, *z, *h;  // input arrays, or null
    const float4 *pos;           // working buffer records
    const float *ph;
    __device__ __forceinline__ void load(int p, float4 &r, float &hh) const
    {
        if (x) {
            r = make_float4(x[p], y[p], z[p], __int_as_float(p));
            hh = h[p];
        } else {
            r = pos[p];
            hh = ph[p];
        }
    }
    __device__ __forceinline__ float4 load_pos(int p) const
    {
        if (x) return make_float4(x[p], y[p], z[p], __int_as_float(p));
        return pos[p];
    }
};

// What the host reads back after a step.  The device writes it with an
// ordinary store into mapped pinned host memory (no copy engine involved, so
// small read-backs never queue behind a large copy on another stream).
struct Readback {
    Counters c;
    long long total;  // a compressed-row total (btree_find_neighbors_csr / btree_pack_rows)
    int root_b;       // branching factor of node 0
    int pad;
};

// Buffers of the level-synchronous build of big cells.  Level L reads the
// particles from the input (L = 0) or working buffer (L-1)&1 and writes
// working buffer L&1; its big cells are ids[L&1], the next level's ids[(L+1)&1].
struct LevelBufs {
    Src in;
    float4 *wpos[2];
    float *wh[2];
    int *ids[2];
    BigCell *big;
    int *hist, *hoff, *cursor, *tiles;
    SmallItem *small;  // cells of kTinyCap < n <= kSmallCap particles
    SmallItem *tiny;   // cells of n <= kTinyCap (both queues hold cap_small items)
    long long cap_hist;
    int cap_big, cap_tiles;
};

__device__ __forceinline__ Src level_src(const LevelBufs &L, int level)
{
    if (level == 0) return L.in;
    const int k = (level - 1) & 1;
    return Src{nullptr, nullptr, nullptr, nullptr, L.wpos[k], L.wh[k]};
}

}  // namespace bt
