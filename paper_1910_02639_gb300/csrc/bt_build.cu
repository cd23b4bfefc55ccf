// bt_build.cu -- BuildTree (Algorithm 1 of arXiv:1910.02639) on the GPU, for
// one or many particle sets at once.
//
// Level-synchronous for cells with more than kSmallCap particles ("big"
// cells), over all sets together: one pass per candidate branching factor
// computes every particle's sub-cell (Eqs. 2-3) and a global histogram n_j;
// the ratio test (Eq. 4) accepts b or halves it; an exclusive scan of the
// accepted histograms places the sub-cells; a scatter moves each particle to
// its sub-cell.  Cells of at most kSmallCap particles are built to the bottom
// by one warp each, entirely in shared memory (depth-first, explicit stack).
//
// Particle records are float4 (x, y, z, original index as int bits) plus a
// float h, in "tree order" once final: the particles of every cell, and so of
// every sub-tree, occupy one contiguous range, sub-cells in id order.  Each
// set's particles stay inside that set's input range; node i < nsets is the
// root of set i.  Per set: k = 3 or 2 (b^k sub-cells, z not split), or the
// octree (b = 2).
//
// Every level kernel reads its work counts from the device counters and
// stops when the abort flag is set, so the level loop and the ratio loop can
// be driven by the host (reading the counters) or by conditional nodes of a
// CUDA graph (the one-thread kernels set the loop conditions).
#include "bt_internal.cuh"
#include "bt_build.cuh"

#include <cfloat>
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

namespace bt {

namespace cg = cooperative_groups;

// atomicAdd(p, v) by the group's threads together: one atomic per group,
// each thread gets the old value plus the sum of the values of the lower
// ranks.  Every thread of the group passes the same p.
template <class G>
__device__ __forceinline__ int group_atomic_add(const G &g, int *p, int v)
{
    const int incl = cg::inclusive_scan(g, v);
    int base = 0;
    if (g.thread_rank() == g.num_threads() - 1) base = atomicAdd(p, incl);
    return g.shfl(base, g.num_threads() - 1) + incl - v;
}

// The same for the threads of the warp that reach this call together.
__device__ __forceinline__ int warp_atomic_add(int *p, int v)
{
    return group_atomic_add(cg::coalesced_threads(), p, v);
}

// Work units of at most the set's gmax particles over tree positions
// [start, start + cnt).  Sets searched by the compact block shape fill the
// groups array from its end, the others from its start.  kWarpAgg: the
// threads that call together share one atomic per counter (the level
// kernels, one thread per sub-cell, thousands of calls per launch); the
// per-warp small-cell builder takes plain atomics (a few calls per cell;
// aggregating them there gave no measurable gain).
// The counter of a set's list of work units.
__device__ __forceinline__ int *group_counter(const TreeDev &T, int set)
{
    return (T.set_flags[set] & kSetFindCompact) ? &T.ctr->ngroups_c : &T.ctr->ngroups;
}

// Write the work units of [start, start + cnt) at list entries g0, g0 + 1, ...
// (reserved on the set's counter).
__device__ __forceinline__ void emit_write(const TreeDev &T, int set, int g0, int start, int cnt)
{
    const int gm = T.set_gmax[set];
    const int ng = (cnt + gm - 1) / gm;
    const bool compact = (T.set_flags[set] & kSetFindCompact) != 0;
    for (int q = 0; q < ng; q++) {
        if (g0 + q >= T.cap_groups) break;
        const int idx = compact ? T.cap_groups - 1 - (g0 + q) : g0 + q;
        T.groups[idx] = make_int2(start + q * gm, group_pack(set, min(gm, cnt - q * gm)));
    }
    if (g0 + ng > T.cap_groups) atomicOr(&T.ctr->status, kStCapGroups);
}

template <bool kWarpAgg = false>
__device__ __forceinline__ void emit_groups(const TreeDev &T, int set, int start, int cnt)
{
    const int gm = T.set_gmax[set];
    const int ng = (cnt + gm - 1) / gm;
    const bool compact = (T.set_flags[set] & kSetFindCompact) != 0;
    int *ctr = group_counter(T, set);
    const int g0 = kWarpAgg
                       ? group_atomic_add(cg::labeled_partition(cg::coalesced_threads(), (int)compact), ctr, ng)
                       : atomicAdd(ctr, ng);
    emit_write(T, set, g0, start, cnt);
}

__device__ __forceinline__ int set_b0(const TreeDev &T, int set, int count)
{
    if (T.set_flags[set] & kSetOctree) return 2;
    return set_dim(T, set) == 2 ? branching_factor2(count, T.set_s[set])
                                : branching_factor(count, T.set_s[set]);
}

// ------------------------------------------------------------------ bbox
// Per-set bounding boxes (Eq. 2 "bounds of the domain"), plus a check that
// every coordinate and h is finite and h >= 0.
// One block per kRootChunk particles of one set: coalesced loads, a block
// reduction, six atomics per block.
// Block-wide min/max of v (6 values) into the set's bounding box.
__device__ __forceinline__ void bbox_flush(const TreeDev &T, int set, float (&v)[6], float (&red)[6][8])
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 6; k++) {
            const float w = __shfl_xor_sync(~0u, v[k], o);
            v[k] = k < 3 ? fminf(v[k], w) : fmaxf(v[k], w);
        }
    __syncthreads();  // red of the previous flush
    if (lane == 0)
        for (int k = 0; k < 6; k++) red[k][warp] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < 6; k++) {
            float w = lane < nw ? red[k][lane] : (k < 3 ? FLT_MAX : -FLT_MAX);
            for (int o = 4; o > 0; o >>= 1) {
                const float u = __shfl_xor_sync(~0u, w, o);
                w = k < 3 ? fminf(w, u) : fmaxf(w, u);
            }
            if (lane == 0) {
                int *bb = T.set_bbox + 6 * set + k;
                if (k < 3) atomicMin(bb, float_to_ordered(w));
                else atomicMax(bb, float_to_ordered(w));
            }
        }
    }
}

// The box is kept in registers over consecutive chunks of one set and
// added to the set's box once per set and block (a large set's chunks
// would otherwise all take atomics on the same six words).
__global__ void __launch_bounds__(256) k_bbox(TreeDev T, const float *__restrict__ x,
                                              const float *__restrict__ y,
                                              const float *__restrict__ z,
                                              const float *__restrict__ h)
{
    __shared__ float red[6][8];
    const int tid = threadIdx.x, lane = tid & 31;
    const int total = T.set_chunk0[T.nsets];
    bool bad = false;
    int cur = -1;
    float v[6] = {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int c = blockIdx.x; c < total; c += gridDim.x) {
        const int set = set_of_chunk(T.set_chunk0, T.nsets, c);  // the same in the whole block
        if (set != cur) {
            if (cur >= 0) bbox_flush(T, cur, v, red);
            cur = set;
            for (int k = 0; k < 6; k++) v[k] = k < 3 ? FLT_MAX : -FLT_MAX;
        }
        const int p0 = T.set_start[set] + (c - T.set_chunk0[set]) * kRootChunk;
        const int p1 = min(p0 + kRootChunk, T.set_start[set + 1]);
#pragma unroll 4
        for (int p = p0 + tid; p < p1; p += blockDim.x) {
            const float a = x[p], b = y[p], cc = z[p], hh = h[p];
            bad |= !isfinite(a) || !isfinite(b) || !isfinite(cc) || !isfinite(hh) || !(hh >= 0.0f);
            v[0] = fminf(v[0], a); v[1] = fminf(v[1], b); v[2] = fminf(v[2], cc);
            v[3] = fmaxf(v[3], a); v[4] = fmaxf(v[4], b); v[5] = fmaxf(v[5], cc);
        }
    }
    if (cur >= 0) bbox_flush(T, cur, v, red);
    if (__any_sync(~0u, bad) && lane == 0) atomicOr(&T.ctr->status, kStNonfinite);
}

// Per-set tables from the staged records.  n_j <= alpha*s (binary64) is
// n_j <= floor(alpha*s) for integer n_j.
__global__ void k_init_sets(TreeDev T, const SetRec *rec, int *set_start, int *set_s, int *set_na,
                            double *set_beta, int *set_gmax, int *set_chunk0)
{
    const int nsets = T.nsets;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsets; s += gridDim.x * blockDim.x) {
        const SetRec r = rec[s];
        for (int l = 0; l < 3; l++) {
            T.set_bbox[6 * s + l] = INT_MAX;
            T.set_bbox[6 * s + 3 + l] = INT_MIN;
        }
        set_start[s] = r.start;
        set_chunk0[s] = r.chunk0;
        if (s == nsets - 1) {
            set_start[nsets] = r.end;
            set_chunk0[nsets] = r.chunk0 + (r.end - r.start + kRootChunk - 1) / kRootChunk;
        }
        set_s[s] = r.s;
        const double under = __dmul_rn(r.alpha, (double)r.s);
        set_na[s] = under < 0.0 ? -1 : (under >= 2147483647.0 ? INT_MAX : (int)floor(under));
        set_beta[s] = r.beta;
        set_gmax[s] = r.gmax;
        T.set_flags[s] = r.flags;
    }
}

// Roots from the boxes, one thread per set: a set of <= s particles is one
// leaf (work units now, particles copied by k_copy_leaf_roots), a set of
// <= kSmallCap particles goes to the warp builder, a larger one to the big
// levels.
__device__ void root_set(TreeDev &T, int s, const LevelBufs &L)
{
    const int start = T.set_start[s], n = T.set_start[s + 1] - start;
    NodeGeom g;
    for (int l = 0; l < 3; l++) {
        double lo = (double)ordered_to_float(T.set_bbox[6 * s + l]);
        double hi = (double)ordered_to_float(T.set_bbox[6 * s + 3 + l]);
        if (n == 0) { lo = 0.0; hi = 0.0; }
        g.lo[l] = lo == 0.0 ? 0.0 : lo;  // canonical +0
        g.hi[l] = hi == 0.0 ? 0.0 : hi;
    }
    g.start = start;
    g.count = n;
    g.depth = 0;
    g.set = s;
    T.geom[s] = g;
    NodeWalk w;
    make_walk(g, 0, 0, w, set_dim(T, s));
    w.b = 0;  // a leaf until split
    T.walk[s] = w;
    if (n == 0) return;
    if (n <= T.set_s[s]) {
        T.set_flags[s] |= kSetLeafRoot;
        emit_groups(T, s, start, n);
    } else if (n <= kSmallCap) {
        const bool tiny = n <= kTinyCap;
        const int k = atomicAdd(tiny ? &T.ctr->ntiny : &T.ctr->nsmall, 1);
        if (k < T.cap_small) (tiny ? L.tiny : L.small)[k] = SmallItem{s, 2};
        else atomicOr(&T.ctr->status, kStCapSmall);
    } else {
        const int k = atomicAdd(&T.ctr->nbig_next, 1);
        if (k < L.cap_big) {
            L.ids[0][k] = s;
        } else {
            atomicOr(&T.ctr->status, kStCapBig);
            T.ctr->abort = 1;
        }
    }
}

// A build whose input failed the finiteness check stops here (the bounding
// boxes, and so everything below, would be meaningless).
__global__ void k_root_sets(TreeDev T, LevelBufs L)
{
    if (T.ctr->status & kStNonfinite) {
        if (blockIdx.x == 0 && threadIdx.x == 0) T.ctr->abort = 1;
        return;
    }
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < T.nsets; s += gridDim.x * blockDim.x)
        root_set(T, s, L);
}

// Sets that are one leaf: their particles are final where they are (one
// block per root-pass chunk; blocks of other sets return at once).
__global__ void k_copy_leaf_roots(TreeDev T, const float *__restrict__ x, const float *__restrict__ y,
                                  const float *__restrict__ z, const float *__restrict__ h)
{
    if (T.ctr->abort) return;
    const int total = T.set_chunk0[T.nsets];
    for (int c = blockIdx.x; c < total; c += gridDim.x) {
        const int set = set_of_chunk(T.set_chunk0, T.nsets, c);
        if (!(T.set_flags[set] & kSetLeafRoot)) continue;  // uniform over the block
        const int p0 = T.set_start[set] + (c - T.set_chunk0[set]) * kRootChunk;
        const int p1 = min(p0 + kRootChunk, T.set_start[set + 1]);
        for (int i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
            T.spos[i] = make_float4(x[i], y[i], z[i], __int_as_float(i));
            T.sh[i] = h[i];
            T.inv[i] = i;
        }
    }
}

// ------------------------------------------------------------------ big cells
// Every level kernel reads its work counts from the device counters, so the
// same kernels run host-driven (the host reads the counters between steps)
// or inside a CUDA graph whose loops are conditional nodes.

// One thread: whether another level follows; sets the graph's loop condition.
__global__ void k_level_go(Counters *ctr, int advance, cudaGraphConditionalHandle h, int graph)
{
    if (advance) ctr->level += 1;
    const int go = ctr->nbig_next > 0 && !ctr->abort && ctr->level < kDepthMax;
    ctr->level_go = go;
    if (graph) cudaGraphSetConditional(h, go);
}

// One thread: the cells queued by the previous level become this level's.
__global__ void k_level_begin(Counters *ctr)
{
    ctr->nbig = ctr->nbig_next;
    ctr->nbig_next = 0;
    ctr->ratio_it = 0;
    ctr->again = 0;
}

__global__ void k_big_setup(TreeDev T, LevelBufs L)
{
    const Counters *ctr = T.ctr;
    if (ctr->abort) return;
    const int nb = ctr->nbig;
    const int *ids = L.ids[ctr->level & 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        const int node = ids[i];
        const NodeGeom &g = T.geom[node];
        const int b0 = set_b0(T, g.set, g.count);
        BigCell c;
        c.node = node;
        c.b0 = b0;
        c.b = b0;
        c.hist_n = ncells(b0, set_dim(T, g.set));
        c.chunk_n = (g.count + kBigChunk - 1) / kBigChunk;
        c.hist_base = 0;
        c.chunk_base = 0;
        c.state = 0;
        c.slot0 = 0;
        c.u = 0;
        c.ne = 0;
        c.lastj = -1;
        c.halved = 0;
        c.set = g.set;
        c.w[0] = c.w[1] = c.w[2] = 0.0;
        L.big[i] = c;
    }
}

// One block: exclusive scans of histogram sizes and chunk counts over the
// level's cells; reserves the level's sub-cells; capacity checks.
__global__ void __launch_bounds__(1024) k_big_scan(TreeDev T, LevelBufs L,
                                                   cudaGraphConditionalHandle hratio, int graph)
{
    __shared__ long long sh_h[1024], sh_c[1024];
    __shared__ long long carry_h, carry_c;
    Counters *ctr = T.ctr;
    if (ctr->abort) {
        if (threadIdx.x == 0) {
            ctr->ratio_go = 0;
            if (graph) cudaGraphSetConditional(hratio, 0);
        }
        return;
    }
    const int nb = ctr->nbig;
    BigCell *big = L.big;
    if (threadIdx.x == 0) { carry_h = 0; carry_c = 0; }
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        long long vh = i < nb ? big[i].hist_n : 0;
        long long vc = i < nb ? big[i].chunk_n : 0;
        sh_h[threadIdx.x] = vh;
        sh_c[threadIdx.x] = vc;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            long long ah = threadIdx.x >= o ? sh_h[threadIdx.x - o] : 0;
            long long ac = threadIdx.x >= o ? sh_c[threadIdx.x - o] : 0;
            __syncthreads();
            sh_h[threadIdx.x] += ah;
            sh_c[threadIdx.x] += ac;
            __syncthreads();
        }
        if (i < nb) {
            const long long hb = carry_h + sh_h[threadIdx.x] - vh;
            big[i].hist_base = (int)min(hb, (long long)INT_MAX);
            big[i].chunk_base = (int)(carry_c + sh_c[threadIdx.x] - vc);
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            carry_h += sh_h[1023];
            carry_c += sh_c[1023];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long ht = carry_h;
        const bool fit_hist = ht <= L.cap_hist && ht < INT_MAX;
        const bool fit_slots = (long long)ctr->nslots + ht <= (long long)T.cap_slots;
        const int ok = fit_hist && fit_slots;
        ctr->hist_total = ok ? (int)ht : 0;
        ctr->chunk_total = ok ? (int)carry_c : 0;
        if (ok) {
            ctr->slot_base = ctr->nslots;
            ctr->nslots += (int)ht;
        } else {
            ctr->hist_need = ht;
            atomicOr(&ctr->status, fit_hist ? kStCapSlots : kStCapBig);
            ctr->abort = 1;
        }
        ctr->ratio_go = ok;
        if (graph) cudaGraphSetConditional(hratio, ok);
    }
}

__global__ void __launch_bounds__(256) k_zero_hist(const Counters *ctr, int *hist)
{
    if (ctr->abort) return;
    const int n = ctr->hist_total;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) hist[e] = 0;
}

__device__ __forceinline__ int find_cell_by_chunk(const BigCell *big, int nb, int chunk)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (big[mid].chunk_base <= chunk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_cell_by_hist(const BigCell *big, int nb, int e)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (big[mid].hist_base <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per-block walk parameters of the block's cell for its current b.
__device__ __forceinline__ void block_cell_params(const TreeDev &T, const BigCell &c,
                                                  NodeGeom &g, NodeWalk &w)
{
    __shared__ NodeGeom s_g;
    __shared__ NodeWalk s_w;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_g = T.geom[c.node];
        make_walk(s_g, c.b, 0, s_w, set_dim(T, c.set));
    }
    __syncthreads();
    g = s_g;
    w = s_w;
}

__device__ __forceinline__ int sub_cell_id(const float4 &p, const NodeWalk &w, const NodeGeom &g, int b)
{
    int c0 = coord_fast(p.x, w, g, 0, b);
    int c1 = coord_fast(p.y, w, g, 1, b);
    int c2 = coord_fast(p.z, w, g, 2, b);
    return c0 + b * (c1 + b * c2);
}

// Histogram pass of one candidate b for every pending big cell.  A cell
// with at most kPrivBins sub-cells is counted in shared memory first and
// added to the global histogram once per non-empty bin and block: with few
// bins, thousands of particles of a block would otherwise serialise on the
// same few global counters.
constexpr int kPrivBins = 4096;
static_assert(kPrivBins <= 4096 && kBigChunk <= 4096, "sub-cell and rank packed in 12 bits each");

__global__ void __launch_bounds__(256, 4) k_big_hist(TreeDev T, LevelBufs L)
{
    __shared__ int sh_bin[kPrivBins];
    const Counters *ctr = T.ctr;
    if (ctr->abort) return;
    const int nb = ctr->nbig;
    const int total = ctr->chunk_total;
    const BigCell *big = L.big;
    int *hist = L.hist;
    const Src src = level_src(L, ctr->level);
    for (int chunk = blockIdx.x; chunk < total; chunk += gridDim.x) {
        int ci = find_cell_by_chunk(big, nb, chunk);
        BigCell c = big[ci];
        if (c.state != 0) continue;  // uniform across the block
        NodeGeom g;
        NodeWalk w;
        block_cell_params(T, c, g, w);  // (begins with a block barrier)
        int p0 = g.start + (chunk - c.chunk_base) * kBigChunk;
        int p1 = min(p0 + kBigChunk, g.start + g.count);
        int *hc = hist + c.hist_base;
        const int nc = ncells(c.b, set_dim(T, c.set));
        if (nc > kPrivBins) {
            // one global atomic per sub-cell and warp (inputs often arrive
            // in spatial runs: neighbours in a warp share sub-cells); two
            // particles per thread and step, so that twice the loads are in
            // flight
            const int lane = threadIdx.x & 31;
            for (int pb = p0; pb < p1; pb += 2 * blockDim.x) {
                const int pa = pb + threadIdx.x, pc = pa + blockDim.x;
                float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rc = ra;
                if (pa < p1) ra = src.load_pos(pa);
                if (pc < p1) rc = src.load_pos(pc);
                const int ja = pa < p1 ? sub_cell_id(ra, w, g, c.b) : -1 - lane;
                const int jc = pc < p1 ? sub_cell_id(rc, w, g, c.b) : -1 - lane;
                const unsigned sa = __match_any_sync(~0u, ja);
                const unsigned sc = __match_any_sync(~0u, jc);
                const unsigned lt = (1u << lane) - 1u;
                if (ja >= 0 && (sa & lt) == 0) atomicAdd(&hc[ja], __popc(sa));
                if (jc >= 0 && (sc & lt) == 0) atomicAdd(&hc[jc], __popc(sc));
            }
            continue;
        }
        for (int j = threadIdx.x; j < nc; j += blockDim.x) sh_bin[j] = 0;
        __syncthreads();
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            float4 r = src.load_pos(p);
            atomicAdd(&sh_bin[sub_cell_id(r, w, g, c.b)], 1);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += blockDim.x) {
            const int v = sh_bin[j];
            if (v) atomicAdd(&hc[j], v);
        }
    }
}

// Per-cell statistics of the current histogram (Eq. 4 numerator, non-empty
// sub-cells), accumulated over the whole level by all blocks.
__global__ void __launch_bounds__(256) k_big_count(TreeDev T, LevelBufs L)
{
    const Counters *ctr = T.ctr;
    if (ctr->abort) return;
    const int nb = ctr->nbig;
    const int total = ctr->hist_total;
    BigCell *big = L.big;
    const int *hist = L.hist;
    __shared__ int s_red[4][8];  // per warp: cell (or -2: mixed), u, ne, last j
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e0 = blockIdx.x * blockDim.x; e0 < total; e0 += gridDim.x * blockDim.x) {
        const int e = e0 + threadIdx.x;
        int ci = -1, u = 0, ne = 0, lj = -1;
        if (e < total) {
            ci = find_cell_by_hist(big, nb, e);
            const BigCell &c = big[ci];
            const int j = e - c.hist_base;
            if (c.state == 0 && j < ncells(c.b, set_dim(T, c.set))) {
                const int v = hist[e];
                u = v <= T.set_na[c.set];
                ne = v > 0;
                lj = v > 0 ? j : -1;
            } else {
                ci = -1;
            }
        }
        // one atomic per block when the whole block lies in one cell (the
        // common case: cells are long contiguous runs of e; a level with one
        // huge cell would otherwise put every warp's atomics on one line),
        // else one per warp, else per lane
        const unsigned same = __match_any_sync(~0u, ci);
        if (same == 0xffffffffu) {
            int su = u, sne = ne, slj = lj;
            for (int o = 16; o > 0; o >>= 1) {
                su += __shfl_xor_sync(~0u, su, o);
                sne += __shfl_xor_sync(~0u, sne, o);
                slj = max(slj, __shfl_xor_sync(~0u, slj, o));
            }
            if (lane == 0) { s_red[0][warp] = ci; s_red[1][warp] = su; s_red[2][warp] = sne; s_red[3][warp] = slj; }
        } else {
            if (lane == 0) s_red[0][warp] = -2;
            if (ci >= 0) {
                if (u) atomicAdd(&big[ci].u, u);
                if (ne) atomicAdd(&big[ci].ne, ne);
                if (lj >= 0) atomicMax(&big[ci].lastj, lj);
            }
        }
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x >> 5;
            const int wc = lane < nw ? s_red[0][lane] : -1;
            const int c0 = __shfl_sync(~0u, wc, 0);
            const bool one = __all_sync(~0u, lane >= nw || wc == c0) && c0 >= 0;
            if (one) {  // every warp of the block in cell c0
                int su = lane < nw ? s_red[1][lane] : 0, sne = lane < nw ? s_red[2][lane] : 0;
                int slj = lane < nw ? s_red[3][lane] : -1;
                for (int o = 4; o > 0; o >>= 1) {
                    su += __shfl_xor_sync(~0u, su, o);
                    sne += __shfl_xor_sync(~0u, sne, o);
                    slj = max(slj, __shfl_xor_sync(~0u, slj, o));
                }
                if (lane == 0) {
                    if (su) atomicAdd(&big[c0].u, su);
                    if (sne) atomicAdd(&big[c0].ne, sne);
                    if (slj >= 0) atomicMax(&big[c0].lastj, slj);
                }
            } else if (lane < nw && wc >= 0) {  // per warp
                if (s_red[1][lane]) atomicAdd(&big[wc].u, s_red[1][lane]);
                if (s_red[2][lane]) atomicAdd(&big[wc].ne, s_red[2][lane]);
                if (s_red[3][lane] >= 0) atomicMax(&big[wc].lastj, s_red[3][lane]);
            }
        }
        __syncthreads();  // s_red is reused by the next step
    }
}

// Ratio test (Eq. 4), one thread per big cell: accept b or halve it.
__device__ __forceinline__ void decide_cell(const TreeDev &T, BigCell &c)
{
    c.halved = 0;
    if (c.state != 0) return;
    if (c.b > 2 && ratio_halves(T, c.set, c.u, c.b)) {
        c.b = max(2, c.b / 2);
        c.halved = 1;
        c.u = 0;
        c.ne = 0;
        c.lastj = -1;
        T.ctr->again = 1;
    } else {
        c.state = 1;
    }
}

__global__ void k_big_decide(TreeDev T, LevelBufs L)
{
    if (T.ctr->abort) return;
    const int nb = T.ctr->nbig;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x)
        decide_cell(T, L.big[i]);
}


// Clear the histogram of every cell whose b was just halved.
__global__ void __launch_bounds__(256) k_big_zero(const Counters *ctr, LevelBufs L)
{
    if (ctr->abort) return;
    const int nb = ctr->nbig;
    const int total = ctr->hist_total;
    const BigCell *big = L.big;
    int *hist = L.hist;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const BigCell &c = big[find_cell_by_hist(big, nb, e)];
        if (c.halved) hist[e] = 0;
    }
}

// One thread, after a ratio pass: another pass iff some cell halved b.
__global__ void k_ratio_end(Counters *ctr, cudaGraphConditionalHandle h, int graph)
{
    ctr->ratio_it += 1;
    ctr->ratio_total += 1;
    const int go = ctr->again && !ctr->abort && ctr->ratio_it < 16;
    ctr->again = 0;
    ctr->ratio_go = go;
    if (graph) cudaGraphSetConditional(h, go);
}

// After acceptance, one thread per cell: no-progress guard, walk
// parameters, sub-cell widths, slot placement.
__device__ void finish_cell(const TreeDev &T, BigCell &c, int slot_level_base);

__global__ void k_big_finish(TreeDev T, LevelBufs L)
{
    if (T.ctr->abort) return;
    const int nb = T.ctr->nbig;
    const int base = T.ctr->slot_base;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x)
        finish_cell(T, L.big[i], base);
}

__device__ void finish_cell(const TreeDev &T, BigCell &c, int slot_level_base)
{
    const int b = c.b;
    const int k = set_dim(T, c.set);
    const NodeGeom g = T.geom[c.node];
    for (int l = 0; l < 3; l++) c.w[l] = cell_width(g.lo[l], g.hi[l], dim_b(b, k, l));
    bool leaf = false;
    if (c.ne == 1) {
        const int lj = c.lastj;
        int cc[3] = {lj % b, (lj / b) % b, lj / (b * b)};
        bool same = true;
        for (int l = 0; l < 3; l++) {
            double clo, chi;
            child_bounds_w(g.lo[l], g.hi[l], c.w[l], dim_b(b, k, l), cc[l], clo, chi);
            if (clo != g.lo[l] || chi != g.hi[l]) same = false;
        }
        leaf = same;
    }
    if (leaf) {
        c.state = 2;
        NodeWalk w;
        make_walk(g, 0, 0, w, k);
        w.b = 0;
        T.walk[c.node] = w;
        atomicAdd(&T.ctr->noversized, 1);
        atomicOr(&T.ctr->status, kStOversized);
        emit_groups(T, c.set, g.start, g.count);
        return;
    }
    c.slot0 = slot_level_base + c.hist_base;
    NodeWalk w;
    make_walk(g, b, c.slot0, w, k);
    T.walk[c.node] = w;
    atomicMax(&T.ctr->max_depth, g.depth + 1);
}

// Emit the sub-cells of every accepted big cell: slots, child nodes, queues,
// leaf work units; cursor[e] = first tree position of sub-cell e.
__global__ void __launch_bounds__(256) k_big_emit(TreeDev T, LevelBufs L)
{
    Counters *ctr = T.ctr;
    if (ctr->abort) return;
    const int nb = ctr->nbig;
    const int total = ctr->hist_total;
    const int dst_buf = ctr->level & 1;
    const BigCell *big = L.big;
    const int *hist = L.hist, *hoff = L.hoff;
    int *cursor = L.cursor;
    int *next_big = L.ids[(ctr->level + 1) & 1];
    SmallItem *small = L.small;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int ci = find_cell_by_hist(big, nb, e);
        const BigCell c = big[ci];
        if (c.state != 1) continue;
        const int b = c.b;
        const int kd = set_dim(T, c.set);
        const int j = e - c.hist_base;
        if (j >= ncells(b, kd)) continue;
        const NodeGeom &g = T.geom[c.node];
        const int s = T.set_s[c.set];
        const int cnt = hist[e];
        const int start = g.start + (hoff[e] - hoff[c.hist_base]);
        cursor[e] = start;
        const int depth = g.depth + 1;
        int child = -1;
        if (cnt > s && depth < kDepthMax) {
            child = warp_atomic_add(&T.ctr->nnodes, 1);
            if (child >= T.cap_nodes) {
                atomicOr(&T.ctr->status, kStCapNodes);
                child = -1;
            } else {
                NodeGeom ng;
                int cc[3] = {j % b, (j / b) % b, j / (b * b)};
                for (int l = 0; l < 3; l++)
                    child_bounds_w(g.lo[l], g.hi[l], c.w[l], dim_b(b, kd, l), cc[l], ng.lo[l], ng.hi[l]);
                ng.start = start;
                ng.count = cnt;
                ng.depth = depth;
                ng.set = c.set;
                T.geom[child] = ng;
                if (cnt > kSmallCap) {
                    const int k = warp_atomic_add(&T.ctr->nbig_next, 1);
                    if (k < L.cap_big) {
                        next_big[k] = child;
                    } else {
                        atomicOr(&T.ctr->status, kStCapBig);
                        T.ctr->abort = 1;
                    }
                } else if (cnt > kTinyCap) {
                    int k = warp_atomic_add(&T.ctr->nsmall, 1);
                    if (k < T.cap_small) small[k] = SmallItem{child, dst_buf};
                    else atomicOr(&T.ctr->status, kStCapSmall);
                } else {
                    int k = warp_atomic_add(&T.ctr->ntiny, 1);
                    if (k < T.cap_small) L.tiny[k] = SmallItem{child, dst_buf};
                    else atomicOr(&T.ctr->status, kStCapSmall);
                }
            }
        } else if (cnt > 0) {
            if (cnt > s) {
                atomicAdd(&T.ctr->noversized, 1);
                atomicOr(&T.ctr->status, kStOversized);
            }
            if (!(T.set_flags[c.set] & kSetPackLeaves)) {
                emit_groups<true>(T, c.set, start, cnt);
            } else {
                // leaf sub-cells 2i and 2i+1 (adjacent in tree order) share
                // a work unit when both are leaves and fit together
                const int nc = ncells(b, kd), gm = T.set_gmax[c.set];
                const int jp = j ^ 1;  // the partner sub-cell
                bool paired = false;
                if (jp < nc) {
                    const int cp = hist[c.hist_base + jp];
                    const bool leafp = cp > 0 && !(cp > s && depth < kDepthMax);
                    paired = leafp && cnt + cp <= gm;
                }
                if (!paired) emit_groups<true>(T, c.set, start, cnt);
                else if ((j & 1) == 0) emit_groups<true>(T, c.set, start, cnt + hist[c.hist_base + jp]);
            }
        }
        T.slots[c.slot0 + j] = Slot{start, cnt, child, 0};
    }
}

// Move every particle of an accepted big cell to its sub-cell.  Leaf
// sub-cells are final: they go straight to tree order; others to the
// working buffer `dst` for the next level / the warp builder.
__device__ __forceinline__ void scatter_one(const TreeDev &T, const BigCell &c, int j, int pos,
                                            const float4 &r, float hh, float4 *dst_pos, float *dst_h)
{
    if (T.slots[c.slot0 + j].child < 0) {  // a leaf: final position
        T.spos[pos] = r;
        T.sh[pos] = hh;
        T.inv[__float_as_int(r.w)] = pos;
    } else {
        dst_pos[pos] = r;
        dst_h[pos] = hh;
    }
}

// Move every particle of the level's big cells to its sub-cell's range.  A
// cell with at most kPrivBins sub-cells ranks the block's particles per
// sub-cell in shared memory and reserves each sub-cell's run with one global
// atomic (the order within a sub-cell is not part of any result).
__global__ void __launch_bounds__(256) k_big_scatter(TreeDev T, LevelBufs L)
{
    __shared__ int sh_bin[kPrivBins];
    __shared__ int sh_jr[kBigChunk];  // per particle: sub-cell << 12 | rank within the block
    const Counters *ctr = T.ctr;
    if (ctr->abort) return;
    const int nb = ctr->nbig;
    const int total = ctr->chunk_total;
    const BigCell *big = L.big;
    const Src src = level_src(L, ctr->level);
    int *cursor = L.cursor;
    float4 *dst_pos = L.wpos[ctr->level & 1];
    float *dst_h = L.wh[ctr->level & 1];
    for (int chunk = blockIdx.x; chunk < total; chunk += gridDim.x) {
        int ci = find_cell_by_chunk(big, nb, chunk);
        BigCell c = big[ci];
        NodeGeom g;
        NodeWalk w;
        block_cell_params(T, c, g, w);  // (begins with a block barrier)
        int p0 = g.start + (chunk - c.chunk_base) * kBigChunk;
        int p1 = min(p0 + kBigChunk, g.start + g.count);
        if (c.state == 2) {  // stayed a leaf: final where it is
            for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
                float4 r;
                float hh;
                src.load(p, r, hh);
                T.spos[p] = r;
                T.sh[p] = hh;
                T.inv[__float_as_int(r.w)] = p;
            }
            continue;
        }
        const int nc = ncells(c.b, set_dim(T, c.set));
        if (nc > kPrivBins) {
            // one global atomic per sub-cell and warp; ranks within the warp;
            // two particles per thread and step (twice the loads and atomics
            // in flight)
            const int lane = threadIdx.x & 31;
            const unsigned lt = (1u << lane) - 1u;
            for (int pb = p0; pb < p1; pb += 2 * blockDim.x) {
                const int pa = pb + threadIdx.x, pc = pa + blockDim.x;
                float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rc = ra;
                float ha = 0.f, hc2 = 0.f;
                if (pa < p1) src.load(pa, ra, ha);
                if (pc < p1) src.load(pc, rc, hc2);
                const int ja = pa < p1 ? sub_cell_id(ra, w, g, c.b) : -1 - lane;
                const int jc = pc < p1 ? sub_cell_id(rc, w, g, c.b) : -1 - lane;
                const unsigned sa = __match_any_sync(~0u, ja);
                const unsigned sc = __match_any_sync(~0u, jc);
                const int la = __ffs(sa) - 1, lc = __ffs(sc) - 1;
                int ata = 0, atc = 0;
                if (ja >= 0 && lane == la) ata = atomicAdd(&cursor[c.hist_base + ja], __popc(sa));
                if (jc >= 0 && lane == lc) atc = atomicAdd(&cursor[c.hist_base + jc], __popc(sc));
                ata = __shfl_sync(~0u, ata, la);
                atc = __shfl_sync(~0u, atc, lc);
                if (ja >= 0) scatter_one(T, c, ja, ata + __popc(sa & lt), ra, ha, dst_pos, dst_h);
                if (jc >= 0) scatter_one(T, c, jc, atc + __popc(sc & lt), rc, hc2, dst_pos, dst_h);
            }
            continue;
        }
        for (int j = threadIdx.x; j < nc; j += blockDim.x) sh_bin[j] = 0;
        __syncthreads();
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int j = sub_cell_id(src.load_pos(p), w, g, c.b);
            sh_jr[p - p0] = j << 12 | atomicAdd(&sh_bin[j], 1);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += blockDim.x) {
            const int v = sh_bin[j];
            if (v) sh_bin[j] = atomicAdd(&cursor[c.hist_base + j], v);
        }
        __syncthreads();
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            float4 r;
            float hh;
            src.load(p, r, hh);
            const int jr = sh_jr[p - p0], j = jr >> 12;
            scatter_one(T, c, j, sh_bin[j] + (jr & 4095), r, hh, dst_pos, dst_h);
        }
    }
}

// ------------------------------------------------------------------ scan
// Exclusive scan of int32 counts (sums fit in int32).
constexpr int kScanTile = 4096;

// The scans below run over the level histogram: n = hist_total (nothing
// when the build was aborted).
__device__ __forceinline__ int scan_n(const Counters *ctr) { return ctr->abort ? 0 : ctr->hist_total; }

__global__ void __launch_bounds__(256) k_scan_tiles(const Counters *ctr, const int *in, int *tile_sum)
{
    const int n = scan_n(ctr);
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    __shared__ int ws[8];
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int t0 = tile * kScanTile;
        int s = 0;
        for (int i = t0 + threadIdx.x; i < min(t0 + kScanTile, n); i += blockDim.x) s += in[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(~0u, s, o);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < 8; k++) t += ws[k];
            tile_sum[tile] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_scan_tile_sums(const Counters *ctr, int *tile_sum)
{
    const int ntiles = (scan_n(ctr) + kScanTile - 1) / kScanTile;
    __shared__ int sh[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < ntiles ? tile_sum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int a = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += a;
            __syncthreads();
        }
        if (i < ntiles) tile_sum[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sh[1023];
        __syncthreads();
    }
}

__device__ void scan_apply_tile(const int *in, int n, int tile, const int *tile_off, int *out);

__global__ void __launch_bounds__(256) k_scan_apply(const Counters *ctr, const int *in,
                                                    const int *tile_off, int *out)
{
    const int n = scan_n(ctr);
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) scan_apply_tile(in, n, tile, tile_off, out);
}

// 256 threads x 16 items of one tile.
__device__ void scan_apply_tile(const int *in, int n, int tile, const int *tile_off, int *out)
{
    __shared__ int ws[8];
    int t0 = tile * kScanTile;
    int v[16];
    int s = 0;
    for (int k = 0; k < 16; k++) {
        int i = t0 + threadIdx.x * 16 + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        int a = __shfl_up_sync(~0u, incl, o);
        if (lane >= o) incl += a;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    int woff = 0;
    for (int k = 0; k < wid; k++) woff += ws[k];
    int run = tile_off[tile] + woff + incl - s;
    for (int k = 0; k < 16; k++) {
        int i = t0 + threadIdx.x * 16 + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    __syncthreads();  // ws is reused by the block's next tile
}

// ------------------------------------------------------------------ warp builder
struct Frame {
    double lo[3], hi[3];
    double w[3];  // sub-cell widths once split
    int a, m, node, depth;
    int b, slot0, next;
    int emit;   // emit work units for the leaves below this cell
    int eself;  // emit this cell itself as one or two work units
};

constexpr int kSmallWarps = 4;
constexpr int kHistMax = 512;  // >= b0^k for any cell of <= kSmallCap particles and s >= 1
constexpr int kTinyHistMax = 64;  // the same for <= kTinyCap particles (s = 1: b = 4)
static_assert(kSmallCap % 32 == 0 && kTinyCap % 32 == 0, "whole particles per lane");

// Per warp; the warps' histograms (2 x hist ints each: counts and offsets)
// follow the kSmallWarps records.
template <int CAP>
struct SmallSmem {
    float x[CAP], y[CAP], z[CAP];  // one array per field, so that
    int id[CAP];                   // the in-place scatter moves one
    float h[CAP];                  // field at a time
    short key[CAP];
    Frame fr[kDepthMax + 2];
    NodeWalk w;
};

// v[pos[k]] = v[k] for k < m (pos a permutation of 0..m-1), in place: each
// lane holds its (at most CAP / 32) values in registers meanwhile.
template <int CAP, class V>
__device__ __forceinline__ void permute_field(V *v, const short *pos, int m, int lane)
{
    V r[CAP / 32];
#pragma unroll
    for (int q = 0; q < CAP / 32; q++)
        if (lane + 32 * q < m) r[q] = v[lane + 32 * q];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < CAP / 32; q++)
        if (lane + 32 * q < m) v[pos[lane + 32 * q]] = r[q];
    __syncwarp();
}

__device__ __forceinline__ int warp_sum(int v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
    return v;
}

// One warp builds the whole sub-tree of one cell of <= CAP particles: an
// instance for cells of up to kSmallCap particles and a leaner one (fewer
// registers and less shared memory: 24 warps per SM instead of 16) for the many
// cells of up to kTinyCap.
template <int CAP>
__global__ void __launch_bounds__(32 * kSmallWarps, CAP == kTinyCap ? 6 : 4)
    k_small(TreeDev T, const SmallItem *items, Src src0, Src src1, Src srcin)
{
    if (T.ctr->abort) return;
    constexpr bool kTiny = CAP == kTinyCap;
    const int nitems = min(kTiny ? T.ctr->ntiny : T.ctr->nsmall, T.cap_small);
    int *const next_ctr = kTiny ? &T.ctr->tiny_next : &T.ctr->small_next;
    const int hcells = kTiny ? T.tiny_hist : T.small_hist;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wid = threadIdx.x >> 5;
    SmallSmem<CAP> &S = reinterpret_cast<SmallSmem<CAP> *>(smem_raw)[wid];
    int *const hist = reinterpret_cast<int *>(smem_raw + kSmallWarps * sizeof(SmallSmem<CAP>)) +
                      wid * 2 * hcells;
    int *const off = hist + hcells;
    const int lane = threadIdx.x & 31;

    // cells are taken one at a time from a shared counter (their costs differ
    // widely), by a grid of as many warps as are resident; the next cell's
    // index is taken while the current one is built
    int it_next = 0, mdep = 0;  // mdep: deepest node made by this warp (lane 0)
    if (lane == 0) it_next = atomicAdd(next_ctr, 1);
    for (;;) {
        const int it = __shfl_sync(~0u, it_next, 0);
        if (it >= nitems) break;
        if (lane == 0) it_next = atomicAdd(next_ctr, 1);
        const SmallItem item = items[it];
        const NodeGeom G = T.geom[item.node];
        const int base = G.start, m0 = G.count;
        const int set = G.set;
        const int s_set = T.set_s[set];
        const int na = T.set_na[set];
        const int gm_set = T.set_gmax[set];
        const bool octree = (T.set_flags[set] & kSetOctree) != 0;
        const bool pack = (T.set_flags[set] & kSetPackLeaves) != 0;
        const int kd = set_dim(T, set);
        const Src src = item.src == 0 ? src0 : (item.src == 1 ? src1 : srcin);
        for (int k = lane; k < m0; k += 32) {
            float4 r;
            float hh;
            src.load(base + k, r, hh);
            S.x[k] = r.x;
            S.y[k] = r.y;
            S.z[k] = r.z;
            S.id[k] = __float_as_int(r.w);
            S.h[k] = hh;
        }
        if (lane == 0) {
            Frame &f = S.fr[0];
            for (int l = 0; l < 3; l++) { f.lo[l] = G.lo[l]; f.hi[l] = G.hi[l]; }
            f.a = 0; f.m = m0; f.node = item.node; f.depth = G.depth;
            f.b = 0; f.slot0 = 0; f.next = 0;
            f.emit = m0 > kWholeMax;
            f.eself = m0 <= kWholeMax;
        }
        int sp = 1;
        bool direct = false;  // particles already written to their final places
        __syncwarp();
        while (sp > 0) {
            Frame &F = S.fr[sp - 1];
            if (F.b == 0) {
                // ---- split cell F (Algorithm 1, Steps 1-3)
                const int a = F.a, m = F.m;
                NodeGeom g;
                for (int l = 0; l < 3; l++) { g.lo[l] = F.lo[l]; g.hi[l] = F.hi[l]; }
                g.start = base + a; g.count = m; g.depth = F.depth; g.set = set;
                int b = octree ? 2 : (kd == 2 ? branching_factor2(m, s_set) : branching_factor(m, s_set));
                for (;;) {
                    if (lane == 0) make_walk(g, b, 0, S.w, kd);
                    __syncwarp();
                    const NodeWalk w = S.w;
                    const int ncell = ncells(b, kd);
                    for (int j = lane; j < ncell; j += 32) hist[j] = 0;
                    __syncwarp();
                    for (int k = lane; k < m; k += 32) {
                        int j = sub_cell_id(make_float4(S.x[a + k], S.y[a + k], S.z[a + k], 0.0f), w, g, b);
                        S.key[a + k] = (short)j;
                        atomicAdd(&hist[j], 1);
                    }
                    __syncwarp();
                    int u = 0;
                    for (int j = lane; j < ncell; j += 32) u += hist[j] <= na;
                    u = warp_sum(u);
                    if (b > 2 && ratio_halves(T, set, u, b)) {
                        b = max(2, b / 2);
                        __syncwarp();
                        continue;
                    }
                    break;
                }
                const int ncell = ncells(b, kd);
                // no-progress guard; internal sub-cells
                int ne = 0, lj = -1, nint = 0;
                for (int j = lane; j < ncell; j += 32) {
                    const int cnt = hist[j];
                    if (cnt > 0) { ne++; lj = j; }
                    nint += cnt > s_set;
                }
                ne = warp_sum(ne);
                nint = F.depth + 1 < kDepthMax ? warp_sum(nint) : 0;
                for (int o = 16; o > 0; o >>= 1) lj = max(lj, __shfl_xor_sync(~0u, lj, o));
                // a cell that splits takes its sub-cells' slots now: the
                // atomic's latency overlaps the scan and the emission below
                // (and, when it is one work unit, that unit's list entry)
                int slot0 = 0, ge = -1;
                if (lane == 0 && ne != 1) {
                    slot0 = atomicAdd(&T.ctr->nslots, ncell);
                    if (F.eself && m <= gm_set) ge = atomicAdd(group_counter(T, set), 1);
                }
                // the binary64 sub-cell widths are needed only for child boxes
                if (ne == 1 || nint > 0) {
                    if (lane == 0)
                        for (int l = 0; l < 3; l++) F.w[l] = cell_width(g.lo[l], g.hi[l], dim_b(b, kd, l));
                    __syncwarp();
                }
                bool leaf = false;
                if (ne == 1) {
                    int cc[3] = {lj % b, (lj / b) % b, lj / (b * b)};
                    bool same = true;
                    for (int l = 0; l < 3; l++) {
                        double clo, chi;
                        child_bounds_w(g.lo[l], g.hi[l], F.w[l], dim_b(b, kd, l), cc[l], clo, chi);
                        if (clo != g.lo[l] || chi != g.hi[l]) same = false;
                    }
                    leaf = same;
                }
                if (leaf) {
                    if (lane == 0) {
                        NodeWalk w;
                        make_walk(g, 0, 0, w, kd);
                        w.b = 0;
                        T.walk[F.node] = w;
                        atomicAdd(&T.ctr->noversized, 1);
                        atomicOr(&T.ctr->status, kStOversized);
                        if (F.emit || F.eself) emit_groups(T, set, base + a, m);
                    }
                    sp--;
                    __syncwarp();
                    continue;
                }
                // exclusive scan of the histogram
                {
                    int carry = 0;
                    for (int j0 = 0; j0 < ncell; j0 += 32) {
                        int j = j0 + lane;
                        int v = j < ncell ? hist[j] : 0;
                        int incl = v;
                        for (int o = 1; o < 32; o <<= 1) {
                            int t = __shfl_up_sync(~0u, incl, o);
                            if (lane >= o) incl += t;
                        }
                        if (j < ncell) off[j] = carry + incl - v;
                        carry += __shfl_sync(~0u, incl, 31);
                    }
                }
                __syncwarp();
                // a cell of <= kWholeMax particles becomes work units of its own
                if (F.eself && lane == 0) {
                    if (m <= gm_set) {
                        if (ge >= 0) emit_write(T, set, ge, base + a, m);
                        else emit_groups(T, set, base + a, m);
                    } else {
                        // two units split at the sub-cell boundary nearest the
                        // middle (sub-cell ids run x fastest: low ids are low z)
                        int bnd = 0, best = m;
                        for (int j = 0; j <= ncell; j++) {
                            const int o = j < ncell ? off[j] : m;
                            const int d = abs(2 * o - m);
                            if (d < best) { best = d; bnd = o; }
                        }
                        if (bnd == 0 || bnd == m) {
                            emit_groups(T, set, base + a, m);
                        } else {
                            emit_groups(T, set, base + a, bnd);
                            emit_groups(T, set, base + a + bnd, m - bnd);
                        }
                    }
                }
                if (lane == 0) {
                    if (ne == 1) slot0 = atomicAdd(&T.ctr->nslots, ncell);
                    if (slot0 + ncell > T.cap_slots) {
                        atomicOr(&T.ctr->status, kStCapSlots);
                        slot0 = -1;
                    }
                }
                slot0 = __shfl_sync(~0u, slot0, 0);
                __syncwarp();
                if (slot0 < 0) {  // out of slot capacity: abandon this sub-tree (host rebuilds)
                    sp = 0;
                    break;
                }
                for (int j = lane; j < ncell; j += 32) {
                    const int cnt = hist[j];
                    const int start = base + a + off[j];
                    const int depth = F.depth + 1;
                    int child = -1;
                    if (cnt > s_set && depth < kDepthMax) {
                        child = atomicAdd(&T.ctr->nnodes, 1);
                        if (child >= T.cap_nodes) {
                            atomicOr(&T.ctr->status, kStCapNodes);
                            child = -1;
                        } else {
                            NodeGeom cg;
                            int cc[3] = {j % b, (j / b) % b, j / (b * b)};
                            for (int l = 0; l < 3; l++)
                                child_bounds_w(g.lo[l], g.hi[l], F.w[l], dim_b(b, kd, l), cc[l], cg.lo[l],
                                               cg.hi[l]);
                            cg.start = start; cg.count = cnt; cg.depth = depth; cg.set = set;
                            T.geom[child] = cg;
                        }
                    } else if (cnt > 0) {
                        if (cnt > s_set) {
                            atomicAdd(&T.ctr->noversized, 1);
                            atomicOr(&T.ctr->status, kStOversized);
                        }
                        if (F.emit && !pack) emit_groups(T, set, start, cnt);
                    }
                    T.slots[slot0 + j] = Slot{start, cnt, child, 0};
                }
                if (F.emit && pack && lane == 0) {
                    // sibling leaves in sub-cell order are adjacent in tree
                    // order: pack runs of them along one x-row of sub-cells
                    // (so that a unit stays compact) into units of <= gmax
                    const int gm = T.set_gmax[set];
                    const int depth = F.depth + 1;
                    int ps = 0, pc = 0, prow = -1;
                    for (int j = 0; j < ncell; j++) {
                        const int cnt = hist[j];
                        if (cnt == 0) continue;
                        const int start = base + a + off[j];
                        if (cnt > s_set && depth < kDepthMax) {  // an internal sub-cell
                            if (pc > 0) emit_groups(T, set, ps, pc);
                            pc = 0;
                            continue;
                        }
                        const int row = j / b;
                        if (pc > 0 && pc + cnt <= gm && start == ps + pc && row == prow) {
                            pc += cnt;
                        } else {
                            if (pc > 0) emit_groups(T, set, ps, pc);
                            ps = start;
                            pc = cnt;
                            prow = row;
                        }
                    }
                    if (pc > 0) emit_groups(T, set, ps, pc);
                }
                __syncwarp();  // S.hist / S.off are rewritten by the scatter below
                if (lane == 0) {
                    NodeWalk w = S.w;  // made for this b above
                    w.slot0 = slot0;
                    T.walk[F.node] = w;
                    mdep = max(mdep, F.depth + 1);
                }
                if (sp == 1 && m0 <= 32 && nint == 0) {
                    // the whole sub-tree is this node and its leaves: each
                    // lane moves its one particle straight to its final place
                    const bool v = lane < m;
                    const int j = v ? S.key[lane] : ncell + lane;
                    const unsigned same = __match_any_sync(~0u, j);
                    if (v) {
                        const int pos = base + off[j] + __popc(same & ((1u << lane) - 1u));
                        const int id = S.id[lane];
                        T.spos[pos] = make_float4(S.x[lane], S.y[lane], S.z[lane], __int_as_float(id));
                        T.sh[pos] = S.h[lane];
                        T.inv[id] = pos;
                    }
                    direct = true;
                    sp = 0;
                    __syncwarp();
                    break;
                }
                // scatter in place: every lane holds its particles in
                // registers while their new positions are taken
                for (int j = lane; j < ncell; j += 32) hist[j] = off[j];
                __syncwarp();
                for (int k = lane; k < m; k += 32)
                    S.key[a + k] = (short)atomicAdd(&hist[S.key[a + k]], 1);  // now the position
                __syncwarp();
                permute_field<CAP>(S.x + a, S.key + a, m, lane);
                permute_field<CAP>(S.y + a, S.key + a, m, lane);
                permute_field<CAP>(S.z + a, S.key + a, m, lane);
                permute_field<CAP>(S.h + a, S.key + a, m, lane);
                permute_field<CAP>(S.id + a, S.key + a, m, lane);
                if (lane == 0) { F.b = b; F.slot0 = slot0; F.next = 0; }
                __syncwarp();
            } else {
                // ---- descend into the next internal sub-cell
                const int ncell = ncells(F.b, kd);
                int found = -1;
                while (F.next < ncell && found < 0) {
                    int j = F.next + lane;
                    bool isint = false;
                    if (j < ncell) isint = T.slots[F.slot0 + j].child >= 0;
                    unsigned bal = __ballot_sync(~0u, isint);
                    if (bal) found = F.next + __ffs(bal) - 1;
                    __syncwarp();
                    if (lane == 0) F.next = bal ? found + 1 : F.next + 32;
                    __syncwarp();
                }
                if (found < 0) {
                    sp--;
                    __syncwarp();
                    continue;
                }
                if (lane == 0) {
                    const Slot s = T.slots[F.slot0 + found];
                    Frame &C = S.fr[sp];
                    const int b = F.b;
                    int cc[3] = {found % b, (found / b) % b, found / (b * b)};
                    for (int l = 0; l < 3; l++)
                        child_bounds_w(F.lo[l], F.hi[l], F.w[l], dim_b(b, kd, l), cc[l], C.lo[l], C.hi[l]);
                    C.a = s.start - base; C.m = s.count; C.node = s.child; C.depth = F.depth + 1;
                    C.b = 0; C.slot0 = 0; C.next = 0;
                    C.emit = F.emit && s.count > kWholeMax;
                    C.eself = F.emit && s.count <= kWholeMax;
                }
                sp++;
                __syncwarp();
            }
        }
        __syncwarp();
        if (!direct)
            for (int k = lane; k < m0; k += 32) {
                const int id = S.id[k];
                T.spos[base + k] = make_float4(S.x[k], S.y[k], S.z[k], __int_as_float(id));
                T.sh[base + k] = S.h[k];
                T.inv[id] = base + k;
            }
        __syncwarp();
    }
    if (lane == 0 && mdep > 0) atomicMax(&T.ctr->max_depth, mdep);
}

size_t small_smem_bytes(int hist_cells, int cap)
{
    const size_t rec = cap == kTinyCap ? sizeof(SmallSmem<kTinyCap>) : sizeof(SmallSmem<kSmallCap>);
    return (rec + 2 * sizeof(int) * (size_t)hist_cells) * kSmallWarps;
}

// ------------------------------------------------------------------ host side
static inline int grid_for(long long work, int per_block, int max_blocks)
{
    long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

void launch_init_sets(const TreeDev &T, const SetRec *rec, int *set_start, int *set_s, int *set_na,
                      double *set_beta, int *set_gmax, int *set_chunk0, cudaStream_t st)
{
    note_launch();
    k_init_sets<<<grid_for(T.nsets, 256, 1 << 16), 256, 0, st>>>(T, rec, set_start, set_s, set_na,
                                                                 set_beta, set_gmax, set_chunk0);
}

void launch_bbox(const TreeDev &T, const float *x, const float *y, const float *z, const float *h,
                 long long chunks, int sms, cudaStream_t st)
{
    note_launch();
    k_bbox<<<grid_for(chunks, 1, sms * 8), 256, 0, st>>>(T, x, y, z, h);
}

void launch_roots(const TreeDev &T, const LevelBufs &L, long long chunks, int sms, cudaStream_t st)
{
    note_launch();
    k_root_sets<<<grid_for(T.nsets, 128, 1 << 16), 128, 0, st>>>(T, L);
    note_launch();
    k_copy_leaf_roots<<<grid_for(chunks, 1, sms * 8), 256, 0, st>>>(T, L.in.x, L.in.y, L.in.z, L.in.h);
}

void launch_level_go(Counters *ctr, int advance, cudaGraphConditionalHandle h, int graph, cudaStream_t st)
{
    note_launch();
    k_level_go<<<1, 1, 0, st>>>(ctr, advance, h, graph);
}

void launch_level_start(const TreeDev &T, const LevelBufs &L, const LevelHints &H, int sms,
                        cudaGraphConditionalHandle hratio, int graph, cudaStream_t st)
{
    note_launch();
    k_level_begin<<<1, 1, 0, st>>>(T.ctr);
    note_launch();
    k_big_setup<<<grid_for(H.nbig, 256, sms * 4), 256, 0, st>>>(T, L);
    note_launch();
    k_big_scan<<<1, 1024, 0, st>>>(T, L, hratio, graph);
}

void launch_level_zero(const TreeDev &T, const LevelBufs &L, const LevelHints &H, int sms, cudaStream_t st)
{
    note_launch();
    k_zero_hist<<<grid_for(H.hist, 256 * 4, sms * 8), 256, 0, st>>>(T.ctr, L.hist);
}

void launch_ratio_pass(const TreeDev &T, const LevelBufs &L, const LevelHints &H, int sms,
                       cudaGraphConditionalHandle hratio, int graph, cudaStream_t st)
{
    note_launch();
    k_big_hist<<<grid_for(H.chunks, 1, sms * 8), 256, 0, st>>>(T, L);
    note_launch();
    k_big_count<<<grid_for(H.hist, 256, sms * 8), 256, 0, st>>>(T, L);
    note_launch();
    k_big_decide<<<grid_for(H.nbig, 128, sms * 4), 128, 0, st>>>(T, L);
    note_launch();
    k_big_zero<<<grid_for(H.hist, 256, sms * 8), 256, 0, st>>>(T.ctr, L);
    note_launch();
    k_ratio_end<<<1, 1, 0, st>>>(T.ctr, hratio, graph);
}

void launch_level_finish(const TreeDev &T, const LevelBufs &L, const LevelHints &H, int sms,
                         cudaGraphConditionalHandle hlevel, int graph, cudaStream_t st)
{
    const int tiles = (int)((H.hist + kScanTile - 1) / kScanTile);
    note_launch();
    k_big_finish<<<grid_for(H.nbig, 128, sms * 4), 128, 0, st>>>(T, L);
    note_launch();
    k_scan_tiles<<<grid_for(tiles, 1, sms * 8), 256, 0, st>>>(T.ctr, L.hist, L.tiles);
    note_launch();
    k_scan_tile_sums<<<1, 1024, 0, st>>>(T.ctr, L.tiles);
    note_launch();
    k_scan_apply<<<grid_for(tiles, 1, sms * 8), 256, 0, st>>>(T.ctr, L.hist, L.tiles, L.hoff);
    note_launch();
    k_big_emit<<<grid_for(H.hist, 256, sms * 16), 256, 0, st>>>(T, L);
    note_launch();
    k_big_scatter<<<grid_for(H.chunks, 1, sms * 8), 256, 0, st>>>(T, L);
    launch_level_go(T.ctr, 1, hlevel, graph, st);
}

int scan_tile_count(long long n) { return (int)((n + kScanTile - 1) / kScanTile) + 1; }

template <int CAP>
static void launch_small_cap(const TreeDev &T, const LevelBufs &L, long long nitems_hint, int sms,
                             cudaStream_t st)
{
    if (nitems_hint <= 0) return;
    const Src s0{nullptr, nullptr, nullptr, nullptr, L.wpos[0], L.wh[0]};
    const Src s1{nullptr, nullptr, nullptr, nullptr, L.wpos[1], L.wh[1]};
    const size_t smem = small_smem_bytes(CAP == kTinyCap ? T.tiny_hist : T.small_hist, CAP);
    // as many blocks as are resident at once (the warps take cells from a
    // counter until none is left)
    static thread_local size_t occ_smem = 0;
    static thread_local int occ_blocks = 0;
    if (occ_smem != smem) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small<CAP>, 32 * kSmallWarps, smem) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        occ_smem = smem;
        occ_blocks = per_sm;
    }
    const int blocks = grid_for(nitems_hint, kSmallWarps, sms * occ_blocks);
    note_launch();
    k_small<CAP><<<blocks, 32 * kSmallWarps, smem, st>>>(T, CAP == kTinyCap ? L.tiny : L.small, s0, s1, L.in);
}

void launch_small(const TreeDev &T, const LevelBufs &L, long long nsmall_hint, long long ntiny_hint, int sms,
                  cudaStream_t st)
{
    launch_small_cap<kTinyCap>(T, L, ntiny_hint, sms, st);
    launch_small_cap<kSmallCap>(T, L, nsmall_hint, sms, st);
}

cudaError_t build_init_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_small<kSmallCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)small_smem_bytes(kHistMax, kSmallCap));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_small<kTinyCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)small_smem_bytes(kTinyHistMax, kTinyCap));
}

// One thread: copy the counters (and node 0's b) into the mapped host mirror.
__global__ void k_readback(const Counters *__restrict__ ctr, const NodeWalk *__restrict__ walk0,
                           Readback *out)
{
    out->c = *ctr;
    out->root_b = walk0 ? walk0->b : 0;
    __threadfence_system();
}

__global__ void k_readback_total(const long long *__restrict__ total, Readback *out)
{
    out->total = *total;
    __threadfence_system();
}

void launch_readback(const Counters *ctr, const NodeWalk *walk0, Readback *out, cudaStream_t st)
{
    k_readback<<<1, 1, 0, st>>>(ctr, walk0, out);
}

void launch_readback_total(const long long *total, Readback *out, cudaStream_t st)
{
    k_readback_total<<<1, 1, 0, st>>>(total, out);
}

__global__ void k_init_counters(Counters *ctr, int nroots)
{
    Counters c = {};
    c.nnodes = nroots;  // nodes 0 .. nroots-1 are the set roots
    *ctr = c;
}

void launch_init_counters(Counters *ctr, int nroots, cudaStream_t st)
{
    note_launch();
    k_init_counters<<<1, 1, 0, st>>>(ctr, nroots);
}

}  // namespace bt
