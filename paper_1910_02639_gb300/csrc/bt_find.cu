// bt_find.cu -- FindNeighbors (Algorithm 2 of arXiv:1910.02639) on the GPU,
// optionally fused with the SPH density sum (M4 cubic spline).
//
// Work unit: a group of <= 32 particles contiguous in tree order (a leaf, a
// cell of <= 32 particles, a run of sibling leaves, or a slice of an
// oversized leaf) of one particle set, one block at a time (blocks are
// persistent and stride over the groups).  Two block shapes, chosen per set:
// 8 warps with a 1024-candidate window, or 4 warps with 512.  Per group:
//   1. warp 0 loads the queries; then all threads walk the tree once for the
//      union of their search intervals (Eqs. 5-6 applied to the group's query
//      box), frontier by frontier, collecting contiguous particle ranges
//      (x-runs of sub-cells in Eq. 3 order; internal sub-cells of <= 256
//      particles are taken whole) as 32-particle jobs;
//   2. all warps stream the jobs with several coalesced float4 loads in
//      flight per lane and keep the candidates within 2*h_max of the group's
//      bounding box;
//   3. the kept candidates are sorted by original index (bitonic, registers);
//      in scan mode (very wide groups) they are collected already sorted;
//   4. stage A: every 32-candidate chunk is tested against every query with
//      an FP32 filter whose error band is certified; pairs inside the band
//      are decided by the binary64 definition; one ballot per (query, chunk);
//   5. stage B: per query, the ballots are compacted (prefix sums) into a
//      list of hit positions which the warp writes out lane-parallel as the
//      ascending, capped row, accumulating the density terms in that order
//      when fused.
// Groups whose candidate set exceeds the buffer, or spans too many original
// indices for 32-bit sort keys, are processed in windows of original index
// (same results, more passes).  The same kernel also counts only (compressed
// rows, first pass), writes rows at given offsets (second pass), and keeps
// only j > i (half rows).
#include "bt_internal.cuh"
#include "bt_sort.cuh"
#include "bt_find.cuh"

#include <cfloat>
#include <mutex>

namespace bt {

// Two block shapes, chosen per particle set (BT_SET_FIND_COMPACT): 8 warps
// per work unit with a 1024-candidate window, or 4 warps with a 512-candidate
// window (more work units resident per SM).  Same results.
template <int NT_, int CAP_, int SLOT_BITS_>
struct FindCfg {
    static constexpr int NT = NT_;              // threads per work unit
    static constexpr int WARPS = NT_ / 32;
    static constexpr int CAP = CAP_;            // candidates per window
    static constexpr int SLOT_BITS = SLOT_BITS_;  // log2(CAP)
    static constexpr int CHUNKS = CAP_ / 32;
    static constexpr int JOB_MAX = CAP_ / 2;    // 32-particle jobs per group walk
};
using CfgWide = FindCfg<256, 1024, 10>;
using CfgCompact = FindCfg<128, 512, 9>;
constexpr int kSpanMax = (1 << 22) - 1;    // original-index span of one window
constexpr int kFrontMax = 64;              // tree nodes per walk frontier
constexpr int kDescendMin = 256;           // internal sub-cells up to this size are scanned whole
                                           // (fewer walk levels on deep trees; 32 was 2-26 % slower)
constexpr int kFindChunk = 1;              // groups per block step (more: heavy neighbours
                                           // land on one block and stretch the tail)
constexpr int kHitBatch = 256;             // hit positions staged per warp and pass
constexpr int kUnroll = 2;                 // gather jobs in flight per warp (more spills registers)
constexpr int kSortThreads = 128;          // warps 0-3 sort; the others wait
constexpr float kPiF = 3.14159265358979f;

template <class C>
struct FindSmem {
    float4 cand[C::CAP];        // x, y, z, original index (bits)
    float cmass[C::CAP];
    uint32_t key[C::CAP];       // (orig - kmin) << C::SLOT_BITS | slot, sorted
    uint32_t mask[kGroupMax * C::CHUNKS];
    // density partial sums: slot k of query p holds the terms whose position
    // in p's ascending neighbour list is k mod 32, so the summation order
    // depends on the list alone (not on windows or work-unit composition)
    float qacc[kGroupMax][32];
    int2 jobs[C::JOB_MAX];       // (first tree position, length <= 32)
    float4 q[kGroupMax];      // x, y, z, R_lo
    float qrhi[kGroupMax];
    float qh[kGroupMax];
    int qorig[kGroupMax];
    int qself[kGroupMax];     // sorted position of the query itself, or -1
    int qlow[kGroupMax];      // half rows: candidates below this sorted position are dropped
    int qcnt[kGroupMax];
    // Three arrays of three phases of a work unit share their storage: the
    // walk's frontiers (once per unit, first), the histogram of the window
    // planning (gather), and the hit positions of stage B (last, per window).
    union {
        struct {
            int front[2][kFrontMax];  // walk frontiers
            int fr_rx0[kFrontMax], fr_rx1[kFrontMax], fr_ry0[kFrontMax], fr_ny[kFrontMax];
            int fr_rz0[kFrontMax], fr_row0[kFrontMax], fr_b[kFrontMax], fr_off[kFrontMax + 1];
        };
        int hist[256];
        unsigned short hits[C::WARPS][kHitBatch];
    };
    float box[13];            // PL[3] PH[3] QL[3] QH[3] T
    int njobs, nfront, nnext, ncand, kmin, kmax, range_ovf, ovf_lo, ovf_hi;
    int jfail, cover, gstart, gcount, whi, ctot;
    int wcnt[2][C::WARPS];  // per-warp kept counts (scan mode), double-buffered
    int gset, set_lo, set_hi;  // the group's particle set and its index range
    int split;                 // the unit went to the split pass
};

struct FindArgs {
    TreeDev T;
    int ngmax;
    int32_t *nbrs;
    int32_t *counts;
    const float *smass;  // masses in tree order (density only)
    float *rho;
    int ngroups;  // >= 0: work units of this list; < 0: read on the device
    int list;     // 0: the wide-shape list (front of T.groups); 1: the compact list (back)
    // compressed rows: row i at nbrs + row_off[i], length row_off[i+1] - row_off[i]
    // (null: fixed rows of ngmax); count_only: counts (and density), no rows
    const long long *row_off;
    int count_only;
    int half;  // rows hold only j > i (each pair once when h is uniform)
};

__device__ __forceinline__ float warp_min(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(~0u, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(~0u, v, o));
    return v;
}

// Binary64 predicate of the definition (Algorithm 2 / Sec. 3.2).
__device__ __forceinline__ bool exact_neighbor(float4 p, float hp, float4 qd)
{
    double dx = __dsub_rn((double)qd.x, (double)p.x);
    double dy = __dsub_rn((double)qd.y, (double)p.y);
    double dz = __dsub_rn((double)qd.z, (double)p.z);
    double d = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    d = __dadd_rn(d, __dmul_rn(dz, dz));
    double two_h = __dmul_rn(2.0, (double)hp);
    return d < __dmul_rn(two_h, two_h);
}

// Append a contiguous particle range as 32-particle jobs.
template <class C>
__device__ __forceinline__ void add_range(FindSmem<C> &S, int s, int len)
{
    if (len <= 0) return;
    const int nj = (len + 31) >> 5;
    atomicAdd(&S.ctot, len);
    const int j0 = atomicAdd(&S.njobs, nj);
    if (j0 + nj <= C::JOB_MAX) {
        for (int k = 0; k < nj; k++) S.jobs[j0 + k] = make_int2(s + 32 * k, min(32, len - 32 * k));
    } else {
        // jobs [0, jfail) were all written; everything else is covered by
        // [ovf_lo, ovf_hi)
        atomicMin(&S.jfail, j0);
        atomicMin(&S.ovf_lo, s);
        atomicMax(&S.ovf_hi, s + len);
        S.range_ovf = 1;
    }
}

// All threads: the tree walk for the group's query box, one frontier of
// nodes at a time; the rows of all frontier nodes are spread over the block.
template <class C>
__device__ void group_walk(const TreeDev &T, FindSmem<C> &S)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        S.njobs = 0;
        S.ctot = 0;
        S.cover = 0;
        S.range_ovf = 0;
        S.jfail = C::JOB_MAX;
        S.ovf_lo = INT_MAX;
        S.ovf_hi = INT_MIN;
        S.front[0][0] = S.gset;  // root of the group's set
        S.nfront = 1;
        S.nnext = 0;
    }
    __syncthreads();
    const float QL0 = S.box[6], QL1 = S.box[7], QL2 = S.box[8];
    const float QH0 = S.box[9], QH1 = S.box[10], QH2 = S.box[11];
    int cur = 0;
    for (;;) {
        const int nf = S.nfront;
        if (nf == 0) break;
        // per-node ranges
        if (tid < nf) {
            const NodeWalk W = T.walk[S.front[cur][tid]];
            int rows = 0;
            if (W.b == 0) {
                add_range(S, W.start, W.count);
            } else {
                int rx0, rx1, ry0, ry1, rz0, rz1;
                walk_range(QL0, QH0, W, 0, rx0, rx1);
                walk_range(QL1, QH1, W, 1, ry0, ry1);
                walk_range(QL2, QH2, W, 2, rz0, rz1);
                if (rx1 >= rx0 && ry1 >= ry0 && rz1 >= rz0) {
                    rows = (ry1 - ry0 + 1) * (rz1 - rz0 + 1);
                    S.fr_rx0[tid] = rx0;
                    S.fr_rx1[tid] = rx1;
                    S.fr_ry0[tid] = ry0;
                    S.fr_ny[tid] = ry1 - ry0 + 1;
                    S.fr_rz0[tid] = rz0;
                    S.fr_row0[tid] = W.slot0;
                    S.fr_b[tid] = W.b;
                }
            }
            S.fr_off[tid] = rows;
        }
        __syncthreads();
        if (tid < 32) {  // exclusive prefix of rows over the frontier
            int carry = 0;
            for (int i0 = 0; i0 < nf; i0 += 32) {
                const int i = i0 + tid;
                const int v = i < nf ? S.fr_off[i] : 0;
                int incl = v;
                for (int o = 1; o < 32; o <<= 1) {
                    int t = __shfl_up_sync(~0u, incl, o);
                    if (tid >= o) incl += t;
                }
                if (i < nf) S.fr_off[i] = carry + incl - v;
                carry += __shfl_sync(~0u, incl, 31);
            }
            if (tid == 0) S.fr_off[nf] = carry;
        }
        __syncthreads();
        const int total = S.fr_off[nf];
        for (int r = tid; r < total; r += C::NT) {
            int lo = 0, hi = nf - 1;  // frontier node owning row r
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.fr_off[mid] <= r) lo = mid; else hi = mid - 1;
            }
            const int lr = r - S.fr_off[lo];
            const int ny = S.fr_ny[lo], b = S.fr_b[lo];
            const int cy = S.fr_ry0[lo] + lr % ny;
            const int cz = S.fr_rz0[lo] + lr / ny;
            const int row = S.fr_row0[lo] + b * (cy + b * cz);
            const int rx0 = S.fr_rx0[lo], rx1 = S.fr_rx1[lo];
            int cs = 0, cl = 0;
            for (int cx0 = rx0; cx0 <= rx1; cx0 += 4) {
                Slot sl[4];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (cx0 + u <= rx1) sl[u] = T.slots[row + cx0 + u];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (cx0 + u > rx1) break;
                    if (sl[u].child >= 0 && sl[u].count > kDescendMin) {
                        add_range(S, cs, cl);
                        cl = 0;
                        const int k = atomicAdd(&S.nnext, 1);
                        if (k < kFrontMax) S.front[cur ^ 1][k] = sl[u].child;
                        else add_range(S, sl[u].start, sl[u].count);  // whole sub-tree
                    } else if (sl[u].count > 0) {
                        if (cl == 0) cs = sl[u].start;
                        cl = sl[u].start + sl[u].count - cs;
                    }
                }
            }
            add_range(S, cs, cl);
        }
        __syncthreads();
        if (tid == 0) {
            S.nfront = min(S.nnext, kFrontMax);
            S.nnext = 0;
        }
        cur ^= 1;
        __syncthreads();
    }
    if (S.range_ovf) {
        // Too many jobs: replace them by the one range that covers them all
        // (a superset, and no particle appears twice).
        if (tid < 32) {
            int lo = S.ovf_lo, hi = S.ovf_hi;
            const int nj = min(S.jfail, C::JOB_MAX);
            for (int r = tid; r < nj; r += 32) {
                const int2 jb = S.jobs[r];
                lo = min(lo, jb.x);
                hi = max(hi, jb.x + jb.y);
            }
            for (int o = 16; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(~0u, lo, o));
                hi = max(hi, __shfl_xor_sync(~0u, hi, o));
            }
            if (tid == 0) {
                S.jobs[0] = make_int2(lo, hi - lo);
                S.njobs = (hi - lo + 31) >> 5;
                S.ctot = hi - lo;
                S.cover = 1;
                atomicOr(&T.ctr->status, kStWalk);
            }
        }
        __syncthreads();
    }
}

// Stream the candidates of the collected jobs.  mode 0: collect those with
// original index in [wlo, whi) into the buffer; mode 1: histogram them into
// 256 bins of width W starting at wlo.
template <bool DENS, class C>
__device__ void group_gather(const FindArgs &A, FindSmem<C> &S, int mode, int wlo, int whi, int W)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float PL0 = S.box[0], PL1 = S.box[1], PL2 = S.box[2];
    const float PH0 = S.box[3], PH1 = S.box[4], PH2 = S.box[5];
    const float T2 = S.box[12];
    const int njobs = S.njobs;
    const bool cover = S.cover;
    const int2 cv = S.jobs[0];
    const unsigned lt = (1u << lane) - 1;
    int kmin = INT_MAX, kmax = INT_MIN;
    for (int j0 = warp * kUnroll; j0 < njobs; j0 += C::WARPS * kUnroll) {
        float4 c[kUnroll];
        float mm[kUnroll];
        bool keep[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int job = j0 + u;
            int t = 0;
            bool ok = false;
            if (job < njobs) {
                const int2 jb = cover ? make_int2(cv.x + 32 * job, min(32, cv.y - 32 * job)) : S.jobs[job];
                ok = lane < jb.y;
                t = jb.x + lane;
            }
            c[u] = ok ? __ldg(&A.T.spos[t]) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (DENS) mm[u] = ok ? __ldg(&A.smass[t]) : 0.0f;
            keep[u] = ok;
        }
        unsigned bal[kUnroll];
        int tot = 0;
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int orig = __float_as_int(c[u].w);
            const float ex = fmaxf(fmaxf(__fsub_rn(PL0, c[u].x), __fsub_rn(c[u].x, PH0)), 0.0f);
            const float ey = fmaxf(fmaxf(__fsub_rn(PL1, c[u].y), __fsub_rn(c[u].y, PH1)), 0.0f);
            const float ez = fmaxf(fmaxf(__fsub_rn(PL2, c[u].z), __fsub_rn(c[u].z, PH2)), 0.0f);
            const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
            keep[u] = keep[u] && d2 <= T2 && orig >= wlo && orig < whi;
            if (mode == 0) {
                bal[u] = __ballot_sync(~0u, keep[u]);
                tot += __popc(bal[u]);
            } else if (keep[u]) {
                atomicAdd(&S.hist[(int)((unsigned)(orig - wlo) / (unsigned)W)], 1);
            }
        }
        if (mode == 0 && tot > 0) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&S.ncand, tot);
            base = __shfl_sync(~0u, base, 0);
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (keep[u]) {
                    const int slot = base + __popc(bal[u] & lt);
                    if (slot < C::CAP) {
                        S.cand[slot] = c[u];
                        if (DENS) S.cmass[slot] = mm[u];
                    }
                    const int orig = __float_as_int(c[u].w);
                    kmin = min(kmin, orig);
                    kmax = max(kmax, orig);
                }
                base += __popc(bal[u]);
            }
        }
    }
    if (mode == 0) {
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(~0u, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(~0u, kmax, o));
        }
        if (lane == 0 && kmin <= kmax) {
            atomicMin(&S.kmin, kmin);
            atomicMax(&S.kmax, kmax);
        }
    }
}

__device__ __forceinline__ float m4_shape(float q)
{
    const float t = 2.0f - q;
    const float w2 = 0.25f * t * t * t;
    const float w1 = fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f);
    return q < 1.0f ? w1 : (q < 2.0f ? w2 : 0.0f);
}

template <int E>
__device__ __forceinline__ void sort_keys(uint32_t *buf)
{
    block_sort<kSortThreads, E>(buf);
}

// Packed pairs of FP32 lanes (sm_100+ f32x2 arithmetic, round-to-nearest per
// element, the same results as the scalar operations).
__device__ __forceinline__ unsigned long long f2_pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Stage A for two candidates per lane (one from each of two chunks): the
// squared FP32 distances to query P, two at a time.  Same arithmetic as
// test_chunk: d2 = fma(dz, dz, fma(dy, dy, dx * dx)).
__device__ __forceinline__ void dist2_pair(const float4 &P, unsigned long long qx,
                                           unsigned long long qy, unsigned long long qz, float &d1,
                                           float &d2)
{
    const unsigned long long dx = f2_sub(qx, f2_pack(P.x, P.x));
    const unsigned long long dy = f2_sub(qy, f2_pack(P.y, P.y));
    const unsigned long long dz = f2_sub(qz, f2_pack(P.z, P.z));
    const unsigned long long r = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
    f2_unpack(r, d1, d2);
}

// One FP32 filter step of stage A: the ballot of hits of query P over this
// lane's candidate Q, and whether the pair lies in the uncertain band.
__device__ __forceinline__ unsigned test_chunk(const float4 &P, float rhi, const float4 &Q,
                                               bool valid, bool &amb)
{
    const float dx = Q.x - P.x, dy = Q.y - P.y, dz = Q.z - P.z;
    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const bool hit = valid && d2 < P.w;
    amb |= valid && !hit && d2 <= rhi;
    return __ballot_sync(~0u, hit);
}

template <class C>
__device__ __forceinline__ void fix_band(FindSmem<C> &S, int c, int gcount, const float4 &Q, int lane)
{
    for (int p = 0; p < gcount; p++) {
        const float4 P = S.q[p];
        const float dx = Q.x - P.x, dy = Q.y - P.y, dz = Q.z - P.z;
        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (!(d2 < P.w) && d2 <= S.qrhi[p] && exact_neighbor(P, S.qh[p], Q))
            atomicOr(&S.mask[p * C::CHUNKS + c], 1u << lane);
    }
}

// Sort, test and emit the candidates of the current window.
// `presorted`: the candidates were collected in ascending original index
// and their keys are already in S.key (scan mode).
template <bool DENS, class C>
__device__ void group_window(const FindArgs &A, FindSmem<C> &S, bool presorted)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = S.ncand;  // <= C::CAP here
    const int gcount = S.gcount;
    if (m == 0) return;
    const int kmin = S.kmin;
    if (!presorted) {
        int npad = kSortThreads;
        while (npad < m) npad <<= 1;
        for (int s = tid; s < npad; s += C::NT) {
            uint32_t k = 0xffffffffu;
            if (s < m) k = ((uint32_t)(__float_as_int(S.cand[s].w) - kmin) << C::SLOT_BITS) | (uint32_t)s;
            S.key[s] = k;
        }
        __syncthreads();
        if (tid < kSortThreads) {
            switch (npad) {
            case kSortThreads: sort_keys<1>(S.key); break;
            case 2 * kSortThreads: sort_keys<2>(S.key); break;
            case 4 * kSortThreads: sort_keys<4>(S.key); break;
            default:
                if constexpr (C::CAP > 4 * kSortThreads) sort_keys<8>(S.key);
                break;
            }
        }
        __syncthreads();
    }
    // sorted position of each query itself (it is its own candidate when its
    // original index lies in this window)
    if (tid < gcount) {
        const int o = S.qorig[tid];
        const uint32_t want = (uint32_t)(o - kmin);
        int lo = 0, hi = m;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((S.key[mid] >> C::SLOT_BITS) < want) lo = mid + 1; else hi = mid;
        }
        S.qself[tid] = (o >= kmin && lo < m && (S.key[lo] >> C::SLOT_BITS) == want) ? lo : -1;
        // half rows keep j > i only: drop every candidate up to the query itself
        S.qlow[tid] = o < kmin ? 0 : (S.qself[tid] >= 0 ? lo + 1 : lo);
    }

    // ---- stage A: one ballot per (query, chunk); two chunks per pass
    const int nch = (m + 31) >> 5;
    const bool halves = nch <= 16;  // stage B: two lanes per chunk
    for (int c = warp; c < nch; c += 2 * C::WARPS) {
        const int c2 = c + C::WARPS;
        if (C::WARPS == 8 && c2 >= nch) {
            // 8-warp shape: a chunk without a partner takes one candidate per
            // lane (cheaper than a half-empty packed pass; measured 4-6 %
            // faster on near-uniform sets; with 4 warps it measured slower)
            const int k1 = c * 32 + lane;
            const bool v1 = k1 < m;
            float4 Q1 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (v1) Q1 = S.cand[S.key[k1] & (C::CAP - 1)];
            bool amb1 = false;
            for (int p = 0; p < gcount; p++) {
                const unsigned b1 = test_chunk(S.q[p], S.qrhi[p], Q1, v1, amb1);
                if (lane == 0) S.mask[p * C::CHUNKS + c] = b1;
            }
            __syncwarp();
            if (__any_sync(~0u, amb1)) {
                if (amb1) fix_band(S, c, gcount, Q1, lane);
                __syncwarp();
            }
            continue;
        }
        const bool has2 = c2 < nch;
        const int k1 = c * 32 + lane, k2 = c2 * 32 + lane;
        const bool v1 = k1 < m, v2 = k2 < m;
        float4 Q1 = make_float4(0.f, 0.f, 0.f, 0.f), Q2 = Q1;
        if (v1) Q1 = S.cand[S.key[k1] & (C::CAP - 1)];
        if (v2) Q2 = S.cand[S.key[k2] & (C::CAP - 1)];
        bool amb1 = false, amb2 = false;
        const unsigned long long qx = f2_pack(Q1.x, Q2.x), qy = f2_pack(Q1.y, Q2.y),
                                 qz = f2_pack(Q1.z, Q2.z);
        for (int p = 0; p < gcount; p++) {
            const float4 P = S.q[p];
            const float rhi = S.qrhi[p];
            float d1, d2;
            dist2_pair(P, qx, qy, qz, d1, d2);
            const bool h1 = v1 && d1 < P.w, h2 = v2 && d2 < P.w;
            amb1 |= v1 && !h1 && d1 <= rhi;
            amb2 |= v2 && !h2 && d2 <= rhi;
            const unsigned b1 = __ballot_sync(~0u, h1);
            const unsigned b2 = __ballot_sync(~0u, h2);
            if (lane == 0) {
                S.mask[p * C::CHUNKS + c] = b1;
                if (has2) S.mask[p * C::CHUNKS + c2] = b2;
            }
        }
        __syncwarp();
        if (__any_sync(~0u, amb1)) {
            if (amb1) fix_band(S, c, gcount, Q1, lane);
            __syncwarp();
        }
        if (__any_sync(~0u, amb2)) {
            if (amb2) fix_band(S, c2, gcount, Q2, lane);
            __syncwarp();
        }
    }
    __syncthreads();

    // ---- stage B: per query, compact the ballots into hit positions, then
    // write the row (and the density terms) lane-parallel in ascending order.
    unsigned short *hl = S.hits[warp];
    for (int p = warp; p < gcount; p += C::WARPS) {
        // lane -> (chunk, half): with at most 16 chunks every chunk's mask
        // is split over two lanes (16 candidates each), so the extraction
        // loop below runs half as long; lanes stay in candidate order
        const int ch = halves ? (lane >> 1) : lane;
        uint32_t mk = ch < nch ? S.mask[p * C::CHUNKS + ch] : 0u;
        const int sr = S.qself[p];
        if (sr >= 0 && ch == (sr >> 5)) mk &= ~(1u << (sr & 31));
        if (A.half) {
            const int low = S.qlow[p];
            const int c0 = ch * 32;
            if (c0 + 32 <= low) mk = 0u;
            else if (c0 < low) mk &= ~((1u << (low - c0)) - 1u);
        }
        const int sh16 = halves ? (lane & 1) * 16 : 0;
        if (halves) mk = (mk >> sh16) & 0xffffu;
        const int bitbase = ch * 32 + sh16;  // candidate of bit 0 of mk
        const int cnt = __popc(mk);
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(~0u, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(~0u, incl, 31);
        const int excl = incl - cnt;
        const int base = S.qcnt[p];
        const long long qo = S.qorig[p];
        int32_t *row = A.row_off ? A.nbrs + A.row_off[qo] : A.nbrs + qo * A.ngmax;
        const long long rowcap = A.count_only ? 0
                                 : (A.row_off ? A.row_off[qo + 1] - A.row_off[qo] : (long long)A.ngmax);
        const float4 P = S.q[p];
        const float inv_h = DENS ? __frcp_rn(S.qh[p]) : 0.0f;
        // lane L takes the list positions congruent to L mod 32 and continues
        // its slot of the running density sum
        const int i0 = (lane - base) & 31;
        float acc = DENS ? S.qacc[p][lane] : 0.0f;
        for (int b0 = 0; b0 < total; b0 += kHitBatch) {
            if (total <= kHitBatch) {
                uint32_t mm = mk;
                int r = excl;
                while (mm) {
                    hl[r++] = (unsigned short)(bitbase + __ffs(mm) - 1);
                    mm &= mm - 1;
                }
            } else if (excl < b0 + kHitBatch && excl + cnt > b0) {
                uint32_t mm = mk;
                int r = excl;
                while (mm) {
                    const int bit = __ffs(mm) - 1;
                    mm &= mm - 1;
                    if (r >= b0 && r < b0 + kHitBatch) hl[r - b0] = (unsigned short)(bitbase + bit);
                    r++;
                }
            }
            __syncwarp();
            const int nb = min(kHitBatch, total - b0);
            // two list positions per step (i, i + 32) so that their
            // shared-memory loads overlap; the density terms are still
            // added in position order
            for (int i = i0; i < nb; i += 64) {
                const bool two = i + 32 < nb;
                const uint32_t key1 = S.key[hl[i]];
                const uint32_t key2 = two ? S.key[hl[i + 32]] : 0u;
                const int pos = base + b0 + i;
                const int vbase = kmin - S.set_lo;
                if (pos < rowcap) row[pos] = vbase + (int)(key1 >> C::SLOT_BITS);
                if (two && pos + 32 < rowcap) row[pos + 32] = vbase + (int)(key2 >> C::SLOT_BITS);
                if (DENS) {
                    const int s1 = key1 & (C::CAP - 1), s2 = key2 & (C::CAP - 1);
                    const float4 Q1 = S.cand[s1];
                    const float4 Q2 = S.cand[s2];
                    const float m1 = S.cmass[s1], m2 = S.cmass[s2];
                    const float dx1 = Q1.x - P.x, dy1 = Q1.y - P.y, dz1 = Q1.z - P.z;
                    const float dx2 = Q2.x - P.x, dy2 = Q2.y - P.y, dz2 = Q2.z - P.z;
                    const float e1 = fmaf(dz1, dz1, fmaf(dy1, dy1, dx1 * dx1));
                    const float e2 = fmaf(dz2, dz2, fmaf(dy2, dy2, dx2 * dx2));
                    const float q1 = e1 > 0.0f ? e1 * rsqrtf(e1) * inv_h : 0.0f;
                    const float q2 = e2 > 0.0f ? e2 * rsqrtf(e2) * inv_h : 0.0f;
                    const float w1 = m4_shape(q1), w2 = m4_shape(q2);
                    acc = fmaf(m1, w1, acc);
                    if (two) acc = fmaf(m2, w2, acc);
                }
            }
            __syncwarp();
        }
        if (DENS) S.qacc[p][lane] = acc;
        if (lane == 0) S.qcnt[p] = base + total;
    }
    __syncthreads();
}

// Scan mode, for a group whose query box holds a large part of its set (very
// large h): instead of re-streaming the candidates once per window, walk the
// set in ascending original index through the inverse permutation, keep the
// particles inside the box, and cut windows of at most C::CAP candidates that
// arrive already sorted.  Block-wide: one round = C::NT indices.
template <bool DENS, class C>
__device__ void group_scan(const FindArgs &A, FindSmem<C> &S)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float PL0 = S.box[0], PL1 = S.box[1], PL2 = S.box[2];
    const float PH0 = S.box[3], PH1 = S.box[4], PH2 = S.box[5];
    const float T2 = S.box[12];
    const unsigned lt = (1u << lane) - 1;
    const int jend = S.set_hi;
    int j0 = S.set_lo;
    int buf = 0;
    while (j0 < jend) {
        const int kmin = j0;
        int base = 0;  // candidates kept so far in this window (same in all threads)
        int j = j0;
        for (; j < jend; j += C::NT) {
            if (j - kmin > kSpanMax - C::NT) break;  // keys must fit their bits
            const int idx = j + tid;
            bool keep = false;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            float mm = 0.0f;
            if (idx < jend) {
                const int p = __ldg(&A.T.inv[idx]);
                c = __ldg(&A.T.spos[p]);
                if (DENS) mm = __ldg(&A.smass[p]);
                const float ex = fmaxf(fmaxf(__fsub_rn(PL0, c.x), __fsub_rn(c.x, PH0)), 0.0f);
                const float ey = fmaxf(fmaxf(__fsub_rn(PL1, c.y), __fsub_rn(c.y, PH1)), 0.0f);
                const float ez = fmaxf(fmaxf(__fsub_rn(PL2, c.z), __fsub_rn(c.z, PH2)), 0.0f);
                keep = fmaf(ez, ez, fmaf(ey, ey, ex * ex)) <= T2;
            }
            const unsigned bal = __ballot_sync(~0u, keep);
            if (lane == 0) S.wcnt[buf][warp] = __popc(bal);
            __syncthreads();
            int before = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < C::WARPS; w++) {
                const int v = S.wcnt[buf][w];
                before += w < warp ? v : 0;
                tot += v;
            }
            buf ^= 1;
            if (base + tot > C::CAP) break;  // uniform: this round opens the next window
            if (keep) {
                const int slot = base + before + __popc(bal & lt);
                S.cand[slot] = c;
                if (DENS) S.cmass[slot] = mm;
                S.key[slot] = ((uint32_t)(idx - kmin) << C::SLOT_BITS) | (uint32_t)slot;
            }
            base += tot;
        }
        if (tid == 0) {
            S.ncand = base;
            S.kmin = kmin;
        }
        __syncthreads();
        group_window<DENS>(A, S, true);
        j0 = j;
    }
}

// The free middle of the groups array: the 8-warp units fill it from the
// front (nf0 of them), the compact ones from the back; room entries are left.
__device__ __forceinline__ void free_part(const TreeDev &T, int &nf0, int &room)
{
    nf0 = T.ctr->abort ? 0 : min(T.ctr->ngroups, T.cap_groups);
    const int nc0 = T.ctr->abort ? 0 : min(T.ctr->ngroups_c, T.cap_groups - nf0);
    room = T.cap_groups - nf0 - nc0;
}

// Reserve one-query units there for the gc queries of a unit starting at
// tree position first; false (placeholders of count 0 written) when the
// free part is full: the unit is then searched whole by its own block.
__device__ __noinline__ bool split_unit(const TreeDev &T, int first, int gc, int set)
{
    int nf0, room;
    free_part(T, nf0, room);
    const int k = atomicAdd(&T.ctr->nsplit, gc);
    const int fit = max(0, min(gc, room - k));
    for (int i = 0; i < fit; i++)
        T.groups[nf0 + k + i] = make_int2(fit == gc ? first + i : 0, group_pack(set, fit == gc ? 1 : 0));
    return fit == gc;
}

template <class C, bool DENS>
__global__ void __launch_bounds__(C::NT, C::NT == 128 ? 9 : 1024 / C::NT) k_find(FindArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FindSmem<C> &S = *reinterpret_cast<FindSmem<C> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TreeDev &T = A.T;
    // ngroups < 0: read the count the build left on the device (graph form).
    // The wide-shape list runs forward from the start of T.groups, the
    // compact one backward from its end (clamped so that both stay inside).
    // The split pass (list 2) reads the units written into the free middle.
    int ngroups = A.ngroups;
    const int2 *G;
    if (A.list == 2) {
        int nf0, room;
        free_part(T, nf0, room);
        ngroups = min(T.ctr->nsplit, room);
        G = T.groups + nf0;
    } else {
        if (ngroups < 0) {
            const int nf = T.ctr->abort ? 0 : min(T.ctr->ngroups, T.cap_groups);
            ngroups = A.list == 0 ? nf : (T.ctr->abort ? 0 : min(T.ctr->ngroups_c, T.cap_groups - nf));
        }
        G = A.list == 0 ? T.groups : T.groups + (T.cap_groups - ngroups);
    }
    const int nchunks = (ngroups + kFindChunk - 1) / kFindChunk;

    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const int g1 = min(chunk * kFindChunk + kFindChunk, ngroups);
        for (int g = chunk * kFindChunk; g < g1; g++) {
            __syncthreads();
            if (A.list == 2 && group_count(G[g].y) == 0) continue;  // placeholder of a split that did not fit
            if (DENS)
                for (int i = tid; i < kGroupMax * 32; i += C::NT) (&S.qacc[0][0])[i] = 0.0f;
            // ---- queries (warp 0), FP32 only: RN(2h * 2h) is the float
            // rounding of the exact binary64 (2h)^2.
            if (tid < 32) {
                const int2 grp0 = G[g];
                const int2 grp = make_int2(grp0.x, group_count(grp0.y));
                const bool v = lane < grp.y;
                float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
                float h = 0.0f;
                if (v) {
                    r = T.spos[grp.x + lane];
                    h = T.sh[grp.x + lane];
                }
                const float two_h = 2.0f * h;
                const float r32 = __fmul_rn(two_h, two_h);
                float rlo = -1.0f, rhi = __int_as_float(0x7f800000);
                if (r32 >= 0x1p-100f && r32 <= 0x1p100f) {
                    rlo = __fmul_rd(r32, 1.0f - 0x1p-18f);
                    rhi = __fmul_ru(r32, 1.0f + 0x1p-18f);
                }
                const float rs = __fmul_ru(two_h, 1.0f + 0x1p-20f);
                if (v) {
                    S.q[lane] = make_float4(r.x, r.y, r.z, rlo);
                    S.qrhi[lane] = rhi;
                    S.qh[lane] = h;
                    S.qorig[lane] = __float_as_int(r.w);
                    S.qcnt[lane] = 0;
                }
                const float big = FLT_MAX;
                float pl0 = v ? r.x : big, pl1 = v ? r.y : big, pl2 = v ? r.z : big;
                float ph0 = v ? r.x : -big, ph1 = v ? r.y : -big, ph2 = v ? r.z : -big;
                float ql0 = v ? __fsub_rd(r.x, rs) : big, ql1 = v ? __fsub_rd(r.y, rs) : big;
                float ql2 = v ? __fsub_rd(r.z, rs) : big;
                float qh0 = v ? __fadd_ru(r.x, rs) : -big, qh1 = v ? __fadd_ru(r.y, rs) : -big;
                float qh2 = v ? __fadd_ru(r.z, rs) : -big;
                float rsm = v ? rs : 0.0f;
                pl0 = warp_min(pl0); pl1 = warp_min(pl1); pl2 = warp_min(pl2);
                ph0 = warp_max(ph0); ph1 = warp_max(ph1); ph2 = warp_max(ph2);
                ql0 = warp_min(ql0); ql1 = warp_min(ql1); ql2 = warp_min(ql2);
                qh0 = warp_max(qh0); qh1 = warp_max(qh1); qh2 = warp_max(qh2);
                rsm = warp_max(rsm);
                if (lane == 0) {
                    S.box[0] = pl0; S.box[1] = pl1; S.box[2] = pl2;
                    S.box[3] = ph0; S.box[4] = ph1; S.box[5] = ph2;
                    S.box[6] = ql0; S.box[7] = ql1; S.box[8] = ql2;
                    S.box[9] = qh0; S.box[10] = qh1; S.box[11] = qh2;
                    S.box[12] = __fmul_ru(__fmul_ru(rsm, rsm), 1.0f + 0x1p-19f);
                    S.gstart = grp.x;
                    S.gcount = grp.y;
                    const int gs = group_set(grp0.y);
                    S.gset = gs;
                    S.set_lo = T.set_start[gs];
                    S.set_hi = T.set_start[gs + 1];
                }
            }
            __syncthreads();
            group_walk(T, S);

            // ---- scan mode when re-streaming the candidates per window would
            // cost more than one pass over the whole set (C^2 / C::CAP > 3/4 n)
            const long long ctot = S.ctot;
            const long long nset = S.set_hi - S.set_lo;
            const bool scan = ctot > 2 * C::CAP && 3 * nset * C::CAP < 4 * ctot * ctot;
            // A unit whose candidates need scan mode or many windows is split:
            // its queries become work units of one query each in the free
            // part of the groups array, searched by the split pass on many
            // blocks at once (same lists and densities; one block would
            // otherwise hold the whole tail of the launch).
            if ((scan || ctot > 8 * C::CAP) && A.list != 2 && S.gcount > 1) {
                if (tid == 0) S.split = split_unit(T, S.gstart, S.gcount, S.gset);
                __syncthreads();
                if (S.split) continue;
            }
            if (scan && tid == 0) atomicOr(&T.ctr->status, kStWalk);
            if (scan) group_scan<DENS>(A, S);

            // ---- windows over original index (within the set)
            int wlo = S.set_lo;
            const int wend = scan ? wlo : S.set_hi;
            for (; wlo < wend;) {
                int whi = INT_MAX;
                if (tid == 0) {
                    S.ncand = 0;
                    S.kmin = INT_MAX;
                    S.kmax = INT_MIN;
                }
                __syncthreads();
                group_gather<DENS>(A, S, 0, wlo, whi, 1);
                __syncthreads();
                const bool fits = S.ncand <= C::CAP && (S.ncand == 0 || S.kmax - S.kmin < kSpanMax);
                if (!fits) {
                    // choose the largest window [wlo, whi) that fits, by histograms
                    long long span = (long long)wend - wlo;
                    if (tid == 0) atomicOr(&T.ctr->status, kStWalk);
                    for (;;) {
                        const int Wd = (int)((span + 255) / 256);
                        for (int i = tid; i < 256; i += C::NT) S.hist[i] = 0;
                        __syncthreads();
                        group_gather<DENS>(A, S, 1, wlo, (int)min((long long)INT_MAX, wlo + span), Wd);
                        __syncthreads();
                        if (tid == 0) {
                            long long cum = 0;
                            int k = 0;
                            while (k < 256 && (long long)k * Wd < span && cum + S.hist[k] <= C::CAP &&
                                   (long long)(k + 1) * Wd <= kSpanMax) {
                                cum += S.hist[k];
                                k++;
                            }
                            S.whi = k > 0 ? (int)min((long long)wlo + (long long)k * Wd, (long long)wlo + span)
                                          : -1;
                        }
                        __syncthreads();
                        if (S.whi >= 0) break;
                        span = Wd;
                        __syncthreads();
                    }
                    whi = S.whi;
                    if (tid == 0) {
                        S.ncand = 0;
                        S.kmin = INT_MAX;
                        S.kmax = INT_MIN;
                    }
                    __syncthreads();
                    group_gather<DENS>(A, S, 0, wlo, whi, 1);
                    __syncthreads();
                }
                group_window<DENS>(A, S, false);
                if (whi == INT_MAX || whi >= wend) break;
                wlo = whi;
            }

            // ---- results
            if (tid < S.gcount) {
                const int c = S.qcnt[tid];
                A.counts[S.qorig[tid]] = c;
                if (!A.count_only && !A.row_off && c > A.ngmax) atomicOr(&T.ctr->status, kStNgmax);
            }
            if (DENS) {
                for (int p = warp; p < S.gcount; p += C::WARPS) {
                    float a = S.qacc[p][lane];
                    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(~0u, a, o);
                    if (lane == 0) {
                        const float hh = S.qh[p];
                        const float mp = A.smass[S.gstart + p];
                        A.rho[S.qorig[p]] = (mp + a) / (kPiF * hh * hh * hh);
                    }
                }
            }
        }
    }
}

__global__ void k_mass_to_tree(const float4 *__restrict__ spos, const float *__restrict__ m,
                               float *__restrict__ smass, int n)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        smass[t] = m[__float_as_int(spos[t].w)];
}

size_t find_smem_bytes() { return sizeof(FindSmem<CfgWide>); }

// resident blocks per SM of k_find<CfgWide/CfgCompact, false/true>
static int g_find_per_sm[2][2] = {{1, 1}, {1, 1}};

template <class C, bool DENS>
static cudaError_t find_attr(int *per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(k_find<C, DENS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(FindSmem<C>));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_find<C, DENS>, C::NT, sizeof(FindSmem<C>));
    if (*per_sm < 1) *per_sm = 1;
    return e;
}

cudaError_t find_init_attributes()
{
    cudaError_t e = find_attr<CfgWide, false>(&g_find_per_sm[0][0]);
    if (e == cudaSuccess) e = find_attr<CfgWide, true>(&g_find_per_sm[0][1]);
    if (e == cudaSuccess) e = find_attr<CfgCompact, false>(&g_find_per_sm[1][0]);
    if (e == cudaSuccess) e = find_attr<CfgCompact, true>(&g_find_per_sm[1][1]);
    return e;
}

template <class C>
static void launch_find_list(const FindArgs &A, int list, int ngroups, int sms, cudaStream_t st)
{
    FindArgs B = A;
    B.list = list;
    B.ngroups = ngroups;
    if (ngroups == 0) return;
    const bool dens = A.rho != nullptr;
    long long blocks = (long long)sms * g_find_per_sm[list == 1 ? 1 : 0][dens ? 1 : 0];
    if (ngroups > 0) {
        const long long nchunks = (ngroups + kFindChunk - 1) / kFindChunk;
        if (blocks > nchunks) blocks = nchunks;
    }
    note_launch();
    if (dens)
        k_find<C, true><<<(int)blocks, C::NT, sizeof(FindSmem<C>), st>>>(B);
    else
        k_find<C, false><<<(int)blocks, C::NT, sizeof(FindSmem<C>), st>>>(B);
}

cudaError_t launch_find_rows(FindArgs A, const TreeDev &T, int ngroups, int ngroups_c, const float *m,
                             int sms, cudaStream_t st);

// ngroups / ngroups_c: work units of the wide / compact lists, or -1 to read
// both counts on the device (graph form: both kernels are launched).
cudaError_t launch_find(const TreeDev &T, int ngroups, int ngroups_c, int ngmax, int32_t *nbrs,
                        int32_t *counts, const float *m, float *smass, float *rho, int sms,
                        cudaStream_t st)
{
    FindArgs A;
    A.T = T;
    A.ngmax = ngmax;
    A.nbrs = nbrs;
    A.counts = counts;
    A.smass = smass;
    A.rho = rho;
    A.ngroups = 0;
    A.list = 0;
    A.row_off = nullptr;
    A.count_only = 0;
    A.half = 0;
    return launch_find_rows(A, T, ngroups, ngroups_c, m, sms, st);
}

cudaError_t launch_find_rows(FindArgs A, const TreeDev &T, int ngroups, int ngroups_c, const float *m,
                             int sms, cudaStream_t st)
{
    // the masses in tree order are written here, then read by k_find
    float *smass = const_cast<float *>(A.smass);
    float *rho = A.rho;
    if (ngroups == 0 && ngroups_c == 0) return cudaSuccess;
    if (rho) {
        int nb = (T.n + 255) / 256;
        if (nb > sms * 8) nb = sms * 8;
        if (nb < 1) nb = 1;
        note_launch();
        k_mass_to_tree<<<nb, 256, 0, st>>>(T.spos, m, smass, T.n);
    }
    cudaMemsetAsync(&T.ctr->nsplit, 0, sizeof(int), st);
    launch_find_list<CfgWide>(A, 0, ngroups, sms, st);
    launch_find_list<CfgCompact>(A, 1, ngroups_c, sms, st);
    launch_find_list<CfgWide>(A, 2, -1, sms, st);  // the units split above (count on the device)
    return cudaGetLastError();
}

// ---------------------------------------------------------------- compressed rows
constexpr int kScan64Tile = 2048;

// Exclusive scan of int32 counts [n] into int64 offsets [n + 1] (three
// passes: tile sums, one block over the tile sums, per-tile apply).
// cap: each count is taken as min(count, cap).
__global__ void __launch_bounds__(256) k_scan64_tiles(const int32_t *in, long long n, int cap,
                                                      long long *tsum)
{
    __shared__ long long ws[8];
    const long long t0 = (long long)blockIdx.x * kScan64Tile;
    long long s = 0;
    for (long long i = t0 + threadIdx.x; i < min(t0 + kScan64Tile, n); i += blockDim.x) s += min(in[i], cap);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(~0u, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k = 0; k < 8; k++) t += ws[k];
        tsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_scan64_sums(long long *tsum, int ntiles, long long *total)
{
    __shared__ long long sh[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += 1024) {
        const int i = base + threadIdx.x;
        const long long v = i < ntiles ? tsum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const long long a = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += a;
            __syncthreads();
        }
        if (i < ntiles) tsum[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(256) k_scan64_apply(const int32_t *in, long long n, int cap,
                                                      const long long *toff, long long *out)
{
    // 256 threads x 8 items
    __shared__ long long ws[8];
    const long long t0 = (long long)blockIdx.x * kScan64Tile;
    long long v[8];
    long long s = 0;
    for (int k = 0; k < 8; k++) {
        const long long i = t0 + threadIdx.x * 8 + k;
        v[k] = i < n ? min(in[i], cap) : 0;
        s += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const long long a = __shfl_up_sync(~0u, incl, o);
        if (lane >= o) incl += a;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    long long woff = 0;
    for (int k = 0; k < wid; k++) woff += ws[k];
    long long run = toff[blockIdx.x] + woff + incl - s;
    for (int k = 0; k < 8; k++) {
        const long long i = t0 + threadIdx.x * 8 + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
}

__global__ void k_copy_total(const long long *total, long long *dst) { *dst = *total; }

long long csr_scratch_elems(long long n) { return (n + kScan64Tile - 1) / kScan64Tile + 2; }

void launch_scan64(const int32_t *counts, long long n, int cap, long long *offsets, long long *scratch,
                   cudaStream_t st);

cudaError_t launch_find_csr_count(const TreeDev &T, int ngroups, int ngroups_c, int32_t *counts,
                                  const float *m, float *smass, float *rho, long long *offsets,
                                  long long *scratch, int half, int sms, cudaStream_t st)
{
    FindArgs A;
    A.half = half;
    A.T = T;
    A.ngmax = 0;
    A.nbrs = nullptr;
    A.counts = counts;
    A.smass = smass;
    A.rho = rho;
    A.ngroups = 0;
    A.list = 0;
    A.row_off = nullptr;
    A.count_only = 1;
    cudaError_t e = launch_find_rows(A, T, ngroups, ngroups_c, m, sms, st);
    if (e != cudaSuccess) return e;
    launch_scan64(counts, T.n, INT_MAX, offsets, scratch, st);
    return cudaGetLastError();
}

void launch_scan64(const int32_t *counts, long long n, int cap, long long *offsets, long long *scratch,
                   cudaStream_t st)
{
    const int ntiles = (int)((n + kScan64Tile - 1) / kScan64Tile);
    long long *total = scratch + ntiles;
    if (ntiles > 0) {
        note_launch(3);
        k_scan64_tiles<<<ntiles, 256, 0, st>>>(counts, n, cap, scratch);
        k_scan64_sums<<<1, 1024, 0, st>>>(scratch, ntiles, total);
        k_scan64_apply<<<ntiles, 256, 0, st>>>(counts, n, cap, scratch, offsets);
    } else {
        cudaMemsetAsync(total, 0, sizeof(long long), st);
    }
    note_launch();
    k_copy_total<<<1, 1, 0, st>>>(total, offsets + n);
}

// Pack fixed rows into compressed rows: row i's first min(counts[i], ngmax)
// entries go to csr[offsets[i] ..].  One warp per row, coalesced.
__global__ void __launch_bounds__(256) k_pack_rows(const int32_t *__restrict__ rows,
                                                   const int32_t *__restrict__ counts, long long n,
                                                   int ngmax, const long long *__restrict__ offsets,
                                                   int32_t *__restrict__ csr)
{
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const int c = min(counts[i], ngmax);
        const int32_t *src = rows + i * ngmax;
        int32_t *dst = csr + offsets[i];
        for (int k = lane; k < c; k += 32) dst[k] = src[k];
    }
}

void launch_pack_rows(const int32_t *rows, const int32_t *counts, long long n, int ngmax,
                      const long long *offsets, int32_t *csr, int sms, cudaStream_t st)
{
    long long blocks = (n + 7) / 8;
    if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
    if (blocks < 1) blocks = 1;
    note_launch();
    k_pack_rows<<<(int)blocks, 256, 0, st>>>(rows, counts, n, ngmax, offsets, csr);
}

cudaError_t launch_find_csr_rows(const TreeDev &T, int ngroups, int ngroups_c, const long long *offsets,
                                 int32_t *nbrs, int32_t *counts, int half, int sms, cudaStream_t st)
{
    FindArgs A;
    A.half = half;
    A.T = T;
    A.ngmax = 0;
    A.nbrs = nbrs;
    A.counts = counts;
    A.smass = nullptr;
    A.rho = nullptr;
    A.ngroups = 0;
    A.list = 0;
    A.row_off = offsets;
    A.count_only = 0;
    return launch_find_rows(A, T, ngroups, ngroups_c, nullptr, sms, st);
}

// ---------------------------------------------------------------- no-alloc form
// Some callers cannot allocate device memory at the point where they search
// (an allocator-free real-time loop, a host framework that owns all memory
// and forbids allocation after set-up).  For them the fused search keeps its
// scratch -- the masses permuted to tree order -- in this file-scope array
// instead of a buffer allocated on first use.  Every GPU that loads the
// library holds it (8 MB) until the process exits.
constexpr long long kNoAllocMaxN = 1LL << 21;
static __device__ __align__(256) float g_noalloc_smass[kNoAllocMaxN];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

long long noalloc_max_particles() { return kNoAllocMaxN; }

// Device address of the static scratch array on the current device, looked
// up once per device (a host-side name of a __device__ array is not a device
// address).  The first call on a device does the look-up.
static cudaError_t noalloc_scratch(float **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        float *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_smass);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

cudaError_t launch_find_density_noalloc(const TreeDev &T, int ngroups, int ngroups_c, int ngmax,
                                        int32_t *nbrs, int32_t *counts, const float *m, float *rho,
                                        int sms, cudaStream_t st)
{
    if ((long long)T.n > kNoAllocMaxN) return cudaErrorInvalidValue;
    float *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return e;
    // k_mass_to_tree overwrites scratch[0, n) before k_find reads it, so
    // nothing left by an earlier call needs clearing.
    return launch_find(T, ngroups, ngroups_c, ngmax, nbrs, counts, m, scratch, rho, sms, st);
}

// ---------------------------------------------------------------- density
// Consumer form: rho from existing rows (first min(count, ngmax) entries).
__global__ void __launch_bounds__(256) k_density(TreeDev T, const float *__restrict__ m,
                                                 const int32_t *__restrict__ nbrs,
                                                 const int32_t *__restrict__ counts, int ngmax,
                                                 float *__restrict__ rho)
{
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < T.n; i += nw) {
        const int ti = T.inv[i];
        const float4 P = T.spos[ti];
        const float h = T.sh[ti];
        const float inv_h = __frcp_rn(h);
        const int c = min(counts[i], ngmax);
        const int32_t *row = nbrs + (long long)i * ngmax;
        const int off = T.set_start[T.nsets == 1 ? 0 : find_set(T.set_start, T.nsets, i)];
        float acc = 0.0f;
        for (int k = lane; k < c; k += 32) {
            const int j = off + row[k];
            const float4 Q = T.spos[T.inv[j]];
            const float dx = Q.x - P.x, dy = Q.y - P.y, dz = Q.z - P.z;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float q = d2 > 0.0f ? d2 * rsqrtf(d2) * inv_h : 0.0f;
            acc = fmaf(m[j], m4_shape(q), acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(~0u, acc, o);
        if (lane == 0) rho[i] = (m[i] + acc) / (kPiF * h * h * h);
    }
}

cudaError_t launch_density(const TreeDev &T, const float *m, const int32_t *nbrs,
                           const int32_t *counts, int ngmax, float *rho, int sms, cudaStream_t st)
{
    if (T.n <= 0) return cudaSuccess;
    long long blocks = ((long long)T.n + 7) / 8;
    if (blocks > sms * 16) blocks = sms * 16;
    note_launch();
    k_density<<<(int)blocks, 256, 0, st>>>(T, m, nbrs, counts, ngmax, rho);
    return cudaGetLastError();
}

}  // namespace bt
