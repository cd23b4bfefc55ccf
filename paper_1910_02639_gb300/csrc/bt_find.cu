// bt_find.cu -- FindNeighbors (Algorithm 2 of arXiv:1910.02639) on the GPU,
// optionally fused with the SPH density sum (M4 cubic spline).
//
// Work unit: a group of <= 32 particles that are contiguous in tree order (a
// leaf, a small cell, or a 32-slice of an oversized leaf), one 128-thread
// block at a time.  Per group:
//   1. warp 0 loads the queries and walks the tree once for the union of
//      their search intervals (Eqs. 5-6 on the group's query box), collecting
//      contiguous particle ranges (whole x-runs of sub-cells, Eq. 3 order);
//   2. all warps stream the candidates of those ranges (coalesced float4
//      loads) and keep those within 2*h_max of the group's bounding box;
//   3. the kept candidates are sorted by original index (bitonic, registers);
//   4. each candidate chunk of 32 is tested against every query with an FP32
//      filter whose error band is certified; the rare pairs inside the band
//      are decided by the binary64 definition; one ballot per (query, chunk);
//   5. per query, the ballots are turned into the ascending, capped row with
//      a warp prefix sum (and the density sum is accumulated in that order).
// Groups whose candidate set is larger than the buffer, or spans too many
// original indices for 32-bit sort keys, are processed in windows of
// original index (same results, more passes).
#include "bt_internal.cuh"
#include "bt_sort.cuh"
#include "bt_find.cuh"

#include <cfloat>

namespace bt {

constexpr int kCap = 1024;                 // candidates per window
constexpr int kSlotBits = 10;              // log2(kCap)
constexpr int kSpanMax = (1 << 22) - 1;    // original-index span of one window
constexpr int kChunks = kCap / 32;
constexpr int kRangeMax = 256;
constexpr int kStackMax = 128;
constexpr int kDescendMin = 32;            // smaller internal sub-cells are scanned whole
constexpr int kFindChunk = 4;              // consecutive groups per block step
constexpr float kPiF = 3.14159265358979f;

struct FindSmem {
    float4 cand[kCap];
    float cmass[kCap];
    uint32_t key[kCap];
    uint32_t mask[kGroupMax * kChunks];
    unsigned short rank_of[kCap];
    float4 q[kGroupMax];      // x, y, z, R_lo
    float qrhi[kGroupMax];
    float qh[kGroupMax];
    int qorig[kGroupMax];
    int qself[kGroupMax];
    int qcnt[kGroupMax];
    float qacc[kGroupMax];
    int2 ranges[kRangeMax];
    int stack[kStackMax];
    int hist[256];
    float box[13];            // PL[3] PH[3] QL[3] QH[3] T
    int nrange, nstack, ncand, kmin, kmax, range_ovf, ovf_lo, ovf_hi;
    int gstart, gcount, wlo, whi, mode_w;
};

struct FindArgs {
    TreeDev T;
    int ngmax;
    int32_t *nbrs;
    int32_t *counts;
    const float *smass;  // masses in tree order (density only)
    float *rho;
    int ngroups;
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

__device__ __forceinline__ void add_range(FindSmem &S, int s, int len)
{
    if (len <= 0) return;
    int r = atomicAdd(&S.nrange, 1);
    if (r < kRangeMax - 1) {
        S.ranges[r] = make_int2(s, len);
    } else {
        atomicMin(&S.ovf_lo, s);
        atomicMax(&S.ovf_hi, s + len);
        S.range_ovf = 1;
    }
}

// Warp 0: the tree walk for the group's query box.
__device__ void group_walk(const TreeDev &T, FindSmem &S, int lane)
{
    if (lane == 0) {
        S.nrange = 0;
        S.nstack = 0;
        S.range_ovf = 0;
        S.ovf_lo = INT_MAX;
        S.ovf_hi = INT_MIN;
    }
    __syncwarp();
    const float QL0 = S.box[6], QL1 = S.box[7], QL2 = S.box[8];
    const float QH0 = S.box[9], QH1 = S.box[10], QH2 = S.box[11];
    if (lane == 0) {
        S.stack[0] = 0;
        S.nstack = 1;
    }
    __syncwarp();
    while (S.nstack > 0) {
        const int nid = S.stack[S.nstack - 1];
        __syncwarp();
        if (lane == 0) S.nstack--;
        const NodeWalk W = T.walk[nid];
        __syncwarp();
        if (W.b == 0) {
            if (lane == 0) add_range(S, W.start, W.count);
            __syncwarp();
            continue;
        }
        int rx0, rx1, ry0, ry1, rz0, rz1;
        walk_range(QL0, QH0, W, 0, rx0, rx1);
        walk_range(QL1, QH1, W, 1, ry0, ry1);
        walk_range(QL2, QH2, W, 2, rz0, rz1);
        if (rx1 < rx0 || ry1 < ry0 || rz1 < rz0) continue;
        const int ny = ry1 - ry0 + 1;
        const int nyz = ny * (rz1 - rz0 + 1);
        for (int idx = lane; idx < nyz; idx += 32) {
            const int cy = ry0 + idx % ny;
            const int cz = rz0 + idx / ny;
            const int row = W.slot0 + W.b * (cy + W.b * cz);
            int cs = 0, cl = 0;
            for (int cx = rx0; cx <= rx1; cx++) {
                const Slot sl = T.slots[row + cx];
                if (sl.child >= 0 && sl.count > kDescendMin) {
                    add_range(S, cs, cl);
                    cl = 0;
                    int k = atomicAdd(&S.nstack, 1);
                    if (k < kStackMax) {
                        S.stack[k] = sl.child;
                    } else {
                        atomicSub(&S.nstack, 1);
                        add_range(S, sl.start, sl.count);
                    }
                } else if (sl.count > 0) {
                    if (cl == 0) cs = sl.start;
                    cl = sl.start + sl.count - cs;
                }
            }
            add_range(S, cs, cl);
        }
        __syncwarp();
    }
    __syncwarp();
    if (S.range_ovf) {
        // Too many ranges: replace the list by the one range that covers them
        // all (a superset, and no particle appears twice).
        int lo = S.ovf_lo, hi = S.ovf_hi;
        for (int r = lane; r < kRangeMax - 1; r += 32) {
            const int2 rg = S.ranges[r];
            lo = min(lo, rg.x);
            hi = max(hi, rg.x + rg.y);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(~0u, lo, o));
            hi = max(hi, __shfl_xor_sync(~0u, hi, o));
        }
        __syncwarp();
        if (lane == 0) {
            S.ranges[0] = make_int2(lo, hi - lo);
            S.nrange = 1;
            atomicOr(&T.ctr->status, kStWalk);
        }
    }
    __syncwarp();
}

// Stream the candidates of the collected ranges.  mode 0: collect those with
// original index in [wlo, whi) into the buffer; mode 1: histogram them into
// 256 bins of width W starting at wlo.
template <bool DENS>
__device__ void group_gather(const FindArgs &A, FindSmem &S, int mode, int wlo, int whi, int W)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float PL0 = S.box[0], PL1 = S.box[1], PL2 = S.box[2];
    const float PH0 = S.box[3], PH1 = S.box[4], PH2 = S.box[5];
    const float T2 = S.box[12];
    const int gstart = S.gstart, gcount = S.gcount;
    int kmin = INT_MAX, kmax = INT_MIN;
    const int nr = S.nrange;
    for (int r = warp; r < nr; r += 4) {
        const int2 rg = S.ranges[r];
        for (int off = 0; off < rg.y; off += 32) {
            const int t = rg.x + off + lane;
            bool keep = false;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            int orig = 0;
            if (off + lane < rg.y) {
                c = __ldg(&A.T.spos[t]);
                orig = __float_as_int(c.w);
                float ex = fmaxf(fmaxf(__fsub_rn(PL0, c.x), __fsub_rn(c.x, PH0)), 0.0f);
                float ey = fmaxf(fmaxf(__fsub_rn(PL1, c.y), __fsub_rn(c.y, PH1)), 0.0f);
                float ez = fmaxf(fmaxf(__fsub_rn(PL2, c.z), __fsub_rn(c.z, PH2)), 0.0f);
                float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                keep = d2 <= T2 && orig >= wlo && orig < whi;
            }
            if (mode == 0) {
                const unsigned bal = __ballot_sync(~0u, keep);
                if (bal == 0) continue;
                int base = 0;
                if (lane == 0) base = atomicAdd(&S.ncand, __popc(bal));
                base = __shfl_sync(~0u, base, 0);
                if (keep) {
                    const int slot = base + __popc(bal & ((1u << lane) - 1));
                    if (slot < kCap) {
                        S.cand[slot] = c;
                        if (DENS) S.cmass[slot] = __ldg(&A.smass[t]);
                        if (t >= gstart && t < gstart + gcount) S.qself[t - gstart] = slot;
                    }
                    kmin = min(kmin, orig);
                    kmax = max(kmax, orig);
                }
            } else if (keep) {
                atomicAdd(&S.hist[(int)((unsigned)(orig - wlo) / (unsigned)W)], 1);
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
    if (q < 1.0f) return fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f);
    if (q < 2.0f) {
        float t = 2.0f - q;
        return 0.25f * t * t * t;
    }
    return 0.0f;
}

// Sort, test and emit the candidates of the current window.
template <bool DENS>
__device__ void group_window(const FindArgs &A, FindSmem &S)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = S.ncand;  // <= kCap here
    const int gcount = S.gcount;
    if (m == 0) return;
    const int kmin = S.kmin;
    int npad = 128;
    while (npad < m) npad <<= 1;
    for (int s = tid; s < npad; s += 128) {
        uint32_t k = 0xffffffffu;
        if (s < m) k = ((uint32_t)(__float_as_int(S.cand[s].w) - kmin) << kSlotBits) | (uint32_t)s;
        S.key[s] = k;
    }
    __syncthreads();
    block_sort_n(S.key, npad);
    for (int k = tid; k < m; k += 128) S.rank_of[S.key[k] & (kCap - 1)] = (unsigned short)k;
    __syncthreads();

    // ---- stage A: one ballot per (query, chunk)
    const int nch = (m + 31) >> 5;
    for (int c = warp; c < nch; c += 4) {
        const int k = c * 32 + lane;
        const bool valid = k < m;
        float4 Q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) Q = S.cand[S.key[k] & (kCap - 1)];
        bool amb = false;
        for (int p = 0; p < gcount; p++) {
            const float4 P = S.q[p];
            const float rhi = S.qrhi[p];
            const float dx = Q.x - P.x, dy = Q.y - P.y, dz = Q.z - P.z;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const bool hit = valid && d2 < P.w;
            amb |= valid && !hit && d2 <= rhi;
            const unsigned bal = __ballot_sync(~0u, hit);
            if (lane == 0) S.mask[p * kChunks + c] = bal;
        }
        __syncwarp();
        if (__any_sync(~0u, amb)) {
            if (amb) {
                for (int p = 0; p < gcount; p++) {
                    const float4 P = S.q[p];
                    const float rhi = S.qrhi[p];
                    const float dx = Q.x - P.x, dy = Q.y - P.y, dz = Q.z - P.z;
                    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    if (!(d2 < P.w) && d2 <= rhi && exact_neighbor(P, S.qh[p], Q))
                        atomicOr(&S.mask[p * kChunks + c], 1u << lane);
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();

    // ---- stage B: ascending rows by prefix sums of the ballots
    for (int p = warp; p < gcount; p += 4) {
        uint32_t mk = lane < nch ? S.mask[p * kChunks + lane] : 0u;
        const int self = S.qself[p];
        if (self >= 0) {
            const int sr = S.rank_of[self];
            if (lane == (sr >> 5)) mk &= ~(1u << (sr & 31));
        }
        const int cnt = __popc(mk);
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(~0u, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(~0u, incl, 31);
        int pos = S.qcnt[p] + incl - cnt;
        int32_t *row = A.nbrs + (long long)S.qorig[p] * A.ngmax;
        const float4 P = S.q[p];
        const float inv_h = 1.0f / S.qh[p];
        float acc = 0.0f;
        while (mk) {
            const int bit = __ffs(mk) - 1;
            mk &= mk - 1;
            const uint32_t key = S.key[lane * 32 + bit];
            if (pos < A.ngmax) row[pos] = kmin + (int)(key >> kSlotBits);
            pos++;
            if (DENS) {
                const int slot = key & (kCap - 1);
                const float4 Q = S.cand[slot];
                const float dx = Q.x - P.x, dy = Q.y - P.y, dz = Q.z - P.z;
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                acc = fmaf(S.cmass[slot], m4_shape(sqrtf(d2) * inv_h), acc);
            }
        }
        if (DENS) {
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(~0u, acc, o);
        }
        if (lane == 0) {
            S.qcnt[p] += total;
            if (DENS) S.qacc[p] += acc;
        }
    }
    __syncthreads();
}

template <bool DENS>
__global__ void __launch_bounds__(128) k_find(FindArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FindSmem &S = *reinterpret_cast<FindSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    const TreeDev &T = A.T;
    const int nchunks = (A.ngroups + kFindChunk - 1) / kFindChunk;

    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const int g1 = min(chunk * kFindChunk + kFindChunk, A.ngroups);
        for (int g = chunk * kFindChunk; g < g1; g++) {
            __syncthreads();
            const int2 grp = T.groups[g];
            // ---- queries (warp 0)
            if (tid < 32) {
                const bool v = lane < grp.y;
                float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
                float h = 0.0f;
                if (v) {
                    r = T.spos[grp.x + lane];
                    h = T.sh[grp.x + lane];
                }
                const double two_h = __dmul_rn(2.0, (double)h);
                const double R64 = __dmul_rn(two_h, two_h);
                float rlo = -1.0f, rhi = FLT_MAX;
                if (R64 >= 0x1p-100 && R64 <= 0x1p100) {
                    const float r32 = __double2float_rn(R64);
                    rlo = __fmul_rd(r32, 1.0f - 0x1p-18f);
                    rhi = __fmul_ru(r32, 1.0f + 0x1p-18f);
                }
                const float rs = __fmul_ru(__fmul_ru(h, 2.0f), 1.0f + 0x1p-20f);
                if (v) {
                    S.q[lane] = make_float4(r.x, r.y, r.z, rlo);
                    S.qrhi[lane] = rhi;
                    S.qh[lane] = h;
                    S.qorig[lane] = __float_as_int(r.w);
                    S.qcnt[lane] = 0;
                    S.qacc[lane] = 0.0f;
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
                }
                __syncwarp();
                group_walk(T, S, lane);
            }
            __syncthreads();

            // ---- windows over original index
            int wlo = 0;
            for (;;) {
                int whi = INT_MAX;
                if (tid == 0) {
                    S.ncand = 0;
                    S.kmin = INT_MAX;
                    S.kmax = INT_MIN;
                }
                if (tid < kGroupMax) S.qself[tid] = -1;
                __syncthreads();
                group_gather<DENS>(A, S, 0, wlo, whi, 1);
                __syncthreads();
                const bool fits = S.ncand <= kCap && (S.ncand == 0 || S.kmax - S.kmin < kSpanMax);
                if (!fits) {
                    // choose the largest window [wlo, whi) that fits, by histograms
                    long long span = (long long)T.n - wlo;
                    if (tid == 0) atomicOr(&T.ctr->status, kStWalk);
                    for (;;) {
                        const int Wd = (int)((span + 255) / 256);
                        for (int i = tid; i < 256; i += 128) S.hist[i] = 0;
                        __syncthreads();
                        group_gather<DENS>(A, S, 1, wlo, (int)min((long long)INT_MAX, wlo + span), Wd);
                        __syncthreads();
                        if (tid == 0) {
                            long long cum = 0;
                            int k = 0;
                            while (k < 256 && (long long)k * Wd < span && cum + S.hist[k] <= kCap &&
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
                    if (tid < kGroupMax) S.qself[tid] = -1;
                    __syncthreads();
                    group_gather<DENS>(A, S, 0, wlo, whi, 1);
                    __syncthreads();
                }
                group_window<DENS>(A, S);
                if (whi == INT_MAX || whi >= T.n) break;
                wlo = whi;
            }

            // ---- results
            if (tid < S.gcount) {
                const int c = S.qcnt[tid];
                const int o = S.qorig[tid];
                A.counts[o] = c;
                if (c > A.ngmax) atomicOr(&T.ctr->status, kStNgmax);
                if (DENS) {
                    const float h = S.qh[tid];
                    const float mp = A.smass[S.gstart + tid];
                    A.rho[o] = (mp + S.qacc[tid]) / (kPiF * h * h * h);
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

size_t find_smem_bytes() { return sizeof(FindSmem); }

cudaError_t find_init_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_find<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(FindSmem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_find<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(FindSmem));
}

cudaError_t launch_find(const TreeDev &T, int ngroups, int ngmax, int32_t *nbrs, int32_t *counts,
                        const float *m, float *smass, float *rho, int sms, cudaStream_t st)
{
    FindArgs A;
    A.T = T;
    A.ngmax = ngmax;
    A.nbrs = nbrs;
    A.counts = counts;
    A.smass = smass;
    A.rho = rho;
    A.ngroups = ngroups;
    if (ngroups <= 0) return cudaSuccess;
    int per_sm = 0;
    const bool dens = rho != nullptr;
    if (dens) {
        int nb = (T.n + 255) / 256;
        if (nb > sms * 8) nb = sms * 8;
        k_mass_to_tree<<<nb, 256, 0, st>>>(T.spos, m, smass, T.n);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_find<true>, 128, sizeof(FindSmem));
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_find<false>, 128, sizeof(FindSmem));
    }
    if (per_sm < 1) per_sm = 1;
    long long nchunks = (ngroups + kFindChunk - 1) / kFindChunk;
    long long blocks = (long long)sms * per_sm;
    if (blocks > nchunks) blocks = nchunks;
    if (dens)
        k_find<true><<<(int)blocks, 128, sizeof(FindSmem), st>>>(A);
    else
        k_find<false><<<(int)blocks, 128, sizeof(FindSmem), st>>>(A);
    return cudaGetLastError();
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
        const float inv_h = 1.0f / h;
        const int c = min(counts[i], ngmax);
        const int32_t *row = nbrs + (long long)i * ngmax;
        float acc = 0.0f;
        for (int k = lane; k < c; k += 32) {
            const int j = row[k];
            const float4 Q = T.spos[T.inv[j]];
            const float dx = Q.x - P.x, dy = Q.y - P.y, dz = Q.z - P.z;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            acc = fmaf(m[j], m4_shape(sqrtf(d2) * inv_h), acc);
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
    k_density<<<(int)blocks, 256, 0, st>>>(T, m, nbrs, counts, ngmax, rho);
    return cudaGetLastError();
}

}  // namespace bt
