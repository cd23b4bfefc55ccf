// bt_api.cu -- the C ABI (include/btree.h): tree handle, buffers, and the
// host side of BuildTree (level loop over cells with > kSmallCap particles).
#include "bt_build.cuh"
#include "bt_find.cuh"
#include "bt_internal.cuh"

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

using namespace bt;

namespace bt {
static std::atomic<uint64_t> g_launches{0};
void note_launch(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }
}  // namespace bt

struct btree {
    int64_t n = 0;
    int s = 16;
    double alpha = 0.5, beta = 0.5;
    bt_allocator al{};
    bool has_al = false;
    cudaStream_t st = nullptr;
    int device = 0, sms = 1;

    int64_t cap_n = 0;
    int cap_nodes = 0, cap_slots = 0, cap_groups = 0, cap_small = 0, cap_big = 0;
    int64_t cap_hist = 0;
    int64_t cap_smass = 0;

    NodeGeom *geom = nullptr;
    NodeWalk *walk = nullptr;
    Slot *slots = nullptr;
    int2 *groups = nullptr;
    float4 *spos = nullptr;
    float *sh = nullptr;
    int *inv = nullptr;
    float4 *wpos[2] = {nullptr, nullptr};
    float *wh[2] = {nullptr, nullptr};
    int *hist = nullptr, *hoff = nullptr, *cursor = nullptr, *tiles = nullptr;
    BigCell *big = nullptr;
    int *big_ids[2] = {nullptr, nullptr};
    SmallItem *small = nullptr;
    Counters *ctr = nullptr;
    Counters *hctr = nullptr;  // pinned host mirror
    float *smass = nullptr;
    // per-set tables (device) and their pinned host staging
    int nsets = 0, cap_sets = 0;
    int *set_start = nullptr, *set_s = nullptr, *set_na = nullptr, *set_gmax = nullptr;
    int *set_flags = nullptr, *set_bbox = nullptr;
    double *set_beta = nullptr;
    SetRec *set_rec = nullptr;  // device copy of the staged records
    SetRec *h_rec = nullptr;    // [cap_sets] pinned staging

    int ngroups = 0;
    bt_info info{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;

int to_status(cudaError_t e)
{
    if (e == cudaSuccess) return BT_OK;
    if (e == cudaErrorMemoryAllocation) return BT_ERR_OOM;
    return BT_ERR_CUDA;
}

void *dev_alloc(btree *t, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (t->has_al) return t->al.alloc(t->al.ctx, bytes, t->st);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, t->st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(btree *t, void *p)
{
    if (!p) return;
    if (t->has_al) t->al.free(t->al.ctx, p, t->st);
    else cudaFreeAsync(p, t->st);
}

template <typename T>
bool realloc_dev(btree *t, T *&p, int64_t old_count, int64_t new_count, bool keep)
{
    T *q = static_cast<T *>(dev_alloc(t, sizeof(T) * (size_t)new_count));
    if (!q) return false;
    if (keep && p && old_count > 0)
        cudaMemcpyAsync(q, p, sizeof(T) * (size_t)old_count, cudaMemcpyDeviceToDevice, t->st);
    dev_free(t, p);
    p = q;
    return true;
}

void free_all(btree *t)
{
    dev_free(t, t->geom); dev_free(t, t->walk); dev_free(t, t->slots); dev_free(t, t->groups);
    dev_free(t, t->spos); dev_free(t, t->sh); dev_free(t, t->inv);
    for (int k = 0; k < 2; k++) { dev_free(t, t->wpos[k]); dev_free(t, t->wh[k]); dev_free(t, t->big_ids[k]); }
    dev_free(t, t->hist); dev_free(t, t->hoff); dev_free(t, t->cursor); dev_free(t, t->tiles);
    dev_free(t, t->big); dev_free(t, t->small); dev_free(t, t->ctr); dev_free(t, t->smass);
    dev_free(t, t->set_start); dev_free(t, t->set_s); dev_free(t, t->set_na); dev_free(t, t->set_gmax);
    dev_free(t, t->set_flags); dev_free(t, t->set_bbox); dev_free(t, t->set_beta); dev_free(t, t->set_rec);
    t->set_start = t->set_s = t->set_na = t->set_gmax = nullptr;
    t->set_flags = t->set_bbox = nullptr;
    t->set_beta = nullptr;
    t->set_rec = nullptr;
    t->cap_sets = 0;
    t->geom = nullptr; t->walk = nullptr; t->slots = nullptr; t->groups = nullptr;
    t->spos = nullptr; t->sh = nullptr; t->inv = nullptr;
    for (int k = 0; k < 2; k++) { t->wpos[k] = nullptr; t->wh[k] = nullptr; t->big_ids[k] = nullptr; }
    t->hist = t->hoff = t->cursor = t->tiles = nullptr;
    t->big = nullptr; t->small = nullptr; t->ctr = nullptr; t->smass = nullptr;
    t->cap_n = 0; t->cap_nodes = t->cap_slots = t->cap_groups = t->cap_small = t->cap_big = 0;
    t->cap_hist = 0; t->cap_smass = 0;
}

TreeDev view(const btree *t)
{
    TreeDev T;
    T.n = (int)t->n;
    T.nsets = t->nsets;
    T.set_start = t->set_start;
    T.set_s = t->set_s;
    T.set_na = t->set_na;
    T.set_beta = t->set_beta;
    T.set_gmax = t->set_gmax;
    T.set_flags = t->set_flags;
    T.set_bbox = t->set_bbox;
    T.geom = t->geom;
    T.walk = t->walk;
    T.slots = t->slots;
    T.groups = t->groups;
    T.spos = t->spos;
    T.sh = t->sh;
    T.inv = t->inv;
    T.ctr = t->ctr;
    T.cap_nodes = t->cap_nodes;
    T.cap_slots = t->cap_slots;
    T.cap_groups = t->cap_groups;
    T.cap_small = t->cap_small;
    return T;
}

// Per-particle buffers and first estimates of the tree-size capacities.
int ensure_particle_caps(btree *t, int64_t n)
{
    const int64_t nn = n > 0 ? n : 1;
    if (t->cap_n < nn) {
        int64_t c = nn;
        bool ok = realloc_dev(t, t->spos, 0, c, false) && realloc_dev(t, t->sh, 0, c, false) &&
                  realloc_dev(t, t->inv, 0, c, false) && realloc_dev(t, t->wpos[0], 0, c, false) &&
                  realloc_dev(t, t->wpos[1], 0, c, false) && realloc_dev(t, t->wh[0], 0, c, false) &&
                  realloc_dev(t, t->wh[1], 0, c, false);
        if (!ok) return BT_ERR_OOM;
        t->cap_n = c;
    }
    const int64_t s = t->s;
    const int64_t ns = std::max(t->nsets, 1);
    int64_t want_groups = nn + 1;
    int64_t want_small = nn / (s + 1) + 2 + ns;
    int64_t want_big = nn / (kSmallCap + 1) + 2;
    if (t->cap_groups < want_groups) {
        if (!realloc_dev(t, t->groups, 0, want_groups, false)) return BT_ERR_OOM;
        t->cap_groups = (int)want_groups;
    }
    if (t->cap_small < want_small) {
        if (!realloc_dev(t, t->small, 0, want_small, false)) return BT_ERR_OOM;
        t->cap_small = (int)want_small;
    }
    if (t->cap_big < want_big) {
        if (!realloc_dev(t, t->big, 0, want_big, false) ||
            !realloc_dev(t, t->big_ids[0], 0, want_big, false) ||
            !realloc_dev(t, t->big_ids[1], 0, want_big, false))
            return BT_ERR_OOM;
        t->cap_big = (int)want_big;
    }
    int64_t want_nodes = std::min<int64_t>(INT32_MAX / 2, 3 * nn / (s + 1) + 1024 + ns);
    if (t->cap_nodes < want_nodes) {
        if (!realloc_dev(t, t->geom, 0, want_nodes, false) || !realloc_dev(t, t->walk, 0, want_nodes, false))
            return BT_ERR_OOM;
        t->cap_nodes = (int)want_nodes;
    }
    int64_t want_slots = std::min<int64_t>(INT32_MAX / 2, 16 * nn / s + 4096);
    if (t->cap_slots < want_slots) {
        if (!realloc_dev(t, t->slots, 0, want_slots, false)) return BT_ERR_OOM;
        t->cap_slots = (int)want_slots;
    }
    if (!t->ctr) {
        t->ctr = static_cast<Counters *>(dev_alloc(t, sizeof(Counters)));
        if (!t->ctr) return BT_ERR_OOM;
    }
    return BT_OK;
}

int ensure_hist(btree *t, int64_t need)
{
    if (t->cap_hist >= need) return BT_OK;
    int64_t c = std::max<int64_t>(need, 4096);
    if (!realloc_dev(t, t->hist, 0, c, false) || !realloc_dev(t, t->hoff, 0, c, false) ||
        !realloc_dev(t, t->cursor, 0, c, false) ||
        !realloc_dev(t, t->tiles, 0, scan_tile_count((int)c) + 1, false))
        return BT_ERR_OOM;
    t->cap_hist = c;
    return BT_OK;
}

// Device tables and pinned staging for nsets particle sets.
int ensure_set_caps(btree *t, int nsets)
{
    if (t->cap_sets >= nsets && t->set_start) return BT_OK;
    const int c = std::max(nsets, 1);
    if (!realloc_dev(t, t->set_start, 0, c + 1, false) || !realloc_dev(t, t->set_s, 0, c, false) ||
        !realloc_dev(t, t->set_na, 0, c, false) || !realloc_dev(t, t->set_gmax, 0, c, false) ||
        !realloc_dev(t, t->set_beta, 0, c, false) || !realloc_dev(t, t->set_rec, 0, c, false) ||
        !realloc_dev(t, t->set_flags, 0, c, false) || !realloc_dev(t, t->set_bbox, 0, 6 * c, false))
        return BT_ERR_OOM;
    // the previous build has finished reading the staging (builds end synchronised)
    if (t->h_rec) cudaFreeHost(t->h_rec);
    t->h_rec = nullptr;
    if (cudaMallocHost(&t->h_rec, sizeof(SetRec) * (size_t)c) != cudaSuccess) {
        cudaGetLastError();
        return BT_ERR_OOM;
    }
    t->cap_sets = c;
    return BT_OK;
}

int read_counters(btree *t)
{
    cudaMemcpyAsync(t->hctr, t->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, t->st);
    cudaError_t e = cudaStreamSynchronize(t->st);
    if (e != cudaSuccess) return to_status(e);
    return to_status(cudaGetLastError());
}

constexpr int kRetry = 100;

int do_build(btree *t, const float *x, const float *y, const float *z, const float *h)
{
    const int ns = t->nsets;
    cudaStream_t st = t->st;
    TreeDev T = view(t);
    // per-set tables (staged on the host by the caller)
    cudaMemcpyAsync(t->set_rec, t->h_rec, sizeof(SetRec) * (size_t)ns, cudaMemcpyHostToDevice, st);
    launch_init_counters(t->ctr, st);
    launch_set_int(&t->ctr->nnodes, ns, st);  // nodes 0..ns-1 are the roots
    launch_init_sets(T, t->set_rec, t->set_start, t->set_s, t->set_na, t->set_beta, t->set_gmax, st);
    cudaEventRecord(t->ev0, st);
    launch_bbox(T, x, y, z, h, t->sms, st);
    launch_root_sets(T, t->big_ids[0], t->small, st);
    launch_copy_leaf_roots(T, x, y, z, h, t->sms, st);
    int rc = read_counters(t);
    if (rc != BT_OK) return rc;
    if (t->hctr->status & kStNonfinite) return BT_ERR_NONFINITE;
    if (t->hctr->status & kStCapSmall) return kRetry;

    {
        Src in{x, y, z, h, nullptr, nullptr};
        Src src = in;
        int nb = t->hctr->nbig_next;
        int cur = 0, dst = 0;
        int64_t nslots = 0;
        while (nb > 0) {
            launch_big_setup(T, t->big, t->big_ids[cur], nb, st);
            if ((rc = read_counters(t)) != BT_OK) return rc;
            if (t->hctr->status & kStCapBig) return BT_ERR_CAPACITY;
            const int hist_total = t->hctr->hist_total;
            const int chunks = t->hctr->chunk_total;
            if ((rc = ensure_hist(t, hist_total)) != BT_OK) return rc;
            if (nslots + hist_total > t->cap_slots) {
                int64_t c = std::max<int64_t>((int64_t)t->cap_slots * 2, nslots + hist_total + 4096);
                if (c > INT32_MAX / 2) return BT_ERR_CAPACITY;
                if (!realloc_dev(t, t->slots, nslots, c, true)) return BT_ERR_OOM;
                t->cap_slots = (int)c;
                T = view(t);
            }
            cudaMemsetAsync(t->hist, 0, sizeof(int) * (size_t)hist_total, st);
            for (int it = 0; it < 16; it++) {
                launch_set_int(&t->ctr->again, 0, st);
                launch_big_hist(T, t->big, nb, chunks, src, t->hist, t->sms, st);
                launch_big_ratio(T, t->big, nb, t->hist, hist_total, t->sms, st);
                if ((rc = read_counters(t)) != BT_OK) return rc;
                if (!t->hctr->again) break;
                launch_big_zero(t->big, nb, t->hist, hist_total, t->sms, st);
            }
            launch_big_finish(T, t->big, nb, (int)nslots, st);
            nslots += hist_total;
            launch_set_int(&t->ctr->nslots, (int)nslots, st);
            launch_scan(t->hist, hist_total, t->tiles, t->hoff, st);
            launch_set_int(&t->ctr->nbig_next, 0, st);
            launch_big_emit(T, t->big, nb, hist_total, t->hist, t->hoff, t->cursor, dst,
                            t->big_ids[cur ^ 1], t->small, t->sms, st);
            launch_big_scatter(T, t->big, nb, chunks, src, t->cursor, t->wpos[dst], t->wh[dst],
                               t->sms, st);
            if ((rc = read_counters(t)) != BT_OK) return rc;
            if (t->hctr->status & (kStCapNodes | kStCapSlots | kStCapGroups | kStCapSmall)) return kRetry;
            nb = t->hctr->nbig_next;
            if (nb > t->cap_big) return BT_ERR_CAPACITY;
            cur ^= 1;
            src = Src{nullptr, nullptr, nullptr, nullptr, t->wpos[dst], t->wh[dst]};
            dst ^= 1;
        }
        if ((rc = read_counters(t)) != BT_OK) return rc;
        const int nsmall = t->hctr->nsmall;
        Src s0{nullptr, nullptr, nullptr, nullptr, t->wpos[0], t->wh[0]};
        Src s1{nullptr, nullptr, nullptr, nullptr, t->wpos[1], t->wh[1]};
        launch_small(T, t->small, std::min(nsmall, t->cap_small), s0, s1, in, t->sms, st);
    }
    cudaEventRecord(t->ev1, st);
    if ((rc = read_counters(t)) != BT_OK) return rc;
    const Counters &c = *t->hctr;
    if (c.status & (kStCapNodes | kStCapSlots | kStCapGroups | kStCapSmall)) return kRetry;
    t->ngroups = c.ngroups;
    NodeWalk w0;
    cudaMemcpyAsync(&w0, t->walk, sizeof(NodeWalk), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return BT_ERR_CUDA;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, t->ev0, t->ev1);
    bt_info &I = t->info;
    I.n = t->n;
    I.bucket_size = t->s;
    I.max_depth = c.max_depth;
    I.num_nodes = c.nnodes;
    I.num_slots = c.nslots;
    I.num_groups = c.ngroups;
    I.root_b = w0.b;
    I.num_oversized = c.noversized;
    I.build_ms = ms;
    return (c.status & kStOversized) ? BT_WARN_OVERSIZED_LEAF : BT_OK;
}

bool is_finite_d(double v) { return std::isfinite(v); }

}  // namespace

// Shared front end of btree_build and btree_build_batched: the per-set
// records must already be staged in t->h_rec.
static int build_core(btree *t, const float *x, const float *y, const float *z, const float *h)
{
    int rc = BT_OK;
    for (int attempt = 0; attempt < 6; attempt++) {
        rc = ensure_particle_caps(t, t->n);
        if (rc != BT_OK) break;
        rc = do_build(t, x, y, z, h);
        if (rc != kRetry) break;
        // grow the tree-size buffers and build again
        int64_t cn = std::min<int64_t>((int64_t)t->cap_nodes * 2, INT32_MAX / 2);
        int64_t cs = std::min<int64_t>((int64_t)t->cap_slots * 2, INT32_MAX / 2);
        int64_t cm = std::min<int64_t>((int64_t)t->cap_small * 2 + 1024, INT32_MAX / 2);
        if (!realloc_dev(t, t->geom, 0, cn, false) || !realloc_dev(t, t->walk, 0, cn, false) ||
            !realloc_dev(t, t->slots, 0, cs, false) || !realloc_dev(t, t->small, 0, cm, false)) {
            rc = BT_ERR_OOM;
            break;
        }
        t->cap_nodes = (int)cn;
        t->cap_slots = (int)cs;
        t->cap_small = (int)cm;
        rc = BT_ERR_CAPACITY;
    }
    return rc;
}

// Creates or re-targets the handle (allocator, stream); nullptr on failure.
static btree *prepare_handle(btree_t **out, const bt_allocator *alloc, void *stream, int *rc)
{
    std::call_once(g_attr_once, [] {
        g_attr_err = build_init_attributes();
        if (g_attr_err == cudaSuccess) g_attr_err = find_init_attributes();
    });
    if (g_attr_err != cudaSuccess) {
        *rc = to_status(g_attr_err);
        return nullptr;
    }
    btree *t = *out;
    bool fresh = false;
    if (!t) {
        t = new (std::nothrow) btree();
        if (!t) {
            *rc = BT_ERR_OOM;
            return nullptr;
        }
        fresh = true;
        cudaGetDevice(&t->device);
        cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, t->device);
        if (cudaMallocHost(&t->hctr, sizeof(Counters)) != cudaSuccess ||
            cudaEventCreate(&t->ev0) != cudaSuccess || cudaEventCreate(&t->ev1) != cudaSuccess) {
            cudaGetLastError();
            delete t;
            *rc = BT_ERR_CUDA;
            return nullptr;
        }
        *out = t;
    }
    if (alloc) {
        if (!fresh && !t->has_al) free_all(t);  // buffers came from another allocator
        t->al = *alloc;
        t->has_al = true;
    } else if (t->has_al) {
        free_all(t);
        t->has_al = false;
    }
    t->st = static_cast<cudaStream_t>(stream);
    *rc = BT_OK;
    return t;
}

static void stage_set(btree *t, int i, int64_t start, int64_t end, int s, double alpha, double beta,
                      int flags, int gmax)
{
    SetRec &r = t->h_rec[i];
    r.start = (int)start;
    r.end = (int)end;
    r.s = s;
    r.flags = flags;
    r.gmax = gmax;
    r.pad = 0;
    r.alpha = alpha;
    r.beta = beta;
}

extern "C" {

int btree_build(const float *x, const float *y, const float *z, const float *h, int64_t n,
                int bucket_size, double alpha, double beta, const bt_allocator *alloc, void *stream,
                btree_t **out)
{
    if (!out || n < 0 || n >= (int64_t)INT32_MAX || bucket_size < 1 || bucket_size > (1 << 20) ||
        !is_finite_d(alpha) || !is_finite_d(beta))
        return BT_ERR_ARG;
    if (n > 0 && (!x || !y || !z || !h)) return BT_ERR_ARG;
    if (alloc && (!alloc->alloc || !alloc->free)) return BT_ERR_ARG;
    int rc;
    btree *t = prepare_handle(out, alloc, stream, &rc);
    if (!t) return rc;
    t->n = n;
    t->s = bucket_size;
    t->alpha = alpha;
    t->beta = beta;
    t->nsets = 1;
    if ((rc = ensure_set_caps(t, 1)) != BT_OK) return rc;
    stage_set(t, 0, 0, n, bucket_size, alpha, beta, 0, kGroupMax);
    return build_core(t, x, y, z, h);
}

int btree_build_batched(const float *x, const float *y, const float *z, const float *h,
                        const int64_t *offsets, int nsets, const bt_set_params *params,
                        const bt_allocator *alloc, void *stream, btree_t **out)
{
    if (!out || !offsets || nsets < 1 || nsets > (1 << 24)) return BT_ERR_ARG;
    if (offsets[0] != 0) return BT_ERR_ARG;
    for (int i = 0; i < nsets; i++)
        if (offsets[i + 1] < offsets[i]) return BT_ERR_ARG;
    const int64_t n = offsets[nsets];
    if (n >= (int64_t)INT32_MAX) return BT_ERR_ARG;
    if (n > 0 && (!x || !y || !z || !h)) return BT_ERR_ARG;
    if (alloc && (!alloc->alloc || !alloc->free)) return BT_ERR_ARG;
    int smin = 1 << 20;
    for (int i = 0; i < nsets; i++) {
        const int s = params ? params[i].bucket_size : 16;
        const double a = params ? params[i].alpha : 0.5, b = params ? params[i].beta : 0.5;
        if (s < 1 || s > (1 << 20) || !is_finite_d(a) || !is_finite_d(b)) return BT_ERR_ARG;
        if (params && (params[i].flags & ~BT_SET_OCTREE)) return BT_ERR_ARG;
        if (params && (params[i].group_size < 0 || params[i].group_size > kGroupMax)) return BT_ERR_ARG;
        smin = std::min(smin, s);
    }
    int rc;
    btree *t = prepare_handle(out, alloc, stream, &rc);
    if (!t) return rc;
    t->n = n;
    t->s = smin;
    t->alpha = params ? params[0].alpha : 0.5;
    t->beta = params ? params[0].beta : 0.5;
    t->nsets = nsets;
    if ((rc = ensure_set_caps(t, nsets)) != BT_OK) return rc;
    for (int i = 0; i < nsets; i++) {
        const int s = params ? params[i].bucket_size : 16;
        const double a = params ? params[i].alpha : 0.5, b = params ? params[i].beta : 0.5;
        const int f = params && (params[i].flags & BT_SET_OCTREE) ? kSetOctree : 0;
        const int g = params && params[i].group_size > 0 ? params[i].group_size : kGroupMax;
        stage_set(t, i, offsets[i], offsets[i + 1], s, a, b, f, g);
    }
    return build_core(t, x, y, z, h);
}

int btree_find_neighbors(const btree_t *t, int ngmax, int32_t *neighbors, int32_t *counts, void *stream)
{
    if (!t || ngmax < 1 || (t->n > 0 && (!neighbors || !counts))) return BT_ERR_ARG;
    if (t->n == 0) return BT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return to_status(launch_find(view(t), t->ngroups, ngmax, neighbors, counts, nullptr, nullptr,
                                 nullptr, t->sms, st));
}

int btree_find_neighbors_density(const btree_t *tc, const float *m, int ngmax, int32_t *neighbors,
                                 int32_t *counts, float *rho, void *stream)
{
    btree *t = const_cast<btree *>(tc);
    if (!t || ngmax < 1 || (t->n > 0 && (!neighbors || !counts || !m || !rho))) return BT_ERR_ARG;
    if (t->n == 0) return BT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (t->cap_smass < t->n) {
        cudaStream_t keep = t->st;
        t->st = st;
        bool ok = realloc_dev(t, t->smass, 0, t->n, false);
        t->st = keep;
        if (!ok) return BT_ERR_OOM;
        t->cap_smass = t->n;
    }
    return to_status(launch_find(view(t), t->ngroups, ngmax, neighbors, counts, m, t->smass, rho,
                                 t->sms, st));
}

int btree_find_neighbors_density_noalloc(const btree_t *t, const float *m, int ngmax,
                                         int32_t *neighbors, int32_t *counts, float *rho,
                                         void *stream)
{
    if (!t || ngmax < 1 || (t->n > 0 && (!neighbors || !counts || !m || !rho))) return BT_ERR_ARG;
    if (t->n > noalloc_max_particles()) return BT_ERR_CAPACITY;
    if (t->n == 0) return BT_OK;
    return to_status(launch_find_density_noalloc(view(t), t->ngroups, ngmax, neighbors, counts, m,
                                                 rho, t->sms, static_cast<cudaStream_t>(stream)));
}

int64_t btree_noalloc_max_particles(void) { return noalloc_max_particles(); }

int sph_density(const btree_t *t, const float *m, const int32_t *neighbors, const int32_t *counts,
                int ngmax, float *rho, void *stream)
{
    if (!t || ngmax < 1 || (t->n > 0 && (!m || !neighbors || !counts || !rho))) return BT_ERR_ARG;
    if (t->n == 0) return BT_OK;
    return to_status(launch_density(view(t), m, neighbors, counts, ngmax, rho, t->sms,
                                    static_cast<cudaStream_t>(stream)));
}

int btree_status(btree_t *t, void *stream, int *out)
{
    if (!t || !out) return BT_ERR_ARG;
    unsigned st = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (t->ctr) {
        cudaMemcpyAsync(&t->hctr->status, &t->ctr->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return to_status(e);
        st = t->hctr->status;
        cudaMemsetAsync(&t->ctr->status, 0, sizeof(unsigned), s);
        cudaStreamSynchronize(s);
    }
    int r = BT_OK;
    if (st & kStOversized) r = BT_WARN_OVERSIZED_LEAF;
    if (st & kStNgmax) r = BT_WARN_NGMAX;
    if (st & (kStCapNodes | kStCapSlots | kStCapGroups | kStCapSmall | kStCapBig)) r = BT_ERR_CAPACITY;
    if (st & kStNonfinite) r = BT_ERR_NONFINITE;
    *out = r;
    return BT_OK;
}

int btree_get_info(const btree_t *t, bt_info *info)
{
    if (!t || !info) return BT_ERR_ARG;
    *info = t->info;
    return BT_OK;
}

int btree_export(const btree_t *t, void *stream, double *node_lo, double *node_hi, int32_t *node_b,
                 int32_t *node_depth, int32_t *node_start, int32_t *node_count, int32_t *node_slot0,
                 int32_t *slot_start, int32_t *slot_count, int32_t *slot_child, int32_t *order)
{
    if (!t) return BT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nn = t->info.num_nodes, ns = t->info.num_slots, n = t->n;
    NodeGeom *g = nullptr;
    NodeWalk *w = nullptr;
    Slot *sl = nullptr;
    float4 *sp = nullptr;
    int rc = BT_OK;
    if (cudaMallocHost(&g, sizeof(NodeGeom) * (size_t)(nn + 1)) != cudaSuccess ||
        cudaMallocHost(&w, sizeof(NodeWalk) * (size_t)(nn + 1)) != cudaSuccess ||
        cudaMallocHost(&sl, sizeof(Slot) * (size_t)(ns + 1)) != cudaSuccess ||
        cudaMallocHost(&sp, sizeof(float4) * (size_t)(n + 1)) != cudaSuccess) {
        rc = BT_ERR_OOM;
    } else {
        if (nn) {
            cudaMemcpyAsync(g, t->geom, sizeof(NodeGeom) * nn, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(w, t->walk, sizeof(NodeWalk) * nn, cudaMemcpyDeviceToHost, s);
        }
        if (ns) cudaMemcpyAsync(sl, t->slots, sizeof(Slot) * ns, cudaMemcpyDeviceToHost, s);
        if (n) cudaMemcpyAsync(sp, t->spos, sizeof(float4) * n, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = to_status(e);
        } else {
            for (int64_t i = 0; i < nn; i++) {
                for (int l = 0; l < 3; l++) {
                    if (node_lo) node_lo[3 * i + l] = g[i].lo[l];
                    if (node_hi) node_hi[3 * i + l] = g[i].hi[l];
                }
                if (node_b) node_b[i] = w[i].b;
                if (node_depth) node_depth[i] = g[i].depth;
                if (node_start) node_start[i] = g[i].start;
                if (node_count) node_count[i] = g[i].count;
                if (node_slot0) node_slot0[i] = w[i].slot0;
            }
            for (int64_t k = 0; k < ns; k++) {
                if (slot_start) slot_start[k] = sl[k].start;
                if (slot_count) slot_count[k] = sl[k].count;
                if (slot_child) slot_child[k] = sl[k].child;
            }
            if (order)
                for (int64_t i = 0; i < n; i++) {
                    float v = sp[i].w;
                    int32_t o;
                    std::memcpy(&o, &v, 4);
                    order[i] = o;
                }
        }
    }
    cudaFreeHost(g);
    cudaFreeHost(w);
    cudaFreeHost(sl);
    cudaFreeHost(sp);
    return rc;
}

void btree_free(btree_t *t)
{
    if (!t) return;
    free_all(t);
    if (t->hctr) cudaFreeHost(t->hctr);
    if (t->h_rec) cudaFreeHost(t->h_rec);
    if (t->ev0) cudaEventDestroy(t->ev0);
    if (t->ev1) cudaEventDestroy(t->ev1);
    delete t;
}

const char *btree_strerror(int status)
{
    switch (status) {
    case BT_OK: return "ok";
    case BT_ERR_ARG: return "invalid argument";
    case BT_ERR_OOM: return "device allocation failed";
    case BT_ERR_CUDA: return "CUDA error";
    case BT_ERR_TIMEOUT: return "bounded device-side wait timed out";
    case BT_ERR_NONFINITE: return "non-finite position or smoothing length, or h < 0";
    case BT_ERR_CAPACITY: return "internal buffer capacity exceeded";
    case BT_WARN_NGMAX: return "some particle has more than ngmax neighbours (rows capped)";
    case BT_WARN_OVERSIZED_LEAF: return "some leaf holds more than bucket_size particles";
    default: return "unknown status";
    }
}

const char *btree_version(void) { return "btree-gb300 0.1 (sm_103a)"; }

uint64_t btree_kernel_launches(void) { return bt::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
