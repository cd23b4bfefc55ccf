// bt_api.cu -- the C ABI (include/btree.h): tree handle, buffers, the host
// side of BuildTree (the level loop over cells with > kSmallCap particles,
// host-driven or captured as a CUDA graph with device-driven loops), and the
// search, compressed-row and read-back entry points.
#include "bt_build.cuh"
#include "bt_find.cuh"
#include "bt_internal.cuh"

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <new>

using namespace bt;

namespace bt {
static std::atomic<uint64_t> g_launches{0};
// Launches issued while capturing a graph are counted when the graph runs.
static thread_local bool g_capturing = false;
void note_launch(int k)
{
    if (!g_capturing) g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed);
}
}  // namespace bt

// Everything a captured graph bakes in; an unchanged key relaunches it.
struct GraphKey {
    TreeDev T;
    LevelBufs L;
    const SetRec *rec;  // mapped staging of the per-set records
    const float *m;
    float *smass, *rho;
    int32_t *nbrs, *counts;
    int ngmax, sms;
    long long root_chunks;  // sets the grid of the root passes
};


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
    Counters *hctr = nullptr;  // = &rb->c: the host's copy of the counters
    Readback *rb = nullptr;    // mapped pinned host memory ...
    Readback *rb_dev = nullptr;  // ... and its device address
    float *smass = nullptr;
    // per-set tables (device) and their pinned host staging
    int nsets = 0, cap_sets = 0;
    int *set_start = nullptr, *set_s = nullptr, *set_na = nullptr, *set_gmax = nullptr;
    int *set_chunk0 = nullptr;
    long long root_chunks = 0;  // root-pass blocks over all sets
    int *set_flags = nullptr, *set_bbox = nullptr;
    double *set_beta = nullptr;
    SetRec *h_rec = nullptr;    // [cap_sets] mapped pinned staging, read by k_init_sets
    SetRec *h_rec_dev = nullptr;

    int ngroups = 0, ngroups_c = 0;  // work units of the wide / compact lists
    bt_info info{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t hist_need_seen = 0;  // largest level histogram asked for so far
    // compressed rows: per-particle counts, scan scratch, pinned total
    int32_t *csr_counts = nullptr;
    long long *csr_scratch = nullptr;
    int64_t cap_csr = 0;

    // graph form: private capture streams, the executable graph and its key
    cudaStream_t gs[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    // asynchronous rebuilds: the build alone as a graph (its own executable),
    // launched without waiting once an earlier build of the same size has set
    // the buffer capacities.  `pending`: its host-side finish (counters, info)
    // is still to be read; ev_staged: its per-set records were read;
    // ev_built: it finished (counters in mapped host memory).
    cudaGraphExec_t gexec_b = nullptr;
    GraphKey gkey_b{};
    bool pending = false;
    cudaEvent_t ev_staged = nullptr, ev_built = nullptr;
    int64_t async_n = -1;
    int async_nsets = -1;
    SetRec *async_rec = nullptr;  // host copy of the records of the last synchronous build
    int cap_async_rec = 0;
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
    dev_free(t, t->csr_counts); dev_free(t, t->csr_scratch);
    t->csr_counts = nullptr;
    t->csr_scratch = nullptr;
    t->cap_csr = 0;
    dev_free(t, t->set_start); dev_free(t, t->set_s); dev_free(t, t->set_na); dev_free(t, t->set_gmax);
    dev_free(t, t->set_flags); dev_free(t, t->set_bbox); dev_free(t, t->set_beta);
    dev_free(t, t->set_chunk0);
    t->set_start = t->set_s = t->set_na = t->set_gmax = t->set_chunk0 = nullptr;
    t->set_flags = t->set_bbox = nullptr;
    t->set_beta = nullptr;
    t->cap_sets = 0;
    t->geom = nullptr; t->walk = nullptr; t->slots = nullptr; t->groups = nullptr;
    t->spos = nullptr; t->sh = nullptr; t->inv = nullptr;
    for (int k = 0; k < 2; k++) { t->wpos[k] = nullptr; t->wh[k] = nullptr; t->big_ids[k] = nullptr; }
    t->hist = t->hoff = t->cursor = t->tiles = nullptr;
    t->big = nullptr; t->small = nullptr; t->ctr = nullptr; t->smass = nullptr;
    t->cap_n = 0; t->cap_nodes = t->cap_slots = t->cap_groups = t->cap_small = t->cap_big = 0;
    t->cap_hist = 0; t->cap_smass = 0;
    t->async_n = -1;  // the capacities are gone: the next build is synchronous
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
    T.set_chunk0 = t->set_chunk0;
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
    T.small_hist = small_hist_cells((int)std::max<int64_t>(t->s, 1));
    T.tiny_hist = small_hist_cells((int)std::max<int64_t>(t->s, 1), kTinyCap);
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
        if (!realloc_dev(t, t->small, 0, 2 * want_small, false)) return BT_ERR_OOM;  // two queues
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

// Histogram capacity.  A big cell of c > kSmallCap particles has
// b0^3 < max(8, 3.375 c/s) histogram entries (b0 >= 3 means cbrt(c/s) > 2,
// so b0 < cbrt(c/s) + 1 < 1.5 cbrt(c/s)), and a level's cells are disjoint:
// one level never needs more than n max(8/257, 3.375/s_min) entries.
int ensure_hist(btree *t)
{
    const double per = std::max(8.0 / (double)(kSmallCap + 1), 3.375 / (double)t->s);
    const int64_t need = std::max<int64_t>((int64_t)std::ceil((double)t->n * per) + 64,
                                           t->hist_need_seen);
    if (t->cap_hist >= need) return BT_OK;
    int64_t c = std::max<int64_t>(need, 4096);
    if (c >= INT32_MAX) return BT_ERR_CAPACITY;
    if (!realloc_dev(t, t->hist, 0, c, false) || !realloc_dev(t, t->hoff, 0, c, false) ||
        !realloc_dev(t, t->cursor, 0, c, false) ||
        !realloc_dev(t, t->tiles, 0, scan_tile_count(c) + 1, false))
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
        !realloc_dev(t, t->set_chunk0, 0, c + 1, false) ||
        !realloc_dev(t, t->set_beta, 0, c, false) ||
        !realloc_dev(t, t->set_flags, 0, c, false) || !realloc_dev(t, t->set_bbox, 0, 6 * c, false))
        return BT_ERR_OOM;
    // the previous build has finished reading the staging (builds end synchronised)
    if (t->h_rec) cudaFreeHost(t->h_rec);
    t->h_rec = nullptr;
    if (cudaHostAlloc(&t->h_rec, sizeof(SetRec) * (size_t)c, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&t->h_rec_dev, t->h_rec, 0) != cudaSuccess) {
        cudaGetLastError();
        return BT_ERR_OOM;
    }
    t->cap_sets = c;
    return BT_OK;
}

int read_counters(btree *t, cudaStream_t st)
{
    launch_readback(t->ctr, t->cap_nodes > 0 ? t->walk : nullptr, t->rb_dev, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return to_status(e);
    return to_status(cudaGetLastError());
}

LevelBufs lview(const btree *t, const float *x, const float *y, const float *z, const float *h)
{
    LevelBufs L;
    L.in = Src{x, y, z, h, nullptr, nullptr};
    for (int k = 0; k < 2; k++) {
        L.wpos[k] = t->wpos[k];
        L.wh[k] = t->wh[k];
        L.ids[k] = t->big_ids[k];
    }
    L.big = t->big;
    L.hist = t->hist;
    L.hoff = t->hoff;
    L.cursor = t->cursor;
    L.tiles = t->tiles;
    L.small = t->small;
    L.tiny = t->small ? t->small + t->cap_small : nullptr;
    L.cap_hist = t->cap_hist;
    L.cap_big = t->cap_big;
    L.cap_tiles = scan_tile_count(t->cap_hist);
    return L;
}

constexpr int kRetry = 100;
constexpr unsigned kCapBits = kStCapNodes | kStCapSlots | kStCapGroups | kStCapSmall | kStCapBig;

// Timing events: inside a capture an ordinary record only orders streams of
// the capture; an external record is a real node of the graph.
void record_event(cudaEvent_t ev, cudaStream_t st, bool capture)
{
    if (capture) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else cudaEventRecord(ev, st);
}

// The steps before the level loop (both forms of the build).
void launch_build_head(btree *t, const TreeDev &T, const LevelBufs &L, cudaStream_t st,
                       bool capture = false)
{
    launch_init_counters(t->ctr, t->nsets, st);
    launch_init_sets(T, t->h_rec_dev, t->set_start, t->set_s, t->set_na, t->set_beta, t->set_gmax,
                     t->set_chunk0, st);
    if (capture && t->ev_staged) record_event(t->ev_staged, st, true);
    record_event(t->ev0, st, capture);
    launch_bbox(T, L.in.x, L.in.y, L.in.z, L.in.h, t->root_chunks, t->sms, st);
    launch_roots(T, L, t->root_chunks, t->sms, st);
}

// After the build (counters on the host): retry on capacity, info.
int finish_build(btree *t, cudaStream_t st)
{
    const Counters &c = *t->hctr;
    if (c.status & kStNonfinite) return BT_ERR_NONFINITE;
    if (c.abort || (c.status & kCapBits) || (int64_t)c.ngroups + c.ngroups_c > t->cap_groups) {
        t->hist_need_seen = std::max<int64_t>(t->hist_need_seen, c.hist_need);
        return kRetry;
    }
    t->ngroups = c.ngroups;
    t->ngroups_c = c.ngroups_c;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, t->ev0, t->ev1) != cudaSuccess) {
        cudaGetLastError();
        ms = 0.0f;
    }
    bt_info &I = t->info;
    I.n = t->n;
    I.bucket_size = t->s;
    I.max_depth = c.max_depth;
    I.num_nodes = c.nnodes;
    I.num_slots = c.nslots;
    I.num_groups = c.ngroups + c.ngroups_c;
    I.root_b = t->rb->root_b;
    I.num_oversized = c.noversized;
    I.build_ms = ms;
    return (c.status & kStOversized) ? BT_WARN_OVERSIZED_LEAF : BT_OK;
}

// Host-driven BuildTree: the host reads the device counters after each step
// of the level loop and of the ratio loop (Eq. 4) to decide what follows.
int do_build(btree *t, const float *x, const float *y, const float *z, const float *h)
{
    cudaStream_t st = t->st;
    const TreeDev T = view(t);
    const LevelBufs L = lview(t, x, y, z, h);
    launch_build_head(t, T, L, st);
    launch_level_go(t->ctr, 0, 0, 0, st);
    int rc = read_counters(t, st);
    if (rc != BT_OK) return rc;
    if (t->hctr->status & kStNonfinite) return BT_ERR_NONFINITE;
    while (t->hctr->level_go) {
        LevelHints H{t->hctr->nbig_next, 0, 0};
        launch_level_start(T, L, H, t->sms, 0, 0, st);
        if ((rc = read_counters(t, st)) != BT_OK) return rc;
        if (t->hctr->abort) break;
        H.hist = t->hctr->hist_total;
        H.chunks = t->hctr->chunk_total;
        launch_level_zero(T, L, H, t->sms, st);
        do {
            launch_ratio_pass(T, L, H, t->sms, 0, 0, st);
            if ((rc = read_counters(t, st)) != BT_OK) return rc;
        } while (t->hctr->ratio_go);
        launch_level_finish(T, L, H, t->sms, 0, 0, st);
        if ((rc = read_counters(t, st)) != BT_OK) return rc;
    }
    if (!t->hctr->abort)
        launch_small(T, L, std::min(t->hctr->nsmall, t->cap_small), std::min(t->hctr->ntiny, t->cap_small),
                     t->sms, st);
    cudaEventRecord(t->ev1, st);
    if ((rc = read_counters(t, st)) != BT_OK) return rc;
    return finish_build(t, st);
}

// ---------------------------------------------------------------- graph form
// A conditional while-node after the work captured so far on `st`; returns
// its body graph.  Later work on `st` follows the node.
cudaError_t add_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, ed, nd, &p);
    if (e != cudaSuccess) return e;
    *body = p.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

cudaError_t capture_graph_of(cudaStream_t st, cudaGraph_t *g)
{
    cudaStreamCaptureStatus cs;
    return cudaStreamGetCaptureInfo(st, &cs, nullptr, g, nullptr, nullptr, nullptr);
}


// Captures build + find (+ density) on the handle's private streams.  The
// level loop and the ratio loop are while-nodes whose conditions the level
// kernels set on the device.
cudaError_t capture_step(btree *t, const GraphKey &K, cudaGraph_t *out)
{
    cudaStream_t s0 = t->gs[0], s1 = t->gs[1], s2 = t->gs[2];
    const TreeDev &T = K.T;
    const LevelBufs &L = K.L;
    const LevelHints Hc{t->cap_big, t->cap_hist, t->n / kBigChunk + t->cap_big + 1};
    cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (err == cudaSuccess && x != cudaSuccess) err = x; };
    cudaGraph_t g0 = nullptr, lbody = nullptr, rbody = nullptr;
    cudaGraphConditionalHandle hlevel = 0, hratio = 0;
    launch_build_head(t, T, L, s0, true);
    chk(capture_graph_of(s0, &g0));
    if (err == cudaSuccess) chk(cudaGraphConditionalHandleCreate(&hlevel, g0, 0, cudaGraphCondAssignDefault));
    launch_level_go(t->ctr, 0, hlevel, 1, s0);
    if (err == cudaSuccess) chk(add_while(s0, hlevel, &lbody));
    if (err == cudaSuccess) {
        chk(cudaStreamBeginCaptureToGraph(s1, lbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (err == cudaSuccess) {
            chk(cudaGraphConditionalHandleCreate(&hratio, lbody, 0, cudaGraphCondAssignDefault));
            launch_level_start(T, L, Hc, t->sms, hratio, 1, s1);
            launch_level_zero(T, L, Hc, t->sms, s1);
            if (err == cudaSuccess) chk(add_while(s1, hratio, &rbody));
            if (err == cudaSuccess) {
                chk(cudaStreamBeginCaptureToGraph(s2, rbody, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
                if (err == cudaSuccess) {
                    launch_ratio_pass(T, L, Hc, t->sms, hratio, 1, s2);
                    chk(cudaStreamEndCapture(s2, &rbody));
                }
            }
            launch_level_finish(T, L, Hc, t->sms, hlevel, 1, s1);
            chk(cudaStreamEndCapture(s1, &lbody));
        }
    }
    launch_small(T, L, t->cap_small, t->cap_small, t->sms, s0);
    record_event(t->ev1, s0, true);
    if (!K.nbrs) {
        // the build alone: counters to mapped host memory, then its event
        launch_readback(t->ctr, t->walk, t->rb_dev, s0);
        if (t->ev_built) record_event(t->ev_built, s0, true);
    }
    if (K.nbrs) chk(launch_find(T, -1, -1, K.ngmax, K.nbrs, K.counts, K.m, K.smass, K.rho, t->sms, s0));
    cudaGraph_t g = nullptr;
    chk(cudaStreamEndCapture(s0, &g));
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return err;
    }
    *out = g;
    return cudaSuccess;
}

// Kernels one run of the captured graph launched (for the launch counter).
uint64_t graph_launches(const Counters &c, bool find, bool dens)
{
    // head: init_counters, init_sets, bbox, root_sets, copy_leaf_roots, level_go;
    // per level: begin, setup, scan, zero, finish, 3 scans, emit, scatter, level_go;
    // per ratio pass: hist, count, decide, zero, ratio_end; then the two warp
    // builders and find (find: the two work-unit lists and the pass over the
    // units split by them)
    return 6 + 11 * (uint64_t)c.level + 5 * (uint64_t)c.ratio_total + 2 + (find ? 3 + (dens ? 1 : 0) : 0);
}

// Launches the captured step (captured again when a pointer or size
// changed); the build-only graph and the build + find graph are kept apart.
cudaError_t launch_step_graph(btree *t, const GraphKey &K, cudaStream_t user)
{
    const bool build_only = K.nbrs == nullptr;
    cudaGraphExec_t &gx = build_only ? t->gexec_b : t->gexec;
    GraphKey &gk = build_only ? t->gkey_b : t->gkey;
    if (!gx || std::memcmp(&K, &gk, sizeof(GraphKey)) != 0) {
        cudaGraph_t g = nullptr;
        g_capturing = true;
        cudaError_t e = capture_step(t, K, &g);
        g_capturing = false;
        if (e != cudaSuccess) return e;
        bool updated = false;
        if (gx) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(gx, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(gx);
                gx = nullptr;
            }
        }
        if (!updated) e = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            gx = nullptr;
            return e;
        }
        std::memcpy(&gk, &K, sizeof(GraphKey));
    }
    return cudaGraphLaunch(gx, user);
}

// The host-side end of an asynchronous build: wait for it, read its
// counters, account its launches.  A build that ran out of capacity (or saw
// non-finite input) reports it here, and the next build runs synchronously
// with retries.
int finish_pending(btree *t)
{
    if (!t->pending) return BT_OK;
    t->pending = false;
    cudaError_t e = cudaEventSynchronize(t->ev_built);
    if (e != cudaSuccess) return to_status(e);
    note_launch((int)(graph_launches(*t->hctr, false, false) + 1));
    const int rc = finish_build(t, t->st);
    if (rc == kRetry || rc < 0) t->async_n = -1;
    return rc == kRetry ? BT_ERR_CAPACITY : rc;
}

// The build alone, as one graph launch on `user`, without waiting for it.
int run_graph_build_async(btree *t, const float *x, const float *y, const float *z, const float *h,
                          cudaStream_t user)
{
    for (int k = 0; k < 3; k++)
        if (!t->gs[k] && cudaStreamCreateWithFlags(&t->gs[k], cudaStreamNonBlocking) != cudaSuccess)
            return BT_ERR_CUDA;
    GraphKey K;
    std::memset(&K, 0, sizeof(K));
    K.T = view(t);
    K.L = lview(t, x, y, z, h);
    K.rec = t->h_rec_dev;
    K.sms = t->sms;
    K.root_chunks = t->root_chunks;
    cudaError_t e = launch_step_graph(t, K, user);
    if (e != cudaSuccess) return to_status(e);
    t->pending = true;
    return BT_OK;
}

int run_graph_step(btree *t, const float *x, const float *y, const float *z, const float *h,
                   const float *m, int ngmax, int32_t *nbrs, int32_t *counts, float *rho,
                   cudaStream_t user)
{
    for (int k = 0; k < 3; k++)
        if (!t->gs[k] && cudaStreamCreateWithFlags(&t->gs[k], cudaStreamNonBlocking) != cudaSuccess)
            return BT_ERR_CUDA;
    GraphKey K;
    std::memset(&K, 0, sizeof(K));
    K.T = view(t);
    K.L = lview(t, x, y, z, h);
    K.rec = t->h_rec_dev;
    K.m = m;
    K.smass = m ? t->smass : nullptr;
    K.rho = rho;
    K.nbrs = nbrs;
    K.counts = counts;
    K.ngmax = ngmax;
    K.sms = t->sms;
    K.root_chunks = t->root_chunks;
    // the graph runs on the private stream s0's ordering inside; it is
    // launched on the caller's stream
    cudaError_t e = launch_step_graph(t, K, user);
    if (e != cudaSuccess) return to_status(e);
    int rc = read_counters(t, user);
    if (rc != BT_OK) return rc;
    note_launch((int)graph_launches(*t->hctr, nbrs != nullptr, m != nullptr));
    return finish_build(t, user);
}

bool is_finite_d(double v) { return std::isfinite(v); }

}  // namespace

// Shared front end of the builds: the per-set records must already be staged
// in t->h_rec.  `graph`: build (+ find) as one CUDA graph.
static int build_core(btree *t, const float *x, const float *y, const float *z, const float *h,
                      bool graph = false, const float *m = nullptr, int ngmax = 0,
                      int32_t *nbrs = nullptr, int32_t *counts = nullptr, float *rho = nullptr,
                      cudaStream_t user = nullptr)
{
    int rc = BT_OK;
    // steady state: the sizes of the last synchronous build, whose capacities
    // held -- the build runs as one graph launch and the call returns at once
    if (!graph && t->n > 0 && t->async_n == t->n && t->async_nsets == t->nsets && t->ev_built &&
        t->async_rec && std::memcmp(t->async_rec, t->h_rec, sizeof(SetRec) * (size_t)t->nsets) == 0) {
        rc = run_graph_build_async(t, x, y, z, h, t->st);
        if (rc == BT_OK) return BT_OK;
        cudaGetLastError();  // could not launch it: build synchronously
    }
    for (int attempt = 0; attempt < 6; attempt++) {
        rc = ensure_particle_caps(t, t->n);
        if (rc == BT_OK) rc = ensure_hist(t);
        if (rc == BT_OK && m && t->cap_smass < t->n) {
            if (!realloc_dev(t, t->smass, 0, std::max<int64_t>(t->n, 1), false)) rc = BT_ERR_OOM;
            else t->cap_smass = std::max<int64_t>(t->n, 1);
        }
        if (rc != BT_OK) break;
        rc = graph ? run_graph_step(t, x, y, z, h, m, ngmax, nbrs, counts, rho, user)
                   : do_build(t, x, y, z, h);
        if (rc != kRetry) break;
        // grow the tree-size buffers and build again
        int64_t cn = std::min<int64_t>((int64_t)t->cap_nodes * 2, INT32_MAX / 2);
        int64_t cs = std::min<int64_t>((int64_t)t->cap_slots * 2, INT32_MAX / 2);
        int64_t cm = std::min<int64_t>((int64_t)t->cap_small * 2 + 1024, INT32_MAX / 2);
        if (!realloc_dev(t, t->geom, 0, cn, false) || !realloc_dev(t, t->walk, 0, cn, false) ||
            !realloc_dev(t, t->slots, 0, cs, false) || !realloc_dev(t, t->small, 0, 2 * cm, false)) {
            rc = BT_ERR_OOM;
            break;
        }
        t->cap_nodes = (int)cn;
        t->cap_slots = (int)cs;
        t->cap_small = (int)cm;
        rc = BT_ERR_CAPACITY;
    }
    if (rc >= 0 && !graph) {
        // the same sets and parameters (new positions allowed) may now be
        // rebuilt asynchronously in these buffers
        if (t->cap_async_rec < t->nsets) {
            std::free(t->async_rec);
            t->async_rec = static_cast<SetRec *>(std::malloc(sizeof(SetRec) * (size_t)t->nsets));
            t->cap_async_rec = t->async_rec ? t->nsets : 0;
        }
        if (t->async_rec) {
            std::memcpy(t->async_rec, t->h_rec, sizeof(SetRec) * (size_t)t->nsets);
            t->async_n = t->n;
            t->async_nsets = t->nsets;
        }
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
        if (cudaHostAlloc(&t->rb, sizeof(Readback), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(&t->rb_dev, t->rb, 0) != cudaSuccess ||
            cudaEventCreate(&t->ev0) != cudaSuccess || cudaEventCreate(&t->ev1) != cudaSuccess) {
            cudaGetLastError();
            delete t;
            *rc = BT_ERR_CUDA;
            return nullptr;
        }
        t->hctr = &t->rb->c;
        if (cudaEventCreateWithFlags(&t->ev_staged, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&t->ev_built, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            t->ev_staged = t->ev_built = nullptr;  // no asynchronous rebuilds then
        }
        *out = t;
    } else if (t->pending) {
        // the previous asynchronous build must be finished (its records are
        // restaged and its buffers may be reallocated below)
        finish_pending(t);
    }
    if (alloc) {
        // buffers from another allocator (or the default) go back to it first
        const bool same = t->has_al && t->al.ctx == alloc->ctx && t->al.alloc == alloc->alloc &&
                          t->al.free == alloc->free;
        if (!fresh && !same) free_all(t);
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
    // sets are staged in order: the blocks of set i follow those of set i - 1
    r.chunk0 = i == 0 ? 0 : (int)t->root_chunks;
    t->root_chunks = r.chunk0 + (end - start + kRootChunk - 1) / kRootChunk;
    r.alpha = alpha;
    r.beta = beta;
}

// ------------------------------------------------------------------ arithmetic rates
namespace bt {

constexpr int kRateChains = 8;  // independent FMA chains per thread

__device__ __forceinline__ float rate_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rate_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ unsigned long long rate_fma(unsigned long long a, unsigned long long b,
                                                       unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

template <class V>
__global__ void __launch_bounds__(256) k_fma_rate(V *sink, int iters, V b, V c, V a0)
{
    V a[kRateChains];
#pragma unroll
    for (int k = 0; k < kRateChains; k++) a[k] = a0;
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int k = 0; k < kRateChains; k++) a[k] = rate_fma(a[k], b, c);
    bool keep = false;
#pragma unroll
    for (int k = 0; k < kRateChains; k++) keep |= a[k] == b;  // never true: keeps the chains live
    if (keep) sink[threadIdx.x] = a[0];
}

template <class V>
static cudaError_t time_rate(cudaStream_t st, int sms, int iters, V b, V c, V a0, double flops_per_fma,
                             double *gflops)
{
    V *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 256 * sizeof(V));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8;
    note_launch();
    k_fma_rate<V><<<blocks, 256, 0, st>>>(sink, iters / 8, b, c, a0);  // warm-up
    cudaEventRecord(e0, st);
    note_launch();
    k_fma_rate<V><<<blocks, 256, 0, st>>>(sink, iters, b, c, a0);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && gflops)
        *gflops = flops_per_fma * kRateChains * (double)iters * blocks * 256 / (ms * 1e6);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return e;
}

static unsigned long long pack2(float f)
{
    unsigned u;
    std::memcpy(&u, &f, sizeof(u));
    return ((unsigned long long)u << 32) | u;
}

static int arith_rates(cudaStream_t st, double *fp32, double *fp32x2, double *fp64)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = time_rate<float>(st, sms, 16384, 0.9999999f, 1e-7f, 1.0f, 2.0, fp32);
    if (e == cudaSuccess) {
        e = time_rate<unsigned long long>(st, sms, 16384, pack2(0.9999999f), pack2(1e-7f), pack2(1.0f), 4.0,
                                          fp32x2);
    }
    if (e == cudaSuccess) e = time_rate<double>(st, sms, 512, 0.9999999999, 1e-12, 1.0, 2.0, fp64);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

}  // namespace bt

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

static int stage_batched(const float *x, const float *y, const float *z, const float *h,
                         const int64_t *offsets, int nsets, const bt_set_params *params,
                         const bt_allocator *alloc, void *stream, btree_t **out, btree **tp)
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
        if (params && (params[i].flags & ~(BT_SET_OCTREE | BT_SET_FIND_COMPACT | BT_SET_2D | BT_SET_PACK_LEAVES)))
            return BT_ERR_ARG;
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
        const int f = (params && (params[i].flags & BT_SET_OCTREE) ? kSetOctree : 0) |
                      (params && (params[i].flags & BT_SET_FIND_COMPACT) ? kSetFindCompact : 0) |
                      (params && (params[i].flags & BT_SET_2D) ? kSetTwoD : 0) |
                      (params && (params[i].flags & BT_SET_PACK_LEAVES) ? kSetPackLeaves : 0);
        const int g = params && params[i].group_size > 0 ? params[i].group_size : kGroupMax;
        stage_set(t, i, offsets[i], offsets[i + 1], s, a, b, f, g);
    }
    *tp = t;
    return BT_OK;
}

int btree_build_batched(const float *x, const float *y, const float *z, const float *h,
                        const int64_t *offsets, int nsets, const bt_set_params *params,
                        const bt_allocator *alloc, void *stream, btree_t **out)
{
    btree *t = nullptr;
    int rc = stage_batched(x, y, z, h, offsets, nsets, params, alloc, stream, out, &t);
    if (rc != BT_OK) return rc;
    return build_core(t, x, y, z, h);
}

int btree_build_find_batched(const float *x, const float *y, const float *z, const float *h,
                             const float *m, const int64_t *offsets, int nsets,
                             const bt_set_params *params, int ngmax, int32_t *neighbors,
                             int32_t *counts, float *rho, const bt_allocator *alloc, void *stream,
                             btree_t **out)
{
    if (ngmax < 1 || !offsets || nsets < 1) return BT_ERR_ARG;
    if (offsets[nsets] > 0 && (!neighbors || !counts || (m && !rho))) return BT_ERR_ARG;
    btree *t = nullptr;
    int rc = stage_batched(x, y, z, h, offsets, nsets, params, alloc, stream, out, &t);
    if (rc != BT_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool any = t->n > 0;
    rc = build_core(t, x, y, z, h, true, any ? m : nullptr, ngmax, any ? neighbors : nullptr,
                    counts, any && m ? rho : nullptr, st);
    if (rc < 0 || !any) return rc;
    const unsigned stw = t->hctr->status;
    if (stw & kStNgmax) return BT_WARN_NGMAX;
    return rc;
}

int btree_find_neighbors(const btree_t *t, int ngmax, int32_t *neighbors, int32_t *counts, void *stream)
{
    if (!t || ngmax < 1 || (t->n > 0 && (!neighbors || !counts))) return BT_ERR_ARG;
    if (t->n == 0) return BT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool dc = t->pending;  // counts not on the host yet: read on the device
    return to_status(launch_find(view(t), dc ? -1 : t->ngroups, dc ? -1 : t->ngroups_c, ngmax, neighbors, counts,
                                 nullptr, nullptr, nullptr, t->sms, st));
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
    const bool dc = t->pending;  // counts not on the host yet: read on the device
    return to_status(launch_find(view(t), dc ? -1 : t->ngroups, dc ? -1 : t->ngroups_c, ngmax, neighbors, counts,
                                 m, t->smass, rho, t->sms, st));
}

int btree_find_neighbors_density_noalloc(const btree_t *t, const float *m, int ngmax,
                                         int32_t *neighbors, int32_t *counts, float *rho,
                                         void *stream)
{
    if (!t || ngmax < 1 || (t->n > 0 && (!neighbors || !counts || !m || !rho))) return BT_ERR_ARG;
    if (t->n > noalloc_max_particles()) return BT_ERR_CAPACITY;
    if (t->n == 0) return BT_OK;
    // the scratch address is looked up for the current device: it must be
    // the tree's
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device) return BT_ERR_ARG;
    const bool dc = t->pending;  // counts not on the host yet: read on the device
    return to_status(launch_find_density_noalloc(view(t), dc ? -1 : t->ngroups, dc ? -1 : t->ngroups_c, ngmax,
                                                 neighbors, counts, m, rho, t->sms,
                                                 static_cast<cudaStream_t>(stream)));
}

int64_t btree_noalloc_max_particles(void) { return noalloc_max_particles(); }

int btree_pack_rows(const btree_t *tc, const int32_t *rows, const int32_t *counts, int ngmax,
                    int64_t *offsets, int32_t *csr, int64_t capacity, int64_t *total, void *stream)
{
    btree *t = const_cast<btree *>(tc);
    if (!t || ngmax < 1 || !offsets || capacity < 0 || (t->n > 0 && (!rows || !counts))) return BT_ERR_ARG;
    const int prc = finish_pending(t);
    if (prc < 0) return prc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = t->n;
    if (n == 0) {
        cudaMemsetAsync(offsets, 0, sizeof(int64_t), st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return BT_ERR_CUDA;
        if (total) *total = 0;
        return BT_OK;
    }
    if (t->cap_csr < n) {
        cudaStream_t keep = t->st;
        t->st = st;
        const bool ok = realloc_dev(t, t->csr_counts, 0, n, false) &&
                        realloc_dev(t, t->csr_scratch, 0, csr_scratch_elems(n), false);
        t->st = keep;
        if (!ok) return BT_ERR_OOM;
        t->cap_csr = n;
    }
    launch_scan64(counts, n, ngmax, reinterpret_cast<long long *>(offsets), t->csr_scratch, st);
    launch_readback_total(reinterpret_cast<const long long *>(offsets + n), t->rb_dev, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return to_status(e);
    const int64_t tot = t->rb->total;
    if (total) *total = tot;
    if (!csr) return BT_OK;
    if (tot > capacity) return BT_ERR_CAPACITY;
    launch_pack_rows(rows, counts, n, ngmax, reinterpret_cast<const long long *>(offsets), csr, t->sms, st);
    return to_status(cudaGetLastError());
}

int btree_find_neighbors_csr(const btree_t *tc, int flags, const float *m, float *rho, int64_t *offsets,
                             int32_t *neighbors, int64_t capacity, int64_t *total, void *stream)
{
    btree *t = const_cast<btree *>(tc);
    if (!t || !offsets || (m == nullptr) != (rho == nullptr) || capacity < 0) return BT_ERR_ARG;
    if ((flags & ~BT_FIND_HALF) || ((flags & BT_FIND_HALF) && m)) return BT_ERR_ARG;
    const int half = (flags & BT_FIND_HALF) ? 1 : 0;
    const int prc = finish_pending(t);
    if (prc < 0) return prc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = t->n;
    if (n == 0) {
        cudaMemsetAsync(offsets, 0, sizeof(int64_t), st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return BT_ERR_CUDA;
        if (total) *total = 0;
        return BT_OK;
    }
    // scratch (allocated on this stream)
    cudaStream_t keep = t->st;
    t->st = st;
    bool ok = true;
    if (t->cap_csr < n) {
        ok = realloc_dev(t, t->csr_counts, 0, n, false) &&
             realloc_dev(t, t->csr_scratch, 0, csr_scratch_elems(n), false);
        if (ok) t->cap_csr = n;
    }
    if (ok && m && t->cap_smass < n) {
        ok = realloc_dev(t, t->smass, 0, n, false);
        if (ok) t->cap_smass = n;
    }
    t->st = keep;
    if (!ok) return BT_ERR_OOM;
    const TreeDev T = view(t);
    cudaError_t e = launch_find_csr_count(T, t->ngroups, t->ngroups_c, t->csr_counts, m, t->smass, rho,
                                          reinterpret_cast<long long *>(offsets), t->csr_scratch, half,
                                          t->sms, st);
    if (e != cudaSuccess) return to_status(e);
    launch_readback_total(reinterpret_cast<const long long *>(offsets + n), t->rb_dev, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return to_status(e);
    const int64_t tot = t->rb->total;
    if (total) *total = tot;
    if (!neighbors) return BT_OK;
    if (tot > capacity) return BT_ERR_CAPACITY;
    return to_status(launch_find_csr_rows(T, t->ngroups, t->ngroups_c,
                                          reinterpret_cast<const long long *>(offsets), neighbors,
                                          t->csr_counts, half, t->sms, st));
}

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
    const int prc = finish_pending(t);
    if (prc == BT_ERR_CUDA) return prc;
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

int btree_get_info(const btree_t *tc, bt_info *info)
{
    if (!tc || !info) return BT_ERR_ARG;
    btree *t = const_cast<btree *>(tc);
    const int rc = finish_pending(t);
    if (rc < 0) return rc;
    *info = t->info;
    return BT_OK;
}

int btree_export(const btree_t *t, void *stream, double *node_lo, double *node_hi, int32_t *node_b,
                 int32_t *node_depth, int32_t *node_start, int32_t *node_count, int32_t *node_slot0,
                 int32_t *slot_start, int32_t *slot_count, int32_t *slot_child, int32_t *order)
{
    if (!t) return BT_ERR_ARG;
    const int prc = finish_pending(const_cast<btree *>(t));
    if (prc < 0) return prc;
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
    if (t->pending) cudaEventSynchronize(t->ev_built);
    if (t->gexec) cudaGraphExecDestroy(t->gexec);
    if (t->gexec_b) cudaGraphExecDestroy(t->gexec_b);
    if (t->ev_staged) cudaEventDestroy(t->ev_staged);
    if (t->ev_built) cudaEventDestroy(t->ev_built);
    std::free(t->async_rec);
    for (int k = 0; k < 3; k++)
        if (t->gs[k]) cudaStreamDestroy(t->gs[k]);
    free_all(t);
    if (t->rb) cudaFreeHost(t->rb);
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

int btree_arith_rates(void *stream, double *fp32_gflops, double *fp32x2_gflops, double *fp64_gflops)
{
    return bt::arith_rates(static_cast<cudaStream_t>(stream), fp32_gflops, fp32x2_gflops, fp64_gflops);
}

uint64_t btree_kernel_launches(void) { return bt::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
