// bt_build.cuh -- launchers of the BuildTree kernels (bt_build.cu).
#pragma once
#include "bt_internal.cuh"

namespace bt {

// Grid sizes of a level's kernels: the host's knowledge of the work (exact
// when it read the counters, capacities inside a graph).  The kernels read
// the true counts from the device and loop over them.
struct LevelHints {
    long long nbig;    // big cells
    long long hist;    // histogram entries
    long long chunks;  // kBigChunk particle blocks
};

void launch_init_counters(Counters *ctr, int nroots, cudaStream_t st);
void launch_init_sets(const TreeDev &T, const SetRec *rec, int *set_start, int *set_s, int *set_na,
                      double *set_beta, int *set_gmax, int *set_chunk0, cudaStream_t st);
void launch_bbox(const TreeDev &T, const float *x, const float *y, const float *z, const float *h,
                 long long chunks, int sms, cudaStream_t st);
void launch_roots(const TreeDev &T, const LevelBufs &L, long long chunks, int sms, cudaStream_t st);
void launch_level_go(Counters *ctr, int advance, cudaGraphConditionalHandle h, int graph, cudaStream_t st);
void launch_level_start(const TreeDev &T, const LevelBufs &L, const LevelHints &H, int sms,
                        cudaGraphConditionalHandle hratio, int graph, cudaStream_t st);
void launch_level_zero(const TreeDev &T, const LevelBufs &L, const LevelHints &H, int sms, cudaStream_t st);
void launch_ratio_pass(const TreeDev &T, const LevelBufs &L, const LevelHints &H, int sms,
                       cudaGraphConditionalHandle hratio, int graph, cudaStream_t st);
void launch_level_finish(const TreeDev &T, const LevelBufs &L, const LevelHints &H, int sms,
                         cudaGraphConditionalHandle hlevel, int graph, cudaStream_t st);
// The warp builders: cells of <= kTinyCap particles, then the rest up to kSmallCap.
void launch_small(const TreeDev &T, const LevelBufs &L, long long nsmall_hint, long long ntiny_hint, int sms,
                  cudaStream_t st);
int scan_tile_count(long long n);
size_t small_smem_bytes(int hist_cells, int cap);
// Small read-backs into mapped pinned host memory (see Readback).
void launch_readback(const Counters *ctr, const NodeWalk *walk0, Readback *out, cudaStream_t st);
void launch_readback_total(const long long *total, Readback *out, cudaStream_t st);
cudaError_t build_init_attributes();

}  // namespace bt
