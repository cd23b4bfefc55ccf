// bt_build.cuh -- launchers of the BuildTree kernels (bt_build.cu).
#pragma once
#include "bt_internal.cuh"

namespace bt {

void launch_init_sets(const TreeDev &T, const SetRec *rec, int *set_start, int *set_s, int *set_na,
                      double *set_beta, int *set_gmax, cudaStream_t st);
void launch_bbox(const TreeDev &T, const float *x, const float *y, const float *z, const float *h,
                 int sms, cudaStream_t st);
void launch_root_sets(const TreeDev &T, int *big_ids, SmallItem *small, cudaStream_t st);
void launch_copy_leaf_roots(const TreeDev &T, const float *x, const float *y, const float *z,
                            const float *h, int sms, cudaStream_t st);
void launch_big_setup(const TreeDev &T, BigCell *big, const int *ids, int nb, cudaStream_t st);
void launch_big_hist(const TreeDev &T, const BigCell *big, int nb, int chunks, Src src, int *hist,
                     int sms, cudaStream_t st);
void launch_big_ratio(const TreeDev &T, BigCell *big, int nb, const int *hist, int hist_total, int sms,
                      cudaStream_t st);
void launch_big_zero(const BigCell *big, int nb, int *hist, int hist_total, int sms, cudaStream_t st);
void launch_big_finish(const TreeDev &T, BigCell *big, int nb, int slot_level_base, cudaStream_t st);
void launch_scan(const int *in, int n, int *tile_buf, int *out, cudaStream_t st);
int scan_tile_count(int n);
void launch_big_emit(const TreeDev &T, const BigCell *big, int nb, int hist_total, const int *hist,
                     const int *hoff, int *cursor, int dst_buf, int *next_big, SmallItem *small,
                     int sms, cudaStream_t st);
void launch_big_scatter(const TreeDev &T, const BigCell *big, int nb, int chunks, Src src,
                        int *cursor, float4 *dst_pos, float *dst_h, int sms, cudaStream_t st);
void launch_small(const TreeDev &T, const SmallItem *items, int nitems, Src src0, Src src1,
                  Src srcin, int sms, cudaStream_t st);
void launch_init_counters(Counters *ctr, cudaStream_t st);
void launch_set_int(int *p, int v, cudaStream_t st);
size_t small_smem_bytes();
cudaError_t build_init_attributes();

}  // namespace bt
