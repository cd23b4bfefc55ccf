// bt_find.cuh -- launchers of the FindNeighbors and density kernels (bt_find.cu).
#pragma once
#include "bt_internal.cuh"

namespace bt {

cudaError_t launch_find(const TreeDev &T, int ngroups, int ngroups_c, int ngmax, int32_t *nbrs,
                        int32_t *counts, const float *m, float *smass, float *rho, int sms,
                        cudaStream_t st);
cudaError_t launch_density(const TreeDev &T, const float *m, const int32_t *nbrs,
                           const int32_t *counts, int ngmax, float *rho, int sms, cudaStream_t st);
cudaError_t launch_find_density_noalloc(const TreeDev &T, int ngroups, int ngroups_c, int ngmax,
                                        int32_t *nbrs, int32_t *counts, const float *m, float *rho,
                                        int sms, cudaStream_t st);
long long noalloc_max_particles();
// Compressed rows: the counting pass (density fused when rho != null) and the
// exclusive scan into offsets [n + 1]; then the row-writing pass.  scratch:
// csr_scratch_elems(n) int64.
long long csr_scratch_elems(long long n);
cudaError_t launch_find_csr_count(const TreeDev &T, int ngroups, int ngroups_c, int32_t *counts,
                                  const float *m, float *smass, float *rho, long long *offsets,
                                  long long *scratch, int half, int sms, cudaStream_t st);
// Exclusive scan of min(counts, cap) into offsets [n + 1]; pack fixed rows
// into compressed rows.
void launch_scan64(const int32_t *counts, long long n, int cap, long long *offsets, long long *scratch,
                   cudaStream_t st);
void launch_pack_rows(const int32_t *rows, const int32_t *counts, long long n, int ngmax,
                      const long long *offsets, int32_t *csr, int sms, cudaStream_t st);
cudaError_t launch_find_csr_rows(const TreeDev &T, int ngroups, int ngroups_c, const long long *offsets,
                                 int32_t *nbrs, int32_t *counts, int half, int sms, cudaStream_t st);
size_t find_smem_bytes();
cudaError_t find_init_attributes();

}  // namespace bt
