// Host-side launchers of the sm_103a kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace selinv {

// counts kernel launches issued by the library (reported by selinv_launch_count)
void note_launch(int n = 1);

cudaError_t configure_selinv_kernels();
// large = 1 for supernodes with s > 32 (128 KB of shared memory), 0 otherwise
cudaError_t launch_linv(int dtype, const ProbDesc *d, const int2 *work, int nwork, int large, cudaStream_t st,
                        int with_dinv = 1);
cudaError_t launch_dinv(int dtype, const ProbDesc *d, const int2 *work, int nwork, cudaStream_t st);
cudaError_t launch_lhat(int dtype, int bucket, const ProbDesc *d, const Item *items, int n,
                        cudaStream_t st);
cudaError_t launch_selinv(int dtype, int bucket, const ProbDesc *d, const Item *items, int n,
                          cudaStream_t st);
cudaError_t configure_ozaki_kernels();
cudaError_t configure_tc_kernels();
cudaError_t launch_selinv_tc(int tn, const ProbDesc *d, const Item *items, int n, long long *slab,
                             long long wait_limit, cudaStream_t st);
cudaError_t launch_tc_reduce(int tn, const ProbDesc *d, const Item *items, const int4 *red, int n,
                             const long long *slab, cudaStream_t st);
cudaError_t configure_tcw_kernels();
cudaError_t launch_selinv_tcw(int cplx, const ProbDesc *d, const Item *items, int n, long long *slab,
                              long long wait_limit, cudaStream_t st);
cudaError_t launch_lhat_tcw(const ProbDesc *d, const Item *items, int n, long long wait_limit, cudaStream_t st);
cudaError_t launch_syrk_tcw(const ProbDesc *d, const Item *items, int n, long long wait_limit, cudaStream_t st);
cudaError_t launch_tcw_reduce(int cplx, const ProbDesc *d, const Item *items, const int4 *red, int n,
                              const long long *slab, cudaStream_t st);
cudaError_t launch_diag_fin(const ProbDesc *d, const Item *items, int n, cudaStream_t st);
cudaError_t launch_diag_tc(int tn, int cplx, const ProbDesc *d, const Item *items, int n, long long wait_limit,
                           cudaStream_t st);
cudaError_t launch_lhat_digits_z(const ProbDesc *d, const int2 *work, int nwork, cudaStream_t st);
cudaError_t launch_diag_fin_z(const ProbDesc *d, const Item *items, int n, cudaStream_t st);
cudaError_t launch_check_finite(const void *x, int64_t n_doubles, int *status, cudaStream_t st);
cudaError_t launch_selinv_persist(int dtype, const ProbDesc *d, const Item *items, const int8_t *buckets,
                                  int n, int *ticket, long long spin_limit, int wait_on_unset,
                                  cudaStream_t st);
cudaError_t launch_linv_digits(const ProbDesc *d, const int2 *work, int nwork, cudaStream_t st);
cudaError_t launch_lhat_oz(int tn, const ProbDesc *d, const Item *items, int n, cudaStream_t st);
cudaError_t launch_selinv_tiny(int dtype, const ProbDesc *d, const Item *items, int n, cudaStream_t st);
cudaError_t launch_push(int dtype, int kind, int bucket, const ProbDesc *d, const Item *items, int n,
                        cudaStream_t st);
cudaError_t launch_lhat_digits(const ProbDesc *d, const int2 *work, int nwork, cudaStream_t st);
cudaError_t launch_diag_oz(const ProbDesc *d, const Item *items, int n, cudaStream_t st);
cudaError_t launch_selinv_oz(int tn, const ProbDesc *d, const Item *items, int n, cudaStream_t st);

}  // namespace selinv
