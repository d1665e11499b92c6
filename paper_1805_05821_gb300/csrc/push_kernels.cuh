// Launchers of the small push kernels (prep, column write, gather/scatter of basis columns).
#pragma once
#include "internal.cuh"

namespace foa {

cudaError_t launch_prep(DevState *st, const double *H, const double *B, double *pre, int kmax, int first,
                        int jcap, cudaStream_t s, int batch = 0, foa_dmd_push_info *info_out = nullptr);
cudaError_t launch_colwrite(int dtype, void *V, const void *src, bool from_x, DevState *st, int64_t n,
                            int64_t nrows, int kmax, int sms, cudaStream_t s);
cudaError_t launch_gather(int dtype, const void *V, void *dst, int64_t ld, int64_t n, int kmax, int col0, int ncols,
                          int sms, cudaStream_t s);
cudaError_t launch_scatter(int dtype, void *V, const void *src, int64_t ld, int64_t n, int kmax, int col0, int ncols,
                           int sms, cudaStream_t s);

}  // namespace foa
