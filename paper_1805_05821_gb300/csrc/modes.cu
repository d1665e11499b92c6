// DMD modes Phi_i = V_{1:m} U_r z_i (Alg. 1): Phi = V Y with Y = [Re y_0, Im y_0, ...]
// (m x ncols, FP64).  SIMT form: each CTA stages 32-row tiles of the row-tiled V in shared
// memory and every thread accumulates ncols/8 outputs of one row.
#include <cstdlib>

#include "api_internal.cuh"
#include "eig_internal.cuh"

namespace foa {

template <typename S>
__global__ void __launch_bounds__(256) modes_simt_kernel(const S *V, int kmax, int64_t n, int ntiles, int m,
                                                         const double *Y, int ldy, int ncols,
                                                         typename Compute<S>::T *phi, int64_t ldp) {
  using C = typename Compute<S>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  C *ys = reinterpret_cast<C *>(smem);                                  // m x ncols (row k: ncols values)
  S *vt = reinterpret_cast<S *>(smem + ((size_t(m) * ncols * sizeof(C) + 15) / 16) * 16);  // 32 x m
  for (int t = threadIdx.x; t < m * ncols; t += blockDim.x) {
    const int k = t / ncols, c = t % ncols;
    ys[t] = static_cast<C>(Y[k + int64_t(c) * ldy]);
  }
  const int row = threadIdx.x & 31, grp = threadIdx.x >> 5;  // 8 column groups
  const int cpg = (ncols + 7) / 8;
  const int c0 = grp * cpg, c1 = min(ncols, c0 + cpg);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    const S *src = V + int64_t(tile) * kmax * kTile;
    for (int t = threadIdx.x; t < m * kTile; t += blockDim.x) vt[t] = src[t];
    __syncthreads();
    C acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = C(0);
    for (int k = 0; k < m; ++k) {
      const C v = to_c(vt[k * kTile + row]);
      const C *yk = ys + k * ncols;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (c0 + i < c1) acc[i] += v * yk[c0 + i];
    }
    const int64_t r = int64_t(tile) * kTile + row;
    if (r < n) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (c0 + i < c1) phi[r + int64_t(c0 + i) * ldp] = acc[i];
    }
  }
}

int launch_modes_tc(foa_dmd *h, int m, const double *Y, int ldy, int ncols, float *phi, int64_t ld_phi, float *Bop,
                    int *err);

int launch_modes(foa_dmd *h, int m, const double *Y, int ldy, int ncols, void *phi, int64_t ld_phi) {
  if (ncols > 64) return FOA_DMD_EINVAL;
  // FP32 storage: tensor cores (tcgen05, kind::tf32 with a three-term split).  FOA_DMD_MODES_SIMT=1
  // selects the SIMT kernel instead (used by the tests as an independent cross-check).
  const char *simt = getenv("FOA_DMD_MODES_SIMT");
  if (h->dtype == FOA_DMD_F32 && !(simt && simt[0] == '1'))
    return launch_modes_tc(h, m, Y, ldy, ncols, static_cast<float *>(phi), ld_phi, h->eig->bop, h->eig->isc + ISC_ERR);
  const int cs = compute_size(h->dtype), s = dtype_size(h->dtype);
  // A CTA keeps the m x nc block of Y and one 32 x m tile of V in shared memory.  When all ncols
  // columns of Y do not fit (FP64 storage past m = 280 at 64 columns), the columns are split
  // into launches of nc columns each (a multiple of 8), and V is read once per launch.
  constexpr size_t kSmemMax = 232448;
  const size_t vbytes = size_t(kTile) * m * s;
  auto smem_for = [&](int nc) { return ((size_t(m) * nc * cs + 15) / 16) * 16 + vbytes; };
  int nc_max = ncols;
  while (nc_max > 8 && smem_for(nc_max) > kSmemMax) nc_max = (nc_max - 1) / 8 * 8;
  if (smem_for(nc_max) > kSmemMax) return FOA_DMD_EINVAL;
  const int grid = h->ntiles < h->sms * 2 ? h->ntiles : h->sms * 2;
  const int64_t es = cs;  // phi holds the compute type (FP64 for FP64 storage, FP32 otherwise)
  cudaError_t e = cudaSuccess;
  for (int c0 = 0; c0 < ncols && e == cudaSuccess; c0 += nc_max) {
    const int nc = ncols - c0 < nc_max ? ncols - c0 : nc_max;
    const size_t smem = smem_for(nc);
    const double *Yc = Y + int64_t(c0) * ldy;
    void *pc = static_cast<unsigned char *>(phi) + int64_t(c0) * ld_phi * es;
    switch (h->dtype) {
      case FOA_DMD_F64:
        e = cudaFuncSetAttribute(modes_simt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e == cudaSuccess)
          modes_simt_kernel<double><<<grid, 256, smem, h->stream>>>(static_cast<const double *>(h->V), h->kmax, h->n,
                                                                    h->ntiles, m, Yc, ldy, nc, static_cast<double *>(pc),
                                                                    ld_phi);
        break;
      case FOA_DMD_F32:
        e = cudaFuncSetAttribute(modes_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e == cudaSuccess)
          modes_simt_kernel<float><<<grid, 256, smem, h->stream>>>(static_cast<const float *>(h->V), h->kmax, h->n,
                                                                   h->ntiles, m, Yc, ldy, nc, static_cast<float *>(pc),
                                                                   ld_phi);
        break;
      default:
        e = cudaFuncSetAttribute(modes_simt_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem));
        if (e == cudaSuccess)
          modes_simt_kernel<__nv_bfloat16><<<grid, 256, smem, h->stream>>>(
              static_cast<const __nv_bfloat16 *>(h->V), h->kmax, h->n, h->ntiles, m, Yc, ldy, nc,
              static_cast<float *>(pc), ld_phi);
        break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (c0 > 0) h->launches += 1;
  }
  return cuda_status(e);
}

}  // namespace foa
