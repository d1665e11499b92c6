// Small kernels around the streaming passes: the beta_pre column of Alg. 1, the
// append of the new basis vector v_{j+1} = w / h_{j+1,j} and the gather of basis columns to a dense layout.
#include "internal.cuh"
#include "push_kernels.cuh"

namespace foa {

cudaError_t launch_pass_f64(int mode, int nc, const PassArgs &a, int grid, cudaStream_t s);
cudaError_t launch_pass_f32(int mode, int nc, const PassArgs &a, int grid, cudaStream_t s);
cudaError_t launch_pass_bf16(int mode, int nc, const PassArgs &a, int grid, cudaStream_t s);
cudaError_t launch_lag(int dtype, int mode, int nc, const PassArgs &a, int grid, cudaStream_t s);

cudaError_t launch_pass(int dtype, int mode, int nc, const PassArgs &a, int grid, cudaStream_t s) {
  if (mode == PASS_A2 || mode == PASS_FIN) return launch_lag(dtype, mode, nc, a, grid, s);
  switch (dtype) {
    case FOA_DMD_F64: return launch_pass_f64(mode, nc, a, grid, s);
    case FOA_DMD_F32: return launch_pass_f32(mode, nc, a, grid, s);
    default: return launch_pass_bf16(mode, nc, a, grid, s);
  }
}

int pass_nc_for(int jcap) {
  const int need = (jcap + kWarps - 1) / kWarps;
  return need <= 8 ? 8 : need <= 16 ? 16 : need <= 32 ? 32 : need <= 48 ? 48 : 64;
}

// Decide whether the push proceeds and compute beta_pre (Alg. 1):
//   beta_pre_1 = sum_{l=1}^{j-1} h_{1,l} beta_{l,j},  beta_pre_i = sum_{l=i-1}^{j-1} h_{i,l} beta_{l,j}
// One warp per entry i; lanes split l, FP64 warp reduction.
__global__ void prep_kernel(DevState *st, const double *H, const double *B, double *pre, int kmax, int first,
                            int batch, foa_dmd_push_info *info_out) {
  const int q = st->q;
  const int stopped = st->stopped || (batch && st->halt);
  const bool full = q >= kmax;
  const bool mismatch = first ? (q != 0) : (q == 0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->pushes += 1;
    int status = -1;
    if (stopped) status = FOA_DMD_ESTOPPED;
    else if (full) status = FOA_DMD_EFULL;
    else if (mismatch) status = FOA_DMD_EINVAL;
    if (status >= 0) {
      st->active = 0;
      st->status = status;
      foa_dmd_push_info inf;
      inf.h_last = __longlong_as_double(0x7ff8000000000000ll);
      inf.indicator = inf.h_last;
      inf.x_norm = inf.h_last;
      inf.q = q;
      inf.status = status;
      st->info = inf;
      if (info_out) *info_out = inf;
    } else {
      st->active = 1;
      st->j = q;
      st->status = -1;
      if (q > 0) {
        const double bjj = B[int64_t(q - 1) * (kmax + 1)];
        st->bjj = bjj;
        st->inv_bjj = 1.0 / bjj;
      }
    }
  }
  if (stopped || full || mismatch || first) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= q) return;
  const int l0 = i == 0 ? 0 : i - 1;
  double acc = 0.0;
  for (int l = l0 + lane; l <= q - 2; l += 32) acc += H[i + int64_t(l) * kmax] * B[l + int64_t(q - 1) * kmax];
  acc = warp_sum(acc);
  if (lane == 0) pre[i] = acc;
}

// v_{j+1} = w / h_{j+1,j} (or v_1 = x / beta_11 on the first push), stored in the row-tiled V.
template <typename S, typename Src>
__global__ void colwrite_kernel(S *V, const Src *src, DevState *st, int64_t n, int64_t nrows, int kmax) {
  if (!st->active || st->status != FOA_DMD_OK) return;
  using C = typename Compute<S>::T;
  const int col = st->j;
  const C scale = static_cast<C>(st->inv_nu);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < nrows; r += stride) {
    const C v = (r < n) ? static_cast<C>(to_c(src[r])) : C(0);
    V[((r >> 5) * kmax + col) * kTile + (r & 31)] = Store<S>::from(v * scale);
  }
}

template <typename S>
__global__ void gather_kernel(const S *V, S *dst, int64_t ld, int64_t n, int kmax, int col0, int ncols) {
  const int64_t total = n * ncols;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t r = e % n;
    const int c = int(e / n);
    dst[r + int64_t(c) * ld] = V[((r >> 5) * kmax + col0 + c) * kTile + (r & 31)];
  }
}

template <typename S>
__global__ void scatter_kernel(S *V, const S *src, int64_t ld, int64_t n, int kmax, int col0, int ncols) {
  const int64_t total = n * ncols;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t r = e % n;
    const int c = int(e / n);
    V[((r >> 5) * kmax + col0 + c) * kTile + (r & 31)] = src[r + int64_t(c) * ld];
  }
}

static int grid_for(int64_t work, int threads, int sms) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = int64_t(sms) * 8;
  if (g > cap) g = cap;
  return int(g < 1 ? 1 : g);
}

cudaError_t launch_prep(DevState *st, const double *H, const double *B, double *pre, int kmax, int first,
                        int jcap, cudaStream_t s, int batch, foa_dmd_push_info *info_out) {
  const int grid = first ? 1 : (jcap + 7) / 8;
  prep_kernel<<<grid, 256, 0, s>>>(st, H, B, pre, kmax, first, batch, info_out);
  return cudaGetLastError();
}

cudaError_t launch_colwrite(int dtype, void *V, const void *src, bool from_x, DevState *st, int64_t n,
                            int64_t nrows, int kmax, int sms, cudaStream_t s) {
  const int grid = grid_for(nrows, 256, sms);
  switch (dtype) {
    case FOA_DMD_F64:
      colwrite_kernel<double, double><<<grid, 256, 0, s>>>(static_cast<double *>(V), static_cast<const double *>(src),
                                                            st, from_x ? n : nrows, nrows, kmax);
      break;
    case FOA_DMD_F32:
      if (from_x)
        colwrite_kernel<float, float><<<grid, 256, 0, s>>>(static_cast<float *>(V), static_cast<const float *>(src),
                                                            st, n, nrows, kmax);
      else
        colwrite_kernel<float, float><<<grid, 256, 0, s>>>(static_cast<float *>(V), static_cast<const float *>(src),
                                                            st, nrows, nrows, kmax);
      break;
    default:
      if (from_x)
        colwrite_kernel<__nv_bfloat16, __nv_bfloat16><<<grid, 256, 0, s>>>(
            static_cast<__nv_bfloat16 *>(V), static_cast<const __nv_bfloat16 *>(src), st, n, nrows, kmax);
      else
        colwrite_kernel<__nv_bfloat16, float><<<grid, 256, 0, s>>>(static_cast<__nv_bfloat16 *>(V),
                                                                   static_cast<const float *>(src), st, nrows,
                                                                   nrows, kmax);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather(int dtype, const void *V, void *dst, int64_t ld, int64_t n, int kmax, int col0, int ncols,
                          int sms, cudaStream_t s) {
  const int grid = grid_for(n * ncols, 256, sms);
  switch (dtype) {
    case FOA_DMD_F64:
      gather_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double *>(V), static_cast<double *>(dst), ld, n,
                                                 kmax, col0, ncols);
      break;
    case FOA_DMD_F32:
      gather_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(V), static_cast<float *>(dst), ld, n,
                                                kmax, col0, ncols);
      break;
    default:
      gather_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(V),
                                                        static_cast<__nv_bfloat16 *>(dst), ld, n, kmax, col0, ncols);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_scatter(int dtype, void *V, const void *src, int64_t ld, int64_t n, int kmax, int col0, int ncols,
                           int sms, cudaStream_t s) {
  const int grid = grid_for(n * ncols, 256, sms);
  switch (dtype) {
    case FOA_DMD_F64:
      scatter_kernel<double><<<grid, 256, 0, s>>>(static_cast<double *>(V), static_cast<const double *>(src), ld, n,
                                                  kmax, col0, ncols);
      break;
    case FOA_DMD_F32:
      scatter_kernel<float><<<grid, 256, 0, s>>>(static_cast<float *>(V), static_cast<const float *>(src), ld, n,
                                                 kmax, col0, ncols);
      break;
    default:
      scatter_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<__nv_bfloat16 *>(V),
                                                         static_cast<const __nv_bfloat16 *>(src), ld, n, kmax, col0,
                                                         ncols);
      break;
  }
  return cudaGetLastError();
}

}  // namespace foa
