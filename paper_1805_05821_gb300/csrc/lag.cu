// Instantiations and launcher of the lagged first pass of the two-pass push (lag.cuh).
#include "lag.cuh"
#include "lag_ws.cuh"
#include "lag_fused.cuh"

namespace foa {

template <typename S, int NC, bool FIN>
static cudaError_t launch_lag_one(const PassArgs &a, int grid, cudaStream_t s) {
  auto k = lag_kernel<S, NC, FIN>;
  static bool configured = false;  // per instantiation; the smem limit is the opt-in maximum
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<grid, kThreads, a.smem_total, s>>>(a);
  return cudaGetLastError();
}

template <typename S, int NC>
static cudaError_t launch_lag_ws_one(const PassArgs &a, int grid, cudaStream_t s) {
  auto k = lag_ws_kernel<S, NC>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<grid, kThreads, a.smem_total, s>>>(a);
  return cudaGetLastError();
}

template <typename S, int FC>
static cudaError_t launch_lag_fused_one(const PassArgs &a, int grid, cudaStream_t s) {
  auto k = lag_fused_kernel<S, FC>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<grid, kConsumers, a.smem_total, s>>>(a);  // no producer warp
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_lag_t(int mode, int nc, const PassArgs &a, int grid, cudaStream_t s) {
  if (mode == PASS_FIN) return launch_lag_one<S, 8, true>(a, grid, s);
  if constexpr (sizeof(typename Compute<S>::T) == 4) {
    // FP32/BF16: stages of one or two tiles held in registers, else the warp-specialised kernel
    // (row and column sweeps on different warps)
    const int fc = fused_columns(a);
    if (fc == 16) return launch_lag_fused_one<S, 16>(a, grid, s);
    if (fc == 24) return launch_lag_fused_one<S, 24>(a, grid, s);
    if (fc == 32) return launch_lag_fused_one<S, 32>(a, grid, s);
    switch (nc) {
      case 8: return launch_lag_ws_one<S, 8>(a, grid, s);
      case 16: return launch_lag_ws_one<S, 16>(a, grid, s);
      case 32: return launch_lag_ws_one<S, 32>(a, grid, s);
      case 48: return launch_lag_ws_one<S, 48>(a, grid, s);
      default: return launch_lag_ws_one<S, 64>(a, grid, s);
    }
  }
  switch (nc) {
    case 8: return launch_lag_one<S, 8, false>(a, grid, s);
    case 16: return launch_lag_one<S, 16, false>(a, grid, s);
    case 32: return launch_lag_one<S, 32, false>(a, grid, s);
    case 48: return launch_lag_one<S, 48, false>(a, grid, s);
    default: return launch_lag_one<S, 64, false>(a, grid, s);
  }
}

cudaError_t launch_lag(int dtype, int mode, int nc, const PassArgs &a, int grid, cudaStream_t s) {
  switch (dtype) {
    case FOA_DMD_F64: return launch_lag_t<double>(mode, nc, a, grid, s);
    case FOA_DMD_F32: return launch_lag_t<float>(mode, nc, a, grid, s);
    default: return launch_lag_t<__nv_bfloat16>(mode, nc, a, grid, s);
  }
}

}  // namespace foa
