// Instantiations of the streaming-pass kernel for __nv_bfloat16 storage.
#include "pass.cuh"
#include "pass_ws.cuh"
#include "pass_fused.cuh"

namespace foa {

template <int MODE, int NC>
static cudaError_t launch_one(const PassArgs &a, int grid, cudaStream_t s) {
  auto k = pass_kernel<__nv_bfloat16, MODE, NC>;
  static bool configured = false;  // per instantiation; the smem limit is the opt-in maximum
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<grid, kThreads, a.smem_total, s>>>(a);
  return cudaGetLastError();
}

// passes with column dots: the warp-specialised kernel
template <int MODE, int NC>
static cudaError_t launch_ws_one(const PassArgs &a, int grid, cudaStream_t s) {
  auto k = pass_ws_kernel<__nv_bfloat16, MODE, NC>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<grid, kThreads, a.smem_total, s>>>(a);
  return cudaGetLastError();
}

// wide-basis stages (one or two tiles) held in registers: pass_fused_kernel
template <int MODE, int FC>
static cudaError_t launch_fused_one(const PassArgs &a, int grid, cudaStream_t s) {
  auto k = pass_fused_kernel<__nv_bfloat16, MODE, FC>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<grid, kConsumers, a.smem_total, s>>>(a);  // no producer warp
  return cudaGetLastError();
}

// passes with column dots (A, B, B2): the register-held kernel where its column groups fit,
// else the warp-specialised one
template <int MODE>
static cudaError_t launch_dots(int nc, const PassArgs &a, int grid, cudaStream_t s) {
  const int fc = fused_columns(a);
  if (fc == 16) return launch_fused_one<MODE, 16>(a, grid, s);
  if (fc == 24) return launch_fused_one<MODE, 24>(a, grid, s);
  if (fc == 32) return launch_fused_one<MODE, 32>(a, grid, s);
  switch (nc) {
    case 8: return launch_ws_one<MODE, 8>(a, grid, s);
    case 16: return launch_ws_one<MODE, 16>(a, grid, s);
    case 32: return launch_ws_one<MODE, 32>(a, grid, s);
    case 48: return launch_ws_one<MODE, 48>(a, grid, s);
    default: return launch_ws_one<MODE, 64>(a, grid, s);
  }
}

cudaError_t launch_pass_bf16(int mode, int nc, const PassArgs &a, int grid, cudaStream_t s) {
  switch (mode) {
    case PASS_A: return launch_dots<PASS_A>(nc, a, grid, s);
    case PASS_B: return launch_dots<PASS_B>(nc, a, grid, s);
    case PASS_B2: return launch_dots<PASS_B2>(nc, a, grid, s);
    case PASS_C: return launch_one<PASS_C, 8>(a, grid, s);
    default: return launch_one<PASS_FIRST, 8>(a, grid, s);
  }
}

}  // namespace foa
