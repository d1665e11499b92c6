// Block push: shared declarations of the block passes over V (block_pass.cuh, instantiated in
// block_pass_f32.cu / block_pass_bf16.cu) and of the Cholesky QR kernels and host loop (block.cu).
#pragma once
#include <cmath>

#include "api_internal.cuh"

namespace foa {
namespace blk {

enum BlockMode : int { BLK_A = 0, BLK_B = 1, BLK_C = 2 };
constexpr int kMaxP = 4;
// A block column whose new direction R_ii is below kBlockResolveUnits * u_s * ||psi|| is not
// pushed by the block form (FOA_DMD_ERESOLVE): block CGS2 in the storage precision no longer keeps
// such columns orthogonal to V (measured: orthogonality lost about 100 columns after R_ii reached
// 7 u_fp32 ||psi|| on noise-floor snapshots).
constexpr double kBlockResolveUnits = 16.0;
__host__ __device__ inline double unit_roundoff(int dtype) {
  return dtype == FOA_DMD_F64 ? 0x1p-53 : dtype == FOA_DMD_F32 ? 0x1p-24 : 0x1p-8;
}

struct BlockState {
  int32_t j;        // basis size before the block
  int32_t pb;       // snapshots in the block
  int32_t m1;       // leading columns factored by the first Cholesky step
  int32_t ncommit;  // columns committed by the block
  int32_t status;
  int32_t err;
  uint32_t ticket[8];
  double xnorm[kMaxP];
  double R1[kMaxP * kMaxP], R2[kMaxP * kMaxP], R[kMaxP * kMaxP];
  double G[kMaxP * kMaxP];
};

struct BlockArgs {
  const void *V;
  const void *X;        // caller's block: snapshot k at X + k*ldx (storage dtype)
  int64_t ldx;
  float *W;             // P working vectors, each nrows floats
  double *W64;          // W R1^-1 in FP64 (P x nrows): Cholesky QR keeps FP64 past the Gram matrix
  double *C1, *C;       // j x P coefficients (column k at k*kmax)
  double *partials, *gpart;
  uint32_t *gcount;
  BlockState *bs;
  DevState *st;
  double *H, *B;
  int64_t n, nrows;
  int32_t ntiles, kmax, j, slots, x_aligned;
  int32_t slot_bytes, base_off, base_stride, off_ws, off_coef, off_dot, off_comb, off_red, off_bar, smem_total;
  double tol;
  double resolve;       // kBlockResolveUnits * u_s
};

// four consecutive rows of one column (16-byte aligned FP32, 8-byte aligned BF16) as floats
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

// upper Cholesky of the leading block of a P x P matrix (column-major, leading dimension kMaxP);
// returns the columns factored (the first failing pivot, or p)
__device__ inline int chol_up(int p, const double *G, double *R) {
  for (int i = 0; i < kMaxP * kMaxP; ++i) R[i] = 0.0;
  for (int i = 0; i < p; ++i) {
    double d = G[i + i * kMaxP];
    for (int k = 0; k < i; ++k) d -= R[k + i * kMaxP] * R[k + i * kMaxP];
    if (!(d > 0.0)) return i;
    const double rii = sqrt(d);
    R[i + i * kMaxP] = rii;
    for (int c = i + 1; c < p; ++c) {
      double t = G[i + c * kMaxP];
      for (int k = 0; k < i; ++k) t -= R[k + i * kMaxP] * R[k + c * kMaxP];
      R[i + c * kMaxP] = t / rii;
    }
  }
  return p;
}

// Cross-CTA reduction of len doubles over the T threads of each CTA (deterministic: CTA order
// within groups of 8, then group order); returns true in the last CTA, with the sums in dot[0..len).
template <int T>
__device__ bool block_reduce(const BlockArgs &a, double *dot, int len, int mode, volatile int *sflag, int tid) {
  double *mypart = a.partials + size_t(blockIdx.x) * len;
  for (int c = tid; c < len; c += T) mypart[c] = dot[c];
  __threadfence();
  named_bar_sync(1, T);
  const int ngroups = (gridDim.x + kGroup - 1) / kGroup;
  const int grp = blockIdx.x / kGroup;
  const int gfirst = grp * kGroup;
  const int gsize = min(kGroup, int(gridDim.x) - gfirst);
  if (tid == 0) {
    const unsigned t = atomicAdd(&a.gcount[grp], 1u);
    sflag[2] = (t == unsigned(gsize - 1)) ? 1 : 0;
  }
  named_bar_sync(1, T);
  if (!sflag[2]) return false;
  __threadfence();
  double *gp = a.gpart + size_t(grp) * len;
  for (int c = tid; c < len; c += T) {
    double t = 0.0;
    for (int b = 0; b < gsize; ++b) t += __ldcg(a.partials + size_t(gfirst + b) * len + c);
    gp[c] = t;
  }
  __threadfence();
  named_bar_sync(1, T);
  if (tid == 0) {
    a.gcount[grp] = 0u;
    const unsigned t = atomicAdd(&a.bs->ticket[mode], 1u);
    sflag[2] = (t == unsigned(ngroups - 1)) ? 1 : 0;
  }
  named_bar_sync(1, T);
  if (!sflag[2]) return false;
  __threadfence();
  for (int c = tid; c < len; c += T) {
    double t = 0.0;
    for (int g = 0; g < ngroups; ++g) t += __ldcg(a.gpart + size_t(g) * len + c);
    dot[c] = t;
  }
  if (tid == 0) a.bs->ticket[mode] = 0u;
  named_bar_sync(1, T);
  return true;
}

// Shape of a block pass at basis size j: T threads a CTA (256: two CTAs per SM, basis up to 256
// columns; 512: one CTA per SM, up to 512) and fc columns per thread (a kernel instance: 2, 4, 6
// or 8 for T = 256, 6 or 8 for T = 512; fc * P a multiple of 8).
inline void block_pass_shape(int j, int P, int &T, int &fc) {
  T = j <= 256 ? 256 : 512;
  const int G1 = T / 8;
  const int nc = (j + G1 - 1) / G1;
  fc = nc <= 2 ? 2 : nc <= 4 ? 4 : nc <= 6 ? 6 : 8;
  if (P == 2 && fc == 6) fc = 8;
  if (fc * P < 8) fc = 8 / P;
}

// launchers of the block passes (one per storage type)
cudaError_t launch_block_pass_f32(int mode, int T, int fc, int P, const BlockArgs &a, int grid, cudaStream_t s);
cudaError_t launch_block_pass_bf16(int mode, int T, int fc, int P, const BlockArgs &a, int grid, cudaStream_t s);

}  // namespace blk
}  // namespace foa
