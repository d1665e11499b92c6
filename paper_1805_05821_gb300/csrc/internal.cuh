// Internal declarations of the GB300 FOA-DMD library: device state, launch parameters and the
// inline-PTX helpers (mbarrier, bulk async copy) shared by the kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "foa_dmd.h"

namespace foa {

constexpr int kTile = 32;          // rows per tile of the row-tiled V layout
constexpr int kWarps = 8;          // consumer warps of a streaming-pass CTA
constexpr int kConsumers = kWarps * 32;
constexpr int kThreads = kConsumers + 32;  // + one producer warp that issues the bulk copies
constexpr int kMaxK = 512;         // largest k_max
constexpr int kGroup = 8;          // CTAs per first-level group of the cross-CTA reduction
constexpr int kMaxR = 64;          // largest number of tiles in one pipeline stage
constexpr int kMaxSlots = 8;

// pass kinds (PASS_B2, PASS_A2 and PASS_FIN are the two-pass push: see lag.cuh)
enum PassMode : int { PASS_A = 0, PASS_B = 1, PASS_C = 2, PASS_FIRST = 3, PASS_B2 = 4, PASS_A2 = 5, PASS_FIN = 6 };

// Device-resident state of one stream.  The host only knows an upper bound of q while pushes
// are in flight; every kernel reads the true values here, so a launch sequence stays correct
// (and capturable in a CUDA graph) whatever the outcome of earlier pushes.
struct DevState {
  int32_t q;         // committed basis size
  int32_t j;         // basis size of the push in progress (index of the column it appends)
  int32_t active;    // 1 while the push in progress proceeds
  int32_t stopped;   // a breakdown froze the stream
  int32_t status;    // foa_dmd_status of the most recent push
  int32_t err;       // sticky device error (bounded wait ran out)
  int32_t pushes;    // number of pushes issued (for the indicator schedule)
  int32_t halt;      // a failed push inside foa_dmd_push_batch skips the rest of the batch
  double inv_bjj;    // 1 / beta_{j,j}
  double bjj;        // beta_{j,j}
  double x_norm;     // ||x||_2 of the push in progress
  double nu;         // h_{j+1,j}
  double inv_nu;     // 1 / h_{j+1,j}
  int32_t pending;   // two-pass push: column pend_col is committed but not yet written to V
  int32_t pend_col;
  double pad1[2];
  uint32_t ticket[8];// per-pass arrival counters of the last reduction level
  foa_dmd_push_info info;  // result of the most recent push
};

// Per-launch parameters of a streaming pass over V.
struct PassArgs {
  const void *V;         // row-tiled storage: element (row r, col c) at ((r/32)*kmax + c)*32 + r%32
  const void *x;         // snapshot (PASS_A, PASS_FIRST), storage dtype, n elements
  void *w;               // working vector, compute dtype, ntiles*32 elements (zero beyond n)
  const double *coef;    // FP64 coefficients of the pass (beta_pre, h or s)
  const double *coef2;   // PASS_A2 / PASS_FIN: s of the pending column
  double *partials;      // [grid][kmax+1]
  double *gpart;         // [ngroups][kmax+1]
  uint32_t *gcount;      // [ngroups]
  DevState *st;
  double *H;             // H-bar, kmax x kmax column-major (ld = kmax)
  double *B;             // beta,  kmax x kmax column-major
  double *pre;           // beta_pre of the push in progress (j entries)
  double *hvec;          // h (after pass A), h + s (after pass B)
  double *svec;          // s (after pass B)
  foa_dmd_push_info *info_out;  // optional extra copy of the push result (device)
  int64_t n;
  int32_t ntiles;
  int32_t kmax;
  int32_t R;             // tiles per stage
  int32_t slots;         // pipeline depth
  int32_t nstages;       // ceil(ntiles / R)
  int32_t jcap;          // upper bound of j used to size shared memory
  int32_t reorth;
  int32_t x_aligned;     // x may be fetched with bulk copies
  int32_t batch;         // inside foa_dmd_push_batch: a failed push sets DevState::halt
  int32_t form;          // 1: QR view (PASS_A projects x itself; PASS_C commits [h; nu])
  double tol;            // breakdown tolerance
  // shared-memory layout (bytes)
  int32_t slot_bytes, base_off;   // within a slot: V tiles at 0, base vector at base_off
  int32_t off_ws, off_coef, off_dot, off_comb, off_norm, off_bar, smem_total;
  int32_t base2_off;     // PASS_A2 / PASS_FIN: w' slice within a slot
  int32_t off_vnew, off_coef2;
  int32_t variant;       // FP32/BF16 passes A, B, B2: 0 = stage in registers where it fits, 1 = shared memory
};

// ------------------------------------------------------------------------------------------
// inline PTX helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2^31 cycles (about a second at GB300 clocks).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}
// ------------------------------------------------------------------------------------------
// Self-checking build (compiled with -DFOA_DMD_CHECKED; build.build(checked=True)): every bulk
// copy checks its shared-memory destination against the CTA's shared window and the 16-byte
// alignment of both addresses and of the size, and the streaming producers check each tile index
// against the tile count.  A failed check sets a bit in this translation unit's check word
// (foa_dmd_check_status ORs the words of all units) and skips the access, so nothing faults: the
// pipeline that misses the copy ends in its bounded wait.  Without the macro the checks vanish.
// ------------------------------------------------------------------------------------------
enum CheckBits : unsigned { kChkSmem = 1u, kChkAlign = 2u, kChkTile = 4u };
#ifdef FOA_DMD_CHECKED
static __device__ unsigned foa_check_word;
__device__ __forceinline__ bool foa_check(bool ok, unsigned bit) {
  if (!ok) atomicOr(&foa_check_word, bit);
  return ok;
}
int foa_check_register(cudaError_t (*read_and_clear)(unsigned *));
static cudaError_t foa_check_read_unit(unsigned *out) {
  unsigned v = 0, z = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, foa_check_word, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(foa_check_word, &z, sizeof(z));
  *out |= v;
  return e;
}
static const int foa_check_registered_ = foa_check_register(&foa_check_read_unit);
#define FOA_CHECK(cond, bit) foa_check((cond), (bit))
#else
#define FOA_CHECK(cond, bit) true
#endif

// One-dimensional bulk copy global -> shared, completing on an mbarrier (transaction bytes).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
#ifdef FOA_DMD_CHECKED
  {
    uint32_t total;
    asm("mov.u32 %0, %%total_smem_size;" : "=r"(total));
    const uint32_t d = smem_addr(dst);
    if (!FOA_CHECK(((d | uint32_t(reinterpret_cast<uintptr_t>(src)) | bytes) & 15u) == 0 && bytes != 0 &&
                       (smem_addr(bar) & 7u) == 0,
                   kChkAlign))
      return;
    if (!FOA_CHECK(uint64_t(d) + bytes <= total, kChkSmem)) return;
  }
#endif
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// Named barrier that also ORs a predicate over the participating threads.
__device__ __forceinline__ int named_bar_or(int id, int count, int pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n barrier.cta.red.or.pred q, %2, %3, p;\n selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred), "r"(id), "r"(count)
      : "memory");
  return r;
}

// two adjacent rows of one column (8-byte or 4-byte aligned): FP32 values
__device__ __forceinline__ float2 ld_pair(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 ld_pair(const __nv_bfloat16 *p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}
__device__ __forceinline__ float2 ld_pair(const double *p) {
  return make_float2(float(p[0]), float(p[1]));  // not used on the FP64 path
}

// storage -> compute conversions
__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename S> struct Store;
template <> struct Store<double> { static __device__ __forceinline__ double from(double v) { return v; } };
template <> struct Store<float> { static __device__ __forceinline__ float from(float v) { return v; } };
template <> struct Store<__nv_bfloat16> {
  static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};
template <typename S> struct Compute { using T = float; };
template <> struct Compute<double> { using T = double; };

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

inline int dtype_size(int dt) { return dt == FOA_DMD_F64 ? 8 : dt == FOA_DMD_F32 ? 4 : 2; }
inline int compute_size(int dt) { return dt == FOA_DMD_F64 ? 8 : 4; }

// launchers (push kernels)
cudaError_t launch_pass(int dtype, int mode, int nc, const PassArgs &a, int grid, cudaStream_t s);
int pass_nc_for(int jcap);

}  // namespace foa
