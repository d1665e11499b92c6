// Block push: P snapshots at once (the block form of the QR view of Sec. 3.1; the §8 block-push
// variant).  Per block X_b = [psi_{j+1} .. psi_{j+P}], with V the current basis (j columns):
//   BLK_A  (one pass over V)  C1 = V^T X_b and ||psi_k||^2
//   BLK_B  (one pass over V)  W = X_b - V C1,  C2 = V^T W,  C = C1 + C2
//   BLK_C  (one pass over V)  W = W - V C2,    G = W^T W, then G = R1^T R1 (Cholesky, FP64)
//   BLK_Q1 (rows of W only)   W1 = W R1^-1 (FP64), G2 = W1^T W1 = R2^T R2, R = R2 R1, breakdown test,
//                             beta block column [C; R], Hbar columns by forward substitution
//   BLK_Q2 (rows of W only)   Q = W1 R2^-1 -> V columns j .. j+P-1
// V is read three times per block instead of three times per snapshot.  The passes share the
// single-stream machinery: a producer warp streams row-tiled V and the P base slices into a
// shared-memory ring with bulk copies on mbarriers; eight consumer warps make the row sweep
// (thread <- row pair x column group, P outputs per row) and the column sweep (quarter-warps take
// four columns, a lane four rows, P products per column); FP32 products, per-CTA FP64 partials
// and a deterministic two-level cross-CTA reduction.  FP32/BF16 storage.  From the Gram matrix
// on, the Cholesky QR works in FP64 (exact products of the FP32 W, W R1^-1 and Q in FP64): stored
// in FP32, W R1^-1 would carry u_fp32 kappa(W)^2 and lose orthogonality once a block's directions
// span more than ~sqrt(1/u_fp32) in size.
#include <cmath>
#include <cstring>

#include "api_internal.cuh"
#include "push_kernels.cuh"

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
  int32_t ntiles, kmax, j, R, slots, nstages, x_aligned;
  int32_t slot_bytes, base_off, base_stride, off_ws, off_coef, off_dot, off_comb, off_red, off_bar, smem_total;
  double tol;
  double resolve;       // kBlockResolveUnits * u_s
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

// Eight consecutive stage rows of one column (or one base slice), 32-byte aligned: two 16-byte
// loads for FP32 (in the other order when swap, which keeps a wavefront's lanes on distinct
// banks), one for BF16.
__device__ __forceinline__ void ld8(const float *p, bool swap, float (&v)[8]) {
  const float4 f = *reinterpret_cast<const float4 *>(p + (swap ? 4 : 0));
  const float4 g = *reinterpret_cast<const float4 *>(p + (swap ? 0 : 4));
  const float4 lo = swap ? g : f, hi = swap ? f : g;
  v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
  v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
}
__device__ __forceinline__ void ld8(const __nv_bfloat16 *p, bool, float (&v)[8]) {
  const uint4 u = *reinterpret_cast<const uint4 *>(p);
  const uint32_t q[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q[i]));
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

// P consecutive floats (P = 2 or 4, 8- or 16-byte aligned) in one shared-memory access
template <int P>
__device__ __forceinline__ void ldp(const float *p, float (&v)[P]) {
  if constexpr (P == 4) {
    const float4 f = *reinterpret_cast<const float4 *>(p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  } else {
    const float2 f = *reinterpret_cast<const float2 *>(p);
    v[0] = f.x; v[1] = f.y;
  }
}
template <int P>
__device__ __forceinline__ void stp(float *p, const float (&v)[P]) {
  if constexpr (P == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}

// Cross-CTA reduction of len doubles (deterministic: CTA order within groups of 8, then group
// order); returns true in the last CTA, with the sums in dot[0..len).
__device__ bool block_reduce(const BlockArgs &a, double *dot, int len, int mode, volatile int *sflag, int tid) {
  double *mypart = a.partials + size_t(blockIdx.x) * len;
  for (int c = tid; c < len; c += kConsumers) mypart[c] = dot[c];
  __threadfence();
  named_bar_sync(1, kConsumers);
  const int ngroups = (gridDim.x + kGroup - 1) / kGroup;
  const int grp = blockIdx.x / kGroup;
  const int gfirst = grp * kGroup;
  const int gsize = min(kGroup, int(gridDim.x) - gfirst);
  if (tid == 0) {
    const unsigned t = atomicAdd(&a.gcount[grp], 1u);
    sflag[2] = (t == unsigned(gsize - 1)) ? 1 : 0;
  }
  named_bar_sync(1, kConsumers);
  if (!sflag[2]) return false;
  __threadfence();
  double *gp = a.gpart + size_t(grp) * len;
  for (int c = tid; c < len; c += kConsumers) {
    double t = 0.0;
    for (int b = 0; b < gsize; ++b) t += __ldcg(a.partials + size_t(gfirst + b) * len + c);
    gp[c] = t;
  }
  __threadfence();
  named_bar_sync(1, kConsumers);
  if (tid == 0) {
    a.gcount[grp] = 0u;
    const unsigned t = atomicAdd(&a.bs->ticket[mode], 1u);
    sflag[2] = (t == unsigned(ngroups - 1)) ? 1 : 0;
  }
  named_bar_sync(1, kConsumers);
  if (!sflag[2]) return false;
  __threadfence();
  for (int c = tid; c < len; c += kConsumers) {
    double t = 0.0;
    for (int g = 0; g < ngroups; ++g) t += __ldcg(a.gpart + size_t(g) * len + c);
    dot[c] = t;
  }
  if (tid == 0) a.bs->ticket[mode] = 0u;
  named_bar_sync(1, kConsumers);
  return true;
}

// upper Cholesky of the leading block of a P x P matrix (column-major); returns the columns
// factored (the first failing pivot, or p)
__device__ int chol_up(int p, const double *G, double *R) {
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

// Column sweep layout: thread t takes rows 8*(t%4) .. +7 of each tile and the columns
// t/4 + 64*u, u < CT (CT = ceil(j/64) <= 8), so a thread keeps CT*P FP32 accumulators and the
// P values of its eight rows, and every V element is read from shared memory once.  Two CTAs per
// SM (96 registers a thread); one CTA's sweeps overlap the other's.
template <typename S, int MODE, int CT, int P>
__global__ void __launch_bounds__(kThreads, 2) block_kernel(const BlockArgs a) {
  constexpr bool kRow = (MODE != BLK_A);   // row sweep (BLK_B, BLK_C)
  constexpr bool kCol = (MODE != BLK_C);   // column sweep (BLK_A, BLK_B)
  extern __shared__ __align__(128) unsigned char smem[];
  if (!a.st->active) return;
  const int j = a.j;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *slots = smem;
  float *wsb = reinterpret_cast<float *>(smem + a.off_ws);     // 2 x P x R*32 (row sweep results)
  float *cf = reinterpret_cast<float *>(smem + a.off_coef);    // j x P coefficients (row sweep)
  double *dot = reinterpret_cast<double *>(smem + a.off_dot);  // reduction vector
  float *comb = reinterpret_cast<float *>(smem + a.off_comb);  // row-sweep group partials
  double *red = reinterpret_cast<double *>(smem + a.off_red);  // kConsumers x P(P+1)/2 (Gram) or P (norms)
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.off_bar);
  uint64_t *empty = full + kMaxSlots;
  volatile int *sflag = reinterpret_cast<volatile int *>(empty + kMaxSlots);
  constexpr int NG = P * (P + 1) / 2;
  const int len = (MODE == BLK_C) ? P * P : (MODE == BLK_A ? j * P + P : j * P);
  if (tid == 0) {
    for (int i = 0; i < a.slots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kWarps);
    }
    sflag[0] = 0;
    sflag[2] = 0;
    mbar_fence_init();
  }
  if (kRow) {
    const double *coef = (MODE == BLK_B) ? a.C1 : a.C;  // BLK_C: C holds C2 until BLK_C's epilogue
    for (int e = tid; e < j * P; e += kThreads) cf[e] = float(coef[(e % P) * a.kmax + e / P]);
  }
  for (int c = tid; c < len; c += kThreads) dot[c] = 0.0;
  __syncthreads();

  const S *Vg = static_cast<const S *>(a.V);
  const int64_t tile_elems = int64_t(a.kmax) * kTile;
  const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(j) * sizeof(S);
  constexpr bool kBaseX = (MODE != BLK_C);  // BLK_A/BLK_B read the snapshots, BLK_C the working W
  const int bes = kBaseX ? int(sizeof(S)) : 4;

  if (warp == kWarps) {
    // ---------------------------------------------------------------- producer warp
    if (lane == 0) {
      int it = 0;
      for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
        const int slot = it % a.slots;
        if (it >= a.slots && !mbar_wait(&empty[slot], ((it / a.slots) - 1) & 1)) {
          sflag[0] = 1;
          atomicExch(&a.bs->err, FOA_DMD_ETIMEOUT);
          break;
        }
        if (sflag[0]) break;
        const int t0 = s * a.R;
        const int nt = min(a.R, a.ntiles - t0);
        const int64_t r0 = int64_t(t0) * kTile;
        const bool bb = kBaseX ? (a.x_aligned && r0 + int64_t(nt) * kTile <= a.n) : true;
        const uint32_t bbytes = bb ? uint32_t(nt) * kTile * bes : 0u;
        unsigned char *dst = slots + size_t(slot) * a.slot_bytes;
        mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * tile_bytes + P * bbytes);
        for (int k = 0; k < nt; ++k)
          bulk_g2s(dst + size_t(k) * tile_bytes, Vg + int64_t(t0 + k) * tile_elems, tile_bytes, &full[slot]);
        if (bbytes)
          for (int k = 0; k < P; ++k) {
            const void *src = kBaseX ? static_cast<const void *>(static_cast<const S *>(a.X) + k * a.ldx + r0)
                                     : static_cast<const void *>(a.W + int64_t(k) * a.nrows + r0);
            bulk_g2s(dst + a.base_off + k * a.base_stride, src, bbytes, &full[slot]);
          }
      }
    }
    return;
  }

  // ------------------------------------------------------------------ consumer warps
  float acc[kCol ? CT * P : 1];
#pragma unroll
  for (int q = 0; q < (kCol ? CT * P : 1); ++q) acc[q] = 0.f;
  float nrm[P];  // BLK_A: ||x_k||^2 of the rows this thread saw (threads 0-3 cover every row)
#pragma unroll
  for (int k = 0; k < P; ++k) nrm[k] = 0.f;
  double gram[NG];  // BLK_C: W^T W of the rows this thread finished (pair (k, l), l >= k, in order)
#pragma unroll
  for (int q = 0; q < NG; ++q) gram[q] = 0.0;
  double gslot[P];  // BLK_C, shared finish: products (k, k+i) of the rows' outputs k = tid % P
#pragma unroll
  for (int i = 0; i < P; ++i) gslot[i] = 0.0;
  const int rg = tid & 3, cg = tid >> 2;  // column sweep: row group (8 rows) and column group
  // Fold the accumulators into the CTA's FP64 dot vector: the four threads of a column group
  // (adjacent lanes) reduce-scatter their P partial sums, so that thread rg ends with p = rg and
  // one FP64 add per column and warp suffices.
  auto flush = [&]() {
    if constexpr (kCol) {
#pragma unroll
      for (int u = 0; u < CT; ++u) {
        const int c = cg + 64 * u;
        float r;
        if constexpr (P == 4) {
          const bool hi = (rg & 2) != 0;
          float x0 = hi ? acc[u * P + 2] : acc[u * P + 0], x1 = hi ? acc[u * P + 3] : acc[u * P + 1];
          const float y0 = hi ? acc[u * P + 0] : acc[u * P + 2], y1 = hi ? acc[u * P + 1] : acc[u * P + 3];
          x0 += __shfl_xor_sync(0xffffffffu, y0, 2);
          x1 += __shfl_xor_sync(0xffffffffu, y1, 2);
          const bool od = (rg & 1) != 0;
          r = od ? x1 : x0;
          r += __shfl_xor_sync(0xffffffffu, od ? x0 : x1, 1);
        } else {
          float x0 = acc[u * P + 0], x1 = acc[u * P + 1];
          x0 += __shfl_xor_sync(0xffffffffu, x0, 2);
          x1 += __shfl_xor_sync(0xffffffffu, x1, 2);
          const bool od = (rg & 1) != 0;
          r = od ? x1 : x0;
          r += __shfl_xor_sync(0xffffffffu, od ? x0 : x1, 1);
        }
        if (c < j && rg < P) dot[c * P + rg] += double(r);
#pragma unroll
        for (int k = 0; k < P; ++k) acc[u * P + k] = 0.f;
      }
    }
  };
  int since_flush = 0;
  int it = 0;
  for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
    const int slot = it % a.slots;
    if (!sflag[0] && !mbar_wait(&full[slot], (it / a.slots) & 1)) {
      sflag[0] = 1;
      atomicExch(&a.bs->err, FOA_DMD_ETIMEOUT);
    }
    const int t0 = s * a.R;
    const int nt = min(a.R, a.ntiles - t0);
    const int RS = nt * kTile;
    const int64_t r0 = int64_t(t0) * kTile;
    const unsigned char *sbase = slots + size_t(slot) * a.slot_bytes;
    const S *vs = reinterpret_cast<const S *>(sbase);
    const bool bb = kBaseX ? (a.x_aligned && r0 + int64_t(RS) <= a.n) : true;
    // double buffer: rows of stage s+1 may be finished while slower warps still read stage s's
    float *ws = wsb + (it & 1) * (P * a.R * kTile);
    // base value k of stage row `row`
    auto base_at = [&](int k, int row) -> float {
      if (bb) {
        if constexpr (kBaseX) return to_c(reinterpret_cast<const S *>(sbase + a.base_off + k * a.base_stride)[row]);
        else return reinterpret_cast<const float *>(sbase + a.base_off + k * a.base_stride)[row];
      }
      const int64_t r = r0 + row;
      return (r < a.n) ? float(to_c(static_cast<const S *>(a.X)[k * a.ldx + r])) : 0.f;
    };

    if constexpr (kRow) {
      // ---------------- row sweep: w_k = base_k - sum_c V_rc coef_{c,k}
      auto finish_row = [&](int row, const float *accv) {
        const int64_t r = r0 + row;
        float wv[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
          wv[k] = base_at(k, row) - accv[k];
          a.W[int64_t(k) * a.nrows + r] = wv[k];
          ws[k * (a.R * kTile) + row] = wv[k];
        }
        if constexpr (MODE == BLK_C) {
          int q = 0;
#pragma unroll
          for (int k = 0; k < P; ++k)
#pragma unroll
            for (int l = k; l < P; ++l) gram[q++] += double(wv[k]) * double(wv[l]);  // exact products
        }
      };
      const int PR = RS >> 1;
      const int G1 = (PR >= kConsumers) ? 1 : (kConsumers / PR);
      if (tid < (G1 == 1 ? kConsumers : G1 * PR)) {
        const int g = (G1 == 1) ? 0 : tid / PR;
        const int cpg = (j + G1 - 1) / G1;
        const int c0 = g * cpg, c1 = min(j, c0 + cpg);
        for (int pr = (G1 == 1 ? tid : tid % PR); pr < PR; pr += (G1 == 1 ? kConsumers : PR)) {
          const int row = 2 * pr;
          const S *vr = vs + (row >> 5) * (kTile * j) + (row & 31);
          float a0[P], a1[P];
#pragma unroll
          for (int k = 0; k < P; ++k) a0[k] = a1[k] = 0.f;
#pragma unroll 4
          for (int c = c0; c < c1; ++c) {
            const float2 v = ld_pair(vr + c * kTile);
            float q[P];
            ldp<P>(cf + c * P, q);  // the P coefficients of column c (one 8- or 16-byte load)
#pragma unroll
            for (int k = 0; k < P; ++k) {
              a0[k] = fmaf(v.x, q[k], a0[k]);
              a1[k] = fmaf(v.y, q[k], a1[k]);
            }
          }
          if (G1 > 1) {
            stp<P>(comb + (g * RS + row) * P, a0);
            stp<P>(comb + (g * RS + row + 1) * P, a1);
          } else {
            finish_row(row, a0);
            finish_row(row + 1, a1);
          }
        }
      }
      if (G1 > 1) {
        named_bar_sync(1, kConsumers);
        // one (row, k) output per thread, the P outputs of a row on adjacent lanes; BLK_C's Gram
        // products of the row are shared among those lanes (lane k takes the pairs (k, k+i))
        for (int e0 = 0; e0 < RS * P; e0 += kConsumers) {
          const int e = e0 + tid;
          if (e < RS * P) {  // warp-uniform: RS * P is a multiple of 64
            const int row = e / P, k = e % P;
            float sum = 0.f;
#pragma unroll 4
            for (int g = 0; g < G1; ++g) sum += comb[(g * RS + row) * P + k];
            const float wv = base_at(k, row) - sum;
            a.W[int64_t(k) * a.nrows + (r0 + row)] = wv;
            ws[k * (a.R * kTile) + row] = wv;
            if constexpr (MODE == BLK_C) {
#pragma unroll
              for (int i = 0; i < P; ++i) {
                const float wl = __shfl_down_sync(0xffffffffu, wv, i);
                if (k + i < P) gslot[i] += double(wv) * double(wl);  // exact products
              }
            }
          }
        }
      }
      named_bar_sync(1, kConsumers);  // ws complete
    }

    if constexpr (kCol) {
      // ---------------- column sweep: d_{c,k} = sum_r V_rc base_{r,k}
      const bool swap = (cg & 1) != 0;  // odd column groups read their two row quads in the other order
      for (int kt = 0; kt < nt; ++kt) {
        const int row0 = kt * kTile + 8 * rg;
        float w[8][P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
          float t[8];
          if constexpr (MODE == BLK_B) {
            ld8(ws + k * (a.R * kTile) + row0, false, t);
          } else if (bb) {
            ld8(reinterpret_cast<const S *>(sbase + a.base_off + k * a.base_stride) + row0, false, t);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) t[i] = base_at(k, row0 + i);
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) w[i][k] = t[i];
        }
        if (MODE == BLK_A && cg == 0) {
#pragma unroll
          for (int k = 0; k < P; ++k)
#pragma unroll
            for (int i = 0; i < 8; ++i) nrm[k] = fmaf(w[i][k], w[i][k], nrm[k]);
        }
        const S *vt = vs + kt * (kTile * j) + 8 * rg;
#pragma unroll
        for (int u = 0; u < CT; ++u) {
          const int c = cg + 64 * u;
          if (c < j) {
            float v[8];
            ld8(vt + c * kTile, swap, v);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
              for (int k = 0; k < P; ++k) acc[u * P + k] = fmaf(v[i], w[i][k], acc[u * P + k]);
          }
        }
        if (++since_flush == 4) {  // 32 products per thread and column
          flush();
          since_flush = 0;
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }
  flush();
  // per-thread norms / Gram into the reduction vector (fixed order over threads)
  if constexpr (MODE == BLK_A) {
#pragma unroll
    for (int k = 0; k < P; ++k) red[tid * P + k] = double(nrm[k]);
    named_bar_sync(1, kConsumers);
    if (tid < P) {
      double t = 0.0;
      for (int i = 0; i < kConsumers; ++i) t += red[i * P + tid];
      dot[j * P + tid] = t;
    }
  } else if constexpr (MODE == BLK_C) {
    {
      const int kt = tid % P;  // the output index of this thread in the shared finish
      int q = 0;
#pragma unroll
      for (int k = 0; k < P; ++k)
#pragma unroll
        for (int l = k; l < P; ++l, ++q)
          if (k == kt) gram[q] += gslot[l - k];
    }
#pragma unroll
    for (int q = 0; q < NG; ++q) red[tid * NG + q] = gram[q];
    named_bar_sync(1, kConsumers);
    if (tid < NG) {
      double t = 0.0;
      for (int i = 0; i < kConsumers; ++i) t += red[i * NG + tid];
      int k = 0, q = tid;
      while (q >= P - k) {
        q -= P - k;
        ++k;
      }
      const int l = k + q;
      dot[k + l * P] = t;
      dot[l + k * P] = t;
    }
  }
  named_bar_sync(1, kConsumers);
  if (!block_reduce(a, dot, len, MODE, sflag, tid)) return;
  // ---------------- the last CTA: the scalar part
  if constexpr (MODE == BLK_A) {
    for (int e = tid; e < j * P; e += kConsumers) a.C1[(e % P) * a.kmax + e / P] = dot[e];
    if (tid < P) a.bs->xnorm[tid] = sqrt(dot[j * P + tid]);
  } else if constexpr (MODE == BLK_B) {
    for (int e = tid; e < j * P; e += kConsumers) {
      const int c = e / P, k = e % P;
      a.C[k * a.kmax + c] = dot[e];  // C2 for the row sweep of BLK_C; C = C1 + C2 is formed there
    }
  } else {
    if (tid == 0) {
      BlockState *bs = a.bs;
      for (int k = 0; k < P; ++k)
        for (int l = 0; l < P; ++l) bs->G[k + l * kMaxP] = dot[k + l * P];
      bs->m1 = chol_up(P, bs->G, bs->R1);
    }
    named_bar_sync(1, kConsumers);
    // C = C1 + C2 (C2 was the row sweep's coefficient)
    for (int e = tid; e < j * P; e += kConsumers) {
      const int c = e / P, k = e % P;
      a.C[k * a.kmax + c] = a.C1[k * a.kmax + c] + a.C[k * a.kmax + c];
    }
  }
}

// W1 = W R1^-1 on the leading m1 columns (FP64), G2 = W1^T W1 (per CTA partials), and in the last CTA:
// R2, R = R2 R1, the breakdown test, the beta block column, the Hbar columns, the device state.
template <int P>
__global__ void __launch_bounds__(256) blockq1_kernel(BlockArgs a, foa_dmd_push_info *info_out) {
  __shared__ double red[256 * P * P];
  __shared__ double dot[P * P];
  __shared__ volatile int sflag[4];
  const int tid = threadIdx.x;
  if (!a.st->active) return;
  BlockState *bs = a.bs;
  const int m1 = __ldcg(&bs->m1);
  double R1[P * P];
#pragma unroll
  for (int i = 0; i < P * P; ++i) R1[i] = __ldcg(&bs->R1[(i % P) + (i / P) * kMaxP]);
  double g[P * P];
#pragma unroll
  for (int i = 0; i < P * P; ++i) g[i] = 0.0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + tid; r < a.nrows; r += stride) {
    float w[P];
#pragma unroll
    for (int k = 0; k < P; ++k) w[k] = a.W[int64_t(k) * a.nrows + r];
    // w1_c = (w_c - sum_{k<c} w1_k R1_{k,c}) / R1_{c,c}, in FP64 for the small triangular solve
    double w1[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      double t = w[c];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= w1[k] * R1[k + c * P];
      w1[c] = (c < m1) ? t / R1[c + c * P] : 0.0;
    }
#pragma unroll
    for (int c = 0; c < P; ++c) a.W64[int64_t(c) * a.nrows + r] = w1[c];
#pragma unroll
    for (int k = 0; k < P; ++k)
#pragma unroll
      for (int l = 0; l < P; ++l) g[k + l * P] += w1[k] * w1[l];
  }
#pragma unroll
  for (int i = 0; i < P * P; ++i) red[tid * P * P + i] = g[i];
  __syncthreads();
  if (tid < P * P) {
    double t = 0.0;
    for (int i = 0; i < 256; ++i) t += red[i * P * P + tid];
    dot[tid] = t;
  }
  __syncthreads();
  // deterministic cross-CTA reduction (groups of 8 CTAs, then groups)
  const int len = P * P;
  double *mypart = a.partials + size_t(blockIdx.x) * len;
  if (tid < len) mypart[tid] = dot[tid];
  __threadfence();
  __syncthreads();
  const int ngroups = (gridDim.x + kGroup - 1) / kGroup;
  const int grp = blockIdx.x / kGroup;
  const int gfirst = grp * kGroup;
  const int gsize = min(kGroup, int(gridDim.x) - gfirst);
  if (tid == 0) {
    const unsigned t = atomicAdd(&a.gcount[grp], 1u);
    sflag[2] = (t == unsigned(gsize - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (!sflag[2]) return;
  __threadfence();
  if (tid < len) {
    double t = 0.0;
    for (int b = 0; b < gsize; ++b) t += __ldcg(a.partials + size_t(gfirst + b) * len + tid);
    a.gpart[size_t(grp) * len + tid] = t;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    a.gcount[grp] = 0u;
    const unsigned t = atomicAdd(&bs->ticket[3], 1u);
    sflag[2] = (t == unsigned(ngroups - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (!sflag[2]) return;
  __threadfence();
  if (tid < len) {
    double t = 0.0;
    for (int gq = 0; gq < ngroups; ++gq) t += __ldcg(a.gpart + size_t(gq) * len + tid);
    dot[tid] = t;
  }
  if (tid == 0) bs->ticket[3] = 0u;
  __syncthreads();
  // ---------------- the last CTA
  const int j = a.j;
  const int K = a.kmax;
  if (tid == 0) {
    double G2[kMaxP * kMaxP];
    for (int i = 0; i < kMaxP * kMaxP; ++i) G2[i] = 0.0;
    for (int k = 0; k < m1; ++k)
      for (int l = 0; l < m1; ++l) G2[k + l * kMaxP] = dot[k + l * P];
    const int m = m1 > 0 ? chol_up(m1, G2, bs->R2) : 0;
    // R = R2 R1: rows r < m for every column c (columns past the factored block keep their
    // coefficients on the factored directions)
    for (int i = 0; i < kMaxP * kMaxP; ++i) bs->R[i] = 0.0;
    for (int c = 0; c < P; ++c)
      for (int r = 0; r < m && r <= c; ++r) {
        double t = 0.0;
        const int kmx = c < m1 - 1 ? c : m1 - 1;
        for (int k = r; k <= kmx; ++k) t += bs->R2[r + k * kMaxP] * bs->R1[k + c * kMaxP];
        bs->R[r + c * kMaxP] = t;
      }
    int nc = 0, status = FOA_DMD_OK;
    for (int i = 0; i < P; ++i) {
      const double rii = bs->R[i + i * kMaxP];
      if (!isfinite(rii) || !isfinite(bs->xnorm[i])) {
        status = FOA_DMD_ENONFINITE;
        break;
      }
      if (!(i < m && rii > a.tol * bs->xnorm[i])) {
        status = FOA_DMD_EBREAKDOWN;
        break;
      }
      if (rii < a.resolve * bs->xnorm[i]) {  // below the block form's resolution: not committed
        status = FOA_DMD_ERESOLVE;
        break;
      }
      nc = i + 1;
    }
    bs->ncommit = nc;
    bs->status = status;
  }
  __syncthreads();
  const int nc = bs->ncommit;
  const int status = bs->status;
  // beta block column
  for (int i = 0; i < nc; ++i) {
    const int col = j + i;
    for (int r = tid; r < j; r += blockDim.x) a.B[r + int64_t(col) * K] = __ldcg(a.C + int64_t(i) * K + r);
    for (int r = tid; r <= i; r += blockDim.x) a.B[j + r + int64_t(col) * K] = bs->R[r + i * kMaxP];
  }
  __syncthreads();
  // Hbar columns by forward substitution, one new snapshot after the other
  const int ncols = nc + ((status == FOA_DMD_EBREAKDOWN) ? 1 : 0);
  for (int i = 0; i < ncols; ++i) {
    const int jc = j - 1 + i, jj = j + i;
    const double bjj = a.B[jc + int64_t(jc) * K];
    for (int r = tid; r < jj; r += blockDim.x) {
      const double brc = (r < j) ? __ldcg(a.C + int64_t(i) * K + r) : bs->R[(r - j) + i * kMaxP];
      const int l0 = r == 0 ? 0 : r - 1;
      double acc = 0.0;
      for (int l = l0; l <= jc - 1; ++l) acc += a.H[r + int64_t(l) * K] * a.B[l + int64_t(jc) * K];
      a.H[r + int64_t(jc) * K] = (brc - acc) / bjj;
    }
    __syncthreads();
    if (tid == 0) {
      const double sub = (i < nc) ? bs->R[i + i * kMaxP] / bjj : 0.0;
      a.H[jj + int64_t(jc) * K] = sub;
      foa_dmd_push_info inf;
      inf.h_last = sub;
      inf.indicator = __longlong_as_double(0x7ff8000000000000ll);
      inf.x_norm = bs->xnorm[i];
      inf.q = j + ((i < nc) ? i + 1 : i);
      inf.status = (i < nc) ? FOA_DMD_OK : status;
      if (info_out) info_out[i] = inf;
      a.st->info = inf;
    }
    __syncthreads();
  }
  if (tid == 0) {
    DevState *st = a.st;
    st->q = j + nc;
    st->status = status;
    if (status == FOA_DMD_EBREAKDOWN) st->stopped = 1;
    if (info_out)
      for (int i = ncols; i < P; ++i) {
        foa_dmd_push_info inf;
        inf.h_last = __longlong_as_double(0x7ff8000000000000ll);
        inf.indicator = inf.h_last;
        inf.x_norm = bs->xnorm[i];
        inf.q = j + nc;
        inf.status = (status == FOA_DMD_EBREAKDOWN) ? FOA_DMD_ESTOPPED : status;
        info_out[i] = inf;
      }
  }
}

// Q = W1 R2^-1 -> V columns j .. j+ncommit-1 (row-tiled), rows beyond n zero
template <typename S, int P>
__global__ void blockq2_kernel(BlockArgs a) {
  if (!a.st->active) return;
  const BlockState *bs = a.bs;
  const int nc = __ldcg(&bs->ncommit);
  if (nc == 0) return;
  double R2[P * P];
#pragma unroll
  for (int i = 0; i < P * P; ++i) R2[i] = __ldcg(&bs->R2[(i % P) + (i / P) * kMaxP]);
  S *V = static_cast<S *>(const_cast<void *>(a.V));
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < a.nrows; r += stride) {
    double q[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      double t = a.W64[int64_t(c) * a.nrows + r];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= q[k] * R2[k + c * P];
      q[c] = t / R2[c + c * P];
    }
#pragma unroll
    for (int c = 0; c < P; ++c)
      if (c < nc) V[((r >> 5) * a.kmax + a.j + c) * kTile + (r & 31)] = Store<S>::from(float(r < a.n ? q[c] : 0.0));
  }
}

// device-state gate of a block push (the prep of a single push, for P snapshots)
__global__ void block_prep_kernel(DevState *st, BlockState *bs, int j, int pb, int kmax) {
  if (threadIdx.x != 0) return;
  const bool ok = !st->stopped && st->q == j && j + pb <= kmax && j >= 1;
  st->active = ok ? 1 : 0;
  st->j = j;
  if (!ok) st->status = st->stopped ? FOA_DMD_ESTOPPED : (j + pb > kmax ? FOA_DMD_EFULL : FOA_DMD_EINVAL);
  bs->j = j;
  bs->pb = pb;
  bs->m1 = 0;
  bs->ncommit = 0;
  bs->status = -1;
}

}  // namespace blk
}  // namespace foa

using namespace foa;
using namespace foa::blk;

namespace {

struct BlockWork {
  float *W = nullptr;
  double *W64 = nullptr;
  double *C1 = nullptr, *C = nullptr;
  BlockState *bs = nullptr;
  foa_dmd_push_info *info = nullptr;
};

template <typename S, int MODE, int CT, int P>
cudaError_t launch_block_one(const BlockArgs &a, int grid, cudaStream_t s) {
  auto k = block_kernel<S, MODE, CT, P>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<grid, kThreads, a.smem_total, s>>>(a);
  return cudaGetLastError();
}

template <typename S, int MODE, int P>
cudaError_t launch_block_ct(int ct, const BlockArgs &a, int grid, cudaStream_t s) {
  switch (ct) {
    case 1: return launch_block_one<S, MODE, 1, P>(a, grid, s);
    case 2: return launch_block_one<S, MODE, 2, P>(a, grid, s);
    case 4: return launch_block_one<S, MODE, 4, P>(a, grid, s);
    case 6: return launch_block_one<S, MODE, 6, P>(a, grid, s);
    default: return launch_block_one<S, MODE, 8, P>(a, grid, s);
  }
}

template <typename S, int P>
cudaError_t launch_block_mode(int mode, int ct, const BlockArgs &a, int grid, cudaStream_t s) {
  switch (mode) {
    case BLK_A: return launch_block_ct<S, BLK_A, P>(ct, a, grid, s);
    case BLK_B: return launch_block_ct<S, BLK_B, P>(ct, a, grid, s);
    default: return launch_block_ct<S, BLK_C, P>(ct, a, grid, s);
  }
}

// shared-memory layout and grid of a block pass at basis size j: two CTAs per SM when two ring
// slots fit in half the shared memory, else one CTA per SM
bool block_geom(const foa_dmd *h, int P, int j, bool two, BlockArgs &a, int &grid) {
  const int s = dtype_size(h->dtype);
  const int64_t tile_bytes = int64_t(kTile) * j * s;
  int R = 1;
  while (R * 2 <= kMaxR && (R * 2) * tile_bytes <= 32768) R *= 2;
  auto up = [](int64_t v, int64_t al) { return (v + al - 1) / al * al; };
  const int64_t base_stride = up(int64_t(R) * kTile * 4, 128);
  const int64_t slot = up(R * tile_bytes, 128) + P * base_stride;
  const int64_t other = up(2 * int64_t(P) * R * kTile * 4, 128) + up(int64_t(j) * P * 4, 16) +
                        up(int64_t(j * P + P * P + P) * 8, 16) + int64_t(512) * P * 4 +
                        int64_t(kConsumers) * (P * (P + 1) / 2 > P ? P * (P + 1) / 2 : P) * 8 + 2 * kMaxSlots * 8 + 64;
  if (two && 2 * slot + other > int64_t(112) * 1024) two = false;
  int slots = int((int64_t(two ? 112 : 200) * 1024 - other) / slot);
  if (slots > 4) slots = 4;
  if (slots < 2) return false;
  a.R = R;
  a.slots = slots;
  a.slot_bytes = int(slot);
  a.base_off = int(up(R * tile_bytes, 128));
  a.base_stride = int(base_stride);
  int64_t off = slot * slots;
  a.off_ws = int(off);
  off += up(2 * int64_t(P) * R * kTile * 4, 128);
  a.off_coef = int(off);
  off += up(int64_t(j) * P * 4, 16);
  a.off_dot = int(off);
  off += up(int64_t(j * P + P * P + P) * 8, 16);
  a.off_comb = int(off);
  off += int64_t(512) * P * 4;
  a.off_red = int(off);
  off += int64_t(kConsumers) * (P * (P + 1) / 2 > P ? P * (P + 1) / 2 : P) * 8;
  a.off_bar = int(off);
  off += 2 * kMaxSlots * 8 + 64;
  a.smem_total = int(off);
  if (a.smem_total > 232448) return false;
  a.ntiles = h->ntiles;
  a.n = h->n;
  a.nrows = h->nrows;
  a.nstages = (h->ntiles + R - 1) / R;
  const int sms = h->sms - (h->opts.indicator_every > 0 ? 1 : 0);
  const int per_sm = two ? 2 : 1;
  grid = a.nstages < sms * per_sm ? a.nstages : sms * per_sm;
  return true;
}

// columns per thread of the column sweep (block_kernel's CT): ceil(j / 64), rounded up to an instance
int ct_for(int j) {
  const int need = (j + 63) / 64;
  return need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : need <= 6 ? 6 : 8;
}

// one block of P snapshots (P = 2 or 4) on a stream with q >= 1 basis vectors
template <int P>
int enqueue_block(foa_dmd *h, BlockWork &bw, const void *X, int64_t ldx, foa_dmd_push_info *info_out) {
  const int j = h->q_host;
  BlockArgs a;
  memset(&a, 0, sizeof(a));
  int grid = 0;
  const int ct = ct_for(j);
  if (!block_geom(h, P, j, true, a, grid)) return FOA_DMD_EINVAL;
  a.V = h->V;
  a.X = X;
  a.ldx = ldx;
  a.W = bw.W;
  a.W64 = bw.W64;
  a.C1 = bw.C1;
  a.C = bw.C;
  a.partials = h->partials;
  a.gpart = h->gpart;
  a.gcount = h->gcount;
  a.bs = bw.bs;
  a.st = h->st;
  a.H = h->H;
  a.B = h->B;
  a.kmax = h->kmax;
  a.j = j;
  a.x_aligned = (reinterpret_cast<uintptr_t>(X) & 15u) == 0 && ((ldx * dtype_size(h->dtype)) & 15) == 0;
  a.tol = h->tol;
  a.resolve = kBlockResolveUnits * unit_roundoff(h->dtype);
  cudaStream_t s = h->stream;
  block_prep_kernel<<<1, 32, 0, s>>>(h->st, bw.bs, j, P, h->kmax);
  cudaError_t e = cudaGetLastError();
  const double sz = dtype_size(h->dtype), n = double(h->n);
  for (int mode = BLK_A; mode <= BLK_C && e == cudaSuccess; ++mode) {
    ProfScope ps(h, mode == BLK_A ? 0 : mode == BLK_B ? 1 : 2, n * j * sz + P * n * (mode == BLK_A ? sz : 8.0));
    if (h->dtype == FOA_DMD_F32) e = launch_block_mode<float, P>(mode, ct, a, grid, s);
    else e = launch_block_mode<__nv_bfloat16, P>(mode, ct, a, grid, s);
    h->launches += 1;
  }
  if (e == cudaSuccess) {
    const int g = h->sms * 4;
    blockq1_kernel<P><<<g, 256, 0, s>>>(a, info_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    ProfScope ps(h, 3, n * P * 4 + n * P * sz);
    if (h->dtype == FOA_DMD_F32) blockq2_kernel<float, P><<<h->sms * 4, 256, 0, s>>>(a);
    else blockq2_kernel<__nv_bfloat16, P><<<h->sms * 4, 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  h->launches += 3;
  return cuda_status(e);
}

}  // namespace

extern "C" int foa_dmd_push_block(foa_dmd_t *h, const void *X_dev, int32_t p, int64_t ld, int32_t block,
                                  foa_dmd_push_info *infos) {
  if (!h || !X_dev || p < 0 || ld < h->n || (block != 2 && block != 4)) return FOA_DMD_EINVAL;
  if (h->dtype == FOA_DMD_F64) return FOA_DMD_EINVAL;  // FP32/BF16 storage only
  if (((ld * dtype_size(h->dtype)) & 15) != 0) return FOA_DMD_EINVAL;
  if (p == 0) return FOA_DMD_OK;
  int rc = flush_pending(h);  // a two-pass stream's newest column
  if (rc) return rc;
  rc = sync_state(h, nullptr);
  if (rc) return rc;
  if (h->stopped_host) return FOA_DMD_ESTOPPED;
  BlockWork bw;
  cudaError_t e = cudaMalloc(&bw.W, size_t(kMaxP) * h->nrows * 4);
  if (e == cudaSuccess) e = cudaMalloc(&bw.W64, size_t(kMaxP) * h->nrows * 8);
  if (e == cudaSuccess) e = cudaMalloc(&bw.C1, size_t(kMaxP) * h->kmax * 8);
  if (e == cudaSuccess) e = cudaMalloc(&bw.C, size_t(kMaxP) * h->kmax * 8);
  if (e == cudaSuccess) e = cudaMalloc(&bw.bs, sizeof(BlockState));
  if (e == cudaSuccess) e = cudaMalloc(&bw.info, sizeof(foa_dmd_push_info) * kMaxP);
  if (e == cudaSuccess) e = cudaMemsetAsync(bw.bs, 0, sizeof(BlockState), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(bw.W, 0, size_t(kMaxP) * h->nrows * 4, h->stream);
  rc = cuda_status(e);
  const char *X = static_cast<const char *>(X_dev);
  const size_t colbytes = size_t(ld) * dtype_size(h->dtype);
  int t = 0;
  while (rc == FOA_DMD_OK && t < p) {
    foa_dmd_push_info got[kMaxP];
    int took = 0;
    if (h->q_host == 0 || p - t < block || h->q_host + block > h->kmax) {
      // single push: the first snapshot of a stream, a remainder, or the last columns before k_max
      if (h->q_host >= h->kmax) {
        for (; t < p; ++t)
          if (infos) {
            infos[t].status = FOA_DMD_EFULL;
            infos[t].q = h->kmax;
            infos[t].h_last = infos[t].indicator = infos[t].x_norm = NAN;
          }
        rc = FOA_DMD_EFULL;
        break;
      }
      rc = enqueue_push(h, X + size_t(t) * colbytes, false, bw.info);
      if (rc == FOA_DMD_OK) rc = flush_pending(h);  // a two-pass handle: the column is written now
      if (rc) break;
      took = 1;
    } else {
      rc = block == 4 ? enqueue_block<4>(h, bw, X + size_t(t) * colbytes, ld, bw.info)
                      : enqueue_block<2>(h, bw, X + size_t(t) * colbytes, ld, bw.info);
      if (rc) break;
      took = block;
    }
    e = cudaMemcpyAsync(got, bw.info, sizeof(foa_dmd_push_info) * took, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      rc = cuda_status(e);
      break;
    }
    rc = sync_state(h, nullptr);
    if (rc) break;
    int32_t berr = 0;
    if (took > 1) {
      e = cudaMemcpy(&berr, &bw.bs->err, sizeof(int32_t), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess || berr) {
        rc = e != cudaSuccess ? cuda_status(e) : berr;
        break;
      }
    }
    int first_bad = FOA_DMD_OK;
    for (int i = 0; i < took; ++i) {
      if (infos) infos[t + i] = got[i];
      if (got[i].status != FOA_DMD_OK && first_bad == FOA_DMD_OK) first_bad = got[i].status;
    }
    t += took;
    if (first_bad != FOA_DMD_OK) {
      if (infos)
        for (int u = t; u < p; ++u) {
          infos[u] = got[took - 1];
          infos[u].status = first_bad == FOA_DMD_ERESOLVE ? FOA_DMD_ERESOLVE : FOA_DMD_ESTOPPED;
        }
      rc = first_bad;
      break;
    }
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(bw.W);
  cudaFree(bw.W64);
  cudaFree(bw.C1);
  cudaFree(bw.C);
  cudaFree(bw.bs);
  cudaFree(bw.info);
  return rc;
}
