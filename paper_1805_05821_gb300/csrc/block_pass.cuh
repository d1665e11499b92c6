// Streaming passes of the block push over V (block CGS2 for P = 2 or 4 snapshots; the block form
// of the QR view of Sec. 3.1).  With V the current basis (j columns) and X_b the block:
//   BLK_A  C1 = V^T X_b and ||psi_k||^2                          (column sweep)
//   BLK_B  W = X_b - V C1,  C2 = V^T W                            (row sweep, then column sweep)
//   BLK_C  W = W - V C2 and the Gram matrix W^T W (exact FP64 products of the FP32 W)
//                                                                  (row sweep)
// Layout.  A pipeline stage is one 32-row tile of the row-tiled V (32*j contiguous elements) and
// the P base slices of its rows (X_b for BLK_A/BLK_B, W for BLK_C), brought into a ring slot by
// bulk copies on an mbarrier.  Thread t of a T-thread CTA owns the row quad rq = t % 8 of every
// tile and the columns c = g + G1*u (g = t / 8, G1 = T / 8, u < FC).  Per stage it copies its
// V fragment (4 rows x FC columns) and its base values into registers; at the first CTA barrier
// the slot is free and one elected thread refills it.  From the registers:
//   row sweep:    P partial sums per row of the fragment, paired over rows (two rows per packed
//                 FP32 FMA against coefficient pairs (q, q) kept in shared memory), combined over
//                 the G1 column groups through shared memory by one thread per (row, output);
//   column sweep: P products per column and row, paired over outputs, one FP32 accumulator pair per
//                 column and output pair, folded every kBlockFlush stages by a reduce-scatter over
//                 the eight lanes of the column group; each lane keeps the running sums of the
//                 outputs it receives as compensated (Kahan) FP32 pairs, widened to FP64 once.
// Columns c >= j read column j - 1 instead (no predicated loads): the row sweep's coefficients are
// zero there and the column sweep never writes those outputs.  Packed FMAs (__ffma2_rn) round each
// lane like fmaf.  The cross-CTA reduction is deterministic (fixed CTA groups); the last CTA
// finishes the pass (coefficients, norms, the first Cholesky step).  A bounded wait that runs out
// records FOA_DMD_ETIMEOUT in the block state, stops the refills and lets the CTA run to its end.
#pragma once
#include <type_traits>

#include "block_internal.cuh"

namespace foa {
namespace blk {

constexpr int kBlockFlush = 8;  // stages between folds: 32 products per FP32 accumulator

// Sum of NV values (NV >= 8) over the eight lanes of a column group, scattered: on return the
// lane holds in x[0 .. NV/8) the totals of the indices off .. off + NV/8 - 1 (off returned).
template <int NV>
__device__ __forceinline__ int reduce_scatter8(float (&x)[NV], int rq) {
  static_assert(NV >= 8 && NV % 8 == 0, "eight lanes, NV/8 values each");
  int off = 0;
#pragma unroll
  for (int lvl = 0; lvl < 3; ++lvl) {
    const int o = 4 >> lvl;
    const int h = NV >> (lvl + 1);
    const bool up = (rq & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? x[i] : x[i + h];
      const float keep = up ? x[i + h] : x[i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    off += up ? h : 0;
  }
  return off;
}

template <typename S, int MODE, int T, int FC, int P>
__global__ void __launch_bounds__(T, 512 / T) block_pass_kernel(const BlockArgs a) {
  static_assert(P == 2 || P == 4, "blocks of 2 or 4");
  static_assert(FC * P >= 8, "at least eight column outputs a thread");
  constexpr bool kRow = (MODE != BLK_A);
  constexpr bool kCol = (MODE != BLK_C);
  constexpr int G1 = T / 8;
  constexpr int KP = P / 2;
  constexpr int NG = P * (P + 1) / 2;
  using BaseT = typename std::conditional<MODE == BLK_C, float, S>::type;

  extern __shared__ __align__(128) unsigned char smem[];
  if (!a.st->active) return;
  const int j = a.j;
  const int tid = threadIdx.x;
  const int rq = tid & 7, g = tid >> 3;
  unsigned char *slots = smem;
  float2 *cfd = reinterpret_cast<float2 *>(smem + a.off_coef);  // (q, q): column c, output k at c*P + k
  float *comb = reinterpret_cast<float *>(smem + a.off_comb);   // row-sweep partials [g][k][row]
  // new w of the stage: row r in slot (r % 4) * 8 + r / 4 (P values), so that the eight lanes of a
  // column group reading row 4 rq + i of their quads touch eight consecutive slots
  float *ws = reinterpret_cast<float *>(smem + a.off_ws);
  double *dot = reinterpret_cast<double *>(smem + a.off_dot);
  double *red = reinterpret_cast<double *>(smem + a.off_red);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.off_bar);
  volatile int *sflag = reinterpret_cast<volatile int *>(full + kMaxSlots);  // [0] abort [2] last
  const int len = (MODE == BLK_C) ? P * P : (MODE == BLK_A ? j * P + P : j * P);
  if (tid == 0) {
    for (int i = 0; i < a.slots; ++i) mbar_init(&full[i], 1);
    sflag[0] = 0;
    sflag[2] = 0;
    mbar_fence_init();
  }
  if constexpr (kRow) {
    const double *coef = (MODE == BLK_B) ? a.C1 : a.C;  // BLK_C: C holds C2 until BLK_C's epilogue
    for (int e = tid; e < G1 * FC * P; e += T) {
      const int c = e / P, k = e % P;
      const float q = c < j ? float(coef[k * a.kmax + c]) : 0.f;
      cfd[e] = make_float2(q, q);
    }
  }
  for (int c = tid; c < len; c += T) dot[c] = 0.0;
  __syncthreads();

  const S *Vg = static_cast<const S *>(a.V);
  const int64_t tile_elems = int64_t(a.kmax) * kTile;
  const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(j) * sizeof(S);
  const BaseT *bg = (MODE == BLK_C) ? reinterpret_cast<const BaseT *>(a.W) : static_cast<const BaseT *>(a.X);
  const int64_t bld = (MODE == BLK_C) ? a.nrows : a.ldx;  // distance between the P base vectors
  // the base slice of tile t comes with the copy when it is 16-byte aligned and inside n
  auto base_bulk = [&](int t) { return MODE == BLK_C || (a.x_aligned && int64_t(t + 1) * kTile <= a.n); };
  constexpr int kIssuer = T - 1;  // not one of the row finishers (t < 32 P)
  auto issue = [&](int slot, int t) {
    const uint32_t bbytes = base_bulk(t) ? uint32_t(kTile * sizeof(BaseT)) : 0u;
    unsigned char *dst = slots + size_t(slot) * a.slot_bytes;
    mbar_arrive_expect_tx(&full[slot], tile_bytes + P * bbytes);
    if (FOA_CHECK(t >= 0 && t < a.ntiles, kChkTile)) bulk_g2s(dst, Vg + int64_t(t) * tile_elems, tile_bytes, &full[slot]);
    if (bbytes)
      for (int k = 0; k < P; ++k)
        bulk_g2s(dst + a.base_off + k * a.base_stride, bg + k * bld + int64_t(t) * kTile, bbytes, &full[slot]);
  };
  if (tid == kIssuer)
    for (int k = 0; k < a.slots; ++k) {
      const int t = blockIdx.x + k * gridDim.x;
      if (t >= a.ntiles) break;
      issue(k, t);
    }

  // this thread's columns: c_u = g + G1 u (those below j are real)
  float2 acc[kCol ? FC * KP : 1];  // column sweep: (output 2kp, output 2kp+1) of column c_u
#pragma unroll
  for (int i = 0; i < (kCol ? FC * KP : 1); ++i) acc[i] = make_float2(0.f, 0.f);
  float nrm[P];     // BLK_A, threads of group 0: ||x_k||^2 over the stages since the last fold
  double nrm64[P];  //   and the folded sums
#pragma unroll
  for (int k = 0; k < P; ++k) nrm[k] = 0.f, nrm64[k] = 0.0;
  constexpr int NQ = (NG + P - 1) / P;  // Gram pairs a finisher takes
  double gram[NQ];  // BLK_C, finisher (k, lane): sums of the products of pairs q = k + P i
  int gk[NQ], gl[NQ];  //   pair q = (gk, gl), gl >= gk, in the order (0,0), (0,1), ..., (P-1,P-1)
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    gram[i] = 0.0;
    int kk = 0, r = (tid >> 5) + P * i;
    while (r >= P - kk && kk < P) r -= P - kk++;
    gk[i] = min(kk, P - 1);
    gl[i] = min(kk + r, P - 1);
  }

  constexpr int NO = kCol ? FC * P / 8 : 1;  // column outputs a lane receives at each fold
  float ks[NO], kc[NO];                       // their running sums and compensations (Kahan)
#pragma unroll
  for (int i = 0; i < NO; ++i) ks[i] = kc[i] = 0.f;
  int koff = 0;                               // index u*P + k of the lane's first output
  auto flush = [&]() {
    if constexpr (kCol) {
      float x[FC * P];
#pragma unroll
      for (int u = 0; u < FC; ++u)
#pragma unroll
        for (int kp = 0; kp < KP; ++kp) {
          x[u * P + 2 * kp] = acc[u * KP + kp].x;
          x[u * P + 2 * kp + 1] = acc[u * KP + kp].y;
          acc[u * KP + kp] = make_float2(0.f, 0.f);
        }
      koff = reduce_scatter8<FC * P>(x, rq);
#pragma unroll
      for (int i = 0; i < NO; ++i) {
        const float y = x[i] - kc[i];
        const float tt = ks[i] + y;
        kc[i] = (tt - ks[i]) - y;
        ks[i] = tt;
      }
      if (MODE == BLK_A && g == 0)
#pragma unroll
        for (int k = 0; k < P; ++k) nrm64[k] += double(nrm[k]), nrm[k] = 0.f;
    }
  };

  int since = 0;
  int slot = 0;
  uint32_t phase = 0;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    if (!sflag[0] && !mbar_wait(&full[slot], phase)) {
      sflag[0] = 1;
      atomicExch(&a.bs->err, FOA_DMD_ETIMEOUT);
    }
    const unsigned char *sb = slots + size_t(slot) * a.slot_bytes;
    const S *vt = reinterpret_cast<const S *>(sb);
    const int64_t r0 = int64_t(t) * kTile;
    const bool bb = base_bulk(t);
    // ---------------- registers: the V fragment and the base values
    float4 v[FC];
#pragma unroll
    for (int u = 0; u < FC; ++u) v[u] = ld4(vt + min(g + G1 * u, j - 1) * kTile + 4 * rq);
    float4 xb[kCol && !kRow ? P : 1];  // BLK_A: rows 4rq .. 4rq+3 of the P snapshots
    float bval = 0.f;                  // BLK_B/BLK_C row finisher (k, row) = (t / 32, t % 32)
    if constexpr (MODE == BLK_A) {
#pragma unroll
      for (int k = 0; k < P; ++k) {
        if (bb) {
          xb[k] = ld4(reinterpret_cast<const S *>(sb + a.base_off + k * a.base_stride) + 4 * rq);
        } else {
          float e[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int64_t r = r0 + 4 * rq + i;
            e[i] = r < a.n ? float(to_c(bg[k * bld + r])) : 0.f;
          }
          xb[k] = make_float4(e[0], e[1], e[2], e[3]);
        }
      }
    } else if (tid < 32 * P) {
      const int k = tid >> 5, row = tid & 31;
      if (bb) bval = to_c(reinterpret_cast<const BaseT *>(sb + a.base_off + k * a.base_stride)[row]);
      else bval = (r0 + row < a.n) ? float(to_c(bg[k * bld + r0 + row])) : 0.f;
    }
    // ---------------- row sweep: partial sums of the rows' P outputs over this thread's columns
    if constexpr (kRow) {
      float2 part[P][2];  // output k: rows (0, 1) and (2, 3) of the quad
#pragma unroll
      for (int k = 0; k < P; ++k) part[k][0] = part[k][1] = make_float2(0.f, 0.f);
      // every u (no per-column branch, so the loads pipeline): the coefficients are zero past j
#pragma unroll
      for (int u = 0; u < FC; ++u) {
        const float4 *qp = reinterpret_cast<const float4 *>(cfd + (g + G1 * u) * P);
        const float2 lo = make_float2(v[u].x, v[u].y), hi = make_float2(v[u].z, v[u].w);
#pragma unroll
        for (int kp = 0; kp < KP; ++kp) {
          const float4 q = qp[kp];  // (q_2kp, q_2kp, q_2kp+1, q_2kp+1)
          const float2 q0 = make_float2(q.x, q.y), q1 = make_float2(q.z, q.w);
          part[2 * kp][0] = __ffma2_rn(lo, q0, part[2 * kp][0]);
          part[2 * kp][1] = __ffma2_rn(hi, q0, part[2 * kp][1]);
          part[2 * kp + 1][0] = __ffma2_rn(lo, q1, part[2 * kp + 1][0]);
          part[2 * kp + 1][1] = __ffma2_rn(hi, q1, part[2 * kp + 1][1]);
        }
      }
#pragma unroll
      for (int k = 0; k < P; ++k)
        *reinterpret_cast<float4 *>(comb + (g * P + k) * kTile + 4 * rq) =
            make_float4(part[k][0].x, part[k][0].y, part[k][1].x, part[k][1].y);
    }
    named_bar_sync(1, T);  // every thread holds its fragment (the slot is free); comb complete
    if (tid == kIssuer && !sflag[0]) {
      const int tn = t + a.slots * gridDim.x;
      if (tn < a.ntiles) issue(slot, tn);
    }
    if constexpr (kRow) {
      // ---------------- finish: w = base - sum over the column groups (one thread per row, output)
      if (tid < 32 * P) {
        const int k = tid >> 5, row = tid & 31;
        const float *cp = comb + k * kTile + row;
        float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
        for (int gg = 0; gg < G1; gg += 2) {
          s0 += cp[gg * P * kTile];
          s1 += cp[(gg + 1) * P * kTile];
        }
        const float wv = bval - (s0 + s1);
        a.W[int64_t(k) * a.nrows + r0 + row] = wv;
        ws[((row & 3) * 8 + (row >> 2)) * P + k] = wv;
      }
      named_bar_sync(1, T);  // ws complete; comb free
    }
    if constexpr (kCol) {
      // ---------------- column sweep: products of the fragment with the rows' P base values
      float2 w2[4][KP];  // row i of the quad: (output 2kp, output 2kp+1)
      if constexpr (MODE == BLK_B) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float *wr = ws + (i * 8 + rq) * P;  // row 4 rq + i
          if constexpr (P == 4) {
            const float4 f = *reinterpret_cast<const float4 *>(wr);
            w2[i][0] = make_float2(f.x, f.y);
            w2[i][1] = make_float2(f.z, f.w);
          } else {
            w2[i][0] = *reinterpret_cast<const float2 *>(wr);
          }
        }
      } else {
#pragma unroll
        for (int kp = 0; kp < KP; ++kp) {
          const float4 e = xb[2 * kp], f = xb[2 * kp + 1];
          w2[0][kp] = make_float2(e.x, f.x);
          w2[1][kp] = make_float2(e.y, f.y);
          w2[2][kp] = make_float2(e.z, f.z);
          w2[3][kp] = make_float2(e.w, f.w);
        }
        if (g == 0)
#pragma unroll
          for (int k = 0; k < P; ++k) {
            const float4 e = xb[k];
            nrm[k] = fmaf(e.x, e.x, fmaf(e.y, e.y, fmaf(e.z, e.z, fmaf(e.w, e.w, nrm[k]))));
          }
      }
#pragma unroll
      for (int u = 0; u < FC; ++u) {  // outputs of columns past j are never written
        const float vr[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 vv = make_float2(vr[i], vr[i]);
#pragma unroll
          for (int kp = 0; kp < KP; ++kp) acc[u * KP + kp] = __ffma2_rn(vv, w2[i][kp], acc[u * KP + kp]);
        }
      }
      if (++since == kBlockFlush) {
        flush();
        since = 0;
      }
    }
    if constexpr (MODE == BLK_C) {
      // Gram products of the stage's rows, pair q = k + P i on finisher (k, lane): the FP64 work
      // spread over P warps, lane l reading ws slot l (row (l % 8) * 4 + l / 8)
      if (tid < 32 * P) {
        const int k = tid >> 5, l = tid & 31;
        float w[P];
        if constexpr (P == 4) {
          const float4 f = *reinterpret_cast<const float4 *>(ws + l * P);
          w[0] = f.x, w[1] = f.y, w[2] = f.z, w[3] = f.w;
        } else {
          const float2 f = *reinterpret_cast<const float2 *>(ws + l * P);
          w[0] = f.x, w[1] = f.y;
        }
#pragma unroll
        for (int i = 0; i < NQ; ++i)
          if (k + P * i < NG) gram[i] += double(w[gk[i]]) * double(w[gl[i]]);  // exact products
      }
    }
    if (++slot == a.slots) {
      slot = 0;
      phase ^= 1u;
    }
  }
  if (since) flush();
  if constexpr (kCol) {
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      const int idx = koff + i;
      const int c = g + G1 * (idx / P);
      if (c < j) dot[c * P + (idx % P)] = double(ks[i]) - double(kc[i]);
    }
  }
  // per-thread norms / Gram into the reduction vector (fixed order over threads)
  if constexpr (MODE == BLK_A) {
    if (tid < 8)
#pragma unroll
      for (int k = 0; k < P; ++k) red[tid * P + k] = nrm64[k] + double(nrm[k]);
    named_bar_sync(1, T);
    if (tid < P) {
      double s = 0.0;
      for (int i = 0; i < 8; ++i) s += red[i * P + tid];
      dot[j * P + tid] = s;
    }
  } else if constexpr (MODE == BLK_C) {
    if (tid < 32 * P) {
      const int k = tid >> 5, l = tid & 31;
#pragma unroll
      for (int i = 0; i < NQ; ++i)
        if (k + P * i < NG) red[(k + P * i) * 32 + l] = gram[i];
    }
    named_bar_sync(1, T);
    if (tid < NG) {
      double s = 0.0;
      for (int i = 0; i < 32; ++i) s += red[tid * 32 + i];
      int k = 0, q = tid;
      while (q >= P - k) q -= P - k++;
      const int l = k + q;
      dot[k + l * P] = s;
      dot[l + k * P] = s;
    }
  }
  named_bar_sync(1, T);
  if (!block_reduce<T>(a, dot, len, MODE, sflag, tid)) return;
  // ---------------- the last CTA: the scalar part
  if constexpr (MODE == BLK_A) {
    for (int e = tid; e < j * P; e += T) a.C1[(e % P) * a.kmax + e / P] = dot[e];
    if (tid < P) a.bs->xnorm[tid] = sqrt(dot[j * P + tid]);
  } else if constexpr (MODE == BLK_B) {
    for (int e = tid; e < j * P; e += T) {
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
    named_bar_sync(1, T);
    // C = C1 + C2 (C2 was the row sweep's coefficient)
    for (int e = tid; e < j * P; e += T) {
      const int c = e / P, k = e % P;
      a.C[k * a.kmax + c] = a.C1[k * a.kmax + c] + a.C[k * a.kmax + c];
    }
  }
}

template <typename S, int MODE, int T, int FC, int P>
cudaError_t launch_block_pass_one(const BlockArgs &a, int grid, cudaStream_t s) {
  auto k = block_pass_kernel<S, MODE, T, FC, P>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<grid, T, a.smem_total, s>>>(a);
  return cudaGetLastError();
}

template <typename S, int MODE, int P>
cudaError_t launch_block_pass_shape(int T, int fc, const BlockArgs &a, int grid, cudaStream_t s) {
  if (T == 512) {
    if constexpr (P == 4)
      if (fc == 6) return launch_block_pass_one<S, MODE, 512, 6, P>(a, grid, s);
    return launch_block_pass_one<S, MODE, 512, 8, P>(a, grid, s);
  }
  if (fc == 8) return launch_block_pass_one<S, MODE, 256, 8, P>(a, grid, s);
  if (fc == 4) return launch_block_pass_one<S, MODE, 256, 4, P>(a, grid, s);
  if constexpr (P == 4) {
    if (fc == 6) return launch_block_pass_one<S, MODE, 256, 6, P>(a, grid, s);
    return launch_block_pass_one<S, MODE, 256, 2, P>(a, grid, s);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
cudaError_t launch_block_pass(int mode, int T, int fc, int P, const BlockArgs &a, int grid, cudaStream_t s) {
  if (P == 4) {
    if (mode == BLK_A) return launch_block_pass_shape<S, BLK_A, 4>(T, fc, a, grid, s);
    if (mode == BLK_B) return launch_block_pass_shape<S, BLK_B, 4>(T, fc, a, grid, s);
    return launch_block_pass_shape<S, BLK_C, 4>(T, fc, a, grid, s);
  }
  if (mode == BLK_A) return launch_block_pass_shape<S, BLK_A, 2>(T, fc, a, grid, s);
  if (mode == BLK_B) return launch_block_pass_shape<S, BLK_B, 2>(T, fc, a, grid, s);
  return launch_block_pass_shape<S, BLK_C, 2>(T, fc, a, grid, s);
}

}  // namespace blk
}  // namespace foa
