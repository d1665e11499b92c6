// Warp-specialised streaming pass for the FP32/BF16 storage forms, for the passes that need both
// sweeps over a staged block of V (PASS_A, PASS_B, PASS_B2; see pass.cuh for what each computes).
//
// The two sweeps depend on each other within a stage (the column dots need the new w of every
// row) but not across stages, so they run on different warps and overlap:
//   warps 0-3 (row group):    sweep 1 of stage s: row-local GEMV-N -> w of the stage's rows,
//                             written to w (global) and to the stage's ws buffer;
//   warps 4-7 (column group): sweep 2 of stage s-1 (or earlier): column dots against ws;
//   warp 8 (producer):        bulk copies of stages s+1, s+2, ... into the slot ring.
// Hand-offs are mbarriers: full[slot] (producer -> both groups), ws_full[b] (row -> column group,
// ws double-buffered by stage parity), ws_empty[b] (column -> row group), empty[slot] (both groups
// -> producer).  Every wait is bounded.  The cross-CTA reduction and the scalar part of the step
// are pass_epilogue, as in pass_kernel.
#pragma once
#include "pass.cuh"

namespace foa {

constexpr int kRowWarps = 4;                  // row group: warps 0..3
constexpr int kColWarps = kWarps - kRowWarps; // column group: warps 4..7
constexpr int kRowThreads = kRowWarps * 32;

template <typename S, int MODE, int NC>
__global__ void __launch_bounds__(kThreads, 2) pass_ws_kernel(const PassArgs a) {
  static_assert(sizeof(typename Compute<S>::T) == 4, "FP32/BF16 storage only");
  static_assert(MODE == PASS_A || MODE == PASS_B || MODE == PASS_B2, "passes with column dots only");
  constexpr bool kBaseX = (MODE == PASS_A);
  constexpr bool kNorm = (MODE == PASS_A || MODE == PASS_B2);
  using BaseT = typename std::conditional<kBaseX, S, float>::type;

  extern __shared__ __align__(128) unsigned char smem[];
  DevState *st = a.st;
  if (!st->active) return;
  const int j = st->j;
  if (j < 1 || j > a.jcap) return;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  unsigned char *slots = smem;
  float *wsb = reinterpret_cast<float *>(smem + a.off_ws);     // 2 x R*32: w of a stage's rows
  float *cf = reinterpret_cast<float *>(smem + a.off_coef);    // coefficients, zero padded
  double *dot = reinterpret_cast<double *>(smem + a.off_dot);
  float *combb = reinterpret_cast<float *>(smem + a.off_comb); // 2 x 256: row-sweep group partials
  double *nrm = reinterpret_cast<double *>(smem + a.off_norm);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.off_bar);
  uint64_t *empty = full + kMaxSlots;
  volatile int *sflag = reinterpret_cast<volatile int *>(empty + kMaxSlots);  // [0] abort [2] last
  uint64_t *ws_full = empty + kMaxSlots + 2;
  uint64_t *ws_empty = ws_full + 2;

  // QR view (a.form): pass A projects x itself (w = x, no pre-vector)
  const bool qr_a = (MODE == PASS_A) && a.form != 0;
  const float cscale = (MODE == PASS_A && !qr_a) ? float(st->inv_bjj) : 1.f;
  if (tid == 0) {
    for (int i = 0; i < a.slots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kWarps);  // all eight consumer warps release a slot
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ws_full[b], kRowWarps);
      mbar_init(&ws_empty[b], kColWarps);
    }
    sflag[0] = 0;
    sflag[2] = 0;
    mbar_fence_init();
  }
  for (int c = tid; c < ((j + 7) & ~3); c += kThreads) cf[c] = c < j ? static_cast<float>(a.coef[c]) : 0.f;
  for (int c = tid; c <= j; c += kThreads) dot[c] = 0.0;
  __syncthreads();

  const S *Vg = static_cast<const S *>(a.V);
  const int64_t tile_elems = int64_t(a.kmax) * kTile;
  const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(j) * sizeof(S);

  if (warp == kWarps) {
    // ---------------------------------------------------------------- producer warp
    if (lane == 0) {
      const BaseT *baseg = kBaseX ? static_cast<const BaseT *>(a.x) : static_cast<const BaseT *>(a.w);
      int it = 0;
      for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
        const int slot = it % a.slots;
        if (it >= a.slots && !mbar_wait(&empty[slot], ((it / a.slots) - 1) & 1)) {
          sflag[0] = 1;
          atomicExch(&st->err, FOA_DMD_ETIMEOUT);
          break;
        }
        if (sflag[0]) break;
        const int t0 = s * a.R;
        const int nt = min(a.R, a.ntiles - t0);
        const int64_t r0 = int64_t(t0) * kTile;
        const bool base_bulk = kBaseX ? (a.x_aligned && r0 + int64_t(nt) * kTile <= a.n) : true;
        const uint32_t bbytes = base_bulk ? uint32_t(nt) * kTile * sizeof(BaseT) : 0u;
        unsigned char *dst = slots + size_t(slot) * a.slot_bytes;
        mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * tile_bytes + bbytes);
        if (FOA_CHECK(t0 >= 0 && t0 + nt <= a.ntiles, kChkTile))
          for (int k = 0; k < nt; ++k)
            bulk_g2s(dst + size_t(k) * tile_bytes, Vg + int64_t(t0 + k) * tile_elems, tile_bytes, &full[slot]);
        if (bbytes) bulk_g2s(dst + a.base_off, baseg + r0, bbytes, &full[slot]);
      }
    }
    return;
  }

  if (warp < kRowWarps) {
    // ------------------------------------------------------------ row group: sweep 1
    const int rt = tid;  // 0 .. kRowThreads-1
    float nsum = 0.f, ncomp = 0.f;  // compensated sum of squares, folded into FP64 at the end
    auto nrm_add = [&](float v) {
      const float y = v - ncomp;
      const float t = nsum + y;
      ncomp = (t - nsum) - y;
      nsum = t;
    };
    int it = 0;
    for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
      const int slot = it % a.slots;
      const int b = it & 1;
      if (!sflag[0] && !mbar_wait(&full[slot], (it / a.slots) & 1)) {
        sflag[0] = 1;
        atomicExch(&st->err, FOA_DMD_ETIMEOUT);
      }
      // ws[b] is free once the column group has finished stage it-2
      if (it >= 2 && !sflag[0] && !mbar_wait(&ws_empty[b], ((it >> 1) - 1) & 1)) {
        sflag[0] = 1;
        atomicExch(&st->err, FOA_DMD_ETIMEOUT);
      }
      float *ws = wsb + b * (a.R * kTile);
      float *cb = combb + b * 256;
      const int t0 = s * a.R;
      const int nt = min(a.R, a.ntiles - t0);
      const int RS = nt * kTile;
      const int64_t r0 = int64_t(t0) * kTile;
      const unsigned char *sbase = slots + size_t(slot) * a.slot_bytes;
      const S *vs = reinterpret_cast<const S *>(sbase);
      const bool base_bulk = kBaseX ? (a.x_aligned && r0 + int64_t(RS) <= a.n) : true;
      const BaseT *bs = reinterpret_cast<const BaseT *>(sbase + a.base_off);
      const BaseT *bg = kBaseX ? static_cast<const BaseT *>(a.x) : static_cast<const BaseT *>(a.w);

      auto finish_row = [&](int row, float acc) {
        const int64_t r = r0 + row;
        float base;
        if (base_bulk) base = to_c(bs[row]);
        else base = (r < a.n) ? float(to_c(bg[r])) : 0.f;
        const float wc = (MODE == PASS_A) ? (base - acc) * cscale : (base - acc);
        static_cast<float *>(a.w)[r] = wc;
        ws[row] = wc;
        if constexpr (MODE == PASS_A) nrm_add(base * base);
        else if constexpr (MODE == PASS_B2) nrm_add(wc * wc);
      };
      if (qr_a) {
        for (int row = rt; row < RS; row += kRowThreads) finish_row(row, 0.f);
      } else {
        // a thread owns a pair of adjacent rows and a group of columns (a multiple of 4); 16-byte
        // coefficient broadcasts, four FP32 chains per row
        const int P = RS >> 1;
        const int G1 = (P >= kRowThreads) ? 1 : (kRowThreads / P);
        if (rt < (G1 == 1 ? kRowThreads : G1 * P)) {
          const int g = (G1 == 1) ? 0 : rt / P;
          const int cpg = (((j + G1 - 1) / G1) + 3) & ~3;
          const int c0 = g * cpg;
          const int c1 = min(j, c0 + cpg);
          for (int pr = (G1 == 1 ? rt : rt % P); pr < P; pr += (G1 == 1 ? kRowThreads : P)) {
            const int row = 2 * pr;
            const S *vr = vs + (row >> 5) * (kTile * j) + (row & 31);
            float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
            int c = c0;
            for (; c + 4 <= c1; c += 4) {
              const float4 q = *reinterpret_cast<const float4 *>(cf + c);
              float2 v[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) v[u] = ld_pair(vr + (c + u) * kTile);
              a0[0] = fmaf(v[0].x, q.x, a0[0]); a1[0] = fmaf(v[0].y, q.x, a1[0]);
              a0[1] = fmaf(v[1].x, q.y, a0[1]); a1[1] = fmaf(v[1].y, q.y, a1[1]);
              a0[2] = fmaf(v[2].x, q.z, a0[2]); a1[2] = fmaf(v[2].y, q.z, a1[2]);
              a0[3] = fmaf(v[3].x, q.w, a0[3]); a1[3] = fmaf(v[3].y, q.w, a1[3]);
            }
            if (c < c1) {  // 1-3 columns left; the padded coefficients are zero beyond them
              const float4 q = *reinterpret_cast<const float4 *>(cf + c);
              float2 v[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) v[u] = (c + u < c1) ? ld_pair(vr + (c + u) * kTile) : make_float2(0.f, 0.f);
              a0[0] = fmaf(v[0].x, q.x, a0[0]); a1[0] = fmaf(v[0].y, q.x, a1[0]);
              a0[1] = fmaf(v[1].x, q.y, a0[1]); a1[1] = fmaf(v[1].y, q.y, a1[1]);
              a0[2] = fmaf(v[2].x, q.z, a0[2]); a1[2] = fmaf(v[2].y, q.z, a1[2]);
              a0[3] = fmaf(v[3].x, q.w, a0[3]); a1[3] = fmaf(v[3].y, q.w, a1[3]);
            }
            const float s0 = (a0[0] + a0[1]) + (a0[2] + a0[3]);
            const float s1 = (a1[0] + a1[1]) + (a1[2] + a1[3]);
            if (G1 > 1) {
              cb[g * RS + row] = s0;
              cb[g * RS + row + 1] = s1;
            } else {
              finish_row(row, s0);
              finish_row(row + 1, s1);
            }
          }
        }
        if (G1 > 1) {
          named_bar_sync(2, kRowThreads);  // row group only
          if (rt < RS) {
            float acc = 0.f;
            for (int g = 0; g < G1; ++g) acc += cb[g * RS + rt];
            finish_row(rt, acc);
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&ws_full[b]);  // release: this warp's ws and w writes
        mbar_arrive(&empty[slot]);
      }
    }
    nrm[tid] = kNorm ? double(nsum) - double(ncomp) : 0.0;
  } else {
    // --------------------------------------------------------- column group: sweep 2
    const int cw = warp - kRowWarps;
    const int hl = lane & 15, half = lane >> 4;
    float acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.f;
    // column c = cw + kColWarps * (2*kk + half): half-warps take alternate columns of the warp's
    // set, a lane covers two adjacent rows
    auto flush = [&]() {
#pragma unroll
      for (int kk = 0; kk < NC; ++kk) {
        const int c = cw + kColWarps * (2 * kk + half);
        if (cw + kColWarps * (2 * kk) < j) {  // warp-uniform: the first half-warp's column exists
          float v = (c < j) ? acc[kk] : 0.f;
#pragma unroll
          for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (hl == 0 && c < j) dot[c] += static_cast<double>(v);
          acc[kk] = 0.f;
        }
      }
    };
    int since_flush = 0;
    int it = 0;
    for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
      const int slot = it % a.slots;
      const int b = it & 1;
      if (!sflag[0] && !mbar_wait(&full[slot], (it / a.slots) & 1)) {
        sflag[0] = 1;
        atomicExch(&st->err, FOA_DMD_ETIMEOUT);
      }
      if (!sflag[0] && !mbar_wait(&ws_full[b], (it >> 1) & 1)) {
        sflag[0] = 1;
        atomicExch(&st->err, FOA_DMD_ETIMEOUT);
      }
      const float *ws = wsb + b * (a.R * kTile);
      const int t0 = s * a.R;
      const int nt = min(a.R, a.ntiles - t0);
      const S *vs = reinterpret_cast<const S *>(slots + size_t(slot) * a.slot_bytes);
      for (int kt = 0; kt < nt; ++kt) {
        const float2 wv = *reinterpret_cast<const float2 *>(ws + kt * kTile + 2 * hl);
        const S *vt = vs + kt * (kTile * j) + 2 * hl;
#pragma unroll
        for (int kk = 0; kk < NC; ++kk) {
          const int c = cw + kColWarps * (2 * kk + half);
          if (c < j) {
            const float2 v = ld_pair(vt + c * kTile);
            acc[kk] = fmaf(v.x, wv.x, fmaf(v.y, wv.y, acc[kk]));
          }
        }
      }
      since_flush += nt;
      if (since_flush >= 16) {  // 32 products per lane and column
        flush();
        since_flush = 0;
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&ws_empty[b]);
        mbar_arrive(&empty[slot]);
      }
    }
    flush();
    nrm[tid] = 0.0;
  }
  pass_epilogue<MODE>(a, st, dot, nrm, sflag, j, tid);
}

}  // namespace foa
