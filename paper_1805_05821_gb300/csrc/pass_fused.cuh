// Streaming pass with the stage held in registers (FP32/BF16 storage, passes A, B and B2 when a
// pipeline stage is one or two 32-row tiles, i.e. the wide-basis part of a run).
//
// A thread owns a fixed pair of adjacent rows of every stage and a fixed group of columns
// (16 or 32 threads share a column group).  Per stage it loads its V fragment (2 rows x FC
// columns) into registers once; from the registers,
//   row sweep:     partial sums of the GEMV-N for its two rows, combined across the column groups
//                  through shared memory, the new w of the stage's rows (as pass_kernel);
//   column sweep:  its columns' dot products with the two new w values, one FP32 accumulator
//                  per column, folded every 16 stages (32 products per lane) by a shuffle tree
//                  over the threads of the column group into the CTA's FP64 dot vector.
// There is no producer warp: the CTA is the eight compute warps (two CTAs of 256 threads per SM,
// up to 128 registers a thread for the fragment), and one elected thread refills a ring slot as
// soon as the first CTA barrier of the stage shows every thread holding its fragment.
// The cross-CTA reduction and the scalar step are pass_epilogue.
#pragma once
#include "pass.cuh"

namespace foa {

// Columns per thread of the register-held pass for this launch (16, 24 or 32), or 0 when the stage
// is wider than two tiles, the column groups would exceed 32 columns, or the launch asks for the
// shared-memory form (PassArgs::variant).
inline int fused_columns(const PassArgs &a) {
  if (a.variant != 0 || a.R > 2) return 0;
  const int G1 = kConsumers / (a.R * (kTile / 2));
  const int cpg = (((a.jcap + G1 - 1) / G1) + 3) & ~3;
  return cpg <= 16 ? 16 : cpg <= 24 ? 24 : cpg <= 32 ? 32 : 0;
}

template <typename S, int MODE, int FC>
__global__ void __launch_bounds__(kConsumers, 2) pass_fused_kernel(const PassArgs a) {
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
  unsigned char *slots = smem;
  float *ws = reinterpret_cast<float *>(smem + a.off_ws);      // w of the stage's rows
  float *cf = reinterpret_cast<float *>(smem + a.off_coef);    // coefficients, zero padded
  double *dot = reinterpret_cast<double *>(smem + a.off_dot);
  float *comb = reinterpret_cast<float *>(smem + a.off_comb);  // row-sweep group partials
  double *nrm = reinterpret_cast<double *>(smem + a.off_norm);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.off_bar);
  volatile int *sflag = reinterpret_cast<volatile int *>(full + 2 * kMaxSlots);  // [0] abort [2] last

  const bool qr_a = (MODE == PASS_A) && a.form != 0;
  const float cscale = (MODE == PASS_A && !qr_a) ? float(st->inv_bjj) : 1.f;
  if (tid == 0) {
    for (int i = 0; i < a.slots; ++i) mbar_init(&full[i], 1);
    sflag[0] = 0;
    sflag[2] = 0;
    mbar_fence_init();
  }
  // fixed mapping: PF row pairs per full stage (R tiles), G1 column groups of cpg columns
  const int PF = a.R * (kTile / 2);                   // 16 (R = 1) or 32 (R = 2)
  const int G1 = kConsumers / PF;                     // 16 or 8
  const int cpg = (((j + G1 - 1) / G1) + 3) & ~3;     // <= FC (host check)
  // coefficients zero-padded past every group's FC-wide window (G1*cpg + FC <= j + 88 < jcap + 96)
  for (int c = tid; c < G1 * cpg + FC; c += kConsumers) cf[c] = c < j ? static_cast<float>(a.coef[c]) : 0.f;
  for (int c = tid; c <= j; c += kConsumers) dot[c] = 0.0;
  __syncthreads();

  const S *Vg = static_cast<const S *>(a.V);
  const int64_t tile_elems = int64_t(a.kmax) * kTile;
  const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(j) * sizeof(S);

  // one elected thread issues the copies of a stage: R whole tiles of V and the stage's slice of x
  // (pass A) or w; a partial x slice (unaligned x, ragged end) is read from global memory instead
  const BaseT *bg = kBaseX ? static_cast<const BaseT *>(a.x) : static_cast<const BaseT *>(a.w);
  constexpr int kIssuer = kConsumers - 1;  // not one of the row finishers (tid < 64)
  auto issue = [&](int slot, int s) {
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
    if (bbytes) bulk_g2s(dst + a.base_off, bg + r0, bbytes, &full[slot]);
  };
  if (tid == kIssuer)
    for (int k = 0; k < a.slots; ++k) {
      const int s = blockIdx.x + k * gridDim.x;
      if (s >= a.nstages) break;
      issue(k, s);
    }

  // ------------------------------------------------------------------ compute
  const int g = tid / PF, pr = tid % PF;
  const int c0 = g * cpg;
  const int nc = max(0, min(j, c0 + cpg) - c0);       // this thread's columns
  float cacc[FC];
#pragma unroll
  for (int u = 0; u < FC; ++u) cacc[u] = 0.f;
  float nsum = 0.f, ncomp = 0.f;
  auto nrm_add = [&](float v) {
    const float y = v - ncomp;
    const float t = nsum + y;
    ncomp = (t - nsum) - y;
    nsum = t;
  };
  auto flush = [&]() {
    // sum over the PF threads of the column group (lanes of one half-warp or one warp)
#pragma unroll
    for (int u = 0; u < FC; ++u) {
      float v = cacc[u];
      if (PF == 32) v += __shfl_xor_sync(0xffffffffu, v, 16);
#pragma unroll
      for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (pr == 0 && u < nc) dot[c0 + u] += static_cast<double>(v);
      cacc[u] = 0.f;
    }
  };
  int since_flush = 0;
  int it = 0;
  for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
    const int slot = it % a.slots;
    if (!sflag[0] && !mbar_wait(&full[slot], (it / a.slots) & 1)) {
      sflag[0] = 1;
      atomicExch(&st->err, FOA_DMD_ETIMEOUT);
    }
    const int t0 = s * a.R;
    const int nt = min(a.R, a.ntiles - t0);
    const int RS = nt * kTile;
    const int64_t r0 = int64_t(t0) * kTile;
    const unsigned char *sbase = slots + size_t(slot) * a.slot_bytes;
    const S *vs = reinterpret_cast<const S *>(sbase);
    const bool base_bulk = kBaseX ? (a.x_aligned && r0 + int64_t(RS) <= a.n) : true;
    // ---------------- the thread's V fragment and its finish row's base value
    const int row = 2 * pr;
    const bool has_rows = row < RS;
    float2 v[FC];
    {
      const S *vr = vs + (row >> 5) * (kTile * j) + (row & 31);
#pragma unroll
      for (int u = 0; u < FC; ++u) v[u] = (has_rows && u < nc) ? ld_pair(vr + (c0 + u) * kTile) : make_float2(0.f, 0.f);
    }
    float base = 0.f;
    if (tid < RS) {
      if (base_bulk) base = to_c(reinterpret_cast<const BaseT *>(sbase + a.base_off)[tid]);
      else base = (r0 + tid < a.n) ? float(to_c(bg[r0 + tid])) : 0.f;
    }
    // ---------------- row sweep from registers
    if (!qr_a) {
      float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
      for (int u = 0; u < FC; u += 4) {
        const float4 q = *reinterpret_cast<const float4 *>(cf + c0 + u);  // zero beyond j
        a0 = fmaf(v[u].x, q.x, a0); b0 = fmaf(v[u].y, q.x, b0);
        a1 = fmaf(v[u + 1].x, q.y, a1); b1 = fmaf(v[u + 1].y, q.y, b1);
        a0 = fmaf(v[u + 2].x, q.z, a0); b0 = fmaf(v[u + 2].y, q.z, b0);
        a1 = fmaf(v[u + 3].x, q.w, a1); b1 = fmaf(v[u + 3].y, q.w, b1);
      }
      comb[g * (2 * PF) + row] = a0 + a1;
      comb[g * (2 * PF) + row + 1] = b0 + b1;
    }
    named_bar_sync(1, kConsumers);  // every thread holds its fragment: the slot is free
    if (tid == kIssuer && !sflag[0]) {
      const int sn = s + a.slots * gridDim.x;
      if (sn < a.nstages) issue(slot, sn);
    }
    if (tid < RS) {
      float acc = 0.f;
      if (!qr_a)
        for (int gg = 0; gg < G1; ++gg) acc += comb[gg * (2 * PF) + tid];
      const float wc = (MODE == PASS_A) ? (base - acc) * cscale : (base - acc);
      static_cast<float *>(a.w)[r0 + tid] = wc;
      ws[tid] = wc;
      if constexpr (MODE == PASS_A) nrm_add(base * base);
      else if constexpr (MODE == PASS_B2) nrm_add(wc * wc);
    }
    named_bar_sync(1, kConsumers);  // ws complete
    // ---------------- column sweep from registers
    if (has_rows) {
      const float2 wv = *reinterpret_cast<const float2 *>(ws + row);
#pragma unroll
      for (int u = 0; u < FC; ++u) cacc[u] = fmaf(v[u].x, wv.x, fmaf(v[u].y, wv.y, cacc[u]));
    }
    if (++since_flush == 16) {  // 32 products per thread and column
      flush();
      since_flush = 0;
    }
  }
  flush();
  nrm[tid] = kNorm ? double(nsum) - double(ncomp) : 0.0;
  pass_epilogue<MODE>(a, st, dot, nrm, sflag, j, tid);
}

}  // namespace foa
