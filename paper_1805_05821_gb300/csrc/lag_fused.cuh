// Lagged first pass of the two-pass push with the stage held in registers (FP32/BF16 storage,
// stages of one or two 32-row tiles): the arithmetic of lag_ws_kernel on the thread layout of
// pass_fused_kernel (no producer warp, two CTAs of 256 threads per SM).
//   row sweep:     per row pair, sum_c V_rc beta_pre_c and sum_c V_rc s_c over the stored columns,
//                  from the thread's V fragment, combined across the column groups through shared
//                  memory; the finisher of row r appends v_r = (w'_r - sum V s)/h to column jp of
//                  V and forms w_r = (x_r - sum V beta_pre - v_r beta_pre_jp)/beta_jj;
//   column sweep:  the stored columns' dots with w from the registers; the appended column's dot
//                  sum_r v_r w_r accumulates in FP64 in the row finishers.
#pragma once
#include "lag_ws.cuh"
#include "pass_fused.cuh"

namespace foa {

template <typename S, int FC>
__global__ void __launch_bounds__(kConsumers, 2) lag_fused_kernel(const PassArgs a) {
  static_assert(sizeof(typename Compute<S>::T) == 4, "FP32/BF16 storage only");
  extern __shared__ __align__(128) unsigned char smem[];
  DevState *st = a.st;
  if (!st->active) return;
  const int pend = st->pending;
  const int jp = st->pend_col;          // index of the pending column
  const int j = st->j;                  // columns of this push's projection (pending one included)
  const int jt = pend ? jp : j;         // columns already stored in V
  if (j < 1 || j > a.jcap || (pend && jp != j - 1)) return;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  unsigned char *slots = smem;
  float *ws = reinterpret_cast<float *>(smem + a.off_ws);      // w of the stage's rows
  float *cfp = reinterpret_cast<float *>(smem + a.off_coef);   // beta_pre (j, zero padded)
  float *cfs = reinterpret_cast<float *>(smem + a.off_coef2);  // s of the pending column (jt, zero padded)
  double *dot = reinterpret_cast<double *>(smem + a.off_dot);
  float *combp = reinterpret_cast<float *>(smem + a.off_comb);  // row-sweep group partials, beta_pre
  float *combs = combp + 2 * kConsumers;                        //                          s
  double *nrm = reinterpret_cast<double *>(smem + a.off_norm);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.off_bar);
  volatile int *sflag = reinterpret_cast<volatile int *>(full + 2 * kMaxSlots);  // [0] abort [2] last

  const float inv_nu = float(st->inv_nu);
  const float inv_bjj = float(st->inv_bjj);
  if (tid == 0) {
    for (int i = 0; i < a.slots; ++i) mbar_init(&full[i], 1);
    sflag[0] = 0;
    sflag[2] = 0;
    mbar_fence_init();
  }
  // fixed mapping as pass_fused_kernel, over the stored columns
  const int PF = a.R * (kTile / 2);
  const int G1 = kConsumers / PF;
  const int cpg = (((jt + G1 - 1) / G1) + 3) & ~3;  // <= FC (host check)
  // zero padding past every group's window: G1*cpg + FC <= jt + 88 < jcap + 96, and > j
  for (int c = tid; c < G1 * cpg + FC; c += kConsumers) {
    cfp[c] = c < j ? static_cast<float>(a.coef[c]) : 0.f;
    cfs[c] = (pend && c < jt) ? static_cast<float>(a.coef2[c]) : 0.f;
  }
  for (int c = tid; c <= j; c += kConsumers) dot[c] = 0.0;
  __syncthreads();

  S *Vg = static_cast<S *>(const_cast<void *>(a.V));
  const S *xg = static_cast<const S *>(a.x);
  const float *wg = static_cast<const float *>(a.w);
  const int64_t tile_elems = int64_t(a.kmax) * kTile;
  const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(jt) * sizeof(S);

  // one elected thread issues the copies of a stage: R tiles of V, the x slice and the w' slice
  constexpr int kIssuer = kConsumers - 1;  // not one of the row finishers (tid < 64)
  auto issue = [&](int slot, int s) {
    const int t0 = s * a.R;
    const int nt = min(a.R, a.ntiles - t0);
    const int64_t r0 = int64_t(t0) * kTile;
    const bool xb = a.x_aligned && r0 + int64_t(nt) * kTile <= a.n;
    const uint32_t xbytes = xb ? uint32_t(nt) * kTile * sizeof(S) : 0u;
    const uint32_t wbytes = pend ? uint32_t(nt) * kTile * 4u : 0u;
    unsigned char *dst = slots + size_t(slot) * a.slot_bytes;
    mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * tile_bytes + xbytes + wbytes);
    if (tile_bytes)
      if (FOA_CHECK(t0 >= 0 && t0 + nt <= a.ntiles, kChkTile))
        for (int k = 0; k < nt; ++k)
          bulk_g2s(dst + size_t(k) * tile_bytes, Vg + int64_t(t0 + k) * tile_elems, tile_bytes, &full[slot]);
    if (xbytes) bulk_g2s(dst + a.base_off, xg + r0, xbytes, &full[slot]);
    if (wbytes) bulk_g2s(dst + a.base2_off, wg + r0, wbytes, &full[slot]);
  };
  if (tid == kIssuer)
    for (int k = 0; k < a.slots; ++k) {
      const int s = blockIdx.x + k * gridDim.x;
      if (s >= a.nstages) break;
      issue(k, s);
    }

  const int g = tid / PF, pr = tid % PF;
  const int c0 = g * cpg;
  const int nc = max(0, min(jt, c0 + cpg) - c0);  // this thread's stored columns
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
  double pacc = 0.0;  // the appended column's dot, rows finished by this thread
  auto flush = [&]() {
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
  float *wout = static_cast<float *>(a.w);
  const float bp_pend = pend ? cfp[jp] : 0.f;
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
    const bool xb = a.x_aligned && r0 + int64_t(RS) <= a.n;
    // ---------------- the thread's V fragment and its finish row's x and w' values
    const int row = 2 * pr;
    const bool has_rows = row < RS;
    float2 v[FC];
    {
      const S *vr = vs + (row >> 5) * (kTile * jt) + (row & 31);
#pragma unroll
      for (int u = 0; u < FC; ++u) v[u] = (has_rows && u < nc) ? ld_pair(vr + (c0 + u) * kTile) : make_float2(0.f, 0.f);
    }
    float xv = 0.f, wpv = 0.f;
    if (tid < RS) {
      const int64_t r = r0 + tid;
      xv = xb ? float(to_c(reinterpret_cast<const S *>(sbase + a.base_off)[tid]))
              : ((r < a.n) ? float(to_c(xg[r])) : 0.f);
      if (pend) wpv = reinterpret_cast<const float *>(sbase + a.base2_off)[tid];
    }
    // ---------------- row sweep from registers: two coefficient vectors
    {
      float pa0 = 0.f, pa1 = 0.f, pb0 = 0.f, pb1 = 0.f;  // beta_pre: rows row, row+1 (two chains)
      float sa0 = 0.f, sa1 = 0.f, sb0 = 0.f, sb1 = 0.f;  // s
#pragma unroll
      for (int u = 0; u < FC; u += 4) {
        const float4 qp = *reinterpret_cast<const float4 *>(cfp + c0 + u);
        const float4 qs = *reinterpret_cast<const float4 *>(cfs + c0 + u);
        pa0 = fmaf(v[u].x, qp.x, pa0); pb0 = fmaf(v[u].y, qp.x, pb0);
        pa1 = fmaf(v[u + 1].x, qp.y, pa1); pb1 = fmaf(v[u + 1].y, qp.y, pb1);
        pa0 = fmaf(v[u + 2].x, qp.z, pa0); pb0 = fmaf(v[u + 2].y, qp.z, pb0);
        pa1 = fmaf(v[u + 3].x, qp.w, pa1); pb1 = fmaf(v[u + 3].y, qp.w, pb1);
        sa0 = fmaf(v[u].x, qs.x, sa0); sb0 = fmaf(v[u].y, qs.x, sb0);
        sa1 = fmaf(v[u + 1].x, qs.y, sa1); sb1 = fmaf(v[u + 1].y, qs.y, sb1);
        sa0 = fmaf(v[u + 2].x, qs.z, sa0); sb0 = fmaf(v[u + 2].y, qs.z, sb0);
        sa1 = fmaf(v[u + 3].x, qs.w, sa1); sb1 = fmaf(v[u + 3].y, qs.w, sb1);
      }
      combp[g * (2 * PF) + row] = pa0 + pa1;
      combp[g * (2 * PF) + row + 1] = pb0 + pb1;
      combs[g * (2 * PF) + row] = sa0 + sa1;
      combs[g * (2 * PF) + row + 1] = sb0 + sb1;
    }
    named_bar_sync(1, kConsumers);  // every thread holds its fragment: the slot is free
    if (tid == kIssuer && !sflag[0]) {
      const int sn = s + a.slots * gridDim.x;
      if (sn < a.nstages) issue(slot, sn);
    }
    if (tid < RS) {
      float ap = 0.f, as = 0.f;
      for (int gg = 0; gg < G1; ++gg) {
        ap += combp[gg * (2 * PF) + tid];
        as += combs[gg * (2 * PF) + tid];
      }
      const int64_t r = r0 + tid;
      float vn = 0.f;
      if (pend) {
        const S vq = Store<S>::from((wpv - as) * inv_nu);
        Vg[((r >> 5) * a.kmax + jp) * kTile + (r & 31)] = vq;
        vn = to_c(vq);
      }
      const float wc = (xv - (ap + vn * bp_pend)) * inv_bjj;
      wout[r] = wc;
      ws[tid] = wc;
      nrm_add(xv * xv);
      pacc = fma(double(vn), double(wc), pacc);
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
  nrm[tid] = double(nsum) - double(ncomp);
  // the appended column's partials, one per warp (the row-sweep buffers are free after the loop)
  double *pend_part = reinterpret_cast<double *>(combp);
  double pw = pacc;
#pragma unroll
  for (int o = 16; o; o >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, o);
  if (lane == 0) pend_part[warp] = pend ? pw : 0.0;
  lag_epilogue(a, st, dot, nrm, pend ? pend_part : nullptr, sflag, j, jt, tid);
}

}  // namespace foa
