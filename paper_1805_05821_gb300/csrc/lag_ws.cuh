// Warp-specialised lagged first pass of the two-pass push for the FP32/BF16 storage forms (the
// arithmetic of lag_kernel<FIN = false> in lag.cuh; the warp roles and hand-offs of pass_ws.cuh):
//   warps 0-3 (row group):    per row of stage s, v = (w' - V s)/h appended to column jp of V,
//                             w = (x - V beta_pre)/beta_jj (the pending column included), ||x||^2;
//                             the stage's w and v go to the ws and vnew buffers (double-buffered);
//   warps 4-7 (column group): h = V^T w over the stored columns and the appended one;
//   warp 8 (producer):        bulk copies of the V tiles, the x slice and the w' slice.
#pragma once
#include "lag.cuh"

namespace foa {

constexpr int kLagRowWarps = 4;
constexpr int kLagColWarps = kWarps - kLagRowWarps;
constexpr int kLagRowThreads = kLagRowWarps * 32;

// Cross-CTA reduction of the lagged first pass (as pass_epilogue), then h and ||x|| of the push.
// On entry every thread has added its column partials into dot[0..j) and stored its norm partial
// in nrm[tid]; pend_part, when given, holds eight per-warp partials of the appended column's dot,
// written before the call and summed here in a fixed order into dot[jt].
__device__ __forceinline__ void lag_epilogue(const PassArgs &a, DevState *st, double *dot, double *nrm,
                                             const double *pend_part, volatile int *sflag, const int j,
                                             const int jt, const int tid) {
  named_bar_sync(1, kConsumers);
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < kConsumers; ++i) t += nrm[i];
    dot[j] = t;
    if (pend_part) {
      double p = 0.0;
      for (int w = 0; w < kWarps; ++w) p += pend_part[w];
      dot[jt] = p;
    }
  }
  named_bar_sync(1, kConsumers);
  const int len = j + 1;
  double *mypart = a.partials + size_t(blockIdx.x) * (a.kmax + 1);
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
  if (!sflag[2]) return;
  __threadfence();
  double *gp = a.gpart + size_t(grp) * (a.kmax + 1);
  for (int c = tid; c < len; c += kConsumers) {
    double t = 0.0;
    for (int bq = 0; bq < gsize; ++bq) t += __ldcg(a.partials + size_t(gfirst + bq) * (a.kmax + 1) + c);
    gp[c] = t;
  }
  __threadfence();
  named_bar_sync(1, kConsumers);
  if (tid == 0) {
    a.gcount[grp] = 0u;
    const unsigned t = atomicAdd(&st->ticket[PASS_A2], 1u);
    sflag[2] = (t == unsigned(ngroups - 1)) ? 1 : 0;
  }
  named_bar_sync(1, kConsumers);
  if (!sflag[2]) return;
  __threadfence();
  for (int c = tid; c < len; c += kConsumers) {
    double t = 0.0;
    for (int g = 0; g < ngroups; ++g) t += __ldcg(a.gpart + size_t(g) * (a.kmax + 1) + c);
    dot[c] = t;
  }
  if (tid == 0) st->ticket[PASS_A2] = 0u;
  named_bar_sync(1, kConsumers);
  for (int c = tid; c < j; c += kConsumers) a.hvec[c] = dot[c];
  if (tid == 0) {
    st->x_norm = sqrt(dot[j]);
    st->pending = 0;  // every CTA has read the flag and appended its rows of the column
  }
}

template <typename S, int NC>
__global__ void __launch_bounds__(kThreads, 2) lag_ws_kernel(const PassArgs a) {
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
  float *wsb = reinterpret_cast<float *>(smem + a.off_ws);      // 2 x R*32: w of a stage
  float *vnb = reinterpret_cast<float *>(smem + a.off_vnew);    // 2 x R*32: the appended column
  float *cfp = reinterpret_cast<float *>(smem + a.off_coef);    // beta_pre (j, zero padded)
  float *cfs = reinterpret_cast<float *>(smem + a.off_coef2);   // s of the pending column (jt, zero padded)
  double *dot = reinterpret_cast<double *>(smem + a.off_dot);
  float *combb = reinterpret_cast<float *>(smem + a.off_comb);  // 2 buffers x (p, s) x 256
  double *nrm = reinterpret_cast<double *>(smem + a.off_norm);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.off_bar);
  uint64_t *empty = full + kMaxSlots;
  volatile int *sflag = reinterpret_cast<volatile int *>(empty + kMaxSlots);  // [0] abort [2] last
  uint64_t *ws_full = empty + kMaxSlots + 2;
  uint64_t *ws_empty = ws_full + 2;

  const float inv_nu = float(st->inv_nu);
  const float inv_bjj = float(st->inv_bjj);
  if (tid == 0) {
    for (int i = 0; i < a.slots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ws_full[b], kLagRowWarps);
      mbar_init(&ws_empty[b], kLagColWarps);
    }
    sflag[0] = 0;
    sflag[2] = 0;
    mbar_fence_init();
  }
  for (int c = tid; c < ((j + 7) & ~3); c += kThreads) cfp[c] = c < j ? static_cast<float>(a.coef[c]) : 0.f;
  for (int c = tid; c < ((jt + 7) & ~3); c += kThreads) cfs[c] = (pend && c < jt) ? static_cast<float>(a.coef2[c]) : 0.f;
  for (int c = tid; c <= j; c += kThreads) dot[c] = 0.0;
  __syncthreads();

  S *Vg = static_cast<S *>(const_cast<void *>(a.V));
  const int64_t tile_elems = int64_t(a.kmax) * kTile;
  const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(jt) * sizeof(S);

  if (warp == kWarps) {
    // ---------------------------------------------------------------- producer warp
    if (lane == 0) {
      const S *xg = static_cast<const S *>(a.x);
      const float *wg = static_cast<const float *>(a.w);
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
        const bool xb = a.x_aligned && r0 + int64_t(nt) * kTile <= a.n;
        const uint32_t xbytes = xb ? uint32_t(nt) * kTile * sizeof(S) : 0u;
        const uint32_t wbytes = pend ? uint32_t(nt) * kTile * 4u : 0u;
        unsigned char *dst = slots + size_t(slot) * a.slot_bytes;
        mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * tile_bytes + xbytes + wbytes);
        if (FOA_CHECK(t0 >= 0 && t0 + nt <= a.ntiles, kChkTile))
          for (int k = 0; k < nt; ++k)
            bulk_g2s(dst + size_t(k) * tile_bytes, Vg + int64_t(t0 + k) * tile_elems, tile_bytes, &full[slot]);
        if (xbytes) bulk_g2s(dst + a.base_off, xg + r0, xbytes, &full[slot]);
        if (wbytes) bulk_g2s(dst + a.base2_off, wg + r0, wbytes, &full[slot]);
      }
    }
    return;
  }

  if (warp < kLagRowWarps) {
    // ------------------------------------------------------------ row group: sweep 1
    const int rt = tid;
    float nsum = 0.f, ncomp = 0.f;
    auto nrm_add = [&](float v) {
      const float y = v - ncomp;
      const float t = nsum + y;
      ncomp = (t - nsum) - y;
      nsum = t;
    };
    const S *xg = static_cast<const S *>(a.x);
    float *wout = static_cast<float *>(a.w);
    const float bp_pend = pend ? cfp[jp] : 0.f;
    int it = 0;
    for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
      const int slot = it % a.slots;
      const int b = it & 1;
      if (!sflag[0] && !mbar_wait(&full[slot], (it / a.slots) & 1)) {
        sflag[0] = 1;
        atomicExch(&st->err, FOA_DMD_ETIMEOUT);
      }
      if (it >= 2 && !sflag[0] && !mbar_wait(&ws_empty[b], ((it >> 1) - 1) & 1)) {
        sflag[0] = 1;
        atomicExch(&st->err, FOA_DMD_ETIMEOUT);
      }
      float *ws = wsb + b * (a.R * kTile);
      float *vnew = vnb + b * (a.R * kTile);
      float *cbp = combb + b * 512;
      float *cbs = cbp + 256;
      const int t0 = s * a.R;
      const int nt = min(a.R, a.ntiles - t0);
      const int RS = nt * kTile;
      const int64_t r0 = int64_t(t0) * kTile;
      const unsigned char *sbase = slots + size_t(slot) * a.slot_bytes;
      const S *vs = reinterpret_cast<const S *>(sbase);
      const bool xb = a.x_aligned && r0 + int64_t(RS) <= a.n;
      const S *xs = reinterpret_cast<const S *>(sbase + a.base_off);
      const float *wps = reinterpret_cast<const float *>(sbase + a.base2_off);

      // accp = sum_{c<jt} V_rc beta_pre_c, accs = sum_{c<jt} V_rc s_c
      auto finish_row = [&](int row, float accp, float accs) {
        const int64_t r = r0 + row;
        float vn = 0.f;
        if (pend) {
          const S vq = Store<S>::from((wps[row] - accs) * inv_nu);
          Vg[((r >> 5) * a.kmax + jp) * kTile + (r & 31)] = vq;
          vn = to_c(vq);
        }
        vnew[row] = vn;
        const float xv = xb ? float(to_c(xs[row])) : ((r < a.n) ? float(to_c(xg[r])) : 0.f);
        accp += vn * bp_pend;
        const float wc = (xv - accp) * inv_bjj;
        wout[r] = wc;
        ws[row] = wc;
        nrm_add(xv * xv);
      };
      const int P = RS >> 1;
      const int G1 = (P >= kLagRowThreads) ? 1 : (kLagRowThreads / P);
      if (rt < (G1 == 1 ? kLagRowThreads : G1 * P)) {
        const int g = (G1 == 1) ? 0 : rt / P;
        const int cpg = (((jt + G1 - 1) / G1) + 3) & ~3;
        const int c0 = g * cpg, c1 = min(jt, c0 + cpg);
        for (int pr = (G1 == 1 ? rt : rt % P); pr < P; pr += (G1 == 1 ? kLagRowThreads : P)) {
          const int row = 2 * pr;
          const S *vr = vs + (row >> 5) * (kTile * jt) + (row & 31);
          float pa0 = 0.f, pa1 = 0.f, pb0 = 0.f, pb1 = 0.f;  // beta_pre: rows row, row+1 (two chains)
          float sa0 = 0.f, sa1 = 0.f, sb0 = 0.f, sb1 = 0.f;  // s
          auto step4 = [&](int c, const float2 (&v)[4]) {
            const float4 qp = *reinterpret_cast<const float4 *>(cfp + c);
            const float4 qs = *reinterpret_cast<const float4 *>(cfs + c);
            pa0 = fmaf(v[0].x, qp.x, pa0); pb0 = fmaf(v[0].y, qp.x, pb0);
            pa1 = fmaf(v[1].x, qp.y, pa1); pb1 = fmaf(v[1].y, qp.y, pb1);
            pa0 = fmaf(v[2].x, qp.z, pa0); pb0 = fmaf(v[2].y, qp.z, pb0);
            pa1 = fmaf(v[3].x, qp.w, pa1); pb1 = fmaf(v[3].y, qp.w, pb1);
            sa0 = fmaf(v[0].x, qs.x, sa0); sb0 = fmaf(v[0].y, qs.x, sb0);
            sa1 = fmaf(v[1].x, qs.y, sa1); sb1 = fmaf(v[1].y, qs.y, sb1);
            sa0 = fmaf(v[2].x, qs.z, sa0); sb0 = fmaf(v[2].y, qs.z, sb0);
            sa1 = fmaf(v[3].x, qs.w, sa1); sb1 = fmaf(v[3].y, qs.w, sb1);
          };
          int c = c0;
          for (; c + 4 <= c1; c += 4) {
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = ld_pair(vr + (c + u) * kTile);
            step4(c, v);
          }
          if (c < c1) {  // 1-3 columns left; the padded coefficients are zero beyond them
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = (c + u < c1) ? ld_pair(vr + (c + u) * kTile) : make_float2(0.f, 0.f);
            step4(c, v);
          }
          if (G1 > 1) {
            cbp[g * RS + row] = pa0 + pa1;
            cbp[g * RS + row + 1] = pb0 + pb1;
            cbs[g * RS + row] = sa0 + sa1;
            cbs[g * RS + row + 1] = sb0 + sb1;
          } else {
            finish_row(row, pa0 + pa1, sa0 + sa1);
            finish_row(row + 1, pb0 + pb1, sb0 + sb1);
          }
        }
      }
      if (G1 > 1) {
        named_bar_sync(2, kLagRowThreads);
        if (rt < RS) {
          float ap = 0.f, as = 0.f;
          for (int g = 0; g < G1; ++g) {
            ap += cbp[g * RS + rt];
            as += cbs[g * RS + rt];
          }
          finish_row(rt, ap, as);
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&ws_full[b]);
        mbar_arrive(&empty[slot]);
      }
    }
    nrm[tid] = double(nsum) - double(ncomp);
  } else {
    // --------------------------------------------------------- column group: sweep 2
    const int cw = warp - kLagRowWarps;
    const int hl = lane & 15, half = lane >> 4;
    float acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.f;
    auto flush = [&]() {
#pragma unroll
      for (int kk = 0; kk < NC; ++kk) {
        const int c = cw + kLagColWarps * (2 * kk + half);
        if (cw + kLagColWarps * (2 * kk) < j) {  // warp-uniform
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
      const float *vnew = vnb + b * (a.R * kTile);
      const int t0 = s * a.R;
      const int nt = min(a.R, a.ntiles - t0);
      const S *vs = reinterpret_cast<const S *>(slots + size_t(slot) * a.slot_bytes);
      for (int kt = 0; kt < nt; ++kt) {
        const float2 wv = *reinterpret_cast<const float2 *>(ws + kt * kTile + 2 * hl);
        const float2 vn2 = *reinterpret_cast<const float2 *>(vnew + kt * kTile + 2 * hl);
        const S *vt = vs + kt * (kTile * jt) + 2 * hl;
#pragma unroll
        for (int kk = 0; kk < NC; ++kk) {
          const int c = cw + kLagColWarps * (2 * kk + half);
          if (c < jt) {
            const float2 v = ld_pair(vt + c * kTile);
            acc[kk] = fmaf(v.x, wv.x, fmaf(v.y, wv.y, acc[kk]));
          } else if (c == jt && pend) {
            acc[kk] = fmaf(vn2.x, wv.x, fmaf(vn2.y, wv.y, acc[kk]));
          }
        }
      }
      since_flush += nt;
      if (since_flush >= 16) {
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

  lag_epilogue(a, st, dot, nrm, nullptr, sflag, j, jt, tid);
}

}  // namespace foa
