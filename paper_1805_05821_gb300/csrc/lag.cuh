// First pass of the two-pass push (a reading of the CGS2 projections and norm of Alg. 1 that reads V twice per push
// instead of three times).  Pass B of push j (PASS_B2 in pass.cuh) leaves the new direction
// pending: w' (w after the first projection) stays in the working vector, s = V^T w' in svec,
// and h_{j+1,j} comes from ||w' - V s||^2 = ||w'||^2 - ||s||^2.  The next push appends
// v_{j+1} = (w' - V s) / h_{j+1,j} while it streams the same V tiles for its own first pass:
//
//   lag_kernel<FIN = false>  (PASS_A2), per row r:
//       v_r = (w'_r - sum_{c<jp} V_rc s_c) / h          -> column jp of V (when a column is pending)
//       w_r = (x_r - sum_{c<j} V_rc beta_pre_c) / beta_jj,   then h = V^T w over j columns, ||x||^2
//   lag_kernel<FIN = true>   (PASS_FIN): only the append, before anything reads V (modes, basis
//       copies, checkpoints).
//
// Layout, pipeline (producer warp + bulk copies on mbarriers, eight consumer warps, double-
// buffered w slice), deterministic two-level reduction and bounded waits are those of
// pass_kernel; a slot holds the V tiles (jp columns), the x slice and the w' slice.  Rows at
// and beyond n hold zeros in V, w and w', so the appended column is zero there as well.
#pragma once
#include "internal.cuh"

namespace foa {

// Two CTAs per SM for the FP32/BF16 forms while the column accumulators fit (as pass_kernel).
template <typename S, int NC, bool FIN>
constexpr int lag_min_blocks() {
  return (sizeof(typename Compute<S>::T) == 4 && (FIN || NC <= 48)) ? 2 : 1;
}

template <typename S, int NC, bool FIN>
__global__ void __launch_bounds__(kThreads, lag_min_blocks<S, NC, FIN>()) lag_kernel(const PassArgs a) {
  using C = typename Compute<S>::T;
  constexpr bool kFp64 = sizeof(C) == 8;
  constexpr int kCombStride = kFp64 ? 256 : 512;  // entries of one row-combine vector
  extern __shared__ __align__(128) unsigned char smem[];
  DevState *st = a.st;
  if (!FIN && !st->active) return;
  const int pend = st->pending;
  if (FIN && !pend) return;
  const int jp = st->pend_col;            // index of the pending column
  const int j = FIN ? jp : st->j;         // columns of this push's projection (pending one included)
  const int jt = pend ? jp : j;           // columns already stored in V
  if (j < 1 || j > a.jcap || (pend && !FIN && jp != j - 1)) return;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  unsigned char *slots = smem;
  C *wsb = reinterpret_cast<C *>(smem + a.off_ws);       // 2 x R*32
  C *vnew = reinterpret_cast<C *>(smem + a.off_vnew);    // R*32: the appended column of the stage
  C *cfp = reinterpret_cast<C *>(smem + a.off_coef);     // beta_pre (j, zero padded)
  C *cfs = reinterpret_cast<C *>(smem + a.off_coef2);    // s of the pending column (jt, zero padded)
  double *dot = reinterpret_cast<double *>(smem + a.off_dot);
  C *comb = reinterpret_cast<C *>(smem + a.off_comb);    // 2 x kCombStride
  double *nrm = reinterpret_cast<double *>(smem + a.off_norm);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.off_bar);
  uint64_t *empty = full + kMaxSlots;
  volatile int *sflag = reinterpret_cast<volatile int *>(empty + kMaxSlots);  // [0] abort [2] last

  const C inv_nu = C(st->inv_nu);
  const C inv_bjj = FIN ? C(0) : C(st->inv_bjj);
  if (tid == 0) {
    for (int i = 0; i < a.slots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kWarps);
    }
    sflag[0] = 0;
    sflag[2] = 0;
    mbar_fence_init();
  }
  for (int c = tid; c < ((j + 7) & ~3); c += kThreads) cfp[c] = (!FIN && c < j) ? static_cast<C>(a.coef[c]) : C(0);
  for (int c = tid; c < ((jt + 7) & ~3); c += kThreads) cfs[c] = (pend && c < jt) ? static_cast<C>(a.coef2[c]) : C(0);
  for (int c = tid; c <= j; c += kThreads) dot[c] = 0.0;
  __syncthreads();

  S *Vg = static_cast<S *>(const_cast<void *>(a.V));
  const int64_t tile_elems = int64_t(a.kmax) * kTile;
  const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(jt) * sizeof(S);

  if (warp == kWarps) {
    // ---------------------------------------------------------------- producer warp
    if (lane == 0) {
      const S *xg = static_cast<const S *>(a.x);
      const C *wg = static_cast<const C *>(a.w);
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
        const bool xb = !FIN && a.x_aligned && r0 + int64_t(nt) * kTile <= a.n;
        const uint32_t xbytes = xb ? uint32_t(nt) * kTile * sizeof(S) : 0u;
        const uint32_t wbytes = pend ? uint32_t(nt) * kTile * sizeof(C) : 0u;
        unsigned char *dst = slots + size_t(slot) * a.slot_bytes;
        mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * tile_bytes + xbytes + wbytes);
        if (tile_bytes)
          if (FOA_CHECK(t0 >= 0 && t0 + nt <= a.ntiles, kChkTile))
            for (int k = 0; k < nt; ++k)
              bulk_g2s(dst + size_t(k) * tile_bytes, Vg + int64_t(t0 + k) * tile_elems, tile_bytes, &full[slot]);
        if (xbytes) bulk_g2s(dst + a.base_off, xg + r0, xbytes, &full[slot]);
        if (wbytes) bulk_g2s(dst + a.base2_off, wg + r0, wbytes, &full[slot]);
      }
    }
    return;
  }

  // ------------------------------------------------------------------ consumer warps
  constexpr int NACC = FIN ? 1 : (kFp64 ? NC : (NC + 1) / 2);
  C acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = C(0);
  C nsum = C(0), ncomp = C(0);  // ||x||^2, compensated per thread, folded into FP64 at the end
  auto nrm_add = [&](C v) {
    const C y = v - ncomp;
    const C t = nsum + y;
    ncomp = (t - nsum) - y;
    nsum = t;
  };
  auto flush = [&]() {
    if constexpr (!FIN) {
      if constexpr (kFp64) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const int c = warp + kWarps * k;
          if (c < j) {
            const C v = warp_sum(acc[k]);
            if (lane == 0) dot[c] += static_cast<double>(v);
            acc[k] = C(0);
          }
        }
      } else {
        const int half = lane >> 4;
#pragma unroll
        for (int kk = 0; kk < NACC; ++kk) {
          const int c = warp + kWarps * (2 * kk + half);
          if (warp + kWarps * (2 * kk) < j) {  // warp-uniform
            float v = (c < j) ? acc[kk] : 0.f;
#pragma unroll
            for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((lane & 15) == 0 && c < j) dot[c] += static_cast<double>(v);
            acc[kk] = 0.f;
          }
        }
      }
    }
  };
  int since_flush = 0;
  int it = 0;
  const S *xg = static_cast<const S *>(a.x);
  C *wout = static_cast<C *>(a.w);
  const C bp_pend = (!FIN && pend) ? cfp[jp] : C(0);

  for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
    const int slot = it % a.slots;
    if (!sflag[0] && !mbar_wait(&full[slot], (it / a.slots) & 1)) {
      sflag[0] = 1;
      atomicExch(&st->err, FOA_DMD_ETIMEOUT);
    }
    C *ws = wsb + (it & 1) * (a.R * kTile);
    const int t0 = s * a.R;
    const int nt = min(a.R, a.ntiles - t0);
    const int RS = nt * kTile;
    const int64_t r0 = int64_t(t0) * kTile;
    const unsigned char *sbase = slots + size_t(slot) * a.slot_bytes;
    const S *vs = reinterpret_cast<const S *>(sbase);
    const bool xb = !FIN && a.x_aligned && r0 + int64_t(RS) <= a.n;
    const S *xs = reinterpret_cast<const S *>(sbase + a.base_off);
    const C *wps = reinterpret_cast<const C *>(sbase + a.base2_off);

    // accp = sum_{c<jt} V_rc beta_pre_c, accs = sum_{c<jt} V_rc s_c
    auto finish_row = [&](int row, C accp, C accs) {
      const int64_t r = r0 + row;
      C vn = C(0);
      if (pend) {
        const S vq = Store<S>::from((wps[row] - accs) * inv_nu);
        Vg[((r >> 5) * a.kmax + jp) * kTile + (r & 31)] = vq;
        vn = to_c(vq);
        vnew[row] = vn;
      }
      if constexpr (!FIN) {
        const C xv = xb ? C(to_c(xs[row])) : ((r < a.n) ? C(to_c(xg[r])) : C(0));
        accp += vn * bp_pend;
        const C wc = (xv - accp) * inv_bjj;
        wout[r] = wc;
        ws[row] = wc;
        nrm_add(xv * xv);
      }
    };

    // ---------------- sweep 1: row-local part (GEMV-N against beta_pre and s)
    if constexpr (kFp64) {
      const int G = (RS >= kConsumers) ? 1 : (kConsumers / RS);
      if (tid < (G == 1 ? kConsumers : G * RS)) {
        const int g = (G == 1) ? 0 : tid / RS;
        const int cpg = (jt + G - 1) / G;
        const int c0 = g * cpg, c1 = min(jt, c0 + cpg);
        for (int row = (G == 1 ? tid : tid % RS); row < RS; row += (G == 1 ? kConsumers : RS)) {
          const S *vr = vs + (row >> 5) * (kTile * jt) + (row & 31);
          C p0 = C(0), p1 = C(0), s0 = C(0), s1 = C(0);
          int c = c0;
          for (; c + 2 <= c1; c += 2) {
            const C v0 = to_c(vr[c * kTile]), v1 = to_c(vr[(c + 1) * kTile]);
            p0 = fma(v0, cfp[c], p0);
            p1 = fma(v1, cfp[c + 1], p1);
            s0 = fma(v0, cfs[c], s0);
            s1 = fma(v1, cfs[c + 1], s1);
          }
          if (c < c1) {
            const C v0 = to_c(vr[c * kTile]);
            p0 = fma(v0, cfp[c], p0);
            s0 = fma(v0, cfs[c], s0);
          }
          if (G > 1) {
            comb[g * RS + row] = p0 + p1;
            comb[kCombStride + g * RS + row] = s0 + s1;
          } else {
            finish_row(row, p0 + p1, s0 + s1);
          }
        }
      }
      if (G > 1) {
        named_bar_sync(1, kConsumers);
        if (tid < RS) {
          C ap = C(0), as = C(0);
          for (int g = 0; g < G; ++g) {
            ap += comb[g * RS + tid];
            as += comb[kCombStride + g * RS + tid];
          }
          finish_row(tid, ap, as);
        }
      }
    } else {
      // a thread owns a pair of adjacent rows and a group of columns (a multiple of 4); 16-byte
      // coefficient broadcasts (both coefficient arrays are zero padded)
      const int P = RS >> 1;
      const int G1 = (P >= kConsumers) ? 1 : (kConsumers / P);
      if (tid < (G1 == 1 ? kConsumers : G1 * P)) {
        const int g = (G1 == 1) ? 0 : tid / P;
        const int cpg = (((jt + G1 - 1) / G1) + 3) & ~3;
        const int c0 = g * cpg, c1 = min(jt, c0 + cpg);
        for (int pr = (G1 == 1 ? tid : tid % P); pr < P; pr += (G1 == 1 ? kConsumers : P)) {
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
            comb[g * RS + row] = pa0 + pa1;
            comb[g * RS + row + 1] = pb0 + pb1;
            comb[kCombStride + g * RS + row] = sa0 + sa1;
            comb[kCombStride + g * RS + row + 1] = sb0 + sb1;
          } else {
            finish_row(row, pa0 + pa1, sa0 + sa1);
            finish_row(row + 1, pb0 + pb1, sb0 + sb1);
          }
        }
      }
      if (G1 > 1) {
        named_bar_sync(1, kConsumers);
        if (tid < RS) {
          float ap = 0.f, as = 0.f;
          for (int g = 0; g < G1; ++g) {
            ap += comb[g * RS + tid];
            as += comb[kCombStride + g * RS + tid];
          }
          finish_row(tid, ap, as);
        }
      }
    }
    named_bar_sync(1, kConsumers);  // ws and vnew complete

    // ---------------- sweep 2: h = V^T w over the stored columns and the appended one
    if constexpr (!FIN) {
      if constexpr (kFp64) {
        for (int kt = 0; kt < nt; ++kt) {
          const C wv = ws[kt * kTile + lane];
          const S *vt = vs + kt * (kTile * jt) + lane;
          const C vnl = pend ? vnew[kt * kTile + lane] : C(0);
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const int c = warp + kWarps * k;
            if (c < jt) acc[k] = fma(to_c(vt[c * kTile]), wv, acc[k]);
            else if (c == jt && pend) acc[k] = fma(vnl, wv, acc[k]);
          }
        }
      } else {
        const int hl = lane & 15, half = lane >> 4;
        for (int kt = 0; kt < nt; ++kt) {
          const float2 wv = *reinterpret_cast<const float2 *>(ws + kt * kTile + 2 * hl);
          const S *vt = vs + kt * (kTile * jt) + 2 * hl;
          const float2 vn2 =
              pend ? *reinterpret_cast<const float2 *>(vnew + kt * kTile + 2 * hl) : make_float2(0.f, 0.f);
#pragma unroll
          for (int kk = 0; kk < NACC; ++kk) {
            const int c = warp + kWarps * (2 * kk + half);
            if (c < jt) {
              const float2 v = ld_pair(vt + c * kTile);
              acc[kk] = fmaf(v.x, wv.x, fmaf(v.y, wv.y, acc[kk]));
            } else if (c == jt && pend) {
              acc[kk] = fmaf(vn2.x, wv.x, fmaf(vn2.y, wv.y, acc[kk]));
            }
          }
        }
        since_flush += nt;
        if (since_flush >= 16) {  // 32 products per lane and column
          flush();
          since_flush = 0;
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }

  if constexpr (FIN) {
    // the last CTA to finish clears the pending flag
    named_bar_sync(1, kConsumers);
    if (tid == 0) {
      __threadfence();
      const unsigned t = atomicAdd(&st->ticket[PASS_FIN], 1u);
      if (t == gridDim.x - 1) {
        st->ticket[PASS_FIN] = 0u;
        st->pending = 0;
      }
    }
  } else {
    flush();
    nrm[tid] = double(nsum) - double(ncomp);
    named_bar_sync(1, kConsumers);
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < kConsumers; ++i) t += nrm[i];
      dot[j] = t;
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
      for (int b = 0; b < gsize; ++b) t += __ldcg(a.partials + size_t(gfirst + b) * (a.kmax + 1) + c);
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
}

}  // namespace foa
