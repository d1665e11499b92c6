// Streaming passes over the basis V for one modified-FOA push (the pre-vector, the CGS2
// projections and the norm of Alg. 1; the streaming form of Alg. 4).  The pass kinds:
//
//   PASS_A      pre-vector w = (x - V beta_pre) / beta_jj,  first projection h = V^T w,  ||x||^2
//               (QR view: w = x)
//   PASS_B      w = w - V h,  reorthogonalisation s = V^T w
//   PASS_C      w = w - V s,  ||w||^2 (h_{j+1,j} = ||w||)
//   PASS_FIRST  ||x||^2 of the first snapshot (beta_11 = ||psi_1||)
//   PASS_B2     pass B of the two-pass push, plus ||w||^2 and the commit of h_{j+1,j} from
//               ||w - V s||^2 = ||w||^2 - ||s||^2; the new column stays pending (lag.cuh)
//
// Layout and schedule.  V is row-tiled: a tile of 32 rows stores its k_max columns one after
// another (32 contiguous elements per column), so the leading j columns of a tile are one
// contiguous block of 32*j elements.  A pipeline stage is R consecutive tiles; a producer warp
// fetches each stage's tiles (and the 32R-row slice of x or w) into a shared-memory ring with
// one-dimensional bulk async copies completing on mbarriers, and the consumer warps make two
// sweeps over the staged block, so V is read from HBM exactly once per pass:
//   sweep 1 (row-local GEMV-N): the new w of every row of the stage;
//   sweep 2 (GEMV-T split over rows): the column dots, one register accumulator per owned column,
//           folded into FP64 every 32 products per lane.
// pass_kernel (this file) runs pass C and PASS_FIRST for every storage type and passes A, B, B2
// for FP64 storage, with all eight consumer warps on sweep 1 and then on sweep 2.  For FP32/BF16
// storage passes A, B and B2 run in pass_ws_kernel (pass_ws.cuh), which puts the two sweeps on
// different warps so that they overlap across stages.  Both end in pass_epilogue.
//
// Every wait is bounded; a timeout records FOA_DMD_ETIMEOUT in the device state and the CTA
// stops waiting (its results are discarded by the host).
#pragma once
#include "internal.cuh"

namespace foa {

// Cross-CTA reduction and the scalar part of the step, shared by the streaming-pass kernels.
// On entry every consumer thread (tid < kConsumers) has added its column partials into dot[0..j)
// and stored its norm partial in nrm[tid]; dot[j] receives the CTA's norm.  Each CTA leaves its
// FP64 partial vector in global memory; the last CTA of every group of 8 CTAs (atomic ticket)
// sums its group in CTA order, and the last group sums the group partials in group order, so the
// reduction is deterministic.  That last CTA then applies the scalar part of the step.
template <int MODE>
__device__ __forceinline__ void pass_epilogue(const PassArgs &a, DevState *st, double *dot, double *nrm,
                                              volatile int *sflag, const int j, const int tid) {
  constexpr bool kNorm = (MODE == PASS_A || MODE == PASS_C || MODE == PASS_FIRST || MODE == PASS_B2);
  named_bar_sync(1, kConsumers);
  const int len = j + 1;
  if (tid == 0) {
    if constexpr (kNorm) {
      double t = 0.0;
      for (int i = 0; i < kConsumers; ++i) t += nrm[i];
      dot[j] = t;
    }
  }
  named_bar_sync(1, kConsumers);
  double *mypart = a.partials + size_t(blockIdx.x) * (a.kmax + 1);
  for (int c = tid; c < len; c += kConsumers) mypart[c] = dot[c];
  __threadfence();
  named_bar_sync(1, kConsumers);

  // ---------------- two-level deterministic reduction (last arriving CTA of each group)
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
    const unsigned t = atomicAdd(&st->ticket[MODE], 1u);
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
  if (tid == 0) st->ticket[MODE] = 0u;
  named_bar_sync(1, kConsumers);

  // ---------------- scalar part of the step (one CTA)
  if constexpr (MODE == PASS_A) {
    for (int c = tid; c < j; c += kConsumers) a.hvec[c] = dot[c];
    if (tid == 0) st->x_norm = sqrt(dot[j]);
  } else if constexpr (MODE == PASS_B) {
    for (int c = tid; c < j; c += kConsumers) {
      a.svec[c] = dot[c];
      a.hvec[c] = a.hvec[c] + dot[c];  // h = h + s
    }
  } else if constexpr (MODE == PASS_C) {
    if (a.form) {
      // QR view: beta column [h; nu]; Hbar column from beta_{:,2:} = Hbar beta (Eq. matmulhbeta) by
      // forward substitution, Hbar_{i,j} = (h_i - beta_pre_i) / beta_jj, Hbar_{j+1,j} = nu / beta_jj
      const double nu = sqrt(dot[j]);
      const double xn = st->x_norm;
      const double bjj = st->bjj;
      int status;
      if (!isfinite(nu) || !isfinite(xn)) status = FOA_DMD_ENONFINITE;
      else if (!(nu > a.tol * xn)) status = FOA_DMD_EBREAKDOWN;
      else status = FOA_DMD_OK;
      const int64_t ld = a.kmax;
      if (status != FOA_DMD_ENONFINITE)
        for (int c = tid; c < j; c += kConsumers) a.H[c + int64_t(j - 1) * ld] = (a.hvec[c] - a.pre[c]) / bjj;
      if (status == FOA_DMD_OK)
        for (int c = tid; c < j; c += kConsumers) a.B[c + int64_t(j) * ld] = a.hvec[c];
      named_bar_sync(1, kConsumers);
      if (tid == 0) {
        const double hsub = nu / bjj;
        if (status == FOA_DMD_OK) {
          a.H[j + int64_t(j - 1) * ld] = hsub;
          a.B[j + int64_t(j) * ld] = nu;
          st->nu = nu;
          st->inv_nu = 1.0 / nu;  // v_{j+1} = w / nu
          st->q = j + 1;
        } else if (status == FOA_DMD_EBREAKDOWN) {
          a.H[j + int64_t(j - 1) * ld] = 0.0;
          st->stopped = 1;
        }
        st->status = status;
        if (status != FOA_DMD_OK && a.batch) st->halt = 1;
        foa_dmd_push_info inf;
        inf.h_last = hsub;
        inf.indicator = __longlong_as_double(0x7ff8000000000000ll);
        inf.x_norm = xn;
        inf.q = st->q;
        inf.status = status;
        st->info = inf;
        if (a.info_out) *a.info_out = inf;
      }
      return;
    }
    const double nu = sqrt(dot[j]);
    const double xn = st->x_norm;
    const double bjj = st->bjj;
    int status;
    if (!isfinite(nu) || !isfinite(xn)) status = FOA_DMD_ENONFINITE;
    else if (!(nu * bjj > a.tol * xn)) status = FOA_DMD_EBREAKDOWN;
    else status = FOA_DMD_OK;
    const int64_t ld = a.kmax;
    if (status != FOA_DMD_ENONFINITE) {
      for (int c = tid; c < j; c += kConsumers) a.H[c + int64_t(j - 1) * ld] = a.hvec[c];
    }
    if (status == FOA_DMD_OK) {
      // beta column: beta_{i,j+1} = beta_pre_i + h_{i,j} beta_{j,j}; beta_{j+1,j+1} = h_{j+1,j} beta_{j,j}
      for (int c = tid; c < j; c += kConsumers) a.B[c + int64_t(j) * ld] = a.pre[c] + a.hvec[c] * bjj;
    }
    named_bar_sync(1, kConsumers);
    if (tid == 0) {
      if (status == FOA_DMD_OK) {
        a.H[j + int64_t(j - 1) * ld] = nu;
        a.B[j + int64_t(j) * ld] = nu * bjj;
        st->nu = nu;
        st->inv_nu = 1.0 / nu;
        st->q = j + 1;
      } else if (status == FOA_DMD_EBREAKDOWN) {
        a.H[j + int64_t(j - 1) * ld] = 0.0;
        st->stopped = 1;
      }
      st->status = status;
      if (status != FOA_DMD_OK && a.batch) st->halt = 1;
      foa_dmd_push_info inf;
      inf.h_last = nu;
      inf.indicator = __longlong_as_double(0x7ff8000000000000ll);
      inf.x_norm = xn;
      inf.q = st->q;
      inf.status = status;
      st->info = inf;
      if (a.info_out) *a.info_out = inf;
    }
  } else if constexpr (MODE == PASS_B2) {
    // s = V^T w' and h += s as in PASS_B, then h_{j+1,j} without a third pass: w still holds w' (after the
    // first projection) and s = V^T w', so ||w' - V s||^2 = ||w'||^2 - ||s||^2 for orthonormal V.
    double *ssq = nrm;  // per-thread partial sums of s_c^2, in column order within a thread
    double t = 0.0;
    for (int c = tid; c < j; c += kConsumers) {
      const double sc = dot[c];
      a.svec[c] = sc;
      a.hvec[c] = a.hvec[c] + sc;
      t += sc * sc;
    }
    ssq[tid] = t;
    named_bar_sync(1, kConsumers);
    if (tid == 0) {
      double ss = 0.0;
      for (int i = 0; i < kConsumers; ++i) ss += ssq[i];
      const double d = dot[j] - ss;
      ssq[0] = d > 0.0 ? sqrt(d) : 0.0;
    }
    named_bar_sync(1, kConsumers);
    const double nu = ssq[0];
    const double xn = st->x_norm;
    const double bjj = st->bjj;
    int status;
    if (!isfinite(nu) || !isfinite(xn) || !isfinite(dot[j])) status = FOA_DMD_ENONFINITE;
    else if (!(nu * bjj > a.tol * xn)) status = FOA_DMD_EBREAKDOWN;
    else status = FOA_DMD_OK;
    const int64_t ld = a.kmax;
    if (status != FOA_DMD_ENONFINITE) {
      for (int c = tid; c < j; c += kConsumers) a.H[c + int64_t(j - 1) * ld] = a.hvec[c];
    }
    if (status == FOA_DMD_OK) {
      for (int c = tid; c < j; c += kConsumers) a.B[c + int64_t(j) * ld] = a.pre[c] + a.hvec[c] * bjj;
    }
    named_bar_sync(1, kConsumers);
    if (tid == 0) {
      if (status == FOA_DMD_OK) {
        a.H[j + int64_t(j - 1) * ld] = nu;
        a.B[j + int64_t(j) * ld] = nu * bjj;
        st->nu = nu;
        st->inv_nu = 1.0 / nu;
        st->q = j + 1;
        st->pending = 1;  // v_{j+1} = (w' - V s) / nu is written by the next pass over V
        st->pend_col = j;
      } else if (status == FOA_DMD_EBREAKDOWN) {
        a.H[j + int64_t(j - 1) * ld] = 0.0;
        st->stopped = 1;
      }
      st->status = status;
      if (status != FOA_DMD_OK && a.batch) st->halt = 1;
      foa_dmd_push_info inf;
      inf.h_last = nu;
      inf.indicator = __longlong_as_double(0x7ff8000000000000ll);
      inf.x_norm = xn;
      inf.q = st->q;
      inf.status = status;
      st->info = inf;
      if (a.info_out) *a.info_out = inf;
    }
  } else if constexpr (MODE == PASS_FIRST) {
    if (tid == 0) {
      const double b = sqrt(dot[0]);
      int status;
      if (!isfinite(b)) status = FOA_DMD_ENONFINITE;
      else if (!(b > 0.0)) status = FOA_DMD_EBREAKDOWN;
      else status = FOA_DMD_OK;
      if (status == FOA_DMD_OK) {
        a.B[0] = b;  // beta_11 = ||psi_1||
        st->nu = b;
        st->inv_nu = 1.0 / b;
        st->q = 1;
      } else if (status == FOA_DMD_EBREAKDOWN) {
        st->stopped = 1;
      }
      st->x_norm = b;
      st->status = status;
      if (status != FOA_DMD_OK && a.batch) st->halt = 1;
      foa_dmd_push_info inf;
      inf.h_last = b;
      inf.indicator = __longlong_as_double(0x7ff8000000000000ll);
      inf.x_norm = b;
      inf.q = st->q;
      inf.status = status;
      st->info = inf;
      if (a.info_out) *a.info_out = inf;
    }
  }
}

// Two CTAs per SM for the FP32/BF16 forms while the column accumulators fit (NC <= 48, i.e.
// j <= 384): one CTA's barrier phases then overlap the other's compute.
template <typename S, int NC>
constexpr int pass_min_blocks() {
  return (sizeof(typename Compute<S>::T) == 4 && NC <= 48) ? 2 : 1;
}

template <typename S, int MODE, int NC>
__global__ void __launch_bounds__(kThreads, pass_min_blocks<S, NC>()) pass_kernel(const PassArgs a) {
  using C = typename Compute<S>::T;
  constexpr bool kFp64 = sizeof(C) == 8;
  constexpr bool kDots = (MODE == PASS_A || MODE == PASS_B || MODE == PASS_B2);
  constexpr bool kNorm = (MODE == PASS_A || MODE == PASS_C || MODE == PASS_FIRST || MODE == PASS_B2);
  constexpr bool kBaseX = (MODE == PASS_A || MODE == PASS_FIRST);
  using BaseT = typename std::conditional<kBaseX, S, C>::type;

  extern __shared__ __align__(128) unsigned char smem[];
  DevState *st = a.st;
  if (!st->active) return;
  const int j = (MODE == PASS_FIRST) ? 0 : st->j;
  if (MODE != PASS_FIRST && (j < 1 || j > a.jcap)) return;
  if (MODE == PASS_FIRST && st->j != 0) return;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  unsigned char *slots = smem;
  C *wsb = reinterpret_cast<C *>(smem + a.off_ws);  // 2 x R*32 entries
  C *cf = reinterpret_cast<C *>(smem + a.off_coef);
  double *dot = reinterpret_cast<double *>(smem + a.off_dot);
  double *comb = reinterpret_cast<double *>(smem + a.off_comb);
  double *nrm = reinterpret_cast<double *>(smem + a.off_norm);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.off_bar);
  uint64_t *empty = full + kMaxSlots;
  volatile int *sflag = reinterpret_cast<volatile int *>(empty + kMaxSlots);  // [0] abort [1] issued [2] last

  // QR view (a.form): pass A projects x itself (w = x, no pre-vector)
  const bool qr_a = (MODE == PASS_A) && a.form != 0;
  const double cscale = (MODE == PASS_A && !qr_a) ? st->inv_bjj : 1.0;
  if (tid == 0) {
    for (int i = 0; i < a.slots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kWarps);  // every consumer warp releases the slot after its column sweep
    }
    sflag[0] = 0;
    sflag[1] = 0;
    sflag[2] = 0;
    mbar_fence_init();
  }
  for (int c = tid; c < ((j + 7) & ~3); c += kThreads) cf[c] = c < j ? static_cast<C>(a.coef[c]) : C(0);
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
        if (it >= a.slots) {
          if (!mbar_wait(&empty[slot], ((it / a.slots) - 1) & 1)) {
            sflag[0] = 1;
            atomicExch(&st->err, FOA_DMD_ETIMEOUT);
            break;
          }
        }
        if (sflag[0]) break;
        const int t0 = s * a.R;
        const int nt = min(a.R, a.ntiles - t0);
        const int64_t r0 = int64_t(t0) * kTile;
        const bool base_bulk = kBaseX ? (a.x_aligned && r0 + int64_t(nt) * kTile <= a.n) : true;
        const uint32_t bbytes = base_bulk ? uint32_t(nt) * kTile * sizeof(BaseT) : 0u;
        unsigned char *dst = slots + size_t(slot) * a.slot_bytes;
        mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * tile_bytes + bbytes);
        if (tile_bytes) {
          if (FOA_CHECK(t0 >= 0 && t0 + nt <= a.ntiles, kChkTile))
            for (int k = 0; k < nt; ++k)
              bulk_g2s(dst + size_t(k) * tile_bytes, Vg + int64_t(t0 + k) * tile_elems, tile_bytes, &full[slot]);
        }
        if (bbytes) bulk_g2s(dst + a.base_off, baseg + r0, bbytes, &full[slot]);
        sflag[1] = it + 1;
      }
    }
    return;
  }

  // ------------------------------------------------------------------ consumer warps
  constexpr int NACC = kFp64 ? NC : (NC + 1) / 2;
  C acc[kDots ? NACC : 1];
#pragma unroll
  for (int k = 0; k < (kDots ? NACC : 1); ++k) acc[k] = C(0);
  // sum of squares for the norms: compensated (Kahan) in the compute type per thread, folded into
  // FP64 once at the end
  C nsum = C(0), ncomp = C(0);
  auto nrm_add = [&](C v) {
    const C y = v - ncomp;
    const C t = nsum + y;
    ncomp = (t - nsum) - y;
    nsum = t;
  };
  int since_flush = 0;
  int it = 0;

  auto flush = [&]() {
    if constexpr (kDots) {
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
          if (warp + kWarps * (2 * kk) < j) {  // warp-uniform: at least the first half-warp's column exists
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


  for (int s = blockIdx.x; s < a.nstages; s += gridDim.x, ++it) {
    const int slot = it % a.slots;
    // Every thread waits for the stage itself.  A wait that runs out records the error and the
    // CTA carries on (its results are discarded by the host); the barrier sequence stays the same
    // for all threads, and after the first timeout no thread waits again, so nothing can hang.
    if (!sflag[0] && !mbar_wait(&full[slot], (it / a.slots) & 1)) {
      sflag[0] = 1;
      atomicExch(&st->err, FOA_DMD_ETIMEOUT);
    }
    C *ws = wsb + (it & 1) * (a.R * kTile);  // double buffer: the next row sweep may start early
    const int t0 = s * a.R;
    const int nt = min(a.R, a.ntiles - t0);
    const int RS = nt * kTile;
    const int64_t r0 = int64_t(t0) * kTile;
    const unsigned char *sbase = slots + size_t(slot) * a.slot_bytes;
    const S *vs = reinterpret_cast<const S *>(sbase);
    const bool base_bulk = kBaseX ? (a.x_aligned && r0 + int64_t(RS) <= a.n) : true;
    const BaseT *bs = reinterpret_cast<const BaseT *>(sbase + a.base_off);
    const BaseT *bg = kBaseX ? static_cast<const BaseT *>(a.x) : static_cast<const BaseT *>(a.w);

    // ---------------- sweep 1: row-local part
    auto finish_row = [&](int row, C acc) {
      const int64_t r = r0 + row;
      C base;
      if (base_bulk) base = to_c(bs[row]);
      else base = (r < a.n) ? C(to_c(bg[r])) : C(0);
      if constexpr (MODE == PASS_FIRST) {
        nrm_add(base * base);
      } else {
        const C wc = (MODE == PASS_A) ? (base - acc) * C(cscale) : (base - acc);
        static_cast<C *>(a.w)[r] = wc;
        ws[row] = wc;
        if constexpr (MODE == PASS_A) nrm_add(base * base);
        else if constexpr (MODE == PASS_C || MODE == PASS_B2) nrm_add(wc * wc);
      }
    };
    if (qr_a) {
      for (int row = tid; row < RS; row += kConsumers) finish_row(row, C(0));
    } else {
      if constexpr (kFp64) {
        const int G = (RS >= kConsumers || j == 0) ? 1 : (kConsumers / RS);
        const int active_rows_threads = (G == 1) ? kConsumers : G * RS;
        if (tid < active_rows_threads) {
          const int g = (G == 1) ? 0 : tid / RS;
          const int cpg = (j + G - 1) / G;
          const int c0 = g * cpg;
          const int c1 = min(j, c0 + cpg);
          for (int row = (G == 1 ? tid : tid % RS); row < RS; row += (G == 1 ? kConsumers : RS)) {
            const S *vr = vs + (row >> 5) * (kTile * j) + (row & 31);
            double accd = 0.0;
            float accf = 0.f;
            if constexpr (kFp64) {
              double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
              int c = c0;
              for (; c + 4 <= c1; c += 4) {
                b0 = fma(to_c(vr[(c + 0) * kTile]), cf[c + 0], b0);
                b1 = fma(to_c(vr[(c + 1) * kTile]), cf[c + 1], b1);
                b2 = fma(to_c(vr[(c + 2) * kTile]), cf[c + 2], b2);
                b3 = fma(to_c(vr[(c + 3) * kTile]), cf[c + 3], b3);
              }
              for (; c < c1; ++c) b0 = fma(to_c(vr[c * kTile]), cf[c], b0);
              accd = (b0 + b1) + (b2 + b3);
            } else {
              // FP32: four independent chains over the thread's columns (no FP64 in the row loop:
              // the FP64 pipe of this part is ~1/64 of FP32)
              float b[8];
    #pragma unroll
              for (int u = 0; u < 8; ++u) b[u] = 0.f;
              int c = c0;
              for (; c + 8 <= c1; c += 8) {
                float v[8];
    #pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = to_c(vr[(c + u) * kTile]);
    #pragma unroll
                for (int u = 0; u < 8; ++u) b[u] = fmaf(v[u], cf[c + u], b[u]);
              }
    #pragma unroll
              for (int u = 0; u < 8; ++u)
                if (c + u < c1) b[u] = fmaf(to_c(vr[(c + u) * kTile]), cf[c + u], b[u]);
              accf = ((b[0] + b[1]) + (b[2] + b[3])) + ((b[4] + b[5]) + (b[6] + b[7]));
            }
            if (G > 1) {
              if constexpr (kFp64) comb[g * RS + row] = accd;
              else reinterpret_cast<float *>(comb)[g * RS + row] = accf;
            } else {
              // finish the row here
              const int64_t r = r0 + row;
              C base;
              if (base_bulk) base = to_c(bs[row]);
              else base = (r < a.n) ? C(to_c(bg[r])) : C(0);
              if constexpr (MODE == PASS_FIRST) {
                nrm_add(base * base);
              } else {
                const C acc = kFp64 ? C(accd) : C(accf);
                const C wc = (MODE == PASS_A) ? (base - acc) * C(cscale) : (base - acc);
                static_cast<C *>(a.w)[r] = wc;
                ws[row] = wc;
                if constexpr (MODE == PASS_A) nrm_add(base * base);
                else if constexpr (MODE == PASS_C || MODE == PASS_B2) nrm_add(wc * wc);
              }
            }
          }
        }
        if (G > 1) {
          named_bar_sync(1, kConsumers);
          if (tid < RS) {
            const int row = tid;
            C acc = C(0);
            if constexpr (kFp64) {
              for (int g = 0; g < G; ++g) acc += comb[g * RS + row];
            } else {
              const float *cb = reinterpret_cast<const float *>(comb);
              for (int g = 0; g < G; ++g) acc += cb[g * RS + row];
            }
            const int64_t r = r0 + row;
            C base;
            if (base_bulk) base = to_c(bs[row]);
            else base = (r < a.n) ? C(to_c(bg[r])) : C(0);
            const C wc = (MODE == PASS_A) ? (base - acc) * C(cscale) : (base - acc);
            static_cast<C *>(a.w)[r] = wc;
            ws[row] = wc;
            if constexpr (MODE == PASS_A) nrm_add(base * base);
            else if constexpr (MODE == PASS_C || MODE == PASS_B2) nrm_add(wc * wc);
          }
        }

      } else {
        // FP32 / BF16 storage: a thread owns a pair of adjacent rows (one 8-byte or 4-byte load
        // gives both) and a group of columns; coefficients come as 16-byte broadcasts (cf is
        // zero padded), four FP32 chains per row.
        const int P = RS >> 1;
        const int G1 = (P >= kConsumers || j == 0) ? 1 : (kConsumers / P);
        float *cb = reinterpret_cast<float *>(comb);
        if (tid < (G1 == 1 ? kConsumers : G1 * P)) {
          const int g = (G1 == 1) ? 0 : tid / P;
          const int cpg = (((j + G1 - 1) / G1) + 3) & ~3;
          const int c0 = g * cpg;
          const int c1 = min(j, c0 + cpg);
          for (int pr = (G1 == 1 ? tid : tid % P); pr < P; pr += (G1 == 1 ? kConsumers : P)) {
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
            if (c < c1) {
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
          named_bar_sync(1, kConsumers);
          if (tid < RS) {
            float acc = 0.f;
            for (int g = 0; g < G1; ++g) acc += cb[g * RS + tid];
            finish_row(tid, acc);
          }
        }
      }
    }
    named_bar_sync(1, kConsumers);  // ws complete

    // ---------------- sweep 2: column dot products over the staged rows
    if constexpr (kDots) {
      if constexpr (kFp64) {
        for (int kt = 0; kt < nt; ++kt) {
          const C wv = ws[kt * kTile + lane];
          const S *vt = vs + kt * (kTile * j) + lane;
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const int c = warp + kWarps * k;
            if (c < j) acc[k] = fma(to_c(vt[c * kTile]), wv, acc[k]);
          }
        }
      } else {
        // half-warps take alternate columns of the warp's set; a lane covers two adjacent rows
        const int hl = lane & 15, half = lane >> 4;
        for (int kt = 0; kt < nt; ++kt) {
          const float2 wv = *reinterpret_cast<const float2 *>(ws + kt * kTile + 2 * hl);
          const S *vt = vs + kt * (kTile * j) + 2 * hl;
#pragma unroll
          for (int kk = 0; kk < NACC; ++kk) {
            const int c = warp + kWarps * (2 * kk + half);
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
      }
    }
    // this warp is done with the slot
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }
  flush();
  nrm[tid] = kNorm ? double(nsum) - double(ncomp) : 0.0;
  pass_epilogue<MODE>(a, st, dot, nrm, sflag, j, tid);
}

}  // namespace foa
