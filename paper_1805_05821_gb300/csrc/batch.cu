// Batched streams: one call advances every active stream of a batch by one push (Alg. 4 with
// p = 1 per stream) in a single cooperative persistent kernel launch, capturable in a CUDA graph.
//
// plan_kernel (1 CTA) reads every stream's device state and the caller's pointer array and
// builds the work list: phase 0 = beta_pre of each active stream (Alg. 1 steps 5-8), phases
// 1-3 = the streaming passes A, B, C (steps 9-15) cut into chunks of whole pipeline stages,
// phase 4 = the append of the new basis vector (step 15).  The persistent kernel takes items
// from one global counter in list order.  An item of phase p of stream s waits (bounded) until
// stream s has finished phase p-1; because every item of phase p-1 precedes it in the list and
// all CTAs are co-resident, that wait always ends.  The last finisher of a (stream, phase) sums
// the chunk partials in chunk order (deterministic) and applies the scalar part of the step.
// Stage processing matches the single-stream pass kernel: bulk async copies of whole row tiles
// into a shared-memory double buffer, a row-local sweep and a column sweep per stage.
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.cuh"
#include "push_kernels.cuh"

namespace foa {
namespace bt {

constexpr int THREADS = 256;
constexpr int SLOT_V = 64 * 1024;     // V bytes per stage slot (one 32-row tile at k_max = 512, FP32)
constexpr int SLOT_B = 8 * 1024;      // base vector bytes per slot
constexpr int SLOTS = 2;
constexpr int MAX_R = 64;
constexpr int64_t CHUNK_BYTES = 16ll << 20;  // V bytes per work item
constexpr int NC = 64;                // column accumulators per warp (k_max <= 512)

struct StreamDesc {
  int64_t n;
  int64_t v_off;    // element offset of the stream's V in the pool
  int64_t w_off;    // element offset of w
  int64_t mat_off;  // double offset of its k_max x k_max H-bar and beta
  int64_t vec_off;  // double offset of its pre/h/s vectors (3 x k_max)
  int64_t part_off; // double offset of its chunk partials
  int32_t ntiles;
  int32_t kmax;
  int32_t max_chunks;
  int32_t pad;
};

struct BState {
  int32_t q, j, active, stopped, status, err, first, pad;
  double bjj, inv_bjj, x_norm, nu, inv_nu, h_last;
};

struct Plan {
  int32_t R, nstages, cs, nchunks;  // per stream (tiles per stage, stages, stages per chunk, chunks)
};

struct BatchArgs {
  const StreamDesc *sd;
  BState *st;
  Plan *plan;
  int32_t *offs;       // (5 * S + 1): item offsets, phase-major, stream-minor
  int32_t *total;
  uint32_t *counter;   // global work counter
  uint32_t *tickets;   // [S][5]
  int32_t *done;       // [S]: last finished phase (-1 before phase 0)
  void *V;             // pool (storage dtype)
  float *W;            // pool of w vectors (FP32)
  double *H, *B;       // pools
  double *vec;         // pools of pre/h/s
  double *part;        // chunk partials
  const void *const *x;  // caller's pointers (device array of S)
  double *h_last;      // caller's output array (device, S)
  double tol;
  int32_t S;
  int32_t *err;        // sticky
};

template <typename S>
__device__ __forceinline__ float ldc(const S *p, int64_t i) {
  return to_c(p[i]);
}

// ---------------------------------------------------------------------------- plan
__global__ void plan_kernel(BatchArgs a, int ssize) {
  const int S = a.S;
  extern __shared__ int32_t cnt[];  // 5 * S counts
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const StreamDesc d = a.sd[s];
    BState &b = a.st[s];
    const bool has_x = a.x[s] != nullptr;
    const int q = b.q;
    int active = has_x && !b.stopped && q < d.kmax;
    b.active = active;
    b.j = q;
    b.first = (q == 0) ? 1 : 0;
    if (active) b.status = -1;
    else if (has_x) b.status = b.stopped ? FOA_DMD_ESTOPPED : FOA_DMD_EFULL;
    if (a.h_last) a.h_last[s] = __longlong_as_double(0x7ff8000000000000ll);
    const int j = q;
    const int64_t tb = int64_t(kTile) * (j > 0 ? j : 0) * ssize;
    int R = MAX_R;
    if (j > 0) {
      R = 1;
      while (R * 2 <= MAX_R && int64_t(R * 2) * tb <= SLOT_V) R *= 2;
    }
    Plan p;
    p.R = R;
    p.nstages = (d.ntiles + R - 1) / R;
    const int64_t stage_bytes = j > 0 ? int64_t(R) * tb : int64_t(R) * kTile * ssize;
    int cs = int(CHUNK_BYTES / (stage_bytes > 0 ? stage_bytes : 1));
    if (cs < 1) cs = 1;
    p.cs = cs;
    p.nchunks = (p.nstages + cs - 1) / cs;
    if (p.nchunks > d.max_chunks) {  // keep within the partials buffer
      p.cs = (p.nstages + d.max_chunks - 1) / d.max_chunks;
      p.nchunks = (p.nstages + p.cs - 1) / p.cs;
    }
    a.plan[s] = p;
    const bool first = (j == 0);
    cnt[0 * S + s] = (active && !first) ? 1 : 0;                 // beta_pre
    cnt[1 * S + s] = active ? p.nchunks : 0;                     // pass A (or the first-snapshot norm)
    cnt[2 * S + s] = (active && !first) ? p.nchunks : 0;         // pass B
    cnt[3 * S + s] = (active && !first) ? p.nchunks : 0;         // pass C
    cnt[4 * S + s] = active ? p.nchunks : 0;                     // append
    a.done[s] = (active && !first) ? -1 : 0;  // streams without a beta_pre item start at phase 1
    for (int ph = 0; ph < 5; ++ph) a.tickets[s * 5 + ph] = 0u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int i = 0; i < 5 * S; ++i) {
      a.offs[i] = run;
      run += cnt[i];
    }
    a.offs[5 * S] = run;
    *a.total = run;
    *a.counter = 0u;
  }
}

// ---------------------------------------------------------------------------- helpers
__device__ __forceinline__ double block_sum_d(double v, double *red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < THREADS / 32; ++i) t += red[i];
  __syncthreads();
  return t;
}

// spin (bounded) until stream s has finished phase p-1
__device__ bool wait_phase(const BatchArgs &a, int s, int p) {
  volatile int32_t *d = a.done + s;
  if (*d >= p - 1) return true;
  const long long t0 = clock64();
  while (*d < p - 1) {
    if (clock64() - t0 > (1ll << 33)) return false;
    __nanosleep(200);
  }
  return true;
}

template <typename S>
__global__ void __launch_bounds__(THREADS, 1) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *slotmem = smem;                                          // SLOTS x (SLOT_V + SLOT_B)
  float *ws = reinterpret_cast<float *>(smem + SLOTS * (SLOT_V + SLOT_B));  // MAX_R*32
  float *cf = ws + MAX_R * kTile;                                         // kMaxK
  double *dot = reinterpret_cast<double *>(cf + kMaxK);                   // kMaxK + 1
  double *comb = dot + kMaxK + 2;                                         // 256
  double *red = comb + THREADS;                                           // 32
  __shared__ uint64_t full[SLOTS];
  __shared__ int s_item, s_stream, s_phase, s_chunk, s_last, s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < SLOTS; ++i) mbar_init(&full[i], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const int S_ = a.S;
  const int total = *a.total;
  uint32_t it = 0;  // stages consumed by this CTA (mbarrier phase tracking)
  while (true) {
    __syncthreads();  // everyone is done with the previous item's descriptors
    if (tid == 0) {
      const int item = int(atomicAdd(a.counter, 1u));
      s_item = item;
      s_fail = 0;
      if (item < total) {
        // phase and stream by binary search over the item offsets
        int lo = 0, hi = 5 * S_;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (a.offs[mid] <= item) lo = mid;
          else hi = mid;
        }
        while (lo + 1 <= 5 * S_ && a.offs[lo + 1] <= item) ++lo;  // skip empty entries
        s_phase = lo / S_;
        s_stream = lo % S_;
        s_chunk = item - a.offs[lo];
        if (!wait_phase(a, s_stream, s_phase)) {
          s_fail = 1;
          atomicExch(a.err, FOA_DMD_ETIMEOUT);
        }
        __threadfence();  // acquire: the finished phase's results are visible below
      }
    }
    __syncthreads();
    if (s_item >= total || s_fail) break;
    const int sidx = s_stream, ph = s_phase, chunk = s_chunk;
    const StreamDesc d = a.sd[sidx];
    BState *bs = a.st + sidx;
    const Plan pl = a.plan[sidx];
    const int j = __ldcg(&bs->j);
    const bool first = __ldcg(&bs->first) != 0;
    const int K = d.kmax;
    double *Hs = a.H + d.mat_off, *Bs = a.B + d.mat_off;
    double *pre = a.vec + d.vec_off, *hv = pre + K, *sv = hv + K;
    S *Vs = static_cast<S *>(a.V) + d.v_off;
    float *w = a.W + d.w_off;
    const S *x = static_cast<const S *>(a.x[sidx]);
    const int64_t nrows = int64_t(d.ntiles) * kTile;

    if (ph == 0) {
      // ---------------------------------------------------------------- beta_pre (steps 5-8)
      if (tid == 0) {
        bs->bjj = Bs[int64_t(j - 1) * (K + 1)];
        bs->inv_bjj = 1.0 / bs->bjj;
      }
      for (int i = warp; i < j; i += THREADS / 32) {
        const int l0 = i == 0 ? 0 : i - 1;
        double acc = 0.0;
        for (int l = l0 + lane; l <= j - 2; l += 32) acc += Hs[i + int64_t(l) * K] * Bs[l + int64_t(j - 1) * K];
        acc = warp_sum(acc);
        if (lane == 0) pre[i] = acc;
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicExch(a.done + sidx, 0);
      continue;
    }
    const int s0 = chunk * pl.cs;
    const int s1 = min(pl.nstages, s0 + pl.cs);
    if (ph == 4) {
      // ---------------------------------------------------------------- append v_{j+1} (step 15)
      if (__ldcg(&bs->status) == FOA_DMD_OK) {
        const int64_t r0 = int64_t(s0) * pl.R * kTile, r1 = min(nrows, int64_t(s1) * pl.R * kTile);
        const float sc = float(__ldcg(&bs->inv_nu));
        for (int64_t r = r0 + tid; r < r1; r += THREADS) {
          const float v = first ? ((r < d.n) ? ldc(x, r) : 0.f) : w[r];
          Vs[((r >> 5) * K + j) * kTile + (r & 31)] = Store<S>::from(v * sc);
        }
      }
      continue;
    }
    // ---------------------------------------------------------------- streaming pass (A, B, C)
    const int mode = first ? PASS_FIRST : (ph == 1 ? PASS_A : ph == 2 ? PASS_B : PASS_C);
    const bool dots = (mode == PASS_A || mode == PASS_B);
    const int jj = first ? 0 : j;
    const double *coef = (mode == PASS_A) ? pre : (mode == PASS_B) ? hv : sv;
    const double cscale = (mode == PASS_A) ? __ldcg(&bs->inv_bjj) : 1.0;
    for (int c = tid; c < jj; c += THREADS) cf[c] = float(__ldcg(coef + c));
    for (int c = tid; c <= jj; c += THREADS) dot[c] = 0.0;
    float acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.f;
    double nacc = 0.0;
    int since_flush = 0;
    const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(jj) * sizeof(S);
    const bool base_x = (mode == PASS_A || mode == PASS_FIRST);
    const bool x_aligned = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    __syncthreads();
    auto issue = [&](int stage, int slot) {
      const int t0 = stage * pl.R;
      const int nt = min(pl.R, d.ntiles - t0);
      const int64_t r0 = int64_t(t0) * kTile;
      unsigned char *dst = slotmem + size_t(slot) * (SLOT_V + SLOT_B);
      const bool bb = base_x ? (x_aligned && r0 + int64_t(nt) * kTile <= d.n) : true;
      const uint32_t bbytes = bb ? uint32_t(nt) * kTile * (base_x ? sizeof(S) : 4) : 0u;
      mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * tile_bytes + bbytes);
      if (tile_bytes)
        for (int k = 0; k < nt; ++k)
          bulk_g2s(dst + size_t(k) * tile_bytes, Vs + (int64_t(t0 + k) * K) * kTile, tile_bytes, &full[slot]);
      if (bbytes) {
        if (base_x) bulk_g2s(dst + SLOT_V, x + r0, bbytes, &full[slot]);
        else bulk_g2s(dst + SLOT_V, w + r0, bbytes, &full[slot]);
      }
    };
    if (tid == 0) {
      for (int k = 0; k < SLOTS && s0 + k < s1; ++k) issue(s0 + k, int((it + k) % SLOTS));
    }
    for (int stg = s0; stg < s1; ++stg, ++it) {
      const int slot = int(it % SLOTS);
      const int bad = mbar_wait(&full[slot], (it / SLOTS) & 1) ? 0 : 1;
      if (__syncthreads_or(bad)) {
        if (tid == 0) atomicExch(a.err, FOA_DMD_ETIMEOUT);
        return;  // the handle is unusable after a timeout
      }
      const int t0 = stg * pl.R;
      const int nt = min(pl.R, d.ntiles - t0);
      const int RS = nt * kTile;
      const int64_t r0 = int64_t(t0) * kTile;
      const unsigned char *sb = slotmem + size_t(slot) * (SLOT_V + SLOT_B);
      const S *vs = reinterpret_cast<const S *>(sb);
      const bool bb = base_x ? (x_aligned && r0 + int64_t(RS) <= d.n) : true;
      // sweep 1
      const int G = (RS >= THREADS || jj == 0) ? 1 : (THREADS / RS);
      float nst = 0.f;
      if (tid < (G == 1 ? THREADS : G * RS)) {
        const int g = (G == 1) ? 0 : tid / RS;
        const int cpg = (jj + G - 1) / G;
        const int c0 = g * cpg, c1 = min(jj, c0 + cpg);
        for (int row = (G == 1 ? tid : tid % RS); row < RS; row += (G == 1 ? THREADS : RS)) {
          const S *vr = vs + (row >> 5) * (kTile * jj) + (row & 31);
          double accd = 0.0;
          for (int cb = c0; cb < c1; cb += 32) {
            const int ce = min(c1, cb + 32);
            float b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
            int c = cb;
            for (; c + 4 <= ce; c += 4) {
              b0 = fmaf(to_c(vr[(c + 0) * kTile]), cf[c + 0], b0);
              b1 = fmaf(to_c(vr[(c + 1) * kTile]), cf[c + 1], b1);
              b2 = fmaf(to_c(vr[(c + 2) * kTile]), cf[c + 2], b2);
              b3 = fmaf(to_c(vr[(c + 3) * kTile]), cf[c + 3], b3);
            }
            for (; c < ce; ++c) b0 = fmaf(to_c(vr[c * kTile]), cf[c], b0);
            accd += double((b0 + b1) + (b2 + b3));
          }
          if (G > 1) {
            comb[g * RS + row] = accd;
          } else {
            const int64_t r = r0 + row;
            double base;
            if (base_x) base = bb ? double(to_c(reinterpret_cast<const S *>(sb + SLOT_V)[row]))
                                  : ((r < d.n) ? double(ldc(x, r)) : 0.0);
            else base = double(reinterpret_cast<const float *>(sb + SLOT_V)[row]);
            if (mode == PASS_FIRST) {
              const float xv = float(base);
              nst = fmaf(xv, xv, nst);
            } else {
              const double wn = (mode == PASS_A) ? (base - accd) * cscale : (base - accd);
              const float wc = float(wn);
              w[r] = wc;
              ws[row] = wc;
              if (mode == PASS_A) {
                const float xv = float(base);
                nst = fmaf(xv, xv, nst);
              } else if (mode == PASS_C) {
                nst = fmaf(wc, wc, nst);
              }
            }
          }
        }
      }
      if (G > 1) {
        __syncthreads();
        if (tid < RS) {
          double accd = 0.0;
          for (int g = 0; g < G; ++g) accd += comb[g * RS + tid];
          const int64_t r = r0 + tid;
          double base;
          if (base_x) base = bb ? double(to_c(reinterpret_cast<const S *>(sb + SLOT_V)[tid]))
                                : ((r < d.n) ? double(ldc(x, r)) : 0.0);
          else base = double(reinterpret_cast<const float *>(sb + SLOT_V)[tid]);
          const double wn = (mode == PASS_A) ? (base - accd) * cscale : (base - accd);
          const float wc = float(wn);
          w[r] = wc;
          ws[tid] = wc;
          if (mode == PASS_A) {
            const float xv = float(base);
            nst = fmaf(xv, xv, nst);
          } else if (mode == PASS_C) {
            nst = fmaf(wc, wc, nst);
          }
        }
      }
      nacc += double(nst);
      __syncthreads();
      // sweep 2
      if (dots) {
        for (int kt = 0; kt < nt; ++kt) {
          const float wv = ws[kt * kTile + lane];
          const S *vt = vs + kt * (kTile * jj) + lane;
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const int c = warp + (THREADS / 32) * k;
            if (c < jj) acc[k] = fmaf(to_c(vt[c * kTile]), wv, acc[k]);
          }
        }
        since_flush += nt;
        if (since_flush >= 32) {
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const int c = warp + (THREADS / 32) * k;
            if (c < jj) {
              const float v = warp_sum(acc[k]);
              if (lane == 0) dot[c] += double(v);
              acc[k] = 0.f;
            }
          }
          since_flush = 0;
        }
      }
      __syncthreads();
      if (tid == 0 && stg + SLOTS < s1) issue(stg + SLOTS, slot);
    }
    // flush and write this chunk's partial
    if (dots) {
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const int c = warp + (THREADS / 32) * k;
        if (c < jj) {
          const float v = warp_sum(acc[k]);
          if (lane == 0) dot[c] += double(v);
        }
      }
    }
    const double ntot = block_sum_d(nacc, red);
    if (tid == 0) dot[jj] = ntot;
    __syncthreads();
    double *pp = a.part + d.part_off + int64_t(chunk) * (K + 1);
    for (int c = tid; c <= jj; c += THREADS) pp[c] = dot[c];
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned t = atomicAdd(a.tickets + sidx * 5 + ph, 1u);
      s_last = (t == unsigned(pl.nchunks - 1)) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) continue;
    __threadfence();
    // ------------------------------------------------------------------ last chunk: reduce + scalar part
    for (int c = tid; c <= jj; c += THREADS) {
      double t = 0.0;
      for (int b = 0; b < pl.nchunks; ++b) t += __ldcg(a.part + d.part_off + int64_t(b) * (K + 1) + c);
      dot[c] = t;
    }
    __syncthreads();
    if (mode == PASS_A) {
      for (int c = tid; c < jj; c += THREADS) hv[c] = dot[c];
      if (tid == 0) bs->x_norm = sqrt(dot[jj]);
    } else if (mode == PASS_B) {
      for (int c = tid; c < jj; c += THREADS) {
        sv[c] = dot[c];
        hv[c] = __ldcg(hv + c) + dot[c];
      }
    } else if (mode == PASS_C) {
      const double nu = sqrt(dot[jj]);
      const double xn = __ldcg(&bs->x_norm), bjj = __ldcg(&bs->bjj);
      int status;
      if (!isfinite(nu) || !isfinite(xn)) status = FOA_DMD_ENONFINITE;
      else if (!(nu * bjj > a.tol * xn)) status = FOA_DMD_EBREAKDOWN;
      else status = FOA_DMD_OK;
      if (status != FOA_DMD_ENONFINITE)
        for (int c = tid; c < jj; c += THREADS) Hs[c + int64_t(jj - 1) * K] = __ldcg(hv + c);
      if (status == FOA_DMD_OK)
        for (int c = tid; c < jj; c += THREADS) Bs[c + int64_t(jj) * K] = __ldcg(pre + c) + __ldcg(hv + c) * bjj;
      __syncthreads();
      if (tid == 0) {
        if (status == FOA_DMD_OK) {
          Hs[jj + int64_t(jj - 1) * K] = nu;
          Bs[jj + int64_t(jj) * K] = nu * bjj;
          bs->nu = nu;
          bs->inv_nu = 1.0 / nu;
          bs->q = jj + 1;
          if (a.h_last) a.h_last[sidx] = nu;
        } else if (status == FOA_DMD_EBREAKDOWN) {
          Hs[jj + int64_t(jj - 1) * K] = 0.0;
          bs->stopped = 1;
        }
        bs->h_last = nu;
        bs->status = status;
      }
    } else {  // first snapshot
      if (tid == 0) {
        const double b = sqrt(dot[0]);
        int status = !isfinite(b) ? FOA_DMD_ENONFINITE : (!(b > 0.0) ? FOA_DMD_EBREAKDOWN : FOA_DMD_OK);
        if (status == FOA_DMD_OK) {
          Bs[0] = b;
          bs->inv_nu = 1.0 / b;
          bs->nu = b;
          bs->q = 1;
          if (a.h_last) a.h_last[sidx] = b;
        } else if (status == FOA_DMD_EBREAKDOWN) {
          bs->stopped = 1;
        }
        bs->x_norm = b;
        bs->h_last = b;
        bs->status = status;
      }
    }
    __threadfence();
    __syncthreads();
    // first snapshot: passes B and C do not exist, so completing the norm completes phase 3
    if (tid == 0) atomicExch(a.done + sidx, (mode == PASS_FIRST) ? 3 : ph);
  }
}

}  // namespace bt
}  // namespace foa

using namespace foa;
using namespace foa::bt;

struct foa_dmd_batch {
  int S = 0, dtype = 0, sms = 0;
  cudaStream_t stream = nullptr;
  double tol = 0.0;
  std::vector<StreamDesc> sd_host;
  StreamDesc *sd = nullptr;
  BState *st = nullptr;
  Plan *plan = nullptr;
  int32_t *offs = nullptr, *total = nullptr, *done = nullptr, *err = nullptr;
  uint32_t *counter = nullptr, *tickets = nullptr;
  void *V = nullptr;
  float *W = nullptr;
  double *H = nullptr, *B = nullptr, *vec = nullptr, *part = nullptr;
  size_t smem = 0;
};

static void batch_free(foa_dmd_batch *b) {
  void *ptrs[] = {b->sd, b->st, b->plan, b->offs, b->total, b->done, b->err, b->counter, b->tickets, b->V, b->W,
                  b->H, b->B, b->vec, b->part};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

extern "C" int foa_dmd_batch_create(int32_t S, const int64_t *n, const int32_t *k_max, int32_t dtype,
                                    const foa_dmd_opts *opts, foa_dmd_batch_t **out) {
  if (!out) return FOA_DMD_EINVAL;
  *out = nullptr;
  if (S < 1 || !n || !k_max || (dtype != FOA_DMD_F32 && dtype != FOA_DMD_BF16)) return FOA_DMD_EINVAL;
  for (int s = 0; s < S; ++s)
    if (n[s] < 1 || k_max[s] < 2 || k_max[s] > kMaxK) return FOA_DMD_EINVAL;
  int sms = 0;
  int rc = check_device(&sms);
  if (rc) return rc;
  foa_dmd_batch *b = new (std::nothrow) foa_dmd_batch();
  if (!b) return FOA_DMD_ENOMEM;
  b->S = S;
  b->dtype = dtype;
  b->sms = sms;
  foa_dmd_opts o;
  if (opts) o = *opts;
  else foa_dmd_opts_default(&o);
  b->stream = static_cast<cudaStream_t>(o.cuda_stream);
  b->tol = o.breakdown_tol > 0.0 ? o.breakdown_tol : default_tol(dtype);
  const int es = dtype_size(dtype);
  int64_t voff = 0, woff = 0, moff = 0, vecoff = 0, poff = 0;
  b->sd_host.resize(S);
  for (int s = 0; s < S; ++s) {
    StreamDesc &d = b->sd_host[s];
    d.n = n[s];
    d.kmax = k_max[s];
    d.ntiles = int32_t((n[s] + kTile - 1) / kTile);
    const int64_t nrows = int64_t(d.ntiles) * kTile;
    d.v_off = voff;
    voff += nrows * d.kmax + 64;  // keep every stream's V 128-byte aligned
    voff = (voff + 63) / 64 * 64;
    d.w_off = woff;
    woff += nrows + 32;
    woff = (woff + 31) / 32 * 32;
    d.mat_off = moff;
    moff += int64_t(d.kmax) * d.kmax;
    d.vec_off = vecoff;
    vecoff += 3 * int64_t(d.kmax);
    d.max_chunks = int32_t(int64_t(nrows) * d.kmax * es / CHUNK_BYTES + 2);
    d.part_off = poff;
    poff += int64_t(d.max_chunks) * (d.kmax + 1);
    d.pad = 0;
  }
  cudaError_t e = cudaSuccess;
#define BAL(p, bytes)                                         \
  do {                                                        \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(p), (bytes)); \
  } while (0)
  BAL(b->sd, sizeof(StreamDesc) * S);
  BAL(b->st, sizeof(BState) * S);
  BAL(b->plan, sizeof(Plan) * S);
  BAL(b->offs, sizeof(int32_t) * (5 * S + 1));
  BAL(b->total, sizeof(int32_t));
  BAL(b->done, sizeof(int32_t) * S);
  BAL(b->err, sizeof(int32_t));
  BAL(b->counter, sizeof(uint32_t));
  BAL(b->tickets, sizeof(uint32_t) * 5 * S);
  BAL(b->V, size_t(voff) * es);
  BAL(b->W, size_t(woff) * 4);
  BAL(b->H, size_t(moff) * 8);
  BAL(b->B, size_t(moff) * 8);
  BAL(b->vec, size_t(vecoff) * 8);
  BAL(b->part, size_t(poff) * 8);
#undef BAL
  if (e == cudaSuccess) e = cudaMemcpy(b->sd, b->sd_host.data(), sizeof(StreamDesc) * S, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->st, 0, sizeof(BState) * S);
  if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(b->V, 0, size_t(voff) * es);
  if (e == cudaSuccess) e = cudaMemset(b->W, 0, size_t(woff) * 4);
  if (e == cudaSuccess) e = cudaMemset(b->H, 0, size_t(moff) * 8);
  if (e == cudaSuccess) e = cudaMemset(b->B, 0, size_t(moff) * 8);
  b->smem = size_t(SLOTS) * (SLOT_V + SLOT_B) + size_t(MAX_R) * kTile * 4 + size_t(kMaxK) * 4 +
            size_t(kMaxK + 2) * 8 + size_t(THREADS) * 8 + 32 * 8;
  if (e == cudaSuccess) {
    e = cudaFuncSetAttribute(dtype == FOA_DMD_F32 ? (const void *)batch_kernel<float>
                                                   : (const void *)batch_kernel<__nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(b->smem));
  }
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    return cuda_status(e);
  }
  *out = b;
  return FOA_DMD_OK;
}

extern "C" int foa_dmd_batch_push(foa_dmd_batch_t *b, const void *const *x_dev, double *h_last_dev) {
  if (!b || !x_dev) return FOA_DMD_EINVAL;
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.sd = b->sd;
  a.st = b->st;
  a.plan = b->plan;
  a.offs = b->offs;
  a.total = b->total;
  a.counter = b->counter;
  a.tickets = b->tickets;
  a.done = b->done;
  a.V = b->V;
  a.W = b->W;
  a.H = b->H;
  a.B = b->B;
  a.vec = b->vec;
  a.part = b->part;
  a.x = x_dev;
  a.h_last = h_last_dev;
  a.tol = b->tol;
  a.S = b->S;
  a.err = b->err;
  plan_kernel<<<1, 256, size_t(5) * b->S * 4, b->stream>>>(a, dtype_size(b->dtype));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  // one CTA per SM, all co-resident (cooperative launch), so the in-kernel phase waits always end
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->sms);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (b->dtype == FOA_DMD_F32) e = cudaLaunchKernelEx(&cfg, batch_kernel<float>, a);
  else e = cudaLaunchKernelEx(&cfg, batch_kernel<__nv_bfloat16>, a);
  return cuda_status(e);
}

extern "C" int foa_dmd_batch_get_state(foa_dmd_batch_t *b, int32_t s, int32_t *q, int32_t *status, double *Hbar,
                                       double *beta, int32_t ld) {
  if (!b || s < 0 || s >= b->S) return FOA_DMD_EINVAL;
  const StreamDesc &d = b->sd_host[s];
  if (ld < d.kmax) return FOA_DMD_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int32_t err = 0;
  BState st;
  e = cudaMemcpy(&err, b->err, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&st, b->st + s, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (err) return err;
  if (q) *q = st.q;
  if (status) *status = st.status;
  const int K = d.kmax;
  if (Hbar) e = cudaMemcpy2D(Hbar, size_t(ld) * 8, b->H + d.mat_off, size_t(K) * 8, size_t(K) * 8, K,
                             cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && beta)
    e = cudaMemcpy2D(beta, size_t(ld) * 8, b->B + d.mat_off, size_t(K) * 8, size_t(K) * 8, K, cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

extern "C" int foa_dmd_batch_get_basis(foa_dmd_batch_t *b, int32_t s, int32_t col0, int32_t ncols, void *dst_dev,
                                       int64_t ld) {
  if (!b || s < 0 || s >= b->S || !dst_dev) return FOA_DMD_EINVAL;
  const StreamDesc &d = b->sd_host[s];
  if (col0 < 0 || ncols < 0 || col0 + ncols > d.kmax || ld < d.n) return FOA_DMD_EINVAL;
  if (ncols == 0) return FOA_DMD_OK;
  const char *base = static_cast<const char *>(b->V) + size_t(d.v_off) * dtype_size(b->dtype);
  return cuda_status(launch_gather(b->dtype, base, dst_dev, ld, d.n, d.kmax, col0, ncols, b->sms, b->stream));
}

extern "C" void foa_dmd_batch_destroy(foa_dmd_batch_t *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
}
