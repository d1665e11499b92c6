// Batched streams: one call advances every active stream of a batch by one push (Alg. 4 with
// p = 1 per stream) in a single cooperative persistent kernel launch, capturable in a CUDA graph.
//
// plan_kernel (1 CTA) reads every stream's device state and the caller's pointer array and
// builds the work list: phase 0 = beta_pre of each active stream (Alg. 1 steps 5-8), phases
// 1-3 = the streaming passes A, B, C (steps 9-15) cut into chunks of whole pipeline stages,
// phase 4 = the append of the new basis vector (step 15).  Items are taken from one global
// counter in list order (phase-major).  An item of phase p of stream s starts once stream s has
// finished phase p-1 (bounded wait); every item of phase p-1 precedes it in the list and all CTAs
// are co-resident, so that wait always ends.  The last finisher of a (stream, phase) sums the
// chunk partials in chunk order (deterministic) and applies the scalar part of the step.
//
// Inside a CTA the roles are those of the single-stream warp-specialised pass: warp 8 fetches
// items, waits for their dependencies, publishes them to the consumers through a two-deep item
// ring and streams their stages into a shared-memory slot ring with bulk async copies; warps 0-3
// make the row-local sweep of each stage, warps 4-7 the column dots of the previous one.  The
// producer runs ahead into the next item while the consumers finish the current one.
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.cuh"
#include "push_kernels.cuh"

namespace foa {
namespace bt {

constexpr int MAX_R = 64;             // tiles per stage
constexpr int SLOT_B = MAX_R * 32 * 4;  // base-vector bytes per slot (x or w of one stage)
constexpr int MAX_SLOTS = 4;
constexpr int NCB = 64;               // column accumulators per column-group lane (k_max <= 512)
constexpr int ROW_WARPS = 4, COL_WARPS = 4, ROW_THREADS = ROW_WARPS * 32;

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
  int32_t slot_v;      // V bytes per stage slot (a whole tile of the widest stream fits)
  int32_t nslots;      // slot ring depth
  int64_t chunk_bytes; // V bytes per work item
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
      while (R * 2 <= MAX_R && int64_t(R * 2) * tb <= a.slot_v) R *= 2;
    }
    Plan p;
    p.R = R;
    p.nstages = (d.ntiles + R - 1) / R;
    const int64_t stage_bytes = j > 0 ? int64_t(R) * tb : int64_t(R) * kTile * ssize;
    int cs = int(a.chunk_bytes / (stage_bytes > 0 ? stage_bytes : 1));
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
struct Item {
  int32_t valid, stream, phase, chunk;
};

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

// Decode an item index into (phase, stream, chunk) by binary search over the item offsets.
__device__ void decode_item(const BatchArgs &a, int item, int &phase, int &stream, int &chunk) {
  const int S = a.S;
  int lo = 0, hi = 5 * S;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.offs[mid] <= item) lo = mid;
    else hi = mid;
  }
  while (lo + 1 <= 5 * S && a.offs[lo + 1] <= item) ++lo;  // skip empty entries
  phase = lo / S;
  stream = lo % S;
  chunk = item - a.offs[lo];
}

template <typename S>
__global__ void __launch_bounds__(kThreads, 1) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int slot_bytes = a.slot_v + SLOT_B;
  unsigned char *slotmem = smem;                                                    // nslots x slot
  float *wsb = reinterpret_cast<float *>(smem + size_t(a.nslots) * slot_bytes);    // 2 x MAX_R*32
  float *cf = wsb + 2 * MAX_R * kTile;                                              // kMaxK + 8
  double *dot = reinterpret_cast<double *>(cf + kMaxK + 8);                         // kMaxK + 2
  float *combb = reinterpret_cast<float *>(dot + kMaxK + 2);                        // 2 x 256
  double *nrm = reinterpret_cast<double *>(combb + 512);                            // 256
  __shared__ uint64_t full[MAX_SLOTS], empty[MAX_SLOTS], ws_full[2], ws_empty[2], item_full[2], item_empty[2];
  __shared__ Item ring[2];
  __shared__ int s_abort, s_last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < a.nslots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ws_full[b], ROW_WARPS);
      mbar_init(&ws_empty[b], COL_WARPS);
      mbar_init(&item_full[b], 1);
      mbar_init(&item_empty[b], 1);
    }
    s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const int total = *a.total;
  auto fail = [&]() {
    s_abort = 1;
    atomicExch(a.err, FOA_DMD_ETIMEOUT);
  };

  if (warp == kWarps) {
    // ---------------------------------------------------------------- producer warp
    if (lane != 0) return;
    uint32_t it = 0;  // stages issued
    for (int k = 0;; ++k) {
      const int r = k & 1;
      if (k >= 2 && !mbar_wait(&item_empty[r], ((k >> 1) - 1) & 1)) {
        fail();
        return;
      }
      const int item = int(atomicAdd(a.counter, 1u));
      Item d;
      d.valid = item < total && !s_abort;
      if (d.valid) {
        decode_item(a, item, d.phase, d.stream, d.chunk);
        if (!wait_phase(a, d.stream, d.phase)) {
          fail();
          d.valid = 0;
        }
        __threadfence();  // the finished phase's results are visible to the consumers
      }
      ring[r] = d;
      mbar_arrive(&item_full[r]);  // release: the descriptor
      if (!d.valid) return;
      if (d.phase < 1 || d.phase > 3) continue;  // beta_pre and append move no staged data
      const StreamDesc sd = a.sd[d.stream];
      const Plan pl = a.plan[d.stream];
      const BState *bs = a.st + d.stream;
      const bool first = __ldcg(&bs->first) != 0;
      const int j = first ? 0 : __ldcg(&bs->j);
      const int mode = first ? PASS_FIRST : (d.phase == 1 ? PASS_A : d.phase == 2 ? PASS_B : PASS_C);
      const bool base_x = (mode == PASS_A || mode == PASS_FIRST);
      const S *Vs = static_cast<const S *>(a.V) + sd.v_off;
      const S *x = static_cast<const S *>(a.x[d.stream]);
      const float *w = a.W + sd.w_off;
      const bool x_aligned = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
      const uint32_t tile_bytes = uint32_t(kTile) * uint32_t(j) * sizeof(S);
      const int s0 = d.chunk * pl.cs, s1 = min(pl.nstages, s0 + pl.cs);
      for (int stg = s0; stg < s1; ++stg, ++it) {
        const int slot = int(it % a.nslots);
        if (it >= uint32_t(a.nslots) && !mbar_wait(&empty[slot], ((it / a.nslots) - 1) & 1)) {
          fail();
          return;
        }
        const int t0 = stg * pl.R;
        const int nt = min(pl.R, sd.ntiles - t0);
        const int64_t r0 = int64_t(t0) * kTile;
        unsigned char *dst = slotmem + size_t(slot) * slot_bytes;
        const bool bb = base_x ? (x_aligned && r0 + int64_t(nt) * kTile <= sd.n) : true;
        const uint32_t bbytes = bb ? uint32_t(nt) * kTile * (base_x ? sizeof(S) : 4) : 0u;
        mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * tile_bytes + bbytes);
        if (tile_bytes)
          for (int q = 0; q < nt; ++q)
            bulk_g2s(dst + size_t(q) * tile_bytes, Vs + int64_t(t0 + q) * sd.kmax * kTile, tile_bytes, &full[slot]);
        if (bbytes) {
          if (base_x) bulk_g2s(dst + a.slot_v, x + r0, bbytes, &full[slot]);
          else bulk_g2s(dst + a.slot_v, w + r0, bbytes, &full[slot]);
        }
      }
    }
  }

  // ------------------------------------------------------------------ consumer warps
  const bool rowg = warp < ROW_WARPS;
  uint32_t it = 0;  // stages consumed (same sequence as the producer's)
  float acc[NCB / 2];
  for (int k = 0;; ++k) {
    const int r = k & 1;
    if (!s_abort && !mbar_wait(&item_full[r], (k >> 1) & 1)) fail();
    const Item d = ring[r];
    named_bar_sync(1, kConsumers);  // every consumer has read the descriptor
    if (tid == 0) mbar_arrive(&item_empty[r]);
    if (!d.valid || s_abort) break;
    const int sidx = d.stream, ph = d.phase, chunk = d.chunk;
    const StreamDesc sd = a.sd[sidx];
    BState *bs = a.st + sidx;
    const Plan pl = a.plan[sidx];
    const int j = __ldcg(&bs->j);
    const bool first = __ldcg(&bs->first) != 0;
    const int K = sd.kmax;
    double *Hs = a.H + sd.mat_off, *Bs = a.B + sd.mat_off;
    double *pre = a.vec + sd.vec_off, *hv = pre + K, *sv = hv + K;
    S *Vs = static_cast<S *>(a.V) + sd.v_off;
    float *w = a.W + sd.w_off;
    const S *x = static_cast<const S *>(a.x[sidx]);
    const int64_t nrows = int64_t(sd.ntiles) * kTile;

    if (ph == 0) {
      // ---------------------------------------------------------------- beta_pre (steps 5-8)
      if (tid == 0) {
        const double bjj = __ldcg(Bs + int64_t(j - 1) * (K + 1));
        bs->bjj = bjj;
        bs->inv_bjj = 1.0 / bjj;
      }
      for (int i = warp; i < j; i += kWarps) {
        const int l0 = i == 0 ? 0 : i - 1;
        double s_ = 0.0;
        for (int l = l0 + lane; l <= j - 2; l += 32) s_ += __ldcg(Hs + i + int64_t(l) * K) * __ldcg(Bs + l + int64_t(j - 1) * K);
        s_ = warp_sum(s_);
        if (lane == 0) pre[i] = s_;
      }
      __threadfence();
      named_bar_sync(1, kConsumers);
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
        for (int64_t rr = r0 + tid; rr < r1; rr += kConsumers) {
          const float v = first ? ((rr < sd.n) ? float(to_c(x[rr])) : 0.f) : __ldcg(w + rr);
          Vs[((rr >> 5) * K + j) * kTile + (rr & 31)] = Store<S>::from(v * sc);
        }
      }
      continue;
    }
    // ---------------------------------------------------------------- streaming pass (A, B, C)
    const int mode = first ? PASS_FIRST : (ph == 1 ? PASS_A : ph == 2 ? PASS_B : PASS_C);
    const bool dots = (mode == PASS_A || mode == PASS_B);
    const int jj = first ? 0 : j;
    const double *coef = (mode == PASS_A) ? pre : (mode == PASS_B) ? hv : sv;
    const float cscale = (mode == PASS_A) ? float(__ldcg(&bs->inv_bjj)) : 1.f;
    for (int c = tid; c < ((jj + 7) & ~3); c += kConsumers) cf[c] = c < jj ? float(__ldcg(coef + c)) : 0.f;
    for (int c = tid; c <= jj; c += kConsumers) dot[c] = 0.0;
    const bool x_aligned = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    const bool base_x = (mode == PASS_A || mode == PASS_FIRST);
    named_bar_sync(1, kConsumers);
    if (rowg) {
      // ------------------------------------------------------------ row group: sweep 1
      const int rt = tid;
      float nsum = 0.f, ncomp = 0.f;
      auto nrm_add = [&](float v) {
        const float y = v - ncomp;
        const float t = nsum + y;
        ncomp = (t - nsum) - y;
        nsum = t;
      };
      for (int stg = s0; stg < s1; ++stg, ++it) {
        const int slot = int(it % a.nslots);
        const int b = int(it & 1);
        if (!s_abort && !mbar_wait(&full[slot], (it / a.nslots) & 1)) fail();
        if (it >= 2 && !s_abort && !mbar_wait(&ws_empty[b], ((it >> 1) - 1) & 1)) fail();
        float *ws = wsb + b * (MAX_R * kTile);
        float *cb = combb + b * 256;
        const int t0 = stg * pl.R;
        const int nt = min(pl.R, sd.ntiles - t0);
        const int RS = nt * kTile;
        const int64_t r0 = int64_t(t0) * kTile;
        const unsigned char *sb = slotmem + size_t(slot) * slot_bytes;
        const S *vs = reinterpret_cast<const S *>(sb);
        const bool bb = base_x ? (x_aligned && r0 + int64_t(RS) <= sd.n) : true;
        auto finish_row = [&](int row, float accv) {
          const int64_t rr = r0 + row;
          float base;
          if (base_x) base = bb ? float(to_c(reinterpret_cast<const S *>(sb + a.slot_v)[row]))
                                : ((rr < sd.n) ? float(to_c(x[rr])) : 0.f);
          else base = reinterpret_cast<const float *>(sb + a.slot_v)[row];
          if (mode == PASS_FIRST) {
            nrm_add(base * base);
            return;
          }
          const float wc = (mode == PASS_A) ? (base - accv) * cscale : (base - accv);
          w[rr] = wc;
          ws[row] = wc;
          if (mode == PASS_A) nrm_add(base * base);
          else if (mode == PASS_C) nrm_add(wc * wc);
        };
        if (jj == 0) {
          for (int row = rt; row < RS; row += ROW_THREADS) finish_row(row, 0.f);
        } else {
          // row pairs, column groups of a multiple of 4, 16-byte coefficient broadcasts
          const int P = RS >> 1;
          const int G1 = (P >= ROW_THREADS) ? 1 : (ROW_THREADS / P);
          if (rt < (G1 == 1 ? ROW_THREADS : G1 * P)) {
            const int g = (G1 == 1) ? 0 : rt / P;
            const int cpg = (((jj + G1 - 1) / G1) + 3) & ~3;
            const int c0 = g * cpg, c1 = min(jj, c0 + cpg);
            for (int pr = (G1 == 1 ? rt : rt % P); pr < P; pr += (G1 == 1 ? ROW_THREADS : P)) {
              const int row = 2 * pr;
              const S *vr = vs + (row >> 5) * (kTile * jj) + (row & 31);
              float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
              for (int c = c0; c < c1; c += 4) {
                const float4 q = *reinterpret_cast<const float4 *>(cf + c);
                float2 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = (c + u < c1) ? ld_pair(vr + (c + u) * kTile) : make_float2(0.f, 0.f);
                a0[0] = fmaf(v[0].x, q.x, a0[0]); a1[0] = fmaf(v[0].y, q.x, a1[0]);
                a0[1] = fmaf(v[1].x, q.y, a0[1]); a1[1] = fmaf(v[1].y, q.y, a1[1]);
                a0[2] = fmaf(v[2].x, q.z, a0[2]); a1[2] = fmaf(v[2].y, q.z, a1[2]);
                a0[3] = fmaf(v[3].x, q.w, a0[3]); a1[3] = fmaf(v[3].y, q.w, a1[3]);
              }
              const float sa = (a0[0] + a0[1]) + (a0[2] + a0[3]);
              const float sb_ = (a1[0] + a1[1]) + (a1[2] + a1[3]);
              if (G1 > 1) {
                cb[g * RS + row] = sa;
                cb[g * RS + row + 1] = sb_;
              } else {
                finish_row(row, sa);
                finish_row(row + 1, sb_);
              }
            }
          }
          if (G1 > 1) {
            named_bar_sync(2, ROW_THREADS);
            if (rt < RS) {
              float s_ = 0.f;
              for (int g = 0; g < G1; ++g) s_ += cb[g * RS + rt];
              finish_row(rt, s_);
            }
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
      const int cw = warp - ROW_WARPS;
      const int hl = lane & 15, half = lane >> 4;
#pragma unroll
      for (int q = 0; q < NCB / 2; ++q) acc[q] = 0.f;
      auto flush = [&]() {
#pragma unroll
        for (int kk = 0; kk < NCB / 2; ++kk) {
          const int c = cw + COL_WARPS * (2 * kk + half);
          if (cw + COL_WARPS * (2 * kk) < jj) {  // warp-uniform
            float v = (c < jj) ? acc[kk] : 0.f;
#pragma unroll
            for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (hl == 0 && c < jj) dot[c] += double(v);
            acc[kk] = 0.f;
          }
        }
      };
      int since_flush = 0;
      for (int stg = s0; stg < s1; ++stg, ++it) {
        const int slot = int(it % a.nslots);
        const int b = int(it & 1);
        if (!s_abort && !mbar_wait(&full[slot], (it / a.nslots) & 1)) fail();
        if (!s_abort && !mbar_wait(&ws_full[b], (it >> 1) & 1)) fail();
        if (dots) {
          const float *ws = wsb + b * (MAX_R * kTile);
          const int t0 = stg * pl.R;
          const int nt = min(pl.R, sd.ntiles - t0);
          const S *vs = reinterpret_cast<const S *>(slotmem + size_t(slot) * slot_bytes);
          for (int kt = 0; kt < nt; ++kt) {
            const float2 wv = *reinterpret_cast<const float2 *>(ws + kt * kTile + 2 * hl);
            const S *vt = vs + kt * (kTile * jj) + 2 * hl;
#pragma unroll
            for (int kk = 0; kk < NCB / 2; ++kk) {
              const int c = cw + COL_WARPS * (2 * kk + half);
              if (c < jj) {
                const float2 v = ld_pair(vt + c * kTile);
                acc[kk] = fmaf(v.x, wv.x, fmaf(v.y, wv.y, acc[kk]));
              }
            }
          }
          since_flush += nt;
          if (since_flush >= 16) {
            flush();
            since_flush = 0;
          }
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&ws_empty[b]);
          mbar_arrive(&empty[slot]);
        }
      }
      if (dots) flush();
      nrm[tid] = 0.0;
    }
    // ---------------------------------------------------------------- this chunk's partial
    named_bar_sync(1, kConsumers);
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < kConsumers; ++i) t += nrm[i];
      dot[jj] = t;
    }
    named_bar_sync(1, kConsumers);
    double *pp = a.part + sd.part_off + int64_t(chunk) * (K + 1);
    for (int c = tid; c <= jj; c += kConsumers) pp[c] = dot[c];
    __threadfence();
    named_bar_sync(1, kConsumers);
    if (tid == 0) {
      const unsigned t = atomicAdd(a.tickets + sidx * 5 + ph, 1u);
      s_last = (t == unsigned(pl.nchunks - 1)) ? 1 : 0;
    }
    named_bar_sync(1, kConsumers);
    if (!s_last) continue;
    __threadfence();
    // ------------------------------------------------------------------ last chunk: reduce + scalar part
    for (int c = tid; c <= jj; c += kConsumers) {
      double t = 0.0;
      for (int q = 0; q < pl.nchunks; ++q) t += __ldcg(a.part + sd.part_off + int64_t(q) * (K + 1) + c);
      dot[c] = t;
    }
    named_bar_sync(1, kConsumers);
    if (mode == PASS_A) {
      for (int c = tid; c < jj; c += kConsumers) hv[c] = dot[c];
      if (tid == 0) bs->x_norm = sqrt(dot[jj]);
    } else if (mode == PASS_B) {
      for (int c = tid; c < jj; c += kConsumers) {
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
        for (int c = tid; c < jj; c += kConsumers) Hs[c + int64_t(jj - 1) * K] = __ldcg(hv + c);
      if (status == FOA_DMD_OK)
        for (int c = tid; c < jj; c += kConsumers) Bs[c + int64_t(jj) * K] = __ldcg(pre + c) + __ldcg(hv + c) * bjj;
      named_bar_sync(1, kConsumers);
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
        const double bn = sqrt(dot[0]);
        int status = !isfinite(bn) ? FOA_DMD_ENONFINITE : (!(bn > 0.0) ? FOA_DMD_EBREAKDOWN : FOA_DMD_OK);
        if (status == FOA_DMD_OK) {
          Bs[0] = bn;
          bs->inv_nu = 1.0 / bn;
          bs->nu = bn;
          bs->q = 1;
          if (a.h_last) a.h_last[sidx] = bn;
        } else if (status == FOA_DMD_EBREAKDOWN) {
          bs->stopped = 1;
        }
        bs->x_norm = bn;
        bs->h_last = bn;
        bs->status = status;
      }
    }
    __threadfence();
    named_bar_sync(1, kConsumers);
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
  int32_t slot_v = 0, nslots = 0;
  int64_t chunk_bytes = 0;
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
  // a stage slot holds one whole 32-row tile of the widest stream; the ring is as deep as fits
  int kmax_max = 2;
  for (int s = 0; s < S; ++s) kmax_max = k_max[s] > kmax_max ? k_max[s] : kmax_max;
  b->slot_v = int32_t((int64_t(kTile) * kmax_max * es + 127) / 128 * 128);
  if (b->slot_v < 16384) b->slot_v = 16384;
  const size_t fixed = size_t(2) * MAX_R * kTile * 4 + size_t(kMaxK + 8) * 4 + size_t(kMaxK + 2) * 8 + 512 * 4 +
                       size_t(kConsumers) * 8;
  int nslots = MAX_SLOTS;
  while (nslots > 2 && size_t(nslots) * (b->slot_v + SLOT_B) + fixed > size_t(220) * 1024) --nslots;
  b->nslots = nslots;
  b->chunk_bytes = 16ll << 20;  // V bytes per work item
  b->smem = size_t(nslots) * (b->slot_v + SLOT_B) + fixed;
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
    d.max_chunks = int32_t(int64_t(nrows) * d.kmax * es / b->chunk_bytes + 2);
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
  a.slot_v = b->slot_v;
  a.nslots = b->nslots;
  a.chunk_bytes = b->chunk_bytes;
  plan_kernel<<<1, 256, size_t(5) * b->S * 4, b->stream>>>(a, dtype_size(b->dtype));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  // one CTA per SM, all co-resident (cooperative launch), so the in-kernel phase waits always end
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->sms);
  cfg.blockDim = dim3(kThreads);
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
