// Batched streams: one call advances every active stream of a batch by one push (Alg. 4 with
// p = 1 per stream), as a fixed sequence of six launches that a CUDA graph can capture (every
// per-push decision is read from device memory):
//
//   plan_kernel     reads every stream's device state and the caller's pointer array, decides
//                   which streams push, and cuts each stream's passes into work items of whole
//                   pipeline stages (about 8 MB of V each);
//   prep_kernel     beta_pre of every active stream (Alg. 1), one CTA per stream;
//   bpass_kernel    pass A, then pass B, then pass C (pre-vector, CGS2, norm; Alg. 1) of all streams, one
//                   launch per pass: two CTAs of 256 threads per SM take items from a counter;
//   append_kernel   v_{j+1} = w / h_{j+1,j} (Alg. 1) of every stream that pushed.
//
// Launch order is the only dependency between the passes of a stream, so no CTA ever waits for
// another.  A pass item streams its stages through a shared-memory ring (two to six slots, as many
// stages as 100 KB holds) filled by one elected thread with bulk async copies (mbarrier
// completion), and every thread holds a fixed row pair and a fixed group of at most 16 (32 when a
// stage is one tile of more than 256 columns) columns of each stage in registers: from the
// registers it forms its partial GEMV-N sums (row sweep, combined across the column groups through
// shared memory) and, once the stage's new w is in shared memory, its columns' dot products
// (column sweep): the register-held layout of the single-stream passes, with two CTAs of 256
// threads per SM so that one CTA's barriers overlap the other's work.  A stage is R tiles of 32
// rows, R the largest power of two <= 8 with R*j <= 256 (stages of up to 32 KB of FP32, three to a
// ring), or one tile when j > 256.  Each item writes its FP64 partial sums; the last item of a (stream, pass)
// adds them in item order (deterministic) and applies the scalar step.
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.cuh"
#include "push_kernels.cuh"

namespace foa {
namespace bt {

constexpr int kBT = 256;                    // threads of a pass CTA (two CTAs per SM)
constexpr int kBW = kBT / 32;               // its warps
constexpr int kMaxRB = 8;                   // tiles per stage
constexpr int kRowsMax = kMaxRB * kTile;    // rows per stage
constexpr int kStageCols = 256;             // R * j <= this while R > 1: stages of <= 32 KB (FP32)
constexpr int kRingBytes = 102400;          // the stage ring of a CTA (two 50 KB slots hold j <= 399)
constexpr int kMaxBSlots = 6;
constexpr int kCf = 640;                    // padded coefficient vector (>= 16 * 32 + 32)
constexpr int64_t kItemBytes = 8ll << 20;   // V bytes per work item ...
constexpr int kItemStages = 256;            // ... and at most this many stages
enum { PH_A = 0, PH_B = 1, PH_C = 2, PH_APP = 3, NPH = 4 };

// shared-memory layout of bpass_kernel (bytes); two CTAs share an SM's 228 KB
constexpr size_t kOffWs = size_t(kRingBytes);
constexpr size_t kOffCf = kOffWs + size_t(kRowsMax) * 4;
constexpr size_t kOffComb = kOffCf + size_t(kCf) * 4;
constexpr size_t kOffDot = kOffComb + size_t(2 * kBT) * 4;
constexpr size_t kOffDotw = kOffDot + size_t(kMaxK + 8) * 8;
constexpr size_t kOffNred = kOffDotw + size_t(kBW * 16) * 8;
constexpr size_t kOffBar = kOffNred + size_t(kBW) * 8;
constexpr size_t kBSmem = kOffBar + size_t(kMaxBSlots) * 8;
static_assert(2 * (kBSmem + 1024 + 64) <= 233472, "two bpass_kernel CTAs per SM");

struct StreamDesc {
  int64_t n;
  int64_t v_off;    // element offset of the stream's V in the pool
  int64_t w_off;    // element offset of w
  int64_t mat_off;  // double offset of its k_max x k_max H-bar and beta
  int64_t vec_off;  // double offset of its pre/h/s vectors (3 x k_max)
  int64_t part_off; // double offset of its item partials
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
  int32_t R, nstages, cs, nchunks;  // tiles per stage, stages, stages per item, items
};

struct BatchArgs {
  const StreamDesc *sd;
  BState *st;
  Plan *plan;
  int32_t *offs;       // NPH x (S + 1): item offsets of each phase, stream-major
  int32_t *total;      // NPH
  uint32_t *counter;   // NPH work counters
  uint32_t *tickets;   // S x NPH
  void *V;             // pool (storage dtype)
  float *W;            // pool of w vectors (FP32)
  double *H, *B;       // pools
  double *vec;         // pools of pre/h/s
  double *part;        // item partials
  const void *const *x;  // caller's pointers (device array of S)
  double *h_last;      // caller's output array (device, S)
  double tol;
  int32_t S;
  int32_t *err;        // sticky
};

// ---------------------------------------------------------------------------- plan
__host__ __device__ __forceinline__ int stage_tiles(int j) {
  if (j <= 0) return kMaxRB;
  int R = 1;
  while (R * 2 <= kMaxRB && (R * 2) * j <= kStageCols) R *= 2;
  return R;
}

__global__ void plan_kernel(BatchArgs a, int ssize) {
  const int S = a.S;
  extern __shared__ int32_t cnt[];  // NPH * S counts
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const StreamDesc d = a.sd[s];
    BState &b = a.st[s];
    const bool has_x = a.x[s] != nullptr;
    const int q = b.q;
    const int active = has_x && !b.stopped && q < d.kmax;
    b.active = active;
    b.j = q;
    b.first = (q == 0) ? 1 : 0;
    if (active) b.status = -1;
    else if (has_x) b.status = b.stopped ? FOA_DMD_ESTOPPED : FOA_DMD_EFULL;
    if (a.h_last) a.h_last[s] = __longlong_as_double(0x7ff8000000000000ll);
    const int j = q;
    Plan p;
    p.R = stage_tiles(j);
    p.nstages = (d.ntiles + p.R - 1) / p.R;
    const int64_t stage_bytes = int64_t(p.R) * kTile * (j > 0 ? j : 1) * ssize;
    p.cs = int(kItemBytes / stage_bytes);
    if (p.cs > kItemStages) p.cs = kItemStages;
    if (p.cs < 1) p.cs = 1;
    p.nchunks = (p.nstages + p.cs - 1) / p.cs;
    if (p.nchunks > d.max_chunks) {  // keep within the partials buffer
      p.cs = (p.nstages + d.max_chunks - 1) / d.max_chunks;
      p.nchunks = (p.nstages + p.cs - 1) / p.cs;
    }
    a.plan[s] = p;
    const bool first = (j == 0);
    cnt[PH_A * S + s] = active ? p.nchunks : 0;               // pass A (or the first snapshot's norm)
    cnt[PH_B * S + s] = (active && !first) ? p.nchunks : 0;   // pass B
    cnt[PH_C * S + s] = (active && !first) ? p.nchunks : 0;   // pass C
    cnt[PH_APP * S + s] = active ? p.nchunks : 0;             // append
    for (int ph = 0; ph < NPH; ++ph) a.tickets[s * NPH + ph] = 0u;
  }
  __syncthreads();
  if (threadIdx.x < NPH) {
    const int ph = threadIdx.x;
    int run = 0;
    for (int s = 0; s < S; ++s) {
      a.offs[ph * (S + 1) + s] = run;
      run += cnt[ph * S + s];
    }
    a.offs[ph * (S + 1) + S] = run;
    a.total[ph] = run;
    a.counter[ph] = 0u;
  }
}

// beta_pre (Alg. 1): beta_pre_1 = sum_{l=1}^{j-1} h_{1,l} beta_{l,j},
// beta_pre_i = sum_{l=i-1}^{j-1} h_{i,l} beta_{l,j}; one CTA per stream, one warp per entry.
__global__ void prep_kernel(BatchArgs a) {
  const int s = blockIdx.x;
  BState *bs = a.st + s;
  if (!bs->active || bs->first) return;
  const StreamDesc sd = a.sd[s];
  const int j = bs->j, K = sd.kmax;
  const double *Hs = a.H + sd.mat_off, *Bs = a.B + sd.mat_off;
  double *pre = a.vec + sd.vec_off;
  if (threadIdx.x == 0) {
    const double bjj = Bs[int64_t(j - 1) * (K + 1)];
    bs->bjj = bjj;
    bs->inv_bjj = 1.0 / bjj;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < j; i += nw) {
    const int l0 = i == 0 ? 0 : i - 1;
    double t = 0.0;
    for (int l = l0 + lane; l <= j - 2; l += 32) t += Hs[i + int64_t(l) * K] * Bs[l + int64_t(j - 1) * K];
    t = warp_sum(t);
    if (lane == 0) pre[i] = t;
  }
}

// (phase, item) -> (stream, chunk) by binary search over the phase's item offsets
__device__ __forceinline__ void decode_item(const BatchArgs &a, int ph, int item, int &stream, int &chunk) {
  const int32_t *o = a.offs + ph * (a.S + 1);
  int lo = 0, hi = a.S;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (o[mid] <= item) lo = mid;
    else hi = mid;
  }
  while (lo + 1 < a.S && o[lo + 1] <= item) ++lo;  // skip streams without items
  stream = lo;
  chunk = item - o[lo];
}

// ---------------------------------------------------------------------------- the passes
// Per-item constants of the stage loop.
struct ItemGeo {
  int R, PF, G1, cpg, c0, nc, g, pr, ns;
  uint32_t tile_bytes, base_off, slot_bytes;
  int64_t tile_elems;
};

// The stages [s0, s1) of one item: per stage, the thread's V fragment (two rows x nc <= FC columns)
// goes to registers, the row sweep's group partials to comb, the finished rows' w to global and
// shared memory, and the column sweep's products to FP32 accumulators folded every 16 stages into
// FP64 (dot for column groups inside a warp, dotw per warp for groups that span several warps).
template <typename S, int FC>
__device__ __forceinline__ void run_stages(const BatchArgs &a, const StreamDesc &sd, const ItemGeo &ig, int mode,
                                           int j, int s0, int s1, float cscale, const S *x, float *w,
                                           unsigned char *slots, uint64_t *full, float *ws, const float *cf,
                                           float *comb, double *dot, double *dotw, uint32_t &par, int &s_abort,
                                           float &nsum, float &ncomp) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kIssuer = kBT - 1;
  const bool dots = (mode == PASS_A || mode == PASS_B);
  const bool base_x = (mode == PASS_A || mode == PASS_FIRST);
  const bool x_aligned = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
  const S *Vs = static_cast<const S *>(a.V) + sd.v_off;
  const int R = ig.R, PF = ig.PF, G1 = ig.G1, c0 = ig.c0, nc = ig.nc, g = ig.g, ns = ig.ns;
  auto issue = [&](int slot, int stg) {
    const int t0 = stg * R;
    const int nt = min(R, sd.ntiles - t0);
    const int64_t r0 = int64_t(t0) * kTile;
    const bool bb = base_x ? (x_aligned && r0 + int64_t(nt) * kTile <= sd.n) : true;
    const uint32_t bbytes = bb ? uint32_t(nt) * kTile * (base_x ? uint32_t(sizeof(S)) : 4u) : 0u;
    unsigned char *dst = slots + size_t(slot) * ig.slot_bytes;
    mbar_arrive_expect_tx(&full[slot], uint32_t(nt) * ig.tile_bytes + bbytes);
    if (ig.tile_bytes && FOA_CHECK(t0 >= 0 && t0 + nt <= sd.ntiles, kChkTile))
      for (int q = 0; q < nt; ++q)
        bulk_g2s(dst + size_t(q) * ig.tile_bytes, Vs + int64_t(t0 + q) * ig.tile_elems, ig.tile_bytes, &full[slot]);
    if (bbytes) {
      if (base_x) bulk_g2s(dst + ig.base_off, x + r0, bbytes, &full[slot]);
      else bulk_g2s(dst + ig.base_off, w + r0, bbytes, &full[slot]);
    }
  };
  const int nst = s1 - s0;
  if (tid == kIssuer && !s_abort)
    for (int k = 0; k < ns && k < nst; ++k) issue(k, s0 + k);
  float cacc[FC];
#pragma unroll
  for (int u = 0; u < FC; ++u) cacc[u] = 0.f;
  auto nrm_add = [&](float v) {
    const float y = v - ncomp;
    const float t = nsum + y;
    ncomp = (t - nsum) - y;
    nsum = t;
  };
  auto flush = [&]() {
#pragma unroll
    for (int u = 0; u < FC; ++u) {
      float v = cacc[u];
      if (PF >= 32) v += __shfl_xor_sync(0xffffffffu, v, 16);
#pragma unroll
      for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (u < nc) {
        if (PF <= 32) {
          if ((lane & (PF - 1)) == 0) dot[c0 + u] += double(v);   // the group is this warp or half-warp
        } else if (lane == 0) {
          dotw[warp * 16 + u] += double(v);                       // FC == 16 here (R >= 4)
        }
      }
      cacc[u] = 0.f;
    }
  };
  int since_flush = 0;
  for (int k = 0; k < nst; ++k) {
    const int stg = s0 + k;
    const int slot = k % ns;
    if (!s_abort && !mbar_wait(&full[slot], (par >> slot) & 1u)) {
      s_abort = 1;
      atomicExch(a.err, FOA_DMD_ETIMEOUT);
    }
    par ^= 1u << slot;
    const int t0 = stg * R;
    const int nt = min(R, sd.ntiles - t0);
    const int RS = nt * kTile;
    const int64_t r0 = int64_t(t0) * kTile;
    const unsigned char *sbase = slots + size_t(slot) * ig.slot_bytes;
    const S *vs = reinterpret_cast<const S *>(sbase);
    const bool bb = base_x ? (x_aligned && r0 + int64_t(RS) <= sd.n) : true;
    // ---- the thread's V fragment and its finish rows' base values
    const int row = 2 * ig.pr;
    const bool has_rows = row < RS && j > 0;
    float2 v[FC];
    {
      const S *vr = vs + (row >> 5) * (kTile * j) + (row & 31);
#pragma unroll
      for (int u = 0; u < FC; ++u) v[u] = (has_rows && u < nc) ? ld_pair(vr + (c0 + u) * kTile) : make_float2(0.f, 0.f);
    }
    float base[kRowsMax / kBT];
#pragma unroll
    for (int h = 0; h < kRowsMax / kBT; ++h) {
      const int rr = tid + h * kBT;
      base[h] = 0.f;
      if (rr < RS) {
        if (base_x) base[h] = bb ? float(to_c(reinterpret_cast<const S *>(sbase + ig.base_off)[rr]))
                                 : ((r0 + rr < sd.n) ? float(to_c(x[r0 + rr])) : 0.f);
        else base[h] = reinterpret_cast<const float *>(sbase + ig.base_off)[rr];
      }
    }
    // ---- row sweep from registers
    if (j > 0) {
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
    __syncthreads();  // every thread holds its fragment and base: the slot is free
    if (tid == kIssuer && !s_abort && k + ns < nst) issue(slot, stg + ns);
#pragma unroll
    for (int h = 0; h < kRowsMax / kBT; ++h) {
      const int rr = tid + h * kBT;
      if (rr < RS) {
        if (mode == PASS_FIRST) {
          nrm_add(base[h] * base[h]);
        } else {
          float acc = 0.f;
          for (int gg = 0; gg < G1; ++gg) acc += comb[gg * (2 * PF) + rr];
          const float wc = (mode == PASS_A) ? (base[h] - acc) * cscale : (base[h] - acc);
          w[r0 + rr] = wc;
          ws[rr] = wc;
          if (mode == PASS_A) nrm_add(base[h] * base[h]);
          else if (mode == PASS_C) nrm_add(wc * wc);
        }
      }
    }
    __syncthreads();  // ws complete
    // ---- column sweep from registers
    if (dots) {
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
  }
  if (dots) flush();
}

template <typename S>
__global__ void __launch_bounds__(kBT, 2) bpass_kernel(BatchArgs a, int ph) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *slots = smem;
  float *ws = reinterpret_cast<float *>(smem + kOffWs);       // new w of the stage's rows
  float *cf = reinterpret_cast<float *>(smem + kOffCf);       // coefficients, zero padded
  float *comb = reinterpret_cast<float *>(smem + kOffComb);   // row-sweep group partials
  double *dot = reinterpret_cast<double *>(smem + kOffDot);
  double *dotw = reinterpret_cast<double *>(smem + kOffDotw); // [warp][16] column sums (R >= 4)
  double *nred = reinterpret_cast<double *>(smem + kOffNred);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kOffBar);
  __shared__ int s_item, s_abort, s_last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < kMaxBSlots; ++i) mbar_init(&full[i], 1);
    s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const int total = a.total[ph];
  // Ring slots are laid out per item (as many stages of the item's size as the ring holds): an
  // item starts with an empty ring, so only the barriers' phases carry over: bit b of par is the
  // parity barrier b completes next (every thread waits on the same barriers in the same order).
  uint32_t par = 0u;
  for (;;) {
    if (tid == 0) s_item = s_abort ? total : int(atomicAdd(a.counter + ph, 1u));
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    int sidx, chunk;
    decode_item(a, ph, item, sidx, chunk);
    const StreamDesc sd = a.sd[sidx];
    BState *bs = a.st + sidx;
    const Plan pl = a.plan[sidx];
    const bool first = bs->first != 0;
    const int j = first ? 0 : bs->j;
    const int K = sd.kmax;
    const int mode = first ? PASS_FIRST : (ph == PH_A ? PASS_A : ph == PH_B ? PASS_B : PASS_C);
    const bool dots = (mode == PASS_A || mode == PASS_B);
    double *Hs = a.H + sd.mat_off, *Bs = a.B + sd.mat_off;
    double *pre = a.vec + sd.vec_off, *hv = pre + K, *sv = hv + K;
    float *w = a.W + sd.w_off;
    const S *x = static_cast<const S *>(a.x[sidx]);
    const float cscale = (mode == PASS_A) ? float(bs->inv_bjj) : 1.f;
    // the fixed mapping of this stream's stages: PF row pairs, G1 column groups of cpg columns
    ItemGeo ig;
    ig.R = pl.R;
    ig.PF = ig.R * (kTile / 2);
    ig.G1 = kBT / ig.PF;
    ig.cpg = j > 0 ? ((((j + ig.G1 - 1) / ig.G1) + 3) & ~3) : 0;  // <= 16, or <= 32 when R = 1
    ig.g = tid / ig.PF;
    ig.pr = tid % ig.PF;
    ig.c0 = ig.g * ig.cpg;
    ig.nc = max(0, min(j, ig.c0 + ig.cpg) - ig.c0);
    ig.tile_bytes = uint32_t(kTile) * uint32_t(j) * sizeof(S);
    ig.tile_elems = int64_t(K) * kTile;
    ig.base_off = uint32_t(ig.R) * ig.tile_bytes;                           // 16-byte multiple
    ig.slot_bytes = (ig.base_off + uint32_t(ig.R) * kTile * 4u + 127u) & ~127u;
    ig.ns = int(uint32_t(kRingBytes) / ig.slot_bytes);
    if (ig.ns > kMaxBSlots) ig.ns = kMaxBSlots;                              // >= 1 (j < 400: >= 2)
    const double *coef = (mode == PASS_A) ? pre : (mode == PASS_B) ? hv : sv;
    const int fcmax = ig.cpg > 16 ? 32 : 16;
    for (int c = tid; c < ig.G1 * ig.cpg + fcmax; c += kBT) cf[c] = (c < j) ? float(coef[c]) : 0.f;
    for (int c = tid; c <= j; c += kBT) dot[c] = 0.0;
    for (int c = tid; c < kBW * 16; c += kBT) dotw[c] = 0.0;
    __syncthreads();
    const int s0 = chunk * pl.cs, s1 = min(pl.nstages, s0 + pl.cs);
    float nsum = 0.f, ncomp = 0.f;
    if (ig.cpg > 16)
      run_stages<S, 32>(a, sd, ig, mode, j, s0, s1, cscale, x, w, slots, full, ws, cf, comb, dot, dotw, par,
                        s_abort, nsum, ncomp);
    else
      run_stages<S, 16>(a, sd, ig, mode, j, s0, s1, cscale, x, w, slots, full, ws, cf, comb, dot, dotw, par,
                        s_abort, nsum, ncomp);
    // ---- this item's partial: column sums (warp order for groups that span warps), the norm in a
    // fixed tree
    double nv = double(nsum) - double(ncomp);
    nv = warp_sum(nv);
    if (lane == 0) nred[warp] = nv;
    __syncthreads();
    if (dots && ig.PF > 32)
      for (int c = tid; c < j; c += kBT) {
        const int gc = c / ig.cpg, u = c - gc * ig.cpg;
        const int w0 = gc * (ig.PF / 32), w1 = w0 + ig.PF / 32;
        double t = 0.0;
        for (int wq = w0; wq < w1; ++wq) t += dotw[wq * 16 + u];
        dot[c] = t;
      }
    if (tid == 0) {
      double t = 0.0;
      for (int wq = 0; wq < kBW; ++wq) t += nred[wq];
      dot[j] = t;
    }
    __syncthreads();
    double *pp = a.part + sd.part_off + int64_t(chunk) * (K + 1);
    for (int c = tid; c <= j; c += kBT) pp[c] = dot[c];
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned t = atomicAdd(a.tickets + sidx * NPH + ph, 1u);
      s_last = (t == unsigned(pl.nchunks - 1)) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) continue;
    __threadfence();
    // ------------------------------------------------------------ last item: reduce + scalar step
    for (int c = tid; c <= j; c += kBT) {
      double t = 0.0;
      for (int q = 0; q < pl.nchunks; ++q) t += __ldcg(a.part + sd.part_off + int64_t(q) * (K + 1) + c);
      dot[c] = t;
    }
    __syncthreads();
    if (mode == PASS_A) {
      for (int c = tid; c < j; c += kBT) hv[c] = dot[c];
      if (tid == 0) bs->x_norm = sqrt(dot[j]);
    } else if (mode == PASS_B) {
      for (int c = tid; c < j; c += kBT) {
        sv[c] = dot[c];
        hv[c] = hv[c] + dot[c];
      }
    } else if (mode == PASS_C) {
      const double nu = sqrt(dot[j]);
      const double xn = bs->x_norm, bjj = bs->bjj;
      int status;
      if (!isfinite(nu) || !isfinite(xn)) status = FOA_DMD_ENONFINITE;
      else if (!(nu * bjj > a.tol * xn)) status = FOA_DMD_EBREAKDOWN;
      else status = FOA_DMD_OK;
      if (status != FOA_DMD_ENONFINITE)
        for (int c = tid; c < j; c += kBT) Hs[c + int64_t(j - 1) * K] = hv[c];
      if (status == FOA_DMD_OK)
        for (int c = tid; c < j; c += kBT) Bs[c + int64_t(j) * K] = pre[c] + hv[c] * bjj;
      __syncthreads();
      if (tid == 0) {
        if (status == FOA_DMD_OK) {
          Hs[j + int64_t(j - 1) * K] = nu;
          Bs[j + int64_t(j) * K] = nu * bjj;
          bs->nu = nu;
          bs->inv_nu = 1.0 / nu;
          bs->q = j + 1;
          if (a.h_last) a.h_last[sidx] = nu;
        } else if (status == FOA_DMD_EBREAKDOWN) {
          Hs[j + int64_t(j - 1) * K] = 0.0;
          bs->stopped = 1;
        }
        bs->h_last = nu;
        bs->status = status;
      }
    } else {  // first snapshot: beta_11 = ||x||
      if (tid == 0) {
        const double bn = sqrt(dot[0]);
        const int status = !isfinite(bn) ? FOA_DMD_ENONFINITE : (!(bn > 0.0) ? FOA_DMD_EBREAKDOWN : FOA_DMD_OK);
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
    __syncthreads();
  }
}

// append v_{j+1} = w / h_{j+1,j} (v_1 = x / ||x|| for a first snapshot), one item per pass item
template <typename S>
__global__ void append_kernel(BatchArgs a) {
  __shared__ int s_item;
  const int total = a.total[PH_APP];
  for (;;) {
    if (threadIdx.x == 0) s_item = int(atomicAdd(a.counter + PH_APP, 1u));
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= total) return;
    int sidx, chunk;
    decode_item(a, PH_APP, item, sidx, chunk);
    const BState *bs = a.st + sidx;
    if (bs->status != FOA_DMD_OK) continue;
    const StreamDesc sd = a.sd[sidx];
    const Plan pl = a.plan[sidx];
    const bool first = bs->first != 0;
    const int j = first ? 0 : bs->j, K = sd.kmax;
    const int64_t nrows = int64_t(sd.ntiles) * kTile;
    const int64_t r0 = int64_t(chunk) * pl.cs * pl.R * kTile;
    const int64_t r1 = min(nrows, int64_t(chunk + 1) * pl.cs * pl.R * kTile);
    const float sc = float(bs->inv_nu);
    S *Vs = static_cast<S *>(a.V) + sd.v_off;
    const float *w = a.W + sd.w_off;
    const S *x = static_cast<const S *>(a.x[sidx]);
    for (int64_t rr = r0 + threadIdx.x; rr < r1; rr += blockDim.x) {
      const float v = first ? ((rr < sd.n) ? float(to_c(x[rr])) : 0.f) : w[rr];
      Vs[((rr >> 5) * K + j) * kTile + (rr & 31)] = Store<S>::from(v * sc);
    }
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
  int32_t *offs = nullptr, *total = nullptr, *err = nullptr;
  uint32_t *counter = nullptr, *tickets = nullptr;
  void *V = nullptr;
  float *W = nullptr;
  double *H = nullptr, *B = nullptr, *vec = nullptr, *part = nullptr;
};

static void batch_free(foa_dmd_batch *b) {
  void *ptrs[] = {b->sd, b->st, b->plan, b->offs, b->total, b->err, b->counter, b->tickets, b->V, b->W,
                  b->H, b->B, b->vec, b->part};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

// the largest number of work items a pass of this stream can have (over every basis size j)
static int32_t max_items(int32_t ntiles, int32_t kmax, int es) {
  int32_t best = 1;
  for (int j = 0; j < kmax; ++j) {
    const int R = stage_tiles(j);
    const int64_t nstages = (ntiles + R - 1) / R;
    const int64_t stage_bytes = int64_t(R) * kTile * (j > 0 ? j : 1) * es;
    int64_t cs = kItemBytes / stage_bytes;
    if (cs > kItemStages) cs = kItemStages;
    if (cs < 1) cs = 1;
    const int64_t nc = (nstages + cs - 1) / cs;
    if (nc > best) best = int32_t(nc);
  }
  return best;
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
    d.max_chunks = max_items(d.ntiles, d.kmax, es);
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
  BAL(b->offs, sizeof(int32_t) * NPH * (S + 1));
  BAL(b->total, sizeof(int32_t) * NPH);
  BAL(b->err, sizeof(int32_t));
  BAL(b->counter, sizeof(uint32_t) * NPH);
  BAL(b->tickets, sizeof(uint32_t) * NPH * S);
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
    const void *kern = dtype == FOA_DMD_F32 ? (const void *)bpass_kernel<float> : (const void *)bpass_kernel<__nv_bfloat16>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kBSmem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
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
  cudaStream_t s = b->stream;
  nvtxRangePushA("foa_dmd batch push");
  // the fixed launch sequence of one round: plan, beta_pre, passes A, B, C, append
  plan_kernel<<<1, 256, size_t(NPH) * b->S * 4, s>>>(a, dtype_size(b->dtype));
  prep_kernel<<<b->S, 256, 0, s>>>(a);
  for (int ph = PH_A; ph <= PH_C; ++ph) {
    if (b->dtype == FOA_DMD_F32) bpass_kernel<float><<<2 * b->sms, kBT, kBSmem, s>>>(a, ph);
    else bpass_kernel<__nv_bfloat16><<<2 * b->sms, kBT, kBSmem, s>>>(a, ph);
  }
  if (b->dtype == FOA_DMD_F32) append_kernel<float><<<b->sms * 4, 256, 0, s>>>(a);
  else append_kernel<__nv_bfloat16><<<b->sms * 4, 256, 0, s>>>(a);
  nvtxRangePop();
  return cuda_status(cudaGetLastError());
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
