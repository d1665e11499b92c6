// Block push: P snapshots at once (the block form of the QR view of Sec. 3.1; the §8 block-push
// variant).  Per block X_b = [psi_{j+1} .. psi_{j+P}], with V the current basis (j columns):
//   BLK_A  (one pass over V)  C1 = V^T X_b and ||psi_k||^2
//   BLK_B  (one pass over V)  W = X_b - V C1,  C2 = V^T W,  C = C1 + C2
//   BLK_C  (one pass over V)  W = W - V C2,    G = W^T W, then G = R1^T R1 (Cholesky, FP64)
//   BLK_Q1 (rows of W only)   W1 = W R1^-1 (FP64), G2 = W1^T W1 = R2^T R2, R = R2 R1, breakdown test,
//                             beta block column [C; R], Hbar columns by forward substitution
//   BLK_Q2 (rows of W only)   Q = W1 R2^-1 -> V columns j .. j+P-1
// V is read three times per block instead of three times per snapshot.  The three passes over V
// are block_pass.cuh (register-held fragments, packed FP32 FMAs, per-CTA FP64 partials and a
// deterministic two-level cross-CTA reduction; FP32/BF16 storage).  From the Gram matrix on, the
// Cholesky QR works in FP64 (exact products of the FP32 W, W R1^-1 and Q in FP64): stored in FP32,
// W R1^-1 would carry u_fp32 kappa(W)^2 and lose orthogonality once a block's directions span more
// than ~sqrt(1/u_fp32) in size.
#include <cmath>
#include <cstring>

#include "block_internal.cuh"
#include "push_kernels.cuh"

namespace foa {
namespace blk {

// W1 = W R1^-1 on the leading m1 columns (FP64), G2 = W1^T W1 (per CTA partials), and in the last CTA:
// R2, R = R2 R1, the breakdown test, the beta block column, the Hbar columns, the device state.
template <int P>
__global__ void __launch_bounds__(256) blockq1_kernel(BlockArgs a, foa_dmd_push_info *info_out) {
  __shared__ double red[256 * P * P];
  __shared__ double dot[P * P];
  __shared__ volatile int sflag[4];
  const int tid = threadIdx.x;
  if (!a.st->active) return;
  BlockState *bs = a.bs;
  const int m1 = __ldcg(&bs->m1);
  double R1[P * P];
#pragma unroll
  for (int i = 0; i < P * P; ++i) R1[i] = __ldcg(&bs->R1[(i % P) + (i / P) * kMaxP]);
  double g[P * P];
#pragma unroll
  for (int i = 0; i < P * P; ++i) g[i] = 0.0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + tid; r < a.nrows; r += stride) {
    float w[P];
#pragma unroll
    for (int k = 0; k < P; ++k) w[k] = a.W[int64_t(k) * a.nrows + r];
    // w1_c = (w_c - sum_{k<c} w1_k R1_{k,c}) / R1_{c,c}, in FP64 for the small triangular solve
    double w1[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      double t = w[c];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= w1[k] * R1[k + c * P];
      w1[c] = (c < m1) ? t / R1[c + c * P] : 0.0;
    }
#pragma unroll
    for (int c = 0; c < P; ++c) a.W64[int64_t(c) * a.nrows + r] = w1[c];
#pragma unroll
    for (int k = 0; k < P; ++k)
#pragma unroll
      for (int l = 0; l < P; ++l) g[k + l * P] += w1[k] * w1[l];
  }
#pragma unroll
  for (int i = 0; i < P * P; ++i) red[tid * P * P + i] = g[i];
  __syncthreads();
  if (tid < P * P) {
    double t = 0.0;
    for (int i = 0; i < 256; ++i) t += red[i * P * P + tid];
    dot[tid] = t;
  }
  __syncthreads();
  // deterministic cross-CTA reduction (groups of 8 CTAs, then groups)
  const int len = P * P;
  double *mypart = a.partials + size_t(blockIdx.x) * len;
  if (tid < len) mypart[tid] = dot[tid];
  __threadfence();
  __syncthreads();
  const int ngroups = (gridDim.x + kGroup - 1) / kGroup;
  const int grp = blockIdx.x / kGroup;
  const int gfirst = grp * kGroup;
  const int gsize = min(kGroup, int(gridDim.x) - gfirst);
  if (tid == 0) {
    const unsigned t = atomicAdd(&a.gcount[grp], 1u);
    sflag[2] = (t == unsigned(gsize - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (!sflag[2]) return;
  __threadfence();
  if (tid < len) {
    double t = 0.0;
    for (int b = 0; b < gsize; ++b) t += __ldcg(a.partials + size_t(gfirst + b) * len + tid);
    a.gpart[size_t(grp) * len + tid] = t;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    a.gcount[grp] = 0u;
    const unsigned t = atomicAdd(&bs->ticket[3], 1u);
    sflag[2] = (t == unsigned(ngroups - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (!sflag[2]) return;
  __threadfence();
  if (tid < len) {
    double t = 0.0;
    for (int gq = 0; gq < ngroups; ++gq) t += __ldcg(a.gpart + size_t(gq) * len + tid);
    dot[tid] = t;
  }
  if (tid == 0) bs->ticket[3] = 0u;
  __syncthreads();
  // ---------------- the last CTA
  const int j = a.j;
  const int K = a.kmax;
  if (tid == 0) {
    double G2[kMaxP * kMaxP];
    for (int i = 0; i < kMaxP * kMaxP; ++i) G2[i] = 0.0;
    for (int k = 0; k < m1; ++k)
      for (int l = 0; l < m1; ++l) G2[k + l * kMaxP] = dot[k + l * P];
    const int m = m1 > 0 ? chol_up(m1, G2, bs->R2) : 0;
    // R = R2 R1: rows r < m for every column c (columns past the factored block keep their
    // coefficients on the factored directions)
    for (int i = 0; i < kMaxP * kMaxP; ++i) bs->R[i] = 0.0;
    for (int c = 0; c < P; ++c)
      for (int r = 0; r < m && r <= c; ++r) {
        double t = 0.0;
        const int kmx = c < m1 - 1 ? c : m1 - 1;
        for (int k = r; k <= kmx; ++k) t += bs->R2[r + k * kMaxP] * bs->R1[k + c * kMaxP];
        bs->R[r + c * kMaxP] = t;
      }
    int nc = 0, status = FOA_DMD_OK;
    for (int i = 0; i < P; ++i) {
      const double rii = bs->R[i + i * kMaxP];
      if (!isfinite(rii) || !isfinite(bs->xnorm[i])) {
        status = FOA_DMD_ENONFINITE;
        break;
      }
      if (!(i < m && rii > a.tol * bs->xnorm[i])) {
        status = FOA_DMD_EBREAKDOWN;
        break;
      }
      if (rii < a.resolve * bs->xnorm[i]) {  // below the block form's resolution: not committed
        status = FOA_DMD_ERESOLVE;
        break;
      }
      nc = i + 1;
    }
    bs->ncommit = nc;
    bs->status = status;
  }
  __syncthreads();
  const int nc = bs->ncommit;
  const int status = bs->status;
  // beta block column
  for (int i = 0; i < nc; ++i) {
    const int col = j + i;
    for (int r = tid; r < j; r += blockDim.x) a.B[r + int64_t(col) * K] = __ldcg(a.C + int64_t(i) * K + r);
    for (int r = tid; r <= i; r += blockDim.x) a.B[j + r + int64_t(col) * K] = bs->R[r + i * kMaxP];
  }
  __syncthreads();
  // Hbar columns by forward substitution, one new snapshot after the other
  const int ncols = nc + ((status == FOA_DMD_EBREAKDOWN) ? 1 : 0);
  for (int i = 0; i < ncols; ++i) {
    const int jc = j - 1 + i, jj = j + i;
    const double bjj = a.B[jc + int64_t(jc) * K];
    for (int r = tid; r < jj; r += blockDim.x) {
      const double brc = (r < j) ? __ldcg(a.C + int64_t(i) * K + r) : bs->R[(r - j) + i * kMaxP];
      const int l0 = r == 0 ? 0 : r - 1;
      double acc = 0.0;
      for (int l = l0; l <= jc - 1; ++l) acc += a.H[r + int64_t(l) * K] * a.B[l + int64_t(jc) * K];
      a.H[r + int64_t(jc) * K] = (brc - acc) / bjj;
    }
    __syncthreads();
    if (tid == 0) {
      const double sub = (i < nc) ? bs->R[i + i * kMaxP] / bjj : 0.0;
      a.H[jj + int64_t(jc) * K] = sub;
      foa_dmd_push_info inf;
      inf.h_last = sub;
      inf.indicator = __longlong_as_double(0x7ff8000000000000ll);
      inf.x_norm = bs->xnorm[i];
      inf.q = j + ((i < nc) ? i + 1 : i);
      inf.status = (i < nc) ? FOA_DMD_OK : status;
      if (info_out) info_out[i] = inf;
      a.st->info = inf;
    }
    __syncthreads();
  }
  if (tid == 0) {
    DevState *st = a.st;
    st->q = j + nc;
    st->status = status;
    if (status == FOA_DMD_EBREAKDOWN) st->stopped = 1;
    if (info_out)
      for (int i = ncols; i < P; ++i) {
        foa_dmd_push_info inf;
        inf.h_last = __longlong_as_double(0x7ff8000000000000ll);
        inf.indicator = inf.h_last;
        inf.x_norm = bs->xnorm[i];
        inf.q = j + nc;
        inf.status = (status == FOA_DMD_EBREAKDOWN) ? FOA_DMD_ESTOPPED : status;
        info_out[i] = inf;
      }
  }
}

// Q = W1 R2^-1 -> V columns j .. j+ncommit-1 (row-tiled), rows beyond n zero
template <typename S, int P>
__global__ void blockq2_kernel(BlockArgs a) {
  if (!a.st->active) return;
  const BlockState *bs = a.bs;
  const int nc = __ldcg(&bs->ncommit);
  if (nc == 0) return;
  double R2[P * P];
#pragma unroll
  for (int i = 0; i < P * P; ++i) R2[i] = __ldcg(&bs->R2[(i % P) + (i / P) * kMaxP]);
  S *V = static_cast<S *>(const_cast<void *>(a.V));
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < a.nrows; r += stride) {
    double q[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      double t = a.W64[int64_t(c) * a.nrows + r];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= q[k] * R2[k + c * P];
      q[c] = t / R2[c + c * P];
    }
#pragma unroll
    for (int c = 0; c < P; ++c)
      if (c < nc) V[((r >> 5) * a.kmax + a.j + c) * kTile + (r & 31)] = Store<S>::from(float(r < a.n ? q[c] : 0.0));
  }
}

// device-state gate of a block push (the prep of a single push, for P snapshots)
__global__ void block_prep_kernel(DevState *st, BlockState *bs, int j, int pb, int kmax) {
  if (threadIdx.x != 0) return;
  const bool ok = !st->stopped && st->q == j && j + pb <= kmax && j >= 1;
  st->active = ok ? 1 : 0;
  st->j = j;
  if (!ok) st->status = st->stopped ? FOA_DMD_ESTOPPED : (j + pb > kmax ? FOA_DMD_EFULL : FOA_DMD_EINVAL);
  bs->j = j;
  bs->pb = pb;
  bs->m1 = 0;
  bs->ncommit = 0;
  bs->status = -1;
}

}  // namespace blk
}  // namespace foa

using namespace foa;
using namespace foa::blk;

namespace {

struct BlockWork {
  float *W = nullptr;
  double *W64 = nullptr;
  double *C1 = nullptr, *C = nullptr;
  BlockState *bs = nullptr;
  foa_dmd_push_info *info = nullptr;
};

// Shared-memory layout and grid of block pass `mode` at basis size j for a T-thread CTA with fc
// columns a thread: the ring of slots (one V tile and the P base slices each), the coefficient
// pairs, the row-sweep partials, the new w of a stage, the FP64 dot vector, the norm / Gram
// partials and the mbarriers.  T = 256: two CTAs per SM; T = 512: one.
bool block_geom(const foa_dmd *h, int P, int j, int mode, int T, int fc, BlockArgs &a, int &grid) {
  const int s = dtype_size(h->dtype);
  const int G1 = T / 8;
  auto up = [](int64_t v, int64_t al) { return (v + al - 1) / al * al; };
  const int64_t tile_bytes = int64_t(kTile) * j * s;
  const int64_t base_stride = up(int64_t(kTile) * (mode == BLK_C ? 4 : s), 128);
  const int64_t slot = up(tile_bytes, 128) + P * base_stride;
  const bool row = mode != BLK_A;
  const int64_t coef_b = row ? up(int64_t(G1) * fc * P * 8, 128) : 0;
  const int64_t comb_b = row ? up(int64_t(G1) * P * kTile * 4, 128) : 0;
  const int64_t ws_b = row ? up(int64_t(kTile) * P * 4, 128) : 0;
  const int64_t dot_b = up(int64_t(j * P + P * P + P) * 8, 128);
  const int64_t red_b = up(int64_t(kTile) * (P * (P + 1) / 2) * 8, 128);  // >= 8 P norms
  const int64_t bar_b = kMaxSlots * 8 + 64;
  const int64_t other = coef_b + comb_b + ws_b + dot_b + red_b + bar_b;
  const int64_t budget = T == 256 ? int64_t(112) * 1024 : int64_t(220) * 1024;
  int slots = int((budget - other) / slot);
  if (slots > 4) slots = 4;
  if (slots < 2) return false;
  a.slots = slots;
  a.slot_bytes = int(slot);
  a.base_off = int(up(tile_bytes, 128));
  a.base_stride = int(base_stride);
  int64_t off = slot * slots;
  a.off_coef = int(off);
  off += coef_b;
  a.off_comb = int(off);
  off += comb_b;
  a.off_ws = int(off);
  off += ws_b;
  a.off_dot = int(off);
  off += dot_b;
  a.off_red = int(off);
  off += red_b;
  a.off_bar = int(off);
  off += bar_b;
  a.smem_total = int(off);
  if (a.smem_total > 232448) return false;
  a.ntiles = h->ntiles;
  a.n = h->n;
  a.nrows = h->nrows;
  const int sms = h->sms - (h->opts.indicator_every > 0 ? 1 : 0);
  const int per_sm = T == 256 ? 2 : 1;
  grid = a.ntiles < sms * per_sm ? a.ntiles : sms * per_sm;
  return true;
}

// one block of P snapshots (P = 2 or 4) on a stream with q >= 1 basis vectors
template <int P>
int enqueue_block(foa_dmd *h, BlockWork &bw, const void *X, int64_t ldx, foa_dmd_push_info *info_out) {
  const int j = h->q_host;
  BlockArgs a;
  memset(&a, 0, sizeof(a));
  a.V = h->V;
  a.X = X;
  a.ldx = ldx;
  a.W = bw.W;
  a.W64 = bw.W64;
  a.C1 = bw.C1;
  a.C = bw.C;
  a.partials = h->partials;
  a.gpart = h->gpart;
  a.gcount = h->gcount;
  a.bs = bw.bs;
  a.st = h->st;
  a.H = h->H;
  a.B = h->B;
  a.kmax = h->kmax;
  a.j = j;
  a.x_aligned = (reinterpret_cast<uintptr_t>(X) & 15u) == 0 && ((ldx * dtype_size(h->dtype)) & 15) == 0;
  a.tol = h->tol;
  a.resolve = kBlockResolveUnits * unit_roundoff(h->dtype);
  int T = 0, fc = 0;
  block_pass_shape(j, P, T, fc);
  BlockArgs am[3];
  int grid = 0;
  for (int mode = BLK_A; mode <= BLK_C; ++mode) {
    am[mode] = a;
    if (!block_geom(h, P, j, mode, T, fc, am[mode], grid)) return FOA_DMD_EINVAL;
  }
  a.ntiles = am[0].ntiles;
  a.n = am[0].n;
  a.nrows = am[0].nrows;
  cudaStream_t s = h->stream;
  block_prep_kernel<<<1, 32, 0, s>>>(h->st, bw.bs, j, P, h->kmax);
  cudaError_t e = cudaGetLastError();
  const double sz = dtype_size(h->dtype), n = double(h->n);
  for (int mode = BLK_A; mode <= BLK_C && e == cudaSuccess; ++mode) {
    // V once, plus the P base vectors read (X or W) and written (W)
    const double vec = mode == BLK_A ? sz : mode == BLK_B ? sz + 4.0 : 8.0;
    ProfScope ps(h, mode == BLK_A ? 0 : mode == BLK_B ? 1 : 2, n * j * sz + P * n * vec);
    if (h->dtype == FOA_DMD_F32) e = launch_block_pass_f32(mode, T, fc, P, am[mode], grid, s);
    else e = launch_block_pass_bf16(mode, T, fc, P, am[mode], grid, s);
    h->launches += 1;
  }
  if (e == cudaSuccess) {
    const int g = h->sms * 4;
    blockq1_kernel<P><<<g, 256, 0, s>>>(a, info_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    ProfScope ps(h, 3, n * P * 4 + n * P * sz);
    if (h->dtype == FOA_DMD_F32) blockq2_kernel<float, P><<<h->sms * 4, 256, 0, s>>>(a);
    else blockq2_kernel<__nv_bfloat16, P><<<h->sms * 4, 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  h->launches += 3;  // prep, Cholesky QR, Q into V
  return cuda_status(e);
}

}  // namespace

extern "C" int foa_dmd_push_block(foa_dmd_t *h, const void *X_dev, int32_t p, int64_t ld, int32_t block,
                                  foa_dmd_push_info *infos) {
  if (!h || !X_dev || p < 0 || ld < h->n || (block != 2 && block != 4)) return FOA_DMD_EINVAL;
  if (h->dtype == FOA_DMD_F64) return FOA_DMD_EINVAL;  // FP32/BF16 storage only
  if (((ld * dtype_size(h->dtype)) & 15) != 0) return FOA_DMD_EINVAL;
  if (p == 0) return FOA_DMD_OK;
  int rc = flush_pending(h);  // a two-pass stream's newest column
  if (rc) return rc;
  rc = sync_state(h, nullptr);
  if (rc) return rc;
  if (h->stopped_host) return FOA_DMD_ESTOPPED;
  BlockWork bw;
  cudaError_t e = cudaMalloc(&bw.W, size_t(kMaxP) * h->nrows * 4);
  if (e == cudaSuccess) e = cudaMalloc(&bw.W64, size_t(kMaxP) * h->nrows * 8);
  if (e == cudaSuccess) e = cudaMalloc(&bw.C1, size_t(kMaxP) * h->kmax * 8);
  if (e == cudaSuccess) e = cudaMalloc(&bw.C, size_t(kMaxP) * h->kmax * 8);
  if (e == cudaSuccess) e = cudaMalloc(&bw.bs, sizeof(BlockState));
  if (e == cudaSuccess) e = cudaMalloc(&bw.info, sizeof(foa_dmd_push_info) * kMaxP);
  if (e == cudaSuccess) e = cudaMemsetAsync(bw.bs, 0, sizeof(BlockState), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(bw.W, 0, size_t(kMaxP) * h->nrows * 4, h->stream);
  rc = cuda_status(e);
  const char *X = static_cast<const char *>(X_dev);
  const size_t colbytes = size_t(ld) * dtype_size(h->dtype);
  int t = 0;
  while (rc == FOA_DMD_OK && t < p) {
    foa_dmd_push_info got[kMaxP];
    int took = 0;
    if (h->q_host == 0 || p - t < block || h->q_host + block > h->kmax) {
      // single push: the first snapshot of a stream, a remainder, or the last columns before k_max
      if (h->q_host >= h->kmax) {
        for (; t < p; ++t)
          if (infos) {
            infos[t].status = FOA_DMD_EFULL;
            infos[t].q = h->kmax;
            infos[t].h_last = infos[t].indicator = infos[t].x_norm = NAN;
          }
        rc = FOA_DMD_EFULL;
        break;
      }
      rc = enqueue_push(h, X + size_t(t) * colbytes, false, bw.info);
      if (rc == FOA_DMD_OK) rc = flush_pending(h);  // a two-pass handle: the column is written now
      if (rc) break;
      took = 1;
    } else {
      rc = block == 4 ? enqueue_block<4>(h, bw, X + size_t(t) * colbytes, ld, bw.info)
                      : enqueue_block<2>(h, bw, X + size_t(t) * colbytes, ld, bw.info);
      if (rc) break;
      took = block;
    }
    e = cudaMemcpyAsync(got, bw.info, sizeof(foa_dmd_push_info) * took, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      rc = cuda_status(e);
      break;
    }
    rc = sync_state(h, nullptr);
    if (rc) break;
    int32_t berr = 0;
    if (took > 1) {
      e = cudaMemcpy(&berr, &bw.bs->err, sizeof(int32_t), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess || berr) {
        rc = e != cudaSuccess ? cuda_status(e) : berr;
        break;
      }
    }
    int first_bad = FOA_DMD_OK;
    for (int i = 0; i < took; ++i) {
      if (infos) infos[t + i] = got[i];
      if (got[i].status != FOA_DMD_OK && first_bad == FOA_DMD_OK) first_bad = got[i].status;
    }
    t += took;
    if (first_bad != FOA_DMD_OK) {
      if (infos)
        for (int u = t; u < p; ++u) {
          infos[u] = got[took - 1];
          infos[u].status = first_bad == FOA_DMD_ERESOLVE ? FOA_DMD_ERESOLVE : FOA_DMD_ESTOPPED;
        }
      rc = first_bad;
      break;
    }
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(bw.W);
  cudaFree(bw.W64);
  cudaFree(bw.C1);
  cudaFree(bw.C);
  cudaFree(bw.bs);
  cudaFree(bw.info);
  return rc;
}
