// C ABI of the library: handle lifetime, push sequencing, state access, checkpoints, profiling.
// Every numerical step runs in the kernels of this directory; this file only sizes launches,
// orders them on the handle's stream and moves small results to the host.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <unistd.h>

#include "api_internal.cuh"
#include "eig_internal.cuh"
#include "push_kernels.cuh"

using namespace foa;

namespace foa {

static inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

int max_kmax_for(int dtype) { return dtype == FOA_DMD_F64 ? 384 : kMaxK; }

// Shared-memory layout and grid of one streaming pass (the launch geometry depends only on the
// dtype, the pass kind, jcap and n, so identical pushes always get identical launches).
bool make_pass_geom(const Geometry &g, int dtype, int mode, int jcap, int64_t n, int ntiles, int sms, PassArgs &a,
                    int &grid) {
  const int s = dtype_size(dtype), cs = compute_size(dtype);
  const bool lag = (mode == PASS_A2 || mode == PASS_FIN);
  const bool basex = (mode == PASS_A || mode == PASS_FIRST);
  const int base_size = basex ? s : cs;
  const int jj = (mode == PASS_FIRST) ? 0 : jcap;
  const int64_t tile_bytes = int64_t(kTile) * jj * s;
  int R = 1;
  if (jj == 0) {
    R = kMaxR;
  } else {
    while (R * 2 <= kMaxR && (R * 2) * tile_bytes <= g.stage_bytes) R *= 2;
  }
  const int64_t vpart = align_up(R * tile_bytes, 128);
  // the lagged first pass also stages the x slice (storage type) and the w' slice (compute type)
  const int64_t bpart = lag ? align_up(int64_t(R) * kTile * s, 128) + align_up(int64_t(R) * kTile * cs, 128)
                            : align_up(int64_t(R) * kTile * base_size, 128);
  const int64_t slot_bytes = vpart + bpart;
  const int64_t ws_bytes = align_up(2 * int64_t(R) * kTile * cs, 128);
  const int64_t vnew_bytes = lag ? align_up(2 * int64_t(R) * kTile * cs, 128) : 0;  // double-buffered
  const int64_t cf_bytes = align_up(int64_t(jcap + 96) * cs, 16);  // room for the fused pass's padding
  const int64_t cf2_bytes = lag ? cf_bytes : 0;
  const int64_t comb_bytes = lag ? 2 * kConsumers * 8 : kConsumers * 8;
  const int64_t other = ws_bytes + vnew_bytes + cf_bytes + cf2_bytes + align_up(int64_t(jcap + 2) * 8, 16) +
                        comb_bytes + kConsumers * 8 + 2 * kMaxSlots * 8 + 64;
  // two CTAs per SM for FP32/BF16 while two slots fit in half the shared memory; otherwise one CTA
  // per SM with a deeper ring
  const bool two = (cs == 4) &&
                   (2 * slot_bytes + other <= g.smem_budget2) && g.max_ctas_per_sm >= 2;
  const int64_t budget = two ? g.smem_budget2 : g.smem_budget;
  const int64_t inflight = two ? g.inflight_bytes / 2 : g.inflight_bytes;
  int slots = int((budget - other) / slot_bytes);
  const int want = int((inflight + slot_bytes - 1) / slot_bytes) + 1;
  if (slots > want) slots = want;
  if (slots > kMaxSlots) slots = kMaxSlots;
  if (slots < 2) return false;
  a.R = R;
  a.slots = slots;
  a.variant = g.variant;
  a.slot_bytes = int(slot_bytes);
  a.base_off = int(vpart);
  a.base2_off = lag ? int(vpart + align_up(int64_t(R) * kTile * s, 128)) : 0;
  int64_t off = slot_bytes * slots;
  a.off_ws = int(off);
  off += ws_bytes;
  a.off_vnew = int(off);
  off += vnew_bytes;
  a.off_coef = int(off);
  off += cf_bytes;
  a.off_coef2 = int(off);
  off += cf2_bytes;
  a.off_dot = int(off);
  off += align_up(int64_t(jcap + 2) * 8, 16);
  a.off_comb = int(off);
  off += comb_bytes;
  a.off_norm = int(off);
  off += kConsumers * 8;
  a.off_bar = int(off);
  off += 2 * kMaxSlots * 8 + 64;
  a.smem_total = int(off);
  if (a.smem_total > 232448) return false;
  a.ntiles = ntiles;
  a.n = n;
  a.jcap = jcap;
  a.nstages = (ntiles + R - 1) / R;
  const int per_sm = two ? 2 : 1;
  grid = a.nstages < sms * per_sm ? a.nstages : sms * per_sm;
  return true;
}

}  // namespace foa

static const char *kErr[] = {"ok",
                             "invalid argument",
                             "out of memory",
                             "CUDA error or no sm_103 device",
                             "basis full (q == k_max)",
                             "breakdown: snapshot linearly dependent on the previous ones",
                             "stream stopped by an earlier breakdown",
                             "snapshot holds NaN or Inf",
                             "device wait timed out",
                             "checkpoint I/O error",
                             "eigensolver did not converge",
                             "block push cannot resolve the snapshot's new direction; push it singly"};

extern "C" const char *foa_dmd_strerror(int status) {
  if (status < 0 || status > FOA_DMD_ERESOLVE) return "unknown status";
  return kErr[status];
}

extern "C" void foa_dmd_opts_default(foa_dmd_opts *o) {
  if (!o) return;
  o->reorth = 1;
  o->breakdown_tol = 0.0;
  o->indicator_every = 0;
  o->n_lead = 32;
  o->indicator_rank_tol = 0.0;
  o->cuda_stream = nullptr;
  o->form = 0;
}

namespace foa {

double default_tol(int dtype) {
  const double u = dtype == FOA_DMD_F64 ? std::ldexp(1.0, -53) : dtype == FOA_DMD_F32 ? std::ldexp(1.0, -24)
                                                                                        : std::ldexp(1.0, -8);
  return std::sqrt(u);
}

int check_device(int *sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FOA_DMD_ECUDA;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return FOA_DMD_ECUDA;
  if (p.major != 10 || p.minor != 3) return FOA_DMD_ECUDA;
  *sms = p.multiProcessorCount;
  return FOA_DMD_OK;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FOA_DMD_OK;
  if (e == cudaErrorMemoryAllocation) return FOA_DMD_ENOMEM;
  return FOA_DMD_ECUDA;
}

void free_handle_buffers(foa_dmd *h) {
  void *ptrs[] = {h->V, h->w, h->H, h->B, h->pre, h->hvec, h->svec, h->partials, h->gpart, h->gcount, h->st,
                  h->info_dev, h->stage_x};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (auto &e : h->events) {
    cudaEventDestroy(e.start);
    cudaEventDestroy(e.stop);
  }
  for (int b = 0; b < 2; ++b) {
    if (h->stage_free[b]) cudaEventDestroy(h->stage_free[b]);
    if (h->stage_ready[b]) cudaEventDestroy(h->stage_ready[b]);
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  h->events.clear();
  eig_free(h);
}

int sync_state(foa_dmd *h, foa_dmd_push_info *info) {
  DevState st;
  cudaError_t e = cudaMemcpyAsync(&st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  h->q_host = st.q;
  h->stopped_host = st.stopped != 0;
  if (info) *info = st.info;
  if (st.err) return st.err;
  return FOA_DMD_OK;
}

int alloc_handle(foa_dmd *h) {
  const int64_t nrows = h->nrows;
  const int s = dtype_size(h->dtype), cs = compute_size(h->dtype);
  const int K = h->kmax;
  const int maxgrid = h->sms * 8;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes)                                  \
  do {                                                     \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes)); \
  } while (0)
  ALLOC(h->V, size_t(nrows) * K * s);
  ALLOC(h->w, size_t(nrows) * cs);
  ALLOC(h->H, size_t(K) * K * 8);
  ALLOC(h->B, size_t(K) * K * 8);
  ALLOC(h->pre, size_t(K) * 8);
  ALLOC(h->hvec, size_t(K) * 8);
  ALLOC(h->svec, size_t(K) * 8);
  ALLOC(h->partials, size_t(maxgrid) * (K + 1) * 8);
  ALLOC(h->gpart, size_t(maxgrid / kGroup + 1) * (K + 1) * 8);
  ALLOC(h->gcount, size_t(maxgrid / kGroup + 1) * 4);
  ALLOC(h->st, sizeof(DevState));
  ALLOC(h->info_dev, size_t(K + 1) * sizeof(foa_dmd_push_info));
#undef ALLOC
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(h->V, 0, size_t(nrows) * K * s, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->w, 0, size_t(nrows) * cs, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->H, 0, size_t(K) * K * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->B, 0, size_t(K) * K * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->pre, 0, size_t(K) * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->hvec, 0, size_t(K) * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->svec, 0, size_t(K) * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->gcount, 0, size_t(maxgrid / kGroup + 1) * 4, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return cuda_status(e);
}

int launch_pass_h(foa_dmd *h, int mode, int jcap, const void *x, const double *coef, bool batch,
                  foa_dmd_push_info *info_out) {
  PassArgs a;
  memset(&a, 0, sizeof(a));
  int grid = 0;
  // with an indicator schedule one SM is left to the side-stream eigensolve
  const int sms = h->sms - (h->opts.indicator_every > 0 ? 1 : 0);
  if (!make_pass_geom(geom_for(h, mode, jcap), h->dtype, mode, jcap, h->n, h->ntiles, sms, a, grid))
    return FOA_DMD_EINVAL;
  a.V = h->V;
  a.x = x;
  a.w = h->w;
  a.coef = coef;
  a.coef2 = h->svec;
  a.partials = h->partials;
  a.gpart = h->gpart;
  a.gcount = h->gcount;
  a.st = h->st;
  a.H = h->H;
  a.B = h->B;
  a.pre = h->pre;
  a.hvec = h->hvec;
  a.svec = h->svec;
  a.info_out = info_out;
  a.kmax = h->kmax;
  a.reorth = h->opts.reorth;
  a.x_aligned = x ? ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) : 0;
  a.batch = batch ? 1 : 0;
  a.form = h->opts.form;
  a.tol = h->tol;
  const double s = dtype_size(h->dtype), cs = compute_size(h->dtype), n = double(h->n);
  double bytes = 0.0;
  int kind = 0;
  switch (mode) {
    case PASS_A: bytes = n * jcap * s + n * s + n * cs; kind = 0; break;
    case PASS_B: bytes = n * jcap * s + 2 * n * cs; kind = 1; break;
    case PASS_C: bytes = n * jcap * s + 2 * n * cs; kind = 2; break;
    // lagged first pass: V (jcap - 1 stored columns) + x + w' read, the new column and w written
    case PASS_A2: bytes = n * (jcap - 1) * s + n * s + n * cs + n * s + n * cs; kind = 0; break;
    case PASS_B2: bytes = n * jcap * s + 2 * n * cs; kind = 1; break;
    case PASS_FIN: bytes = n * (jcap - 1) * s + n * cs + n * s; kind = 3; break;
    default: bytes = n * s; kind = 3; break;
  }
  ProfScope ps(h, kind, bytes);
  h->launches += 1;
  return cuda_status(launch_pass(h->dtype, mode, pass_nc_for(jcap), a, grid, h->stream));
}

// Enqueue one push (Alg. 4, p = 1).  jcap = host upper bound of q.
int enqueue_push(foa_dmd *h, const void *x, bool batch, foa_dmd_push_info *info_out) {
  const bool first = h->q_host == 0;
  const int jcap = h->q_host;
  int rc = cuda_status(launch_prep(h->st, h->H, h->B, h->pre, h->kmax, first ? 1 : 0, jcap, h->stream, batch ? 1 : 0,
                                   info_out));
  h->launches += 2;  // prep and the column write
  if (rc) return rc;
  if (first) {
    rc = launch_pass_h(h, PASS_FIRST, 0, x, nullptr, batch, info_out);
    if (rc) return rc;
    {
      ProfScope ps(h, 3, double(h->n) * 2 * dtype_size(h->dtype));
      rc = cuda_status(launch_colwrite(h->dtype, h->V, x, true, h->st, h->n, h->nrows, h->kmax, h->sms, h->stream));
    }
    if (rc) return rc;
  } else if (h->opts.reorth == 2) {
    // two-pass push: the lagged first pass appends the column left pending by the previous push
    // (if any) and projects x; the second pass commits h_{j+1,j} and leaves v_{j+1} pending
    h->launches -= 1;  // no column write
    rc = launch_pass_h(h, PASS_A2, jcap, x, h->pre, batch, info_out);
    if (rc) return rc;
    rc = launch_pass_h(h, PASS_B2, jcap, nullptr, h->hvec, batch, info_out);
    if (rc) return rc;
  } else {
    rc = launch_pass_h(h, PASS_A, jcap, x, h->pre, batch, info_out);
    if (rc) return rc;
    if (h->opts.reorth) {
      rc = launch_pass_h(h, PASS_B, jcap, nullptr, h->hvec, batch, info_out);
      if (rc) return rc;
    }
    rc = launch_pass_h(h, PASS_C, jcap, nullptr, h->opts.reorth ? h->svec : h->hvec, batch, info_out);
    if (rc) return rc;
    {
      ProfScope ps(h, 3, double(h->n) * (compute_size(h->dtype) + dtype_size(h->dtype)));
      rc = cuda_status(launch_colwrite(h->dtype, h->V, h->w, false, h->st, h->n, h->nrows, h->kmax, h->sms,
                                       h->stream));
    }
    if (rc) return rc;
  }
  h->q_host += 1;
  return FOA_DMD_OK;
}

// Two-pass push: write the pending basis column (if any) before V is read outside a push.
int flush_pending(foa_dmd *h) {
  if (h->opts.reorth != 2 || h->q_host < 2) return FOA_DMD_OK;
  return launch_pass_h(h, PASS_FIN, h->q_host, nullptr, nullptr, false, nullptr);
}

}  // namespace foa

extern "C" int foa_dmd_create(int64_t n, int32_t k_max, int32_t dtype, const foa_dmd_opts *opts, foa_dmd_t **out) {
  if (!out) return FOA_DMD_EINVAL;
  *out = nullptr;
  if (n < 1 || dtype < 0 || dtype > 2 || k_max < 2 || k_max > max_kmax_for(dtype)) return FOA_DMD_EINVAL;
  if (opts && (opts->reorth < 0 || opts->reorth > 2)) return FOA_DMD_EINVAL;
  if (opts && (opts->form < 0 || opts->form > 1 || (opts->form == 1 && opts->reorth == 2))) return FOA_DMD_EINVAL;
  int sms = 0;
  int rc = check_device(&sms);
  if (rc) return rc;
  foa_dmd *h = new (std::nothrow) foa_dmd();
  if (!h) return FOA_DMD_ENOMEM;
  if (opts) h->opts = *opts;
  else foa_dmd_opts_default(&h->opts);
  if (h->opts.n_lead <= 0) h->opts.n_lead = 32;
  h->n = n;
  h->kmax = k_max;
  h->dtype = dtype;
  h->ntiles = int((n + kTile - 1) / kTile);
  h->nrows = int64_t(h->ntiles) * kTile;
  h->sms = sms;
  h->stream = static_cast<cudaStream_t>(h->opts.cuda_stream);
  h->tol = h->opts.breakdown_tol > 0.0 ? h->opts.breakdown_tol : default_tol(dtype);
  h->geom = Geometry();
  rc = alloc_handle(h);
  if (rc) {
    free_handle_buffers(h);
    delete h;
    return rc;
  }
  *out = h;
  return FOA_DMD_OK;
}

extern "C" void foa_dmd_destroy(foa_dmd_t *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_handle_buffers(h);
  delete h;
}

static int finish_push(foa_dmd *h, foa_dmd_push_info *info, bool force_sync) {
  if (!info && !force_sync) return FOA_DMD_OK;
  foa_dmd_push_info inf;
  int rc = sync_state(h, &inf);
  if (rc) return rc;
  if (h->ind_this_push) inf.indicator = latest_indicator(h, false);
  if (info) *info = inf;
  return inf.status < 0 ? FOA_DMD_ECUDA : inf.status;
}

extern "C" int foa_dmd_push(foa_dmd_t *h, const void *x_dev, foa_dmd_push_info *info) {
  if (!h || !x_dev) return FOA_DMD_EINVAL;
  if (h->stopped_host) return FOA_DMD_ESTOPPED;
  if (h->q_host >= h->kmax) return FOA_DMD_EFULL;
  const bool first = h->q_host == 0;
  int rc = enqueue_push(h, x_dev, false, nullptr);
  if (rc) return rc;
  rc = maybe_indicator(h);
  if (rc) return rc;
  return finish_push(h, info, first);
}

extern "C" int foa_dmd_push_batch(foa_dmd_t *h, const void *X_dev, int32_t p, int64_t ld, foa_dmd_push_info *infos) {
  if (!h || !X_dev || p < 0 || ld < h->n) return FOA_DMD_EINVAL;
  if (p == 0) return FOA_DMD_OK;
  if (((ld * dtype_size(h->dtype)) & 15) != 0) return FOA_DMD_EINVAL;
  if (h->stopped_host) return FOA_DMD_ESTOPPED;
  if (h->q_host >= h->kmax) return FOA_DMD_EFULL;
  cudaError_t e = cudaMemsetAsync(&h->st->halt, 0, sizeof(int32_t), h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  const char *X = static_cast<const char *>(X_dev);
  const size_t colbytes = size_t(ld) * dtype_size(h->dtype);
  int first_rc = FOA_DMD_OK;
  int done = 0;
  for (int t = 0; t < p; ++t) {
    if (h->q_host >= h->kmax) break;
    const bool first = h->q_host == 0;
    foa_dmd_push_info *slot = infos ? h->info_dev + (t % (h->kmax + 1)) : nullptr;
    int rc = enqueue_push(h, X + size_t(t) * colbytes, true, slot);
    if (rc) return rc;
    rc = maybe_indicator(h);
    if (rc) return rc;
    ++done;
    if (first) {  // the first push of a stream is synchronous
      foa_dmd_push_info inf;
      rc = sync_state(h, &inf);
      if (rc) return rc;
      if (inf.status != FOA_DMD_OK) {
        if (infos) {
          infos[t] = inf;
          for (int u = t + 1; u < p; ++u) {
            infos[u] = inf;
            infos[u].status = FOA_DMD_ESTOPPED;
          }
        }
        return inf.status;
      }
    }
    if (infos && (t + 1) % (h->kmax + 1) == 0) {
      e = cudaMemcpyAsync(infos + (t + 1 - (h->kmax + 1)), h->info_dev, size_t(h->kmax + 1) * sizeof(foa_dmd_push_info),
                          cudaMemcpyDeviceToHost, h->stream);
      if (e != cudaSuccess) return cuda_status(e);
    }
  }
  if (infos) {
    const int rem = done % (h->kmax + 1);
    if (rem) {
      e = cudaMemcpyAsync(infos + (done - rem), h->info_dev, size_t(rem) * sizeof(foa_dmd_push_info),
                          cudaMemcpyDeviceToHost, h->stream);
      if (e != cudaSuccess) return cuda_status(e);
    }
    for (int u = done; u < p; ++u) {
      infos[u].status = FOA_DMD_EFULL;
      infos[u].h_last = NAN;
      infos[u].indicator = NAN;
      infos[u].x_norm = NAN;
      infos[u].q = h->kmax;
    }
    int rc = sync_state(h, nullptr);
    if (rc) return rc;
    for (int u = 0; u < p; ++u)
      if (infos[u].status != FOA_DMD_OK) {
        first_rc = infos[u].status;
        break;
      }
    return first_rc;
  }
  return FOA_DMD_OK;
}

// Check words of the translation units of a self-checking build, registered at load time.
static std::vector<cudaError_t (*)(unsigned *)> &check_readers() {
  static std::vector<cudaError_t (*)(unsigned *)> r;
  return r;
}
namespace foa {
int foa_check_register(cudaError_t (*read_and_clear)(unsigned *)) {
  check_readers().push_back(read_and_clear);
  return int(check_readers().size());
}
}  // namespace foa

extern "C" int foa_dmd_check_status(uint32_t *bits) {
  if (!bits) return FOA_DMD_EINVAL;
  *bits = 0;
#ifdef FOA_DMD_CHECKED
  cudaError_t e = cudaDeviceSynchronize();
  unsigned v = 0;
  for (auto rd : check_readers())
    if (e == cudaSuccess) e = rd(&v);
  *bits = v;
  return cuda_status(e);
#else
  return FOA_DMD_EINVAL;  // no checks compiled into this build
#endif
}

// One read per host page of [p, p + bytes) on the calling thread.  Measured on GB300 (Grace host,
// 64 KB pages): copies out of pinned pages that had gone unused for seconds ran at 9-37 GB/s
// instead of 208 GB/s, which made the first pushes of a 103 GB stream copy-bound (37.7 against
// 41.8 snapshots/s from device memory); a CPU read of each page shortly before its copy restored
// the full copy rate (41.3 snapshots/s).  The reads cost about a millisecond per 268 MB snapshot.
// Only host memory (pinned or not) is read: a device or managed pointer is left to the copy,
// which reports it.
static void touch_host_pages(const void *p, size_t bytes) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (at.type != cudaMemoryTypeHost && at.type != cudaMemoryTypeUnregistered) return;
  static const size_t page = sysconf(_SC_PAGESIZE) > 0 ? size_t(sysconf(_SC_PAGESIZE)) : 4096;
  const volatile unsigned char *c = static_cast<const volatile unsigned char *>(p);
  unsigned char acc = 0;
  for (size_t o = 0; o < bytes; o += page) acc = static_cast<unsigned char>(acc ^ c[o]);
  if (bytes) acc = static_cast<unsigned char>(acc ^ c[bytes - 1]);
  (void)acc;
}

extern "C" int foa_dmd_push_host(foa_dmd_t *h, const void *x_host, foa_dmd_push_info *info) {
  if (!h || !x_host) return FOA_DMD_EINVAL;
  if (h->stopped_host) return FOA_DMD_ESTOPPED;
  if (h->q_host >= h->kmax) return FOA_DMD_EFULL;
  const size_t bytes = size_t(h->n) * dtype_size(h->dtype);
  const size_t slot = size_t(align_up(int64_t(bytes), 256));
  cudaError_t e = cudaSuccess;
  if (!h->stage_x) {
    e = cudaMalloc(&h->stage_x, 2 * slot);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&h->stage_free[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->stage_ready[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(h->stage_free[b], h->stream);
    }
    if (e != cudaSuccess) return cuda_status(e);
  }
  // Double-buffered staging: the copy of this snapshot (copy stream) overlaps the previous push
  // (handle stream); a buffer is refilled only after the push that read it has finished.
  const int b = h->stage_flip;
  h->stage_flip ^= 1;
  char *buf = static_cast<char *>(h->stage_x) + (b ? slot : 0);
  touch_host_pages(x_host, bytes);
  e = cudaStreamWaitEvent(h->copy_stream, h->stage_free[b], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf, x_host, bytes, cudaMemcpyHostToDevice, h->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->stage_ready[b], h->copy_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->stage_ready[b], 0);
  if (e != cudaSuccess) return cuda_status(e);
  const bool first = h->q_host == 0;
  int rc = enqueue_push(h, buf, false, nullptr);
  if (rc) return rc;
  e = cudaEventRecord(h->stage_free[b], h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  rc = maybe_indicator(h);
  if (rc) return rc;
  return finish_push(h, info, first);
}

extern "C" int foa_dmd_sync(foa_dmd_t *h, foa_dmd_push_info *info) {
  if (!h) return FOA_DMD_EINVAL;
  foa_dmd_push_info inf;
  int rc = sync_state(h, &inf);
  if (rc) return rc;
  if (info) *info = inf;
  return inf.status < 0 ? FOA_DMD_OK : inf.status;
}

extern "C" int foa_dmd_get_state(foa_dmd_t *h, int32_t *q, int32_t *stopped, double *Hbar, double *beta, int32_t ld) {
  if (!h || ld < h->kmax) return FOA_DMD_EINVAL;
  int rc = sync_state(h, nullptr);
  if (rc) return rc;
  if (q) *q = h->q_host;
  if (stopped) *stopped = h->stopped_host ? 1 : 0;
  const int K = h->kmax;
  cudaError_t e = cudaSuccess;
  if (Hbar) e = cudaMemcpy2D(Hbar, size_t(ld) * 8, h->H, size_t(K) * 8, size_t(K) * 8, K, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && beta)
    e = cudaMemcpy2D(beta, size_t(ld) * 8, h->B, size_t(K) * 8, size_t(K) * 8, K, cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

extern "C" int foa_dmd_get_basis(foa_dmd_t *h, int32_t col0, int32_t ncols, void *dst_dev, int64_t ld) {
  if (!h || !dst_dev || col0 < 0 || ncols < 0 || col0 + ncols > h->kmax || ld < h->n) return FOA_DMD_EINVAL;
  if (ncols == 0) return FOA_DMD_OK;
  const int rc = flush_pending(h);
  if (rc) return rc;
  return cuda_status(launch_gather(h->dtype, h->V, dst_dev, ld, h->n, h->kmax, col0, ncols, h->sms, h->stream));
}

extern "C" int foa_dmd_reset(foa_dmd_t *h) {
  if (!h) return FOA_DMD_EINVAL;
  if (h->ind_stream && h->ind_copied_set) {
    // the side stream's eigensolve works on its own copies once it has read H-bar and beta: the
    // reset's clearing waits for that read only, and the eigensolve may overlap the next pushes
    cudaError_t e0 = cudaStreamWaitEvent(h->stream, h->ind_copied, 0);
    if (e0 != cudaSuccess) return cuda_status(e0);
  }
  h->pushes_host = 0;
  cudaError_t e = cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->H, 0, size_t(h->kmax) * h->kmax * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->B, 0, size_t(h->kmax) * h->kmax * 8, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  // V columns beyond q are never read before they are written, so V need not be cleared.
  h->q_host = 0;
  h->stopped_host = false;
  return FOA_DMD_OK;
}

// ------------------------------------------------------------------------------ checkpoints
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, dtype, kmax, q;
  int64_t n;
  int32_t stopped, pad;
  uint64_t checksum;
};
uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}
}  // namespace

extern "C" int foa_dmd_save(foa_dmd_t *h, const char *path) {
  if (!h || !path) return FOA_DMD_EINVAL;
  int rc = flush_pending(h);
  if (rc) return rc;
  rc = sync_state(h, nullptr);
  if (rc) return rc;
  const int K = h->kmax, q = h->q_host;
  const size_t s = dtype_size(h->dtype);
  std::vector<double> H(size_t(K) * K), B(size_t(K) * K);
  std::vector<char> V(size_t(h->n) * q * s);
  cudaError_t e = cudaMemcpy(H.data(), h->H, H.size() * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(B.data(), h->B, B.size() * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (q > 0) {
    void *tmp = nullptr;
    e = cudaMalloc(&tmp, V.size());
    if (e != cudaSuccess) return cuda_status(e);
    rc = cuda_status(launch_gather(h->dtype, h->V, tmp, h->n, h->n, K, 0, q, h->sms, h->stream));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(h->stream));
    if (!rc) rc = cuda_status(cudaMemcpy(V.data(), tmp, V.size(), cudaMemcpyDeviceToHost));
    cudaFree(tmp);
    if (rc) return rc;
  }
  CkptHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "FOADMD1", 8);
  hd.version = 1;
  hd.dtype = h->dtype;
  hd.kmax = K;
  hd.q = q;
  hd.n = h->n;
  hd.stopped = h->stopped_host ? 1 : 0;
  uint64_t cs = 1469598103934665603ull;
  cs = fnv1a(cs, H.data(), H.size() * 8);
  cs = fnv1a(cs, B.data(), B.size() * 8);
  cs = fnv1a(cs, V.data(), V.size());
  hd.checksum = cs;
  FILE *f = fopen(path, "wb");
  if (!f) return FOA_DMD_EIO;
  bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(H.data(), 8, H.size(), f) == H.size() &&
            fwrite(B.data(), 8, B.size(), f) == B.size() && (V.empty() || fwrite(V.data(), 1, V.size(), f) == V.size());
  ok = (fclose(f) == 0) && ok;
  return ok ? FOA_DMD_OK : FOA_DMD_EIO;
}

extern "C" int foa_dmd_load(const char *path, const foa_dmd_opts *opts, foa_dmd_t **out) {
  if (!path || !out) return FOA_DMD_EINVAL;
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) return FOA_DMD_EIO;
  CkptHeader hd;
  if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, "FOADMD1", 8) != 0 || hd.version != 1 || hd.kmax < 2 ||
      hd.kmax > kMaxK || hd.q < 0 || hd.q > hd.kmax || hd.n < 1 || hd.dtype < 0 || hd.dtype > 2) {
    fclose(f);
    return FOA_DMD_EIO;
  }
  const int K = hd.kmax;
  const size_t s = dtype_size(hd.dtype);
  std::vector<double> H(size_t(K) * K), B(size_t(K) * K);
  std::vector<char> V(size_t(hd.n) * hd.q * s);
  bool ok = fread(H.data(), 8, H.size(), f) == H.size() && fread(B.data(), 8, B.size(), f) == B.size() &&
            (V.empty() || fread(V.data(), 1, V.size(), f) == V.size());
  fclose(f);
  if (!ok) return FOA_DMD_EIO;
  uint64_t cs = 1469598103934665603ull;
  cs = fnv1a(cs, H.data(), H.size() * 8);
  cs = fnv1a(cs, B.data(), B.size() * 8);
  cs = fnv1a(cs, V.data(), V.size());
  if (cs != hd.checksum) return FOA_DMD_EIO;
  foa_dmd_t *h = nullptr;
  int rc = foa_dmd_create(hd.n, K, hd.dtype, opts, &h);
  if (rc) return rc;
  cudaError_t e = cudaMemcpy(h->H, H.data(), H.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->B, B.data(), B.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && hd.q > 0) {
    void *tmp = nullptr;
    e = cudaMalloc(&tmp, V.size());
    if (e == cudaSuccess) e = cudaMemcpy(tmp, V.data(), V.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = launch_scatter(hd.dtype, h->V, tmp, hd.n, hd.n, K, 0, hd.q, h->sms, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
  }
  if (e == cudaSuccess) {
    DevState st;
    memset(&st, 0, sizeof(st));
    st.q = hd.q;
    st.stopped = hd.stopped;
    st.status = FOA_DMD_OK;
    st.info.q = hd.q;
    e = cudaMemcpy(h->st, &st, sizeof(st), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    foa_dmd_destroy(h);
    return cuda_status(e);
  }
  h->q_host = hd.q;
  h->stopped_host = hd.stopped != 0;
  *out = h;
  return FOA_DMD_OK;
}

// ------------------------------------------------------------------------------ profiling
extern "C" int foa_dmd_profile(foa_dmd_t *h, int enable) {
  if (!h) return FOA_DMD_EINVAL;
  h->prof = enable != 0;
  return FOA_DMD_OK;
}

extern "C" int foa_dmd_profile_read(foa_dmd_t *h, foa_dmd_kernel_stats *stats) {
  if (!h || !stats) return FOA_DMD_EINVAL;
  memset(stats, 0, sizeof(*stats));
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  for (size_t i = 0; i < h->prof_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->events[i].start, h->events[i].stop) != cudaSuccess) continue;
    const int k = h->events[i].kind;
    stats->ms[k] += ms;
    stats->bytes[k] += h->events[i].bytes;
    stats->launches[k] += 1;
  }
  stats->total_launches = h->launches;
  h->launches = 0;
  h->prof_used = 0;
  return FOA_DMD_OK;
}

extern "C" int foa_dmd_host_alloc(size_t bytes, void **ptr) {
  if (!ptr || bytes == 0) return FOA_DMD_EINVAL;
  return cuda_status(cudaHostAlloc(ptr, bytes, cudaHostAllocDefault));
}

extern "C" int foa_dmd_host_free(void *ptr) { return cuda_status(cudaFreeHost(ptr)); }

extern "C" int foa_dmd_indicators(foa_dmd_t *h, int32_t *push_index, int32_t *m, double *value, int32_t cap,
                                  int32_t *count) {
  if (!h || !count || cap < 0) return FOA_DMD_EINVAL;
  *count = 0;
  if (!h->ind_stream) return FOA_DMD_OK;
  cudaError_t e = cudaStreamSynchronize(h->ind_stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (h->ind_issued - h->ind_read > kIndRing) h->ind_read = h->ind_issued - kIndRing;
  std::vector<IndRecord> recs(static_cast<size_t>(kIndRing));
  e = cudaMemcpy(recs.data(), h->ind_ring, sizeof(IndRecord) * kIndRing, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  int k = 0;
  for (; h->ind_read < h->ind_issued && k < cap; ++h->ind_read, ++k) {
    const IndRecord &r = recs[size_t(h->ind_read % kIndRing)];
    if (push_index) push_index[k] = r.push;
    if (m) m[k] = r.m;
    if (value) value[k] = r.value;
  }
  h->ind_pending = false;
  *count = k;
  return FOA_DMD_OK;
}
