// Host orchestration of the device eigen path: foa_dmd_eig and the push-time indicator schedule.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.cuh"
#include "eig_internal.cuh"

namespace foa {

static constexpr int kVecGridMax = 64;  // CTAs of the inverse-iteration kernel (each owns LU scratch)
static constexpr int kQrSmemMaxOrder = 160;  // largest order whose matrix (200 KB) the QR iteration keeps in shared memory

static void free_work(EigWork *w) {
  void *ptrs[] = {w->A,  w->U,  w->sig_raw, w->sig, w->G,      w->Q,     w->T,     w->Aqr,   w->wr,
                  w->wi, w->yr, w->yi,      w->ysr, w->ysi,    w->ind,   w->amp_re, w->amp_im, w->out,
                  w->anorm, w->lu, w->tw, w->yplanes, w->perm, w->isc, w->gb, w->bop, w->scal};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete w;
}

void eig_free(foa_dmd *h) {
  if (h->ind_stream) cudaStreamSynchronize(h->ind_stream);
  if (h->eig) free_work(h->eig);
  if (h->ind_eig) free_work(h->ind_eig);
  h->eig = h->ind_eig = nullptr;
  if (h->ind_ring) cudaFree(h->ind_ring);
  h->ind_ring = nullptr;
  if (h->ind_event) cudaEventDestroy(h->ind_event);
  h->ind_event = nullptr;
  if (h->ind_copied) cudaEventDestroy(h->ind_copied);
  h->ind_copied = nullptr;
  h->ind_copied_set = false;
  if (h->ind_stream) cudaStreamDestroy(h->ind_stream);
  h->ind_stream = nullptr;
}

static int eig_alloc(foa_dmd *h, EigWork **slot) {
  if (*slot) return FOA_DMD_OK;
  EigWork *w = new (std::nothrow) EigWork();
  if (!w) return FOA_DMD_ENOMEM;
  *slot = w;
  const int K = h->kmax;
  w->K = K;
  w->vgrid = kVecGridMax;
  const size_t K2 = size_t(K) * K * 8, K1 = size_t(K) * 8;
  cudaError_t e = cudaSuccess;
#define AL(p, b)                                          \
  do {                                                    \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(p), (b)); \
  } while (0)
  AL(w->A, K2); AL(w->U, K2); AL(w->sig_raw, K1); AL(w->sig, K1); AL(w->G, K2); AL(w->Q, K2); AL(w->T, K2);
  AL(w->Aqr, K2); AL(w->wr, K1); AL(w->wi, K1); AL(w->yr, K2); AL(w->yi, K2); AL(w->ysr, K2); AL(w->ysi, K2);
  AL(w->ind, K1); AL(w->amp_re, K1); AL(w->amp_im, K1); AL(w->out, OUT_N * K1); AL(w->anorm, 8);
  AL(w->lu, size_t(w->vgrid) * 2 * K2); AL(w->tw, size_t(w->vgrid) * 2 * K1); AL(w->yplanes, 2 * K2);
  AL(w->perm, size_t(K) * 4); AL(w->isc, ISC_N * 4); AL(w->gb, sizeof(GridBar));
  AL(w->bop, modes_tc_bop_bytes(K));
  AL(w->scal, 2 * 8);
#undef AL
  if (e == cudaSuccess) e = cudaMemset(w->gb, 0, sizeof(GridBar));
  if (e == cudaSuccess) e = cudaMemset(w->isc, 0, ISC_N * 4);
  if (e != cudaSuccess) {
    free_work(w);
    *slot = nullptr;
    return cuda_status(e);
  }
  return FOA_DMD_OK;
}

static double eps_of(int dtype) {
  return dtype == FOA_DMD_F64 ? std::ldexp(1.0, -52) : dtype == FOA_DMD_F32 ? std::ldexp(1.0, -23)
                                                                              : std::ldexp(1.0, -7);
}

struct EigOut {
  int m = 0, r = 0, status = FOA_DMD_OK;
  double hlast = 0.0;
  std::vector<double> out;  // OUT_N x K
};

// Enqueue the eigen path on stream s with workspace w for the projected matrix of size m: all
// launch sizes are bounded by m and the truncated rank r is read on the device, so nothing here
// waits for the GPU.  rank_tol as for foa_dmd_eig.
// copied (nullable) is recorded on s once the enqueued work has read the stream's state (H-bar,
// beta): right after copy_h_kernel on the untruncated path, at the end on the truncated one.
static int enqueue_eig(foa_dmd *h, EigWork *w, cudaStream_t s, int m, double rank_tol, int nsel,
                       cudaEvent_t copied = nullptr) {
  const int K = h->kmax;
  cudaError_t e = cudaMemsetAsync(w->isc, 0, ISC_N * 4, s);
  if (e != cudaSuccess) return cuda_status(e);
  double tol = 0.0;
  if (rank_tol > 0.0) tol = rank_tol;
  else if (rank_tol < 0.0) tol = (m + 1) * eps_of(h->dtype);
  const bool trunc = tol > 0.0;
  if (trunc) {
    // cooperative one-sided Jacobi SVD of beta_m (one CTA of four warps per column pair and round)
    int grid = (m + 1) / 2;
    if (grid > 2 * h->sms) grid = 2 * h->sms;
    if (grid < 1) grid = 1;
    const double *Bp = h->B;
    int ldb = K, mm = m, lda = K, sweeps = 30, *iscp = w->isc;
    double *Ap = w->A, *sigp = w->sig_raw, jt = 4.0 * std::ldexp(1.0, -53) * std::sqrt(double(m));
    GridBar *gbp = w->gb;
    long long spin = kGridSpinCycles;
    int skip = -1;
    if (h->test_skip_cta >= 0) {  // foa_dmd_test_wait_fault (one shot)
      skip = h->test_skip_cta < grid ? h->test_skip_cta : grid - 1;
      spin = h->test_spin_cycles;
      h->test_skip_cta = -1;
    }
    // a barrier that timed out keeps a partial count: every launch starts from a zeroed one
    e = cudaMemsetAsync(w->gb, 0, sizeof(GridBar), s);
    if (e != cudaSuccess) return cuda_status(e);
    void *args[] = {&Bp, &ldb, &mm, &Ap, &lda, &sigp, &iscp, &gbp, &sweeps, &jt, &spin, &skip};
    e = cudaLaunchCooperativeKernel((void *)svd_jacobi_kernel, grid, kSvdThreads, args, 0, s);
    if (e != cudaSuccess) return cuda_status(e);
    svd_finish_kernel<<<1, 512, size_t(m) * 12 + 64, s>>>(w->A, K, m, w->sig_raw, w->U, w->sig, w->isc, tol);
    project_t_kernel<<<h->sms * 2, 256, 0, s>>>(h->H, K, m, w->U, K, w->isc, w->T, K);
    project_g_kernel<<<h->sms * 2, 256, 0, s>>>(w->U, K, m, w->isc, w->T, K, w->G, K);
    hessenberg_kernel<<<1, 512, size_t(m) * 8 + 32 * 8, s>>>(w->G, K, w->Q, K, w->isc);
    h->launches += 5;
  } else {
    copy_h_kernel<<<h->sms, 256, 0, s>>>(h->H, K, m, w->G, K, w->isc, h->B, w->scal);
    if (copied) {
      e = cudaEventRecord(copied, s);
      if (e != cudaSuccess) return cuda_status(e);
    }
    h->launches += 1;
  }
  anorm_kernel<<<1, 512, 0, s>>>(w->G, K, w->isc, w->anorm);
  e = cudaMemcpyAsync(w->Aqr, w->G, size_t(K) * K * 8, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_status(e);
  // The QR iteration works on the r x r matrix (r = m without truncation); r is counted on the
  // device.  The launch offers the band |j - i| <= 3 (7 m doubles) and up to 160^2 doubles for the
  // whole matrix, which the kernel copies to shared memory when r^2 fits (every truncated eig with
  // r <= 160, whatever m).
  const size_t band = 7 * size_t(m);
  const size_t full = std::min(std::min(size_t(m) * m, size_t(kQrSmemMaxOrder) * kQrSmemMaxOrder),
                               size_t(232448 / 8) - band - 512);  // 4 KB left for the static variables
  const size_t qr_smem = (full + band) * 8;
  if (qr_smem > 48 * 1024) {
    e = cudaFuncSetAttribute(hqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(qr_smem));
    if (e != cudaSuccess) return cuda_status(e);
  }
  hqr_kernel<<<1, 512, qr_smem, s>>>(w->Aqr, K, w->isc, w->wr, w->wi, w->isc, int(full));
  EigArgs a;
  memset(&a, 0, sizeof(a));
  a.Hs = w->G;
  a.Q = w->Q;
  a.U = w->U;
  a.H = h->H;
  a.ldH = K;
  a.wr = w->wr;
  a.wi = w->wi;
  a.anorm = w->anorm;
  a.lu = w->lu;
  a.tw = w->tw;
  a.yr = w->yr;
  a.yi = w->yi;
  a.ysr = w->ysr;
  a.ysi = w->ysi;
  a.ind = w->ind;
  a.amp_re = w->amp_re;
  a.amp_im = w->amp_im;
  a.out = w->out;
  a.perm = w->perm;
  a.isc = w->isc;
  a.ld = K;
  a.m = m;
  a.have_q = trunc ? 1 : 0;
  a.have_u = trunc ? 1 : 0;
  a.hlast_p = trunc ? h->H + m + int64_t(m - 1) * K : w->scal;  // h_{m+1,m} (0 after a breakdown)
  a.b11_p = trunc ? h->B : w->scal + 1;
  const int vgrid = m < w->vgrid ? m : w->vgrid;
  const size_t vsmem = (size_t(m) * 10 + size_t(m + 1) / 2 + 64) * 8;
  vectors_kernel<<<vgrid, 256, vsmem, s>>>(a);
  if (nsel > m) nsel = m;
  order_kernel<<<1, 512, size_t(m) * 20 + 64, s>>>(a, nsel);
  h->launches += 4;  // anorm, hqr, vectors, order
  if (trunc && copied) {
    e = cudaEventRecord(copied, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return cuda_status(cudaGetLastError());
}

// Synchronous eigen path on the handle's stream; copies the sorted scalars back.
static int run_eig_body(foa_dmd *h, double rank_tol, int nsel, EigOut &res);
static int run_eig(foa_dmd *h, double rank_tol, int nsel, EigOut &res) {
  nvtxRangePushA("foa_dmd eig");
  const int rc = run_eig_body(h, rank_tol, nsel, res);
  nvtxRangePop();
  return rc;
}

static int run_eig_body(foa_dmd *h, double rank_tol, int nsel, EigOut &res) {
  int rc = sync_state(h, nullptr);
  if (rc) return rc;
  const int q = h->q_host;
  const int m = h->stopped_host ? q : q - 1;
  if (m < 1) return FOA_DMD_EINVAL;
  rc = eig_alloc(h, &h->eig);
  if (rc) return rc;
  EigWork *w = h->eig;
  const int K = h->kmax;
  cudaStream_t s = h->stream;
  rc = enqueue_eig(h, w, s, m, rank_tol, nsel);
  if (rc) return rc;
  res.out.resize(size_t(OUT_N) * K);
  int iscv[ISC_N];
  double hb = 0.0;
  cudaError_t e = cudaMemcpyAsync(res.out.data(), w->out, res.out.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(iscv, w->isc, sizeof(iscv), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, h->H + m + int64_t(m - 1) * K, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  if (iscv[ISC_ERR]) return iscv[ISC_ERR];
  res.m = m;
  res.r = iscv[ISC_R];
  res.hlast = hb;
  res.status = iscv[ISC_STATUS];
  return res.status;
}

// max of the error indicators of the n_lead leading modes into the indicator ring
__global__ void ind_record_kernel(const double *out, int ld, const int *isc, int n_lead, IndRecord *rec, int push,
                                  int m) {
  if (threadIdx.x != 0) return;
  const int r = isc[ISC_R];
  const int nl = r < n_lead ? r : n_lead;
  double v = 0.0;
  for (int i = 0; i < nl; ++i) v = fmax(v, out[OUT_IND * ld + i]);
  if (isc[ISC_STATUS] != FOA_DMD_OK || isc[ISC_ERR] != 0) v = __longlong_as_double(0x7ff8000000000000ll);
  rec->push = push;
  rec->m = m;
  rec->value = v;
}

// interleave the sorted y columns into real planes [Re y_0, Im y_0, Re y_1, ...] (m x 2 ncols)
__global__ void planes_kernel(const double *ysr, const double *ysi, int ld, int m, int ncols, double *Y) {
  const int64_t total = int64_t(m) * ncols;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t / m), i = int(t % m);
    Y[i + int64_t(2 * c) * ld] = ysr[i + int64_t(c) * ld];
    Y[i + int64_t(2 * c + 1) * ld] = ysi[i + int64_t(c) * ld];
  }
}

// The indicator schedule: every indicator_every-th push enqueues the eigen path for the projected
// matrix of that moment on a low-priority side stream (its own workspace), after the push's
// passes.  H-bar's leading m columns never change once written, so the eigensolve overlaps the
// following pushes; the streaming passes leave one SM free for it.  Results go to a device ring
// read by foa_dmd_indicators (and by a push that asks for its info).
int maybe_indicator(foa_dmd *h) {
  h->pushes_host += 1;
  h->ind_this_push = false;
  const int every = h->opts.indicator_every;
  if (every <= 0 || h->pushes_host % every != 0) return FOA_DMD_OK;
  const int m = h->stopped_host ? h->q_host : h->q_host - 1;
  if (m < 1) return FOA_DMD_OK;
  cudaError_t e = cudaSuccess;
  if (!h->ind_stream) {
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->ind_stream, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ind_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ind_copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&h->ind_ring, sizeof(IndRecord) * kIndRing);
    if (e != cudaSuccess) return cuda_status(e);
  }
  int rc = eig_alloc(h, &h->ind_eig);
  if (rc) return rc;
  e = cudaEventRecord(h->ind_event, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->ind_stream, h->ind_event, 0);
  if (e != cudaSuccess) return cuda_status(e);
  rc = enqueue_eig(h, h->ind_eig, h->ind_stream, m, h->opts.indicator_rank_tol, 0, h->ind_copied);
  if (rc) return rc;
  h->ind_copied_set = true;
  IndRecord *rec = static_cast<IndRecord *>(h->ind_ring) + (h->ind_issued % kIndRing);
  ind_record_kernel<<<1, 32, 0, h->ind_stream>>>(h->ind_eig->out, h->kmax, h->ind_eig->isc, h->opts.n_lead, rec,
                                                 h->pushes_host, m);
  h->launches += 1;
  h->ind_issued += 1;
  h->ind_pending = true;
  h->ind_this_push = true;
  return cuda_status(cudaGetLastError());
}

// Latest indicator value (synchronises the side stream); NaN when none was scheduled.
double latest_indicator(foa_dmd *h, bool only_if_pending) {
  if (!h->ind_stream || h->ind_issued == 0 || (only_if_pending && !h->ind_pending)) return NAN;
  IndRecord r;
  cudaError_t e = cudaStreamSynchronize(h->ind_stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(&r, static_cast<IndRecord *>(h->ind_ring) + ((h->ind_issued - 1) % kIndRing), sizeof(r),
                   cudaMemcpyDeviceToHost);
  h->ind_pending = false;
  return e == cudaSuccess ? r.value : NAN;
}

}  // namespace foa

using namespace foa;

extern "C" int foa_dmd_test_wait_fault(foa_dmd_t *h, int32_t skip_cta, int64_t spin_cycles) {
  if (!h || skip_cta < 0 || spin_cycles < 1 || spin_cycles > kGridSpinCycles) return FOA_DMD_EINVAL;
  h->test_skip_cta = skip_cta;
  h->test_spin_cycles = spin_cycles;
  return FOA_DMD_OK;
}

extern "C" int foa_dmd_eig(foa_dmd_t *h, double rank_tol, foa_dmd_eig_result *res) {
  if (!h || !res) return FOA_DMD_EINVAL;
  if (!res->lam_re || !res->lam_im || !res->indicator || !res->amp_re || !res->amp_im) return FOA_DMD_EINVAL;
  if (res->n_modes < 0 || res->vec_cols < 0) return FOA_DMD_EINVAL;
  if (res->n_modes > 0) {
    const int es = h->dtype == FOA_DMD_F64 ? 8 : 4;
    if (!res->phi_dev || res->ld_phi < h->n || ((res->ld_phi * es) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(res->phi_dev) & 15) != 0)
      return FOA_DMD_EINVAL;
  }
  if (res->vec_cols > 0 && (!res->vec_re || !res->vec_im)) return FOA_DMD_EINVAL;
  EigOut o;
  const int nsel = res->n_modes > res->vec_cols ? res->n_modes : res->vec_cols;
  int rc = run_eig(h, rank_tol, nsel, o);
  res->m = o.m;
  res->r = o.r;
  res->h_last = o.hlast;
  if (rc) return rc;
  if (o.r > res->cap) return FOA_DMD_EINVAL;
  const int K = h->kmax;
  for (int i = 0; i < o.r; ++i) {
    res->lam_re[i] = o.out[size_t(OUT_LRE) * K + i];
    res->lam_im[i] = o.out[size_t(OUT_LIM) * K + i];
    res->indicator[i] = o.out[size_t(OUT_IND) * K + i];
    res->amp_re[i] = o.out[size_t(OUT_ARE) * K + i];
    res->amp_im[i] = o.out[size_t(OUT_AIM) * K + i];
  }
  EigWork *w = h->eig;
  cudaError_t e = cudaSuccess;
  if (res->sigma) {
    if (rank_tol != 0.0) e = cudaMemcpy(res->sigma, w->sig, size_t(o.r) * 8, cudaMemcpyDeviceToHost);
    else
      for (int i = 0; i < o.r; ++i) res->sigma[i] = NAN;
  }
  if (e != cudaSuccess) return cuda_status(e);
  const int vc = res->vec_cols < o.r ? res->vec_cols : o.r;
  if (vc > 0) {
    e = cudaMemcpy2D(res->vec_re, size_t(o.m) * 8, w->ysr, size_t(K) * 8, size_t(o.m) * 8, vc, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy2D(res->vec_im, size_t(o.m) * 8, w->ysi, size_t(K) * 8, size_t(o.m) * 8, vc,
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
  }
  const int nm = res->n_modes < o.r ? res->n_modes : o.r;
  if (nm > 0) {
    rc = flush_pending(h);  // two-pass push: the last basis column may still be pending
    if (rc) return rc;
    planes_kernel<<<h->sms, 256, 0, h->stream>>>(w->ysr, w->ysi, K, o.m, nm, w->yplanes);
    h->launches += 2;  // planes and the modes GEMM
    rc = launch_modes(h, o.m, w->yplanes, K, 2 * nm, res->phi_dev, res->ld_phi);
    if (rc) return rc;
    int errv = 0;
    e = cudaMemcpyAsync(&errv, w->isc + ISC_ERR, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (errv) return errv;
  }
  return FOA_DMD_OK;
}
