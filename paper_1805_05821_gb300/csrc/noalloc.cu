// One push without any device allocation: foa_dmd_push_noalloc.
//
// Some callers cannot allocate device memory at the point where they need the update: code
// running under a memory pool or arena that owns all device memory, or plug-ins whose host
// application forbids cudaMalloc/cudaFree on its hot path (those calls may synchronise the
// device or fragment a carefully sized heap).  For them this entry point performs the same push
// as foa_dmd_push on buffers the caller already owns; the library's own per-push scratch (device
// state, beta_pre/h/s vectors, the per-CTA partial sums of the cross-CTA reduction and their
// counters) lives in one file-scope __device__ array of fixed size instead of memory obtained
// with cudaMalloc.  The call waits for its stream to finish the push before it returns.
#include <cstring>

#include "api_internal.cuh"
#include "push_kernels.cuh"

namespace foa {
namespace na {

constexpr int kMaxGrid = 1024;                 // CTAs of one streaming pass
constexpr int kGroups = kMaxGrid / kGroup + 1;
constexpr size_t kStateBytes = 1024;           // DevState, rounded up
constexpr size_t kVecBytes = 3 * size_t(kMaxK) * 8;
constexpr size_t kPartBytes = size_t(kMaxGrid) * (kMaxK + 1) * 8;
constexpr size_t kGpartBytes = size_t(kGroups) * (kMaxK + 1) * 8;
constexpr size_t kCountBytes = 1024;
constexpr size_t kScratchBytes = kStateBytes + kVecBytes + kPartBytes + kGpartBytes + kCountBytes;  // ~4.8 MB

// The scratch shared by every call on a device (held until the process exits).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once per device.
static void *g_addr[64];

// The caller's buffers are the whole stream state.  A breakdown leaves q unchanged and records
// h in H-bar column q (1-based), a column that is still zero on a stream that has not broken
// down; such a stream is marked stopped, so the push reports FOA_DMD_ESTOPPED as a handle would.
__global__ void init_state_kernel(DevState *st, int q, const double *Hbar, int ldh) {
  if (threadIdx.x == 0) {
    int stopped = 0;
    for (int i = 0; i < q && q > 0; ++i) stopped |= Hbar[i + int64_t(q - 1) * ldh] != 0.0;
    st->q = q;
    st->stopped = stopped;
  }
}

}  // namespace na
}  // namespace foa

using namespace foa;
using namespace foa::na;

extern "C" int foa_dmd_push_noalloc(int64_t n, int32_t k_max, int32_t dtype, void *V, double *Hbar, double *beta,
                                    int32_t q, const void *x_dev, void *w_dev, double breakdown_tol,
                                    void *cuda_stream, foa_dmd_push_info *info) {
  if (n < 1 || k_max < 2 || k_max > max_kmax_for(dtype) || dtype < 0 || dtype > 2 || !V || !Hbar || !beta || !x_dev ||
      !w_dev || !info || q < 0)
    return FOA_DMD_EINVAL;
  if (q >= k_max) return FOA_DMD_EFULL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FOA_DMD_ECUDA;
  int sms = 0;
  int rc = check_device(&sms);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the call synchronises its stream and copies to pageable host memory, neither of which a
  // stream capture allows: refuse before anything is enqueued
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &capture) != cudaSuccess || capture != cudaStreamCaptureStatusNone)
    return FOA_DMD_EINVAL;
  if (!g_addr[dev]) {
    // first call on this device: resolve the array's device address (must precede any capture)
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return FOA_DMD_ECUDA;
    g_addr[dev] = p;
  }
  unsigned char *base = static_cast<unsigned char *>(g_addr[dev]);
  DevState *st = reinterpret_cast<DevState *>(base);
  double *vec = reinterpret_cast<double *>(base + kStateBytes);
  double *partials = reinterpret_cast<double *>(base + kStateBytes + kVecBytes);
  double *gpart = reinterpret_cast<double *>(base + kStateBytes + kVecBytes + kPartBytes);
  uint32_t *gcount = reinterpret_cast<uint32_t *>(base + kStateBytes + kVecBytes + kPartBytes + kGpartBytes);

  // A stand-in handle that points at the caller's buffers and the static scratch.
  foa_dmd h;
  foa_dmd_opts_default(&h.opts);
  h.n = n;
  h.kmax = k_max;
  h.dtype = dtype;
  h.ntiles = int((n + kTile - 1) / kTile);
  h.nrows = int64_t(h.ntiles) * kTile;
  h.sms = sms;
  h.stream = s;
  h.tol = breakdown_tol > 0.0 ? breakdown_tol : default_tol(dtype);
  h.V = V;
  h.w = w_dev;
  h.H = Hbar;
  h.B = beta;
  h.pre = vec;
  h.hvec = vec + kMaxK;
  h.svec = vec + 2 * kMaxK;
  h.partials = partials;
  h.gpart = gpart;
  h.gcount = gcount;
  h.st = st;
  h.q_host = q;
  if (sms * h.geom.max_ctas_per_sm > kMaxGrid) return FOA_DMD_EINVAL;
  // everything the kernels expect to start at zero
  cudaError_t e = cudaMemsetAsync(st, 0, kStateBytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(gcount, 0, kCountBytes, s);
  if (e != cudaSuccess) return cuda_status(e);
  foa::na::init_state_kernel<<<1, 32, 0, s>>>(st, q, Hbar, k_max);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  rc = enqueue_push(&h, x_dev, false, nullptr);
  h.V = h.w = nullptr;  // the stand-in owns nothing
  if (rc) return rc;
  // one copy brings back the push result together with the sticky device error word
  DevState out;
  e = cudaMemcpyAsync(&out, st, sizeof(out), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  *info = out.info;
  if (out.err) return out.err;
  return info->status < 0 ? FOA_DMD_ECUDA : info->status;
}
