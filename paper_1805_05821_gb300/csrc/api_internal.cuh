// Host-side handle of one snapshot stream and helpers shared by the API translation units.
#pragma once
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

namespace foa {

// Launch-geometry knobs of the streaming passes (set per handle; the autotuner may change them).
struct Geometry {
  int64_t stage_bytes = 32 * 1024;     // target bytes of V per pipeline stage
  int64_t smem_budget = 220 * 1024;    // shared memory of a CTA when one CTA runs per SM
  int64_t smem_budget2 = 112 * 1024;   // ... when two CTAs share an SM
  int64_t inflight_bytes = 96 * 1024;  // bytes of V each CTA keeps in flight
  int max_ctas_per_sm = 2;
  int variant = 0;  // FP32/BF16 passes A, B, B2: 0 = register-held stage where it fits, 1 = shared memory
};

struct EventPair {
  cudaEvent_t start, stop;
  int kind;
  double bytes;
};

struct EigWork;  // device workspace of the eigensolver (eig.cu)

constexpr int kTuneKinds = 5;     // pass kinds with their own tuned geometry: A, B, C, A2, B2
constexpr int kTuneBuckets = 11;  // j buckets (upper ends 8, 16, 32, 64, 128, 192, ..., 512)

}  // namespace foa

struct foa_dmd {
  int64_t n = 0;
  int kmax = 0;
  int dtype = 0;
  int ntiles = 0;
  int64_t nrows = 0;
  int sms = 0;
  foa_dmd_opts opts;
  cudaStream_t stream = nullptr;
  double tol = 0.0;
  foa::Geometry geom;
  foa::Geometry tuned[foa::kTuneKinds][foa::kTuneBuckets];  // foa_dmd_autotune's choices
  bool tuned_ok[foa::kTuneKinds][foa::kTuneBuckets] = {};
  void *V = nullptr;
  void *w = nullptr;
  double *H = nullptr, *B = nullptr, *pre = nullptr, *hvec = nullptr, *svec = nullptr;
  double *partials = nullptr, *gpart = nullptr;
  uint32_t *gcount = nullptr;
  foa::DevState *st = nullptr;
  foa_dmd_push_info *info_dev = nullptr;
  void *stage_x = nullptr;
  int stage_flip = 0;
  cudaStream_t copy_stream = nullptr;        // host->device snapshot copies (foa_dmd_push_host)
  cudaEvent_t stage_free[2] = {nullptr, nullptr}, stage_ready[2] = {nullptr, nullptr};
  int64_t launches = 0;                      // kernels launched by this handle
  int q_host = 0;
  bool stopped_host = false;
  int pushes_host = 0;
  bool prof = false;
  size_t prof_used = 0;
  std::vector<foa::EventPair> events;
  foa::EigWork *eig = nullptr;
  // push-time indicator (side stream)
  foa::EigWork *ind_eig = nullptr;
  cudaStream_t ind_stream = nullptr;
  cudaEvent_t ind_event = nullptr;
  cudaEvent_t ind_copied = nullptr;  // recorded once the latest indicator eigensolve has read H-bar/beta
  bool ind_copied_set = false;
  void *ind_ring = nullptr;
  int64_t ind_issued = 0, ind_read = 0;
  bool ind_pending = false;
  bool ind_this_push = false;  // the most recent push scheduled an indicator
  // foa_dmd_test_wait_fault: one-shot failure injection into the next cooperative SVD launch
  int test_skip_cta = -1;
  long long test_spin_cycles = 0;
};

namespace foa {
// An NVTX range names every streaming-pass launch (for tools: ncu --nvtx --nvtx-include "foa_dmd pass B/"
// selects the B passes); while profiling is enabled, a CUDA event pair also brackets the launch.
struct ProfScope {
  foa_dmd *h;
  int kind;
  double bytes;
  size_t idx;
  ProfScope(foa_dmd *h_, int kind_, double bytes_) : h(h_), kind(kind_), bytes(bytes_), idx(size_t(-1)) {
    static const char *kNames[4] = {"foa_dmd pass A", "foa_dmd pass B", "foa_dmd pass C", "foa_dmd column write"};
    nvtxRangePushA(kNames[kind & 3]);
    if (!h->prof) return;
    if (h->prof_used == h->events.size()) {
      EventPair p;
      cudaEventCreate(&p.start);
      cudaEventCreate(&p.stop);
      h->events.push_back(p);
    }
    idx = h->prof_used++;
    h->events[idx].kind = kind;
    h->events[idx].bytes = bytes;
    cudaEventRecord(h->events[idx].start, h->stream);
  }
  ~ProfScope() {
    if (idx != size_t(-1)) cudaEventRecord(h->events[idx].stop, h->stream);
    nvtxRangePop();
  }
};

int cuda_status(cudaError_t e);
int sync_state(foa_dmd *h, foa_dmd_push_info *info);
int check_device(int *sms);
double default_tol(int dtype);
int max_kmax_for(int dtype);
bool make_pass_geom(const Geometry &g, int dtype, int mode, int jcap, int64_t n, int ntiles, int sms, PassArgs &a,
                    int &grid);
int launch_pass_h(foa_dmd *h, int mode, int jcap, const void *x, const double *coef, bool batch,
                  foa_dmd_push_info *info_out);
int enqueue_push(foa_dmd *h, const void *x, bool batch, foa_dmd_push_info *info_out);
int flush_pending(foa_dmd *h);
// geometry of a pass launch: the tuned choice for (kind, j bucket) if any, else the handle default
const Geometry &geom_for(const foa_dmd *h, int mode, int jcap);
int tune_bucket(int j);
// eigen path (eig.cu)
void eig_free(foa_dmd *h);
int maybe_indicator(foa_dmd *h);  // the indicator schedule of foa_dmd_opts.indicator_every
double latest_indicator(foa_dmd *h, bool only_if_pending);
constexpr int kIndRing = 1024;
}  // namespace foa
