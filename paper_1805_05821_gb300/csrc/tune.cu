// Autotuner of the streaming-pass launch geometry: foa_dmd_autotune.
//
// The knobs of one pass launch are the V bytes of a pipeline stage (tiles per stage), the V bytes
// a CTA keeps in flight (ring depth) and the CTAs per SM (one CTA with a deep ring, or two CTAs
// whose barrier phases overlap).  The best choice depends on the dtype, the pass kind and the
// basis size j: j fixes the tile width, so it decides how many tiles fit a stage and how the row
// sweep splits columns.  The tuner times every candidate on the handle's own buffers for each
// pass kind the handle's options use and each j bucket, keeps the fastest per (kind, bucket), and
// optionally appends the choices to a text cache keyed on (device arch, dtype, log2 n, kind,
// bucket) that later handles read instead of timing again.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.cuh"
#include "push_kernels.cuh"

namespace foa {

// Upper ends of the j buckets; bucket b holds kTuneEdges[b-1] < j <= kTuneEdges[b].
static const int kTuneEdges[kTuneBuckets] = {8, 16, 32, 64, 128, 192, 256, 320, 384, 448, 512};

int tune_bucket(int j) {
  for (int b = 0; b < kTuneBuckets; ++b)
    if (j <= kTuneEdges[b]) return b;
  return kTuneBuckets - 1;
}

int tune_kind(int mode) {
  switch (mode) {
    case PASS_A: return 0;
    case PASS_B: return 1;
    case PASS_C: return 2;
    case PASS_A2: return 3;
    case PASS_B2: return 4;
    default: return -1;
  }
}

const Geometry &geom_for(const foa_dmd *h, int mode, int jcap) {
  const int k = tune_kind(mode == PASS_FIN ? PASS_A2 : mode);
  if (k < 0) return h->geom;
  const int b = tune_bucket(jcap);
  return h->tuned_ok[k][b] ? h->tuned[k][b] : h->geom;
}

namespace {

// Device state for one timed launch: push in progress at basis size j (with a pending column for
// the lagged pass); unit scalars keep every value finite.
__global__ void tune_state_kernel(DevState *st, int j, int pending) {
  if (threadIdx.x != 0) return;
  st->q = j;
  st->j = j;
  st->active = 1;
  st->stopped = 0;
  st->status = -1;
  st->err = 0;
  st->halt = 0;
  st->inv_bjj = 1.0;
  st->bjj = 1.0;
  st->x_norm = 1.0;
  st->nu = 1.0;
  st->inv_nu = 1.0;
  st->pending = pending;
  st->pend_col = j - 1;
}

struct Candidate {
  int64_t stage, inflight;
  int ctas, variant;
};

const int kKindMode[kTuneKinds] = {PASS_A, PASS_B, PASS_C, PASS_A2, PASS_B2};

int arch_of() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return 0;
  return p.major * 10 + p.minor;
}

int log2_floor(int64_t n) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= n) ++l;
  return l;
}

// Cache lines: "foa_dmd_tune arch dtype log2n kind bucket stage inflight ctas variant ms"
void load_cache(foa_dmd *h, const char *path, int arch, int nb) {
  FILE *f = fopen(path, "r");
  if (!f) return;
  char tag[32];
  int a, dt, l2, kind, b, ctas, variant;
  long long stage, inflight;
  double ms;
  while (fscanf(f, "%31s %d %d %d %d %d %lld %lld %d %d %lf", tag, &a, &dt, &l2, &kind, &b, &stage, &inflight, &ctas,
                &variant, &ms) == 11) {
    if (strcmp(tag, "foa_dmd_tune") != 0 || a != arch || dt != h->dtype || l2 != nb) continue;
    if (kind < 0 || kind >= kTuneKinds || b < 0 || b >= kTuneBuckets) continue;
    if (stage < 4096 || stage > (1 << 20) || inflight < 4096 || inflight > (1 << 20) || ctas < 1 || ctas > 2) continue;
    Geometry g = h->geom;
    g.stage_bytes = stage;
    g.inflight_bytes = inflight;
    g.max_ctas_per_sm = ctas;
    g.variant = (variant == 1) ? 1 : 0;
    h->tuned[kind][b] = g;
    h->tuned_ok[kind][b] = true;
  }
  fclose(f);
}

}  // namespace
}  // namespace foa

using namespace foa;

extern "C" int foa_dmd_autotune(foa_dmd_t *h, const char *cache_path, int32_t flags) {
  if (!h) return FOA_DMD_EINVAL;
  int rc = sync_state(h, nullptr);
  if (rc) return rc;
  if (h->q_host != 0) return FOA_DMD_EINVAL;  // tuning overwrites the stream state
  const int arch = arch_of();
  const int nb = log2_floor(h->n);
  // passes this handle launches
  bool used[kTuneKinds] = {false, false, false, false, false};
  if (h->opts.reorth == 2) {
    used[3] = used[4] = true;
  } else {
    used[0] = used[2] = true;
    used[1] = h->opts.reorth != 0;
  }
  if (cache_path && !(flags & 1)) load_cache(h, cache_path, arch, nb);
  const int jmax = h->kmax - 1;
  int nbuckets = tune_bucket(jmax < 1 ? 1 : jmax) + 1;
  bool need = false;
  for (int k = 0; k < kTuneKinds; ++k)
    for (int b = 0; b < nbuckets; ++b)
      if (used[k] && (!h->tuned_ok[k][b] || (flags & 1))) need = true;
  if (!need) return FOA_DMD_OK;

  const int s = dtype_size(h->dtype), cs = compute_size(h->dtype);
  void *xt = nullptr;
  cudaError_t e = cudaMalloc(&xt, size_t(h->nrows) * s);
  if (e == cudaSuccess) e = cudaMemsetAsync(xt, 0, size_t(h->nrows) * s, h->stream);
  if (e != cudaSuccess) {
    if (xt) cudaFree(xt);
    return cuda_status(e);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<Candidate> cands;
  for (int64_t st : {16384, 32768, 65536})
    for (int64_t inf : {65536, 98304, 147456, 196608})
      for (int c : {1, 2})
        for (int v : {0, 1}) cands.push_back({st, inf, c, v});
  const int sms = h->sms - (h->opts.indicator_every > 0 ? 1 : 0);
  FILE *cache = (cache_path && *cache_path) ? fopen(cache_path, "a") : nullptr;
  for (int k = 0; k < kTuneKinds && rc == FOA_DMD_OK; ++k) {
    if (!used[k]) continue;
    const int mode = kKindMode[k];
    for (int b = 0; b < nbuckets && rc == FOA_DMD_OK; ++b) {
      if (h->tuned_ok[k][b] && !(flags & 1)) continue;
      int j = kTuneEdges[b] < jmax ? kTuneEdges[b] : jmax;
      if (j < 1) j = 1;
      // time on a prefix of V large enough to stream well past L2 (about 2 GB), at most all of it
      const int64_t tile_bytes = int64_t(kTile) * j * s;
      int64_t tiles = int64_t(2) << 30;
      tiles /= tile_bytes;
      if (tiles < int64_t(sms) * 16) tiles = int64_t(sms) * 16;
      if (tiles > h->ntiles) tiles = h->ntiles;
      const int64_t n_t = (tiles == h->ntiles) ? h->n : tiles * kTile;
      double best = 1e30;
      Geometry bestg = h->geom;
      std::vector<std::string> seen;
      for (const Candidate &c : cands) {
        Geometry g = h->geom;
        g.stage_bytes = c.stage;
        g.inflight_bytes = c.inflight;
        g.max_ctas_per_sm = c.ctas;
        g.variant = c.variant;
        // variant 1 (shared-memory stage instead of the register-held one) is an alternative for the
        // FP32/BF16 passes with column dots only; FP64 and pass C have a single form
        if (c.variant == 1 && (h->dtype == FOA_DMD_F64 || mode == PASS_C)) continue;
        PassArgs a;
        memset(&a, 0, sizeof(a));
        int grid = 0;
        if (!make_pass_geom(g, h->dtype, mode, j, n_t, int(tiles), sms, a, grid)) continue;
        char key[96];
        snprintf(key, sizeof(key), "%d/%d/%d/%d/%d", a.R, a.slots, grid, a.smem_total, c.variant);
        bool dup = false;
        for (auto &q : seen) dup = dup || q == key;
        if (dup) continue;  // same launch as an earlier candidate
        seen.push_back(key);
        a.V = h->V;
        a.x = xt;
        a.w = h->w;
        a.coef = h->pre;
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
        a.kmax = h->kmax;
        a.reorth = h->opts.reorth;
        a.x_aligned = 1;
        a.form = h->opts.form;
        a.tol = h->tol;
        const int nc = pass_nc_for(j);
        float times[3];
        int nt = 0;
        for (int rep = 0; rep < 4 && rc == FOA_DMD_OK; ++rep) {
          tune_state_kernel<<<1, 32, 0, h->stream>>>(h->st, j, mode == PASS_A2 ? 1 : 0);
          e = cudaEventRecord(e0, h->stream);
          if (e == cudaSuccess) e = launch_pass(h->dtype, mode, nc, a, grid, h->stream);
          if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) {
            rc = cuda_status(e);
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) times[nt++] = ms;  // the first launch warms up
        }
        if (rc) break;
        DevState st;
        e = cudaMemcpy(&st, h->st, sizeof(st), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess || st.err) {
          rc = e != cudaSuccess ? cuda_status(e) : st.err;
          break;
        }
        // median of three
        float lo = fminf(times[0], fminf(times[1], times[2])), hi = fmaxf(times[0], fmaxf(times[1], times[2]));
        const double med = double(times[0]) + times[1] + times[2] - lo - hi;
        if (med < best) {
          best = med;
          bestg = g;
        }
      }
      if (rc) break;
      h->tuned[k][b] = bestg;
      h->tuned_ok[k][b] = true;
      if (cache)
        fprintf(cache, "foa_dmd_tune %d %d %d %d %d %lld %lld %d %d %.6f\n", arch, h->dtype, nb, k, b,
                (long long)bestg.stage_bytes, (long long)bestg.inflight_bytes, bestg.max_ctas_per_sm, bestg.variant,
                best);
    }
  }
  if (cache) fclose(cache);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(xt);
  // back to an empty stream: state, coefficients, working vector and basis cleared
  const int K = h->kmax;
  e = cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->H, 0, size_t(K) * K * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->B, 0, size_t(K) * K * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->w, 0, size_t(h->nrows) * cs, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->V, 0, size_t(h->nrows) * K * s, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (rc == FOA_DMD_OK && e != cudaSuccess) rc = cuda_status(e);
  h->q_host = 0;
  h->stopped_host = false;
  h->launches = 0;
  return rc;
}

extern "C" int foa_dmd_tuned_geometry(foa_dmd_t *h, int32_t kind, int32_t j, int64_t *stage_bytes,
                                      int64_t *inflight_bytes, int32_t *ctas_per_sm, int32_t *variant,
                                      int32_t *tuned) {
  if (!h || kind < 0 || kind >= kTuneKinds || j < 1) return FOA_DMD_EINVAL;
  const Geometry &g = geom_for(h, kKindMode[kind], j);
  if (stage_bytes) *stage_bytes = g.stage_bytes;
  if (inflight_bytes) *inflight_bytes = g.inflight_bytes;
  if (ctas_per_sm) *ctas_per_sm = g.max_ctas_per_sm;
  if (variant) *variant = g.variant;
  if (tuned) *tuned = h->tuned_ok[kind][tune_bucket(j)] ? 1 : 0;
  return FOA_DMD_OK;
}
