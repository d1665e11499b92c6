// DMD modes on the 5th-generation tensor cores: Phi = V Y (Alg. 1, Phi_i = V U_r z_i)
// for FP32 storage, with tcgen05.mma kind::tf32, accumulators in TMEM and a three-term split
// for FP32-level accuracy:  V Y ~= V_hi Y_hi + V_hi Y_lo + V_lo Y_hi, where x_hi keeps the
// 19 leading bits of x (a TF32 value) and x_lo = x - x_hi.
//
// A CTA owns blocks of 256 rows (8 tiles of the row-tiled V) and runs a K loop over chunks of 16
// basis columns.  Warp roles:
//   warp 8      producer: per chunk, bulk-copies the 8 tiles' 32 x 16 column slices of V and the
//               chunk of the pre-split Y operand into a stage of the shared-memory ring;
//   warps 0-3   converters: read the staged V slice and write V_hi / V_lo in the K-major
//               core-matrix layout the MMA descriptors expect (8 rows x 16 bytes per core matrix);
//   warp 9      MMA issuer (one thread) and TMEM owner: per chunk and per 128-row half, 2 K-steps
//               x 3 products into the accumulator; tcgen05.commit releases the stage;
//   warps 4-7   epilogue: tcgen05.ld of the 2 x (128 x 64) FP32 accumulators, coalesced stores.
// Two accumulator sets (2 x 128 TMEM columns) let the epilogue of one row block overlap the MMAs
// of the next.  Every mbarrier wait is bounded; on a timeout the kernel records
// FOA_DMD_ETIMEOUT and the CTA frees its TMEM before returning.
#include "api_internal.cuh"
#include "eig_internal.cuh"

namespace foa {
namespace tc {

constexpr int KC = 16;            // basis columns per K chunk
constexpr int ROWS = 256;         // rows per block (two M = 128 MMAs)
constexpr int TILES = ROWS / kTile;
constexpr int NOUT = 64;          // MMA N (output columns, zero padded)
constexpr int NS = 3;             // pipeline stages
constexpr int RAW_BYTES = TILES * kTile * KC * 4;     // 16 KB
constexpr int B_BYTES = 2 * NOUT * KC * 4;            // hi + lo, 8 KB
constexpr int A_BYTES = 2 * 2 * 128 * KC * 4;         // 2 halves x hi/lo, 32 KB
constexpr int STAGE_BYTES = RAW_BYTES + B_BYTES + A_BYTES;
constexpr int THREADS = 320;
constexpr int TMEM_COLS = 256;

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// shared-memory matrix descriptor: no swizzle, K-major, core matrices of 8 rows x 16 bytes;
// lbo = byte step between core matrices along K, sbo = byte step between 8-row groups.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version for this architecture
  return d;                // base offset 0, swizzle none
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = 64, M = 128
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(NOUT >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct TcArgs {
  const float *V;
  int kmax;
  int64_t n;
  int ntiles;
  int m;
  const float *Bop;  // pre-split Y: [chunk][hi/lo][8 groups][4 kgroups][8 rows][4 elems]
  float *phi;
  int64_t ldp;
  int ncols;
  int *err;
};

__global__ void __launch_bounds__(THREADS, 1) modes_tc_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full[NS], conv[NS], freed[NS], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblocks = (a.ntiles + TILES - 1) / TILES;
  const int nk = (a.m + KC - 1) / KC;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&conv[i], 1);
      mbar_init(&freed[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 1);
    }
    abort_s = 0;
    mbar_fence_init();
  }
  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_s;
  auto stage_ptr = [&](int s) { return smem + size_t(s) * STAGE_BYTES; };
  auto fail = [&]() {
    abort_s = 1;
    atomicExch(a.err, FOA_DMD_ETIMEOUT);
  };

  if (warp == 8) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int it = 0;
      for (int rb = blockIdx.x; rb < nblocks && !abort_s; rb += gridDim.x) {
        const int t0 = rb * TILES;
        const int nt = min(TILES, a.ntiles - t0);
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % NS;
          if (it >= NS && !mbar_wait(&freed[s], ((it / NS) - 1) & 1)) {
            fail();
            break;
          }
          const int k0 = kc * KC;
          const int cols = min(KC, a.m - k0);
          const uint32_t tb = uint32_t(kTile) * cols * 4;
          unsigned char *st = stage_ptr(s);
          mbar_arrive_expect_tx(&full[s], uint32_t(nt) * tb + B_BYTES);
          for (int t = 0; t < nt; ++t)
            bulk_g2s(st + t * (kTile * KC * 4), a.V + (int64_t(t0 + t) * a.kmax + k0) * kTile, tb, &full[s]);
          bulk_g2s(st + RAW_BYTES, a.Bop + size_t(kc) * (B_BYTES / 4), B_BYTES, &full[s]);
        }
      }
    }
  } else if (warp < 4) {
    // ------------------------------------------------------------ converters (128 threads)
    const int ct = threadIdx.x;  // 0..127
    int it = 0;
    for (int rb = blockIdx.x; rb < nblocks; rb += gridDim.x) {
      const int nt = min(TILES, a.ntiles - rb * TILES);
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int s = it % NS;
        const int bad = mbar_wait(&full[s], (it / NS) & 1) ? 0 : 1;
        if (named_bar_or(1, 128, bad)) {
          if (ct == 0) fail();
          goto conv_done;
        }
        {
          const int cols = min(KC, a.m - kc * KC);
          const float *raw = reinterpret_cast<const float *>(stage_ptr(s));
          unsigned char *A = stage_ptr(s) + RAW_BYTES + B_BYTES;
          // 8 tiles x 4 column quads x 32 rows = 1024 items, 8 per thread
          for (int item = ct; item < TILES * 4 * kTile; item += 128) {
            const int r = item & 31;
            const int c4 = (item >> 5) & 3;
            const int t = item >> 7;
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c = c4 * 4 + e;
              v[e] = (t < nt && c < cols) ? raw[t * (kTile * KC) + c * kTile + r] : 0.f;
            }
            const int half = t >> 2;
            const int R = (t & 3) * kTile + r;  // row within the 128-row half
            const int off = ((R >> 3) * 4 + c4) * 128 + (R & 7) * 16;
            float4 hi, lo;
            hi.x = tf32_hi(v[0]); lo.x = v[0] - hi.x;
            hi.y = tf32_hi(v[1]); lo.y = v[1] - hi.y;
            hi.z = tf32_hi(v[2]); lo.z = v[2] - hi.z;
            hi.w = tf32_hi(v[3]); lo.w = v[3] - hi.w;
            unsigned char *base = A + half * (2 * 128 * KC * 4);
            *reinterpret_cast<float4 *>(base + off) = hi;
            *reinterpret_cast<float4 *>(base + 128 * KC * 4 + off) = lo;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          named_bar_sync(1, 128);
          if (ct == 0) mbar_arrive(&conv[s]);
        }
      }
    }
  conv_done:;
  } else if (warp == 9) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc();
      int it = 0, lb = 0;
      for (int rb = blockIdx.x; rb < nblocks && !abort_s; rb += gridDim.x, ++lb) {
        const int as = lb & 1;
        if (lb >= 2 && !mbar_wait(&acc_empty[as], ((lb >> 1) - 1) & 1)) {
          fail();
          break;
        }
        tc_fence_after();
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % NS;
          if (!mbar_wait(&conv[s], (it / NS) & 1)) {
            fail();
            break;
          }
          tc_fence_after();
          const uint32_t sb = smem_addr(stage_ptr(s));
          const uint32_t bhi = sb + RAW_BYTES, blo = bhi + NOUT * KC * 4;
          const uint32_t abase = sb + RAW_BYTES + B_BYTES;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const uint32_t ahi = abase + half * (2 * 128 * KC * 4), alo = ahi + 128 * KC * 4;
            const uint32_t d = tmem_base + uint32_t(as * 128 + half * NOUT);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
              const uint32_t ko = ks * 2 * 128;  // two core matrices along K per K-step of 8
              const uint64_t dah = make_desc(ahi + ko, 128, 512), dal = make_desc(alo + ko, 128, 512);
              const uint64_t dbh = make_desc(bhi + ko, 128, 512), dbl = make_desc(blo + ko, 128, 512);
              const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
              mma_tf32(d, dah, dbh, idesc, first);
              mma_tf32(d, dah, dbl, idesc, 1u);
              mma_tf32(d, dal, dbh, idesc, 1u);
            }
          }
          mma_commit(&freed[s]);
        }
        mma_commit(&acc_full[as]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 4-7)
    const int q = warp - 4;  // TMEM lane quarter
    int lb = 0;
    for (int rb = blockIdx.x; rb < nblocks; rb += gridDim.x, ++lb) {
      const int as = lb & 1;
      const int bad = mbar_wait(&acc_full[as], (lb >> 1) & 1) ? 0 : 1;
      if (named_bar_or(2, 128, bad)) {
        if (threadIdx.x == 128) fail();
        break;
      }
      tc_fence_after();
      for (int half = 0; half < 2; ++half) {
        const int64_t r = int64_t(rb) * ROWS + half * 128 + q * 32 + lane;
        const uint32_t taddr = tmem_base + (uint32_t(q * 32) << 16) + uint32_t(as * 128 + half * NOUT);
        float v[NOUT];
#pragma unroll
        for (int c = 0; c < NOUT; c += 16) tmem_ld16(taddr + c, v + c);
        tmem_wait_ld();
        if (r < a.n) {
#pragma unroll
          for (int c = 0; c < NOUT; ++c)
            if (c < a.ncols) a.phi[r + int64_t(c) * a.ldp] = v[c];
        }
      }
      tc_fence_before();
      named_bar_sync(2, 128);
      if (threadIdx.x == 128) mbar_arrive(&acc_empty[as]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 9) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// Y (m x ncols, FP64, ld) -> pre-split TF32 operand chunks in the K-major core-matrix layout.
__global__ void split_y_kernel(const double *Y, int ldy, int m, int ncols, float *Bop) {
  const int nk = (m + KC - 1) / KC;
  const int total = nk * NOUT * KC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int chunk = e / (NOUT * KC);
    const int w = e % (NOUT * KC);
    const int nrow = w / KC, kk = w % KC;
    const int k = chunk * KC + kk;
    const double y = (k < m && nrow < ncols) ? Y[k + int64_t(nrow) * ldy] : 0.0;
    const float hi = tf32_hi(float(y));
    const float lo = float(y - double(hi));
    const int off = ((nrow >> 3) * 4 + (kk >> 2)) * 32 + (nrow & 7) * 4 + (kk & 3);
    float *base = Bop + size_t(chunk) * (B_BYTES / 4);
    base[off] = hi;
    base[NOUT * KC + off] = lo;
  }
}

}  // namespace tc

int launch_modes_tc(foa_dmd *h, int m, const double *Y, int ldy, int ncols, float *phi, int64_t ld_phi, float *Bop,
                    int *err) {
  using namespace tc;
  if (ncols > NOUT) return FOA_DMD_EINVAL;
  const int nk = (m + KC - 1) / KC;
  split_y_kernel<<<(nk * NOUT * KC + 255) / 256, 256, 0, h->stream>>>(Y, ldy, m, ncols, Bop);
  const size_t smem = size_t(NS) * STAGE_BYTES;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(modes_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_status(e);
    configured = true;
  }
  const int nblocks = (h->ntiles + TILES - 1) / TILES;
  const int grid = nblocks < h->sms ? nblocks : h->sms;
  TcArgs a;
  a.V = static_cast<const float *>(h->V);
  a.kmax = h->kmax;
  a.n = h->n;
  a.ntiles = h->ntiles;
  a.m = m;
  a.Bop = Bop;
  a.phi = phi;
  a.ldp = ld_phi;
  a.ncols = ncols;
  a.err = err;
  modes_tc_kernel<<<grid, THREADS, smem, h->stream>>>(a);
  h->launches += 2;
  return cuda_status(cudaGetLastError());
}

size_t modes_tc_bop_bytes(int kmax) {
  const int nk = (kmax + tc::KC - 1) / tc::KC;
  return size_t(nk) * tc::B_BYTES;
}

}  // namespace foa
