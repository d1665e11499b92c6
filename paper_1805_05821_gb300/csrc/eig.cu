// Device eigen path of FOA-based DMD (the eigen extraction of Alg. 1 and Alg. 3), all in FP64:
//
//   svd_jacobi_kernel  one-sided (Hestenes) Jacobi SVD of the upper-triangular beta_m, run by a
//                      cooperative grid: each round of the round-robin ordering rotates m/2
//                      independent column pairs, one pair per CTA of four warps; beta_m W =
//                      U Sigma gives U and Sigma without forming W (Sec. 3.2.2 rank truncation).
//   project_t/g_kernel G = U_r^T H_m U_r (copy_h_kernel: G = H_m without truncation).
//   hessenberg_kernel  Householder reduction of G to upper Hessenberg form G = Q Hs Q^T.
//   hqr_kernel         eigenvalues of Hs by the Francis double-shift QR iteration (single CTA;
//                      the sequential steps of the EISPACK routine hqr).
//   vectors_kernel     per eigenvalue: right and left eigenvectors of Hs by inverse iteration
//                      (LU of Hs - lambda I with adjacent-row pivoting), z = Q z_hs normalised
//                      (unit norm, largest entry real positive), the amplitude
//                      c = (w^H b)/(w^H z) with b = beta_11 U_r^T e_1 (Sec. 3.2.4, Eqs.
//                      exrecon/exreconwrt), the error indicator of Sec. 3.2.3 and y = U_r z.
//   order_kernel       ordering by |c| (conjugate pairs share the larger |c|), |lambda|, Im.
//
// The modes Phi = V y_i are formed by the GEMM in modes.cu.
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.cuh"
#include "eig_internal.cuh"

namespace foa {

// ------------------------------------------------------------------------------ grid barrier
// Only used in cooperative launches (all CTAs co-resident).  Bounded spin: a CTA that has waited
// spin_limit clock cycles for the others records FOA_DMD_ETIMEOUT and returns false, and its
// caller returns at once, so a CTA that never arrives ends the whole grid within the limit.
__device__ bool grid_barrier(GridBar *gb, int *err, long long spin_limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned *vgen = &gb->gen;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&gb->count, 1u);
    if (arrived == gridDim.x - 1) {
      gb->count = 0u;
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > spin_limit) {
          ok = 0;
          atomicExch(err, FOA_DMD_ETIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Bounded wait of CTA p for its neighbours p-1 and p+1 (those that exist among np CTAs) to have
// finished `target` rounds of the Jacobi sweep; the columns they rotated are then visible.
__device__ bool wait_neighbours(GridBar *gb, int p, int np, unsigned target, int *err, long long spin_limit) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    const long long t0 = clock64();
    volatile unsigned *rd = gb->round;
    for (int q = p - 1; q <= p + 1 && ok; q += 2) {
      if (q < 0 || q >= np) continue;
      while (rd[q] < target) {
        if (clock64() - t0 > spin_limit) {
          ok = 0;
          atomicExch(err, FOA_DMD_ETIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  __syncthreads();
  return t;
}

__device__ __forceinline__ int block_max_int(int v, int *red) {
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  int t = red[0];
  const int nw = blockDim.x >> 5;
  for (int i = 1; i < nw; ++i) t = max(t, red[i]);
  __syncthreads();
  return t;
}

// ------------------------------------------------------------------------------ SVD
// One-sided Jacobi on the columns of A = beta_m (m x m, ld).  Rotating columns i, j with
// alpha = |a_i|^2, beta = |a_j|^2, gamma = a_i.a_j:  zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t,
// a_i <- c a_i - s a_j,  a_j <- s a_i + c a_j.  Converged when no pair has
// |gamma| > tol sqrt(alpha beta).  Afterwards sigma_i = |a_i| and u_i = a_i / sigma_i.
//
// A CTA of four warps (one per SM sub-partition, so the pair's FP64 work uses all four FP64
// pipes of the SM) takes one column pair at a time: each thread holds up to kSvdRows rows of both
// columns in registers, the three dot products are summed in a fixed order (warp trees, then the
// four warps), thread 0 forms the rotation, and every thread rotates its rows.  The grid has one
// CTA per pair of the round-robin ordering ((m+1)/2 <= 256 CTAs).  In that ordering the two
// columns pair p takes in round r+1 were held in round r by pairs p-1 and p+1 (checked for every
// m <= 512), so between rounds a CTA waits only for its two neighbours' round counters, not for
// the whole grid; one grid barrier per sweep sums the rotation counts for the convergence test.
// Columns are read through L2 (__ldcg): a column that comes back to an SM it visited before must
// not be served from that SM's L1.
//
// skip_cta (normally -1) and spin_limit serve foa_dmd_test_wait_fault: CTA skip_cta returns before
// its first grid-barrier arrival, as a CTA that died would, and the others give up after
// spin_limit cycles.
__global__ void __launch_bounds__(kSvdThreads) svd_jacobi_kernel(const double *B, int ldb, int m, double *A, int lda,
                                                                 double *sig, int *isc, GridBar *gb, int max_sweeps,
                                                                 double tol, long long spin_limit, int skip_cta) {
  int *err = isc + ISC_ERR;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t gtid = int64_t(blockIdx.x) * blockDim.x + tid;
  const int64_t gthreads = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = gtid; e < int64_t(m) * m; e += gthreads) {
    const int r = int(e % m), c = int(e / m);
    A[r + int64_t(c) * lda] = (r <= c) ? B[r + int64_t(c) * ldb] : 0.0;
  }
  if (gtid == 0) isc[ISC_ROT] = 0;
  if (int(blockIdx.x) == skip_cta) return;  // failure injection only (uniform over the CTA)
  if (!grid_barrier(gb, err, spin_limit)) return;
  __shared__ double red[kSvdThreads / 32][3];
  __shared__ double rcs[2];
  __shared__ int rgo, nrot;
  const int mp = m + (m & 1);  // players of the round-robin schedule (m may be odd: one dummy)
  const int npairs = mp / 2;
  const double tol2 = tol * tol;
  const bool nbr = int(gridDim.x) == npairs;  // one pair per CTA: neighbour waits between rounds
  if (max_sweeps > kMaxSweeps) max_sweeps = kMaxSweeps;
  unsigned gr = 0;  // rounds finished by this CTA
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int myrot = 0;  // rotations applied by this CTA in the sweep (thread 0)
    for (int rnd = 0; rnd < mp - 1; ++rnd) {
      if (nbr && gr > 0 && !wait_neighbours(gb, blockIdx.x, npairs, gr, err, spin_limit)) return;
      for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
        const int pa = p, pb = mp - 1 - p;
        const int i = pa == 0 ? 0 : 1 + (pa - 1 + rnd) % (mp - 1);
        const int j = pb == 0 ? 0 : 1 + (pb - 1 + rnd) % (mp - 1);
        if (i >= m || j >= m) continue;  // uniform over the CTA
        double *ai = A + int64_t(i) * lda, *aj = A + int64_t(j) * lda;
        double x[kSvdRows], y[kSvdRows];
        double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
        for (int u = 0; u < kSvdRows; ++u) {
          const int k = tid + u * kSvdThreads;
          x[u] = k < m ? __ldcg(ai + k) : 0.0;
          y[u] = k < m ? __ldcg(aj + k) : 0.0;
          al = fma(x[u], x[u], al);
          be = fma(y[u], y[u], be);
          ga = fma(x[u], y[u], ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (lane == 0) {
          red[warp][0] = al;
          red[warp][1] = be;
          red[warp][2] = ga;
        }
        __syncthreads();
        if (tid == 0) {
          double sa = 0.0, sb = 0.0, sg = 0.0;
          for (int w = 0; w < kSvdThreads / 32; ++w) {
            sa += red[w][0];
            sb += red[w][1];
            sg += red[w][2];
          }
          const int go = (sg != 0.0) && (sg * sg > tol2 * (sa * sb));
          if (go) {
            const double zeta = (sb - sa) / (2.0 * sg);
            const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
            const double c = rsqrt(fma(t, t, 1.0));
            rcs[0] = c;
            rcs[1] = c * t;
            ++myrot;
          }
          rgo = go;
        }
        __syncthreads();
        if (rgo) {
          const double c = rcs[0], sn = rcs[1];
#pragma unroll
          for (int u = 0; u < kSvdRows; ++u) {
            const int k = tid + u * kSvdThreads;
            if (k < m) {
              ai[k] = c * x[u] - sn * y[u];
              aj[k] = sn * x[u] + c * y[u];
            }
          }
        }
      }
      if (nbr) {
        __syncthreads();  // this CTA's rotated columns are written
        if (tid == 0) {
          __threadfence();
          atomicExch(&gb->round[blockIdx.x], gr + 1);
        }
      } else if (!grid_barrier(gb, err, spin_limit)) {
        return;
      }
      ++gr;
    }
    if (tid == 0 && myrot) atomicAdd(&gb->rot[sweep], unsigned(myrot));
    if (!grid_barrier(gb, err, spin_limit)) return;  // every CTA has finished the sweep and added its count
    if (tid == 0) nrot = int(*(volatile unsigned *)&gb->rot[sweep]);
    __syncthreads();
    if (nrot == 0) break;
  }
  if (gtid == 0) isc[ISC_SWEEPS] = sweep;
  // column norms (one warp per column)
  const int warp_g = int(gtid >> 5), nwarps = int(gthreads >> 5);
  for (int c = warp_g; c < m; c += nwarps) {
    const double *ac = A + int64_t(c) * lda;
    double sq = 0.0;
    for (int k = lane; k < m; k += 32) {
      const double v = __ldcg(ac + k);
      sq += v * v;
    }
    sq = warp_sum(sq);
    if (lane == 0) sig[c] = sqrt(sq);
  }
}

// Sort singular values descending (stable by index), form U = A Sigma^{-1} in that order, and
// count the retained rank r = #{sigma_i > tol sigma_1} (at least 1).  Single CTA.
__global__ void svd_finish_kernel(const double *A, int lda, int m, const double *sig_in, double *U, double *sig,
                                  int *isc, double rank_tol) {
  extern __shared__ double sh[];
  double *s = sh;                               // m
  int *pos = reinterpret_cast<int *>(sh + m);   // m
  for (int i = threadIdx.x; i < m; i += blockDim.x) s[i] = sig_in[i];
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    int rank = 0;
    for (int k = 0; k < m; ++k) rank += (s[k] > s[i]) || (s[k] == s[i] && k < i);
    pos[i] = rank;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) sig[pos[i]] = s[i];
  __syncthreads();
  for (int64_t e = threadIdx.x; e < int64_t(m) * m; e += blockDim.x) {
    const int r = int(e % m), c = int(e / m);
    const double sc = s[c] > 0.0 ? 1.0 / s[c] : 0.0;
    U[r + int64_t(pos[c]) * lda] = A[r + int64_t(c) * lda] * sc;
  }
  if (threadIdx.x == 0) {
    double smax = 0.0;
    for (int k = 0; k < m; ++k) smax = fmax(smax, s[k]);
    int r = 0;
    for (int k = 0; k < m; ++k) r += s[k] > rank_tol * smax;
    isc[ISC_R] = r < 1 ? 1 : r;
  }
}

// ------------------------------------------------------------------------------ projection
// T = H_m U_r (m x r), then G = U_r^T T (r x r).  Without truncation G = H_m.
__global__ void project_t_kernel(const double *H, int ldh, int m, const double *U, int ldu, const int *isc,
                                 double *T, int ldt) {
  const int r = isc[ISC_R];
  const int64_t total = int64_t(m) * r;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(e % m), c = int(e / m);
    double s = 0.0;
    const int k0 = i > 0 ? i - 1 : 0;  // H_m is upper Hessenberg
    for (int k = k0; k < m; ++k) s += H[i + int64_t(k) * ldh] * U[k + int64_t(c) * ldu];
    T[i + int64_t(c) * ldt] = s;
  }
}
__global__ void project_g_kernel(const double *U, int ldu, int m, const int *isc, const double *T, int ldt, double *G,
                                 int ldg) {
  const int r = isc[ISC_R];
  const int64_t total = int64_t(r) * r;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(e % r), c = int(e / r);
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += U[k + int64_t(i) * ldu] * T[k + int64_t(c) * ldt];
    G[i + int64_t(c) * ldg] = s;
  }
}
// G = H_m (Hessenberg part), and the two entries of the stream's state the untruncated eigen path
// still needs (h_{m+1,m} for the indicators, beta_11 for the amplitudes), so that nothing after this
// kernel reads H-bar or beta.
__global__ void copy_h_kernel(const double *H, int ldh, int m, double *G, int ldg, int *isc, const double *B,
                              double *scal) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < int64_t(m) * m;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(e % m), c = int(e / m);
    G[i + int64_t(c) * ldg] = (i <= c + 1) ? H[i + int64_t(c) * ldh] : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    isc[ISC_R] = m;
    scal[0] = H[m + int64_t(m - 1) * ldh];
    scal[1] = B[0];
  }
}

// ------------------------------------------------------------------------------ Hessenberg
// Householder reduction G = Q Hs Q^T (single CTA).  Q accumulated explicitly.
__global__ void hessenberg_kernel(double *G, int ldg, double *Q, int ldq, const int *isc) {
  const int n = isc[ISC_R];
  extern __shared__ double sh[];
  double *v = sh;            // n
  double *red = sh + n;      // 32
  __shared__ double s_beta;
  for (int64_t e = threadIdx.x; e < int64_t(n) * n; e += blockDim.x) {
    const int i = int(e % n), c = int(e / n);
    Q[i + int64_t(c) * ldq] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    // reflector for G[k+1:n, k] (identity when the entries below G[k+1,k] are already zero)
    double ss = 0.0;
    for (int i = k + 2 + threadIdx.x; i < n; i += blockDim.x) {
      const double x = G[i + int64_t(k) * ldg];
      ss += x * x;
    }
    ss = block_sum(ss, red);
    if (ss == 0.0) continue;
    const double alpha = G[(k + 1) + int64_t(k) * ldg];
    const double nrm = sqrt(alpha * alpha + ss);
    const double beta = alpha >= 0.0 ? -nrm : nrm;  // new G[k+1,k]
    const double v0 = alpha - beta;
    // v = [1, x(k+2:)/v0], tau = (beta - alpha)/beta
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) v[i] = (i == k + 1) ? 1.0 : G[i + int64_t(k) * ldg] / v0;
    if (threadIdx.x == 0) s_beta = (beta - alpha) / beta;
    __syncthreads();
    const double tau = s_beta;
    // G <- (I - tau v v^T) G : columns k..n-1
    for (int c = k + threadIdx.x; c < n; c += blockDim.x) {
      double d = 0.0;
      for (int i = k + 1; i < n; ++i) d += v[i] * G[i + int64_t(c) * ldg];
      d *= tau;
      for (int i = k + 1; i < n; ++i) G[i + int64_t(c) * ldg] -= d * v[i];
    }
    __syncthreads();
    // G <- G (I - tau v v^T) : all rows;  Q <- Q (I - tau v v^T)
    for (int row = threadIdx.x; row < 2 * n; row += blockDim.x) {
      double *M = row < n ? G : Q;
      const int ldm = row < n ? ldg : ldq;
      const int i = row < n ? row : row - n;
      double d = 0.0;
      for (int c = k + 1; c < n; ++c) d += M[i + int64_t(c) * ldm] * v[c];
      d *= tau;
      for (int c = k + 1; c < n; ++c) M[i + int64_t(c) * ldm] -= d * v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      G[(k + 1) + int64_t(k) * ldg] = beta;
      for (int i = k + 2; i < n; ++i) G[i + int64_t(k) * ldg] = 0.0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ QR iteration
// Eigenvalues of the upper Hessenberg Hs (n x n) by the Francis double-shift QR iteration with
// deflation.  The sequential core follows the published routine hqr of Martin, Peters and
// Wilkinson ("The QR algorithm for real Hessenberg matrices", Numer. Math. 14 (1970) 219-231;
// Handbook for Automatic Computation vol. II, contribution II/14; EISPACK hqr): the negligible-
// subdiagonal search, the exceptional shifts after 10 and 20 iterations without deflation
// (0.75 s and -0.4375 s^2), the search for two small consecutive subdiagonals and the bulge-
// chasing sweep with its p, q, r, x, y, z, w quantities (Golub & Van Loan, Sec. 7.5, give the
// same method).  Works in place on a copy A.  A conjugate pair is stored +Im first.
//
// Layout: the band |j - i| <= 3 (every entry the bulge chase reads, 7 n doubles) lives in shared
// memory; the rest of A in shared memory when n^2 fits the smem_elems doubles offered, else in
// global memory.  Sweep step k applies reflector k to rows k..k+2 (columns k..nn) and then to
// columns k..k+2 (rows l..k+3).  Warp 0 takes the corner, rows/columns k..k+3 (all band
// entries): lanes 0-3 the row update of columns k..k+3, then the column update of rows k..k+3,
// and lane 0 forms reflector k+1 from column k; the other warps apply reflector k to rows k..k+2
// of columns k+4..nn and to columns k..k+2 of rows l..k-1, a fixed thread per column and per
// row.  Those entries are never read by the chase within the sweep, so one CTA barrier per step
// suffices, and every entry receives the same updates in the same order as the sequential sweep.
__global__ void hqr_kernel(double *Ag, int lda, const int *isc_in, double *wr, double *wi, int *isc,
                           int smem_elems) {
  const int n = isc_in[ISC_R];
  extern __shared__ double sh[];
  const int tid = threadIdx.x, lane = tid & 31;
  const int T1 = blockDim.x - 32;  // threads outside warp 0
  double *a = Ag;
  int ld = lda;
  double *band = sh + smem_elems;  // entry (i, j), |j - i| <= 3, at band[7 i + j - i + 3]
  if (int64_t(n) * n <= int64_t(smem_elems)) {
    a = sh;
    ld = n;
    for (int64_t e = tid; e < int64_t(n) * n; e += blockDim.x) {
      const int i = int(e % n), c = int(e / n);
      a[i + int64_t(c) * n] = Ag[i + int64_t(c) * lda];
    }
  }
  for (int e = tid; e < 7 * n; e += blockDim.x) {
    const int i = e / 7, j = i + e % 7 - 3;
    band[e] = (j >= 0 && j < n) ? Ag[i + int64_t(j) * lda] : 0.0;
  }
#define AA(i, j) (*((((j) - (i)) <= 3 && ((i) - (j)) <= 3) ? &band[7 * (i) + (j) - (i) + 3] : &a[(i) + int64_t(j) * ld]))
  __shared__ double red[32];
  __shared__ int ired[32];
  __shared__ double sp, sq, sx, st_, sw, sanorm;
  __shared__ int snn, sits, sskip, sfail;
  __shared__ double rfl[2][5];  // reflector of step k in slot k & 1: x, y, z, q, r
  __shared__ int rskip[2];
  __syncthreads();
  double an = 0.0;
  for (int64_t e = tid; e < int64_t(n) * n; e += blockDim.x) {
    const int i = int(e % n), c = int(e / n);
    if (i <= c + 1) an += fabs(AA(i, c));
  }
  an = block_sum(an, red);
  if (tid == 0) {
    sanorm = an;
    snn = n - 1;
    st_ = 0.0;
    sits = 0;
    sfail = 0;
  }
  __syncthreads();
  const double eps = 2.220446049250313e-16;
  // Reflector of step k from (p, q, r) (the first step m gets them already scaled); records it in
  // slot k & 1 and writes A(k, k-1).  Lane 0 of warp 0 only.  Past the first step (p, q, r) are
  // scaled by the power of two x nearest below max(|p|, |q|, |r|), which is exact: on GB300 a
  // dependent FP64 operation takes about 64 cycles and a division about 420, and the reflector is
  // the chase's critical path, so the division by |p| + |q| + |r| of the sequential routine is
  // replaced; the reflector (p/s, q/s, r/s, q/p, r/p) does not depend on the scale.
  auto reflector = [&](int k, int m, int l, double p, double q, double r, double x) {
    bool go = true;
    if (k != m) {
      const double mx = fmax(fabs(p), fmax(fabs(q), fabs(r)));
      const long long eb = (__double_as_longlong(mx) >> 52) & 0x7ff;  // biased exponent of mx
      if (mx != 0.0 && eb != 0 && eb < 2046) {
        x = __longlong_as_double(eb << 52);                        // 2^(e), e the exponent of mx
        const double ix = __longlong_as_double((2046 - eb) << 52);  // 2^(-e)
        p *= ix;
        q *= ix;
        r *= ix;
      } else if (mx != 0.0) {  // subnormal or near-overflow maximum: the division as in hqr
        x = fabs(p) + fabs(q) + fabs(r);
        const double ix = 1.0 / x;
        p *= ix;
        q *= ix;
        r *= ix;
      } else {
        go = false;
      }
    }
    double s = 0.0;
    if (go) {
      s = copysign(sqrt(p * p + q * q + r * r), p);
      if (s == 0.0) go = false;
    }
    const int b = k & 1;
    if (go) {
      if (k == m) {
        if (l != m) AA(k, k - 1) = -AA(k, k - 1);
      } else {
        AA(k, k - 1) = -s * x;
      }
      p += s;
      const double is = 1.0 / s, ip = 1.0 / p;
      rfl[b][0] = p * is;
      rfl[b][1] = q * is;
      rfl[b][2] = r * is;
      rfl[b][3] = q * ip;
      rfl[b][4] = r * ip;
      rskip[b] = 0;
    } else {
      rskip[b] = 1;
    }
  };
  while (true) {
    const int nn = snn;
    if (nn < 0 || sfail) break;
    // largest l in [1, nn] whose subdiagonal is negligible (0 if none)
    int cand = 0;
    for (int l = 1 + tid; l <= nn; l += blockDim.x) {
      double s = fabs(AA(l - 1, l - 1)) + fabs(AA(l, l));
      if (s == 0.0) s = sanorm;
      if (fabs(AA(l, l - 1)) <= eps * s) cand = max(cand, l);
    }
    const int l = block_max_int(cand, ired);
    if (tid == 0 && l > 0) AA(l, l - 1) = 0.0;
    __syncthreads();
    if (l == nn) {
      if (tid == 0) {
        wr[nn] = AA(nn, nn) + st_;
        wi[nn] = 0.0;
        snn = nn - 1;
        sits = 0;
      }
      __syncthreads();
      continue;
    }
    if (l == nn - 1) {
      if (tid == 0) {
        const double y = AA(nn - 1, nn - 1), x = AA(nn, nn) + st_;
        const double w = AA(nn, nn - 1) * AA(nn - 1, nn);
        const double p = 0.5 * (y - AA(nn, nn));
        const double q = p * p + w;
        double z = sqrt(fabs(q));
        if (q >= 0.0) {
          z = p + copysign(z, p);
          wr[nn - 1] = wr[nn] = x + z;
          if (z != 0.0) wr[nn] = x - w / z;
          wi[nn - 1] = wi[nn] = 0.0;
        } else {
          wr[nn - 1] = wr[nn] = x + p;
          wi[nn - 1] = z;
          wi[nn] = -z;
        }
        snn = nn - 2;
        sits = 0;
      }
      __syncthreads();
      continue;
    }
    if (sits >= 60) {
      if (tid == 0) sfail = 1;
      __syncthreads();
      break;
    }
    // shifts
    if (tid == 0) {
      double x = AA(nn, nn), y = AA(nn - 1, nn - 1), w = AA(nn, nn - 1) * AA(nn - 1, nn);
      if (sits == 10 || sits == 20) {
        st_ += x;
        sx = x;
        const double s = fabs(AA(nn, nn - 1)) + fabs(AA(nn - 1, nn - 2));
        x = y = 0.75 * s;
        w = -0.4375 * s * s;
        sskip = 1;  // diagonal shift pending
      } else {
        sskip = 0;
      }
      sp = x;  // keep x, y, w
      sq = y;
      sw = w;
      sits = sits + 1;
    }
    __syncthreads();
    if (sskip) {
      const double xs = sx;
      for (int i = tid; i <= nn; i += blockDim.x) AA(i, i) -= xs;
      __syncthreads();
    }
    const double X = sp, Y = sq, W = sw;
    // largest m in [l, nn-2] where two consecutive subdiagonals are small (or m = l)
    int mc = l;
    for (int m = l + 1 + tid; m <= nn - 2; m += blockDim.x) {
      const double z = AA(m, m);
      const double r = X - z, s = Y - z;
      double p = (r * s - W) / AA(m + 1, m) + AA(m, m + 1);
      double q = AA(m + 1, m + 1) - z - r - s;
      double rr = AA(m + 2, m + 1);
      const double sc = fabs(p) + fabs(q) + fabs(rr);
      p /= sc;
      q /= sc;
      rr /= sc;
      const double u = fabs(AA(m, m - 1)) * (fabs(q) + fabs(rr));
      const double v = fabs(p) * (fabs(AA(m - 1, m - 1)) + fabs(z) + fabs(AA(m + 1, m + 1)));
      if (u <= eps * v) mc = max(mc, m);
    }
    const int m = block_max_int(mc, ired);
    for (int i = m + 2 + tid; i <= nn; i += blockDim.x) {
      AA(i, i - 2) = 0.0;
      if (i != m + 2) AA(i, i - 3) = 0.0;
    }
    __syncthreads();
    if (tid == 0) {
      const double z = AA(m, m);
      const double r = X - z, s = Y - z;
      double p = (r * s - W) / AA(m + 1, m) + AA(m, m + 1);
      double q = AA(m + 1, m + 1) - z - r - s;
      double rr = AA(m + 2, m + 1);
      const double sc = fabs(p) + fabs(q) + fabs(rr);
      reflector(m, m, l, p / sc, q / sc, rr / sc, 0.0);
    }
    __syncthreads();
    // double-shift QR sweep on rows/columns l..nn, starting at m; one barrier per step
    for (int k = m; k <= nn - 1; ++k) {
      const int b = k & 1;
      const bool three = (k != nn - 1);
      const bool skip = rskip[b] != 0;
      const double x = rfl[b][0], y = rfl[b][1], z = rfl[b][2], q = rfl[b][3], r = rfl[b][4];
      if (tid < 32) {
        // ---- warp 0: the corner, then the next reflector
        double fw = 0.0;  // lane 1 + i: row k + 1 + i of column k after the step
        if (!skip) {
          const int jj = k + lane;
          if (lane < 4 && jj <= nn) {
            double p = AA(k, jj) + q * AA(k + 1, jj);
            if (three) {
              p += r * AA(k + 2, jj);
              AA(k + 2, jj) -= p * z;
            }
            AA(k + 1, jj) -= p * y;
            AA(k, jj) -= p * x;
          }
          __syncwarp();
          const int i = k + lane;
          if (lane < 4 && i <= nn && i <= k + 3) {
            double p = x * AA(i, k) + y * AA(i, k + 1);
            if (three) {
              p += z * AA(i, k + 2);
              AA(i, k + 2) -= p * r;
            }
            AA(i, k + 1) -= p * q;
            const double aik = AA(i, k) - p;
            AA(i, k) = aik;
            fw = aik;
          }
        } else {
          const int i = k + lane;
          if (lane >= 1 && lane < 4 && i <= nn) fw = AA(i, k);
        }
        const double f0 = __shfl_sync(0xffffffffu, fw, 1);
        const double f1 = __shfl_sync(0xffffffffu, fw, 2);
        const double f2 = __shfl_sync(0xffffffffu, fw, 3);
        if (lane == 0 && k + 1 <= nn - 1) reflector(k + 1, m, l, f0, f1, (k + 1 != nn - 1) ? f2 : 0.0, 0.0);
      } else if (!skip) {
        // ---- the other warps: columns k+4..nn (rows k..k+2) and rows l..k-1 (columns k..k+2),
        // at most two of each a thread (n <= 512 < 2 T1); every load issued before any update,
        // so the step waits for one memory round trip
        const int t1 = tid - 32;
        const int j0 = k + 4 + ((t1 - (k + 4)) % T1 + T1) % T1, j1 = j0 + T1;
        const int i0 = l + ((t1 - l) % T1 + T1) % T1, i1 = i0 + T1;
        const bool hj0 = j0 <= nn, hj1 = j1 <= nn, hi0 = i0 <= k - 1, hi1 = i1 <= k - 1;
        double c0[3] = {0.0, 0.0, 0.0}, c1[3] = {0.0, 0.0, 0.0}, r0[3] = {0.0, 0.0, 0.0}, r1[3] = {0.0, 0.0, 0.0};
        if (hj0) {
          c0[0] = AA(k, j0), c0[1] = AA(k + 1, j0);
          if (three) c0[2] = AA(k + 2, j0);
        }
        if (hj1) {
          c1[0] = AA(k, j1), c1[1] = AA(k + 1, j1);
          if (three) c1[2] = AA(k + 2, j1);
        }
        if (hi0) {
          r0[0] = AA(i0, k), r0[1] = AA(i0, k + 1);
          if (three) r0[2] = AA(i0, k + 2);
        }
        if (hi1) {
          r1[0] = AA(i1, k), r1[1] = AA(i1, k + 1);
          if (three) r1[2] = AA(i1, k + 2);
        }
        auto rowupd = [&](double (&v)[3], int jj) {
          double p = v[0] + q * v[1];
          if (three) {
            p += r * v[2];
            AA(k + 2, jj) = v[2] - p * z;
          }
          AA(k + 1, jj) = v[1] - p * y;
          AA(k, jj) = v[0] - p * x;
        };
        auto colupd = [&](double (&v)[3], int i) {
          double p = x * v[0] + y * v[1];
          if (three) {
            p += z * v[2];
            AA(i, k + 2) = v[2] - p * r;
          }
          AA(i, k + 1) = v[1] - p * q;
          AA(i, k) = v[0] - p;
        };
        if (hj0) rowupd(c0, j0);
        if (hj1) rowupd(c1, j1);
        if (hi0) colupd(r0, i0);
        if (hi1) colupd(r1, i1);
      }
      __syncthreads();
    }
  }
  if (tid == 0) isc[ISC_STATUS] = sfail ? FOA_DMD_ENOCONV : FOA_DMD_OK;
#undef AA
}

// ------------------------------------------------------------------------------ vectors
struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cconj(cplx a) { return {a.re, -a.im}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
  }
  const double r = b.re / b.im, d = b.re * r + b.im;
  return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}

// One CTA per eigenvalue with Im >= 0 (the -Im partner of a pair is its conjugate).
__global__ void vectors_kernel(EigArgs e) {
  const int r = e.isc[ISC_R];
  const int m = e.m;
  const double hlast = *e.hlast_p, b11 = *e.b11_p;
  extern __shared__ double sh[];
  double *cr = sh, *ci = sh + r;                 // current LU row / work vector
  double *br = sh + 2 * r, *bi = sh + 3 * r;     // right-hand side / solution
  double *lr = sh + 4 * r, *li = sh + 5 * r;     // multipliers
  int *swp = reinterpret_cast<int *>(sh + 6 * r);  // pivot swaps
  double *red = sh + 6 * r + (r + 1) / 2 + 1;      // 32 doubles
  double *zr_s = red + 32, *zi_s = zr_s + r;       // eigenvector z (r)
  double *wr_s = zi_s + r, *wi_s = wr_s + r;       // left eigenvector w (r)
  __shared__ cplx s_piv, s_l;
  __shared__ int s_swap;
  double *Ur = e.lu + size_t(blockIdx.x) * 2 * size_t(r) * r;  // U of the LU (r x r complex, col-major)
  double *Ui = Ur + size_t(r) * r;
  const double *Hs = e.Hs;
  const int ldh = e.ld;
  const double anorm = e.anorm[0];
  const double tiny = 2.220446049250313e-16 * (anorm > 0.0 ? anorm : 1.0);
  for (int idx = blockIdx.x; idx < r; idx += gridDim.x) {
    const double lre = e.wr[idx], lim = e.wi[idx];
    if (lim < 0.0) continue;  // filled by the +Im partner
    const cplx lam = {lre, lim};
    // ---- LU of A = Hs - lam I with adjacent-row pivoting
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
      cr[c] = Hs[0 + int64_t(c) * ldh] - (c == 0 ? lam.re : 0.0);
      ci[c] = (c == 0 ? -lam.im : 0.0);
    }
    __syncthreads();
    for (int k = 0; k < r - 1; ++k) {
      if (threadIdx.x == 0) {
        const cplx cur = {cr[k], ci[k]};
        const cplx nxt = {Hs[(k + 1) + int64_t(k) * ldh], 0.0};
        const bool sw = cabs2(nxt) > cabs2(cur);
        cplx piv = sw ? nxt : cur, oth = sw ? cur : nxt;
        if (piv.re == 0.0 && piv.im == 0.0) piv.re = tiny;
        s_swap = sw ? 1 : 0;
        s_piv = piv;
        s_l = cdiv(oth, piv);
        swp[k] = s_swap;
        lr[k] = s_l.re;
        li[k] = s_l.im;
      }
      __syncthreads();
      const int sw = s_swap;
      const cplx l = s_l;
      for (int c = k + threadIdx.x; c < r; c += blockDim.x) {
        const cplx cur = {cr[c], ci[c]};
        const cplx nxt = {Hs[(k + 1) + int64_t(c) * ldh] - (c == k + 1 ? lam.re : 0.0), (c == k + 1 ? -lam.im : 0.0)};
        cplx piv = sw ? nxt : cur;
        const cplx oth = sw ? cur : nxt;
        if (c == k) piv = s_piv;
        Ur[k + int64_t(c) * r] = piv.re;
        Ui[k + int64_t(c) * r] = piv.im;
        if (c > k) {
          const cplx nw = csub(oth, cmul(l, piv));
          cr[c] = nw.re;
          ci[c] = nw.im;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      cplx last = {cr[r - 1], ci[r - 1]};
      if (last.re == 0.0 && last.im == 0.0) last.re = tiny;
      Ur[(r - 1) + int64_t(r - 1) * r] = last.re;
      Ui[(r - 1) + int64_t(r - 1) * r] = last.im;
    }
    __syncthreads();
    // ---- two inverse-iteration solves each for A z = b (right) and A^H w = b (left)
    for (int side = 0; side < 2; ++side) {
      for (int c = threadIdx.x; c < r; c += blockDim.x) {
        br[c] = 1.0;
        bi[c] = 0.0;
      }
      __syncthreads();
      for (int itn = 0; itn < 2; ++itn) {
        if (side == 0) {
          // forward elimination on b
          if (threadIdx.x == 0) {
            for (int k = 0; k < r - 1; ++k) {
              if (swp[k]) {
                double t = br[k]; br[k] = br[k + 1]; br[k + 1] = t;
                t = bi[k]; bi[k] = bi[k + 1]; bi[k + 1] = t;
              }
              const cplx l = {lr[k], li[k]};
              const cplx nb = csub({br[k + 1], bi[k + 1]}, cmul(l, {br[k], bi[k]}));
              br[k + 1] = nb.re;
              bi[k + 1] = nb.im;
            }
          }
          __syncthreads();
          // back substitution U z = b, column oriented
          for (int i = r - 1; i >= 0; --i) {
            if (threadIdx.x == 0) {
              const cplx zi_ = cdiv({br[i], bi[i]}, {Ur[i + int64_t(i) * r], Ui[i + int64_t(i) * r]});
              br[i] = zi_.re;
              bi[i] = zi_.im;
            }
            __syncthreads();
            const cplx zv = {br[i], bi[i]};
            for (int k = threadIdx.x; k < i; k += blockDim.x) {
              const cplx u = {Ur[k + int64_t(i) * r], Ui[k + int64_t(i) * r]};
              const cplx nb = csub({br[k], bi[k]}, cmul(u, zv));
              br[k] = nb.re;
              bi[k] = nb.im;
            }
            __syncthreads();
          }
        } else {
          // U^H y = b (forward), then apply E_k^H in reverse
          for (int i = 0; i < r; ++i) {
            if (threadIdx.x == 0) {
              const cplx yv = cdiv({br[i], bi[i]}, cconj({Ur[i + int64_t(i) * r], Ui[i + int64_t(i) * r]}));
              br[i] = yv.re;
              bi[i] = yv.im;
            }
            __syncthreads();
            const cplx yv = {br[i], bi[i]};
            for (int k = i + 1 + threadIdx.x; k < r; k += blockDim.x) {
              const cplx u = cconj({Ur[i + int64_t(k) * r], Ui[i + int64_t(k) * r]});
              const cplx nb = csub({br[k], bi[k]}, cmul(u, yv));
              br[k] = nb.re;
              bi[k] = nb.im;
            }
            __syncthreads();
          }
          if (threadIdx.x == 0) {
            for (int k = r - 2; k >= 0; --k) {
              const cplx l = cconj({lr[k], li[k]});
              const cplx nb = csub({br[k], bi[k]}, cmul(l, {br[k + 1], bi[k + 1]}));
              br[k] = nb.re;
              bi[k] = nb.im;
              if (swp[k]) {
                double t = br[k]; br[k] = br[k + 1]; br[k + 1] = t;
                t = bi[k]; bi[k] = bi[k + 1]; bi[k + 1] = t;
              }
            }
          }
          __syncthreads();
        }
        // normalise
        double s2 = 0.0;
        for (int c = threadIdx.x; c < r; c += blockDim.x) s2 += br[c] * br[c] + bi[c] * bi[c];
        s2 = block_sum(s2, red);
        const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 1.0;
        for (int c = threadIdx.x; c < r; c += blockDim.x) {
          br[c] *= inv;
          bi[c] *= inv;
        }
        __syncthreads();
      }
      // map back to the coordinates of G: v = Q v_hs
      double *dr = side == 0 ? zr_s : wr_s, *di = side == 0 ? zi_s : wi_s;
      for (int i = threadIdx.x; i < r; i += blockDim.x) {
        if (e.have_q) {
          double sr = 0.0, si = 0.0;
          for (int k = 0; k < r; ++k) {
            const double q = e.Q[i + int64_t(k) * e.ld];
            sr += q * br[k];
            si += q * bi[k];
          }
          dr[i] = sr;
          di[i] = si;
        } else {
          dr[i] = br[i];
          di[i] = bi[i];
        }
      }
      __syncthreads();
    }
    // ---- normalise z: unit norm, largest-magnitude entry real positive (lowest index on ties)
    double s2 = 0.0;
    for (int c = threadIdx.x; c < r; c += blockDim.x) s2 += zr_s[c] * zr_s[c] + zi_s[c] * zi_s[c];
    s2 = block_sum(s2, red);
    __shared__ int s_arg;
    if (threadIdx.x == 0) {
      double best = -1.0;
      int arg = 0;
      for (int c = 0; c < r; ++c) {
        const double a2 = zr_s[c] * zr_s[c] + zi_s[c] * zi_s[c];
        if (a2 > best * (1.0 + 1e-12)) {
          best = a2;
          arg = c;
        }
      }
      s_arg = arg;
    }
    __syncthreads();
    {
      const cplx zk = {zr_s[s_arg], zi_s[s_arg]};
      const double az = sqrt(cabs2(zk));
      const double nrm = sqrt(s2);
      const cplx ph = {zk.re / (az * nrm), -zk.im / (az * nrm)};  // conj(zk)/|zk| / |z|
      __syncthreads();
      for (int c = threadIdx.x; c < r; c += blockDim.x) {
        const cplx v = cmul({zr_s[c], zi_s[c]}, ph);
        zr_s[c] = v.re;
        zi_s[c] = v.im;
      }
      __syncthreads();
    }
    // ---- amplitude c = (w^H b) / (w^H z), b = beta_11 U_r^T e_1
    double n1r = 0.0, n1i = 0.0, d1r = 0.0, d1i = 0.0;
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
      const double bc = b11 * (e.have_u ? e.U[0 + int64_t(c) * e.ld] : (c == 0 ? 1.0 : 0.0));
      // conj(w) * b
      n1r += wr_s[c] * bc;
      n1i += -wi_s[c] * bc;
      // conj(w) * z
      d1r += wr_s[c] * zr_s[c] + wi_s[c] * zi_s[c];
      d1i += wr_s[c] * zi_s[c] - wi_s[c] * zr_s[c];
    }
    n1r = block_sum(n1r, red);
    n1i = block_sum(n1i, red);
    d1r = block_sum(d1r, red);
    d1i = block_sum(d1i, red);
    const cplx amp = cdiv({n1r, n1i}, {d1r, d1i});
    // ---- y = U_r z (m entries) into the output column idx
    double *yr = e.yr + int64_t(idx) * e.ld, *yi = e.yi + int64_t(idx) * e.ld;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      if (e.have_u) {
        double sr = 0.0, si = 0.0;
        for (int k = 0; k < r; ++k) {
          const double u = e.U[i + int64_t(k) * e.ld];
          sr += u * zr_s[k];
          si += u * zi_s[k];
        }
        yr[i] = sr;
        yi[i] = si;
      } else {
        yr[i] = zr_s[i];
        yi[i] = zi_s[i];
      }
    }
    __syncthreads();
    // ---- error indicator (Sec. 3.2.3)
    double ind;
    if (!e.have_u) {
      const double zl2 = zr_s[m - 1] * zr_s[m - 1] + zi_s[m - 1] * zi_s[m - 1];
      ind = fabs(hlast) * sqrt(zl2);
    } else {
      // t = H_m y; t <- t - U_r (U_r^T t); ind = sqrt(|t|^2 + |h y_m|^2)
      double *tr = e.tw + size_t(blockIdx.x) * 2 * size_t(e.ld), *ti = tr + e.ld;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int k = (i > 0 ? i - 1 : 0); k < m; ++k) {
          const double h = e.H[i + int64_t(k) * e.ldH];
          sr += h * yr[k];
          si += h * yi[k];
        }
        tr[i] = sr;
        ti[i] = si;
      }
      __syncthreads();
      // u = U_r^T t  (r entries, in br/bi)
      for (int k = threadIdx.x; k < r; k += blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int i = 0; i < m; ++i) {
          const double u = e.U[i + int64_t(k) * e.ld];
          sr += u * tr[i];
          si += u * ti[i];
        }
        br[k] = sr;
        bi[k] = si;
      }
      __syncthreads();
      double acc = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double sr = tr[i], si = ti[i];
        for (int k = 0; k < r; ++k) {
          const double u = e.U[i + int64_t(k) * e.ld];
          sr -= u * br[k];
          si -= u * bi[k];
        }
        acc += sr * sr + si * si;
      }
      acc = block_sum(acc, red);
      const double hy2 = hlast * hlast * (yr[m - 1] * yr[m - 1] + yi[m - 1] * yi[m - 1]);
      ind = sqrt(acc + hy2);
    }
    if (threadIdx.x == 0) {
      e.amp_re[idx] = amp.re;
      e.amp_im[idx] = amp.im;
      e.ind[idx] = ind;
      if (lim > 0.0 && idx + 1 < r) {
        e.amp_re[idx + 1] = amp.re;
        e.amp_im[idx + 1] = -amp.im;
        e.ind[idx + 1] = ind;
      }
    }
    if (lim > 0.0 && idx + 1 < r) {
      double *yr2 = e.yr + int64_t(idx + 1) * e.ld, *yi2 = e.yi + int64_t(idx + 1) * e.ld;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        yr2[i] = yr[i];
        yi2[i] = -yi[i];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ ordering
// key_i = |c_i| (a conjugate pair takes the larger of its two), order by key desc, |lambda| desc,
// Im desc, index asc.  Writes the sorted eigenvalues, indicators, amplitudes and y columns.
__global__ void order_kernel(EigArgs e, int nsel) {
  const int r = e.isc[ISC_R];
  const int m = e.m;
  extern __shared__ double sh[];
  double *key = sh, *lab = sh + r;
  int *pos = reinterpret_cast<int *>(sh + 2 * r);
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    double k = hypot(e.amp_re[i], e.amp_im[i]);
    if (e.wi[i] > 0.0 && i + 1 < r) k = fmax(k, hypot(e.amp_re[i + 1], e.amp_im[i + 1]));
    if (e.wi[i] < 0.0 && i > 0) k = fmax(k, hypot(e.amp_re[i - 1], e.amp_im[i - 1]));
    key[i] = k;
    lab[i] = hypot(e.wr[i], e.wi[i]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    int rank = 0;
    for (int k = 0; k < r; ++k) {
      bool before;
      if (key[k] != key[i]) before = key[k] > key[i];
      else if (lab[k] != lab[i]) before = lab[k] > lab[i];
      else if (e.wi[k] != e.wi[i]) before = e.wi[k] > e.wi[i];
      else before = k < i;
      rank += before;
    }
    pos[i] = rank;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const int p = pos[i];
    e.out[OUT_LRE * e.ld + p] = e.wr[i];
    e.out[OUT_LIM * e.ld + p] = e.wi[i];
    e.out[OUT_IND * e.ld + p] = e.ind[i];
    e.out[OUT_ARE * e.ld + p] = e.amp_re[i];
    e.out[OUT_AIM * e.ld + p] = e.amp_im[i];
    e.perm[p] = i;
  }
  __syncthreads();
  // sorted y columns 0..nsel-1
  for (int64_t t = threadIdx.x; t < int64_t(nsel) * m; t += blockDim.x) {
    const int c = int(t / m), i = int(t % m);
    const int src = e.perm[c];
    e.ysr[i + int64_t(c) * e.ld] = e.yr[i + int64_t(src) * e.ld];
    e.ysi[i + int64_t(c) * e.ld] = e.yi[i + int64_t(src) * e.ld];
  }
}

// sum |Hs| over the Hessenberg band (for the pivot floor of inverse iteration)
__global__ void anorm_kernel(const double *Hs, int ld, const int *isc, double *out) {
  const int n = isc[ISC_R];
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < int64_t(n) * n; e += blockDim.x) {
    const int i = int(e % n), c = int(e / n);
    if (i <= c + 1) s += fabs(Hs[i + int64_t(c) * ld]);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[0] = s;
}

}  // namespace foa
