/*
 * FP64 CPU oracle of the modified Full Orthogonalization Arnoldi (FOA) update of FOA-based
 * DMD (Anantharamu & Mahesh, arXiv:1805.05821): Algorithm 1 steps 2-19 and the streaming
 * update of Algorithm 4, one snapshot per call.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links or calls this file; only the
 * tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * The steps run unfused, one plain loop each, in the order the paper gives them.  Every sum
 * over rows is taken over fixed blocks of ORACLE_BLOCK rows, each summed in index order, and
 * the block sums are then added in block order, so the result does not depend on the number
 * of OpenMP threads.  Build with -O2 -ffp-contract=off: no fused multiply-add anywhere.
 *
 * Storage: V is n x kmax column-major (leading dimension ldv), Hbar is kmax x kmax
 * column-major (ldh, row j holds h_{j+1,j} in 1-based terms), beta is kmax x kmax
 * column-major (ldb).  Indices below are 0-based; comments give the paper's 1-based names.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_BLOCK 4096

/* status codes returned to the Python side of the oracle */
#define ORACLE_OK 0
#define ORACLE_BREAKDOWN 1
#define ORACLE_NOMEM 2

static int64_t nblocks_of(int64_t n) { return (n + ORACLE_BLOCK - 1) / ORACLE_BLOCK; }

/* sum_r a[r]*b[r] over fixed row blocks */
static double dot_blocked(int64_t n, const double *a, const double *b, double *part) {
  int64_t nb = nblocks_of(n);
#pragma omp parallel for schedule(static)
  for (int64_t blk = 0; blk < nb; ++blk) {
    int64_t r0 = blk * ORACLE_BLOCK, r1 = r0 + ORACLE_BLOCK < n ? r0 + ORACLE_BLOCK : n;
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) s += a[r] * b[r];
    part[blk] = s;
  }
  double s = 0.0;
  for (int64_t blk = 0; blk < nb; ++blk) s += part[blk];
  return s;
}

/* out[i] = sum_r V[r,i] * w[r], i < j  (V_{:,1:j}^T w), blocked over rows */
static void gemv_t(int64_t n, int32_t j, const double *V, int64_t ldv, const double *w, double *out,
                   double *part) {
  int64_t nb = nblocks_of(n);
#pragma omp parallel for schedule(static)
  for (int64_t blk = 0; blk < nb; ++blk) {
    int64_t r0 = blk * ORACLE_BLOCK, r1 = r0 + ORACLE_BLOCK < n ? r0 + ORACLE_BLOCK : n;
    for (int32_t i = 0; i < j; ++i) {
      const double *v = V + (int64_t)i * ldv;
      double s = 0.0;
      for (int64_t r = r0; r < r1; ++r) s += v[r] * w[r];
      part[blk * j + i] = s;
    }
  }
  for (int32_t i = 0; i < j; ++i) {
    double s = 0.0;
    for (int64_t blk = 0; blk < nb; ++blk) s += part[blk * j + i];
    out[i] = s;
  }
}

/* y[r] = sum_{i<j} V[r,i] * c[i], summed in column order for every row */
static void gemv_n(int64_t n, int32_t j, const double *V, int64_t ldv, const double *c, double *y) {
  int64_t nb = nblocks_of(n);
#pragma omp parallel for schedule(static)
  for (int64_t blk = 0; blk < nb; ++blk) {
    int64_t r0 = blk * ORACLE_BLOCK, r1 = r0 + ORACLE_BLOCK < n ? r0 + ORACLE_BLOCK : n;
    for (int64_t r = r0; r < r1; ++r) y[r] = 0.0;
    for (int32_t i = 0; i < j; ++i) {
      const double *v = V + (int64_t)i * ldv;
      double ci = c[i];
      for (int64_t r = r0; r < r1; ++r) y[r] += v[r] * ci;
    }
  }
}

/*
 * First push (Alg. 4 steps 4-8 / Alg. 1 steps 2-3): beta_{1,1} = ||psi_1||_2,
 * v_1 = psi_1 / beta_{1,1}.  Returns ORACLE_BREAKDOWN for a zero snapshot.
 */
int foa_oracle_first(int64_t n, double *V, double *B, const double *x, double *out_norm) {
  double *part = (double *)malloc(sizeof(double) * (size_t)nblocks_of(n));
  if (!part) return ORACLE_NOMEM;
  double b = sqrt(dot_blocked(n, x, x, part));
  free(part);
  *out_norm = b;
  if (!(b > 0.0)) return ORACLE_BREAKDOWN;
  B[0] = b;
  for (int64_t r = 0; r < n; ++r) V[r] = x[r] / b;
  return ORACLE_OK;
}

/*
 * One modified-FOA step with j = q >= 1 basis vectors (Alg. 4 steps 9-20 for one snapshot,
 * Alg. 1 steps 4-18 for index j):
 *   beta_pre_1     = sum_{l=1}^{j-1}   h_{1,l} beta_{l,j}                     (step 5)
 *   beta_pre_i     = sum_{l=i-1}^{j-1} h_{i,l} beta_{l,j},  i = 2..j          (steps 6-8)
 *   w              = (psi_{j+1} - V_{1:j} beta_pre) / beta_{j,j}               (step 9)
 *   h              = V^T w;  w = w - V h;  s = V^T w;  h = h + s;  w = w - V s (steps 10-14)
 *   h_{j+1,j}      = ||w||_2;  v_{j+1} = w / h_{j+1,j}                           (step 15)
 *   beta_{i,j+1}   = beta_pre_i + h_{i,j} beta_{j,j},  i = 1..j;
 *   beta_{j+1,j+1} = h_{j+1,j} beta_{j,j}                                       (steps 16-18)
 * reorth = 0 drops the second Gram-Schmidt pass (s = 0, classical Gram-Schmidt once).
 * reorth = 2 is the two-pass reading of the same step: h_{j+1,j} is taken from the Pythagorean
 * identity ||w - V s||^2 = ||w||^2 - ||s||^2 (w after the first projection, s = V^T w), the form
 * that lets a streaming implementation append v_{j+1} during the next snapshot's first pass.
 * A new direction is declared dependent (Sec. 3.2.4: h_{j+1,j} = 0 means psi_{j+1} lies in
 * span{psi_1..psi_j}) when h_{j+1,j} beta_{j,j} <= tol * ||psi_{j+1}||_2; then column j of
 * Hbar gets h with h_{j+1,j} = 0, V and beta are left alone, and ORACLE_BREAKDOWN returns.
 * out[0] = h_{j+1,j}, out[1] = ||psi_{j+1}||_2.
 */
int foa_oracle_step(int64_t n, int32_t j, double *V, int64_t ldv, double *H, int32_t ldh, double *B,
                    int32_t ldb, const double *x, double tol, int reorth, double *out) {
  int64_t nb = nblocks_of(n);
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  double *part = (double *)malloc(sizeof(double) * (size_t)(nb * (j > 1 ? j : 1)));
  double *pre = (double *)calloc((size_t)j, sizeof(double));
  double *h = (double *)calloc((size_t)j, sizeof(double));
  double *s = (double *)calloc((size_t)j, sizeof(double));
  if (!w || !y || !part || !pre || !h || !s) {
    free(w); free(y); free(part); free(pre); free(h); free(s);
    return ORACLE_NOMEM;
  }
#define HB(i, l) H[(int64_t)(l) * ldh + (i)]
#define BT(i, l) B[(int64_t)(l) * ldb + (i)]
  const int32_t jc = j - 1; /* 0-based index of column j */

  /* steps 5-8: beta_pre (empty sums give 0 when j = 1) */
  for (int32_t i = 0; i < j; ++i) {
    int32_t l0 = i == 0 ? 0 : i - 1;
    double acc = 0.0;
    for (int32_t l = l0; l <= j - 2; ++l) acc += HB(i, l) * BT(l, jc);
    pre[i] = acc;
  }
  /* step 9 */
  double bjj = BT(jc, jc);
  gemv_n(n, j, V, ldv, pre, y);
  for (int64_t r = 0; r < n; ++r) w[r] = (x[r] - y[r]) / bjj;
  /* step 10 */
  gemv_t(n, j, V, ldv, w, h, part);
  /* step 11 */
  gemv_n(n, j, V, ldv, h, y);
  for (int64_t r = 0; r < n; ++r) w[r] = w[r] - y[r];
  double w1norm2 = 0.0;
  if (reorth == 2) w1norm2 = dot_blocked(n, w, w, part);
  if (reorth) {
    /* step 12 */
    gemv_t(n, j, V, ldv, w, s, part);
    /* step 13 */
    for (int32_t i = 0; i < j; ++i) h[i] = h[i] + s[i];
    /* step 14 */
    gemv_n(n, j, V, ldv, s, y);
    for (int64_t r = 0; r < n; ++r) w[r] = w[r] - y[r];
  }
  /* step 15 */
  double nu;
  if (reorth == 2) {
    double ss = 0.0;
    for (int32_t i = 0; i < j; ++i) ss += s[i] * s[i];
    double d = w1norm2 - ss;
    nu = sqrt(d > 0.0 ? d : 0.0);
  } else {
    nu = sqrt(dot_blocked(n, w, w, part));
  }
  double xn = sqrt(dot_blocked(n, x, x, part));
  out[0] = nu;
  out[1] = xn;
  for (int32_t i = 0; i < j; ++i) HB(i, jc) = h[i];
  int status = ORACLE_OK;
  if (!(nu * bjj > tol * xn)) {
    HB(j, jc) = 0.0;
    status = ORACLE_BREAKDOWN;
  } else {
    HB(j, jc) = nu;
    double *vn = V + (int64_t)j * ldv;
    for (int64_t r = 0; r < n; ++r) vn[r] = w[r] / nu;
    /* steps 16-18 */
    for (int32_t i = 0; i < j; ++i) BT(i, j) = pre[i] + h[i] * bjj;
    BT(j, j) = nu * bjj;
  }
#undef HB
#undef BT
  free(w); free(y); free(part); free(pre); free(h); free(s);
  return status;
}

/*
 * The QR view of the same push (Sec. 3.1: FOA-based DMD computes a QR factorisation X = V beta
 * of the snapshot matrix; App. B, Eq. matmulhbeta: beta_{:,2:j+1} = Hbar_j beta_j).  The new
 * snapshot is orthogonalised directly (CGS2 on psi_{j+1}, no pre-vector):
 *   h = V^T psi;  w = psi - V h;  s = V^T w;  h = h + s;  w = w - V s;  nu = ||w||_2
 *   beta_{1:j,j+1} = h,  beta_{j+1,j+1} = nu,  v_{j+1} = w / nu
 * and column j of Hbar follows from column j+1 of beta by forward substitution in
 * beta_{:,j+1} = sum_{l<=j} Hbar_{:,l} beta_{l,j}:
 *   Hbar_{i,j} = (beta_{i,j+1} - sum_{l=max(1,i-1)}^{j-1} Hbar_{i,l} beta_{l,j}) / beta_{j,j},  i <= j
 *   Hbar_{j+1,j} = beta_{j+1,j+1} / beta_{j,j}
 * In exact arithmetic this is the same Hbar as foa_oracle_step.  Breakdown reading as there:
 * nu <= tol * ||psi||_2 (nu is the distance of psi from span V), then column j of Hbar gets its
 * first j entries with Hbar_{j+1,j} = 0 and V, beta are left alone.
 * reorth = 0 drops s.  out[0] = Hbar_{j+1,j}, out[1] = ||psi||_2.
 */
int foa_oracle_qr_step(int64_t n, int32_t j, double *V, int64_t ldv, double *H, int32_t ldh, double *B,
                       int32_t ldb, const double *x, double tol, int reorth, double *out) {
  int64_t nb = nblocks_of(n);
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  double *part = (double *)malloc(sizeof(double) * (size_t)(nb * (j > 1 ? j : 1)));
  double *h = (double *)calloc((size_t)j, sizeof(double));
  double *s = (double *)calloc((size_t)j, sizeof(double));
  if (!w || !y || !part || !h || !s) {
    free(w); free(y); free(part); free(h); free(s);
    return ORACLE_NOMEM;
  }
#define HB(i, l) H[(int64_t)(l) * ldh + (i)]
#define BT(i, l) B[(int64_t)(l) * ldb + (i)]
  const int32_t jc = j - 1;
  gemv_t(n, j, V, ldv, x, h, part);
  gemv_n(n, j, V, ldv, h, y);
  for (int64_t r = 0; r < n; ++r) w[r] = x[r] - y[r];
  if (reorth) {
    gemv_t(n, j, V, ldv, w, s, part);
    for (int32_t i = 0; i < j; ++i) h[i] = h[i] + s[i];
    gemv_n(n, j, V, ldv, s, y);
    for (int64_t r = 0; r < n; ++r) w[r] = w[r] - y[r];
  }
  double nu = sqrt(dot_blocked(n, w, w, part));
  double xn = sqrt(dot_blocked(n, x, x, part));
  double bjj = BT(jc, jc);
  /* column j of Hbar from beta_{1:j,j+1} = h by forward substitution */
  for (int32_t i = 0; i < j; ++i) {
    int32_t l0 = i == 0 ? 0 : i - 1;
    double acc = 0.0;
    for (int32_t l = l0; l <= j - 2; ++l) acc += HB(i, l) * BT(l, jc);
    HB(i, jc) = (h[i] - acc) / bjj;
  }
  int status = ORACLE_OK;
  if (!(nu > tol * xn)) {
    HB(j, jc) = 0.0;
    out[0] = 0.0;
    status = ORACLE_BREAKDOWN;
  } else {
    HB(j, jc) = nu / bjj;
    out[0] = nu / bjj;
    double *vn = V + (int64_t)j * ldv;
    for (int64_t r = 0; r < n; ++r) vn[r] = w[r] / nu;
    for (int32_t i = 0; i < j; ++i) BT(i, j) = h[i];
    BT(j, j) = nu;
  }
  out[1] = xn;
#undef HB
#undef BT
  free(w); free(y); free(part); free(h); free(s);
  return status;
}

int foa_oracle_block_rows(void) { return ORACLE_BLOCK; }
