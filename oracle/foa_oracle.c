/*
 * FP64 CPU oracle of the modified Full Orthogonalization Arnoldi (FOA) update of FOA-based
 * DMD (Anantharamu & Mahesh, arXiv:1805.05821): the basis and coefficient updates of Algorithm 1 and the streaming
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
 * First push (Algorithms 1 and 4): beta_{1,1} = ||psi_1||_2,
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
 * One modified-FOA update of Algorithm 1 (Algorithm 4 for one snapshot) with j = q >= 1 basis
 * vectors.  With the stored basis V (n x j, orthonormal), H-bar (upper Hessenberg) and beta (upper
 * triangular, X_{1:j} = V beta), the snapshot psi = psi_{j+1} is taken into the basis through the
 * scaled pre-vector of the last column, not through psi itself (Sec. 3.1):
 *   beta_pre  = H-bar_{1:j,1:j-1} beta_{1:j-1,j}, i.e. beta_pre_i = sum_{l=max(1,i-1)}^{j-1} h_{i,l} beta_{l,j}
 *               (H-bar is upper Hessenberg; beta_pre = 0 for j = 1)
 *   w         = (psi - V beta_pre) / beta_{j,j}
 *   h         = V^T w,  w = w - V h,  s = V^T w,  h = h + s,  w = w - V s    (CGS with one reorthogonalisation)
 *   h_{j+1,j} = ||w||_2,  v_{j+1} = w / h_{j+1,j}
 *   beta_{1:j,j+1} = beta_pre + h beta_{j,j},  beta_{j+1,j+1} = h_{j+1,j} beta_{j,j}
 * so that psi = V_{1:j+1} beta_{1:j+1,j+1} and H-bar gains column j = [h; h_{j+1,j}].
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

  /* beta_pre (empty sums give 0 when j = 1) */
  for (int32_t i = 0; i < j; ++i) {
    int32_t l0 = i == 0 ? 0 : i - 1;
    double acc = 0.0;
    for (int32_t l = l0; l <= j - 2; ++l) acc += HB(i, l) * BT(l, jc);
    pre[i] = acc;
  }
  /* the scaled pre-vector */
  double bjj = BT(jc, jc);
  gemv_n(n, j, V, ldv, pre, y);
  for (int64_t r = 0; r < n; ++r) w[r] = (x[r] - y[r]) / bjj;
  /* first projection */
  gemv_t(n, j, V, ldv, w, h, part);
  gemv_n(n, j, V, ldv, h, y);
  for (int64_t r = 0; r < n; ++r) w[r] = w[r] - y[r];
  double w1norm2 = 0.0;
  if (reorth == 2) w1norm2 = dot_blocked(n, w, w, part);
  if (reorth) {
    /* reorthogonalisation */
    gemv_t(n, j, V, ldv, w, s, part);
    for (int32_t i = 0; i < j; ++i) h[i] = h[i] + s[i];
    gemv_n(n, j, V, ldv, s, y);
    for (int64_t r = 0; r < n; ++r) w[r] = w[r] - y[r];
  }
  /* the new direction's norm h_{j+1,j} */
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
    /* the beta column */
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

/*
 * Block push of p snapshots at once (the block form of the QR view: block classical Gram-Schmidt
 * with reorthogonalisation against V, then a Cholesky QR of the projected block, twice).  In exact
 * arithmetic it gives the same V, beta and Hbar as p single pushes (the QR factorisation of X with
 * a positive diagonal is unique, Sec. 3.1); the rounding differs.  Steps, X_b = [psi_{j+1} ..
 * psi_{j+p}] (n x p, leading dimension ldx):
 *   C1 = V^T X_b;  W = X_b - V C1;  C2 = V^T W;  W = W - V C2;  C = C1 + C2
 *   G = W^T W = R1^T R1 (Cholesky);  W1 = W R1^-1;  G2 = W1^T W1 = R2^T R2;  Q = W1 R2^-1;  R = R2 R1
 *   beta_{1:j, j+1:j+p} = C,  beta_{j+1:j+p, j+1:j+p} = R,  V_{:, j+1:j+p} = Q
 * and the Hbar columns j .. j+p-1 by the forward substitution of foa_oracle_qr_step, one column
 * after the other.  Breakdown: the first block column i with R_ii <= tol * ||psi_{j+1+i}||_2 (or a
 * Cholesky pivot <= 0) is dependent; the columns before it are committed, its Hbar column gets a
 * zero subdiagonal, and ORACLE_BREAKDOWN returns with out[0] = i (columns committed).
 * out[1 + i] = Hbar_{j+1+i, j+i} for the committed columns.
 */
static int chol_upper(int p, const double *G, int ldg, double *R, int ldr) {
  /* G = R^T R for the leading block that stays positive definite, R upper triangular (column-
     major); returns the number of leading columns factored (the first failing pivot, or p) */
  for (int c = 0; c < p; ++c)
    for (int r = 0; r < p; ++r) R[r + c * ldr] = 0.0;
  for (int i = 0; i < p; ++i) {
    double d = G[i + i * ldg];
    for (int k = 0; k < i; ++k) d -= R[k + i * ldr] * R[k + i * ldr];
    if (!(d > 0.0)) return i;
    double rii = sqrt(d);
    R[i + i * ldr] = rii;
    for (int c = i + 1; c < p; ++c) {
      double t = G[i + c * ldg];
      for (int k = 0; k < i; ++k) t -= R[k + i * ldr] * R[k + c * ldr];
      R[i + c * ldr] = t / rii;
    }
  }
  return p;
}

/* W[:, :m] (n rows, column stride n) := W[:, :m] R^-1, R upper triangular (leading dimension ldr) */
static void right_solve_upper(int64_t n, int m, double *W, const double *R, int ldr) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r) {
    for (int c = 0; c < m; ++c) {
      double t = W[r + (int64_t)c * n];
      for (int k = 0; k < c; ++k) t -= W[r + (int64_t)k * n] * R[k + c * ldr];
      W[r + (int64_t)c * n] = t / R[c + c * ldr];
    }
  }
}

/* G = W[:, :m]^T W[:, :m] (leading dimension ldg), each entry a blocked dot product */
static void gram_blocked(int64_t n, int m, const double *W, double *G, int ldg, double *part) {
  for (int a = 0; a < m; ++a)
    for (int b = a; b < m; ++b) {
      double g = dot_blocked(n, W + (int64_t)a * n, W + (int64_t)b * n, part);
      G[a + b * ldg] = g;
      G[b + a * ldg] = g;
    }
}

int foa_oracle_block_step(int64_t n, int32_t j, int32_t p, double *V, int64_t ldv, double *H, int32_t ldh,
                          double *B, int32_t ldb, const double *X, int64_t ldx, double tol, double *out) {
  out[0] = 0.0;
  if (p < 1) return ORACLE_OK;
  int64_t nb = nblocks_of(n);
  double *W = (double *)malloc(sizeof(double) * (size_t)(n * p));
  double *Y = (double *)malloc(sizeof(double) * (size_t)n);
  double *part = (double *)malloc(sizeof(double) * (size_t)(nb * (j > 1 ? j : 1)));
  double *C = (double *)calloc((size_t)(j * p), sizeof(double));
  double *C2 = (double *)calloc((size_t)j, sizeof(double));
  double *G = (double *)calloc((size_t)(p * p), sizeof(double));
  double *R1 = (double *)calloc((size_t)(p * p), sizeof(double));
  double *R2 = (double *)calloc((size_t)(p * p), sizeof(double));
  double *R = (double *)calloc((size_t)(p * p), sizeof(double));
  double *xn = (double *)malloc(sizeof(double) * (size_t)p);
  if (!W || !Y || !part || !C || !C2 || !G || !R1 || !R2 || !R || !xn) {
    free(W); free(Y); free(part); free(C); free(C2); free(G); free(R1); free(R2); free(R); free(xn);
    return ORACLE_NOMEM;
  }
#define HB(i, l) H[(int64_t)(l) * ldh + (i)]
#define BT(i, l) B[(int64_t)(l) * ldb + (i)]
  /* block Gram-Schmidt against V, twice */
  for (int k = 0; k < p; ++k) {
    const double *x = X + (int64_t)k * ldx;
    double *w = W + (int64_t)k * n;
    double *ck = C + (int64_t)k * j;
    xn[k] = sqrt(dot_blocked(n, x, x, part));
    gemv_t(n, j, V, ldv, x, ck, part);                          /* C1 = V^T X_b */
    gemv_n(n, j, V, ldv, ck, Y);
    for (int64_t r = 0; r < n; ++r) w[r] = x[r] - Y[r];          /* W = X_b - V C1 */
    gemv_t(n, j, V, ldv, w, C2, part);                          /* C2 = V^T W */
    gemv_n(n, j, V, ldv, C2, Y);
    for (int64_t r = 0; r < n; ++r) w[r] = w[r] - Y[r];          /* W = W - V C2 */
    for (int i = 0; i < j; ++i) ck[i] = ck[i] + C2[i];          /* C = C1 + C2 */
  }
  /* Cholesky QR twice on the leading columns that stay positive definite */
  gram_blocked(n, p, W, G, p, part);                           /* G = W^T W */
  const int m1 = chol_upper(p, G, p, R1, p);                   /* G = R1^T R1, leading m1 columns */
  int m = m1;
  if (m1 > 0) {
    right_solve_upper(n, m1, W, R1, p);                        /* W1 = W R1^-1 */
    gram_blocked(n, m1, W, G, p, part);                        /* G2 = W1^T W1 */
    m = chol_upper(m1, G, p, R2, p);                           /* G2 = R2^T R2, leading m columns */
    if (m > 0) right_solve_upper(n, m, W, R2, p);              /* Q = W1 R2^-1 */
  }
  /* R = R2 R1: rows r < m are defined for every column c (R1's rows below m1 are not: a column
     past the factored block keeps its coefficients on the factored directions) */
  for (int c = 0; c < p; ++c)
    for (int r = 0; r < m && r <= c; ++r) {
      double t = 0.0;
      const int kmax = c < m1 - 1 ? c : m1 - 1;
      for (int k = r; k <= kmax; ++k) t += R2[r + k * p] * R1[k + c * p];
      R[r + c * p] = t;
    }
  /* the first dependent column: R_ii <= tol ||psi|| (or no factor) */
  int ncommit = 0;
  int status = ORACLE_OK;
  for (int i = 0; i < p; ++i) {
    if (!(i < m && R[i + i * p] > tol * xn[i])) {
      status = ORACLE_BREAKDOWN;
      break;
    }
    ncommit = i + 1;
  }
  /* commits: beta block column, V */
  for (int i = 0; i < ncommit; ++i) {
    const int col = j + i;
    for (int r = 0; r < j; ++r) BT(r, col) = C[r + (int64_t)i * j];
    for (int r = 0; r <= i; ++r) BT(j + r, col) = R[r + i * p];
    double *vn = V + (int64_t)col * ldv;
    const double *qc = W + (int64_t)i * n;
    for (int64_t r = 0; r < n; ++r) vn[r] = qc[r];
  }
  /* Hbar columns by forward substitution (as foa_oracle_qr_step), one per new snapshot; the first
     dependent snapshot's column is formed from its coefficients with a zero subdiagonal */
  const int ncols = ncommit + (status == ORACLE_BREAKDOWN ? 1 : 0);
  for (int i = 0; i < ncols; ++i) {
    const int jc = j - 1 + i;          /* 0-based Hbar column of snapshot j+i (basis size j+i before it) */
    const int jj = j + i;
    const double bjj = BT(jc, jc);
    for (int r = 0; r < jj; ++r) {
      double brc;                      /* beta_{r, jj} of snapshot j+i */
      if (r < j) brc = C[r + (int64_t)i * j];
      else brc = R[(r - j) + i * p];   /* r - j < i <= m: a factored row */
      int l0 = r == 0 ? 0 : r - 1;
      double acc = 0.0;
      for (int l = l0; l <= jc - 1; ++l) acc += HB(r, l) * BT(l, jc);
      HB(r, jc) = (brc - acc) / bjj;
    }
    if (i < ncommit) {
      HB(jj, jc) = R[i + i * p] / bjj;
      out[1 + i] = HB(jj, jc);
    } else {
      HB(jj, jc) = 0.0;
    }
  }
  out[0] = (double)ncommit;
#undef HB
#undef BT
  free(W); free(Y); free(part); free(C); free(C2); free(G); free(R1); free(R2); free(R); free(xn);
  return status;
}

int foa_oracle_block_rows(void) { return ORACLE_BLOCK; }
