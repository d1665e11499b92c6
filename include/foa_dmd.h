/*
 * foa_dmd.h -- C ABI of the GB300 streaming FOA-based DMD library.
 *
 * The library implements the modified Full Orthogonalization Arnoldi (FOA) update of
 * FOA-based projected DMD (Anantharamu & Mahesh, arXiv:1805.05821, Sec. 3.1, Algorithms 1,
 * 3 and 4) and the on-demand extraction of DMD eigenvalues, error indicators, amplitudes and
 * modes (the eigen extraction of Algorithm 1, Sec. 3.2.2-3.2.4).  Every step runs in CUDA kernels built
 * for sm_103a; there is no CPU fallback.  If no suitable GPU is present, foa_dmd_create
 * returns FOA_DMD_ECUDA.
 *
 * Conventions (all entry points):
 *  - Every call returns a status (foa_dmd_status).  On any status other than FOA_DMD_OK and
 *    FOA_DMD_EBREAKDOWN the stream state (H, V, beta, q) is unchanged.
 *  - "device" pointers are CUDA global memory of the current device; "host" pointers are
 *    ordinary (or pinned) host memory.  The caller owns every buffer it passes; the library
 *    keeps no pointer to it after the call's stream work has completed.
 *  - Work is issued on the handle's stream (foa_dmd_opts.cuda_stream).  Calls that take a
 *    host output pointer synchronise that stream before returning; the others are
 *    asynchronous and stream-ordered.
 *  - A handle is not thread-safe.  Different handles are independent.
 *  - Storage dtype: snapshots and the basis V are stored in FP64, FP32 or BF16.  H-bar, beta
 *    and all coefficient arithmetic are FP64 in every case.  With FP32 or BF16 storage the
 *    streaming dot products use FP32 products with FP64 accumulation of blocked partial sums.
 */
#ifndef FOA_DMD_H
#define FOA_DMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct foa_dmd foa_dmd_t;
typedef struct foa_dmd_batch foa_dmd_batch_t;

/* storage dtype of snapshots and of V */
typedef enum { FOA_DMD_F64 = 0, FOA_DMD_F32 = 1, FOA_DMD_BF16 = 2 } foa_dmd_dtype;

typedef enum {
  FOA_DMD_OK = 0,
  FOA_DMD_EINVAL = 1,      /* bad argument (null pointer, size, misaligned buffer, ...) */
  FOA_DMD_ENOMEM = 2,      /* device or host allocation failed */
  FOA_DMD_ECUDA = 3,       /* CUDA error, or no sm_103 device */
  FOA_DMD_EFULL = 4,       /* q == k_max: no room for another basis vector */
  FOA_DMD_EBREAKDOWN = 5,  /* snapshot is linearly dependent on the previous ones (Sec. 3.2.4:
                              h_{j+1,j} = 0); H-bar column j is recorded with h_{j+1,j} = 0,
                              the stream freezes and the j x j projected matrix is exact */
  FOA_DMD_ESTOPPED = 6,    /* push after a breakdown */
  FOA_DMD_ENONFINITE = 7,  /* snapshot holds NaN or Inf; state unchanged */
  FOA_DMD_ETIMEOUT = 8,    /* a bounded device wait ran out and the waiting kernel returned;
                              from foa_dmd_eig the stream state is unchanged and the handle
                              stays usable, after a push call the handle should be destroyed */
  FOA_DMD_EIO = 9,         /* checkpoint file error or checksum mismatch */
  FOA_DMD_ENOCONV = 10,    /* the device eigensolver did not converge */
  FOA_DMD_ERESOLVE = 11    /* foa_dmd_push_block only: a snapshot's new direction is too small
                              for the block form to keep V orthogonal; that snapshot and the
                              rest of the call were not pushed, the stream is not stopped */
} foa_dmd_status;

typedef struct {
  int32_t reorth;          /* 1 (default): classical Gram-Schmidt with one reorthogonalization
                              (CGS2, Alg. 1); 0: one classical Gram-Schmidt pass;
                              2: the same CGS2 step read as two passes over V per push:
                              h_{j+1,j} from ||w||^2 - ||s||^2 (w after the first projection,
                              s = V^T w, Pythagoras for orthonormal V), and v_{j+1} written
                              while the next push streams V.  H-bar, beta and q are committed
                              at the end of each push; the newest basis column is written by
                              the next push or before V is read (foa_dmd_get_basis,
                              foa_dmd_save, foa_dmd_eig modes).  Other values: EINVAL. */
  double breakdown_tol;    /* breakdown when h_{j+1,j} beta_{j,j} <= tol * ||x||_2; <= 0 selects
                              the default sqrt(u) of the storage dtype (2^-26.5, 2^-12, 2^-4) */
  int32_t indicator_every; /* 0 (default): push reports h_{j+1,j} only; m > 0: every m-th push
                              also runs the eigensolve and reports the error indicator */
  int32_t n_lead;          /* number of leading modes (by |amplitude|) the scheduled indicator
                              takes its maximum over; default 32 */
  double indicator_rank_tol; /* rank_tol for the scheduled eigensolve (0: no truncation,
                                < 0: automatic, as for foa_dmd_eig) */
  void *cuda_stream;       /* cudaStream_t for all work of the handle; NULL = default stream */
  int32_t form;            /* 0 (default): the push as Alg. 1 prints it (pre-vector
                              w = (psi - V beta_pre)/beta_jj, beta column from beta_pre + h beta_jj);
                              1: the QR view of the same push (Sec. 3.1): psi is orthogonalised
                              directly (h = V^T psi, CGS2 or CGS1 as reorth says), the beta column
                              is [h; nu] and the Hbar column comes from beta_{:,2:} = Hbar beta
                              (App. B, Eq. matmulhbeta) by forward substitution.  Equal in exact
                              arithmetic; the rounding differs.  form = 1 takes reorth 0 or 1;
                              other combinations: EINVAL.  The batched streams use form 0. */
} foa_dmd_opts;

/* Fill opts with the defaults listed above. */
void foa_dmd_opts_default(foa_dmd_opts *opts);

/* Result of one push. */
typedef struct {
  double h_last;     /* h_{q,q-1} of this push (beta_{1,1} = ||x|| on the first push) */
  double indicator;  /* max over the n_lead leading modes of the error indicator of Sec. 3.2.3
                        (Eq. errordmdvec: |h_{m+1,m}| |e_m^T z_i|, or its truncated form);
                        NaN when this push did not schedule an eigensolve */
  double x_norm;     /* ||x||_2 */
  int32_t q;         /* number of basis vectors after the push */
  int32_t status;    /* foa_dmd_status of this push */
} foa_dmd_push_info;

/*
 * Create a stream of snapshots of length n with room for k_max snapshots
 * (2 <= k_max <= 512).  Allocates V (n x k_max, storage dtype, row-tiled), H-bar and beta
 * (k_max x k_max, FP64) and scratch on the current device (the allocation of Alg. 4 done once, at
 * the maximum size).  opts may be NULL (defaults).  Errors: EINVAL, ENOMEM, ECUDA.
 */
int foa_dmd_create(int64_t n, int32_t k_max, int32_t dtype, const foa_dmd_opts *opts,
                   foa_dmd_t **out);

/*
 * Push one snapshot: Algorithm 4 with p = 1 (the first snapshot's normalisation, otherwise
 * the modified FOA update of Alg. 1).  x_dev: device, n contiguous elements of the handle's dtype, 16-byte
 * aligned.  info: host; NULL makes the call fully asynchronous (no synchronisation), and
 * errors found on the device are then reported by the next synchronising call.  The first
 * push of a stream always synchronises.  Errors: EINVAL, EFULL, EBREAKDOWN, ESTOPPED,
 * ENONFINITE, ETIMEOUT, ECUDA.
 */
int foa_dmd_push(foa_dmd_t *h, const void *x_dev, foa_dmd_push_info *info);

/*
 * Push p snapshots, the columns of X_dev (device, column-major, leading dimension ld >= n,
 * ld a multiple of 16 bytes / element size): Algorithm 4 with batch p.  The arithmetic is
 * bitwise identical to p calls of foa_dmd_push (Sec. 3.1: the streaming and batch forms carry
 * out the same floating-point operations in the same order).  infos: host array of p, or
 * NULL (asynchronous).  Stops at the first push whose status is not OK.
 */
int foa_dmd_push_batch(foa_dmd_t *h, const void *X_dev, int32_t p, int64_t ld,
                       foa_dmd_push_info *infos);

/*
 * Push one snapshot held in host memory: copies x_host (n elements of the handle's dtype;
 * pinned memory from foa_dmd_host_alloc gives full copy bandwidth) to a device staging
 * buffer on the handle's stream, then pushes it as foa_dmd_push does.  Before enqueueing the
 * copy the calling thread reads one byte per host page of x_host (pinned pages left unused for
 * seconds otherwise copy at a fraction of the link's rate).  The call returns once the copy is
 * enqueued; x_host must stay valid until the handle's stream has passed the copy (any later
 * synchronising call, or foa_dmd_sync).
 */
int foa_dmd_push_host(foa_dmd_t *h, const void *x_host, foa_dmd_push_info *info);

/*
 * Push-time error indicators (foa_dmd_opts.indicator_every = m > 0).  Every m-th push enqueues
 * the eigensolve of the projected matrix of that moment on a low-priority side stream, where it
 * overlaps the following pushes (the streaming passes leave one SM free for it).  A push that
 * asks for its info waits for its own indicator.  This call waits for the side stream and
 * returns, oldest first, up to cap records not yet read: the 1-based index of the push that
 * scheduled it (counted since create/reset), the size m of the projected matrix, and the
 * indicator (max over the n_lead leading modes; NaN if the eigensolve failed).  The device
 * keeps the last 1024 records.  Indicators assume the preceding asynchronous pushes succeeded.
 */
int foa_dmd_indicators(foa_dmd_t *h, int32_t *push_index, int32_t *m, double *value, int32_t cap,
                       int32_t *count);

/* Wait for the handle's stream and return the status of the most recent push. */
int foa_dmd_sync(foa_dmd_t *h, foa_dmd_push_info *info);

/*
 * Eigen-decomposition of the projected matrix (the eigen extraction of Alg. 1 and Alg. 3), all
 * on the device in FP64:
 *   m = q-1 (or q after a breakdown), H_m = H-bar(1:m,1:m);
 *   rank_tol > 0: SVD beta_m = U Sigma W^T, r = #{sigma_i > rank_tol sigma_1},
 *                 G = U_r^T H_m U_r;  rank_tol < 0: the same with rank_tol = N eps(dtype)
 *                 (the numerical-rank rule of Sec. 4.1 with N = m+1 snapshots);
 *   rank_tol == 0: no truncation, U_r = I, G = H_m;
 *   (lambda_i, z_i) = eig(G) with ||z_i|| = 1, largest-magnitude entry real positive;
 *   indicators (Sec. 3.2.3): |h_{m+1,m}| |e_m^T z_i|, truncated
 *                 ||[(I - U_r U_r^T) H_m U_r z_i ; h_{m+1,m} e_m^T U_r z_i]||;
 *   amplitudes c (Sec. 3.2.4, Eqs. exrecon/exreconwrt): [z] c = beta_11 U_r^T e_1;
 *   order: |c| descending, then |lambda| descending, then Im(lambda) descending
 *   (a conjugate pair shares the larger |c|, so its +Im member comes first);
 *   modes (Alg. 1): Phi_i = V_{1:m} U_r z_i for the first n_modes in that order.
 * Results go to the caller's buffers in res (see foa_dmd_eig_result).  Synchronises.
 * Errors: EINVAL (m < 1, cap too small, bad phi buffer), ENOCONV, ECUDA.
 */
typedef struct {
  /* inputs */
  int32_t cap;        /* capacity (entries) of each host array below; must be >= r */
  int32_t n_modes;    /* number of leading modes to form into phi_dev (0: no modes) */
  void *phi_dev;      /* device, n x (2 n_modes), column-major, leading dimension ld_phi
                         (>= n, 16-byte multiple): column 2i = Re Phi_i, column 2i+1 = Im Phi_i;
                         FP64 for FP64 storage, FP32 otherwise */
  int64_t ld_phi;
  double *vec_re, *vec_im; /* optional host (m x vec_cols, leading dimension m): U_r z_i */
  int32_t vec_cols;
  /* outputs */
  int32_t m;          /* size of the projected matrix */
  int32_t r;          /* truncated rank (m without truncation) */
  double *lam_re, *lam_im;     /* host, cap entries: eigenvalues, in the order above */
  double *indicator;           /* host, cap: error indicators */
  double *amp_re, *amp_im;     /* host, cap: amplitudes c_i */
  double *sigma;               /* optional host, cap: singular values of beta_m (truncation) */
  double h_last;               /* h_{m+1,m} */
} foa_dmd_eig_result;

int foa_dmd_eig(foa_dmd_t *h, double rank_tol, foa_dmd_eig_result *res);

/*
 * Test hook for the failure path of the bounded device waits (no counterpart in the paper).
 * The next truncated foa_dmd_eig of this handle launches its cooperative SVD with CTA skip_cta
 * (clamped to the grid) returning before its first grid-barrier arrival, as a CTA that died
 * would, and every other CTA giving up after spin_cycles clock cycles (1 .. 2^32; the normal
 * limit is 2^32, about 2 s at 2 GHz).  That eig returns FOA_DMD_ETIMEOUT with the stream state
 * unchanged; the barrier is re-armed at every launch, so the next eig runs normally.  One shot:
 * the request is cleared by the launch it affects.  Errors: EINVAL.
 */
int foa_dmd_test_wait_fault(foa_dmd_t *h, int32_t skip_cta, int64_t spin_cycles);

/*
 * Copy the FP64 state to host buffers (synchronises): q, stopped flag, H-bar and beta as
 * k_max x k_max column-major arrays with leading dimension ld >= k_max (either may be NULL).
 */
int foa_dmd_get_state(foa_dmd_t *h, int32_t *q, int32_t *stopped, double *Hbar, double *beta,
                      int32_t ld);

/*
 * Copy basis columns col0 .. col0+ncols-1 of V into dst_dev (device, n x ncols column-major,
 * leading dimension ld >= n, storage dtype).  V itself is kept row-tiled: rows are grouped in
 * tiles of 32, and each tile stores its k_max columns contiguously, so one push reads every
 * tile's leading q columns as a single contiguous block.
 */
int foa_dmd_get_basis(foa_dmd_t *h, int32_t col0, int32_t ncols, void *dst_dev, int64_t ld);

/* Discard all snapshots (q = 0, not stopped); buffers are kept. */
int foa_dmd_reset(foa_dmd_t *h);

/*
 * Checkpoint: the stream state of Algorithm 3 is exactly (H, V, beta, q).  save writes a
 * header (magic, version, n, k_max, dtype, q, stopped), H-bar, beta and the q basis columns
 * in storage dtype, with an FNV-1a checksum; load recreates a handle from it.  Pushing after
 * load gives bitwise the same results as an uninterrupted run.  Errors: EIO, ENOMEM, ECUDA.
 */
int foa_dmd_save(foa_dmd_t *h, const char *path);
int foa_dmd_load(const char *path, const foa_dmd_opts *opts, foa_dmd_t **out);

/*
 * One push that allocates no device memory, for callers that cannot call cudaMalloc at that
 * point (an arena or pool owns all device memory, or a host application forbids allocation on
 * its hot path).  The paper has no counterpart: it is the arithmetic of foa_dmd_push (Alg. 4
 * with p = 1) on buffers the caller owns, with the library's per-push scratch in a fixed
 * file-scope device array instead of allocated memory.
 *   V:        device, row-tiled basis as described at foa_dmd_get_basis (n rounded up to a
 *             multiple of 32 rows, k_max columns per tile, storage dtype, zero-initialised);
 *   Hbar, beta: device, k_max x k_max FP64 column-major (zero-initialised before the first push);
 *   q:        current number of basis vectors (0 for the first snapshot; after an OK push the
 *             new q is info->q, after EBREAKDOWN q stays as it was);
 *   x_dev:    device, the snapshot (n elements, storage dtype, 16-byte aligned);
 *   w_dev:    device, working vector of ceil(n/32)*32 elements (FP32, or FP64 for FP64 storage),
 *             zero-initialised once; on return it holds the unnormalised new direction;
 *   info:     host, result of the push (q after the push, h_last, status).
 * Limits: k_max <= 512 (384 for FP64); the scratch array holds the partial sums of at most 1024
 * CTAs (about 4.8 MB, kept by every GPU that loads the library until the process exits).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 * should therefore come before any stream capture.  Every call shares the array and clears
 * what must start at zero; calls that overlap on the GPU (different streams or threads) race
 * on it.  The call synchronises cuda_stream before returning, so it cannot be part of a stream
 * capture: while cuda_stream is being captured it returns EINVAL without enqueueing anything.
 * There is no handle to remember a breakdown: the caller's H-bar is the record.  A breakdown
 * (EBREAKDOWN) writes h into H-bar column q (1-based) and leaves q alone; a later call with that
 * q finds the column non-zero and returns ESTOPPED without changing anything (a zero first
 * snapshot records nothing, so a call after it starts the stream afresh).  Errors: EINVAL (sizes
 * beyond the limits, null pointers, a capturing stream), EFULL, EBREAKDOWN, ESTOPPED, ENONFINITE,
 * ETIMEOUT, ECUDA.
 */
int foa_dmd_push_noalloc(int64_t n, int32_t k_max, int32_t dtype, void *V, double *Hbar, double *beta,
                         int32_t q, const void *x_dev, void *w_dev, double breakdown_tol, void *cuda_stream,
                         foa_dmd_push_info *info);

/* Free all resources of the handle (synchronises its stream). NULL is ignored. */
void foa_dmd_destroy(foa_dmd_t *h);

/* Static string for a status code. */
const char *foa_dmd_strerror(int status);

/*
 * Kernel timing.  While enabled, every streaming-pass launch of the handle is bracketed by
 * CUDA events on the handle's stream.  foa_dmd_profile_read synchronises and returns, per
 * kernel kind (0: pass A = pre-vector and h = V^T w, 1: pass B = w -= V h and s = V^T w, 2: pass
 * C = h += s, w -= V s and ||w||, 3: the column write v_{j+1} = w / h_{j+1,j}; with reorth = 2, 0 is the lagged first pass, 1 the second
 * pass and 3 also the finishing column write), the summed event time in ms, the launch count and the
 * algorithmic bytes those launches had to move, plus the number of kernels of any kind the
 * handle launched since the previous read, then clears the counters.
 */
typedef struct {
  double ms[4];
  double bytes[4];
  int64_t launches[4];
  int64_t total_launches;
} foa_dmd_kernel_stats;

int foa_dmd_profile(foa_dmd_t *h, int enable);
int foa_dmd_profile_read(foa_dmd_t *h, foa_dmd_kernel_stats *stats);

/*
 * Block push (no counterpart in Alg. 4, whose p snapshots are pushed one after the other): the
 * snapshots are taken `block` at a time (2 or 4), each block orthogonalised against V by block
 * classical Gram-Schmidt with one reorthogonalisation and then inside the block by Cholesky QR,
 * twice; the beta block column is [C; R] and the H-bar columns follow from beta_{:,2:} = H-bar beta
 * (App. B, Eq. matmulhbeta) by forward substitution, as in the QR view (foa_dmd_opts.form = 1).
 * In exact arithmetic the result is that of p single pushes (X = V beta is the unique QR
 * factorisation with a positive diagonal, Sec. 3.1); the rounding differs, and Cholesky QR loses
 * orthogonality as O(u kappa(W)^2) when a block is nearly dependent on the basis.  V is read three
 * times per block instead of three times per snapshot.
 *   X_dev: device, p snapshots, snapshot t at X_dev + t*ld elements (storage dtype, 16-byte
 *          aligned rows: ld * element size a multiple of 16); block: 2 or 4.
 *   infos: host, p results (or NULL).  The first snapshot of a stream, a remainder shorter than
 *          `block` and the columns just below k_max are pushed singly (with the handle's form).
 * A dependent snapshot inside a block commits the columns before it and stops the stream
 * (EBREAKDOWN; later snapshots ESTOPPED).
 * Resolution limit (no counterpart in the paper; Sec. 3.2.2 explains why the QR form, unlike the
 * modified FOA update, loses accuracy as kappa_2(X) grows): block classical Gram-Schmidt keeps
 * the new columns orthogonal to V only while a snapshot's new direction stays well above the
 * rounding of its projections, R_ii >> u_s ||psi||.  Below R_ii = 16 u_s ||psi|| (u_s the unit
 * roundoff of the storage type; 9.5e-7 for FP32) the block form is not used: the columns before
 * that snapshot are committed, the call returns FOA_DMD_ERESOLVE and reports ERESOLVE for that
 * snapshot and every later one of the call, none of which is pushed, and the stream is NOT
 * stopped: push them with foa_dmd_push, whose modified FOA form stays orthogonal there.  (On
 * 4 x 16^3 fields with 1e-7 noise, without this limit V lost its orthogonality about 100 columns
 * after R_ii fell to 7 u_fp32 ||psi||, and H-bar diverged.)
 * FP32/BF16 storage only (EINVAL for FP64).  The push-time indicator schedule is not run by block
 * pushes.  Synchronises the handle's stream.
 */
int foa_dmd_push_block(foa_dmd_t *h, const void *X_dev, int32_t p, int64_t ld, int32_t block,
                       foa_dmd_push_info *infos);

/*
 * Autotuner of the streaming-pass launch geometry (no counterpart in the paper).  For every pass
 * kind the handle's options use (A/B/C, or the two passes of reorth = 2) and every j bucket up to
 * k_max (upper ends 8, 16, 32, 64, 128, 192, 256, 320, 384, 448, 512), times each candidate
 * (V bytes per pipeline stage 16/32/64 KB x V bytes in flight per CTA 64/96/144/192 KB x one or two
 * CTAs per SM x, for the FP32/BF16 passes with column dots, the register-held or the shared-
 * memory form of the stage) on the handle's own buffers, over a prefix of V of about 2 GB, median
 * of three launches, and keeps the fastest; later pushes of the handle launch with it.
 *   cache_path: NULL, or a text file.  Choices found there for (device arch, dtype, floor(log2 n),
 *               kind, bucket) are used without timing; new choices are appended.
 *   flags:      bit 0 = time again even where the cache has a choice.
 * The handle must hold no snapshots (q == 0, e.g. right after create or reset): tuning overwrites
 * V, H-bar, beta and the working vector, and clears them again before returning.  Errors:
 * EINVAL (q != 0), ENOMEM, ECUDA, ETIMEOUT.  foa_dmd_tuned_geometry reports the geometry a pass
 * of kind (0 A, 1 B, 2 C, 3 lagged first pass, 4 second pass of the two-pass push) at basis size j
 * launches with (variant 0: register-held stage where it fits, 1: shared-memory stage), and whether
 * it was tuned (*tuned = 1) or is the default.
 */
int foa_dmd_autotune(foa_dmd_t *h, const char *cache_path, int32_t flags);
int foa_dmd_tuned_geometry(foa_dmd_t *h, int32_t kind, int32_t j, int64_t *stage_bytes, int64_t *inflight_bytes,
                           int32_t *ctas_per_sm, int32_t *variant, int32_t *tuned);

/*
 * Self-checking builds (the library compiled with -DFOA_DMD_CHECKED, the stand-in for a memory
 * checker): waits for the device, then returns in *bits the checks that failed since the last
 * call and clears them: 1 = a bulk copy's shared-memory destination outside the CTA's shared
 * window, 2 = a bulk copy's address or size not 16-byte aligned (or its mbarrier not 8-byte
 * aligned), 4 = a streaming pass's tile index outside the tile count.  A failed check skips the
 * access (the pipeline that misses it ends in its bounded wait with FOA_DMD_ETIMEOUT), so nothing
 * faults.  In a normal build *bits = 0 and the call returns FOA_DMD_EINVAL.
 */
int foa_dmd_check_status(uint32_t *bits);

/* Pinned host memory for foa_dmd_push_host (cudaHostAlloc / cudaFreeHost). */
int foa_dmd_host_alloc(size_t bytes, void **ptr);
int foa_dmd_host_free(void *ptr);

/*
 * Many independent streams of uneven n and k_max advanced together (all FP32 or all BF16
 * storage).  batch_push advances every stream whose x pointer is non-NULL by one push
 * (Algorithm 4, p = 1 each) in a single persistent kernel launch; streams have their own
 * H-bar, beta, V and q.  x_dev: DEVICE array of S device pointers.  h_last_dev: device array
 * of S doubles receiving h_{q,q-1} of each stream (NaN for inactive or failed streams).
 * Graph-capturable: all per-push decisions are read from device memory.
 * Per-stream statuses are read with foa_dmd_batch_get_state.
 */
int foa_dmd_batch_create(int32_t S, const int64_t *n, const int32_t *k_max, int32_t dtype,
                         const foa_dmd_opts *opts, foa_dmd_batch_t **out);
int foa_dmd_batch_push(foa_dmd_batch_t *b, const void *const *x_dev, double *h_last_dev);
int foa_dmd_batch_get_state(foa_dmd_batch_t *b, int32_t s, int32_t *q, int32_t *status,
                            double *Hbar, double *beta, int32_t ld);
int foa_dmd_batch_get_basis(foa_dmd_batch_t *b, int32_t s, int32_t col0, int32_t ncols,
                            void *dst_dev, int64_t ld);
void foa_dmd_batch_destroy(foa_dmd_batch_t *b);

#ifdef __cplusplus
}
#endif
#endif /* FOA_DMD_H */
