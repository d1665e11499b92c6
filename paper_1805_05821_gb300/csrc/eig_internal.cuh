// Internal declarations of the device eigen path (eig.cu, eig_host.cu, modes.cu).
#pragma once
#include "internal.cuh"

namespace foa {

constexpr int kMaxSweeps = 32;  // Jacobi sweeps at most (the launch asks for 30)

// Cross-CTA synchronisation state of the cooperative Jacobi SVD, zeroed before every launch.
struct GridBar {
  unsigned count;                 // grid barrier: arrivals
  unsigned gen;                   // grid barrier: generation
  unsigned rot[kMaxSweeps];       // rotations applied in each sweep (summed over CTAs)
  unsigned round[kMaxK / 2];      // rounds each CTA has finished (its neighbours wait on it)
};

// integer scalars of one eigen-decomposition (device)
enum { ISC_R = 0, ISC_STATUS = 1, ISC_ERR = 2, ISC_ROT = 3, ISC_SWEEPS = 4, ISC_N = 16 };
// rows of the sorted output block (each ld long)
enum { OUT_LRE = 0, OUT_LIM = 1, OUT_IND = 2, OUT_ARE = 3, OUT_AIM = 4, OUT_N = 5 };

struct EigArgs {
  const double *Hs;   // Hessenberg matrix whose eigenpairs are wanted (r x r, ld)
  const double *Q;    // G = Q Hs Q^T (when have_q)
  const double *U;    // U_r (m x r, ld) when have_u
  const double *H;    // H-bar of the stream (ldH), for the truncated indicator
  int ldH;
  const double *wr, *wi;
  const double *anorm;
  double *lu, *tw;    // per-CTA scratch
  double *yr, *yi;    // y_i = U_r z_i (m x r, ld), unsorted
  double *ysr, *ysi;  // sorted y columns
  double *ind, *amp_re, *amp_im;
  double *out;        // OUT_N x ld sorted scalars
  int *perm;
  int *isc;
  int ld, m;
  int have_q, have_u;
  const double *hlast_p;  // h_{m+1,m} (device)
  const double *b11_p;    // beta_{1,1} (device)
};

// one push-time indicator (device ring written by the indicator stream)
struct IndRecord {
  int32_t push;   // 1-based index of the push that scheduled it
  int32_t m;      // size of the projected matrix
  double value;   // max over the n_lead leading modes
};

struct EigWork {
  int K = 0;
  int vgrid = 0;
  double *A = nullptr, *U = nullptr, *sig_raw = nullptr, *sig = nullptr, *G = nullptr, *Q = nullptr, *T = nullptr,
         *Aqr = nullptr, *wr = nullptr, *wi = nullptr, *yr = nullptr, *yi = nullptr, *ysr = nullptr, *ysi = nullptr,
         *ind = nullptr, *amp_re = nullptr, *amp_im = nullptr, *out = nullptr, *anorm = nullptr, *lu = nullptr,
         *tw = nullptr, *yplanes = nullptr;
  float *bop = nullptr;  // pre-split Y operand of the tensor-core mode product
  double *scal = nullptr;  // untruncated path: h_{m+1,m} and beta_11, copied with H_m
  int *perm = nullptr, *isc = nullptr;
  GridBar *gb = nullptr;
};

constexpr int kSvdThreads = 128;  // threads of a Jacobi SVD CTA (four warps per column pair)
constexpr int kSvdRows = (kMaxK + kSvdThreads - 1) / kSvdThreads;
constexpr long long kGridSpinCycles = 1ll << 32;  // bounded wait of a grid barrier (about 2 s at 2 GHz)
__global__ void svd_jacobi_kernel(const double *B, int ldb, int m, double *A, int lda, double *sig, int *isc,
                                  GridBar *gb, int max_sweeps, double tol, long long spin_limit, int skip_cta);
__global__ void svd_finish_kernel(const double *A, int lda, int m, const double *sig_in, double *U, double *sig,
                                  int *isc, double rank_tol);
__global__ void project_t_kernel(const double *H, int ldh, int m, const double *U, int ldu, const int *isc,
                                 double *T, int ldt);
__global__ void project_g_kernel(const double *U, int ldu, int m, const int *isc, const double *T, int ldt, double *G,
                                 int ldg);
__global__ void copy_h_kernel(const double *H, int ldh, int m, double *G, int ldg, int *isc, const double *B,
                              double *scal);
__global__ void hessenberg_kernel(double *G, int ldg, double *Q, int ldq, const int *isc);
__global__ void hqr_kernel(double *Ag, int lda, const int *isc_in, double *wr, double *wi, int *isc,
                           int smem_elems);
__global__ void vectors_kernel(EigArgs e);
__global__ void order_kernel(EigArgs e, int nsel);
__global__ void anorm_kernel(const double *Hs, int ld, const int *isc, double *out);

size_t modes_tc_bop_bytes(int kmax);
// modes.cu: Phi = V Y (Y: m x ncols real planes, ld), written to phi (ld_phi)
int launch_modes(foa_dmd *h, int m, const double *Y, int ldy, int ncols, void *phi, int64_t ld_phi);

}  // namespace foa
