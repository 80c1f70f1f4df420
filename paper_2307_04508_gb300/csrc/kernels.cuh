// Launch interfaces of the LT-GW kernels (host side).  Every launcher issues
// its kernels on the given stream and returns the launch status; none of them
// synchronises.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ltgw {

enum ScaleMode { SCALE_NONE = 0, SCALE_DIRECT = 1, SCALE_LAPLACE = 2 };

// C_b = alpha * A_b diag(s_b) B_b for b in [0, batch).  With syrk = 1 only the
// lower-triangle tiles are computed and each value is mirrored (A == B^T).
struct GemmF64Args {
  int M = 0, N = 0;
  int64_t K = 0;
  const double *A = nullptr; int64_t lda = 0, strideA = 0;
  const double *B = nullptr; int64_t ldb = 0, strideB = 0;
  double *C = nullptr; int64_t ldc = 0, strideC = 0;
  double alpha = 1.0;
  int scale_mode = SCALE_NONE;
  const double *delta = nullptr;     // [K] pair gaps
  const double *batch_p0 = nullptr;  // [batch] omega (direct) or x_m (Laplace), device
  const double *batch_p1 = nullptr;  // [batch] w_m (Laplace), device
  int syrk = 0;
};
cudaError_t launch_gemm_f64(const GemmF64Args &g, int batch, bool a_kmaj, bool b_kmaj,
                            cudaStream_t s);

// W[b][t][m] = sum_P Bt[t][P][m] (C_b Bt[t])[P][m], C_b is N x N (K-major rows).
struct ColDotArgs {
  int N = 0, ncols = 0, n_tgt = 0;
  const double *C = nullptr; int64_t ldc = 0, strideC = 0;
  const double *Bt = nullptr; int64_t ldb = 0, strideBt = 0;
  double *W = nullptr; int64_t ldw = 0;
};
cudaError_t launch_gemm_coldot(const ColDotArgs &g, int n_batch, cudaStream_t s);

// ---- elementwise / small kernels (elementwise.cu) ----
// delta[i*n_virt + a] = eps[n_occ + a] - eps[n_frozen + i], i < n_occ - n_frozen
cudaError_t launch_pair_gaps(const double *eps, int n_occ, int n_virt, int n_frozen,
                             double *delta, cudaStream_t s);
// Pi_j = alpha * sum_k E[j][k] M_k over n elements per matrix
cudaError_t launch_recombine(const double *M, int n_tau, const double *E, int n_omega,
                             int64_t n_elem, double alpha, double *Pi, cudaStream_t s);
// dst[r][c] = src[r][c0 + c] for a strided 2-D copy of rows (batched)
cudaError_t launch_copy_cols(const double *src, int64_t lds, int64_t c0, double *dst,
                             int64_t ldd, int rows, int64_t cols, int batch,
                             int64_t strideS, int64_t strideD, cudaStream_t s);

// ---- screening (screen.cu) ----
// Sweep-operator inversion of I - Pi_j for n_omega matrices: writes
// C_j = (I - Pi_j)^-1 - I.  X0, X1: [n_omega][N][N] work buffers distinct from C.
cudaError_t launch_screen(const double *Pi, int N, int n_omega, double *X0, double *X1,
                          double *C, int *flags, cudaStream_t s, int *launches);

// ---- eigensolver (eig_f64.cu) ----
struct EigWork {
  double *A = nullptr;      // [n][n] symmetric in, destroyed
  double *V = nullptr;      // [n][n] Householder vectors (row k = v_k)
  double *d = nullptr, *e = nullptr, *tau = nullptr;  // [n]
  double *p = nullptr, *w = nullptr;                  // [n] symv / update vectors
  double *scal = nullptr;                             // [8]
  double *lam = nullptr;                              // [n] kept eigenvalues, descending
  double *X = nullptr;                                // [n][kcap] tridiagonal eigenvectors
  double *lu = nullptr;                               // [5 n kcap] inverse-iteration scratch
  int *count = nullptr;                               // [2]
};
// Tridiagonalise A, count eigenvalues > thresh (returned through count[0]).
cudaError_t launch_eig_tridiag(EigWork &w, int n, double thresh, cudaStream_t s, int *launches);
// Eigenvalues (descending) and eigenvectors for the k largest, Ut = rows [k][n].
cudaError_t launch_eig_vectors(EigWork &w, int n, int k, double *Ut, int *flags,
                               cudaStream_t s, int *launches);

// ---- self-energy, Pade and Newton (sigma_qp.cu) ----
struct SigmaArgs {
  int n_tgt = 0, n_omega = 0, n_orb = 0;   // n_orb: active orbitals in the m-sum
  const double *W = nullptr;               // [n_omega][n_tgt][n_orb]
  const double *eps_m = nullptr;           // [n_orb] active orbital energies
  const double *omega = nullptr, *weight = nullptr;  // [n_omega]
  double eps_F = 0.0;
  double *sigma = nullptr;                 // [n_tgt][n_omega][2]
};
cudaError_t launch_sigma(const SigmaArgs &a, cudaStream_t s);

struct QpArgs {
  int n_tgt = 0, n_omega = 0, pade_stride = 2;
  const double *sigma = nullptr;           // [n_tgt][n_omega][2]
  const double *omega = nullptr;           // [n_omega]
  const double *eps_n = nullptr;           // [n_tgt]
  const double *shift = nullptr;           // [n_tgt]
  double eps_F = 0.0, eta = 0.0, tol = 1e-12;
  int max_iter = 100;
  double *e_qp = nullptr;
  int *status = nullptr;
};
cudaError_t launch_qp(const QpArgs &a, cudaStream_t s);

}  // namespace ltgw
