// Launch interfaces of the LT-GW kernels (host side).  Every launcher issues
// its kernels on the given stream and returns the launch status; none of them
// synchronises.
#pragma once

#include <cuda_bf16.h>

#include <cuda_runtime.h>
#include <stdint.h>

namespace ltgw {

// per-pair factor of Pi's contraction: Delta / (w^2 + Delta^2) (Eq. Pi), w_m Delta
// e^{-Delta^2 x_m} (the M^m form of Eq. LT), or e^{-Delta tau_k} (imaginary-time form)
enum ScaleMode { SCALE_NONE = 0, SCALE_DIRECT = 1, SCALE_LAPLACE = 2, SCALE_EXPTAU = 3 };

// C_b = alpha * A_b diag(s_b) B_b for b in [0, batch).  With syrk = 1 only the
// lower-triangle tiles are computed and each value is mirrored (A == B^T).
template <typename T>
struct GemmArgs {
  int M = 0, N = 0;
  int64_t K = 0;
  const T *A = nullptr; int64_t lda = 0, strideA = 0;
  const T *B = nullptr; int64_t ldb = 0, strideB = 0;
  T *C = nullptr; int64_t ldc = 0, strideC = 0;
  double alpha = 1.0;
  int scale_mode = SCALE_NONE;       // FP64 only
  const double *delta = nullptr;     // [K] pair gaps
  const double *batch_p0 = nullptr;  // [batch] omega (direct) or x_m (Laplace), device
  const double *batch_p1 = nullptr;  // [batch] w_m (Laplace), device
  int syrk = 0;
  double beta = 0.0;      // C = alpha * acc + beta * C
  int64_t ksplit = 0;     // > 0: batch index b covers k in [b*ksplit, (b+1)*ksplit), C_b at b*strideC
};
using GemmF64Args = GemmArgs<double>;
// Tiled GEMM / SYRK on the CUDA cores (instantiated in FP64).
template <typename T>
cudaError_t launch_gemm(const GemmArgs<T> &g, int batch, bool a_kmaj, bool b_kmaj, cudaStream_t s);
inline cudaError_t launch_gemm_f64(const GemmF64Args &g, int batch, bool a_kmaj, bool b_kmaj, cudaStream_t s) {
  return launch_gemm<double>(g, batch, a_kmaj, b_kmaj, s);
}
// Every reflector panel's Gram block in one launch: panel q = rows q*nb ..
// of V (n x n, row j zero outside columns j+1..n-1, nb <= 64), chunk c of its
// columns from q*nb + 1 on (ks wide) into P + (c * npanel + q) * nb * nb
// (ld = the panel's row count; zeros past the panel's end), npanel =
// ceil(nref / nb), ceil((n - 1) / ks) chunks.
cudaError_t launch_gram_panels(const double *V, int n, int nref, int nb, int64_t ks, double *P, cudaStream_t s);

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
// Pi_j = alpha * sum_k E[j][k] M_k over n elements per matrix (n_tau <= 32, any n_omega);
// fp32: FP32 arithmetic (FP64 in and out), for moments of the tensor-core forms
cudaError_t launch_recombine(const double *M, int n_tau, const double *E, int n_omega,
                             int64_t n_elem, double alpha, double *Pi, cudaStream_t s, bool fp32 = false);
// dst[r][c] = src[r][c0 + c] for a strided 2-D copy of rows (batched)
cudaError_t launch_copy_cols(const double *src, int64_t lds, int64_t c0, double *dst,
                             int64_t ldd, int rows, int64_t cols, int batch,
                             int64_t strideS, int64_t strideD, cudaStream_t s);

// ---- screening (screen.cu) ----
// Sweep-operator inversion of I - Pi_j for n_omega matrices: writes
// C_j = (I - Pi_j)^-1 - I.  X0, X1: [n_omega][N][N] work buffers distinct from C.
cudaError_t launch_screen(const double *Pi, int N, int n_omega, double *X0, double *X1,
                          double *C, int *flags, cudaStream_t s, int *launches);

// Blocked form: work = screen_blocked_scratch(N, n_omega) doubles.
size_t screen_blocked_scratch(int N, int n_omega);
cudaError_t launch_screen_blocked(const double *Pi, int N, int n_omega, double *work, double *C, int *flags,
                                  cudaStream_t s, int *launches);

// ---- eigensolver (eig.cu) ----
struct EigWork {
  double *A = nullptr;      // [n][n] symmetric in, destroyed
  double *V = nullptr;      // [n + 64][n] Householder vectors (row k = v_k; rows >= n-2 zero)
  double *d = nullptr, *e = nullptr, *tau = nullptr;  // [n]
  double *p = nullptr, *w = nullptr;                  // [n] symv / update vectors
  double *scal = nullptr;                             // [8]
  double *lam = nullptr;                              // [n] kept eigenvalues, descending
  double *X = nullptr;                                // [n][kcap] tridiagonal eigenvectors
  double *lu = nullptr;                               // [5 n kcap] inverse-iteration scratch
  int *count = nullptr;                               // [2]
  double *wy = nullptr;                               // [WY scratch] see eig.cu
  int64_t wy_r0 = 0;                                  // doubles of wy's first region (W1 scratch)
  double *grid_ws = nullptr;                          // [4 n + 2 n_sm + 8] fused-reduction scratch
  int *flags = nullptr;                               // device error flags
};
// Tridiagonalise A, count eigenvalues > thresh (returned through count[0]).
// V must be zeroed by the caller before the call.
cudaError_t launch_eig_tridiag(EigWork &w, int n, double thresh, cudaStream_t s, int *launches);
// Eigenvalues (descending) and eigenvectors for the k largest, Ut = rows [k][n].
cudaError_t launch_eig_vectors(EigWork &w, int n, int k, double *Ut, int *flags,
                               cudaStream_t s, int *launches);

// ---- split-BF16 tensor-core contraction (tc_gemm.cu) ----
// D_t = A diag(s_t) B^T for t < n_t; A [*][Kp] FP32, B pre-split, scale [n_t][Kp] FP32,
// zero-padded (rows of A and B to 128, Kp to 64).  tiles: device list of
// (tile row of A, tile row of B) pairs.  Output: FP64 partial tiles
// partial[split][group][nt_group][tile][128][128], group = t / nt_group.
enum TcOut { TC_OUT_F64 = 0, TC_OUT_F32 = 1, TC_OUT_COLDOT = 2 };
struct TcGemmArgs {
  const float *A = nullptr, *B = nullptr, *scale = nullptr;
  int64_t Kp = 0;
  int n_t = 0;
  int nt_group = 4;              // scales per CTA (1..4); group = blockIdx.y
  int64_t a_group_stride = 0;    // A of group g starts at A + g * a_group_stride
  const int *tiles = nullptr;
  int64_t k_begin = 0, k_end = 0;   // the pair range [k_begin, k_end) contracted (k_end 0: Kp)
  int64_t k_per_split = 0;
  int64_t drain_k = 2048;        // pairs per FP32 accumulation (bounds its rounding bias)
  int out_mode = TC_OUT_F64;     // F32 requires k_per_split <= drain_k
  int out_colmajor = 0;          // F64 / F32 partial tiles stored [col][row] (coalesced drains)
  double *partial = nullptr;     // TC_OUT_F64
  float *partial32 = nullptr;    // TC_OUT_F32
  // TC_OUT_COLDOT (nt_group = 1): out[split][group][tile row][col] =
  //   sum over the 128 tile rows r of D[r][col] * cd_B[col][r] (cd_B row-major, ld cd_ld)
  const double *cd_B = nullptr;
  int64_t cd_ld = 0;
  int cd_rows = 0, cd_cols = 0;  // valid extent of cd_B's transpose (rows = D rows)
  int n_tile_rows = 0, cd_cols_p = 0;
  float *cd_out = nullptr;
  int *err = nullptr;
  // B pre-split (BF16 hi and lo, row-major [rows_b][Kp]; required): the
  // kernel keeps A in tensor memory and brings the operands in by tiled bulk
  // copies (nt_group <= 2; A groups only stacked, a_group_stride = rows_a Kp,
  // with nt_group = 1).
  const __nv_bfloat16 *B_hi = nullptr, *B_lo = nullptr;
  int64_t rows_a = 0, rows_b = 0;   // padded row counts of A and B (tensor-map extents)
  // single: B is exact in BF16 (B_lo not given) and so is every A value (its
  // lo part is zero): one product per step, A_hi B_hi (integer digit operands)
  int single = 0;
  // FP8 E4M3 form (launch_tc_fp8_gemm): codes qa [n_t][rows_a][Kp], qb [rows_b][Kp] and
  // per-row de-scales ds_a [n_t][rows_a], ds_b [rows_b], applied in the epilogue.
  const uint8_t *A8 = nullptr, *B8 = nullptr;
  const float *ds_a = nullptr, *ds_b = nullptr;
  int groups_fastest = 0;   // set by the launcher: grid order (groups, tiles, splits)
};
cudaError_t launch_tc_split_gemm(const TcGemmArgs &g, int n_tiles, cudaStream_t s);
// hi = bf16(x), lo = bf16(x - hi) elementwise: the split the tensor-core kernels use.
cudaError_t launch_split_bf16(const float *x, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t n, cudaStream_t s);
// FP8 E4M3 operands with per-row scales (mixed.cu): for each row r of X [rows][Kp] (FP32),
// inv = 448 / max|X_r|, qb[r][k] = e4m3(X_rk inv); for each factor row S[t] ([n_t][Kp])
// the FP32 products X_rk S_tk get their own row scale, codes qa[t][r][k].  De-scales
// (1 / inv, 0 for zero rows) in ds_b[r], ds_a[t][r]; code columns Kp..Kq-1 are zero.
// split: rows of 3 Kq codes, the two-term expansion h = e4m3(x inv), l = e4m3(x inv - h)
// in segments h | l | h (A operands) and h | h | l (B operands), so that a contraction
// over the 3 Kq codes sums h_a h_b + l_a h_b + h_a l_b.
cudaError_t launch_fp8_quantize(const float *X, int64_t Kp, int64_t Kq, const float *S, int n_t, int rows,
                                uint8_t *qa, uint8_t *qb, float *ds_a, float *ds_b, cudaStream_t s, int split);
// Rows of X (FP64 [rows][ld], `cols` used; with colscale, X_rk colscale_k as one
// FP64 product) as s balanced base-128 digits of their fixed-point form
// rint(X_r 2^(7 s - e_r)), e_r the exponent of the row's largest magnitude
// (m < 2^e_r): digit i to dA / dB [i][r][Kp] (FP32 / BF16, either may be null; zero
// past cols), e_r to exps[r].  The FP64-accurate product of two sliced operands sums
// 2^(-7(i+j)) (a_i b_j^T) 2^(e_A + e_B) over i + j <= s + 1.
cudaError_t launch_slice_rows(const double *X, int64_t ld, int rows, int64_t cols, int64_t Kp, int s,
                              int64_t slice_stride, float *dA, __nv_bfloat16 *dB, int *exps, cudaStream_t st,
                              const double *colscale = nullptr);
// FP64 factors f[t][k] (k < K) of the Pi contraction per frequency (SCALE_DIRECT,
// p0 = omega), Laplace point (SCALE_LAPLACE, p0 = x, p1 = w) or imaginary-time
// node (SCALE_EXPTAU, p0 = tau), no fused operations.
cudaError_t launch_pi_factor64(const double *delta, int64_t K, int n_t, const double *p0, const double *p1,
                               int mode, double *f, cudaStream_t st);
// D[r][c] = beta D[r][c] + S[r][c] 2^(ea[r] + eb[c]) (rows <= 65535); lower (rows ==
// cols, S symmetric): the entries c <= r scaled, each written to (r, c) and (c, r).
cudaError_t launch_scale_exp2_to(const double *S, int64_t lds, double *D, int64_t ldd, int rows, int cols,
                                 const int *ea, const int *eb, double beta, cudaStream_t st, int lower = 0);
// The slices of X's columns 0..cols-1 as operand rows (X FP64 [rows][ld], the
// contraction index is X's row): digit i of column c to dB[i][c][k] (BF16), its
// exponent to exps[c]; as launch_slice_rows applied to X^T.
cudaError_t launch_slice_cols(const double *X, int64_t ld, int rows, int cols, int64_t Kp, int s,
                              int64_t slice_stride, __nv_bfloat16 *dB, int *exps, cudaStream_t st);
// W[t][c] = sum_r Y[r][t ncols + c] Bt[t][r][c] in FP64 (Bt [n_tgt] x [N][ldb]).
cudaError_t launch_coldot64(const double *Y, int64_t ldy, const double *Bt, int64_t ldb, int64_t strideB, int N,
                            int ncols, int n_tgt, double *W, int64_t ldw, cudaStream_t st);
// X itself quantised per row as an A operand (split: segments h | l | h).
cudaError_t launch_fp8_quantize_a(const float *X, int64_t Kp, int64_t Kq, int rows, uint8_t *q, float *ds,
                                  cudaStream_t s, int split);
// Scaled contraction on FP8 E4M3 codes (tcgen05 kind::f8f6f4): D_t = diag(ds_a[t]) qa[t] qb^T diag(ds_b),
// up to four scales per CTA (nt_group <= 4), Kp (of the codes) and k_per_split multiples of 128;
// partial tiles as launch_tc_split_gemm (column-major).
cudaError_t launch_tc_fp8_gemm(const TcGemmArgs &g, int n_tiles, cudaStream_t s);
size_t tc_gemm_smem_bytes();

// ---- mixed-precision helpers (mixed.cu) ----
// dst[c][r] = (float)src[r][c0 + c] for r < rows, c < cols; zero up to cols_p x rows_p
// (batched over `batch` with strides in elements).
cudaError_t launch_to_f32_transposed(const double *src, int64_t lds, int64_t c0, int rows, int cols,
                                     float *dst, int rows_p, int cols_p, int batch, int64_t strideS,
                                     int64_t strideD, cudaStream_t s);
// out[r][c] = alpha * sum over splits of full-grid partial tiles (tile = I * nJ + J, one
// scale per group: nt_group = 1) for
// r < rows, c < cols; FP64 to out64 (ld ld64) and/or FP32 to out32 (ld ld32; columns
// up to cols32 (default ld32) and rows up to rows_p32 are written, zero beyond the
// data), per group g (strides in elements).
cudaError_t launch_tc_reduce_full(const double *partial, const float *partial32, int splits, int groups,
                                  int n_tiles, int nJ, int rows, int cols, double alpha, double *out64,
                                  int64_t ld64, int64_t stride64, float *out32, int64_t ld32,
                                  int rows_p32, int64_t stride32, cudaStream_t s, int64_t cols32 = -1,
                                  double beta = 0.0);
// out64[r][c] = alpha * (sum of the partials) + beta * out64[r][c], one group.
cudaError_t launch_tc_reduce_full_acc(const double *partial, const float *partial32, int splits, int groups,
                                      int n_tiles, int nJ, int rows, int cols, double alpha, double *out64,
                                      int64_t ld64, double beta, cudaStream_t s);
// W[g][c] = sum over splits and tile rows of cd_out[split][g][I][c], c < cols.
cudaError_t launch_tc_reduce_coldot(const float *cd_out, int splits, int groups, int n_tile_rows,
                                    int cols_p, int cols, double *W, int64_t ldw, cudaStream_t s);
// dst[r][c] = (float)src[r][c] for r < rows, c < cols; zero up to rows_p x cols_p.
cudaError_t launch_to_f32_padded(const double *src, int64_t lds, int rows, int64_t cols, float *dst,
                                 int rows_p, int64_t cols_p, cudaStream_t s);
// scale[t][k] (FP32, zero for k >= K): direct w_t -> D/(w^2+D^2); Laplace (x_t, w_t) -> w D e^{-D^2 x};
// imaginary time tau_t -> e^{-D tau}.
cudaError_t launch_scale_table(const double *delta, int64_t K, int64_t Kp, int n_t, const double *p0,
                               const double *p1, int mode, float *scale, cudaStream_t s);
// M_t = alpha * sum over splits of the partial tiles (FP64 or FP32), full symmetric
// [n_t][N][N] FP64, for a lower tile list (tile_index [nI][nJ]); nt_group scales per
// group; colmajor: partial tiles stored [col][row].
cudaError_t launch_tc_reduce_sym(const double *partial, const float *partial32, int splits, int groups,
                                 int n_tiles, const int *tile_index, int nJ, int n_t, int N, double alpha,
                                 double *M, cudaStream_t s, double beta, int nt_group, int colmajor);
// dst[c][r] = src[r][c0 + c] in FP64 (batched)
cudaError_t launch_transpose_f64(const double *src, int64_t lds, int64_t c0, int rows, int cols, double *dst,
                                 int64_t ldd, int batch, int64_t strideS, int64_t strideD, cudaStream_t s);

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
