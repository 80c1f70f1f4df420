/*
 * ltgw.h - C ABI of the GB300 (sm_103a) LT-GW G0W0 library.
 *
 * The library computes the imaginary-frequency G0W0 self-energy of the
 * analytic-continuation GW method accelerated by a Laplace transformation
 * (LT), natural auxiliary functions (NAF) and the frozen-core approximation,
 * as stated in Toelle, Niemeyer, Neugebauer, arXiv:2307.04508, Sec. 2:
 *
 *   W^c_nm(iw) = sum_PQ R^P_nm {[1 - Pi(iw)]^-1 - 1}_PQ R^Q_nm      (Eq. ScreenedCoulombOrbital)
 *   Pi_PQ(iw)  = -2 s sum_ia R^P_ia D_ia / (w^2 + D_ia^2) R^Q_ia      (Eq. Pi; D_ia = e_a - e_i)
 *   Pi_PQ(iw) ~= -2 s sum_m M^m_PQ exp(-w^2 x_m),
 *   M^m_PQ     = sum_ia R^P_ia w_m D_ia exp(-D_ia^2 x_m) R^Q_ia        (Eq. LT and the M^m form)
 *   Sigma^c_n(iw) = -(1/pi) sum_m int_0^inf dw' z/(z^2 + w'^2) W_nm(iw'),
 *                   z = iw + e_F - e_m                                 (Eq. CorrelationSelfEnergy)
 *   K_PQ = sum_ia R^P_ia R^Q_ia, U = eigenvectors of K above a threshold,
 *   R~ = R U                                                            (Eqs. nafeq, naftrafo)
 *
 * followed by an N-point Pade continuation (Vidberg & Serene 1977) and the
 * quasi-particle equation E = e_n + Re Sigma^c_n(E) + (Sigma_x - V_xc)_n.
 *
 * Conventions shared by every entry point:
 *  - All matrices are row-major float64.  The caller owns every buffer; the
 *    library never frees or keeps a caller pointer beyond the call.
 *  - "any" pointer: host (pageable or pinned) or device memory; the library
 *    detects which and stages host data itself.  "device" pointer: device
 *    memory on the context's device.
 *  - Work is issued on the given CUDA stream (cudaStream_t passed as void*;
 *    NULL = the legacy default stream).  Calls that return host-visible
 *    results synchronise that stream before returning.
 *  - Every call returns an ltgw_status; no exception or abort crosses the ABI.
 *    ltgw_last_error() gives a one-line description of the last failure.
 *  - A context is not thread-safe: one host thread at a time per context.
 *
 * Readings of points the paper leaves open (fixed once, shared with the tests):
 *  - closed-shell spatial orbitals: spin factor s (default 2) multiplies the
 *    -2 of Eq. Pi; the NAF metric sums active occupied-virtual pairs without a
 *    factor 2 and keeps eigenvalues strictly above the threshold;
 *  - frozen-core orbitals leave Pi, K and the m-sum of Sigma and cannot be targets;
 *  - e_F = (e_HOMO + e_LUMO)/2; eta = 0;
 *  - the Pade fraction passes through every second Gauss-Legendre node
 *    (indices 0, 2, 4, ...) in ascending order;
 *  - Newton from e_n, |dE| < 1e-12 Ha, at most 100 steps.
 */
#ifndef LTGW_H
#define LTGW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LTGW_OK = 0,
  LTGW_ERR_BAD_ARG = 1,     /* an argument is out of range or inconsistent          */
  LTGW_ERR_NOMEM = 2,       /* device or pinned-host allocation failed             */
  LTGW_ERR_NOT_SPD = 3,     /* a pivot of 1 - Pi(iw) was not positive              */
  LTGW_ERR_NO_CONVERGE = 4, /* a quasi-particle Newton solve did not converge      */
  LTGW_ERR_DEVICE = 5,      /* a CUDA call failed                                  */
  LTGW_ERR_EIG = 6,         /* the NAF eigensolver failed (non-finite or no vector) */
  LTGW_ERR_NO_NAF = 7,      /* the NAF threshold kept no auxiliary function        */
  LTGW_ERR_TIMEOUT = 8      /* a wait for completions ran out of time              */
} ltgw_status;

enum { LTGW_FP64 = 0, LTGW_BF16X3 = 1, LTGW_FP8 = 2, LTGW_FP8_PI = 3, LTGW_FP64_EMU = 4 };

typedef struct {
  int n_occ;          /* occupied orbitals, frozen core included                  */
  int n_virt;         /* virtual orbitals                                         */
  int n_frozen;       /* lowest occupied orbitals frozen (0 <= n_frozen < n_occ)  */
  int n_aux;          /* auxiliary functions                                      */
  int n_omega;        /* modified Gauss-Legendre points (2..256)                  */
  int n_tau;          /* Laplace / imaginary-time points, use_laplace != 0 (1..32) */
  double omega0;      /* GL map w = omega0 (1+x)/(1-x), Ha (> 0)                  */
  double naf_thresh;  /* < 0: no NAF; >= 0: keep eigenvalues of K above it        */
  int spin;           /* 1 (spin orbitals) or 2 (closed shell)                    */
  int use_laplace;    /* 0: Pi from Eq. Pi; 1: Pi from the Laplace moments M^m     */
                      /* (Eq. LT); 2: imaginary-time (cosine-transform) form,     */
                      /* moments with e^{-Delta tau_k} (ltgw_cosine_grid)         */
  int precision;      /* LTGW_FP64; LTGW_BF16X3: the dense contractions (NAF       */
                      /* metric, projections, Pi, W_nm) on the tensor cores with  */
                      /* split-BF16 operands (see ltgw_polarizability_mixed);     */
                      /* LTGW_FP8: the same with the Pi build and the W_nm        */
                      /* contraction in FP8 E4M3 with per-row scales and two-term */
                      /* expansions (rows are auxiliary functions;                */
                      /* ltgw_polarizability_fp8);                                */
                      /* LTGW_FP8_PI: FP8 for the Pi build only.                  */
                      /* LTGW_FP64_EMU: the FP64 form with the NAF metric, the    */
                      /* projections, Pi and W_nm FP64-accurate on the tensor     */
                      /* cores from 6 integer slices per operand row (see          */
                      /* ltgw_gemm_emulated); results as LTGW_FP64 to ~1e-12.      */
                      /* The eigensolver, screening, Pade and Newton stay FP64.   */
  int reserved;       /* must be 0                                                */
} ltgw_params;

typedef struct {
  int n_naf;                 /* auxiliary functions kept (n_aux without NAF)          */
  int n_pade;                /* points the Pade fraction passes through               */
  int n_tau;                 /* Laplace points used (0 in direct mode)                */
  int naf_near_threshold;    /* eigenvalues within 1e-12*lambda_max of the threshold  */
  double lt_max_rel_err;     /* max |X sum w e^{-X x} - 1| over the library grid's
                                interval (NaN when the caller supplied the grid)      */
  double ms_naf, ms_pi, ms_screen, ms_wnm, ms_sigma_qp, ms_total; /* last solve, device time */
  double ms_pi_kernel;       /* summed device time of the Pi-build kernel launches    */
  int pi_kernel_launches;    /* Pi-build kernel launches in the last solve            */
  int kernel_launches;       /* all kernel launches in the last solve                 */
  double ms_tridiag;         /* device time of the NAF Householder tridiagonalisation */
  double ms_generate;        /* host time spent in the block callback (streamed solve) */
  int tc_autotuned;          /* contraction shapes the autotuner has timed (this context) */
  double ms_naf_metric;      /* NAF stage parts (device time, ltgw_set_timing on): the */
  double ms_eig_vectors;     /* metric K (streamed: with the block arrivals), the      */
  double ms_naf_project;     /* eigenpairs after the tridiagonalisation (bisection,    */
                             /* inverse iteration, back-transformation), the projections */
} ltgw_stats;

typedef struct ltgw_ctx ltgw_ctx;

/* Create a context on CUDA device `device` (it becomes current on this thread).
 * The context owns a device workspace that grows to the largest solve seen. */
ltgw_status ltgw_create(ltgw_ctx **out, int device);
void ltgw_destroy(ltgw_ctx *ctx);
const char *ltgw_status_string(ltgw_status s);
const char *ltgw_last_error(const ltgw_ctx *ctx);

/* Turn per-stage CUDA-event timing on (1) or off (0); off by default. */
ltgw_status ltgw_set_timing(ltgw_ctx *ctx, int on);
/* Turn the contraction autotuner on (1) or off (0); off by default.  When on,
 * the first tensor-core contraction of a shape on this context times a few
 * configurations (scales per CTA, K-split count) on the caller's stream and
 * keeps the fastest for later calls with that shape; results then depend on
 * the choice only through FP32 summation order (within the form's
 * tolerance).  Off, every call takes the fixed heuristic and is
 * reproducible bit for bit. */
ltgw_status ltgw_set_autotune(ltgw_ctx *ctx, int on);
/* Device workspace a context holds between calls (it grows to the largest
 * call's need and is kept for the next call). */
size_t ltgw_workspace_bytes(const ltgw_ctx *ctx);
/* Free that workspace (no call of this context may be in flight); the next
 * call allocates again. */
ltgw_status ltgw_trim(ltgw_ctx *ctx);
ltgw_status ltgw_get_stats(const ltgw_ctx *ctx, ltgw_stats *out);

/*
 * One G0W0 solve: the whole path of Sec. 2 from orbital energies and RI
 * tensor blocks to Sigma^c_n(iw) and quasi-particle energies.
 *   eps      any [n_occ+n_virt]            orbital energies, ascending, Ha
 *   B_ov     any [n_aux][n_occ*n_virt]     R^P_ia, pair index i*n_virt+a, all occupied i
 *   B_tgt    any [n_tgt][n_aux][n_occ+n_virt]  R^P_nm for n = targets[t], all m
 *   targets  any [n_tgt]                   orbital indices, n_frozen <= n < n_occ+n_virt
 *   shift    any [n_tgt]                   (Sigma_x - V_xc)_n, Ha
 *   tau_x, tau_w  any [n_tau] or NULL      Laplace grid; NULL: the library fits a
 *                                          minimax grid on the paper's interval.
 *                                          use_laplace = 2: tau_x = tau [n_tau],
 *                                          tau_w = gamma [n_omega][n_tau]; NULL:
 *                                          ltgw_cosine_grid on [gap, span] of the
 *                                          active orbitals
 *   sigma_iw any [n_tgt][n_omega][2]       out: Sigma^c_n(i w_l) (re, im) at the GL nodes
 *   e_qp     any [n_tgt]                   out: quasi-particle energies, Ha
 *   qp_status any [n_tgt]                  out: 0 converged, 1 not
 * Returns LTGW_ERR_NO_CONVERGE (after writing every output) when a state did
 * not converge.  Synchronises `stream`.
 */
ltgw_status ltgw_solve(ltgw_ctx *ctx, const ltgw_params *p, const double *eps,
                       const double *B_ov, const double *B_tgt, const int *targets,
                       int n_tgt, const double *shift, const double *tau_x,
                       const double *tau_w, double *sigma_iw, double *e_qp,
                       int *qp_status, void *stream);

/*
 * Eigenvalue-self-consistent GW (evGW, Sec. 3 and the evGW timings of Sec. 4):
 * ltgw_solve's G0W0, then up to n_cycles further cycles that rebuild Pi, W and
 * Sigma from the previous cycle's quasi-particle energies for the target
 * states and, for every other active orbital, its input energy shifted by the
 * shift (E_QP - eps) of the target nearest to it by orbital index (below and
 * above the window: the lowest and the highest target's shift; frozen core
 * unchanged).  The NAF basis and the projected tensors are formed once; the
 * library's Laplace grid (when tau_x is NULL) is refitted to each cycle's
 * energies.  The quasi-particle equation keeps the input eps_n +
 * (Sigma_x - V_xc)_n as its reference.  Stops early once the quasi-particle
 * HOMO/LUMO gap changes by less than gap_tol (> 0; both states among the
 * targets).  Outputs are those of the last cycle; cycles_done (may be NULL):
 * the cycles run after G0W0.  Other arguments as ltgw_solve.
 */
ltgw_status ltgw_solve_ev(ltgw_ctx *ctx, const ltgw_params *p, const double *eps,
                          const double *B_ov, const double *B_tgt, const int *targets,
                          int n_tgt, const double *shift, const double *tau_x,
                          const double *tau_w, int n_cycles, double gap_tol,
                          double *sigma_iw, double *e_qp, int *qp_status, int *cycles_done,
                          void *stream);

/*
 * The same solve without the occupied-virtual block resident: the caller
 * supplies the RI tensor one block of occupied orbitals at a time.
 *   fill(user, i0, i1, dst, fill_stream) writes R^P_ia for active occupied
 *   orbitals i0 <= i < i1 (n_frozen <= i0 < i1 <= n_occ) into the device
 *   buffer dst [n_aux][(i1-i0)*n_virt] (pair index (i-i0)*n_virt + a), with
 *   its work complete, or issued on fill_stream (a library stream), when it
 *   returns 0; any other return value aborts the solve (LTGW_ERR_BAD_ARG).
 *   dst is free when fill is called (the library has waited for the work
 *   that read it), so fill may write it by any means.  The library keeps two
 *   block buffers: work that fill issues on fill_stream overlaps the
 *   library's work on the previous block, which runs on `stream`.
 * Blocks hold occ_block orbitals (the last may hold fewer) and are requested
 * in ascending order for the NAF metric K = sum over blocks of B B^T
 * (Eq. nafeq).  The tensor-core forms keep each block, transposed and split
 * into BF16 hi / lo (4 bytes per value, n_aux * n_act * n_virt values in
 * all), as the operand of the projection R~ = U^T R (Eq. naftrafo), so they
 * request every block once; the FP64 form requests every block a second time
 * for the projection (the tensor is never resident in FP64).
 * Needs NAF (naf_thresh >= 0).  Other arguments and outputs as for
 * ltgw_solve.  Synchronises `stream` (and fill_stream).
 */
typedef int (*ltgw_block_fn)(void *user, int i0, int i1, double *dst, void *stream);
ltgw_status ltgw_solve_streamed(ltgw_ctx *ctx, const ltgw_params *p, const double *eps,
                                ltgw_block_fn fill, void *user, int occ_block,
                                const double *B_tgt, const int *targets, int n_tgt,
                                const double *shift, const double *tau_x, const double *tau_w,
                                double *sigma_iw, double *e_qp, int *qp_status, void *stream);

/* ---- grids (host only, no context) ------------------------------------- */

/* Modified Gauss-Legendre rule on [0, inf) (Sec. 2 after Eq.
 * CorrelationSelfEnergy): Legendre nodes mapped by w = omega0 (1+x)/(1-x),
 * weights g = w_GL * 2 omega0 / (1-x)^2, ascending.  omega, weight: host [n]. */
ltgw_status ltgw_gl_grid(int n, double omega0, double *omega, double *weight);

/* Minimax Laplace grid (Sec. 3: bounds and epsilon_LT): x_m, w_m (host [n_tau])
 * with 1/X ~ sum_m w_m exp(-X x_m) on [a, b], fitted by a Remez exchange
 * on the relative error.  *max_rel_err receives max |X sum w e^{-X x} - 1|. */
ltgw_status ltgw_laplace_grid(int n_tau, double a, double b, double *x, double *w,
                              double *max_rel_err);

/* Imaginary-time (cosine-transform) grid, the alternative to Eq. LT's
 * factorisation: Delta / (w^2 + Delta^2) = int_0^inf cos(w tau) e^{-Delta tau} dtau
 * ~ sum_k gamma[j][k] e^{-Delta tau_k} for Delta in [dmin, dmax] and each of the
 * n_omega frequencies.  tau (n_tau): geometric from 0.1/dmax to 8/dmin;
 * gamma ([n_omega][n_tau]): per frequency, the least-squares fit over log-spaced
 * Delta of the error scaled by the target's largest value on [dmin, dmax], plus
 * ridge times the squared coefficients of unit-norm columns (a small ridge
 * trades fit error for less cancellation among the coefficients).  max_err: the
 * largest such scaled error over the frequencies on a finer sample;
 * amplification (may be NULL): the largest sum_k |gamma_jk| e^{-Delta tau_k} over
 * the target's largest value, the factor by which the recombination can
 * magnify relative errors of the moments.  Solves use ridge 1e-14 in FP64 and
 * 1e-10 in the tensor-core forms.  Host only. */
ltgw_status ltgw_cosine_grid(int n_tau, double dmin, double dmax, int n_omega, const double *omegas,
                             double ridge, double *tau, double *gamma, double *max_err,
                             double *amplification);

/* ---- single steps on device buffers (for checking and composition) ------ */

/* NAF basis (Eqs. nafeq and NAF eigen-equation): K = B B^T over the n_pairs
 * columns of B (device [n_aux][ld], ld >= n_pairs), eigenpairs of K, and the
 * eigenvectors with eigenvalue > thresh written as the rows of Ut (device
 * [n_aux][n_aux] capacity; rows 0..n_naf-1 used, descending eigenvalue).
 * lambda: device [n_aux] capacity, kept eigenvalues, descending.  Synchronises. */
ltgw_status ltgw_naf_basis(ltgw_ctx *ctx, int n_aux, int64_t n_pairs, const double *B,
                           int64_t ld, double thresh, double *Ut, double *lambda,
                           int *n_naf, void *stream);

/* The same NAF basis as LTGW_BF16X3 solves form it: K on the tensor cores
 * with split-BF16 operands (as ltgw_polarizability_mixed, unit scale), then
 * the same FP64 eigensolver as ltgw_naf_basis.  K carries a relative error of
 * about 1e-6, so the eigenvalues carry about 1e-6 * lambda_max.  Same
 * arguments, layouts and errors as ltgw_naf_basis. */
ltgw_status ltgw_naf_basis_mixed(ltgw_ctx *ctx, int n_aux, int64_t n_pairs, const double *B,
                                 int64_t ld, double thresh, double *Ut, double *lambda,
                                 int *n_naf, void *stream);

/* Polarisability at the GL frequencies `omegas` (host [n_omega]) from the
 * pair block Bt (device [N][n_pairs]) and gaps delta (device [n_pairs]):
 * n_tau == 0 evaluates Eq. Pi directly, n_tau > 0 the Laplace form with the
 * host grid (x, w).  Pi: device [n_omega][N][N], full symmetric.  Stream-ordered. */
ltgw_status ltgw_polarizability(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                const double *delta, int n_omega, const double *omegas,
                                int n_tau, const double *x, const double *w, int spin,
                                double *Pi, void *stream);

/* The same polarisability in the mixed-precision form: every product of the
 * pair sum runs on the tensor cores with BF16 hi/lo split operands
 * (x = bf16(x) + bf16(x - bf16(x)); hi*hi + hi*lo + lo*hi), the per-pair scale
 * applied while the operands are loaded, FP32 accumulation drained to FP64
 * every 2048 pairs (each MMA's FP32 rounding biases sums of one sign by about
 * half an ulp, so the drain length bounds the drift).  Same arguments and
 * layout as ltgw_polarizability; relative error about 1e-5.  Synchronises. */
ltgw_status ltgw_polarizability_mixed(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                      const double *delta, int n_omega, const double *omegas,
                                      int n_tau, const double *x, const double *w, int spin,
                                      double *Pi, void *stream);

/* Pi in the imaginary-time (cosine-transform) form, the alternative to Eq. LT's
 * factorisation (Delta / (w^2 + Delta^2) = int_0^inf cos(w tau) e^{-Delta tau} dtau):
 * M^k = R~ diag(e^{-Delta tau_k}) R~^T for the n_tau points tau (host) and
 * Pi_j = -2 spin sum_k gamma[j][k] M^k (gamma host [n_omega][n_tau], e.g. from
 * ltgw_cosine_grid).  precision: LTGW_FP64, LTGW_BF16X3 (split BF16) or
 * LTGW_FP8 / LTGW_FP8_PI (FP8 E4M3); other arguments as ltgw_polarizability.
 * Synchronises. */
ltgw_status ltgw_polarizability_tau(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                    const double *delta, int n_omega, const double *omegas,
                                    int n_tau, const double *tau, const double *gamma, int spin,
                                    int precision, double *Pi, void *stream);

/* The same polarisability in FP8 E4M3 (not a step of the paper: the
 * low-precision variant of its Pi contraction).  R~ is rounded to FP32, the
 * per-pair factors of Eq. Pi (or of the M^m form) are formed in FP64 and
 * rounded to FP32, and every row of R~ and of each R~ diag(factor) (FP32
 * products) is scaled so that its largest magnitude maps to 448, the largest
 * finite E4M3 value; each scaled value xs is written as the two-term E4M3
 * expansion h + l, h = e4m3(xs), l = e4m3(xs - h) (nearest even, saturating;
 * both in the row's scaled units).  The products h_a h_b + l_a h_b + h_a l_b
 * are summed on the tensor cores (kind::f8f6f4, over three segments of codes)
 * in FP32, drained every 4096 codes, de-scaled per row and summed over
 * K-splits in FP64; each Pi_j (or M^m) is formed on its lower triangle and
 * mirrored.  Relative error against the exact Pi about 1e-4 (a single E4M3
 * term keeps 3 mantissa bits and gives about 4e-3, and 1 meV errors in the
 * quasi-particle energies).  Same arguments and layout as
 * ltgw_polarizability.  Synchronises. */
ltgw_status ltgw_polarizability_fp8(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                    const double *delta, int n_omega, const double *omegas,
                                    int n_tau, const double *x, const double *w, int spin,
                                    double *Pi, void *stream);

/* The polarisability of ltgw_polarizability (Eq. Pi, or with n_tau > 0 the
 * M^m form of Eq. LT) with every contraction FP64-accurate on the tensor
 * cores (not a step of the paper: the FP64 form at tensor-core speed).  Per
 * frequency or Laplace point t the FP64 factors f_t (Delta / (w_t^2 +
 * Delta^2), or w_t Delta exp(-Delta^2 x_t); each operation rounded once)
 * scale R~'s columns (one FP64 product per entry), and M_t = (R~ diag(f_t))
 * R~^T is formed as in ltgw_gemm_emulated with n_slices slices (lower tiles,
 * mirrored; pairs in equal chunks of at most 131072, each sliced on its own, their products
 * added); the direct form writes Pi_j = -2 s M_j, the Laplace form
 * recombines -2 s sum_m exp(-w_j^2 x_m) M^m in FP64.  Relative error about
 * 2^(-7 n_slices) of the largest row products (n_slices = 6: about 1e-12 in
 * Frobenius norm, the FP64 form's results to 1e-8 Ha in the quasi-particle
 * energies).  n_slices in [2, 8]; other arguments, layout and errors as
 * ltgw_polarizability.  Synchronises. */
ltgw_status ltgw_polarizability_emulated(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                         const double *delta, int n_omega, const double *omegas,
                                         int n_tau, const double *x, const double *w, int spin,
                                         int n_slices, double *Pi, void *stream);

/* Screening (Eq. ScreenedCoulombOrbital): C_j = [1 - Pi_j]^-1 - 1 for each of
 * n_omega matrices (device [n_omega][N][N] in and out, may not alias).
 * Synchronises; LTGW_ERR_NOT_SPD if a pivot was not positive. */
ltgw_status ltgw_screen(ltgw_ctx *ctx, int N, int n_omega, const double *Pi, double *C,
                        void *stream);

/* FP64-accurate product C = A B^T on the tensor cores (not a step of the
 * paper: an emulation of FP64 contractions with exact small-integer products).
 * Each row r of A (and of B) is written in fixed point relative to e_r, the
 * exponent of the row's largest magnitude (max|X_r| < 2^e_r):
 * Q = rint(X_r 2^(7 s - e_r)) (ties to even), in s balanced base-128 digits
 * a_1 .. a_s (|a_1| <= 128, |a_i| <= 64 after it); then
 * C = sum over digit pairs with i + j <= s + 1 of 2^(-7(i+j)) a_i b_j^T,
 * times 2^(e_A + e_B).  Every pair's integer products are exact in BF16 and
 * summed exactly (FP32 sums below 2^24 per drain, FP64 after), so the only
 * errors are the dropped digits: about 2^(-7s) of the rows' largest
 * magnitudes (s = 6: about 1e-12 relative Frobenius on products of Gaussian
 * rows).  A [m][lda], B [n][ldb] (k columns used), C [m][ldc]: device, row
 * major; sym: B = A, only the lower tiles are computed and C (ldc = n) is
 * written whole, symmetric.  m <= 65535; n_slices in [2, 8].  A and B must be finite
 * (NaN or Inf give undefined values in C, no error).  A, B are read only and
 * stay the caller's; the slices and partial tiles live in the context's
 * scratch (LTGW_ERR_NOMEM if they do not fit).  Synchronises. */
ltgw_status ltgw_gemm_emulated(ltgw_ctx *ctx, int m, int n, int64_t k, const double *A, int64_t lda,
                               const double *B, int64_t ldb, double *C, int64_t ldc, int sym, int n_slices,
                               void *stream);

/* ---- request server (continuous admission of solves) -------------------- */

/* One G0W0 request: the arguments of ltgw_solve.  Every pointer must stay valid
 * (and outputs unread) until the request's completion has been polled. */
typedef struct {
  ltgw_params p;
  const double *eps, *B_ov, *B_tgt;   /* any; layouts as for ltgw_solve        */
  const int *targets;
  int n_tgt;
  const double *shift, *tau_x, *tau_w;
  double *sigma_iw, *e_qp;            /* outputs, any                          */
  int *qp_status;
} ltgw_request;

typedef struct {
  uint64_t ticket;      /* from ltgw_server_submit                              */
  ltgw_status status;   /* what ltgw_solve returned for the request             */
  double queue_ms;      /* submit -> start of service                           */
  double service_ms;    /* start of service -> results written                  */
  double latency_ms;    /* submit -> results written                            */
  double start_ms;      /* start of service, ms since the server was created    */
  double end_ms;        /* results written, ms since the server was created     */
  char message[120];    /* ltgw_last_error of the solve ("" when status is OK)  */
} ltgw_completion;

typedef struct ltgw_server ltgw_server;

/* A server with n_slots workers on `device`, each with its own context and
 * non-blocking stream (requests in different slots overlap on the device).
 * A request is admitted when a slot is free and the sum of the estimated
 * footprints of the running requests, with its own, stays within
 * hbm_budget_bytes: the oldest that fits first.  A request that does not fit
 * may be passed by later ones that do at most 8 times; after that nothing is
 * admitted ahead of it.  A request whose solve runs out of device memory
 * while others run goes back to the head of the queue with its estimate
 * doubled (at the full budget it runs alone); one that runs out of memory
 * alone is re-run alone once after the idle slots released their workspace,
 * and fails (LTGW_ERR_NOMEM) if it runs out again.  Each slot keeps up to a
 * quarter of the budget, shared among the slots, of workspace between
 * requests; that retained workspace counts against admission. */
ltgw_status ltgw_server_create(ltgw_server **out, int device, int n_slots, size_t hbm_budget_bytes);
/* Queue a request (never blocks on the GPU); LTGW_ERR_NOMEM if its estimated
 * footprint alone exceeds the budget. */
ltgw_status ltgw_server_submit(ltgw_server *srv, const ltgw_request *req, uint64_t *ticket);
/* Move up to max_out completions (oldest first) into out; returns how many. */
int ltgw_server_poll(ltgw_server *srv, ltgw_completion *out, int max_out);
/* Wait until nothing is queued or running; LTGW_ERR_TIMEOUT after timeout_s. */
ltgw_status ltgw_server_wait_all(ltgw_server *srv, double timeout_s);
/* Finish the running requests, drop the queued ones, release everything. */
void ltgw_server_destroy(ltgw_server *srv);
/* Estimated device bytes of one solve (inputs staged + workspace, tensor-core
 * partial tiles included; with NAF the post-NAF size is taken as n_aux / 2). */
size_t ltgw_request_footprint(const ltgw_params *p, int n_tgt);

/* ---- allocation-free screening ------------------------------------------ */

/* Largest n_omega * N * N accepted by ltgw_screen_static. */
#define LTGW_SCREEN_STATIC_MAX_ELEMS (1u << 19)

/* The paper has no counterpart to this entry point.  It computes the same
 * C_j = [1 - Pi_j]^-1 - 1 as ltgw_screen, for callers that cannot allocate
 * device memory when they call: a process whose device memory is already
 * claimed in full by another allocator (a framework's caching allocator or a
 * pre-reserved pool), or a latency-sensitive caller that cannot afford
 * cudaMalloc/cudaFree, which may block and synchronise the device.  It needs
 * no context and calls no allocating routine: its scratch (two sweep buffers
 * of LTGW_SCREEN_STATIC_MAX_ELEMS doubles, 4 MiB each, and an error flag) is a
 * fixed device array that every GPU loading the library holds until the
 * process exits.
 *   N, n_omega  matrix size and count, n_omega * N * N <= LTGW_SCREEN_STATIC_MAX_ELEMS;
 *               larger sizes return LTGW_ERR_BAD_ARG before any GPU work
 *   Pi, C       device [n_omega][N][N] on the current device, distinct
 * Runs on `stream` and synchronises it; LTGW_ERR_NOT_SPD if a pivot was not
 * positive.  A call looks up the array's device address (cudaGetSymbolAddress)
 * on the current device each time it runs outside stream capture, so a device
 * reset between calls is harmless; a call on a capturing stream reuses the
 * address found by an earlier call on that device, so make one call on each
 * device before any stream capture.  All calls share the one array per device,
 * so calls that overlap on the GPU (other streams, other host threads) race. */
ltgw_status ltgw_screen_static(int N, int n_omega, const double *Pi, double *C, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LTGW_H */
