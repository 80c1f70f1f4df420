// FP64 symmetric eigensolver for the natural auxiliary functions (Sec. 2:
// diagonalise K, keep the eigenvectors whose eigenvalue exceeds eps_NAF).
//
//  1. Householder reduction K = Q T Q^T to tridiagonal T (one reflector per
//     step: reflector, symmetric mat-vec, rank-2 update of the trailing block);
//  2. Sturm-sequence count of the eigenvalues of T above the threshold;
//  3. multisection for the kept eigenvalues, one warp each, with T in shared memory;
//  4. inverse iteration for their eigenvectors (tridiagonal LU with row
//     interchanges), with modified Gram-Schmidt inside groups of nearly equal
//     eigenvalues;
//  5. symmetric re-orthonormalisation X <- X (3 - X^T X)/2 twice, which removes
//     the small non-orthogonality inverse iteration leaves between close
//     eigenvalues without leaving the span of X;
//  6. back-transformation U = Q X in compact-WY blocks of 64 reflectors
//     (split-K FP64 GEMMs), written transposed as the rows of Ut.
//
// Only the kept eigenvectors are formed.  Householder convention: H = 1 - tau v v^T,
// v_0 = 1, H x = beta e_1.
#include <float.h>

#include <algorithm>
#include <mutex>
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {
namespace {

constexpr int RB = 1024;  // threads of the single-block kernels

__device__ __forceinline__ double block_sum(double v, double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    if (lane == 0) sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// Reflector for column k: x = A[k+1:n, k].
__global__ void __launch_bounds__(RB) hh_reflector_kernel(const double *A, double *V, double *d,
                                                          double *e, double *tau, double *scal,
                                                          int n, int k) {
  __shared__ double sh[32];
  const int L = n - k - 1;
  double s = 0.0;
  for (int i = 1 + threadIdx.x; i < L; i += blockDim.x) {
    double x = A[(int64_t)(k + 1 + i) * n + k];
    s = fma(x, x, s);
  }
  const double sigma = block_sum(s, sh);
  const double alpha = A[(int64_t)(k + 1) * n + k];
  double t, beta, sc;
  if (sigma == 0.0) {
    t = 0.0; beta = alpha; sc = 0.0;
  } else {
    double nrm = sqrt(alpha * alpha + sigma);
    beta = (alpha >= 0.0) ? -nrm : nrm;
    t = (beta - alpha) / beta;
    sc = 1.0 / (alpha - beta);
  }
  double *v = V + (int64_t)k * n + (k + 1);
  for (int i = threadIdx.x; i < L; i += blockDim.x)
    v[i] = (i == 0) ? 1.0 : A[(int64_t)(k + 1 + i) * n + k] * sc;
  if (threadIdx.x == 0) {
    d[k] = A[(int64_t)k * n + k];
    e[k] = beta;
    tau[k] = t;
    scal[0] = t;
  }
}

// p = tau * A22 v, one warp per row of the trailing block.
__global__ void hh_symv_kernel(const double *__restrict__ A, const double *__restrict__ V,
                               double *__restrict__ p, const double *__restrict__ scal, int n,
                               int k) {
  const int L = n - k - 1;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= L) return;
  const double *row = A + (int64_t)(k + 1 + warp) * n + (k + 1);
  const double *v = V + (int64_t)k * n + (k + 1);
  double s = 0.0;
  for (int j = lane; j < L; j += 32) s = fma(row[j], v[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) p[warp] = scal[0] * s;
}

// w = p - (tau/2)(p.v) v
__global__ void __launch_bounds__(RB) hh_w_kernel(const double *V, const double *p, double *w,
                                                  const double *scal, int n, int k) {
  __shared__ double sh[32];
  const int L = n - k - 1;
  const double *v = V + (int64_t)k * n + (k + 1);
  double s = 0.0;
  for (int i = threadIdx.x; i < L; i += blockDim.x) s = fma(p[i], v[i], s);
  const double gamma = 0.5 * scal[0] * block_sum(s, sh);
  for (int i = threadIdx.x; i < L; i += blockDim.x) w[i] = p[i] - gamma * v[i];
}

// A22 -= v w^T + w v^T
__global__ void hh_update_kernel(double *__restrict__ A, const double *__restrict__ V,
                                 const double *__restrict__ w, int n, int k) {
  const int L = n - k - 1;
  const double *v = V + (int64_t)k * n + (k + 1);
  const int64_t LL = (int64_t)L * L;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < LL;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / L), j = (int)(e - (int64_t)i * L);
    double *a = A + (int64_t)(k + 1 + i) * n + (k + 1 + j);
    *a -= v[i] * w[j] + w[i] * v[j];
  }
}

// ---- persistent Householder reduction (one cooperative launch) ----
// All n-2 reflector steps in one kernel.  Row r of the working matrix belongs
// to one warp for the whole reduction, so each
// row is read and written by one SM only; data one block writes and another
// reads (v, p, the column being reduced, the partial sums) go through L2
// (ld.global.cg).  Rows are dealt round-robin over blocks, then warps.
// Per step: [every block forms the reflector from the column in L2; p = tau
// A22 v on its rows; partial p.v] barrier [rank-2 update + the next column's
// partial norm] barrier.  Grid barriers use release/acquire atomics, are
// bounded (about two seconds) and report through flags.
struct GridBar {
  unsigned count, gen;
  int abort;
};

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ bool grid_barrier(GridBar *gb, int *flags) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = ld_acquire(&gb->gen);
    if (atom_add_acq_rel(&gb->count, 1u) == gridDim.x - 1) {
      gb->count = 0;
      atom_add_acq_rel(&gb->gen, 1u);   // release: the reset and every arrival happen-before
    } else {
      const uint64_t t0 = gtimer();
      unsigned it = 0;
      while (ld_acquire(&gb->gen) == g) {
        if ((++it & 1023) == 0) {
          if (*(volatile int *)&gb->abort) { ok = 0; break; }
          if (gtimer() - t0 > 2000000000ull) {
            atomicExch(&flags[FLAG_EIG], 1);
            atomicExch(&gb->abort, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Fixed-order sum of the per-block partials (identical in every block).
__device__ double sum_partials(const double *part, double *sh) {
  double v = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(part + b);
  return block_sum(v, sh);
}

__global__ void __launch_bounds__(512) hh_persistent_kernel(double *A, double *V, double *d, double *e,
                                                            double *tau, double *P, double *part1, double *part2,
                                                            GridBar *gb, int n, int *flags) {
  extern __shared__ double sm_vp[];   // v[n], p[n]
  __shared__ double sh[32];
  double *sv = sm_vp, *sp = sm_vp + n;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  // rows go round-robin over blocks first, so every SM gets rows
  const int gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const int nw = gridDim.x * wpb;
  // partial norm of column 0 below the subdiagonal
  {
    double acc = 0.0;
    for (int r = gw; r < n; r += nw)
      if (r >= 2 && lane == 0) { double x = A[(int64_t)r * n]; acc += x * x; }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part1[blockIdx.x] = acc;
  }
  if (!grid_barrier(gb, flags)) return;
  for (int k = 0; k + 2 < n; ++k) {
    // ---- reflector for column k (x = A[k+1:n, k]), computed by every block
    const double sigma = sum_partials(part1, sh);
    const double alpha = __ldcg(A + (int64_t)(k + 1) * n + k);
    double t, beta, sc;
    if (sigma == 0.0) {
      t = 0.0; beta = alpha; sc = 0.0;
    } else {
      const double nrm = sqrt(alpha * alpha + sigma);
      beta = (alpha >= 0.0) ? -nrm : nrm;
      t = (beta - alpha) / beta;
      sc = 1.0 / (alpha - beta);
    }
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
      const double v = (j == k + 1) ? 1.0 : __ldcg(A + (int64_t)j * n + k) * sc;
      sv[j] = v;
      if (blockIdx.x == 0) V[(int64_t)k * n + j] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      d[k] = __ldcg(A + (int64_t)k * n + k);
      e[k] = beta;
      tau[k] = t;
    }
    __syncthreads();
    // ---- p = tau A22 v (rows k+1..n-1), partial p.v
    double pv = 0.0;
    for (int r = gw; r < n; r += nw) {
      if (r < k + 1) continue;
      const double *row = A + (int64_t)r * n;
      // 8 independent loads in flight per lane: the row streams from L2
      double a8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int j = k + 1 + lane;
      for (; j + 7 * 32 < n; j += 8 * 32) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = row[j + u * 32];
#pragma unroll
        for (int u = 0; u < 8; ++u) a8[u] = fma(x[u], sv[j + u * 32], a8[u]);
      }
      for (; j < n; j += 32) a8[0] = fma(row[j], sv[j], a8[0]);
      double acc = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        const double pr = t * acc;
        P[r] = pr;
        pv += pr * sv[r];
      }
    }
    pv = block_sum(pv, sh);
    if (threadIdx.x == 0) part2[blockIdx.x] = pv;
    if (!grid_barrier(gb, flags)) return;
    // ---- A22 -= v w^T + w v^T with w = p - (tau/2)(p.v) v; next column's partial norm
    const double gamma = 0.5 * t * sum_partials(part2, sh);
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) sp[j] = __ldcg(P + j) - gamma * sv[j];
    __syncthreads();
    double nx = 0.0;
    for (int r = gw; r < n; r += nw) {
      if (r < k + 1) continue;
      double *row = A + (int64_t)r * n;
      const double vr = sv[r], wr = sp[r];
      int j = k + 1 + lane;
      for (; j + 7 * 32 < n; j += 8 * 32) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = row[j + u * 32];
#pragma unroll
        for (int u = 0; u < 8; ++u) row[j + u * 32] = x[u] - (vr * sp[j + u * 32] + wr * sv[j + u * 32]);
      }
      for (; j < n; j += 32) row[j] -= vr * sp[j] + wr * sv[j];
      __syncwarp();
      if (lane == 0 && r >= k + 3) { const double x = row[k + 1]; nx += x * x; }
    }
    nx = block_sum(nx, sh);
    if (threadIdx.x == 0) part1[blockIdx.x] = nx;
    if (!grid_barrier(gb, flags)) return;
  }
}

// Last diagonal / off-diagonal entries once every reflector is applied.
__global__ void hh_finalize_kernel(const double *A, double *d, double *e, int n) {
  if (threadIdx.x != 0) return;
  if (n >= 2) {
    d[n - 2] = A[(int64_t)(n - 2) * n + (n - 2)];
    e[n - 2] = A[(int64_t)(n - 1) * n + (n - 2)];
  }
  d[n - 1] = A[(int64_t)(n - 1) * n + (n - 1)];
  e[n - 1] = 0.0;
}

// 1/q from the hardware reciprocal estimate refined by three Newton steps
// y <- y (2 - q y) (each step squares the relative error), about 1 ulp: the
// Sturm count below is exact for a matrix perturbed by a few ulps anyway, and
// this avoids the IEEE division sequence, which is costly on this part's
// FP64 pipe.  |q| >= pivmin > 0 keeps q away from zero and subnormals.
__device__ __forceinline__ double recip_nr(double q) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(q));
  y = y * fma(-q, y, 2.0);
  y = y * fma(-q, y, 2.0);
  y = y * fma(-q, y, 2.0);
  return y;
}

// Number of eigenvalues of T below x (signs of the LDL^T pivots of T - x).
__device__ int sturm_count(const double *d, const double *e2, int n, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++c;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] * recip_nr(q);
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++c;
  }
  return c;
}

// scal[1..3] = lower / upper Gershgorin bound, pivmin; count[0] = #eig > thresh.
__global__ void __launch_bounds__(RB) tridiag_bounds_kernel(const double *d, const double *e,
                                                            int n, double thresh, double *scal,
                                                            double *e2, int *count) {
  __shared__ double s_lo[RB], s_hi[RB], s_e[RB];
  double lo = DBL_MAX, hi = -DBL_MAX, em = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i < n - 1) {
      e2[i] = e[i] * e[i];
      em = fmax(em, e2[i]);
    }
  }
  s_lo[threadIdx.x] = lo; s_hi[threadIdx.x] = hi; s_e[threadIdx.x] = em;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_lo[threadIdx.x] = fmin(s_lo[threadIdx.x], s_lo[threadIdx.x + s]);
      s_hi[threadIdx.x] = fmax(s_hi[threadIdx.x], s_hi[threadIdx.x + s]);
      s_e[threadIdx.x] = fmax(s_e[threadIdx.x], s_e[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double pivmin = DBL_MIN * fmax(1.0, s_e[0]);
    scal[1] = s_lo[0] - 2.0 * DBL_EPSILON * fabs(s_lo[0]) - 4.0 * pivmin - 1e-300;
    scal[2] = s_hi[0] + 2.0 * DBL_EPSILON * fabs(s_hi[0]) + 4.0 * pivmin + 1e-300;
    scal[3] = pivmin;
    scal[4] = fmax(fabs(s_lo[0]), fabs(s_hi[0]));  // ||T|| bound
    int below = sturm_count(d, e2, n, thresh, pivmin);
    count[0] = n - below;
    // eigenvalues within 1e-12 * ||T|| of the threshold (tie diagnostics)
    double tol = 1e-12 * scal[4];
    count[1] = sturm_count(d, e2, n, thresh + tol, pivmin) - sturm_count(d, e2, n, thresh - tol, pivmin);
  }
}

// lam[r] = (n-1-r)-th smallest eigenvalue (r-th largest), r < k, by
// multisection with BIS_L lanes per eigenvalue: each lane counts the
// eigenvalues below one of BIS_L interior points, so an interval shrinks
// (BIS_L + 1)-fold per step.  Few lanes per eigenvalue keep the total number
// of FP64 divisions (the cost on this part) near that of plain bisection while
// giving enough threads to hide their latency.  d and e^2 live in shared memory.
constexpr int BIS_L = 4;
__global__ void bisect_kernel(const double *d, const double *e2g, const double *scal, int n,
                              int k, int epw, double *lam) {
  extern __shared__ double sm[];
  double *sd = sm, *se2 = sm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sd[i] = d[i];
    se2[i] = (i < n - 1) ? e2g[i] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int sub = lane % BIS_L, grp = lane / BIS_L;
  const unsigned gmask = ((1u << BIS_L) - 1u) << (grp * BIS_L);
  const int r = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * epw + grp;
  const bool live = grp < epw && r < k;
  const int idx = n - 1 - (live ? r : 0);  // ascending index of the wanted eigenvalue
  double lo = scal[1], hi = scal[2];
  const double pivmin = scal[3];
  bool done = !live;
  for (int it = 0; it < 200; ++it) {
    if (!done && hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) done = true;
    if (__all_sync(0xffffffffu, done)) break;
    const double x = lo + (hi - lo) * (double)(sub + 1) / (double)(BIS_L + 1);
    const bool above = !done && sturm_count(sd, se2, n, x, pivmin) > idx;  // eigenvalue idx < x
    const unsigned b = (__ballot_sync(0xffffffffu, above) & gmask) >> (grp * BIS_L);
    if (!done) {
      const int j = b ? (__ffs(b) - 1) : BIS_L;
      const double nlo = (j == 0) ? lo : lo + (hi - lo) * (double)j / (double)(BIS_L + 1);
      const double nhi = (j == BIS_L) ? hi : lo + (hi - lo) * (double)(j + 1) / (double)(BIS_L + 1);
      if (!(nlo > lo || nhi < hi)) done = true;  // no progress at this resolution
      lo = nlo;
      hi = nhi;
    }
  }
  if (live && sub == 0) lam[r] = 0.5 * (lo + hi);
}

// Inverse iteration for the eigenvectors of T, one thread per group of
// consecutive eigenvalues closer than gtol (groups are orthogonalised
// internally).  X[i*k + r] receives the vector of lam[r].
__global__ void inverse_iteration_kernel(const double *dg, const double *eg, const double *lam,
                                         const double *scal, int n, int k, double *X,
                                         double *lu, int *flags) {
  extern __shared__ double sde[];
  double *d = sde, *e = sde + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { d[i] = dg[i]; e[i] = eg[i]; }
  __syncthreads();
  const int r0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (r0 >= k) return;
  const double tnorm = scal[4];
  const double gtol = 1e-7 * tnorm;
  if (r0 > 0 && lam[r0 - 1] - lam[r0] <= gtol) return;  // not the first of its group
  int r1 = r0 + 1;
  while (r1 < k && lam[r1 - 1] - lam[r1] <= gtol) ++r1;
  // scratch for this thread: dl, dd, du, du2, piv (strided by k for coalescing)
  double *dl = lu, *dd = lu + (int64_t)n * k, *du = lu + 2 * (int64_t)n * k;
  double *du2 = lu + 3 * (int64_t)n * k, *pv = lu + 4 * (int64_t)n * k;
  const double tiny = DBL_EPSILON * fmax(tnorm, DBL_MIN);
  double prev = 0.0;
  for (int r = r0; r < r1; ++r) {
    double lm = lam[r];
    if (r > r0) {
      double pert = 10.0 * DBL_EPSILON * fmax(fabs(lm), tnorm * 1e-3);
      if (prev - lm < pert) lm = prev - pert;
    }
    prev = lm;
#define S(a, i) a[(int64_t)(i) * k + r]
    // LU of T - lm with row interchanges
    for (int i = 0; i < n; ++i) {
      S(dd, i) = d[i] - lm;
      if (i < n - 1) { S(dl, i) = e[i]; S(du, i) = e[i]; }
      S(du2, i) = 0.0;
    }
    for (int i = 0; i < n - 1; ++i) {
      double di = S(dd, i), li = S(dl, i);
      if (fabs(di) >= fabs(li)) {
        S(pv, i) = 0.0;
        if (di == 0.0) { di = tiny; S(dd, i) = di; }
        double f = li / di;
        S(dl, i) = f;
        S(dd, i + 1) -= f * S(du, i);
      } else {
        S(pv, i) = 1.0;
        double f = di / li;
        S(dd, i) = li;
        S(dl, i) = f;
        double tmp = S(du, i);
        S(du, i) = S(dd, i + 1);
        S(dd, i + 1) = tmp - f * S(dd, i + 1);
        if (i < n - 2) {
          S(du2, i) = S(du, i + 1);
          S(du, i + 1) = -f * S(du, i + 1);
        }
      }
    }
    if (S(dd, n - 1) == 0.0) S(dd, n - 1) = tiny;
    for (int i = 0; i < n; ++i)
      if (fabs(S(dd, i)) < tiny) S(dd, i) = copysign(tiny, S(dd, i));
    // start vector: deterministic, no special structure
    for (int i = 0; i < n; ++i) S(X, i) = 1.0 + 0.5 * sin(0.7548776662 * (i + 1) + 0.5698402910 * (r + 1));
    for (int iter = 0; iter < 2; ++iter) {
      // forward: apply L^-1 with the interchanges
      for (int i = 0; i < n - 1; ++i) {
        if (S(pv, i) == 0.0) {
          S(X, i + 1) -= S(dl, i) * S(X, i);
        } else {
          double t = S(X, i);
          S(X, i) = S(X, i + 1);
          S(X, i + 1) = t - S(dl, i) * S(X, i);
        }
      }
      // backward: U^-1
      for (int i = n - 1; i >= 0; --i) {
        double s = S(X, i);
        if (i + 1 < n) s -= S(du, i) * S(X, i + 1);
        if (i + 2 < n) s -= S(du2, i) * S(X, i + 2);
        S(X, i) = s / S(dd, i);
      }
      // orthogonalise against the earlier vectors of this group
      for (int q = r0; q < r; ++q) {
        double dot = 0.0;
        for (int i = 0; i < n; ++i) dot += X[(int64_t)i * k + q] * S(X, i);
        for (int i = 0; i < n; ++i) S(X, i) -= dot * X[(int64_t)i * k + q];
      }
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) nrm += S(X, i) * S(X, i);
      nrm = sqrt(nrm);
      if (!(nrm > 0.0) || !isfinite(nrm)) { atomicExch(&flags[FLAG_EIG], 1); break; }
      double inv = 1.0 / nrm;
      for (int i = 0; i < n; ++i) S(X, i) *= inv;
    }
#undef S
  }
}

// F = (3 I - G) / 2 for a k x k Gram matrix G (in place).
__global__ void lowdin_factor_kernel(double *G, int k) {
  int64_t kk = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kk;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / k), j = (int)(e - (int64_t)i * k);
    G[e] = ((i == j) ? 1.5 : 0.0) - 0.5 * G[e];
  }
}

// ---- compact-WY back-transformation: U = H_0 H_1 ... H_{n-3} X ----
// For a block of nb consecutive reflectors j0..j0+nb-1 (rows of V, zero
// outside j+1..n-1), H_j0 ... H_{j0+nb-1} = 1 - V_b T V_b^T with T upper
// triangular (T_ii = tau_i, T[0:l, l] = -tau_l T[0:l, 0:l] G[0:l, l],
// G = V_b^T V_b).  Blocks are applied from the last to the first:
// Y <- Y - V_b (T (V_b^T Y)).
constexpr int WY_NB = 64;
constexpr int64_t WY_KSPLIT = 64;

// dst[i] = sum_s src[s * stride + i]
__global__ void sum_partials_kernel(const double *__restrict__ src, int nsplit, int64_t stride,
                                    int64_t n, double *__restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int q = 0; q < nsplit; ++q) a += src[q * stride + i];
    dst[i] = a;
  }
}

// T (nb x nb, row-major, upper) from G = V_b^T V_b and tau[j0..j0+nb).
__global__ void wy_build_t_kernel(const double *__restrict__ G, const double *__restrict__ tau,
                                  int j0, int nb, double *__restrict__ T) {
  __shared__ double sT[WY_NB][WY_NB + 1];
  const int i = threadIdx.x;
  for (int q = threadIdx.x; q < WY_NB * WY_NB; q += blockDim.x) sT[q / WY_NB][q % WY_NB] = 0.0;
  __syncthreads();
  if (i < nb) sT[i][i] = tau[j0 + i];
  __syncthreads();
  for (int l = 1; l < nb; ++l) {
    double v = 0.0;
    if (i < l) {
      for (int m = i; m < l; ++m) v += sT[i][m] * G[m * nb + l];
      v *= -tau[j0 + l];
    }
    __syncthreads();
    if (i < l) sT[i][l] = v;
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) T[q] = sT[q / nb][q % nb];
}

// Ut[c][r] = X[r][c]
__global__ void transpose_kernel(const double *__restrict__ X, int n, int k, double *__restrict__ Ut) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    int r = r0 + q, c = c0 + threadIdx.x;
    if (r < n && c < k) tile[q][threadIdx.x] = X[(int64_t)r * k + c];
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    int c = c0 + q, r = r0 + threadIdx.x;
    if (r < n && c < k) Ut[(int64_t)c * n + r] = tile[threadIdx.x][q];
  }
}

// Raise a kernel's dynamic shared-memory limit once, to the most any call
// may use; setting it per call races between host threads (one thread could
// lower it between another thread's set and launch).
cudaError_t allow_max_dynamic_smem(const void *kernel, std::once_flag &flag) {
  cudaError_t result = cudaSuccess;
  std::call_once(flag, [&] {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if ((result = cudaGetDevice(&dev)) != cudaSuccess) return;
    if ((result = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return;
    if ((result = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return;
    result = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes);
  });
  return result;
}
std::once_flag g_smem_hh, g_smem_bisect, g_smem_invit;

}  // namespace

cudaError_t launch_eig_tridiag(EigWork &w, int n, double thresh, cudaStream_t s, int *launches) {
  // one cooperative launch when the grid fits on the device and v, p fit in shared memory
  int dev = 0, nsm = 0, coop = 0, per_sm = 0;
  const size_t smem = 2 * (size_t)n * sizeof(double);
  bool persistent = n > 2 && smem <= 200 * 1024 && w.grid_ws != nullptr;
  if (persistent) {
    persistent = cudaGetDevice(&dev) == cudaSuccess &&
                 cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                 cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
                 allow_max_dynamic_smem((const void *)hh_persistent_kernel, g_smem_hh) == cudaSuccess &&
                 cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hh_persistent_kernel, 512, smem) ==
                     cudaSuccess &&
                 per_sm >= 1;
    cudaGetLastError();
  }
  if (persistent) {
    double *P = w.grid_ws, *part1 = P + n, *part2 = part1 + nsm;
    GridBar *gb = reinterpret_cast<GridBar *>(part2 + nsm);
    cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), s);
    if (e != cudaSuccess) return e;
    void *args[] = {&w.A, &w.V, &w.d, &w.e, &w.tau, &P, &part1, &part2, &gb, (void *)&n, &w.flags};
    e = cudaLaunchCooperativeKernel((const void *)hh_persistent_kernel, dim3(nsm), dim3(512), args, smem, s);
    if (e != cudaSuccess) return e;
    *launches += 1;
  } else {
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    hh_reflector_kernel<<<1, RB, 0, s>>>(w.A, w.V, w.d, w.e, w.tau, w.scal, n, k);
    int symv_blocks = (L * 32 + 255) / 256;
    hh_symv_kernel<<<symv_blocks, 256, 0, s>>>(w.A, w.V, w.p, w.scal, n, k);
    hh_w_kernel<<<1, RB, 0, s>>>(w.V, w.p, w.w, w.scal, n, k);
    int64_t LL = (int64_t)L * L;
    int ub = (int)((LL + 255) / 256);
    if (ub > 152 * 8) ub = 152 * 8;
    hh_update_kernel<<<ub, 256, 0, s>>>(w.A, w.V, w.w, n, k);
    *launches += 4;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  }
  hh_finalize_kernel<<<1, 32, 0, s>>>(w.A, w.d, w.e, n);
  // e2 reuses w.p (length n)
  tridiag_bounds_kernel<<<1, RB, 0, s>>>(w.d, w.e, n, thresh, w.scal, w.p, w.count);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_eig_vectors(EigWork &w, int n, int k, double *Ut, int *flags, cudaStream_t s,
                               int *launches) {
  if (k <= 0) return cudaSuccess;
  size_t smem = 2 * (size_t)n * sizeof(double);
  {
    cudaError_t e = allow_max_dynamic_smem((const void *)bisect_kernel, g_smem_bisect);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem((const void *)inverse_iteration_kernel, g_smem_invit);
    if (e != cudaSuccess) return e;
  }
  {
    // one warp per block and at most 32 / BIS_L eigenvalues per warp, spread
    // so that every SM gets work: the FP64 divisions of the Sturm counts are
    // the cost on this part
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 148;
    cudaGetLastError();
    const int epw = std::max(1, std::min(32 / BIS_L, (k + nsm - 1) / nsm));
    bisect_kernel<<<(k + epw - 1) / epw, 32, smem, s>>>(w.d, w.p, w.scal, n, k, epw, w.lam);
  }
  inverse_iteration_kernel<<<(k + 31) / 32, 32, smem, s>>>(w.d, w.e, w.lam, w.scal, n, k, w.X, w.lu, flags);
  *launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // re-orthonormalise twice: G = X^T X, F = (3 - G)/2, X <- X F
  double *G = w.lu;                       // k*k scratch (inverse-iteration scratch is free now)
  double *Xn = w.lu + (int64_t)k * k;     // n*k scratch
  for (int pass = 0; pass < 2; ++pass) {
    GemmF64Args g;
    g.M = k; g.N = k; g.K = n;
    g.A = w.X; g.lda = k;   // A[kidx][m] = X[i][m]  (M-major)
    g.B = w.X; g.ldb = k;   // B[kidx][n] = X[i][n]  (N-major)
    g.C = G; g.ldc = k;
    g.syrk = 1;
    e = launch_gemm_f64(g, 1, false, false, s);
    if (e != cudaSuccess) return e;
    lowdin_factor_kernel<<<152, 256, 0, s>>>(G, k);
    GemmF64Args h;
    h.M = n; h.N = k; h.K = k;
    h.A = w.X; h.lda = k;   // K-major rows of X
    h.B = G; h.ldb = k;     // N-major
    h.C = Xn; h.ldc = k;
    e = launch_gemm_f64(h, 1, true, false, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(w.X, Xn, (size_t)n * k * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    *launches += 3;
  }
  // compact-WY back-transformation, blocks of WY_NB reflectors from the last
  const int nref = n - 2;  // reflectors 0 .. n-3
  double *Gp = w.wy;                                           // [nsplit][nb][nb]
  const int nsplit_max = (int)((n + WY_KSPLIT - 1) / WY_KSPLIT);
  double *W1p = Gp + (int64_t)nsplit_max * WY_NB * WY_NB;      // [nsplit][nb][k]
  double *Gs = W1p + (int64_t)nsplit_max * WY_NB * k;          // [nb][nb]
  double *W1 = Gs + WY_NB * WY_NB;                             // [nb][k]
  double *Tm = W1 + (int64_t)WY_NB * k;                        // [nb][nb]
  double *W2 = Tm + WY_NB * WY_NB;                             // [nb][k]
  for (int j0 = ((nref - 1) / WY_NB) * WY_NB; nref > 0 && j0 >= 0; j0 -= WY_NB) {
    const int nb = std::min(WY_NB, nref - j0);
    const int r0 = j0 + 1;              // first row where this block's V is non-zero
    const int64_t len = n - r0;
    const int nsplit = (int)((len + WY_KSPLIT - 1) / WY_KSPLIT);
    GemmF64Args g;                      // G partials = V_b V_b^T over row chunks
    g.M = nb; g.N = nb; g.K = len; g.ksplit = WY_KSPLIT;
    g.A = w.V + (int64_t)j0 * n + r0; g.lda = n;
    g.B = w.V + (int64_t)j0 * n + r0; g.ldb = n;
    g.C = Gp; g.ldc = nb; g.strideC = (int64_t)nb * nb;
    e = launch_gemm_f64(g, nsplit, true, true, s);
    if (e != cudaSuccess) return e;
    GemmF64Args h;                      // W1 partials = V_b^T Y over row chunks
    h.M = nb; h.N = k; h.K = len; h.ksplit = WY_KSPLIT;
    h.A = w.V + (int64_t)j0 * n + r0; h.lda = n;
    h.B = w.X + (int64_t)r0 * k; h.ldb = k;
    h.C = W1p; h.ldc = k; h.strideC = (int64_t)nb * k;
    e = launch_gemm_f64(h, nsplit, true, false, s);
    if (e != cudaSuccess) return e;
    sum_partials_kernel<<<64, 256, 0, s>>>(Gp, nsplit, (int64_t)nb * nb, (int64_t)nb * nb, Gs);
    sum_partials_kernel<<<152, 256, 0, s>>>(W1p, nsplit, (int64_t)nb * k, (int64_t)nb * k, W1);
    wy_build_t_kernel<<<1, WY_NB, 0, s>>>(Gs, w.tau, j0, nb, Tm);
    GemmF64Args t2;                     // W2 = T W1
    t2.M = nb; t2.N = k; t2.K = nb;
    t2.A = Tm; t2.lda = nb; t2.B = W1; t2.ldb = k; t2.C = W2; t2.ldc = k;
    e = launch_gemm_f64(t2, 1, true, false, s);
    if (e != cudaSuccess) return e;
    GemmF64Args u;                      // Y[r0:, :] -= V_b^T W2
    u.M = (int)len; u.N = k; u.K = nb;
    u.A = w.V + (int64_t)j0 * n + r0; u.lda = n;   // A[kidx=i][m=r] = V[j0+i][r0+r]
    u.B = W2; u.ldb = k;
    u.C = w.X + (int64_t)r0 * k; u.ldc = k;
    u.alpha = -1.0; u.beta = 1.0;
    e = launch_gemm_f64(u, 1, false, false, s);
    if (e != cudaSuccess) return e;
    *launches += 7;
  }
  dim3 tb(32, 8), tg((k + 31) / 32, (n + 31) / 32);
  transpose_kernel<<<tg, tb, 0, s>>>(w.X, n, k, Ut);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace ltgw
