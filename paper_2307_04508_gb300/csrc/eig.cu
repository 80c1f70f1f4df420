// Symmetric eigensolver for the natural auxiliary functions (Sec. 2:
// diagonalise K, keep the eigenvectors whose eigenvalue exceeds eps_NAF).
//
//  1. Householder reduction K = Q T Q^T to tridiagonal T (one reflector per
//     step: reflector, symmetric mat-vec, rank-2 update of the trailing block);
//  2. Sturm-sequence count of the eigenvalues of T above the threshold;
//  3. multisection for the kept eigenvalues, with T in shared memory;
//  4. inverse iteration for their eigenvectors (tridiagonal LU with row
//     interchanges), with modified Gram-Schmidt inside groups of nearly equal
//     eigenvalues;
//  5. symmetric re-orthonormalisation X <- X (3 - X^T X)/2 twice, which removes
//     the small non-orthogonality inverse iteration leaves between close
//     eigenvalues without leaving the span of X;
//  6. back-transformation U = Q X in compact-WY blocks of 64 reflectors
//     (split-K GEMMs), written transposed as the rows of Ut.
//
// FP64 throughout (both the plain and the mixed-precision solve: only the
// dense contractions around the eigensolver change precision).  Only the kept
// eigenvectors are formed.  Householder convention: H = 1 - tau v v^T,
// v_0 = 1, H x = beta e_1.
//
// On this part an FP64 FMA has a dependent latency of about 64 cycles and an
// IEEE FP64 division about 400 (FP32 FMA: 4), so the sequential recurrences
// (Sturm counts, tridiagonal LU) are written to keep as few operations as
// possible on their dependency chains.
#include <float.h>

#include <algorithm>
#include <mutex>
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {
namespace {

constexpr int RB = 1024;        // threads of the single-block kernels
constexpr int HH_MIN_ROWS = 4;  // fewest rows per block of the fused reduction

template <typename T> struct Lim;
template <> struct Lim<double> {
  static __device__ __forceinline__ double eps() { return DBL_EPSILON; }
  static __device__ __forceinline__ double tiny() { return DBL_MIN; }
  static constexpr double group_tol = 1e-7;   // inverse-iteration groups, relative to ||T||
};

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

// ---- per-step kernels (FP64; used when a cooperative launch is not possible)
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

// ---- fused Householder reduction (one cooperative launch) ----
// All n-2 reflector steps in one kernel with ONE grid barrier per step.
// Writing A^(k) for the matrix after the first k rank-2 updates, reflector k
// comes from row k of A^(k) (= column k by symmetry), p_k = tau_k A^(k)_22 v_k,
// w_k = p_k - (tau_k/2)(p_k.v_k) v_k and A^(k+1)_22 = A^(k)_22 - v_k w_k^T - w_k v_k^T.
// Row r belongs to block r mod G for the whole reduction (held in shared
// memory when the block's rows fit there, else in place in global memory).
// Step k:
//  phase 1 (every block, identical arithmetic, so every block holds the same
//    vectors): normalise v_{k-1}; p_{k-1}.v_{k-1} from the full p_{k-1} (so
//    no per-block partial sums are exchanged); w_{k-1}; row k of A^(k) from
//    row k of A^(k-1), which its owner published during step k-1, minus
//    update k-1; the coefficients of reflector k.  The reflector is kept
//    unnormalised, x = (alpha, x_{k+2}, ...), with v = (1, sc x_{k+2}, ...) and
//    sc = 1/(alpha - beta), so no extra pass is needed before phase 2;
//  phase 2 (own rows r > k): one pass that applies update k-1 and accumulates
//    s_r = sum_j A^(k)[r][j] x_j, then p_k[r] = tau sc (s_r - beta A^(k)[r][k+1]);
//    the owner of row k+1 copies that row to the published buffer;
//  grid barrier.
// p and the published row are double-buffered by step parity, so a block
// still reading step k-1's copies never sees step k's writes.  Data crossing
// blocks goes through L2 (ld.global.cg).  The barrier is bounded (about two
// seconds) and reports through flags.
struct GridBar {
  unsigned count;   // arrivals so far; barrier j (0-based) is passed at count >= G (j + 1)
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

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Grid barrier number j: one release-add per block, then an acquire poll of
// the counter (bounded: about two seconds, then the abort flag and FLAG_EIG).
__device__ bool grid_barrier(GridBar *gb, unsigned j, int *flags) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = gridDim.x * (j + 1);
    red_add_release(&gb->count, 1u);
    if (ld_acquire(&gb->count) < target) {
      const uint64_t t0 = gtimer();
      unsigned it = 0;
      while (ld_acquire(&gb->count) < target) {
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

template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;   // in lane 0
}

template <typename T>
struct HhFusedArgs {
  const double *A0;   // the input matrix (row 0 is read from here at step 0)
  T *A;               // working rows, updated in place when they do not fit in shared memory
  T *V;               // [n][n] reflectors, row k = v_k (columns k+1..n-1 written)
  double *d, *e, *tau;
  T *P;               // [2][n] p of the step, by parity
  T *pub;             // [2][n] the next reflector's row, by parity
  double *tail;       // [2] A^(n-3)[n-1][n-2 .. n-1], for the last 2 x 2 block
  GridBar *gb;
  int *flags;
  int n, R;           // R = rows per block
};

// One lane-strided pass over row[j0:j1): optional update a -= v_r w + w_r v
// (UPD) and the dot with vc.  Eight loads are issued before their use so that
// rows streamed from L2/HBM keep enough requests in flight.
template <typename T, bool UPD>
__device__ __forceinline__ T row_pass(T *row, int j0, int j1, const T *vp, const T *wv, const T *vc, T vr, T wr) {
  const int lane = threadIdx.x & 31;
  T acc0 = 0, acc1 = 0;
  int j = j0 + lane;
  for (; j + 7 * 32 < j1; j += 8 * 32) {
    T x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = row[j + u * 32];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = j + u * 32;
      T a = x[u];
      if (UPD) {
        a = fma(-vr, wv[q], fma(-wr, vp[q], a));
        row[q] = a;
      }
      if (u & 1) acc1 = fma(a, vc[q], acc1); else acc0 = fma(a, vc[q], acc0);
    }
  }
  for (; j < j1; j += 32) {
    T a = row[j];
    if (UPD) {
      a = fma(-vr, wv[j], fma(-wr, vp[j], a));
      row[j] = a;
    }
    acc0 = fma(a, vc[j], acc0);
  }
  return acc0 + acc1;
}

// FP64 instructions are scarce on this part (about 2 per clock per SM), so
// the per-step bookkeeping keeps them off paths that every thread runs: the
// scalars are computed by one thread, and in the FP64 form phase 1 runs on
// HH_P1_FP64 threads only (the FP32 form does all of it in FP32).
constexpr int HH_P1_FP64 = 128;

template <typename T, bool SMEM>
__global__ void __launch_bounds__(512, 1) hh_fused_kernel(HhFusedArgs<T> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = reinterpret_cast<T *>(smem_raw);
  __shared__ T wbuf[2][16];       // per-warp partials: p.v, |x|^2
  __shared__ T s_seg[16], s_a1[16];
  __shared__ T s_st[5];           // x[k], alpha; tau, beta, sc of the step
  const int n = g.n, G = gridDim.x, b = blockIdx.x, R = g.R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int p1 = (sizeof(T) == 8) ? min(HH_P1_FP64, (int)blockDim.x) : (int)blockDim.x;  // phase-1 team
  const int p1w = p1 >> 5;
  T *wv = smem + 2 * n;
  T *rows = smem + 3 * n;   // SMEM: [R][n], local row lr is global row lr * G + b
  const int n_own = (b < n) ? min(R, (n - 1 - b) / G + 1) : 0;
  if (SMEM) {
    for (int lr = 0; lr < n_own; ++lr) {
      const double *src = g.A0 + (int64_t)(lr * G + b) * n;
      for (int j = threadIdx.x; j < n; j += blockDim.x) rows[(int64_t)lr * n + j] = (T)src[j];
    }
  }
  T *vprev = smem + n, *vcur = smem;
  T tau_prev = 0, sc_prev = 0;
  for (int k = 0; k + 2 < n; ++k) {
    // ---- phase 1.  Team thread t owns element j = k + t + m * p1 of every
    // vector it touches, so the loops below need no barrier between them.
    T *x = vcur;
    T s2 = 0;
    if (k == 0) {
      if (threadIdx.x < p1)
        for (int j = threadIdx.x; j < n; j += p1) {
          const T xj = (T)__ldcg(g.A0 + j);
          x[j] = xj;
          if (j >= 2) s2 = fma(xj, xj, s2);
          if (j < 2) s_st[j] = xj;
        }
    } else {
      const T *Pk = g.P + (size_t)((k - 1) & 1) * n;
      const T *pb = g.pub + (size_t)(k & 1) * n;
      // p of step k-1 and the published row k into wv and x by every thread,
      // its loads issued together: one L2 round trip, where the team's loop
      // below (a global store between its loads) would wait once per element
      for (int j0 = k + threadIdx.x; j0 < n; j0 += 4 * blockDim.x) {
        T pv[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * blockDim.x;
          if (j < n) { pv[u] = __ldcg(Pk + j); xv[u] = __ldcg(pb + j); }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * blockDim.x;
          if (j < n) { wv[j] = pv[u]; x[j] = xv[u]; }
        }
      }
      __syncthreads();
      const T pkk = wv[k];   // read before the team's second loop rewrites wv
      T dsum = 0;
      if (threadIdx.x < p1)
        for (int j = k + threadIdx.x; j < n; j += p1) {
          const T vj = (j == k) ? (T)1 : vprev[j] * sc_prev;   // normalise v_{k-1}
          vprev[j] = vj;
          if (b == 0) g.V[(int64_t)(k - 1) * n + j] = vj;
          dsum = fma(wv[j], vj, dsum);
        }
      if (warp < p1w) {
        dsum = warp_sum(dsum);
        if (lane == 0) wbuf[0][warp] = dsum;
      }
      __syncthreads();
      if (threadIdx.x < p1) {
        T pv = 0;
        for (int q = 0; q < p1w; ++q) pv += wbuf[0][q];
        const T gam = (T)0.5 * tau_prev * pv;
        const T wk = pkk - gam;   // v_{k-1}[k] = 1
        for (int j = k + threadIdx.x; j < n; j += p1) {
          const T wj = wv[j] - gam * vprev[j];
          wv[j] = wj;
          const T xj = x[j] - wj - wk * vprev[j];
          x[j] = xj;
          if (j >= k + 2) s2 = fma(xj, xj, s2);
          if (j < k + 2) s_st[j - k] = xj;
        }
      }
    }
    if (warp < p1w) {
      s2 = warp_sum(s2);
      if (lane == 0) wbuf[1][warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // the reflector's scalars, once
      T sigma = 0;
      for (int q = 0; q < p1w; ++q) sigma += wbuf[1][q];
      const T alpha = s_st[1];
      T t = 0, beta = alpha, sc = 0;
      if (sigma != (T)0) {
        const T nrm = sqrt(alpha * alpha + sigma);
        beta = (alpha >= (T)0) ? -nrm : nrm;
        t = (beta - alpha) / beta;
        sc = (T)1 / (alpha - beta);
      }
      s_st[2] = t; s_st[3] = beta; s_st[4] = sc;
      if (b == 0) {
        g.d[k] = s_st[0];
        g.e[k] = beta;
        g.tau[k] = t;
      }
    }
    __syncthreads();
    const T t = s_st[2], beta = s_st[3], sc = s_st[4], tsc = t * sc;
    // ---- phase 2: own rows r > k: update k-1 (k > 0) fused with s_r
    const int lr0 = (k + 1 > b) ? (k + 1 - b + G - 1) / G : 0;
    const int nact = n_own - lr0;
    const int wpr = nact > 0 ? max(1, nwarp / nact) : 1;   // warps per row when rows are few
    T *Pk = g.P + (size_t)(k & 1) * n;
    if (nact > 0) {
      const int L = n - k - 1;
      const int seglen = (((L + wpr - 1) / wpr) + 31) & ~31;
      for (int task = warp; task < nact * wpr; task += nwarp) {
        const int lr = lr0 + task / wpr, seg = task % wpr;
        const int r = lr * G + b;
        T *row = SMEM ? rows + (int64_t)lr * n : g.A + (int64_t)r * n;
        const int j0 = k + 1 + seg * seglen, j1 = min(n, j0 + seglen);
        T acc = 0, a1 = 0;
        if (j0 < j1) {
          if (k == 0) acc = row_pass<T, false>(row, j0, j1, vprev, wv, x, (T)0, (T)0);
          else acc = row_pass<T, true>(row, j0, j1, vprev, wv, x, vprev[r], wv[r]);
        }
        acc = warp_sum(acc);
        if (seg == 0) {   // A^(k)[r][k+1], written by this warp's lane 0
          __syncwarp();
          a1 = row[k + 1];
        }
        if (wpr == 1) {
          if (lane == 0) Pk[r] = tsc * (acc - beta * a1);
        } else if (lane == 0) {
          s_seg[task] = acc;
          if (seg == 0) s_a1[task / wpr] = a1;
        }
      }
    }
    __syncthreads();   // every row update of this step is complete
    if (nact > 0 && wpr > 1 && threadIdx.x < nact) {
      const int r = (lr0 + threadIdx.x) * G + b;
      T a = 0;
      for (int q = 0; q < wpr; ++q) a += s_seg[threadIdx.x * wpr + q];
      Pk[r] = tsc * (a - beta * s_a1[threadIdx.x]);
    }
    // the owner of row k+1 publishes it (A^(k) values, columns k+1..n-1); at the
    // last step the owner of row n-1 also hands over that row's last two entries
    if ((k + 1) % G == b) {
      const int lr = (k + 1) / G;
      const T *rp = SMEM ? rows + (int64_t)lr * n : g.A + (int64_t)(k + 1) * n;
      T *pubp = g.pub + (size_t)((k + 1) & 1) * n;
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) pubp[j] = rp[j];
    }
    if (k == n - 3 && (n - 1) % G == b && threadIdx.x == 0) {
      const T *rp = SMEM ? rows + (int64_t)((n - 1) / G) * n : g.A + (int64_t)(n - 1) * n;
      g.tail[0] = rp[n - 2];
      g.tail[1] = rp[n - 1];
    }
    if (!grid_barrier(g.gb, (unsigned)k, g.flags)) return;
    tau_prev = t;
    sc_prev = sc;
    T *tmp = vprev; vprev = vcur; vcur = tmp;
  }
  // ---- the last 2 x 2 block: normalise v_{n-3}, apply update n-3 to rows n-2, n-1
  if (b == 0 && n >= 3 && threadIdx.x == 0) {
    const int kl = n - 3;
    const T *Pk = g.P + (size_t)(kl & 1) * n;
    const T *pb = g.pub + (size_t)((kl + 1) & 1) * n;
    const T v2 = 1, v1 = vprev[n - 1] * sc_prev;
    g.V[(int64_t)kl * n + n - 2] = v2;
    g.V[(int64_t)kl * n + n - 1] = v1;
    const T p2 = __ldcg(Pk + n - 2), p1v = __ldcg(Pk + n - 1);
    const T gam = (T)0.5 * tau_prev * (p2 * v2 + p1v * v1);
    const T w2 = p2 - gam * v2, w1 = p1v - gam * v1;
    const T a22 = __ldcg(pb + n - 2), a21 = __ldcg(pb + n - 1), a11 = (T)__ldcg(g.tail + 1);
    g.d[n - 2] = fma(-v2, w2, fma(-w2, v2, a22));
    g.e[n - 2] = fma(-v2, w1, fma(-w2, v1, a21));
    g.d[n - 1] = fma(-v1, w1, fma(-w1, v1, a11));
    g.e[n - 1] = 0.0;
  }
}

// Number of eigenvalues of T below x (Sturm): the sign changes along the
// leading principal minors p_0 = 1, p_i = det(T_i - x) with
// p_i = (d_{i-1} - x) p_{i-1} - e_{i-2}^2 p_{i-2}.  This is the LDL^T pivot
// count q_i = p_i / p_{i-1} without the division: one FMA per step sits on the
// dependency chain (e^2 p_{i-2} is ready a step early), against a reciprocal
// and its Newton steps in the quotient form.  The pair (p_{i-1}, p_i) is
// rescaled by an exact power of two whenever the larger exponent leaves
// [-400, 400] (integer operations on the high words), and a minor that comes
// out exactly zero is replaced by pivmin with the sign opposite to p_{i-1}
// (counted as a sign change, like the quotient form's pivot -pivmin).  The range check runs every 8 steps, off
// the chain.
__device__ __forceinline__ bool is_zero_bits(double v) {   // +0 or -0, on the integer pipe
  return ((__double2hiint(v) & 0x7fffffff) | __double2loint(v)) == 0;
}

__device__ int sturm_count(const double *d, const double *e2, int n, double x, double pivmin) {
  double pm = 1.0, p = d[0] - x;
  if (p == 0.0) p = -pivmin;
  bool neg = __double2hiint(p) < 0;
  int c = neg;
  int i = 1;
  while (i < n) {
    // 8 steps between range checks: |p| grows at most 2 (|d| + |e| + |x|) per
    // step and shrinks by at most e^2 per two, so +-400 stays far from overflow.
    // The block's d_i - x and e^2 are formed first, off the FMA chain.
    double dx[8], ee[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = min(i + u, n - 1);
      dx[u] = d[j] - x;
      ee[u] = e2[j - 1];
    }
    const int m = min(8, n - i);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (u < m) {
        double pn = fma(dx[u], p, -(ee[u] * pm));
        if (is_zero_bits(pn))   // -pivmin with the sign opposite to p, on the integer pipe
          pn = __longlong_as_double((~__double_as_longlong(p) & (long long)0x8000000000000000ull) |
                                    __double_as_longlong(pivmin));
        const bool nn = __double2hiint(pn) < 0;
        c += (nn != neg);
        neg = nn;
        pm = p;
        p = pn;
      }
    }
    i += m;
    const int em = max((__double2hiint(p) >> 20) & 0x7ff, (__double2hiint(pm) >> 20) & 0x7ff);
    if (em > 1023 + 400 || em < 1023 - 400) {
      const double f = __hiloint2double((2046 - em) << 20, 0);   // 2^(1023 - em), exact
      p *= f;
      pm *= f;
    }
  }
  return c;
}

// 1/q from the hardware reciprocal estimate and Newton steps y <- y (2 - q y)
// (each squares the relative error): two give a few ulps, one about 2^-46, at
// a fraction of the latency of the IEEE division on this part.  |q| is kept
// away from zero and subnormals by the caller.
template <int STEPS = 2>
__device__ __forceinline__ double recip_nr(double q) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(q));
#pragma unroll
  for (int s = 0; s < STEPS; ++s) y = y * fma(-q, y, 2.0);
  return y;
}

// |a| < |b| on the integer pipe (finite doubles: magnitude order = bit order)
__device__ __forceinline__ bool abs_less(double a, double b) {
  return (__double_as_longlong(a) & 0x7fffffffffffffffll) < (__double_as_longlong(b) & 0x7fffffffffffffffll);
}

// scal[1..3] = lower / upper Gershgorin bound, pivmin; scal[4] = ||T|| bound;
// scal[5] = max e^2; count[0] = #eig > thresh, count[1] = #eig within
// 1e-12 ||T|| of it.
__global__ void __launch_bounds__(RB) tridiag_bounds_kernel(const double *dg, const double *e,
                                                            int n, double thresh, double *scal,
                                                            double *e2g, int *count, bool staged) {
  __shared__ double s_lo[RB], s_hi[RB], s_e[RB];
  // the Sturm counts below walk d and e^2 sequentially: staged in shared
  // memory when they fit, so that each step is not an L2 round trip
  extern __shared__ double s_de[];
  double *sd = staged ? s_de : nullptr, *se2 = staged ? s_de + n : e2g;
  const double *d = staged ? sd : dg;
  double *e2 = se2;
  if (staged)
    for (int i = threadIdx.x; i < n; i += blockDim.x) sd[i] = dg[i];
  double lo = DBL_MAX, hi = -DBL_MAX, em = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    lo = fmin(lo, dg[i] - r);
    hi = fmax(hi, dg[i] + r);
    if (i < n - 1) {
      const double ee = e[i] * e[i];
      e2[i] = ee;
      if (staged) e2g[i] = ee;
      em = fmax(em, ee);
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
  // the three counts (at the threshold and at thresh -/+ tol) run in three warps at once
  __shared__ int s_cnt[3];
  const double pivmin = DBL_MIN * fmax(1.0, s_e[0]);
  const double tn = fmax(fabs(s_lo[0]), fabs(s_hi[0]));  // ||T|| bound
  const double tol = 1e-12 * tn;
  const int w = threadIdx.x >> 5;
  if (w < 3 && (threadIdx.x & 31) == 0) {
    const double x = thresh + (w == 0 ? 0.0 : (w == 1 ? tol : -tol));
    s_cnt[w] = sturm_count(d, e2, n, x, pivmin);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    scal[1] = s_lo[0] - 2.0 * DBL_EPSILON * fabs(s_lo[0]) - 4.0 * pivmin - 1e-300;
    scal[2] = s_hi[0] + 2.0 * DBL_EPSILON * fabs(s_hi[0]) + 4.0 * pivmin + 1e-300;
    scal[3] = pivmin;
    scal[4] = tn;
    scal[5] = s_e[0];
    count[0] = n - s_cnt[0];
    // eigenvalues within tol of the threshold (tie diagnostics)
    count[1] = s_cnt[1] - s_cnt[2];
  }
}

// lam[r] = (n-1-r)-th smallest eigenvalue (r-th largest), r < k, by
// multisection with BIS_L lanes per eigenvalue: each lane counts the
// eigenvalues below one of BIS_L interior points, so an interval shrinks
// (BIS_L + 1)-fold per step.  On this part a warp's FP64 instructions run one
// after another whatever their dependences, so a whole warp per eigenvalue
// (33-fold per step, about 11 steps to full precision) beats fewer lanes with
// more steps.  d and e^2 live in shared memory.
constexpr int BIS_L = 32;
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
  const unsigned gmask = (BIS_L >= 32) ? 0xffffffffu : (((1u << (BIS_L & 31)) - 1u) << (grp * BIS_L));
  const int r = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * epw + grp;
  const bool live = grp < epw && r < k;
  const int idx = n - 1 - (live ? r : 0);  // ascending index of the wanted eigenvalue
  double lo = scal[1], hi = scal[2];
  const double pivmin = scal[3];
  bool done = !live;
  for (int it = 0; it < 200; ++it) {
    if (!done && hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) done = true;
    if (__all_sync(0xffffffffu, done)) break;
    const double x = lo + (hi - lo) * ((double)(sub + 1) * (1.0 / (BIS_L + 1)));
    const bool above = !done && sturm_count(sd, se2, n, x, pivmin) > idx;  // eigenvalue idx < x
    const unsigned b = (__ballot_sync(0xffffffffu, above) & gmask) >> (grp * BIS_L);
    if (!done) {
      const int j = b ? (__ffs(b) - 1) : BIS_L;
      // the same expressions as the lanes' points, so the bracket is exactly two of them
      const double nlo = (j == 0) ? lo : lo + (hi - lo) * ((double)j * (1.0 / (BIS_L + 1)));
      const double nhi = (j == BIS_L) ? hi : lo + (hi - lo) * ((double)(j + 1) * (1.0 / (BIS_L + 1)));
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
//
// The LU factorisation of T - lambda (row interchanges) runs with its
// recurrence carried in registers, so it only reads T and writes the factors:
// multipliers, reciprocals of U's diagonal, U's two super-diagonals and the
// interchange flags.  SMEM: those five arrays and the working vector live in
// shared memory, interleaved by thread (TPB threads per block); otherwise in
// the global scratch lu (strided by k) and X.  The start vector comes from an
// integer hash of (i, r).
constexpr int IV_DL = 0, IV_RDD = 1, IV_DU = 2, IV_DU2 = 3, IV_PV = 4, IV_X = 5;

__device__ __forceinline__ unsigned mix32(unsigned x) {
  x ^= x >> 16; x *= 0x7feb352du;
  x ^= x >> 15; x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

template <typename T>
__device__ __forceinline__ T iv_start(int i, int r) {
  return (T)0.5 + (T)(mix32((unsigned)i * 0x9e3779b9u ^ mix32((unsigned)r + 0x632be5abu)) >> 8) * (T)(1.0 / 16777216.0);
}

template <typename T, bool SMEM>
__global__ void inverse_iteration_kernel(const double *dg, const double *eg, const double *lam,
                                         const double *scal, int n, int k, T *X, T *lu, int *flags) {
  extern __shared__ __align__(16) unsigned char sde_raw[];
  T *d = reinterpret_cast<T *>(sde_raw), *e = d + n;
  T *ws = e + n;                                   // SMEM: [6][n][blockDim.x]
  for (int i = threadIdx.x; i < n; i += blockDim.x) { d[i] = (T)dg[i]; e[i] = (i < n - 1) ? (T)eg[i] : (T)0; }
  __syncthreads();
  const int tl = threadIdx.x, tpb = blockDim.x;
  const int r0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (r0 >= k) return;
  const double tnorm = scal[4];
  const double gtol = Lim<T>::group_tol * tnorm;
  if (r0 > 0 && lam[r0 - 1] - lam[r0] <= gtol) return;  // not the first of its group
  int r1 = r0 + 1;
  while (r1 < k && lam[r1 - 1] - lam[r1] <= gtol) ++r1;
  const T tiny = Lim<T>::eps() * fmax((T)tnorm, Lim<T>::tiny());
  // pivots below tiny in magnitude (zero included) become +-tiny; integer compare
  const long long tiny_bits = __double_as_longlong(tiny);
  auto fix = [&](T x) -> T {
    const long long xb = __double_as_longlong(x);
    return ((xb & 0x7fffffffffffffffll) < tiny_bits) ? __longlong_as_double((xb & (long long)0x8000000000000000ull) | tiny_bits)
                                                   : x;
  };
  double prev = 0.0;
  for (int r = r0; r < r1; ++r) {
    // element i of array a of this thread's vector
#define S(a, i) (SMEM ? ws[((int64_t)(a) * n + (i)) * tpb + tl] : lu[((int64_t)(a) * n + (i)) * k + r])
#define XV(i) (SMEM ? ws[((int64_t)IV_X * n + (i)) * tpb + tl] : X[(int64_t)(i) * k + r])
    double lmd = lam[r];
    if (r > r0) {
      double pert = 10.0 * (double)Lim<T>::eps() * fmax(fabs(lmd), tnorm * 1e-3);
      if (prev - lmd < pert) lmd = prev - pert;
    }
    prev = lmd;
    const T lm = (T)lmd;
    // LU of T - lm with row interchanges; a, b = current diagonal and super-diagonal.
    // One reciprocal per step (of the pivot); U's super-diagonals are stored
    // pre-scaled by it, so the backward sweep has one FMA on its chain.
    {
      // chain per step: pivot choice (integer compare), reciprocal, one FMA;
      // the block's d - lm, c b and a dn are formed beside it
      T a = d[0] - lm, b = e[0];
      for (int i0 = 0; i0 < n - 1; i0 += 8) {
        T dn8[8], c8[8], bn8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = min(i0 + u, n - 2);
          dn8[u] = d[i + 1] - lm;
          c8[u] = e[i];
          bn8[u] = e[i + 1];   // e[n-1] = 0
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u;
          if (i < n - 1) {
            const T c = c8[u], dn = dn8[u], bn = bn8[u];
            const T cb = c * b, adn = a * dn;
            const bool sw = abs_less(a, c);
            const T piv = fix(sw ? c : a);
            const T rp = recip_nr<1>(piv);   // 2^-46: ample for an iteration that refines itself
            const T f = (sw ? a : c) * rp;
            S(IV_DL, i) = f;
            S(IV_RDD, i) = rp;
            S(IV_DU, i) = (sw ? dn : b) * rp;
            S(IV_DU2, i) = sw ? bn * rp : (T)0;
            S(IV_PV, i) = sw ? (T)1 : (T)0;
            const T an = sw ? fma(-adn, rp, b) : fma(-cb, rp, dn);
            b = sw ? -f * bn : bn;
            a = an;
          }
        }
      }
      S(IV_RDD, n - 1) = recip_nr<1>(fix(a));
      S(IV_DU, n - 1) = 0;
      S(IV_DU2, n - 1) = 0;
    }
    for (int iter = 0; iter < 2; ++iter) {
      // forward: apply L^-1 with the interchanges (the start vector on the first
      // pass).  Eight steps' factors and entries are loaded before the chain.
      T xc = (iter == 0) ? iv_start<T>(0, r) : XV(0);
      for (int i0 = 0; i0 < n - 1; i0 += 8) {
        T f8[8], p8[8], x8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = min(i0 + u, n - 2);
          f8[u] = S(IV_DL, i);
          p8[u] = S(IV_PV, i);
          x8[u] = (iter == 0) ? iv_start<T>(i + 1, r) : XV(i + 1);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u;
          if (i < n - 1) {
            T xn = x8[u], out;
            if (p8[u] == (T)0) { out = xc; xn = xn - f8[u] * xc; }
            else { out = xn; xn = xc - f8[u] * xn; }
            XV(i) = out;
            xc = xn;
          }
        }
      }
      XV(n - 1) = xc;
      // backward: U^-1 (rows scaled by 1 / pivot), eight steps' data loaded first
      T x1 = 0, x2 = 0;
      for (int i0 = n - 1; i0 >= 0; i0 -= 8) {
        T du8[8], dv8[8], rd8[8], xv8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = max(i0 - u, 0);
          du8[u] = S(IV_DU, i);
          dv8[u] = S(IV_DU2, i);
          rd8[u] = S(IV_RDD, i);
          xv8[u] = XV(i);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 - u;
          if (i >= 0) {
            const T sv = fma(-du8[u], x1, fma(-dv8[u], x2, xv8[u] * rd8[u]));
            XV(i) = sv;
            x2 = x1;
            x1 = sv;
          }
        }
      }
      // orthogonalise against the earlier vectors of this group (already in X)
      for (int q = r0; q < r; ++q) {
        double dot = 0.0;
        for (int i = 0; i < n; ++i) dot += (double)X[(int64_t)i * k + q] * (double)XV(i);
        const T dt = (T)dot;
        for (int i = 0; i < n; ++i) XV(i) -= dt * X[(int64_t)i * k + q];
      }
      T s0 = 0, s1 = 0, s2 = 0, s3 = 0;   // four chains: FP64 FMA latency is long here
      int i = 0;
      for (; i + 3 < n; i += 4) {
        s0 = fma(XV(i), XV(i), s0); s1 = fma(XV(i + 1), XV(i + 1), s1);
        s2 = fma(XV(i + 2), XV(i + 2), s2); s3 = fma(XV(i + 3), XV(i + 3), s3);
      }
      for (; i < n; ++i) s0 = fma(XV(i), XV(i), s0);
      const double nrm = sqrt((double)((s0 + s1) + (s2 + s3)));
      if (!(nrm > 0.0) || !isfinite(nrm)) { atomicExch(&flags[FLAG_EIG], 1); break; }
      const T inv = (T)(1.0 / nrm);
      if (SMEM && iter == 1) {
        for (int i = 0; i < n; ++i) X[(int64_t)i * k + r] = XV(i) * inv;
      } else {
        for (int i = 0; i < n; ++i) XV(i) *= inv;
      }
    }
#undef S
#undef XV
  }
}

// F = (3 I - G) / 2 for a k x k Gram matrix G (in place).
template <typename T>
__global__ void lowdin_factor_kernel(T *G, int k) {
  int64_t kk = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kk;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / k), j = (int)(e - (int64_t)i * k);
    G[e] = (T)(((i == j) ? 1.5 : 0.0) - 0.5 * (double)G[e]);
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
template <typename T>
__global__ void sum_partials_kernel(const T *__restrict__ src, int nsplit, int64_t stride,
                                    int64_t n, T *__restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T a = 0;
    for (int q = 0; q < nsplit; ++q) a += src[q * stride + i];
    dst[i] = a;
  }
}

// T (row-major, upper, zero-padded to WY_NB x WY_NB) of reflector block b (one
// CTA each) from G_b = V_b^T V_b (Gg + b*WY_NB^2, ld nb) and tau[j0..j0+nb),
// j0 = b*WY_NB.
// Column l: T[0:l, l] = -tau_l T[0:l, 0:l] G[0:l, l]; four threads share
// each row's sum (shorter FMA chains).
template <typename T>
__global__ void wy_build_t_kernel(const T *__restrict__ Gall, const double *__restrict__ tau, int nref,
                                  T *__restrict__ Tall) {
  // dynamic: [2][WY_NB][WY_NB + 1] (over the static limit in FP64)
  extern __shared__ __align__(16) unsigned char wy_raw[];
  T (*sT)[WY_NB + 1] = reinterpret_cast<T (*)[WY_NB + 1]>(wy_raw);
  T (*Gt)[WY_NB + 1] = sT + WY_NB;   // G transposed: column l of G is read along a row
  const int j0 = blockIdx.x * WY_NB, nb = min(WY_NB, nref - j0);
  const T *Gg = Gall + (int64_t)blockIdx.x * WY_NB * WY_NB;
  T *Tm = Tall + (int64_t)blockIdx.x * WY_NB * WY_NB;
  for (int q = threadIdx.x; q < WY_NB * WY_NB; q += blockDim.x) {
    sT[q / WY_NB][q % WY_NB] = 0;
    if (q < nb * nb) Gt[q % nb][q / nb] = Gg[q];
  }
  __syncthreads();
  if (threadIdx.x < nb) sT[threadIdx.x][threadIdx.x] = (T)tau[j0 + threadIdx.x];
  __syncthreads();
  const int i = threadIdx.x >> 2, part = threadIdx.x & 3;   // blockDim = 4 * WY_NB
  for (int l = 1; l < nb; ++l) {
    T v = 0;
    if (i < l)
      for (int m = i + part; m < l; m += 4) v = fma(sT[i][m], Gt[l][m], v);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    __syncthreads();
    if (i < l && part == 0) sT[i][l] = -(T)tau[j0 + l] * v;
    __syncthreads();
  }
  for (int q = threadIdx.x; q < WY_NB * WY_NB; q += blockDim.x) Tm[q] = sT[q / WY_NB][q % WY_NB];   // zero-padded
}

// ---- the compact-WY blocks applied by one cooperative kernel ----
// Launched as G CTAs for each of the S column slices (columns 64 s .. 64 s +
// 63 of Y).  CTA (s, c) owns the row chunks ch = c, c + G, c + 2G, ... of
// WA_RC rows.  For each block b, last to first (rows r0 = 64 b + 1 .. n-1):
//   1. the partial of W1 = V_b Y[r0:, slice] over the own chunks -> Wp[s][c];
//   2. grid barrier; CTA c sums entries c*256 + t (+ G*256 ...) of the
//      slice's partials                                            -> W1[s];
//   3. grid barrier; Y[own rows, slice] -= M_b[own rows] W1[s].
// A CTA reads and writes only its own rows of Y, so step 3 of one block and
// step 1 of the next need no barrier between them.  Each step does
// WA_RC x 64 x 64 FMAs per chunk (64 rows of V_b by the slice, or the chunk's
// rows by 64 columns), so the FP64 work spreads over every SM in units a
// quarter of a 64 x 64 x 64 tile.
constexpr int WA_RC = 32;
constexpr size_t WA_SMEM = (size_t)(64 * (WA_RC + 1) + 64 * 64) * sizeof(double);   // step 3 (the larger)

struct WyApplyArgs {
  const double *V;   // [n + 64][n] reflectors (rows)
  const double *M;   // [nblk][n - 1][64]: M_b[r - 1][i] = (V_b^T T_b)[r][i]
  double *Y;         // [n][k], updated in place
  double *Wp;        // [S * G][64 * 64] partials of W1
  double *W1;        // [S][64 * 64]
  GridBar *gb;
  int *flags;
  int n, k, nref, nblk, G;
};

__global__ void __launch_bounds__(256) wy_apply_kernel(WyApplyArgs g) {
  extern __shared__ __align__(16) double wa_sm[];
  const int s = blockIdx.x / g.G, c = blockIdx.x % g.G;
  const int n = g.n, k = g.k, col0 = 64 * s, ncol = min(64, k - col0);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double *W1s = g.W1 + (int64_t)s * 4096;
  unsigned bar = 0;
  for (int b = g.nblk - 1; b >= 0; --b) {
    const int j0 = 64 * b, nb = min(64, g.nref - j0), r0 = j0 + 1;
    // ---- 1: Vs[r][i] = V_b[i][a + r] (transposed), Ys[r][cc] = Y[a + r][col0 + cc]
    double *Vs = wa_sm, *Ys = wa_sm + WA_RC * 65;
    double acc[4][4] = {};
    for (int ch = c; ch * WA_RC < n; ch += g.G) {
      const int a = max(ch * WA_RC, r0), e = min(n, ch * WA_RC + WA_RC);
      if (a >= e) continue;   // the same for the whole CTA
      const int len = e - a;
      for (int q = tid; q < 64 * WA_RC; q += 256) {
        const int i = q / WA_RC, r = q % WA_RC;
        Vs[r * 65 + i] = (i < nb && r < len) ? g.V[(int64_t)(j0 + i) * n + a + r] : 0.0;
        const int r2 = q >> 6, cc = q & 63;
        Ys[r2 * 64 + cc] = (r2 < len && cc < ncol) ? g.Y[(int64_t)(a + r2) * k + col0 + cc] : 0.0;
      }
      __syncthreads();
      for (int r = 0; r < len; ++r) {
        double av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) av[u] = Vs[r * 65 + ty + 16 * u];
#pragma unroll
        for (int v = 0; v < 4; ++v) bv[v] = Ys[r * 64 + tx + 16 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
      }
      __syncthreads();
    }
    double *Wpc = g.Wp + (int64_t)blockIdx.x * 4096;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) Wpc[(ty + 16 * u) * 64 + tx + 16 * v] = acc[u][v];
    if (!grid_barrier(g.gb, bar++, g.flags)) return;
    // ---- 2: the slice's partials summed, 256 entries per CTA at a time
    const double *Wps = g.Wp + (int64_t)s * g.G * 4096;
    for (int q = c * 256 + tid; q < 4096; q += g.G * 256) {
      double t = 0.0;
      for (int m = 0; m < g.G; ++m) t += __ldcg(Wps + (int64_t)m * 4096 + q);
      W1s[q] = t;
    }
    if (!grid_barrier(g.gb, bar++, g.flags)) return;
    // ---- 3: Ms[i][r] = M_b[a + r - 1][i] (transposed), Ws = W1[s]
    double *Ms = wa_sm, *Ws = wa_sm + 64 * (WA_RC + 1);
    for (int q = tid; q < 4096; q += 256) Ws[q] = __ldcg(W1s + q);
    __syncthreads();
    for (int ch = c; ch * WA_RC < n; ch += g.G) {
      const int a = max(ch * WA_RC, r0), e = min(n, ch * WA_RC + WA_RC);
      if (a >= e) continue;
      const int len = e - a;
      for (int q = tid; q < WA_RC * 64; q += 256) {
        const int r = q >> 6, i = q & 63;
        Ms[i * (WA_RC + 1) + r] = (r < len && i < nb) ? g.M[((int64_t)b * (n - 1) + (a + r - 1)) * 64 + i] : 0.0;
      }
      __syncthreads();
      double upd[2][4] = {};
      for (int i = 0; i < nb; ++i) {
        double av[2], bv[4];
#pragma unroll
        for (int u = 0; u < 2; ++u) av[u] = Ms[i * (WA_RC + 1) + ty + 16 * u];
#pragma unroll
        for (int v = 0; v < 4; ++v) bv[v] = Ws[i * 64 + tx + 16 * v];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) upd[u][v] = fma(av[u], bv[v], upd[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int r = ty + 16 * u;
        if (r >= len) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int cc = tx + 16 * v;
          if (cc < ncol) g.Y[(int64_t)(a + r) * k + col0 + cc] -= upd[u][v];
        }
      }
      __syncthreads();
    }
  }
}

// Ut[c][r] = X[r][c]
template <typename T>
__global__ void transpose_kernel(const T *__restrict__ X, int n, int k, double *__restrict__ Ut) {
  __shared__ T tile[32][33];
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
std::once_flag g_smem_hh[2], g_smem_bisect, g_smem_invit[2], g_smem_bounds, g_smem_wy, g_smem_wa;

// Try the fused reduction in arithmetic T; false when it cannot be launched.
template <typename T>
bool launch_fused(EigWork &w, int n, cudaStream_t s, int *launches, cudaError_t *err) {
  int dev = 0, nsm = 0, coop = 0, optin = 0;
  *err = cudaSuccess;
  bool ok = n > 2 && w.grid_ws != nullptr && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess;
  cudaGetLastError();
  if (!ok) return false;
  const int G = std::min(nsm, std::max(1, (n + HH_MIN_ROWS - 1) / HH_MIN_ROWS));
  const int R = (n + G - 1) / G;
  const size_t reserve = 1024;   // static shared memory of the kernel
  const size_t s_rows = (size_t)(3 + R) * n * sizeof(T), s_vec = (size_t)3 * n * sizeof(T);
  const bool in_smem = s_rows + reserve <= (size_t)optin;
  const size_t smem = in_smem ? s_rows : s_vec;
  if (smem + reserve > (size_t)optin) return false;
  const int fi = in_smem ? 1 : 0;
  const void *kern = in_smem ? (const void *)hh_fused_kernel<T, true> : (const void *)hh_fused_kernel<T, false>;
  int per_sm = 0;
  ok = allow_max_dynamic_smem(kern, g_smem_hh[fi]) == cudaSuccess &&
       cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem) == cudaSuccess && per_sm >= 1;
  cudaGetLastError();
  if (!ok) return false;
  HhFusedArgs<T> g;
  g.A0 = w.A;
  g.A = w.A;   // reduced in place when the rows do not fit in shared memory
  g.V = reinterpret_cast<T *>(w.V);
  g.d = w.d; g.e = w.e; g.tau = w.tau;
  g.P = reinterpret_cast<T *>(w.grid_ws);
  g.pub = g.P + 2 * (size_t)n;
  double *after = w.grid_ws + (4 * (size_t)n * sizeof(T) + sizeof(double) - 1) / sizeof(double);
  g.tail = after;
  g.gb = reinterpret_cast<GridBar *>(after + 2);
  g.flags = w.flags;
  g.n = n; g.R = R;
  *err = cudaMemsetAsync(g.gb, 0, sizeof(GridBar), s);
  if (*err != cudaSuccess) return true;
  void *args[] = {&g};
  *err = cudaLaunchCooperativeKernel(kern, dim3(G), dim3(512), args, smem, s);
  if (*err == cudaSuccess) *launches += 1;
  return true;
}

// Steps 3-6 in arithmetic T.
template <typename T>
cudaError_t eig_vectors_impl(EigWork &w, int n, int k, double *Ut, int *flags, cudaStream_t s, int *launches) {
  const size_t smem = 2 * (size_t)n * sizeof(T);
  {
    cudaError_t e = allow_max_dynamic_smem((const void *)bisect_kernel, g_smem_bisect);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem((const void *)inverse_iteration_kernel<T, true>, g_smem_invit[0]);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem((const void *)inverse_iteration_kernel<T, false>, g_smem_invit[1]);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem((const void *)wy_build_t_kernel<T>, g_smem_wy);
    if (e != cudaSuccess) return e;
  }
  {
    // at most 32 / BIS_L eigenvalues per warp, spread so that every SM gets
    // work; four warps per block, one per scheduler of the SM (the warps of
    // one-warp blocks can share a scheduler, and each FP64 instruction holds
    // it for the whole warp), with one copy of d and e^2 in shared memory
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 148;
    cudaGetLastError();
    const int epw = std::max(1, std::min(32 / BIS_L, (k + nsm - 1) / nsm));
    const int nwarps = (k + epw - 1) / epw;
    bisect_kernel<<<(nwarps + 3) / 4, 128, smem, s>>>(w.d, w.p, w.scal, n, k, epw, w.lam);
  }
  T *X = reinterpret_cast<T *>(w.X), *lu = reinterpret_cast<T *>(w.lu), *V = reinterpret_cast<T *>(w.V);
  {
    // factors in shared memory when at least one thread's share fits
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      optin = 48 * 1024;
    cudaGetLastError();
    // shared-memory factors only when every vector then runs in one wave; FP64
    // instructions cost a warp the same with 2 active lanes as with 32, so
    // otherwise 32 vectors per warp with the factors in L2 is faster
    const size_t budget = (size_t)optin - 1024, per_thread = 6 * (size_t)n * sizeof(T);
    int tpb = smem + per_thread <= budget ? (int)std::min<size_t>(32, (budget - smem) / per_thread) : 0;
    int nsm_iv = 148, dev_iv = 0;
    if (cudaGetDevice(&dev_iv) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm_iv, cudaDevAttrMultiProcessorCount, dev_iv) != cudaSuccess)
      nsm_iv = 148;
    cudaGetLastError();
    if (tpb >= 1 && (k + tpb - 1) / tpb > nsm_iv) tpb = 0;
    if (tpb >= 1)
      inverse_iteration_kernel<T, true><<<(k + tpb - 1) / tpb, tpb, smem + tpb * per_thread, s>>>(
          w.d, w.e, w.lam, w.scal, n, k, X, lu, flags);
    else
      inverse_iteration_kernel<T, false><<<(k + 31) / 32, 32, smem, s>>>(w.d, w.e, w.lam, w.scal, n, k, X, lu, flags);
  }
  *launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // re-orthonormalise: G = X^T X, F = (3 - G)/2, X <- X F.  One pass squares
  // the non-orthogonality inverse iteration leaves (about 1e-12 here).  X^T X
  // is split over its length-n sum (partials in the free inverse-iteration
  // scratch): a 64 x 64 FP64 tile over all n rows would keep one SM busy for
  // milliseconds.
  T *G = lu;                       // k*k scratch (inverse-iteration scratch is free now)
  T *Xn = lu + (int64_t)k * k;     // n*k scratch
  {
    T *Gpart = Xn + (int64_t)n * k;
    const int64_t room = 5 * (int64_t)n * n - (int64_t)k * k - (int64_t)n * k;
    int nsp = (int)std::min<int64_t>((n + 63) / 64, std::max<int64_t>(1, room / ((int64_t)k * k)));
    const int64_t ks = (n + nsp - 1) / nsp;
    nsp = (int)((n + ks - 1) / ks);
    GemmArgs<T> g;
    g.M = k; g.N = k; g.K = n; g.ksplit = ks;
    g.A = X; g.lda = k;   // A[kidx][m] = X[i][m]  (M-major)
    g.B = X; g.ldb = k;   // B[kidx][n] = X[i][n]  (N-major)
    g.C = Gpart; g.ldc = k; g.strideC = (int64_t)k * k;
    g.syrk = 1;
    e = launch_gemm<T>(g, nsp, false, false, s);
    if (e != cudaSuccess) return e;
    sum_partials_kernel<T><<<152, 256, 0, s>>>(Gpart, nsp, (int64_t)k * k, (int64_t)k * k, G);
    lowdin_factor_kernel<T><<<152, 256, 0, s>>>(G, k);
    GemmArgs<T> h;
    h.M = n; h.N = k; h.K = k;
    h.A = X; h.lda = k;   // K-major rows of X
    h.B = G; h.ldb = k;   // N-major
    h.C = Xn; h.ldc = k;
    e = launch_gemm<T>(h, 1, true, false, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(X, Xn, (size_t)n * k * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    *launches += 4;
  }
  // compact-WY back-transformation, blocks of WY_NB reflectors from the last:
  // Y <- Y - M_b (V_b^T Y) with M_b = V_b T_b.  Every block's G, T and M_b are
  // formed first (every G in one launch, the T recurrences in one launch, all
  // M_b in one batched GEMM over rows 1..n-1; V carries WY_NB zero rows past
  // its end for the last block), then the blocks are applied in order: by one
  // cooperative kernel, or two GEMMs each where that kernel cannot launch.
  const int nref = n - 2;  // reflectors 0 .. n-3
  if (nref > 0) {
    const int nblk = (nref + WY_NB - 1) / WY_NB;
    const int nsplit_max = (int)((n + WY_KSPLIT - 1) / WY_KSPLIT);
    // region 0 (w.wy_r0 doubles): W1's split partials and W1 for the
    // block-at-a-time form, or the cooperative kernel's partials and W1
    T *W1p = reinterpret_cast<T *>(w.wy);                        // [nsplit][nb][k]
    T *W1 = W1p + (int64_t)nsplit_max * WY_NB * k;               // [nb][k]
    T *Gs = reinterpret_cast<T *>(w.wy) + w.wy_r0;               // [nblk][nb][nb]
    T *Tm = Gs + (int64_t)nblk * WY_NB * WY_NB;                  // [nblk][WY_NB][WY_NB]
    T *Mall = Tm + (int64_t)nblk * WY_NB * WY_NB;                // [nblk][n-1][WY_NB]
    {
      // every block's G = V_b V_b^T in one launch (column chunks of WY_KSPLIT;
      // a block-at-a-time GEMM keeps only ~n/64 SMs busy), the chunk partials
      // in the M_b region, which is written only after the T recurrences
      T *Gp = Mall;                                              // [nchunk][nblk][nb][nb]
      const int64_t nchunk = (n - 1 + WY_KSPLIT - 1) / WY_KSPLIT;
      e = launch_gram_panels(V, n, nref, WY_NB, WY_KSPLIT, Gp, s);
      if (e != cudaSuccess) return e;
      sum_partials_kernel<T><<<152, 256, 0, s>>>(Gp, (int)nchunk, (int64_t)nblk * WY_NB * WY_NB,
                                                 (int64_t)nblk * WY_NB * WY_NB, Gs);
      *launches += 2;
    }
    wy_build_t_kernel<T><<<nblk, 4 * WY_NB, 2 * WY_NB * (WY_NB + 1) * sizeof(T), s>>>(Gs, w.tau, nref, Tm);
    {
      GemmArgs<T> m;                      // M_b[r-1][c] = sum_i V[j0+i][r] T_b[i][c], r = 1..n-1
      m.M = n - 1; m.N = WY_NB; m.K = WY_NB;
      m.A = V + 1; m.lda = n; m.strideA = (int64_t)WY_NB * n;        // A[kidx=i][m] = V[j0+i][1+m]
      m.B = Tm; m.ldb = WY_NB; m.strideB = (int64_t)WY_NB * WY_NB;
      m.C = Mall; m.ldc = WY_NB; m.strideC = (int64_t)(n - 1) * WY_NB;
      e = launch_gemm<T>(m, nblk, false, false, s);
      if (e != cudaSuccess) return e;
    }
    *launches += 2;
    // the blocks applied by one cooperative kernel when its CTAs fit at once
    // and region 0 holds their partials; otherwise two GEMMs per block
    bool applied = false;
    if (sizeof(T) == sizeof(double)) {
      int dev = 0, nsm = 0, coop = 0, per_sm = 0;
      const int S = (k + 63) / 64;
      if (cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop && S <= nsm &&
          allow_max_dynamic_smem((const void *)wy_apply_kernel, g_smem_wa) == cudaSuccess &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)wy_apply_kernel, 256, WA_SMEM) ==
              cudaSuccess && per_sm >= 1) {
        int G = nsm / S;
        while (G > 1 && (int64_t)(S * G + S) * 4096 > w.wy_r0) --G;
        if ((int64_t)(S * G + S) * 4096 <= w.wy_r0) {
          WyApplyArgs a;
          a.V = reinterpret_cast<const double *>(V);
          a.M = reinterpret_cast<const double *>(Mall);
          a.Y = reinterpret_cast<double *>(X);
          a.Wp = w.wy;
          a.W1 = w.wy + (int64_t)S * G * 4096;
          // the fused reduction's barrier word (that kernel has finished)
          a.gb = reinterpret_cast<GridBar *>(w.grid_ws + 4 * (size_t)n + 2);
          a.flags = flags;
          a.n = n; a.k = k; a.nref = nref; a.nblk = nblk; a.G = G;
          e = cudaMemsetAsync(a.gb, 0, sizeof(GridBar), s);
          if (e != cudaSuccess) return e;
          void *args[] = {&a};
          e = cudaLaunchCooperativeKernel((const void *)wy_apply_kernel, dim3((unsigned)(S * G)), dim3(256), args,
                                          WA_SMEM, s);
          if (e != cudaSuccess) return e;
          *launches += 1;
          applied = true;
        }
      }
      cudaGetLastError();
    }
    for (int bi = nblk - 1; bi >= 0 && !applied; --bi) {
      const int j0 = bi * WY_NB, nb = std::min(WY_NB, nref - j0);
      const int r0 = j0 + 1;
      const int64_t len = n - r0;
      const int nsplit = (int)((len + WY_KSPLIT - 1) / WY_KSPLIT);
      GemmArgs<T> h;                      // W1 partials = V_b^T Y over row chunks
      h.M = nb; h.N = k; h.K = len; h.ksplit = WY_KSPLIT;
      h.A = V + (int64_t)j0 * n + r0; h.lda = n;
      h.B = X + (int64_t)r0 * k; h.ldb = k;
      h.C = W1p; h.ldc = k; h.strideC = (int64_t)nb * k;
      e = launch_gemm<T>(h, nsplit, true, false, s);
      if (e != cudaSuccess) return e;
      sum_partials_kernel<T><<<152, 256, 0, s>>>(W1p, nsplit, (int64_t)nb * k, (int64_t)nb * k, W1);
      GemmArgs<T> u;                      // Y[r0:, :] -= M_b[r0:, 0:nb] W1
      u.M = (int)len; u.N = k; u.K = nb;
      u.A = Mall + (int64_t)bi * (n - 1) * WY_NB + (int64_t)(r0 - 1) * WY_NB; u.lda = WY_NB;   // K-major
      u.B = W1; u.ldb = k;
      u.C = X + (int64_t)r0 * k; u.ldc = k;
      u.alpha = -1.0; u.beta = 1.0;
      e = launch_gemm<T>(u, 1, true, false, s);
      if (e != cudaSuccess) return e;
      *launches += 3;
    }
  }
  dim3 tb(32, 8), tg((k + 31) / 32, (n + 31) / 32);
  transpose_kernel<T><<<tg, tb, 0, s>>>(X, n, k, Ut);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_eig_tridiag(EigWork &w, int n, double thresh, cudaStream_t s, int *launches) {
  cudaError_t e = cudaSuccess;
  const bool fused = launch_fused<double>(w, n, s, launches, &e);
  if (e != cudaSuccess) return e;
  if (!fused) {
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
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    hh_finalize_kernel<<<1, 32, 0, s>>>(w.A, w.d, w.e, n);
    *launches += 1;
  }
  // e2 reuses w.p (length n)
  {
    const size_t st = 2 * (size_t)n * sizeof(double);
    const bool staged = st <= 180 * 1024 &&
                        allow_max_dynamic_smem((const void *)tridiag_bounds_kernel, g_smem_bounds) == cudaSuccess;
    cudaGetLastError();
    tridiag_bounds_kernel<<<1, RB, staged ? st : 0, s>>>(w.d, w.e, n, thresh, w.scal, w.p, w.count, staged);
  }
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_eig_vectors(EigWork &w, int n, int k, double *Ut, int *flags, cudaStream_t s,
                               int *launches) {
  if (k <= 0) return cudaSuccess;
  return eig_vectors_impl<double>(w, n, k, Ut, flags, s, launches);
}

}  // namespace ltgw
