// Screening of Eq. ScreenedCoulombOrbital: C(i w_j) = [1 - Pi(i w_j)]^-1 - 1
// for every frequency, by the symmetric sweep operator (Gauss-Jordan without
// pivoting, stable here because 1 - Pi is symmetric positive definite with all
// eigenvalues >= 1).  After sweeping every pivot the matrix holds -A^-1.
//
// Two forms:
//  * launch_screen: one launch per pivot k for all frequencies, ping-ponging
//    between two buffers (first step forms A = 1 - Pi, last writes C = -X - 1);
//  * launch_screen_blocked: pivot blocks of 64 - the block is inverted by a
//    4-CTA cluster, and the rank-64 update A -= A[:,P] A_PP^-1 A[P,:] runs on
//    the FP64 tiled GEMM (about N/64 x 5 launches instead of N).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {
namespace {

constexpr int SW_ROWS = 4;  // rows of one matrix per block

// grid: x = row group of SW_ROWS rows, y = frequency.  Threads stride over columns.
__global__ void __launch_bounds__(256) sweep_step_kernel(const double *__restrict__ in,
                                                         double *__restrict__ out, int N, int k,
                                                         int first, int last, int *flags) {
  const int b = blockIdx.y;
  const int64_t NN = (int64_t)N * N;
  const double *X = in + b * NN;
  double *Y = out + b * NN;
  const double *rowk = X + (int64_t)k * N;
  double p = rowk[k];
  if (first) p = 1.0 - p;
  if (blockIdx.x == 0 && threadIdx.x == 0 && !(p > 0.0 && isfinite(p)))
    atomicExch(&flags[FLAG_NOT_SPD], 1);
  const double rp = 1.0 / p;
  const double sg = first ? -1.0 : 1.0;  // first step reads 1 - Pi
  for (int q = 0; q < SW_ROWS; ++q) {
    const int i = blockIdx.x * SW_ROWS + q;
    if (i >= N) break;
    const double *rowi = X + (int64_t)i * N;
    double *yi = Y + (int64_t)i * N;
    double aik = sg * rowi[k];
    if (i == k && first) aik = p;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      double akj = sg * rowk[j] + ((first && j == k) ? 1.0 : 0.0);
      double aij = sg * rowi[j] + ((first && i == j) ? 1.0 : 0.0);
      double r;
      if (i == k && j == k) r = -rp;
      else if (i == k) r = akj * rp;
      else if (j == k) r = aik * rp;
      else r = aij - aik * akj * rp;
      if (last) r = -r - (i == j ? 1.0 : 0.0);
      yi[j] = r;
    }
  }
}

// ---- blocked sweep: pivot blocks of SB_B, rank-SB_B updates on the tiled GEMM ----
constexpr int SB_B = 64;

// X = I - Pi
template <typename T>
__global__ void form_a_kernel(const double *__restrict__ Pi, T *__restrict__ X, int N, int64_t total) {
  const int64_t NN = (int64_t)N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = e % NN;
    const int i = (int)(f / N), j = (int)(f - (int64_t)i * N);
    X[e] = (T)((i == j ? 1.0 : 0.0) - Pi[e]);
  }
}

// Z = X[P,P]^-1 for each frequency, by the sweep on a cluster of SB_CL CTAs
// (one CTA per frequency would leave most SMs idle through the bs pivots).
// CTA c of the cluster holds rows SB_RPC*c .. SB_RPC*c + SB_RPC - 1 of the
// block in registers: warp w rows 2w and 2w + 1 of them, lane l columns l and
// l + 32.  At pivot k the warp holding row k forms the reciprocal of the pivot
// and writes row k scaled by it, and the reciprocal, into every CTA's shared
// memory; each CTA keeps its own rows' column k locally; then one cluster
// barrier.  The buffers alternate with the pivot's parity, so the writes for
// pivot k + 1 never meet the reads for pivot k.
constexpr int SB_CL = 4;
constexpr int SB_RPC = SB_B / SB_CL;         // rows per CTA
constexpr int SB_THREADS = SB_RPC / 2 * 32;  // one warp per two rows

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void st_cluster_f64(uint32_t local_addr, unsigned rank, double v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_addr), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote), "d"(v) : "memory");
}

template <typename T>
__global__ void __cluster_dims__(SB_CL, 1, 1) __launch_bounds__(SB_THREADS)
    block_inverse_kernel(const T *__restrict__ X, int N, int p0, int bs, T *__restrict__ Z, int *flags) {
  static_assert(sizeof(T) == sizeof(double), "the pivot row is exchanged as f64");
  __shared__ T rowk[2][SB_B + 1];   // [SB_B]: the pivot's reciprocal
  __shared__ T colk[2][SB_RPC];
  unsigned crank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
  const int b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lr0 = 2 * warp, i0 = (int)crank * SB_RPC + lr0;
  const T *Xb = X + (int64_t)b * N * N;
  T v[2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + r, j = lane + 32 * h;
      v[r][h] = (i < bs && j < bs) ? Xb[(int64_t)(p0 + i) * N + (p0 + j)] : (T)0;
    }
  const uint32_t rowk_addr = (uint32_t)__cvta_generic_to_shared(&rowk[0][0]);
  cluster_sync();   // every CTA of the cluster is running before the first remote write
  for (int k = 0; k < bs; ++k) {
    const int par = k & 1, hk = k >> 5;
    if (lane == (k & 31)) {
      colk[par][lr0] = hk ? v[0][1] : v[0][0];
      colk[par][lr0 + 1] = hk ? v[1][1] : v[1][0];
    }
    if ((int)crank == k / SB_RPC && warp == (k % SB_RPC) >> 1) {   // this warp holds row k
      const int rk = k & 1;
      const T mine = rk ? (hk ? v[1][1] : v[1][0]) : (hk ? v[0][1] : v[0][0]);
      const T piv = __shfl_sync(0xffffffffu, mine, k & 31);
      if (lane == 0 && !(piv > (T)0 && isfinite(piv))) atomicExch(&flags[FLAG_NOT_SPD], 1);
      const T rp = (T)1 / piv;
      const T a0 = (rk ? v[1][0] : v[0][0]) * rp, a1 = (rk ? v[1][1] : v[0][1]) * rp;
      const uint32_t row = rowk_addr + (uint32_t)(par * (SB_B + 1) * sizeof(T));
#pragma unroll
      for (unsigned c = 0; c < SB_CL; ++c) {
        st_cluster_f64(row + lane * sizeof(T), c, a0);
        st_cluster_f64(row + (lane + 32) * sizeof(T), c, a1);
        if (lane == 0) st_cluster_f64(row + SB_B * sizeof(T), c, rp);
      }
    }
    cluster_sync();
    const T rp = rowk[par][SB_B];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + r, j = lane + 32 * h;
        if (i >= bs || j >= bs) continue;
        if (i == k && j == k) v[r][h] = -rp;
        else if (i == k) v[r][h] = rowk[par][j];
        else if (j == k) v[r][h] = colk[par][lr0 + r] * rp;
        else v[r][h] = fma(-colk[par][lr0 + r], rowk[par][j], v[r][h]);
      }
  }
  T *Zb = Z + (int64_t)b * SB_B * SB_B;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + r, j = lane + 32 * h;
      if (i < bs && j < bs) Zb[i * SB_B + j] = -v[r][h];
    }
}

// rowsP[b][r][j] = X[b][p0 + r][j]
template <typename T>
__global__ void copy_rows_kernel(const T *__restrict__ X, int N, int p0, int bs, T *__restrict__ rowsP) {
  const int b = blockIdx.z, r = blockIdx.y;
  const T *src = X + (int64_t)b * N * N + (int64_t)(p0 + r) * N;
  T *dst = rowsP + ((int64_t)b * SB_B + r) * N;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) dst[j] = src[j];
}

// X[:, P] = R, X[P, :] = R^T, X[P, P] = -Z
template <typename T>
__global__ void fix_block_kernel(T *__restrict__ X, int N, int p0, int bs, const T *__restrict__ R,
                                 const T *__restrict__ Z) {
  const int b = blockIdx.y;
  T *Xb = X + (int64_t)b * N * N;
  const T *Rb = R + (int64_t)b * N * SB_B;
  const T *Zb = Z + (int64_t)b * SB_B * SB_B;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)N * bs;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / bs), c = (int)(q % bs);
    const bool inP = i >= p0 && i < p0 + bs;
    const T v = inP ? -Zb[(i - p0) * SB_B + c] : Rb[(int64_t)i * SB_B + c];
    Xb[(int64_t)i * N + p0 + c] = v;
    if (!inP) Xb[(int64_t)(p0 + c) * N + i] = v;   // the P x P block is written once
  }
}

// C = -X - I
template <typename T>
__global__ void finish_c_kernel(const T *__restrict__ X, double *__restrict__ C, int N, int64_t total) {
  const int64_t NN = (int64_t)N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = e % NN;
    const int i = (int)(f / N), j = (int)(f - (int64_t)i * N);
    C[e] = -(double)X[e] - (i == j ? 1.0 : 0.0);
  }
}

template <typename T>
cudaError_t screen_blocked_impl(const double *Pi, int N, int n_omega, T *work, double *C, int *flags,
                                cudaStream_t s, int *launches) {
  const int64_t NN = (int64_t)N * N, total = NN * n_omega;
  T *X = work;
  T *R = X + total;
  T *rowsP = R + (int64_t)n_omega * N * SB_B;
  T *Z = rowsP + (int64_t)n_omega * SB_B * N;
  int eb = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  form_a_kernel<T><<<eb, 256, 0, s>>>(Pi, X, N, total);
  ++*launches;
  for (int p0 = 0; p0 < N; p0 += SB_B) {
    const int bs = std::min(SB_B, N - p0);
    block_inverse_kernel<T><<<dim3(SB_CL, n_omega), SB_THREADS, 0, s>>>(X, N, p0, bs, Z, flags);
    dim3 cg((N + 255) / 256 < 8 ? (N + 255) / 256 : 8, bs, n_omega);
    copy_rows_kernel<T><<<cg, 256, 0, s>>>(X, N, p0, bs, rowsP);
    GemmArgs<T> g;   // R = X[:, P] Z
    g.M = N; g.N = bs; g.K = bs;
    g.A = X + p0; g.lda = N; g.strideA = NN;
    g.B = Z; g.ldb = SB_B; g.strideB = (int64_t)SB_B * SB_B;
    g.C = R; g.ldc = SB_B; g.strideC = (int64_t)N * SB_B;
    cudaError_t e = launch_gemm<T>(g, n_omega, true, false, s);
    if (e != cudaSuccess) return e;
    GemmArgs<T> u;   // X -= R X[P, :]  (= X[:, P] Z X[P, :], symmetric: lower tiles, mirrored)
    u.M = N; u.N = N; u.K = bs; u.syrk = 1;
    u.A = R; u.lda = SB_B; u.strideA = (int64_t)N * SB_B;
    u.B = rowsP; u.ldb = N; u.strideB = (int64_t)SB_B * N;
    u.C = X; u.ldc = N; u.strideC = NN;
    u.alpha = -1.0; u.beta = 1.0;
    e = launch_gemm<T>(u, n_omega, true, false, s);
    if (e != cudaSuccess) return e;
    dim3 fg((int)std::min<int64_t>(((int64_t)N * bs + 255) / 256, 64), n_omega);
    fix_block_kernel<T><<<fg, 256, 0, s>>>(X, N, p0, bs, R, Z);
    *launches += 5;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  finish_c_kernel<T><<<eb, 256, 0, s>>>(X, C, N, total);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_screen(const double *Pi, int N, int n_omega, double *X0, double *X1,
                          double *C, int *flags, cudaStream_t s, int *launches) {
  if (N <= 0 || n_omega <= 0) return cudaSuccess;
  dim3 grid((N + SW_ROWS - 1) / SW_ROWS, n_omega);
  const int threads = N >= 256 ? 256 : (N >= 128 ? 128 : (N >= 64 ? 64 : 32));
  const double *in = Pi;
  for (int k = 0; k < N; ++k) {
    int last = (k == N - 1);
    double *out = last ? C : ((k & 1) ? X1 : X0);
    sweep_step_kernel<<<grid, threads, 0, s>>>(in, out, N, k, k == 0, last, flags);
    ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    in = out;
  }
  return cudaSuccess;
}

}  // namespace ltgw

namespace ltgw {

size_t screen_blocked_scratch(int N, int n_omega) {
  return (size_t)n_omega * ((size_t)N * N + 2 * (size_t)N * SB_B + (size_t)SB_B * SB_B);
}

cudaError_t launch_screen_blocked(const double *Pi, int N, int n_omega, double *work, double *C, int *flags,
                                  cudaStream_t s, int *launches) {
  if (N <= 0 || n_omega <= 0) return cudaSuccess;
  return screen_blocked_impl<double>(Pi, N, n_omega, work, C, flags, s, launches);
}

}  // namespace ltgw
