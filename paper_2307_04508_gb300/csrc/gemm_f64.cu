// FP64 tiled contractions of the LT-GW path on the CUDA cores.
//
//  * scaled SYRK  C_b = alpha * A diag(s_b) A^T   (NAF metric K, Eq. nafeq;
//    Pi(i w) of Eq. Pi; Laplace moments M^m) with the per-pair scale s_b
//    computed from the pair gap inside the operand load;
//  * plain GEMM   C = A B with either operand stored K- or M/N-major
//    (NAF projection, Eq. naftrafo);
//  * GEMM + column dot  W_b[m] = sum_P B[P][m] (C_b B)[P][m]
//    (the P,Q contraction of Eq. ScreenedCoulombOrbital).
//
// GB300's FP64 rate is about 2 DFMA per clock per SM, so a 64x64 tile with a
// 4x4 register micro-tile per thread keeps the FP64 pipe saturated with
// ~0.5 B/clk/SM of global traffic; the tiles stay simple on purpose.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int PAD = 1;

template <typename T>
struct TileSmem {
  T As[BK][BM + PAD];
  T Bs[BK][BN + PAD];
  T sc[BK];
};

// Scale applied to pair (column) k of the A operand for batch entry b.
__device__ __forceinline__ double pair_scale(int mode, double d, double p0, double p1) {
  if (mode == SCALE_DIRECT) return d / (p0 * p0 + d * d);   // D / (w^2 + D^2)
  if (mode == SCALE_LAPLACE) return p1 * d * exp(-d * d * p0);  // w_m D e^{-D^2 x_m}
  if (mode == SCALE_EXPTAU) return exp(-d * p0);                // e^{-D tau_k}
  return 1.0;
}

// Accumulate one BMxBN output tile over the full K range into acc.
// A is MxK (K-major: A[m*lda+k]; else A[k*lda+m]); B is KxN (K-major:
// B[n*ldb+k]; else B[k*ldb+n]).  Scale s(k) multiplies the A operand.
template <typename T, bool A_KMAJ, bool B_KMAJ>
__device__ __forceinline__ void tile_accumulate(T acc[4][4], TileSmem<T> &sm, const T *A,
                                                int64_t lda, const T *B, int64_t ldb,
                                                int m0, int n0, int M, int N, int64_t K,
                                                int scale_mode, const double *delta, double p0,
                                                double p1) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // micro-tile rows ty + 16 i (i < n_rows) lie inside M: the zero-padded rows
  // of a tile at the edge do no FMAs (their accumulators are never stored)
  const int n_rows = min(4, max(0, (M - m0 - ty + 15) / 16));
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    if (scale_mode != SCALE_NONE && tid < BK) {
      int64_t k = k0 + tid;
      sm.sc[tid] = (k < K) ? (T)pair_scale(scale_mode, delta[k], p0, p1) : (T)0;
    }
    if (scale_mode != SCALE_NONE) __syncthreads();
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int idx = tid + r * NT;
      int m, k;
      if (A_KMAJ) { m = idx / BK; k = idx % BK; } else { k = idx / BM; m = idx % BM; }
      int gm = m0 + m;
      int64_t gk = k0 + k;
      T v = 0;
      if (gm < M && gk < K) v = A_KMAJ ? A[(int64_t)gm * lda + gk] : A[gk * lda + gm];
      if (scale_mode != SCALE_NONE) v *= sm.sc[k];
      sm.As[k][m] = v;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      int idx = tid + r * NT;
      int n, k;
      if (B_KMAJ) { n = idx / BK; k = idx % BK; } else { k = idx / BN; n = idx % BN; }
      int gn = n0 + n;
      int64_t gk = k0 + k;
      T v = 0;
      if (gn < N && gk < K) v = B_KMAJ ? B[(int64_t)gn * ldb + gk] : B[gk * ldb + gn];
      sm.Bs[k][n] = v;
    }
    __syncthreads();
    if (n_rows == 4) {
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sm.As[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = sm.Bs[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    } else if (n_rows > 0) {   // the tile's last rows: only the valid ones
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        T b[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = sm.Bs[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (i < n_rows) {
            const T a = sm.As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a, b[j], acc[i][j]);
          }
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, bool A_KMAJ, bool B_KMAJ>
__global__ void __launch_bounds__(NT) gemm_tile_kernel(GemmArgs<T> g) {
  __shared__ TileSmem<T> sm;
  const int b = blockIdx.z;
  int m0, n0;
  if (g.syrk) {
    // lower-triangle tile index -> (bi, bj), bi >= bj
    int t = blockIdx.x;
    int bi = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while (bi * (bi + 1) / 2 > t) --bi;
    int bj = t - bi * (bi + 1) / 2;
    m0 = bi * BM;
    n0 = bj * BN;
  } else {
    m0 = blockIdx.y * BM;
    n0 = blockIdx.x * BN;
  }
  const T *A, *B;
  T *C = g.C + (int64_t)b * g.strideC;
  int64_t K = g.K;
  const double *delta = g.delta;
  double p0 = 0.0, p1 = 0.0;
  if (g.ksplit > 0) {
    const int64_t k0 = (int64_t)b * g.ksplit;
    K = min(g.ksplit, g.K - k0);
    A = g.A + (A_KMAJ ? k0 : k0 * g.lda);
    B = g.B + (B_KMAJ ? k0 : k0 * g.ldb);
    if (delta) delta += k0;
  } else {
    A = g.A + (int64_t)b * g.strideA;
    B = g.B + (int64_t)b * g.strideB;
    p0 = g.batch_p0 ? g.batch_p0[b] : 0.0;
    p1 = g.batch_p1 ? g.batch_p1[b] : 0.0;
  }
  T acc[4][4] = {};
  tile_accumulate<T, A_KMAJ, B_KMAJ>(acc, sm, A, g.lda, B, g.ldb, m0, n0, g.M, g.N, K,
                                     g.scale_mode, delta, p0, p1);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      T v = (T)g.alpha * acc[i][j];
      if (g.beta != 0.0) v += (T)g.beta * C[(int64_t)gm * g.ldc + gn];
      if (g.syrk) {
        if (gm >= gn) {
          C[(int64_t)gm * g.ldc + gn] = v;
          C[(int64_t)gn * g.ldc + gm] = v;
        }
      } else {
        C[(int64_t)gm * g.ldc + gn] = v;
      }
    }
  }
}

// W[b][t][m] = sum_P Bt[t][P][m] * sum_Q C[b][P][Q] Bt[t][Q][m]
// grid: x = column tile of m, y = target t, z = frequency b.
__global__ void __launch_bounds__(NT) gemm_coldot_kernel(ColDotArgs g) {
  __shared__ TileSmem<double> sm;
  __shared__ double red[16][BN];
  const int b = blockIdx.z, t = blockIdx.y;
  const int n0 = blockIdx.x * BN;
  const double *Cb = g.C + (int64_t)b * g.strideC;
  const double *Bt = g.Bt + (int64_t)t * g.strideBt;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double part[4] = {0, 0, 0, 0};
  for (int m0 = 0; m0 < g.N; m0 += BM) {
    double acc[4][4] = {};
    tile_accumulate<double, true, false>(acc, sm, Cb, g.ldc, Bt, g.ldb, m0, n0, g.N, g.ncols, g.N,
                                 SCALE_NONE, nullptr, 0.0, 0.0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int gm = m0 + ty + 16 * i;
      if (gm >= g.N) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gn = n0 + tx + 16 * j;
        if (gn < g.ncols) part[j] = fma(Bt[(int64_t)gm * g.ldb + gn], acc[i][j], part[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) red[ty][tx + 16 * j] = part[j];
  __syncthreads();
  if (threadIdx.x < BN) {
    int gn = n0 + threadIdx.x;
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 16; ++r) s += red[r][threadIdx.x];
    if (gn < g.ncols) g.W[((int64_t)b * g.n_tgt + t) * g.ldw + gn] = s;
  }
}

// Gram blocks of the reflector panels: panel q holds rows j0 = q*nb ..
// j0+nbq-1 of V (row j is zero outside columns j+1..n-1), and chunk c covers
// its columns r0 + c*ks .. r0 + (c+1)*ks - 1 with r0 = j0 + 1.  The chunk's
// partial of G_q = V_q V_q^T goes to P + (c * npanel + q) * nb * nb with
// leading dimension nbq; chunks past the panel's end write zeros, so one sum
// over every chunk index gives every panel's G.  grid: x = chunk, y = panel.
__global__ void __launch_bounds__(NT) gram_panels_kernel(const double *__restrict__ V, int n, int nref,
                                                         int nb, int64_t ks, double *__restrict__ P) {
  __shared__ TileSmem<double> sm;
  const int c = blockIdx.x, q = blockIdx.y;
  const int j0 = q * nb, nbq = min(nb, nref - j0);
  const int64_t r0 = j0 + 1, len = n - r0, k0 = (int64_t)c * ks;
  double acc[4][4] = {};
  if (k0 < len) {
    const double *A = V + (int64_t)j0 * n + r0 + k0;
    tile_accumulate<double, true, true>(acc, sm, A, n, A, n, 0, 0, nbq, nbq, min(ks, len - k0), SCALE_NONE,
                                        nullptr, 0.0, 0.0);
  }
  double *Pq = P + ((int64_t)c * gridDim.y + q) * nb * nb;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = tx + 16 * j;
      if (gm < nbq && gn < nbq) Pq[gm * nbq + gn] = acc[i][j];
    }
  }
}

}  // namespace

cudaError_t launch_gram_panels(const double *V, int n, int nref, int nb, int64_t ks, double *P, cudaStream_t s) {
  if (nref <= 0 || n < 2) return cudaSuccess;
  if (nb <= 0 || nb > BM || ks <= 0) return cudaErrorInvalidValue;
  const int npanel = (nref + nb - 1) / nb;
  const int64_t nchunk = (n - 1 + ks - 1) / ks;   // chunks of the longest panel (q = 0)
  gram_panels_kernel<<<dim3((unsigned)nchunk, (unsigned)npanel), NT, 0, s>>>(V, n, nref, nb, ks, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gemm(const GemmArgs<T> &g, int batch, bool a_kmaj, bool b_kmaj, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return cudaSuccess;
  if (sizeof(T) != sizeof(double) && g.scale_mode != SCALE_NONE) return cudaErrorInvalidValue;
  dim3 grid;
  if (g.syrk) {
    int tm = ceil_div(g.M, BM);
    grid = dim3((unsigned)(tm * (tm + 1) / 2), 1, (unsigned)batch);
  } else {
    grid = dim3((unsigned)ceil_div(g.N, BN), (unsigned)ceil_div(g.M, BM), (unsigned)batch);
  }
  if (a_kmaj && b_kmaj) gemm_tile_kernel<T, true, true><<<grid, NT, 0, s>>>(g);
  else if (a_kmaj && !b_kmaj) gemm_tile_kernel<T, true, false><<<grid, NT, 0, s>>>(g);
  else if (!a_kmaj && b_kmaj) gemm_tile_kernel<T, false, true><<<grid, NT, 0, s>>>(g);
  else gemm_tile_kernel<T, false, false><<<grid, NT, 0, s>>>(g);
  return cudaGetLastError();
}
template cudaError_t launch_gemm<double>(const GemmArgs<double> &, int, bool, bool, cudaStream_t);

cudaError_t launch_gemm_coldot(const ColDotArgs &g, int n_batch, cudaStream_t s) {
  if (g.N <= 0 || g.ncols <= 0 || g.n_tgt <= 0 || n_batch <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(g.ncols, BN), (unsigned)g.n_tgt, (unsigned)n_batch);
  gemm_coldot_kernel<<<grid, NT, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace ltgw
