// Bandwidth-bound helpers of the LT-GW path: pair gaps, the Laplace
// recombination of the moments onto the frequency grid, strided copies.
#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {
namespace {

__global__ void pair_gaps_kernel(const double *eps, int n_occ, int n_virt, int n_frozen,
                                 double *delta) {
  int64_t n_act = n_occ - n_frozen;
  int64_t total = n_act * n_virt;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = p / n_virt, a = p - i * n_virt;
    delta[p] = eps[n_occ + a] - eps[n_frozen + i];
  }
}

// Pi(i w_j) = alpha * sum_k exp(-w_j^2 x_k) M^k (the frequency recombination
// of the Laplace moments).  E[j][k] = exp(-w_j^2 x_k) is precomputed on the
// host.  Each thread owns one matrix element and streams the N_tau moments
// once, writing all N_omega outputs: N_tau reads + N_omega writes per element.
// That is N_omega N_tau FMAs per 8 (N_tau + N_omega) bytes, more than this
// part's FP64 rate feeds (2 FMA per clock per SM against 32 bytes per clock
// of HBM): in FP64 the kernel is bound by the FP64 pipe.  The tensor-core
// forms, whose moments carry about 1e-5 relative error, recombine with FP32
// arithmetic (Acc = float; FP64 in and out), which leaves the kernel bound by
// HBM.
template <int MAXT, typename Acc>
__global__ void recombine_kernel(const double *__restrict__ M, int n_tau,
                                 const double *__restrict__ E, int n_omega, int64_t n_elem,
                                 double alpha, double *__restrict__ Pi) {
  __shared__ Acc sE[64 * MAXT];
  for (int i = threadIdx.x; i < n_omega * n_tau; i += blockDim.x) sE[i] = (Acc)(alpha * E[i]);
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elem;
       e += (int64_t)gridDim.x * blockDim.x) {
    Acc m[MAXT];
#pragma unroll
    for (int k = 0; k < MAXT; ++k) m[k] = (k < n_tau) ? (Acc)__ldcs(M + (int64_t)k * n_elem + e) : (Acc)0;
    for (int j = 0; j < n_omega; ++j) {
      Acc s = 0;
#pragma unroll
      for (int k = 0; k < MAXT; ++k)
        if (k < n_tau) s = fma(sE[j * n_tau + k], m[k], s);
      __stcs(Pi + (int64_t)j * n_elem + e, (double)s);
    }
  }
}

__global__ void copy_cols_kernel(const double *src, int64_t lds, int64_t c0, double *dst,
                                 int64_t ldd, int rows, int64_t cols, int64_t strideS,
                                 int64_t strideD) {
  int b = blockIdx.z;
  int r = blockIdx.y;
  const double *s = src + b * strideS + (int64_t)r * lds + c0;
  double *d = dst + b * strideD + (int64_t)r * ldd;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cols;
       c += (int64_t)gridDim.x * blockDim.x)
    d[c] = s[c];
}

}  // namespace

cudaError_t launch_pair_gaps(const double *eps, int n_occ, int n_virt, int n_frozen,
                             double *delta, cudaStream_t s) {
  int64_t total = (int64_t)(n_occ - n_frozen) * n_virt;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  pair_gaps_kernel<<<blocks, 256, 0, s>>>(eps, n_occ, n_virt, n_frozen, delta);
  return cudaGetLastError();
}

// Frequencies go in launches of up to 64 (the kernel keeps E of one launch in
// shared memory); each launch re-reads the moments.
template <typename Acc>
void recombine_launch(const double *M, int n_tau, const double *E, int nj, int64_t n_elem, double alpha,
                      double *Pj, int blocks, cudaStream_t s) {
  if (n_tau <= 8)
    recombine_kernel<8, Acc><<<blocks, 256, 0, s>>>(M, n_tau, E, nj, n_elem, alpha, Pj);
  else if (n_tau <= 16)
    recombine_kernel<16, Acc><<<blocks, 256, 0, s>>>(M, n_tau, E, nj, n_elem, alpha, Pj);
  else
    recombine_kernel<32, Acc><<<blocks, 256, 0, s>>>(M, n_tau, E, nj, n_elem, alpha, Pj);
}

cudaError_t launch_recombine(const double *M, int n_tau, const double *E, int n_omega,
                             int64_t n_elem, double alpha, double *Pi, cudaStream_t s, bool fp32) {
  if (n_tau > 32 || n_tau < 1 || n_omega < 1) return cudaErrorInvalidValue;
  int blocks = (int)((n_elem + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  for (int j0 = 0; j0 < n_omega; j0 += 64) {
    const int nj = n_omega - j0 < 64 ? n_omega - j0 : 64;
    const double *Ej = E + (int64_t)j0 * n_tau;
    double *Pj = Pi + (int64_t)j0 * n_elem;
    if (fp32)
      recombine_launch<float>(M, n_tau, Ej, nj, n_elem, alpha, Pj, blocks, s);
    else
      recombine_launch<double>(M, n_tau, Ej, nj, n_elem, alpha, Pj, blocks, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_copy_cols(const double *src, int64_t lds, int64_t c0, double *dst,
                             int64_t ldd, int rows, int64_t cols, int batch,
                             int64_t strideS, int64_t strideD, cudaStream_t s) {
  if (rows <= 0 || cols <= 0 || batch <= 0) return cudaSuccess;
  int bx = (int)((cols + 255) / 256);
  if (bx > 64) bx = 64;
  dim3 grid(bx, rows, batch);
  copy_cols_kernel<<<grid, 256, 0, s>>>(src, lds, c0, dst, ldd, rows, cols, strideS, strideD);
  return cudaGetLastError();
}

}  // namespace ltgw
