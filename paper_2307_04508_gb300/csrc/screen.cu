// Screening of Eq. ScreenedCoulombOrbital: C(i w_j) = [1 - Pi(i w_j)]^-1 - 1
// for every frequency, by the symmetric sweep operator (Gauss-Jordan without
// pivoting, stable here because 1 - Pi is symmetric positive definite with all
// eigenvalues >= 1).  After sweeping every pivot the matrix holds -A^-1.
//
// One launch per pivot k covers all frequencies; each element of the output
// depends only on the input, so the step ping-pongs between two buffers.  The
// first step forms A = 1 - Pi on the fly, the last one writes C = -X - 1.
#include <math.h>

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
