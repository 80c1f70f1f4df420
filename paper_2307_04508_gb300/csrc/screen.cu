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

__global__ void sweep_step_kernel(const double *__restrict__ in, double *__restrict__ out,
                                  int N, int k, int first, int last, int *flags) {
  const int b = blockIdx.y;
  const int64_t NN = (int64_t)N * N;
  const double *X = in + b * NN;
  double *Y = out + b * NN;
  auto at = [&](int r, int c) -> double {
    double v = X[(int64_t)r * N + c];
    if (first) v = (r == c ? 1.0 : 0.0) - v;
    return v;
  };
  const double p = at(k, k);
  if (blockIdx.x == 0 && threadIdx.x == 0 && !(p > 0.0 && isfinite(p)))
    atomicExch(&flags[FLAG_NOT_SPD], 1);
  const double rp = 1.0 / p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < NN;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / N), j = (int)(e - (int64_t)i * N);
    double r;
    if (i == k && j == k) r = -rp;
    else if (i == k) r = at(k, j) * rp;
    else if (j == k) r = at(i, k) * rp;
    else r = at(i, j) - at(i, k) * at(k, j) * rp;
    if (last) r = -r - (i == j ? 1.0 : 0.0);
    Y[e] = r;
  }
}

}  // namespace

cudaError_t launch_screen(const double *Pi, int N, int n_omega, double *X0, double *X1,
                          double *C, int *flags, cudaStream_t s, int *launches) {
  if (N <= 0 || n_omega <= 0) return cudaSuccess;
  const int64_t NN = (int64_t)N * N;
  int bx = (int)((NN + 255) / 256);
  int cap = (152 * 8 + n_omega - 1) / n_omega;
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  dim3 grid(bx, n_omega);
  const double *in = Pi;
  for (int k = 0; k < N; ++k) {
    int last = (k == N - 1);
    double *out = last ? C : ((k & 1) ? X1 : X0);
    sweep_step_kernel<<<grid, 256, 0, s>>>(in, out, N, k, k == 0, last, flags);
    ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    in = out;
  }
  return cudaSuccess;
}

}  // namespace ltgw
