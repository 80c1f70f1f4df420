// Seeded synthetic-input generator, device side: the same Philox4x32-10
// counters, keys and Box-Muller normals as philox_gen.c (Salmon et al.,
// SC'11, written from the published definition), for workloads too large to
// generate on the host.  No GW arithmetic lives here.
//
//   key     = (seed & 0xffffffff, (seed >> 32) + stream)
//   counter = (c0, c1, c2, 0)
//   normal  = sqrt(-2 ln u1) cos(2 pi u2), u1 = (x0 + 1) 2^-32, u2 = x1 2^-32
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ double normal_at(uint32_t k0, uint32_t k1, uint32_t a, uint32_t b, uint32_t c) {
  uint32_t x[4] = {a, b, c, 0u};
  philox(x, k0, k1);
  const double u1 = ((double)x[0] + 1.0) * 2.3283064365386963e-10;
  const double u2 = (double)x[1] * 2.3283064365386963e-10;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// out[r][(i - i0) * n_virt + a] = normal(r, i, n_occ + a), r < rows
__global__ void pair_normals_ov_kernel(uint32_t k0, uint32_t k1, int64_t rows, int64_t n_occ, int64_t n_virt,
                                       int64_t i0, int64_t i1, double *out) {
  const int64_t cols = (i1 - i0) * n_virt, total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, q = e - r * cols;
    const int64_t i = i0 + q / n_virt, a = q % n_virt;
    out[e] = normal_at(k0, k1, (uint32_t)r, (uint32_t)i, (uint32_t)(n_occ + a));
  }
}

// out[r][m] = normal(r, min(p, m), max(p, m))
__global__ void pair_normals_row_kernel(uint32_t k0, uint32_t k1, int64_t rows, int64_t n_orb, int64_t p,
                                        double *out) {
  const int64_t total = rows * n_orb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n_orb, m = e - r * n_orb;
    const int64_t lo = p < m ? p : m, hi = p < m ? m : p;
    out[e] = normal_at(k0, k1, (uint32_t)r, (uint32_t)lo, (uint32_t)hi);
  }
}

// out[r][c] = normal(r, c, 0)
__global__ void normal_matrix_kernel(uint32_t k0, uint32_t k1, int64_t rows, int64_t cols, double *out) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    out[e] = normal_at(k0, k1, (uint32_t)r, (uint32_t)c, 0u);
  }
}

int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

}  // namespace

extern "C" {

int synth_dev_pair_normals_ov(uint64_t seed, uint32_t stream, int64_t rows, int64_t n_occ, int64_t n_virt,
                              int64_t i0, int64_t i1, double *out, void *cuda_stream) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) + stream;
  pair_normals_ov_kernel<<<grid_for(rows * (i1 - i0) * n_virt), 256, 0, (cudaStream_t)cuda_stream>>>(
      k0, k1, rows, n_occ, n_virt, i0, i1, out);
  return (int)cudaGetLastError();
}

int synth_dev_pair_normals_row(uint64_t seed, uint32_t stream, int64_t rows, int64_t n_orb, int64_t p, double *out,
                               void *cuda_stream) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) + stream;
  pair_normals_row_kernel<<<grid_for(rows * n_orb), 256, 0, (cudaStream_t)cuda_stream>>>(k0, k1, rows, n_orb, p, out);
  return (int)cudaGetLastError();
}

int synth_dev_normal_matrix(uint64_t seed, uint32_t stream, int64_t rows, int64_t cols, double *out,
                            void *cuda_stream) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) + stream;
  normal_matrix_kernel<<<grid_for(rows * cols), 256, 0, (cudaStream_t)cuda_stream>>>(k0, k1, rows, cols, out);
  return (int)cudaGetLastError();
}

}  // extern "C"
