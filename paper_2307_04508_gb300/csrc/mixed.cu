// Bandwidth-bound helpers of the mixed-precision (split-BF16) path: FP32
// padded operand copies, the per-pair scale table of the polarisability
// (fused into the tensor-core operand load), and the FP64 reduction of the
// split-K partial tiles into full symmetric matrices.
#include <math.h>

#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <climits>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {
namespace {

__global__ void to_f32_padded_kernel(const double *__restrict__ src, int64_t lds, int rows, int64_t cols,
                                     float *__restrict__ dst, int64_t cols_p) {
  const int r = blockIdx.y;
  const double *s = src + (int64_t)r * lds;
  float *d = dst + (int64_t)r * cols_p;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cols_p;
       c += (int64_t)gridDim.x * blockDim.x)
    d[c] = (r < rows && c < cols) ? (float)s[c] : 0.0f;
}

__global__ void scale_table_kernel(const double *__restrict__ delta, int64_t K, int64_t Kp,
                                   const double *__restrict__ p0, const double *__restrict__ p1,
                                   int mode, float *__restrict__ scale) {
  const int t = blockIdx.y;
  const double a = p0 ? p0[t] : 0.0, b = p1 ? p1[t] : 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Kp;
       k += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (k < K) {
      const double d = delta ? delta[k] : 0.0;
      v = (mode == SCALE_DIRECT) ? d / (a * a + d * d)
          : (mode == SCALE_LAPLACE) ? b * d * exp(-d * d * a)
          : (mode == SCALE_EXPTAU) ? exp(-d * a) : 1.0;
    }
    scale[(int64_t)t * Kp + k] = (float)v;
  }
}

// One thread per lower-triangle element (i >= j) of one matrix t.  Partial
// tiles are 128 x 128, four scales per group.
// Sum of FP32 partials as an unevaluated pair hi + lo of FP32 numbers
// (Knuth's TwoSum per term; about 48 significant bits): the FP32 partials
// carry errors of 2^-24 of their own, so the pair's sum equals their FP64 sum
// far below that, and FP32 additions run many times faster than FP64 ones on
// this part (where the FP64 sum made the reductions FP64-bound).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

__global__ void tc_reduce_sym_kernel(const double *__restrict__ partial, const float *__restrict__ partial32,
                                     int splits, int groups, int n_tiles, const int *__restrict__ tile_index,
                                     int nJ, int N, int nt_group, int colmajor, double alpha, double beta,
                                     double *__restrict__ M) {
  const int t = blockIdx.y;
  const int grp = t / nt_group, slot = t % nt_group;
  const int64_t NN = (int64_t)N * N;
  const int64_t ntri = (int64_t)N * (N + 1) / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ntri;
       e += (int64_t)gridDim.x * blockDim.x) {
    // e -> (i, j), i >= j, row-major lower triangle (an FP32 estimate of the
    // row, corrected by integer tests)
    int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((int64_t)(a + 1) * (a + 2) / 2 <= e) ++a;
    while ((int64_t)a * (a + 1) / 2 > e) --a;
    const int b = (int)(e - (int64_t)a * (a + 1) / 2);
    // (a, b), a >= b, b fastest; column-major tiles take (i, j) = (N-1-b, N-1-a) so that
    // consecutive threads read consecutive rows of one column
    const int i = colmajor ? N - 1 - b : a, j = colmajor ? N - 1 - a : b;
    const int tile = tile_index[(i / 128) * nJ + (j / 128)];
    const int64_t in_tile = colmajor ? (int64_t)(j % 128) * 128 + (i % 128) : (int64_t)(i % 128) * 128 + (j % 128);
    double acc = 0.0;
    if (partial32) {
      float hi = 0.0f, lo = 0.0f;
      for (int s = 0; s < splits; ++s)
        two_sum_acc(hi, lo, partial32[((((int64_t)s * groups + grp) * nt_group + slot) * n_tiles + tile) * (128 * 128) +
                                      in_tile]);
      acc = (double)hi + (double)lo;
    } else {
      for (int s = 0; s < splits; ++s)
        acc += partial[((((int64_t)s * groups + grp) * nt_group + slot) * n_tiles + tile) * (128 * 128) + in_tile];
    }
    acc *= alpha;
    if (beta != 0.0) acc += beta * M[t * NN + (int64_t)i * N + j];
    M[t * NN + (int64_t)i * N + j] = acc;
    M[t * NN + (int64_t)j * N + i] = acc;
  }
}

// dst[c][r] = src[r][c0 + c] (FP64 -> FP32), zero padding, 32 x 32 tiles through smem.
__global__ void to_f32_transposed_kernel(const double *__restrict__ src, int64_t lds, int64_t c0, int rows,
                                         int cols, float *__restrict__ dst, int rows_p, int cols_p,
                                         int64_t strideS, int64_t strideD) {
  __shared__ float tile[32][33];
  const int b = blockIdx.z;
  const double *S = src + b * strideS + c0;
  float *D = dst + b * strideD;
  const int r0 = blockIdx.y * 32, cb = blockIdx.x * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + q, c = cb + threadIdx.x;
    tile[q][threadIdx.x] = (r < rows && c < cols) ? (float)S[(int64_t)r * lds + c] : 0.0f;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int c = cb + q, r = r0 + threadIdx.x;
    if (c < cols_p && r < rows_p) D[(int64_t)c * rows_p + r] = tile[threadIdx.x][q];
  }
}

// dst[c][r] = src[r][c0 + c] in FP64, r < rows, c < cols (batched).
__global__ void transpose_f64_kernel(const double *__restrict__ src, int64_t lds, int64_t c0, int rows, int cols,
                                     double *__restrict__ dst, int64_t ldd, int64_t strideS, int64_t strideD) {
  __shared__ double tile[32][33];
  const int b = blockIdx.z;
  const double *S = src + b * strideS + c0;
  double *D = dst + b * strideD;
  const int r0 = blockIdx.y * 32, cb = blockIdx.x * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + q, c = cb + threadIdx.x;
    if (r < rows && c < cols) tile[q][threadIdx.x] = S[(int64_t)r * lds + c];
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int c = cb + q, r = r0 + threadIdx.x;
    if (c < cols && r < rows) D[(int64_t)c * ldd + r] = tile[threadIdx.x][q];
  }
}

// Full-grid partial tiles -> FP64 and/or FP32 padded output, per group.
__global__ void tc_reduce_full_kernel(const double *__restrict__ partial, const float *__restrict__ partial32,
                                      int splits, int groups, int n_tiles, int nJ, int rows, int cols,
                                      double alpha, double *__restrict__ out64, int64_t ld64, int64_t stride64,
                                      float *__restrict__ out32, int64_t ld32, int64_t cols32, int rows_p32,
                                      int64_t stride32, double beta) {
  const int g = blockIdx.z;
  const int r = blockIdx.y;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < (out32 ? cols32 : cols);
       c += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (r < rows && c < cols) {
      const int tile = (r / 128) * nJ + (int)(c / 128);
      const int64_t off = (int64_t)(r % 128) * 128 + (c % 128);
      if (partial32) {
        float hi = 0.0f, lo = 0.0f;
        for (int s = 0; s < splits; ++s)
          two_sum_acc(hi, lo, partial32[(((int64_t)s * groups + g) * n_tiles + tile) * (128 * 128) + off]);
        acc = (double)hi + (double)lo;
      } else {
        for (int s = 0; s < splits; ++s) acc += partial[(((int64_t)s * groups + g) * n_tiles + tile) * (128 * 128) + off];
      }
      acc *= alpha;
      if (out64) {
        double *o = out64 + g * stride64 + (int64_t)r * ld64 + c;
        if (beta != 0.0) acc += beta * *o;
        *o = acc;
      }
    }
    if (out32 && r < rows_p32) out32[g * stride32 + (int64_t)r * ld32 + c] = (float)acc;
  }
}

__global__ void tc_reduce_coldot_kernel(const float *__restrict__ cd, int splits, int groups, int n_tile_rows,
                                        int cols_p, int cols, double *__restrict__ W, int64_t ldw) {
  const int g = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    float hi = 0.0f, lo = 0.0f;
    for (int s = 0; s < splits; ++s)
      for (int I = 0; I < n_tile_rows; ++I) two_sum_acc(hi, lo, cd[(((int64_t)s * groups + g) * n_tile_rows + I) * cols_p + c]);
    W[(int64_t)g * ldw + c] = (double)hi + (double)lo;
  }
}

}  // namespace

cudaError_t launch_to_f32_padded(const double *src, int64_t lds, int rows, int64_t cols, float *dst,
                                 int rows_p, int64_t cols_p, cudaStream_t s) {
  if (rows_p <= 0 || cols_p <= 0) return cudaSuccess;
  int bx = (int)((cols_p + 255) / 256);
  if (bx > 64) bx = 64;
  dim3 grid(bx, rows_p);
  to_f32_padded_kernel<<<grid, 256, 0, s>>>(src, lds, rows, cols, dst, cols_p);
  return cudaGetLastError();
}

cudaError_t launch_scale_table(const double *delta, int64_t K, int64_t Kp, int n_t, const double *p0,
                               const double *p1, int mode, float *scale, cudaStream_t s) {
  if (n_t <= 0) return cudaSuccess;
  int bx = (int)((Kp + 255) / 256);
  if (bx > 152) bx = 152;
  dim3 grid(bx, n_t);
  scale_table_kernel<<<grid, 256, 0, s>>>(delta, K, Kp, p0, p1, mode, scale);
  return cudaGetLastError();
}

cudaError_t launch_tc_reduce_sym(const double *partial, const float *partial32, int splits, int groups,
                                 int n_tiles, const int *tile_index, int nJ, int n_t, int N, double alpha,
                                 double *M, cudaStream_t s, double beta, int nt_group, int colmajor) {
  if (N <= 0 || n_t <= 0) return cudaSuccess;
  int64_t ntri = (int64_t)N * (N + 1) / 2;
  int bx = (int)((ntri + 255) / 256);
  if (bx > 152 * 4) bx = 152 * 4;
  dim3 grid(bx, n_t);
  if (nt_group < 1 || (n_t + nt_group - 1) / nt_group != groups) return cudaErrorInvalidValue;
  tc_reduce_sym_kernel<<<grid, 256, 0, s>>>(partial, partial32, splits, groups, n_tiles, tile_index, nJ, N,
                                            nt_group, colmajor, alpha, beta, M);
  return cudaGetLastError();
}

}  // namespace ltgw

namespace ltgw {

cudaError_t launch_to_f32_transposed(const double *src, int64_t lds, int64_t c0, int rows, int cols,
                                     float *dst, int rows_p, int cols_p, int batch, int64_t strideS,
                                     int64_t strideD, cudaStream_t s) {
  if (rows_p <= 0 || cols_p <= 0 || batch <= 0) return cudaSuccess;
  dim3 block(32, 8), grid((cols_p + 31) / 32, (rows_p + 31) / 32, batch);
  to_f32_transposed_kernel<<<grid, block, 0, s>>>(src, lds, c0, rows, cols, dst, rows_p, cols_p, strideS, strideD);
  return cudaGetLastError();
}

cudaError_t launch_tc_reduce_full(const double *partial, const float *partial32, int splits, int groups,
                                  int n_tiles, int nJ, int rows, int cols, double alpha, double *out64,
                                  int64_t ld64, int64_t stride64, float *out32, int64_t ld32,
                                  int rows_p32, int64_t stride32, cudaStream_t s, int64_t cols32, double beta) {
  if (cols32 < 0) cols32 = ld32;
  const int nrows = out32 ? std::max(rows, rows_p32) : rows;
  const int64_t ncols = out32 ? cols32 : cols;
  if (nrows <= 0 || ncols <= 0 || groups <= 0) return cudaSuccess;
  int bx = (int)((ncols + 255) / 256);
  if (bx > 64) bx = 64;
  dim3 grid(bx, nrows, groups);
  tc_reduce_full_kernel<<<grid, 256, 0, s>>>(partial, partial32, splits, groups, n_tiles, nJ, rows, cols, alpha,
                                             out64, ld64, stride64, out32, ld32, cols32, rows_p32, stride32, beta);
  return cudaGetLastError();
}

cudaError_t launch_tc_reduce_full_acc(const double *partial, const float *partial32, int splits, int groups,
                                      int n_tiles, int nJ, int rows, int cols, double alpha, double *out64,
                                      int64_t ld64, double beta, cudaStream_t s) {
  return launch_tc_reduce_full(partial, partial32, splits, groups, n_tiles, nJ, rows, cols, alpha, out64, ld64, 0,
                               nullptr, 0, 0, 0, s, -1, beta);
}

cudaError_t launch_transpose_f64(const double *src, int64_t lds, int64_t c0, int rows, int cols, double *dst,
                                 int64_t ldd, int batch, int64_t strideS, int64_t strideD, cudaStream_t s) {
  if (rows <= 0 || cols <= 0 || batch <= 0) return cudaSuccess;
  dim3 block(32, 8), grid((cols + 31) / 32, (rows + 31) / 32, batch);
  transpose_f64_kernel<<<grid, block, 0, s>>>(src, lds, c0, rows, cols, dst, ldd, strideS, strideD);
  return cudaGetLastError();
}

cudaError_t launch_tc_reduce_coldot(const float *cd_out, int splits, int groups, int n_tile_rows, int cols_p,
                                    int cols, double *W, int64_t ldw, cudaStream_t s) {
  if (cols <= 0 || groups <= 0) return cudaSuccess;
  int bx = (cols + 255) / 256;
  if (bx > 64) bx = 64;
  dim3 grid(bx, groups);
  tc_reduce_coldot_kernel<<<grid, 256, 0, s>>>(cd_out, splits, groups, n_tile_rows, cols_p, cols, W, ldw);
  return cudaGetLastError();
}


namespace {
__global__ void split_bf16_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ hi,
                                  __nv_bfloat16 *__restrict__ lo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}
}  // namespace

cudaError_t launch_split_bf16(const float *x, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  split_bf16_kernel<<<(int)blocks, 256, 0, s>>>(x, hi, lo, n);
  return cudaGetLastError();
}

namespace {
constexpr int Q8_THREADS = 256;
constexpr float E4M3_MAX = 448.0f;   // largest finite FP8 E4M3 value

__device__ __forceinline__ float block_max(float v, float *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float m = 0.0f;
#pragma unroll
  for (int i = 0; i < Q8_THREADS / 32; ++i) m = fmaxf(m, red[i]);
  return m;
}

// four E4M3 codes (round to nearest even, saturating) of x * inv, packed low byte first
__device__ __forceinline__ uint32_t e4m3x4(float4 x, float inv) {
  const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(x.x * inv, x.y * inv), __NV_SATFINITE, __NV_E4M3);
  const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(x.z * inv, x.w * inv), __NV_SATFINITE, __NV_E4M3);
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

// E4M3 values of four packed codes (exact in FP32)
__device__ __forceinline__ float4 e4m3x4_value(uint32_t c) {
  const __half2_raw a = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(c & 0xffffu), __NV_E4M3);
  const __half2_raw b = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(c >> 16), __NV_E4M3);
  const float2 fa = __half22float2(__half2(a)), fb = __half22float2(__half2(b));
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}

// Codes of x * inv (one term), or (split) of its two-term expansion h + l
// with h = e4m3(x inv) and l = e4m3(x inv - h) (exact in FP32), both in the
// row's scaled units: the row's three segments of Kq codes are written as
// pattern[0..2] of {h, l} (A operands h | l | h, B operands h | h | l, so that
// one accumulator sums h_a h_b + l_a h_b + h_a l_b).
__device__ __forceinline__ void write_codes(uint32_t *row, int64_t k, int64_t q4, float4 x, float inv, int split,
                                            bool a_pattern) {
  const uint32_t h = e4m3x4(x, inv);
  row[k] = h;
  if (!split) return;
  const float4 hv = e4m3x4_value(h);
  const float4 r = make_float4(x.x * inv - hv.x, x.y * inv - hv.y, x.z * inv - hv.z, x.w * inv - hv.w);
  const uint32_t l = e4m3x4(r, 1.0f);
  row[q4 + k] = a_pattern ? l : h;
  row[2 * q4 + k] = a_pattern ? h : l;
}

// One block per row r of X [rows][Kp] (FP32; Kp a multiple of 4): the row's
// scale inv = 448 / max_k |X_rk| and codes qb[r][k] = e4m3(X_rk inv); for each
// of the n_t factor rows S[t] the products p = X_rk S_tk (FP32) get their own
// scale and codes qa[t][r][k].  De-scales 1 / inv (0 for a zero row) go to
// ds_b[r] and ds_a[t][r]; code columns Kp..Kq-1 are zero.  split: each code
// row holds three segments of Kq (the two-term expansion, write_codes).
template <int MAXT>
__global__ void __launch_bounds__(Q8_THREADS)
    fp8_quantize_kernel(const float *__restrict__ X, int64_t Kp, int64_t Kq, const float *__restrict__ S, int n_t,
                        int rows, uint8_t *__restrict__ qa, uint8_t *__restrict__ qb, float *__restrict__ ds_a,
                        float *__restrict__ ds_b, int split) {
  __shared__ float red[Q8_THREADS / 32];
  __shared__ float inv_s[MAXT + 1];
  const int r = blockIdx.x;
  const float4 *xr = reinterpret_cast<const float4 *>(X + (int64_t)r * Kp);
  const int64_t n4 = Kp / 4, q4 = Kq / 4;
  float mb = 0.0f, ma[MAXT];
#pragma unroll
  for (int t = 0; t < MAXT; ++t) ma[t] = 0.0f;
  for (int64_t k = threadIdx.x; k < n4; k += Q8_THREADS) {
    const float4 x = xr[k];
    mb = fmaxf(mb, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
#pragma unroll
    for (int t = 0; t < MAXT; ++t) {
      if (t < n_t) {
        const float4 sv = reinterpret_cast<const float4 *>(S + (int64_t)t * Kp)[k];
        ma[t] = fmaxf(ma[t], fmaxf(fmaxf(fabsf(x.x * sv.x), fabsf(x.y * sv.y)),
                                   fmaxf(fabsf(x.z * sv.z), fabsf(x.w * sv.w))));
      }
    }
  }
  mb = block_max(mb, red);
  if (threadIdx.x == 0) inv_s[MAXT] = mb > 0.0f ? E4M3_MAX / mb : 0.0f;
#pragma unroll
  for (int t = 0; t < MAXT; ++t) {
    if (t < n_t) {
      const float m = block_max(ma[t], red);
      if (threadIdx.x == 0) inv_s[t] = m > 0.0f ? E4M3_MAX / m : 0.0f;
    }
  }
  __syncthreads();
  const float invb = inv_s[MAXT];
  if (threadIdx.x == 0) {
    ds_b[r] = invb > 0.0f ? 1.0f / invb : 0.0f;
    for (int t = 0; t < n_t; ++t) ds_a[(int64_t)t * rows + r] = inv_s[t] > 0.0f ? 1.0f / inv_s[t] : 0.0f;
  }
  const int64_t Ks = split ? 3 * Kq : Kq;   // codes per row
  uint32_t *qbr = qb ? reinterpret_cast<uint32_t *>(qb + (int64_t)r * Ks) : nullptr;
  for (int64_t k = threadIdx.x; k < q4; k += Q8_THREADS) {
    if (k >= n4) {
      for (int seg = 0; seg < (split ? 3 : 1); ++seg) {
        if (qbr) qbr[seg * q4 + k] = 0u;
        for (int t = 0; t < n_t; ++t) reinterpret_cast<uint32_t *>(qa + ((int64_t)t * rows + r) * Ks)[seg * q4 + k] = 0u;
      }
      continue;
    }
    const float4 x = xr[k];
    if (qbr) write_codes(qbr, k, q4, x, invb, split, false);
#pragma unroll
    for (int t = 0; t < MAXT; ++t) {
      if (t < n_t) {
        const float4 sv = reinterpret_cast<const float4 *>(S + (int64_t)t * Kp)[k];
        const float4 p = make_float4(x.x * sv.x, x.y * sv.y, x.z * sv.z, x.w * sv.w);
        write_codes(reinterpret_cast<uint32_t *>(qa + ((int64_t)t * rows + r) * Ks), k, q4, p, inv_s[t], split, true);
      }
    }
  }
}
// One block per row r of X [rows][Kp]: codes of X itself as an A operand
// (split: segments h | l | h), de-scale to ds[r].
__global__ void __launch_bounds__(Q8_THREADS)
    fp8_quantize_a_kernel(const float *__restrict__ X, int64_t Kp, int64_t Kq, int rows, uint8_t *__restrict__ q,
                          float *__restrict__ ds, int split) {
  __shared__ float red[Q8_THREADS / 32];
  const int r = blockIdx.x;
  const float4 *xr = reinterpret_cast<const float4 *>(X + (int64_t)r * Kp);
  const int64_t n4 = Kp / 4, q4 = Kq / 4;
  float m = 0.0f;
  for (int64_t k = threadIdx.x; k < n4; k += Q8_THREADS) {
    const float4 x = xr[k];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
  }
  m = block_max(m, red);
  const float inv = m > 0.0f ? E4M3_MAX / m : 0.0f;
  if (threadIdx.x == 0) ds[r] = inv > 0.0f ? 1.0f / inv : 0.0f;
  const int64_t Ks = split ? 3 * Kq : Kq;
  uint32_t *qr = reinterpret_cast<uint32_t *>(q + (int64_t)r * Ks);
  for (int64_t k = threadIdx.x; k < q4; k += Q8_THREADS) {
    if (k >= n4) {
      for (int seg = 0; seg < (split ? 3 : 1); ++seg) qr[seg * q4 + k] = 0u;
      continue;
    }
    write_codes(qr, k, q4, xr[k], inv, split, true);
  }
}
// One block per row r of X (FP64, row stride ld, `cols` columns; with
// colscale, X_rk colscale_k, one FP64 product): e_r = the exponent of the
// row's largest magnitude m (m = f 2^e_r, f in [0.5, 1); 0 for a zero row),
// the fixed-point row Q = rint(X_r 2^(7 s - e_r)) (exact scaling, ties to
// even), and Q in s balanced base-128 digits, the least significant in
// [-64, 63], the leading one in [-128, 128]: digit i (1 = leading) goes to
// dA[i-1][r][k] (FP32) and/or dB[i-1][r][k] (BF16), exact either way; columns
// cols..Kp-1 are zero.  exps[r] = e_r.
__device__ __forceinline__ double scaled_entry(const double *xr, const double *colscale, int64_t k) {
  return colscale ? __dmul_rn(xr[k], colscale[k]) : xr[k];
}

__global__ void __launch_bounds__(256)
    slice_rows_kernel(const double *__restrict__ X, int64_t ld, int64_t cols, int64_t Kp, int s,
                      int64_t slice_stride, float *__restrict__ dA, __nv_bfloat16 *__restrict__ dB,
                      int *__restrict__ exps, const double *__restrict__ colscale) {
  __shared__ unsigned long long red[8];
  const int r = blockIdx.x;
  const double *xr = X + (int64_t)r * ld;
  unsigned long long mb = 0ull;   // |x| bit patterns order like the values
  for (int64_t k = threadIdx.x; k < cols; k += blockDim.x)
    mb = max(mb, (unsigned long long)__double_as_longlong(scaled_entry(xr, colscale, k)) & 0x7fffffffffffffffull);
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_down_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mb;
  __syncthreads();
  mb = 0ull;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mb = max(mb, red[w]);
  int e = 0;
  if (mb != 0ull) frexp(__longlong_as_double((long long)mb), &e);   // m = f 2^e, f in [0.5, 1)
  if (threadIdx.x == 0 && exps) exps[r] = e;
  for (int64_t k = threadIdx.x; k < Kp; k += blockDim.x) {
    // ldexp scales exactly without forming 2^(7 s - e), which overflows for tiny rows
    long long Q = (k < cols && mb != 0ull) ? __double2ll_rn(ldexp(scaled_entry(xr, colscale, k), 7 * s - e)) : 0ll;
    for (int i = s - 1; i >= 1; --i) {   // balanced digits, least significant first
      const long long t = (Q + 64) >> 7;
      const float d = (float)(Q - (t << 7));
      if (dA) dA[i * slice_stride + (int64_t)r * Kp + k] = d;
      if (dB) dB[i * slice_stride + (int64_t)r * Kp + k] = __float2bfloat16_rn(d);
      Q = t;
    }
    if (dA) dA[(int64_t)r * Kp + k] = (float)Q;
    if (dB) dB[(int64_t)r * Kp + k] = __float2bfloat16_rn((float)Q);
  }
}

// FP64 per-pair factors f[t][k] of the Pi contraction, each operation rounded
// once (no fused multiply-add): Delta / (w_t^2 + Delta^2) (direct, p0 = w),
// (w_t Delta) exp(-Delta Delta x_t) (Laplace, p0 = x, p1 = w), exp(-Delta tau_t)
// (imaginary time, p0 = tau).
__global__ void pi_factor64_kernel(const double *__restrict__ delta, int64_t K, const double *__restrict__ p0,
                                   const double *__restrict__ p1, int mode, double *__restrict__ f) {
  const int t = blockIdx.y;
  const double a = p0[t], b = p1 ? p1[t] : 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
    const double d = delta[k];
    double v;
    if (mode == SCALE_DIRECT)
      v = __ddiv_rn(d, __dadd_rn(__dmul_rn(a, a), __dmul_rn(d, d)));
    else if (mode == SCALE_LAPLACE)
      v = __dmul_rn(__dmul_rn(b, d), exp(__dmul_rn(__dmul_rn(-d, d), a)));
    else
      v = exp(__dmul_rn(-d, a));   // SCALE_EXPTAU: e^{-Delta tau_t}
    f[(int64_t)t * K + k] = v;
  }
}

// D[r][c] = beta D[r][c] + S[r][c] 2^(ea[r] + eb[c]) for r < rows, c < cols
// (the scaling is exact; S may be D with beta = 0).  lower: the product of a
// lower-tile form (S symmetric, rows == cols) whose mirrored upper entries
// must take the lower entry's scale 2^(ea[r] + eb[c]), r >= c: only c <= r
// is read, and each value is written to (r, c) and (c, r).
__global__ void scale_exp2_kernel(const double *S, int64_t lds, double *D, int64_t ldd, int rows, int cols,
                                  const int *__restrict__ ea, const int *__restrict__ eb, double beta, int lower) {
  const int r = blockIdx.y;
  if (r >= rows) return;
  const int er = ea[r];
  const int cend = lower ? min(r + 1, cols) : cols;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cend; c += gridDim.x * blockDim.x) {
    const double v = ldexp(S[(int64_t)r * lds + c], er + eb[c]);
    double *d = D + (int64_t)r * ldd + c;
    const double o = beta != 0.0 ? beta * *d + v : v;
    *d = o;
    if (lower && c != r) D[(int64_t)c * ldd + r] = o;
  }
}

// The slices of X^T's rows, i.e. of X's columns: X FP64 [rows][ld], columns
// 0..cols-1 (each an operand row, contraction index = X's row).  Block: 32
// columns x 8 row lanes.  Pass 1: e_c, the exponent of column c's largest
// magnitude (as in slice_rows_kernel); pass 2: 32 x 32 tiles through shared
// memory, the digits of column c written to dB[i][c][k] (k = X's row, BF16) so
// that a warp's stores run along k.  exps[c] = e_c.
__global__ void __launch_bounds__(256)
    slice_cols_kernel(const double *__restrict__ X, int64_t ld, int rows, int cols, int64_t Kp, int s,
                      int64_t slice_stride, __nv_bfloat16 *__restrict__ dB, int *__restrict__ exps) {
  __shared__ unsigned long long red[8][33];
  __shared__ double tile[32][33];
  __shared__ int e_s[32];
  const int c0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
  const int c = c0 + tx;
  unsigned long long mb = 0ull;
  if (c < cols)
    for (int r = ty; r < rows; r += 8)
      mb = max(mb, (unsigned long long)__double_as_longlong(X[(int64_t)r * ld + c]) & 0x7fffffffffffffffull);
  red[ty][tx] = mb;
  __syncthreads();
  if (ty == 0) {
    for (int q = 1; q < 8; ++q) mb = max(mb, red[q][tx]);
    int e = 0;
    if (mb != 0ull) frexp(__longlong_as_double((long long)mb), &e);
    e_s[tx] = mb != 0ull ? e : INT_MIN;   // INT_MIN: a zero column
    if (c < cols && exps) exps[c] = e;
  }
  __syncthreads();
  for (int r0 = 0; r0 < rows; r0 += 32) {
    for (int q = ty; q < 32; q += 8) {
      const int r = r0 + q;
      tile[q][tx] = (r < rows && c < cols) ? X[(int64_t)r * ld + c] : 0.0;
    }
    __syncthreads();
    // thread (tx, ty): row k = r0 + tx of columns c0 + ty, ty + 8, ...
    const int k = r0 + tx;
    for (int q = ty; q < 32; q += 8) {
      const int cc = c0 + q;
      if (cc >= cols || k >= rows) continue;
      const int e = e_s[q];
      long long Q = e != INT_MIN ? __double2ll_rn(ldexp(tile[tx][q], 7 * s - e)) : 0ll;
      for (int i = s - 1; i >= 1; --i) {
        const long long t = (Q + 64) >> 7;
        dB[i * slice_stride + (int64_t)cc * Kp + k] = __float2bfloat16_rn((float)(Q - (t << 7)));
        Q = t;
      }
      dB[(int64_t)cc * Kp + k] = __float2bfloat16_rn((float)Q);
    }
    __syncthreads();
  }
}

// W[t][c] = sum_r Y[r][t ncols + c] Bt[t][r][c] (FP64), t < n_tgt, c < ncols:
// the column dot of W_nm (Eq. ScreenedCoulombOrbital) on a product Y = C_j Bt.
__global__ void coldot64_kernel(const double *__restrict__ Y, int64_t ldy, const double *__restrict__ Bt,
                                int64_t ldb, int64_t strideB, int N, int ncols, int n_tgt, double *__restrict__ W,
                                int64_t ldw) {
  const int t = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x) {
    double acc = 0.0;
    const double *y = Y + (int64_t)t * ncols + c;
    const double *b = Bt + (int64_t)t * strideB + c;
    for (int r = 0; r < N; ++r) acc = fma(y[(int64_t)r * ldy], b[(int64_t)r * ldb], acc);
    W[(int64_t)t * ldw + c] = acc;
  }
}
}  // namespace

cudaError_t launch_fp8_quantize(const float *X, int64_t Kp, int64_t Kq, const float *S, int n_t, int rows,
                                uint8_t *qa, uint8_t *qb, float *ds_a, float *ds_b, cudaStream_t s, int split) {
  if (rows <= 0) return cudaSuccess;
  if (Kp % 4 || Kq % 16 || Kq < Kp || n_t < 0 || n_t > 32) return cudaErrorInvalidValue;
  if (n_t <= 8)
    fp8_quantize_kernel<8><<<rows, Q8_THREADS, 0, s>>>(X, Kp, Kq, S, n_t, rows, qa, qb, ds_a, ds_b, split);
  else
    fp8_quantize_kernel<32><<<rows, Q8_THREADS, 0, s>>>(X, Kp, Kq, S, n_t, rows, qa, qb, ds_a, ds_b, split);
  return cudaGetLastError();
}

cudaError_t launch_slice_rows(const double *X, int64_t ld, int rows, int64_t cols, int64_t Kp, int s,
                              int64_t slice_stride, float *dA, __nv_bfloat16 *dB, int *exps, cudaStream_t st,
                              const double *colscale) {
  if (rows <= 0) return cudaSuccess;
  if (s < 1 || s > 8 || Kp < cols) return cudaErrorInvalidValue;
  slice_rows_kernel<<<rows, 256, 0, st>>>(X, ld, cols, Kp, s, slice_stride, dA, dB, exps, colscale);
  return cudaGetLastError();
}

cudaError_t launch_pi_factor64(const double *delta, int64_t K, int n_t, const double *p0, const double *p1,
                               int mode, double *f, cudaStream_t st) {
  if (n_t <= 0 || K <= 0) return cudaSuccess;
  int bx = (int)((K + 255) / 256);
  if (bx > 152) bx = 152;
  pi_factor64_kernel<<<dim3(bx, n_t), 256, 0, st>>>(delta, K, p0, p1, mode, f);
  return cudaGetLastError();
}

cudaError_t launch_scale_exp2_to(const double *S, int64_t lds, double *D, int64_t ldd, int rows, int cols,
                                 const int *ea, const int *eb, double beta, cudaStream_t st, int lower) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (rows > 65535 || (lower && rows != cols)) return cudaErrorInvalidValue;
  int bx = (cols + 255) / 256;
  if (bx > 16) bx = 16;
  scale_exp2_kernel<<<dim3(bx, rows), 256, 0, st>>>(S, lds, D, ldd, rows, cols, ea, eb, beta, lower);
  return cudaGetLastError();
}

cudaError_t launch_slice_cols(const double *X, int64_t ld, int rows, int cols, int64_t Kp, int s,
                              int64_t slice_stride, __nv_bfloat16 *dB, int *exps, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (s < 1 || s > 8 || Kp < rows) return cudaErrorInvalidValue;
  slice_cols_kernel<<<(cols + 31) / 32, dim3(32, 8), 0, st>>>(X, ld, rows, cols, Kp, s, slice_stride, dB, exps);
  return cudaGetLastError();
}

cudaError_t launch_coldot64(const double *Y, int64_t ldy, const double *Bt, int64_t ldb, int64_t strideB, int N,
                            int ncols, int n_tgt, double *W, int64_t ldw, cudaStream_t st) {
  if (N <= 0 || ncols <= 0 || n_tgt <= 0) return cudaSuccess;
  int bx = (ncols + 127) / 128;
  if (bx > 64) bx = 64;
  coldot64_kernel<<<dim3(bx, n_tgt), 128, 0, st>>>(Y, ldy, Bt, ldb, strideB, N, ncols, n_tgt, W, ldw);
  return cudaGetLastError();
}

cudaError_t launch_fp8_quantize_a(const float *X, int64_t Kp, int64_t Kq, int rows, uint8_t *q, float *ds,
                                  cudaStream_t s, int split) {
  if (rows <= 0) return cudaSuccess;
  if (Kp % 4 || Kq % 16 || Kq < Kp) return cudaErrorInvalidValue;
  fp8_quantize_a_kernel<<<rows, Q8_THREADS, 0, s>>>(X, Kp, Kq, rows, q, ds, split);
  return cudaGetLastError();
}

}  // namespace ltgw
