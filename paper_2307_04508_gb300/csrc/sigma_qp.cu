// Self-energy on the imaginary axis (Eq. CorrelationSelfEnergy with the
// modified Gauss-Legendre rule), its N-point Pade continuation (Vidberg &
// Serene 1977, appendix: continued fraction through the sample points), and
// the quasi-particle equation E = e_n + Re Sigma^c_n(E) + shift_n solved by
// Newton with the analytic derivative of the fraction.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {
namespace {

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx mk(double a, double b) { return {a, b}; }
__device__ __forceinline__ cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// Smith's algorithm for complex division (Smith, CACM 5, 435 (1962)).
__device__ __forceinline__ cplx operator/(cplx a, cplx b) {
  if (fabs(b.re) >= fabs(b.im)) {
    double r = b.im / b.re, den = b.re + b.im * r;
    return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
  } else {
    double r = b.re / b.im, den = b.re * r + b.im;
    return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
  }
}

// Sigma^c_n(i w_l) = -(1/pi) sum_m sum_j g_j z/(z^2 + w_j^2) W_nm(i w_j),
// z = x + i w_l with x = e_F - e_m.  One block per (target, l); threads over
// m.  With d = z^2 + w_j^2 = (x^2 - w_l^2 + w_j^2) + i 2 x w_l, the term is
// z conj(d) / |d|^2: the parts that depend on m only are formed once per m,
// leaving one real division per (m, j) (FP64 divisions and complex
// arithmetic are what this kernel spends its time on).
__global__ void sigma_kernel(SigmaArgs a) {
  const int t = blockIdx.y, l = blockIdx.x;
  const double wl = a.omega[l];
  double sre = 0.0, sim = 0.0;
  for (int m = threadIdx.x; m < a.n_orb; m += blockDim.x) {
    const double x = a.eps_F - a.eps_m[m];
    const double dre0 = x * x - wl * wl, dim = 2.0 * x * wl;
    const double dim2 = dim * dim, wdim = wl * dim, xdim = x * dim;
    for (int j = 0; j < a.n_omega; ++j) {
      const double wj = a.omega[j];
      const double Wv = a.W[((int64_t)j * a.n_tgt + t) * a.n_orb + m];
      const double dre = dre0 + wj * wj;
      const double inv = 1.0 / fma(dre, dre, dim2);       // 1 / |d|^2
      const double c = a.weight[j] * Wv * inv;
      sre = fma(c, fma(x, dre, wdim), sre);              // Re z conj(d) = x dre + w_l dim
      sim = fma(c, fma(wl, dre, -xdim), sim);            // Im z conj(d) = w_l dre - x dim
    }
  }
  __shared__ double sh_re[32], sh_im[32];
  for (int o = 16; o > 0; o >>= 1) {
    sre += __shfl_down_sync(0xffffffffu, sre, o);
    sim += __shfl_down_sync(0xffffffffu, sim, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh_re[wid] = sre; sh_im[wid] = sim; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0, i = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { r += sh_re[q]; i += sh_im[q]; }
    const double f = -1.0 / 3.14159265358979323846;
    a.sigma[((int64_t)t * a.n_omega + l) * 2 + 0] = f * r;
    a.sigma[((int64_t)t * a.n_omega + l) * 2 + 1] = f * i;
  }
}

constexpr int MAXP = 128;

// 1 / t = conj(t) / |t|^2 (|t| stays far from the FP64 range limits here)
__device__ __forceinline__ cplx crecip(cplx t) {
  const double inv = 1.0 / fma(t.re, t.re, t.im * t.im);
  return {t.re * inv, -t.im * inv};
}

// Continued fraction value and derivative at z, evaluated from the innermost
// level outwards: t_p = 1 + a_p (z - z_{p-1}) / t_{p+1} and its derivative,
// one complex reciprocal per level.
__device__ void pade_eval(const cplx *a, const cplx *zn, int np, cplx z, cplx &val, cplx &dval) {
  cplx t = mk(1.0, 0.0), dt = mk(0.0, 0.0);
  for (int p = np - 1; p >= 1; --p) {
    const cplx rt = crecip(t);
    const cplx num = a[p] * (z - zn[p - 1]);
    const cplx nt = mk(1.0, 0.0) + num * rt;
    const cplx ndt = (a[p] - num * dt * rt) * rt;   // d/dz [num / t]
    t = nt;
    dt = ndt;
  }
  const cplx rt = crecip(t);
  val = a[0] * rt;
  dval = mk(0.0, 0.0) - a[0] * dt * rt * rt;
}

// One thread per target: Pade coefficients through every pade_stride-th node,
// then Newton on f(E) = E - e_n - Re C(E - e_F + i eta) - shift_n.
__global__ void qp_kernel(QpArgs q) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= q.n_tgt) return;
  cplx g[MAXP], a[MAXP], zn[MAXP];
  int np = 0;
  for (int l = 0; l < q.n_omega && np < MAXP; l += q.pade_stride, ++np) {
    zn[np] = mk(0.0, q.omega[l]);
    g[np] = mk(q.sigma[((int64_t)t * q.n_omega + l) * 2], q.sigma[((int64_t)t * q.n_omega + l) * 2 + 1]);
  }
  a[0] = g[0];
  for (int p = 1; p < np; ++p) {
    for (int i = p; i < np; ++i) g[i] = (g[p - 1] - g[i]) / ((zn[i] - zn[p - 1]) * g[i]);
    a[p] = g[p];
  }
  const double en = q.eps_n[t], sh = q.shift[t];
  double E = en;
  int st = 1;
  for (int it = 0; it < q.max_iter; ++it) {
    cplx v, dv;
    pade_eval(a, zn, np, mk(E - q.eps_F, q.eta), v, dv);
    double f = E - en - v.re - sh;
    double fp = 1.0 - dv.re;
    double dE = -f / fp;
    E += dE;
    if (!isfinite(E)) break;
    if (fabs(dE) < q.tol) { st = 0; break; }
  }
  q.e_qp[t] = E;
  q.status[t] = st;
}

}  // namespace

cudaError_t launch_sigma(const SigmaArgs &a, cudaStream_t s) {
  if (a.n_tgt <= 0 || a.n_omega <= 0) return cudaSuccess;
  dim3 grid(a.n_omega, a.n_tgt);
  sigma_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_qp(const QpArgs &q, cudaStream_t s) {
  if (q.n_tgt <= 0) return cudaSuccess;
  if ((q.n_omega + q.pade_stride - 1) / q.pade_stride > MAXP) return cudaErrorInvalidValue;
  qp_kernel<<<(q.n_tgt + 31) / 32, 32, 0, s>>>(q);
  return cudaGetLastError();
}

}  // namespace ltgw
