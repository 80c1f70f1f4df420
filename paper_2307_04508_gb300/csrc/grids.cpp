// Host-side quadrature grids of the LT-GW path.
//
//  * modified Gauss-Legendre rule on [0, inf) for the frequency integral of
//    Eq. CorrelationSelfEnergy: Legendre nodes by Newton's method on the
//    three-term recurrence, mapped by w = w0 (1+x)/(1-x);
//  * minimax Laplace grid for Eq. LT: 1/X ~ sum_m w_m exp(-X x_m) on [a, b]
//    (Sec. 3: a = gap^2 + w_min^2, b = max(largest gap^2, 1e4)), minimising the
//    error of 1/X scaled by a (the criterion the paper's epsilon_LT bounds).
//    Start: the best trapezoid rule in t = log(tau) for 1/X = int exp(t - X e^t) dt
//    over a search of its offset and step; then L_p fits for p = 2..64, which
//    approach the minimax solution; then a Remez exchange on the 2k+1
//    alternation points.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/ltgw.h"

namespace {

const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- Legendre
void legendre_nodes(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 1; j < n; ++j) {
        double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        // refresh the derivative at the converged node
        p0 = 1.0; p1 = z;
        for (int j = 1; j < n; ++j) {
          double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    double wt = 2.0 / ((1.0 - z * z) * dp * dp);
    x[i] = -z;             // ascending
    x[n - 1 - i] = z;
    w[i] = wt;
    w[n - 1 - i] = wt;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// ---------------------------------------------------------------- Laplace fit
// Work on y = X / a in [1, R]; the grid for [a, b] is x_m = alpha_m / a,
// w_m = omega_m / a.  Parameters are logs: alpha = e^p, omega = e^q.  The
// error is absolute in 1/y, i.e. the error of 1/X scaled by a.
struct ExpSum {
  int k = 0;
  std::vector<double> p, q;  // log alpha, log omega
  double s(double y) const {
    double t = 0.0;
    for (int v = 0; v < k; ++v) t += exp(q[v] - exp(p[v]) * y);
    return t;
  }
  double r(double y) const { return 1.0 / y - s(y); }
};

std::vector<double> log_grid(double R, int n) {
  std::vector<double> y(n + 1);
  double lr = log(R);
  for (int i = 0; i <= n; ++i) y[i] = exp(lr * i / n);
  return y;
}

double sup_err(const ExpSum &f, const std::vector<double> &y) {
  double m = 0.0;
  for (double v : y) m = std::max(m, fabs(f.r(v)));
  return m;
}

ExpSum sinc_rule(int k, double t0, double h) {
  ExpSum f;
  f.k = k;
  f.p.resize(k);
  f.q.resize(k);
  for (int v = 0; v < k; ++v) {
    double t = t0 + h * v;
    f.p[v] = t;              // alpha = e^t
    f.q[v] = log(h) + t;     // omega = h e^t
  }
  return f;
}

// Solve the dense system M x = b by Gaussian elimination with partial
// pivoting; returns false when singular.
bool dense_solve(std::vector<double> &M, std::vector<double> &b, int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r * n + c]) > fabs(M[piv * n + c])) piv = r;
    if (!(fabs(M[piv * n + c]) > 1e-300)) return false;
    if (piv != c) {
      for (int j = 0; j < n; ++j) std::swap(M[c * n + j], M[piv * n + j]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = M[r * n + c] / M[c * n + c];
      if (f == 0.0) continue;
      for (int j = c; j < n; ++j) M[r * n + j] -= f * M[c * n + j];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int j = c + 1; j < n; ++j) s -= M[c * n + j] * b[j];
    b[c] = s / M[c * n + c];
  }
  return true;
}

// Minimise sum_i |r(y_i)|^pw for pw = 2, 4, ..., 128 (Levenberg-Marquardt on
// the residuals |r|^{pw/2} sign r): the L_p minimisers approach the minimax
// solution and give Remez a start with the full alternation.
void lp_continuation(ExpSum &f, const std::vector<double> &y) {
  const int k = f.k, m = 2 * k, n = (int)y.size();
  std::vector<double> J((size_t)n * m), fr(n), H(m * m), g(m);
  for (double pw = 2.0; pw <= 64.0; pw *= 2.0) {
    double lam = 1e-2;
    for (int it = 0; it < 40; ++it) {
      double sc = sup_err(f, y);
      if (!(sc > 0.0)) return;
      double obj = 0.0;
      for (int i = 0; i < n; ++i) {
        double yi = y[i], s = 0.0;
        double *Ji = &J[(size_t)i * m];
        for (int v = 0; v < k; ++v) {
          double al = exp(f.p[v]), t = exp(f.q[v] - al * yi);
          s += t;
          Ji[v] = yi * al * t;   // d r / d p_v
          Ji[k + v] = -t;        // d r / d q_v
        }
        double rn = (1.0 / yi - s) / sc;
        double a = fabs(rn);
        double fi = pow(a, 0.5 * pw) * (rn >= 0 ? 1.0 : -1.0);
        double dfac = 0.5 * pw * pow(a, 0.5 * pw - 1.0) / sc;
        for (int c = 0; c < m; ++c) Ji[c] *= dfac;
        fr[i] = fi;
        obj += fi * fi;
      }
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(g.begin(), g.end(), 0.0);
      for (int i = 0; i < n; ++i) {
        const double *Ji = &J[(size_t)i * m];
        for (int a = 0; a < m; ++a) {
          g[a] += Ji[a] * fr[i];
          for (int b = 0; b <= a; ++b) H[a * m + b] += Ji[a] * Ji[b];
        }
      }
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < a; ++b) H[b * m + a] = H[a * m + b];
      bool improved = false;
      for (int tries = 0; tries < 30; ++tries) {
        std::vector<double> M = H, d = g;
        for (int a = 0; a < m; ++a) M[a * m + a] += lam * (H[a * m + a] + 1e-12);
        if (!dense_solve(M, d, m)) { lam *= 5.0; continue; }
        ExpSum t = f;
        for (int v = 0; v < k; ++v) { t.p[v] -= d[v]; t.q[v] -= d[k + v]; }
        double o2 = 0.0;
        bool fin = true;
        for (int i = 0; i < n && fin; ++i) {
          double rr = fabs(t.r(y[i]) / sc);
          double fi = pow(rr, 0.5 * pw);
          o2 += fi * fi;
          fin = isfinite(o2);
        }
        if (fin && o2 < obj) {
          f = t;
          lam = std::max(lam / 3.0, 1e-10);
          improved = true;
          break;
        }
        lam *= 5.0;
      }
      if (!improved) break;
    }
  }
}

// Alternating extrema of r on [1, R]: the largest |r| in each run of equal
// sign, trimmed at the smaller end down to `want` points.
bool find_extrema(const ExpSum &f, double R, int want, std::vector<double> &ys) {
  std::vector<double> y = log_grid(R, 8000);
  std::vector<double> ey, er;
  int cur = 0;
  double by = 1.0, br = 0.0;
  for (double v : y) {
    double r = f.r(v);
    int sg = (r >= 0.0) ? 1 : -1;
    if (cur == 0) { cur = sg; by = v; br = r; continue; }
    if (sg != cur) {
      ey.push_back(by); er.push_back(br);
      cur = sg; by = v; br = r;
    } else if (fabs(r) > fabs(br)) {
      by = v; br = r;
    }
  }
  ey.push_back(by); er.push_back(br);
  while ((int)ey.size() > want) {
    if (fabs(er.front()) < fabs(er.back())) { ey.erase(ey.begin()); er.erase(er.begin()); }
    else { ey.pop_back(); er.pop_back(); }
  }
  if ((int)ey.size() != want) return false;
  ys = ey;
  return true;
}

// Newton on r(y_i) = (-1)^i E (i = 0..2k) in (p, q, E), damped.
bool remez_step(ExpSum &f, const std::vector<double> &ys, double &E) {
  const int k = f.k, n = 2 * k + 1;
  double e0 = 0.0;
  for (int i = 0; i < n; ++i) e0 += f.r(ys[i]) * ((i % 2) ? -1.0 : 1.0);
  E = e0 / n;
  auto resid = [&](const ExpSum &g, double Eg) {
    double fn = 0.0;
    for (int i = 0; i < n; ++i) {
      double Fi = g.r(ys[i]) - ((i % 2) ? -1.0 : 1.0) * Eg;
      fn += Fi * Fi;
    }
    return sqrt(fn);
  };
  for (int it = 0; it < 50; ++it) {
    std::vector<double> J(n * n), F(n);
    for (int i = 0; i < n; ++i) {
      double y = ys[i], sg = (i % 2) ? -1.0 : 1.0, s = 0.0;
      for (int v = 0; v < k; ++v) {
        double al = exp(f.p[v]), t = exp(f.q[v] - al * y);
        s += t;
        J[i * n + v] = y * al * t;
        J[i * n + k + v] = -t;
      }
      J[i * n + 2 * k] = -sg;
      F[i] = 1.0 / y - s - sg * E;
    }
    double fn = resid(f, E);
    if (fn < 1e-15 * std::max(1e-300, fabs(E))) return true;
    if (!dense_solve(J, F, n)) return false;
    double step = 1.0;
    bool ok = false;
    for (int ls = 0; ls < 40; ++ls) {
      ExpSum g = f;
      for (int v = 0; v < k; ++v) { g.p[v] -= step * F[v]; g.q[v] -= step * F[k + v]; }
      double Eg = E - step * F[2 * k];
      if (resid(g, Eg) < fn) { f = g; E = Eg; ok = true; break; }
      step *= 0.5;
    }
    if (!ok) return true;
  }
  return true;
}

}  // namespace

extern "C" ltgw_status ltgw_gl_grid(int n, double omega0, double *omega, double *weight) {
  if (n < 1 || n > 4096 || !(omega0 > 0.0) || !omega || !weight) return LTGW_ERR_BAD_ARG;
  std::vector<double> x, w;
  legendre_nodes(n, x, w);
  for (int i = 0; i < n; ++i) {
    omega[i] = omega0 * (1.0 + x[i]) / (1.0 - x[i]);
    weight[i] = w[i] * 2.0 * omega0 / ((1.0 - x[i]) * (1.0 - x[i]));
  }
  return LTGW_OK;
}

namespace {

// Fitted grids on [1, R] by (k, R), reused by later calls: an exact hit is
// returned as is; a fit for the same k within a factor 8 in R seeds the Remez
// exchange directly.  Process-wide, guarded by a mutex.
struct CachedFit {
  int k;
  double R, err;
  ExpSum f;
};
std::mutex g_fit_mutex;
std::vector<CachedFit> g_fit_cache;

// Remez exchange from `cur`; returns the best grid seen and its error.
void remez_polish(ExpSum &best, double &best_err, ExpSum cur, double R, const std::vector<double> &fine) {
  const int k = cur.k;
  for (int outer = 0; outer < 30; ++outer) {
    std::vector<double> ys;
    if (!find_extrema(cur, R, 2 * k + 1, ys)) break;
    ExpSum trial = cur;
    double E = 0.0;
    if (!remez_step(trial, ys, E)) break;
    bool finite = true;
    for (int v = 0; v < k; ++v) finite = finite && isfinite(trial.p[v]) && isfinite(trial.q[v]);
    if (!finite) break;
    double e = sup_err(trial, fine);
    if (!(e < 1.0)) break;
    cur = trial;
    if (e < best_err) { best_err = e; best = trial; }
    if (fabs(e - fabs(E)) <= 1e-4 * fabs(E)) break;  // equioscillation reached
  }
}

ExpSum fit_unit_interval(int k, double R, double &err_out) {
  const double lr = log(R);
  std::vector<double> fine = log_grid(R, 12000);
  {
    std::lock_guard<std::mutex> lock(g_fit_mutex);
    for (const CachedFit &c : g_fit_cache)
      if (c.k == k && c.R == R) { err_out = c.err; return c.f; }
  }
  ExpSum best;
  double best_err = 1e300;
  // warm start from a cached fit for the same k at a nearby R
  ExpSum seed;
  bool have_seed = false;
  {
    std::lock_guard<std::mutex> lock(g_fit_mutex);
    double bestd = log(8.0);
    for (const CachedFit &c : g_fit_cache)
      if (c.k == k && fabs(log(c.R / R)) < bestd) { bestd = fabs(log(c.R / R)); seed = c.f; have_seed = true; }
  }
  if (have_seed) {
    best = seed;
    best_err = sup_err(seed, fine);
    remez_polish(best, best_err, seed, R, fine);
  }
  if (!have_seed || !(best_err < 1.0)) {
    // 1. best trapezoid rule in t = log(tau) over a coarse search of offset and step
    std::vector<double> coarse = log_grid(R, 300);
    best_err = 1e300;
    for (int ih = 0; ih < 30; ++ih) {
      double h = 0.3 + 3.7 * ih / 29.0;
      for (int it = 0; it < 40; ++it) {
        double t0 = -lr - 6.0 + (lr + 8.0) * it / 39.0;
        ExpSum f = sinc_rule(k, t0, h);
        double e = sup_err(f, coarse);
        if (e < best_err) { best_err = e; best = f; }
      }
    }
    // 2. L_p continuation toward the minimax solution
    ExpSum cur = best;
    lp_continuation(cur, log_grid(R, 800));
    double e_cur = sup_err(cur, fine);
    best_err = sup_err(best, fine);
    if (e_cur < best_err) { best = cur; best_err = e_cur; }
    // 3. Remez exchange polish
    remez_polish(best, best_err, cur, R, fine);
  }
  {
    std::lock_guard<std::mutex> lock(g_fit_mutex);
    if (g_fit_cache.size() < 4096) g_fit_cache.push_back({k, R, best_err, best});
  }
  err_out = best_err;
  return best;
}

}  // namespace

extern "C" ltgw_status ltgw_laplace_grid(int n_tau, double a, double b, double *x, double *w,
                                         double *max_err) {
  if (n_tau < 1 || n_tau > 64 || !(a > 0.0) || !(b > a) || !x || !w) return LTGW_ERR_BAD_ARG;
  const int k = n_tau;
  double err = 0.0;
  ExpSum best = fit_unit_interval(k, b / a, err);
  // map back to [a, b]; ascending x
  std::vector<std::pair<double, double>> g(k);
  for (int v = 0; v < k; ++v) g[v] = {exp(best.p[v]) / a, exp(best.q[v]) / a};
  std::sort(g.begin(), g.end());
  for (int v = 0; v < k; ++v) { x[v] = g[v].first; w[v] = g[v].second; }
  if (max_err) *max_err = err;
  return LTGW_OK;
}

namespace {
// min ||A g - y||^2 + ridge ||C g||^2 for A (m x n, column-major, m >= n),
// C the diagonal that gives A's columns unit norm, by Householder QR of A's
// unit-norm columns stacked over sqrt(ridge) I.  The small ridge keeps the
// coefficients of nearly dependent exponentials from cancelling at large
// magnitude.  False when a column is zero.
bool least_squares(const std::vector<double> &A0, int m, int n, const std::vector<double> &y0, double ridge,
                   std::vector<double> &g) {
  const int mm = m + n;
  std::vector<double> A((size_t)mm * n, 0.0), y(mm, 0.0), cs(n);
  for (int c = 0; c < n; ++c) {
    double s = 0.0;
    for (int r = 0; r < m; ++r) s += A0[(size_t)c * m + r] * A0[(size_t)c * m + r];
    if (!(s > 0.0)) return false;
    cs[c] = 1.0 / sqrt(s);
    for (int r = 0; r < m; ++r) A[(size_t)c * mm + r] = A0[(size_t)c * m + r] * cs[c];
    A[(size_t)c * mm + m + c] = sqrt(ridge);
  }
  for (int r = 0; r < m; ++r) y[r] = y0[r];
  for (int c = 0; c < n; ++c) {
    double *a = &A[(size_t)c * mm];
    double nrm = 0.0;
    for (int r = c; r < mm; ++r) nrm += a[r] * a[r];
    nrm = sqrt(nrm);
    if (!(nrm > 0.0)) return false;
    const double alpha = a[c] > 0.0 ? -nrm : nrm;
    a[c] -= alpha;                                  // v = a - alpha e_c, stored in place
    const double vtv = -2.0 * alpha * a[c];         // |v|^2 = 2 nrm (nrm + |a_c|)
    for (int d = c + 1; d < n; ++d) {
      double *b = &A[(size_t)d * mm];
      double t = 0.0;
      for (int r = c; r < mm; ++r) t += a[r] * b[r];
      t = 2.0 * t / vtv;
      for (int r = c; r < mm; ++r) b[r] -= t * a[r];
    }
    double t = 0.0;
    for (int r = c; r < mm; ++r) t += a[r] * y[r];
    t = 2.0 * t / vtv;
    for (int r = c; r < mm; ++r) y[r] -= t * a[r];
    a[c] = alpha;                                   // R's diagonal
  }
  g.assign(n, 0.0);
  for (int c = n - 1; c >= 0; --c) {
    double s = y[c];
    for (int d = c + 1; d < n; ++d) s -= A[(size_t)d * mm + c] * g[d];
    g[c] = s / A[(size_t)c * mm + c];
  }
  for (int c = 0; c < n; ++c) g[c] *= cs[c];
  return true;
}
}  // namespace

// Imaginary-time (cosine-transform) grid:
//   Delta / (w^2 + Delta^2) = int_0^inf cos(w tau) exp(-Delta tau) dtau
//                           ~ sum_k gamma_jk exp(-Delta tau_k)   for Delta in [dmin, dmax].
// tau_k: geometric from 0.1 / dmax to 8 / dmin (the decay times of the pair
// exponentials; the short ones carry the nearly linear shape Delta / w^2 of
// the high frequencies).  gamma_j: for each frequency w_j the least-squares
// fit over log-spaced Delta of the error scaled by max_Delta of the target,
// with a ridge term ridge |C g|^2 (C: unit-norm columns).  max_err: max over
// frequencies of max_Delta |fit - target| / max_Delta target on a four times
// finer sample; amplification: max over frequencies and Delta of
// sum_k |gamma_jk| e^{-Delta tau_k} / max target, the factor by which the
// recombination can magnify relative errors of M^k.
extern "C" ltgw_status ltgw_cosine_grid(int n_tau, double dmin, double dmax, int n_omega, const double *omegas,
                                        double ridge, double *tau, double *gamma, double *max_err,
                                        double *amplification) {
  if (n_tau < 1 || n_tau > 64 || !(dmin > 0.0) || !(dmax > dmin) || n_omega < 1 || !omegas || !tau || !gamma ||
      !(ridge >= 0.0))
    return LTGW_ERR_BAD_ARG;
  const double t_lo = 0.1 / dmax, t_hi = 8.0 / dmin;
  for (int k = 0; k < n_tau; ++k)
    tau[k] = n_tau == 1 ? sqrt(t_lo * t_hi) : t_lo * pow(t_hi / t_lo, (double)k / (n_tau - 1));
  const int m = 64 * n_tau + 200, mf = 4 * m;
  const double lr = log(dmax / dmin);
  double worst = 0.0, amp = 0.0;
  std::vector<double> A((size_t)m * n_tau), y(m), g;
  for (int j = 0; j < n_omega; ++j) {
    const double w2 = omegas[j] * omegas[j];
    // the target's largest value on [dmin, dmax]: at Delta = w when w lies inside
    const double dpk = std::min(std::max(omegas[j], dmin), dmax), fmax = dpk / (w2 + dpk * dpk);
    for (int s = 0; s < m; ++s) {
      const double d = dmin * exp(lr * s / (m - 1)), f = d / (w2 + d * d);
      for (int k = 0; k < n_tau; ++k) A[(size_t)k * m + s] = exp(-d * tau[k]) / fmax;
      y[s] = f / fmax;
    }
    if (!least_squares(A, m, n_tau, y, ridge, g)) return LTGW_ERR_BAD_ARG;
    for (int k = 0; k < n_tau; ++k) gamma[(size_t)j * n_tau + k] = g[k];
    for (int s = 0; s < mf; ++s) {
      const double d = dmin * exp(lr * s / (mf - 1)), f = d / (w2 + d * d);
      double v = 0.0, va = 0.0;
      for (int k = 0; k < n_tau; ++k) {
        v += g[k] * exp(-d * tau[k]);
        va += fabs(g[k]) * exp(-d * tau[k]);
      }
      worst = std::max(worst, fabs(v - f) / fmax);
      amp = std::max(amp, va / fmax);
    }
  }
  if (max_err) *max_err = worst;
  if (amplification) *amplification = amp;
  return LTGW_OK;
}
