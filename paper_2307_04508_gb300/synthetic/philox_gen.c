/*
 * Seeded synthetic-input generator (host side).
 *
 * This file draws the random numbers that make up the synthetic workloads:
 * standard normals and uniforms from the Philox4x32-10 counter-based
 * generator (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11), written here from that published definition. It holds none
 * of the GW method's arithmetic; both the CPU oracle and the CUDA path consume
 * the arrays it produces.
 *
 * Conventions (shared with the Python wrapper in __init__.py):
 *   key     = (seed & 0xffffffff, (seed >> 32) + stream)      stream tags a use
 *   counter = (c0, c1, c2, 0)                                  caller's indices
 *   normal  = Box-Muller, cos branch: u1 = (x0 + 1) 2^-32, u2 = x1 2^-32
 *   uniform = (x0 + 0.5) 2^-32
 */
#include <math.h>
#include <stdint.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    k[0] += PHILOX_W0;
    k[1] += PHILOX_W1;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static inline void make_key(uint64_t seed, uint32_t stream, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32) + stream;
}

static inline double normal_at(const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2) {
  const double two_m32 = 2.3283064365386963e-10; /* 2^-32 */
  uint32_t ctr[4] = {c0, c1, c2, 0u}, x[4];
  synth_philox4x32_10(ctr, key, x);
  double u1 = ((double)x[0] + 1.0) * two_m32;
  double u2 = (double)x[1] * two_m32;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* out[i] = uniform in [lo, hi) at counter (i, 0, 0) for i in [0, n). */
void synth_uniform(uint64_t seed, uint32_t stream, int64_t n, double lo, double hi,
                   uint32_t c1, double *out) {
  uint32_t key[2];
  make_key(seed, stream, key);
  const double two_m32 = 2.3283064365386963e-10;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, c1, 0u, 0u}, x[4];
    synth_philox4x32_10(ctr, key, x);
    out[i] = lo + (hi - lo) * (((double)x[0] + 0.5) * two_m32);
  }
}

/* out[r*cols + c] = normal at counter (r, c, 0): a dense Gaussian matrix. */
void synth_normal_matrix(uint64_t seed, uint32_t stream, int64_t rows, int64_t cols,
                         double *out) {
  uint32_t key[2];
  make_key(seed, stream, key);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < rows; ++r)
    for (int64_t c = 0; c < cols; ++c)
      out[r * cols + c] = normal_at(key, (uint32_t)r, (uint32_t)c, 0u);
}

/*
 * Symmetric pair normals Z[r, p, q] = normal at counter (r, min(p,q), max(p,q)).
 * Occupied-virtual block: out[r][(i - i0) * n_virt + a] for i in [i0, i1),
 * a in [0, n_virt), with p = i and q = n_occ + a.
 */
void synth_pair_normals_ov(uint64_t seed, uint32_t stream, int64_t n_aux, int64_t n_occ,
                           int64_t n_virt, int64_t i0, int64_t i1, double *out) {
  uint32_t key[2];
  make_key(seed, stream, key);
  const int64_t cols = (i1 - i0) * n_virt;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n_aux; ++r)
    for (int64_t i = i0; i < i1; ++i)
      for (int64_t a = 0; a < n_virt; ++a)
        out[r * cols + (i - i0) * n_virt + a] =
            normal_at(key, (uint32_t)r, (uint32_t)i, (uint32_t)(n_occ + a));
}

/* One orbital row: out[r][m] = normal at counter (r, min(p,m), max(p,m)), m in [0, n_orb). */
void synth_pair_normals_row(uint64_t seed, uint32_t stream, int64_t n_aux, int64_t n_orb,
                            int64_t p, double *out) {
  uint32_t key[2];
  make_key(seed, stream, key);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n_aux; ++r)
    for (int64_t m = 0; m < n_orb; ++m) {
      int64_t lo = p < m ? p : m, hi = p < m ? m : p;
      out[r * n_orb + m] = normal_at(key, (uint32_t)r, (uint32_t)lo, (uint32_t)hi);
    }
}
