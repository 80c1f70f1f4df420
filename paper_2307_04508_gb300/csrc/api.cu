// C ABI of the LT-GW library: argument checking, workspace, host/device
// staging and the order of the steps of Sec. 2 (frozen-core slice -> NAF ->
// Pi -> screening -> W_nm -> Sigma(i w) -> Pade -> Newton).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {
int g_launch_count = 0;
}

using namespace ltgw;

namespace {

// Device bump allocator; grows (free + malloc) only between calls.
struct Arena {
  char *base = nullptr;
  size_t cap = 0, off = 0;
  bool sizing = false;
  size_t need = 0;
  void begin_sizing() { sizing = true; need = 0; off = 0; }
  template <class T>
  T *take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T *p = sizing ? nullptr : reinterpret_cast<T *>(base + off);
    off += std::max<size_t>(n, 1) * sizeof(T);
    if (sizing) need = off;
    return p;
  }
  cudaError_t commit() {
    sizing = false;
    size_t want = need;
    off = 0;
    if (want <= cap) return cudaSuccess;
    if (base) cudaFree(base);
    base = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&base, want);
    if (e != cudaSuccess) { cudaGetLastError(); return e; }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (base) cudaFree(base);
    base = nullptr;
    cap = 0;
  }
};

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

enum Stage { EV_START = 0, EV_NAF, EV_PI0, EV_PI1, EV_PI, EV_SCREEN, EV_WNM, EV_SIGQP, EV_END, EV_TRI0, EV_TRI1,
             EV_K0, EV_VEC1, EV_COUNT };

}  // namespace

struct ltgw_ctx {
  int device = 0;
  ltgw_status st = LTGW_OK;
  std::string err;
  Arena a1, a2, a3;  // a1: inputs; a2: after the NAF count is known; a3: NAF scratch
  int *flags = nullptr;
  bool timing = false;
  cudaEvent_t ev[EV_COUNT] = {};
  // side stream for the copy of inputs first read late in the solve (B_tgt),
  // forked from and joined back to the caller's stream by two events
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // streamed solve: the block callback fills one of two block buffers on its
  // own stream while the caller's stream consumes the other; per buffer, an
  // event when its block has arrived and one when its consumers are done
  cudaStream_t fill_stream = nullptr;
  cudaEvent_t blk_ready[2] = {}, blk_done[2] = {};
  ltgw_stats stats{};
  int launches = 0;
  double pi_tc_flops = 0.0;
  int tri_n = 0;
  double gen_ms = 0.0;
  int n_sm = 148;
  Arena a4;  // tensor-core scratch: tile lists and partial tiles
  Arena a5;  // tensor-core operand copies consumed by the next contraction
  // Autotuner of the tensor-core contractions (off by default): per shape, the
  // (scales per CTA, K-splits) configuration that timed fastest on this GPU.
  struct TcKey {
    int kind, n_tiles, n_t, out_mode;
    int64_t Kp, rows_a, rows_b;
    bool operator<(const TcKey &o) const {
      return std::tie(kind, n_tiles, n_t, out_mode, Kp, rows_a, rows_b) <
             std::tie(o.kind, o.n_tiles, o.n_t, o.out_mode, o.Kp, o.rows_a, o.rows_b);
    }
  };
  struct TcChoice { int nt_group; int64_t splits; };
  bool autotune = false;
  std::map<TcKey, TcChoice> tuned;

  void fail(ltgw_status c, const std::string &m) {
    if (st == LTGW_OK) { st = c; err = m; }
  }
  ltgw_status status() const { return st; }
  void reset() { st = LTGW_OK; err.clear(); launches = 0; }
  void mark(Stage s, cudaStream_t stream) {
    if (timing) cudaEventRecord(ev[s], stream);
  }
  double ms(Stage a, Stage b) {
    float t = 0.f;
    if (!timing) return 0.0;
    if (cudaEventElapsedTime(&t, ev[a], ev[b]) != cudaSuccess) { cudaGetLastError(); return 0.0; }
    return (double)t;
  }
};

#define CHECK_LAUNCH(ctx, expr, nk)                                                              \
  do {                                                                                           \
    cudaError_t _e = (expr);                                                                     \
    (ctx)->launches += (nk);                                                                     \
    if (_e != cudaSuccess) {                                                                     \
      (ctx)->fail(LTGW_ERR_DEVICE, std::string(#expr) + ": " + cudaGetErrorString(_e));          \
      return (ctx)->status();                                                                    \
    }                                                                                            \
  } while (0)

#define REQUIRE(ctx, cond, msg)                                                                  \
  do {                                                                                           \
    if (!(cond)) {                                                                               \
      (ctx)->fail(LTGW_ERR_BAD_ARG, msg);                                                        \
      return (ctx)->status();                                                                    \
    }                                                                                            \
  } while (0)

namespace {

ltgw_status copy_in(ltgw_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return LTGW_OK;
  LTGW_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return LTGW_OK;
}

ltgw_status read_small(ltgw_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return LTGW_OK;
  LTGW_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  LTGW_CUDA(ctx, cudaStreamSynchronize(s));
  return LTGW_OK;
}

ltgw_status check_flags(ltgw_ctx *ctx, cudaStream_t s) {
  int h[FLAG_COUNT];
  if (read_small(ctx, h, ctx->flags, sizeof(h), s) != LTGW_OK) return ctx->status();
  if (h[FLAG_EIG]) ctx->fail(LTGW_ERR_EIG, "NAF eigensolver: inverse iteration produced a non-finite vector");
  if (h[FLAG_NOT_SPD]) ctx->fail(LTGW_ERR_NOT_SPD, "screening: a pivot of 1 - Pi(iw) was not positive");
  if (h[FLAG_TC_TIMEOUT]) ctx->fail(LTGW_ERR_DEVICE, "tensor-core kernel: a pipeline wait timed out");
  return ctx->status();
}

// NAF basis on device data: K = B B^T, eigenvectors with eigenvalue > thresh
// as rows of Ut (descending eigenvalue), their eigenvalues in lam.
ltgw_status naf_metric_tc(ltgw_ctx *ctx, int n, int64_t n_pairs, const double *B, int64_t ld, double *K,
                          cudaStream_t s, double beta = 0.0);

// FP64-accurate C = A B^T from integer slices (defined below).
ltgw_status emu_gemm(ltgw_ctx *ctx, int m, int n, int64_t K, const double *A, int64_t lda, const double *B,
                     int64_t ldb, double *C, int64_t ldc, bool sym, int s, cudaStream_t st);

// K builder for the streamed solve: fills w.A (n x n) itself.
using KBuilder = std::function<ltgw_status(double *K)>;

ltgw_status naf_basis_dev(ltgw_ctx *ctx, Arena &ar, int n, int64_t n_pairs, const double *B,
                          int64_t ld, double thresh, double *Ut, double *lam_out, int *k_out,
                          int *near_out, cudaStream_t s, bool mixed = false, const KBuilder *build_K = nullptr,
                          int emu_slices = 0) {
  EigWork w;
  auto layout = [&](Arena &A) {
    w.A = A.take<double>((size_t)n * n);
    w.V = A.take<double>((size_t)(n + 64) * n);   // 64 zero rows past the last reflector (compact-WY blocks)
    w.d = A.take<double>(n);
    w.e = A.take<double>(n);
    w.tau = A.take<double>(n);
    w.p = A.take<double>(n);
    w.w = A.take<double>(n);
    w.scal = A.take<double>(8);
    w.lam = A.take<double>(n);
    w.X = A.take<double>((size_t)n * n);
    w.lu = A.take<double>((size_t)5 * n * n);
    w.count = A.take<int>(2);
    const int64_t nsplit = (n + 63) / 64, nblk = (n + 63) / 64;
    // compact-WY scratch: W1 and its partials (block-at-a-time form: split
    // partials of 64 x n and W1 64 x n; cooperative form: one 64 x 64 partial
    // per CTA and one W1 per 64-column slice), every block's G and T, and
    // every block's M_b (before the T recurrences: the split partials of G)
    w.wy_r0 = (int64_t)std::max((size_t)nsplit * 64 * (size_t)n + 64 * (size_t)n,
                                ((size_t)ctx->n_sm + (size_t)nsplit) * 64 * 64);
    w.wy = A.take<double>((size_t)w.wy_r0 + 2 * (size_t)nblk * 64 * 64 +
                          (size_t)nblk * std::max((size_t)n * 64, (size_t)nsplit * 64 * 64));
    w.grid_ws = A.take<double>((size_t)4 * n + 2 * (size_t)ctx->n_sm + 8);
  };
  ar.begin_sizing();
  layout(ar);
  if (ar.commit() != cudaSuccess) {
    ctx->fail(LTGW_ERR_NOMEM, "NAF workspace allocation failed");
    return ctx->status();
  }
  layout(ar);
  w.flags = ctx->flags;
  ctx->mark(EV_K0, s);
  if (build_K) {
    if ((*build_K)(w.A) != LTGW_OK) return ctx->status();
  } else if (mixed) {
    if (naf_metric_tc(ctx, n, n_pairs, B, ld, w.A, s) != LTGW_OK) return ctx->status();
  } else if (emu_slices) {
    if (emu_gemm(ctx, n, n, n_pairs, B, ld, B, ld, w.A, n, true, emu_slices, s) != LTGW_OK) return ctx->status();
  } else {
    GemmF64Args g;
    g.M = n; g.N = n; g.K = n_pairs;
    g.A = B; g.lda = ld; g.B = B; g.ldb = ld;
    g.C = w.A; g.ldc = n;
    g.syrk = 1;
    CHECK_LAUNCH(ctx, launch_gemm_f64(g, 1, true, true, s), 1);
  }
  LTGW_CUDA(ctx, cudaMemsetAsync(w.V, 0, (size_t)(n + 64) * n * sizeof(double), s));
  int nl = 0;
  ctx->mark(EV_TRI0, s);
  cudaError_t e = launch_eig_tridiag(w, n, thresh, s, &nl);
  ctx->mark(EV_TRI1, s);
  ctx->tri_n = n;
  ctx->launches += nl;
  if (e != cudaSuccess) { ctx->fail(LTGW_ERR_DEVICE, std::string("eig_tridiag: ") + cudaGetErrorString(e)); return ctx->status(); }
  int cnt[2] = {0, 0};
  if (read_small(ctx, cnt, w.count, sizeof(cnt), s) != LTGW_OK) return ctx->status();
  const int k = cnt[0];
  *k_out = k;
  if (near_out) *near_out = cnt[1];
  if (k <= 0) { ctx->fail(LTGW_ERR_NO_NAF, "NAF threshold kept no auxiliary function"); return ctx->status(); }
  nl = 0;
  e = launch_eig_vectors(w, n, k, Ut, ctx->flags, s, &nl);
  ctx->mark(EV_VEC1, s);
  ctx->launches += nl;
  if (e != cudaSuccess) { ctx->fail(LTGW_ERR_DEVICE, std::string("eig_vectors: ") + cudaGetErrorString(e)); return ctx->status(); }
  if (lam_out) LTGW_CUDA(ctx, cudaMemcpyAsync(lam_out, w.lam, (size_t)k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return LTGW_OK;
}

// Pi at the GL frequencies, direct (n_tau == 0) or through moments M^k and the
// recombination d_E [n_omega][n_tau]: lt_form 1 = the M^m form of Eq. LT
// (factors w_m Delta e^{-Delta^2 x_m}), 2 = imaginary time (factors e^{-Delta tau_k},
// tau_k in d_x).
ltgw_status polarizability_dev(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt, int64_t ldb,
                               const double *delta, int n_omega, const double *d_omega,
                               int n_tau, const double *d_x, const double *d_w, const double *d_E,
                               double *M, int spin, double *Pi, cudaStream_t s, int lt_form) {
  GemmF64Args g;
  g.M = N; g.N = N; g.K = n_pairs;
  g.A = Bt; g.lda = ldb; g.B = Bt; g.ldb = ldb;
  g.ldc = N; g.strideC = (int64_t)N * N;
  g.syrk = 1;
  g.delta = delta;
  ctx->mark(EV_PI0, s);
  if (n_tau == 0) {
    g.C = Pi;
    g.alpha = -2.0 * spin;
    g.scale_mode = SCALE_DIRECT;
    g.batch_p0 = d_omega;
    CHECK_LAUNCH(ctx, launch_gemm_f64(g, n_omega, true, true, s), 1);
    ctx->mark(EV_PI1, s);
  } else {
    g.C = M;
    g.alpha = 1.0;
    g.scale_mode = lt_form == 2 ? SCALE_EXPTAU : SCALE_LAPLACE;
    g.batch_p0 = d_x;
    g.batch_p1 = lt_form == 2 ? nullptr : d_w;
    CHECK_LAUNCH(ctx, launch_gemm_f64(g, n_tau, true, true, s), 1);
    ctx->mark(EV_PI1, s);
    CHECK_LAUNCH(ctx, launch_recombine(M, n_tau, d_E, n_omega, (int64_t)N * N, -2.0 * spin, Pi, s),
                 (n_omega + 63) / 64);
  }
  return LTGW_OK;
}

// Split-K plan: one CTA per SM, so choose the split count that fills whole
// waves best while keeping at least 1024 pairs per CTA.
// K-split count for a tensor-core contraction of `units` output tiles x groups:
// the CTAs of one wave run in lockstep, so the time is about waves x (per-CTA
// overhead + K chunks per CTA); the overhead (TMEM and barrier setup, pipeline
// fill, draining the accumulators) costs about as much as ten 64-pair chunks.
// At least Kp / drain_k splits (up to 64) keep each CTA to one FP32 drain; the
// split length is a multiple of `align` pairs.
int64_t tc_splits(const ltgw_ctx *ctx, int64_t units, int64_t Kp, int64_t drain_k, int64_t align, int64_t *kps_out) {
  const int64_t max_split = std::min<int64_t>(64, std::max<int64_t>(1, Kp / 1024));
  const int64_t min_split = std::min<int64_t>(max_split, (Kp + drain_k - 1) / drain_k);
  const int64_t nchunk = Kp / 64;
  int64_t splits = min_split;
  double best = 1e300;
  for (int64_t sp = min_split; sp <= max_split; ++sp) {
    const int64_t waves = (units * sp + ctx->n_sm - 1) / ctx->n_sm;
    const double cost = (double)waves * (10.0 + (double)((nchunk + sp - 1) / sp));
    if (cost < best) { best = cost; splits = sp; }   // fewer splits on ties
  }
  int64_t kps = ((Kp + splits - 1) / splits + align - 1) / align * align;
  *kps_out = kps;
  return (Kp + kps - 1) / kps;
}

std::vector<int> lower_tiles(int nI, std::vector<int> *tindex) {
  std::vector<int> tiles;
  if (tindex) tindex->assign((size_t)nI * nI, -1);
  for (int I = 0; I < nI; ++I)
    for (int J = 0; J <= I; ++J) {
      if (tindex) (*tindex)[(size_t)I * nI + J] = (int)(tiles.size() / 2);
      tiles.push_back(I);
      tiles.push_back(J);
    }
  return tiles;
}

std::vector<int> full_tiles(int nI, int nJ) {
  std::vector<int> tiles;
  for (int I = 0; I < nI; ++I)
    for (int J = 0; J < nJ; ++J) { tiles.push_back(I); tiles.push_back(J); }
  return tiles;
}

// One split-BF16 contraction on the tensor cores.  Scratch (tile list,
// partials) comes from `ar`; the caller reduces the partials (returned).
struct TcRun {
  double *partial = nullptr;
  float *partial32 = nullptr;
  float *cd_out = nullptr;
  int splits = 1, groups = 1, n_tiles = 0, nt_group = 1;
};

// One configuration of a contraction: scales per CTA, K-split length, output precision.
struct TcPlan {
  int nt_group, groups;
  int64_t splits, kps;
  int out_mode;
};

TcPlan tc_plan(const ltgw_ctx *ctx, const TcGemmArgs &g, int n_tiles, int nt_group, int64_t want_splits) {
  TcPlan p;
  p.nt_group = nt_group;
  p.groups = (g.n_t + nt_group - 1) / nt_group;
  const int64_t align = g.A8 ? 128 : 64;
  const int64_t klen = (g.k_end ? g.k_end : g.Kp) - g.k_begin;   // pairs contracted
  if (g.out_mode == TC_OUT_COLDOT) {
    // the column dot needs the whole contraction (K = the NAF count) in one drain
    p.kps = klen; p.splits = 1; p.out_mode = TC_OUT_COLDOT;
    return p;
  }
  if (want_splits > 0) {
    p.kps = ((klen + want_splits - 1) / want_splits + align - 1) / align * align;
    p.splits = (klen + p.kps - 1) / p.kps;
  } else {
    p.splits = tc_splits(ctx, (int64_t)n_tiles * p.groups, klen, g.drain_k, align, &p.kps);
  }
  p.out_mode = p.kps <= g.drain_k ? TC_OUT_F32 : TC_OUT_F64;
  return p;
}

// Run a contraction.  Scratch (tile list, partials) comes from `ar`; the
// caller reduces the partials (returned with the configuration used).  With
// the autotuner on, the first contraction of a shape times its candidate
// configurations (scales per CTA where the kernel and the caller's reduction
// allow several; the heuristic's K-split count, half and twice it, each
// keeping one FP32 drain per CTA where one can) with CUDA events on the
// stream, keeps the fastest for this context and then runs it.
ltgw_status tc_run(ltgw_ctx *ctx, Arena &ar, TcGemmArgs g, const std::vector<int> &tiles, int coldot_rows,
                   TcRun *run, cudaStream_t s) {
  const int n_tiles = (int)(tiles.size() / 2);
  if (g.out_mode == TC_OUT_COLDOT) g.drain_k = std::max<int64_t>(g.drain_k, (g.k_end ? g.k_end : g.Kp) - g.k_begin);
  const int kind = g.A8 ? 2 : (g.B_hi ? (g.single ? 3 : 1) : 0);
  TcPlan plan = tc_plan(ctx, g, n_tiles, g.nt_group, 0);
  std::vector<TcPlan> cands{plan};
  const ltgw_ctx::TcKey key{kind, n_tiles, g.n_t, g.out_mode, (g.k_end ? g.k_end : g.Kp) - g.k_begin, g.rows_a,
                            g.rows_b};
  bool tune = false;
  if (ctx->autotune && g.out_mode != TC_OUT_COLDOT) {
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
      plan = tc_plan(ctx, g, n_tiles, it->second.nt_group, it->second.splits);
      cands = {plan};
    } else {
      tune = true;
      cands.clear();
      std::vector<int> ntgs{g.nt_group};
      // scales per CTA vary only where the caller reduces with reduce_sym (column-major partials)
      if (g.out_colmajor && g.n_t > 1 && kind == 1) ntgs = {2, 1};
      if (g.out_colmajor && g.n_t > 1 && kind == 2) ntgs = {4, 2, 1};
      const int64_t min_split = std::min<int64_t>(64, ((g.k_end ? g.k_end : g.Kp) - g.k_begin + g.drain_k - 1) / g.drain_k);
      for (int ntg : ntgs) {
        const TcPlan base = tc_plan(ctx, g, n_tiles, ntg, 0);
        for (int64_t sp : {base.splits, base.splits / 2, base.splits * 2}) {
          sp = std::max<int64_t>(std::max<int64_t>(sp, min_split), 1);
          const TcPlan c = tc_plan(ctx, g, n_tiles, ntg, sp);
          if (c.splits > 256) continue;
          bool dup = false;
          for (const TcPlan &o : cands) dup |= (o.nt_group == c.nt_group && o.splits == c.splits);
          if (!dup) cands.push_back(c);
        }
      }
    }
  }
  size_t part64_n = 0, part32_n = 0, cd_n = 0;
  for (const TcPlan &c : cands) {
    const size_t n_part = (size_t)c.splits * c.groups * c.nt_group * n_tiles * 128 * 128;
    if (c.out_mode == TC_OUT_F64) part64_n = std::max(part64_n, n_part);
    if (c.out_mode == TC_OUT_F32) part32_n = std::max(part32_n, n_part);
    if (c.out_mode == TC_OUT_COLDOT) cd_n = (size_t)c.splits * c.groups * coldot_rows * (size_t)g.cd_cols_p;
  }
  int *d_tiles;
  double *part64;
  float *part32, *cd;
  auto layout = [&](Arena &A) {
    d_tiles = A.take<int>(tiles.size());
    part64 = part64_n ? A.take<double>(part64_n) : nullptr;
    part32 = part32_n ? A.take<float>(part32_n) : nullptr;
    cd = cd_n ? A.take<float>(cd_n) : nullptr;
  };
  ar.begin_sizing();
  layout(ar);
  if (ar.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "tensor-core workspace allocation failed"); return ctx->status(); }
  layout(ar);
  copy_in(ctx, d_tiles, tiles.data(), tiles.size() * sizeof(int), s);
  g.tiles = d_tiles;
  g.n_tile_rows = coldot_rows;
  g.err = ctx->flags;
  auto launch = [&](const TcPlan &c) {
    TcGemmArgs h = g;
    h.nt_group = c.nt_group;
    h.k_per_split = c.kps;
    h.out_mode = c.out_mode;
    h.partial = c.out_mode == TC_OUT_F64 ? part64 : nullptr;
    h.partial32 = c.out_mode == TC_OUT_F32 ? part32 : nullptr;
    h.cd_out = c.out_mode == TC_OUT_COLDOT ? cd : nullptr;
    return h.A8 ? launch_tc_fp8_gemm(h, n_tiles, s) : launch_tc_split_gemm(h, n_tiles, s);
  };
  if (tune) {
    cudaEvent_t e0, e1;
    LTGW_CUDA(ctx, cudaEventCreate(&e0));
    LTGW_CUDA(ctx, cudaEventCreate(&e1));
    float best = 1e30f;
    for (const TcPlan &c : cands) {
      float ms = 0.0f;
      CHECK_LAUNCH(ctx, launch(c), 1);   // warm
      cudaEventRecord(e0, s);
      CHECK_LAUNCH(ctx, launch(c), 1);
      cudaEventRecord(e1, s);
      LTGW_CUDA(ctx, cudaEventSynchronize(e1));
      LTGW_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; plan = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tuned[key] = ltgw_ctx::TcChoice{plan.nt_group, plan.splits};
  }
  ctx->stats.tc_autotuned = (int)ctx->tuned.size();
  CHECK_LAUNCH(ctx, launch(plan), 1);
  run->partial = plan.out_mode == TC_OUT_F64 ? part64 : nullptr;
  run->partial32 = plan.out_mode == TC_OUT_F32 ? part32 : nullptr;
  run->cd_out = plan.out_mode == TC_OUT_COLDOT ? cd : nullptr;
  run->splits = (int)plan.splits;
  run->groups = plan.groups;
  run->n_tiles = n_tiles;
  run->nt_group = plan.nt_group;
  return LTGW_OK;
}

// Pi (direct) or the Laplace moments M^k on the tensor cores, split-BF16 or
// (fp8) FP8 E4M3 with per-row scales.  Operand: Af (FP32
// [roundup(N,128)][roundup(n_pairs,64)]) when given, else converted from the
// FP64 block Bt.  Scale table: the per-pair factor of Eq. Pi or of the M^m
// form, applied by the converter warps (split-BF16) or before quantisation (FP8).
ltgw_status polarizability_tc(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt, int64_t ldb,
                              const float *Af_in, const double *delta, int n_omega, const double *d_omega,
                              int n_tau, const double *d_x, const double *d_w, const double *d_E,
                              double *M, int spin, double *Pi, cudaStream_t s, bool fp8, int lt_form) {
  const int64_t Kp = (n_pairs + 63) / 64 * 64, Kq = (n_pairs + 127) / 128 * 128;
  const int nI = (N + 127) / 128, Mp = nI * 128;
  const int n_t = n_tau ? n_tau : n_omega;
  std::vector<int> tindex;
  std::vector<int> tiles = lower_tiles(nI, &tindex);
  float *Af = nullptr, *scale;
  __nv_bfloat16 *Bhi = nullptr, *Blo = nullptr;   // the unscaled operand, pre-split for the TMA-fed kernel
  uint8_t *qa = nullptr, *qb = nullptr;           // FP8 codes: scaled operands [n_t][Mp][3 Kq], B [Mp][3 Kq]
  float *ds_a = nullptr, *ds_b = nullptr;         // FP8 per-row de-scales
  int *d_tindex;
  auto layout = [&](Arena &A) {
    Af = Af_in ? nullptr : A.take<float>((size_t)Mp * Kp);
    scale = A.take<float>((size_t)n_t * Kp);
    if (fp8) {
      qa = A.take<uint8_t>((size_t)n_t * Mp * 3 * Kq);
      qb = A.take<uint8_t>((size_t)Mp * 3 * Kq);
      ds_a = A.take<float>((size_t)n_t * Mp);
      ds_b = A.take<float>((size_t)Mp);
    } else {
      Bhi = A.take<__nv_bfloat16>((size_t)Mp * Kp);
      Blo = A.take<__nv_bfloat16>((size_t)Mp * Kp);
    }
    d_tindex = A.take<int>(tindex.size());
  };
  ctx->a5.begin_sizing();
  layout(ctx->a5);
  if (ctx->a5.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "tensor-core operand allocation failed"); return ctx->status(); }
  layout(ctx->a5);
  const float *A = Af_in ? Af_in : Af;
  copy_in(ctx, d_tindex, tindex.data(), tindex.size() * sizeof(int), s);
  if (!Af_in) CHECK_LAUNCH(ctx, launch_to_f32_padded(Bt, ldb, N, n_pairs, Af, Mp, Kp, s), 1);
  const int mode = n_tau ? (lt_form == 2 ? SCALE_EXPTAU : SCALE_LAPLACE) : SCALE_DIRECT;
  CHECK_LAUNCH(ctx, launch_scale_table(delta, n_pairs, Kp, n_t, n_tau ? d_x : d_omega,
                                       mode == SCALE_LAPLACE ? d_w : nullptr, mode, scale, s), 1);
  TcGemmArgs g;
  if (fp8) {
    // two-term E4M3 expansions of both operands (three products over 3 Kq codes)
    CHECK_LAUNCH(ctx, launch_fp8_quantize(A, Kp, Kq, scale, n_t, Mp, qa, qb, ds_a, ds_b, s, 1), 1);
    // FP32 sums of exact E4M3 products: a 4096-code drain keeps the accumulation
    // bias (about 4e-6) below the expansion's rounding error
    g.A8 = qa; g.B8 = qb; g.ds_a = ds_a; g.ds_b = ds_b; g.Kp = 3 * Kq; g.nt_group = 2; g.drain_k = 4096;
  } else {
    CHECK_LAUNCH(ctx, launch_split_bf16(A, Bhi, Blo, (int64_t)Mp * Kp, s), 1);
    g.A = A; g.B = A; g.scale = scale; g.Kp = Kp; g.nt_group = 2; g.B_hi = Bhi; g.B_lo = Blo;
  }
  g.n_t = n_t; g.rows_a = Mp; g.rows_b = Mp; g.out_colmajor = 1;
  // Pairs go in blocks of at most 64 K-splits x drain_k (one FP32 drain per
  // CTA, partials bounded); each block's partials are added to Pi or M^k.
  TcRun run;
  const int64_t kblk = 64 * g.drain_k;
  ctx->mark(EV_PI0, s);
  for (int64_t k0 = 0; k0 < g.Kp; k0 += kblk) {
    TcGemmArgs gb = g;
    gb.k_begin = k0;
    gb.k_end = std::min(g.Kp, k0 + kblk);
    if (tc_run(ctx, ctx->a4, gb, tiles, 0, &run, s) != LTGW_OK) return ctx->status();
    if (gb.k_end == g.Kp) ctx->mark(EV_PI1, s);
    CHECK_LAUNCH(ctx, launch_tc_reduce_sym(run.partial, run.partial32, run.splits, run.groups, run.n_tiles, d_tindex,
                                           nI, n_t, N, n_tau ? 1.0 : -2.0 * spin, n_tau ? M : Pi, s,
                                           k0 ? 1.0 : 0.0, run.nt_group, 1), 1);
  }
  ctx->pi_tc_flops = (fp8 ? 1.0 : 3.0) * 2.0 * (double)run.n_tiles * 128 * 128 * (double)g.Kp * n_t;   // FP8: Kp = 3 Kq
  if (n_tau) {
    CHECK_LAUNCH(ctx, launch_recombine(M, n_tau, d_E, n_omega, (int64_t)N * N, -2.0 * spin, Pi, s, true),
                 (n_omega + 63) / 64);
  }
  return LTGW_OK;
}

// NAF metric K = B B^T (Eq. nafeq) in the split-BF16 form; K: device [n][n] FP64.
ltgw_status naf_metric_tc(ltgw_ctx *ctx, int n, int64_t n_pairs, const double *B, int64_t ld, double *K,
                          cudaStream_t s, double beta) {
  const int64_t Kp = (n_pairs + 63) / 64 * 64;
  const int nI = (n + 127) / 128, Mp = nI * 128;
  std::vector<int> tindex;
  std::vector<int> tiles = lower_tiles(nI, &tindex);
  float *Af, *ones;
  __nv_bfloat16 *Bhi, *Blo;   // the operand pre-split for the TMA-fed kernel
  int *d_tindex;
  auto layout = [&](Arena &A) {
    Af = A.take<float>((size_t)Mp * Kp);
    ones = A.take<float>((size_t)Kp);
    Bhi = A.take<__nv_bfloat16>((size_t)Mp * Kp);
    Blo = A.take<__nv_bfloat16>((size_t)Mp * Kp);
    d_tindex = A.take<int>(tindex.size());
  };
  ctx->a5.begin_sizing();
  layout(ctx->a5);
  if (ctx->a5.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "tensor-core operand allocation failed"); return ctx->status(); }
  layout(ctx->a5);
  copy_in(ctx, d_tindex, tindex.data(), tindex.size() * sizeof(int), s);
  CHECK_LAUNCH(ctx, launch_to_f32_padded(B, ld, n, n_pairs, Af, Mp, Kp, s), 1);
  CHECK_LAUNCH(ctx, launch_scale_table(nullptr, n_pairs, Kp, 1, nullptr, nullptr, SCALE_NONE, ones, s), 1);
  CHECK_LAUNCH(ctx, launch_split_bf16(Af, Bhi, Blo, (int64_t)Mp * Kp, s), 1);
  TcGemmArgs g;
  g.A = Af; g.B = Af; g.scale = ones; g.Kp = Kp; g.n_t = 1; g.nt_group = 1;
  g.B_hi = Bhi; g.B_lo = Blo; g.rows_a = Mp; g.rows_b = Mp; g.out_colmajor = 1;
  TcRun run;
  if (tc_run(ctx, ctx->a4, g, tiles, 0, &run, s) != LTGW_OK) return ctx->status();
  CHECK_LAUNCH(ctx, launch_tc_reduce_sym(run.partial, run.partial32, run.splits, run.groups, run.n_tiles, d_tindex,
                                         nI, 1, n, 1.0, K, s, beta, run.nt_group, 1), 1);
  return LTGW_OK;
}

// FP64-accurate products from integer slices on the tensor cores.  Each
// operand row is cut into s balanced base-128 digits of its fixed-point form
// (launch_slice_rows); the product sums 2^(-7(i+j)) a_i b_j^T over the digit
// pairs with i + j <= s + 1, every pair on the split-BF16 kernel in its
// one-product mode (A digits in FP32 convert to hi = digit exactly; B digits
// are the hi operand), so its integer products are exact and its FP32 sums too (|sum| <=
// 2^24: drains of 1024 pairs for the leading digits, |a_1 b_1| <= 2^14, and
// 2048 for the others, |a_i b_j| <= 2^13); the pair results
// are added in FP64 in the reduction, then scaled by 2^(e_A + e_B).
constexpr int kEmuSlices = 6;   // slices per operand row in the LTGW_FP64_EMU solve

struct EmuPlan {
  int m = 0, n = 0, s = 0, nIa = 0, nIb = 0, Mpa = 0, Mpb = 0;
  int64_t K = 0, Kp = 0, stra = 0, strb = 0;
  bool lower = false;   // lower tiles of a square product, mirrored
  std::vector<int> tiles, tindex;
  float *dA = nullptr, *ones = nullptr;
  __nv_bfloat16 *dB = nullptr;
  int *ea = nullptr, *eb = nullptr, *d_tindex = nullptr;
  double *factors = nullptr;   // n_factors x K FP64 column factors of A (optional)
  double *tmp = nullptr;       // m x n FP64 (optional): the unscaled sum when C accumulates
};

ltgw_status emu_prepare(ltgw_ctx *ctx, int m, int n, int64_t K, int s, bool lower, int n_factors, EmuPlan *p,
                        cudaStream_t st, bool need_tmp = false) {
  p->m = m; p->n = n; p->s = s; p->K = K; p->lower = lower;
  p->Kp = (K + 63) / 64 * 64;
  p->nIa = (m + 127) / 128; p->nIb = (n + 127) / 128;
  p->Mpa = p->nIa * 128; p->Mpb = p->nIb * 128;
  p->stra = (int64_t)p->Mpa * p->Kp; p->strb = (int64_t)p->Mpb * p->Kp;
  p->tiles = lower ? lower_tiles(p->nIa, &p->tindex) : full_tiles(p->nIa, p->nIb);
  auto layout = [&](Arena &Ar) {
    p->dA = Ar.take<float>((size_t)s * p->stra);
    p->dB = Ar.take<__nv_bfloat16>((size_t)s * p->strb);
    p->ones = Ar.take<float>((size_t)p->Kp);
    p->ea = Ar.take<int>(p->Mpa);
    p->eb = Ar.take<int>(p->Mpb);
    p->d_tindex = lower ? Ar.take<int>(p->tindex.size()) : nullptr;
    p->factors = n_factors ? Ar.take<double>((size_t)n_factors * K) : nullptr;
    p->tmp = need_tmp ? Ar.take<double>((size_t)m * n) : nullptr;
  };
  ctx->a5.begin_sizing();
  layout(ctx->a5);
  if (ctx->a5.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "slice operand allocation failed"); return ctx->status(); }
  layout(ctx->a5);
  if (lower) copy_in(ctx, p->d_tindex, p->tindex.data(), p->tindex.size() * sizeof(int), st);
  // padding rows (and, for column slicing, padding k) stay zero: the slicing
  // writes rows < m (n) only; row slicing writes every k < Kp, column slicing k < K
  LTGW_CUDA(ctx, cudaMemsetAsync(p->dA, 0, (size_t)s * p->stra * sizeof(float), st));
  LTGW_CUDA(ctx, cudaMemsetAsync(p->dB, 0, (size_t)s * p->strb * sizeof(__nv_bfloat16), st));
  LTGW_CUDA(ctx, cudaMemsetAsync(p->ea, 0, p->Mpa * sizeof(int), st));
  LTGW_CUDA(ctx, cudaMemsetAsync(p->eb, 0, p->Mpb * sizeof(int), st));
  CHECK_LAUNCH(ctx, launch_scale_table(nullptr, p->Kp, p->Kp, 1, nullptr, nullptr, SCALE_NONE, p->ones, st), 1);
  return ctx->status();
}

// C = beta C + post * (sliced A) (sliced B)^T from the digits in p->dA / p->dB
// and the exponents p->ea / p->eb.  C [m][ldc]; in the lower form C (ldc = n)
// is written whole and symmetric.  post must be plus or minus a power of two:
// it is folded into the exact 2^(-7L) factors.  beta != 0 needs p->tmp.
ltgw_status emu_pairs(ltgw_ctx *ctx, EmuPlan &p, double post, double *C, int64_t ldc, double beta,
                      cudaStream_t st) {
  if (beta != 0.0 && !p.tmp) { ctx->fail(LTGW_ERR_BAD_ARG, "emulated accumulation without scratch"); return ctx->status(); }
  double *D = beta != 0.0 ? p.tmp : C;
  const int64_t ldd = beta != 0.0 ? p.n : (p.lower ? p.m : ldc);
  bool first = true;
  for (int L = 2; L <= p.s + 1; ++L) {
    for (int i = 1; i < L; ++i) {
      const int j = L - i;
      if (i > p.s || j > p.s) continue;
      TcGemmArgs g;
      g.A = p.dA + (int64_t)(i - 1) * p.stra; g.B = nullptr; g.scale = p.ones; g.Kp = p.Kp; g.n_t = 1;
      g.nt_group = 1;
      g.B_hi = p.dB + (int64_t)(j - 1) * p.strb; g.B_lo = nullptr; g.rows_a = p.Mpa; g.rows_b = p.Mpb;
      g.single = 1;   // digits are exact in BF16: one product per step
      // FP32 sums of integers stay exact below 2^24: |a_1 b_1| <= 2^14 (1024
      // pairs per drain), every other pair has a digit of at most 64 in
      // magnitude, |a_i b_j| <= 2^13 (2048 pairs)
      g.drain_k = (i == 1 && j == 1) ? 1024 : 2048;
      g.out_colmajor = p.lower ? 1 : 0;
      TcRun run;
      if (tc_run(ctx, ctx->a4, g, p.tiles, 0, &run, st) != LTGW_OK) return ctx->status();
      const double alpha = post * ldexp(1.0, -7 * L);
      if (p.lower) {
        CHECK_LAUNCH(ctx, launch_tc_reduce_sym(run.partial, run.partial32, run.splits, run.groups, run.n_tiles,
                                               p.d_tindex, p.nIa, 1, p.m, alpha, D, st, first ? 0.0 : 1.0,
                                               run.nt_group, 1),
                     1);
      } else {
        CHECK_LAUNCH(ctx, launch_tc_reduce_full_acc(run.partial, run.partial32, run.splits, run.groups, run.n_tiles,
                                                    p.nIb, p.m, p.n, alpha, D, ldd, first ? 0.0 : 1.0, st), 1);
      }
      first = false;
    }
  }
  CHECK_LAUNCH(ctx, launch_scale_exp2_to(D, ldd, C, p.lower ? p.m : ldc, p.m, p.n, p.ea, p.eb, beta, st,
                                         p.lower ? 1 : 0), 1);
  return ctx->status();
}

// A (with optional column factors) sliced into p->dA, then emu_pairs.
ltgw_status emu_product(ltgw_ctx *ctx, EmuPlan &p, const double *A, int64_t lda, const double *colscale,
                        double post, double *C, int64_t ldc, cudaStream_t st, double beta = 0.0) {
  CHECK_LAUNCH(ctx, launch_slice_rows(A, lda, p.m, p.K, p.Kp, p.s, p.stra, p.dA, nullptr, p.ea, st, colscale), 1);
  return emu_pairs(ctx, p, post, C, ldc, beta, st);
}

// C = beta C + A A^T (lower form): A sliced once into both operands.
ltgw_status emu_syrk(ltgw_ctx *ctx, EmuPlan &p, const double *A, int64_t lda, double *C, double beta,
                     cudaStream_t st) {
  CHECK_LAUNCH(ctx, launch_slice_rows(A, lda, p.m, p.K, p.Kp, p.s, p.stra, p.dA, p.dB, p.ea, st), 1);
  LTGW_CUDA(ctx, cudaMemcpyAsync(p.eb, p.ea, p.Mpa * sizeof(int), cudaMemcpyDeviceToDevice, st));
  return emu_pairs(ctx, p, 1.0, C, p.m, beta, st);
}

ltgw_status emu_gemm(ltgw_ctx *ctx, int m, int n, int64_t K, const double *A, int64_t lda, const double *B,
                     int64_t ldb, double *C, int64_t ldc, bool sym, int s, cudaStream_t st) {
  EmuPlan p;
  if (emu_prepare(ctx, m, n, K, s, sym, 0, &p, st) != LTGW_OK) return ctx->status();
  if (sym) return emu_syrk(ctx, p, A, lda, C, 0.0, st);
  CHECK_LAUNCH(ctx, launch_slice_rows(B, ldb, n, K, p.Kp, s, p.strb, nullptr, p.dB, p.eb, st), 1);
  return emu_product(ctx, p, A, lda, nullptr, 1.0, C, ldc, st);
}

// Pi from slices (the emulated FP64 form): per frequency (n_tau == 0, Pi_j =
// -2 s M_j written directly) or moment t (lt_form 1: Laplace factors; 2:
// e^{-Delta tau_t}) M_t = (Bt diag(f_t)) Bt^T, then the recombination with
// d_E [n_omega][n_tau].
ltgw_status polarizability_emu(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt, int64_t ldb,
                               const double *delta, int n_omega, const double *d_om, int n_tau, const double *d_x,
                               const double *d_w, const double *d_E, double *d_M, int spin, double *Pi,
                               cudaStream_t s, int lt_form, int n_slices) {
  const int n_t = n_tau ? n_tau : n_omega;
  // pairs in chunks, so that the slices of one chunk are held at a time
  // (6 slices of FP32 A and BF16 B digits: 36 bytes per value); chunks after
  // the first are added (each chunk's product is exact to its own slices)
  const int64_t max_chunk = (int64_t)1 << 17;
  const int64_t n_chunks = (n_pairs + max_chunk - 1) / max_chunk;
  const int64_t chunk = std::min(n_pairs, ((n_pairs + n_chunks - 1) / n_chunks + 63) / 64 * 64);   // balanced
  EmuPlan p;
  if (emu_prepare(ctx, N, N, chunk, n_slices, true, n_t, &p, s, n_pairs > chunk) != LTGW_OK) return ctx->status();
  ctx->mark(EV_PI0, s);
  const int mode = n_tau ? (lt_form == 2 ? SCALE_EXPTAU : SCALE_LAPLACE) : SCALE_DIRECT;
  for (int64_t k0 = 0; k0 < n_pairs; k0 += chunk) {
    const int64_t kc = std::min(chunk, n_pairs - k0);
    p.K = kc;   // the row slicing writes every column < Kp: zeros past kc
    CHECK_LAUNCH(ctx, launch_pi_factor64(delta + k0, kc, n_t, n_tau ? d_x : d_om,
                                         mode == SCALE_LAPLACE ? d_w : nullptr, mode, p.factors, s), 1);
    CHECK_LAUNCH(ctx, launch_slice_rows(Bt + k0, ldb, N, kc, p.Kp, n_slices, p.strb, nullptr, p.dB, p.eb, s), 1);
    for (int t = 0; t < n_t; ++t)
      if (emu_product(ctx, p, Bt + k0, ldb, p.factors + (int64_t)t * kc, n_tau ? 1.0 : -2.0 * spin,
                      (n_tau ? d_M : Pi) + (int64_t)t * N * N, N, s, k0 > 0 ? 1.0 : 0.0) != LTGW_OK)
        return ctx->status();
  }
  ctx->mark(EV_PI1, s);
  if (n_tau)
    CHECK_LAUNCH(ctx, launch_recombine(d_M, n_tau, d_E, n_omega, (int64_t)N * N, -2.0 * spin, Pi, s),
                 (n_omega + 63) / 64);
  return LTGW_OK;
}

// Rows of R~ = U^T R from slices: Ut [N][n_aux] (rows = kept eigenvectors),
// R [n_aux][ld_r] with `cols` columns (pairs or orbitals); out [N][ld_out].
ltgw_status project_emu(ltgw_ctx *ctx, int N, int n_aux, const double *Ut, const double *R, int64_t ld_r,
                        int cols, double *out, int64_t ld_out, int n_slices, cudaStream_t s) {
  EmuPlan p;
  if (emu_prepare(ctx, N, cols, n_aux, n_slices, false, 0, &p, s) != LTGW_OK) return ctx->status();
  CHECK_LAUNCH(ctx, launch_slice_cols(R, ld_r, n_aux, cols, p.Kp, n_slices, p.strb, p.dB, p.eb, s), 1);
  return emu_product(ctx, p, Ut, n_aux, nullptr, 1.0, out, ld_out, s);
}

// W_j[t][c] = sum_PQ Btt[t][P][c] C_j[P][Q] Btt[t][Q][c] (Eq. ScreenedCoulombOrbital):
// Y = C_j Btt (all targets side by side) from slices, then the FP64 column dot.
ltgw_status wnm_emu(ltgw_ctx *ctx, int N, int n_omega, const double *C, int T, int n_orb_act, const double *Btt,
                    int64_t ld_btt, int64_t stride_btt, double *W, int n_slices, cudaStream_t s) {
  const int cols = T * n_orb_act;
  EmuPlan p;
  if (emu_prepare(ctx, N, cols, N, n_slices, false, 0, &p, s, true) != LTGW_OK) return ctx->status();
  for (int t = 0; t < T; ++t)
    CHECK_LAUNCH(ctx, launch_slice_cols(Btt + (int64_t)t * stride_btt, ld_btt, N, n_orb_act, p.Kp, n_slices,
                                        p.strb, p.dB + (int64_t)t * n_orb_act * p.Kp, p.eb + t * n_orb_act, s),
                 1);
  for (int j = 0; j < n_omega; ++j) {
    if (emu_product(ctx, p, C + (int64_t)j * N * N, N, nullptr, 1.0, p.tmp, cols, s) != LTGW_OK)
      return ctx->status();
    CHECK_LAUNCH(ctx, launch_coldot64(p.tmp, cols, Btt, ld_btt, stride_btt, N, n_orb_act, T,
                                      W + (int64_t)j * T * n_orb_act, n_orb_act, s), 1);
  }
  return LTGW_OK;
}

// Operands of the mixed form after the NAF step (Eq. naftrafo in split BF16):
//   Bf       FP32 [roundup(N,128)][roundup(n_ov,64)]   R~_ov, the Pi operand
//   BtT64    FP64 [T][n_orb_act][N]                      R~_tgt transposed (column dot)
//   BtT32    FP32 [roundup(T n_orb_act,128)][roundup(N,64)]  the W_nm operand
// With Ut == nullptr (no NAF) they are copies of the active blocks of B_ov, B_tgt.
// With `window` set, only the ov part runs, for n_ov columns of B_act written
// into columns [col0, col0 + n_ov) of Bf (row stride ld_bf); padding is left
// to the caller.  With Bh_in / Bl_in set (and B_act NULL), the ov block comes
// already transposed and split: BF16 hi / lo [roundup(n_ov,128)][roundup(n_aux,64)].
struct OvWindow {
  int64_t col0 = 0, ld_bf = 0;
};

ltgw_status naf_project_tc(ltgw_ctx *ctx, int N, int n_aux, const double *Ut, const double *B_act, int64_t ld_act,
                           int64_t n_ov, const double *B_tgt, int n_orb, int n_fc, int T, int n_orb_act, float *Bf,
                           double *BtT64, float *BtT32, cudaStream_t s, const OvWindow *window = nullptr,
                           const __nv_bfloat16 *Bh_in = nullptr, const __nv_bfloat16 *Bl_in = nullptr) {
  const int64_t Kp_ov = (n_ov + 63) / 64 * 64;
  const int MpN = (N + 127) / 128 * 128, KpN = (N + 63) / 64 * 64;
  const int64_t rowsT = (int64_t)T * n_orb_act, rowsTp = (rowsT + 127) / 128 * 128;
  if (!Ut) {
    CHECK_LAUNCH(ctx, launch_to_f32_padded(B_act, ld_act, N, n_ov, Bf, MpN, Kp_ov, s), 1);
    CHECK_LAUNCH(ctx, launch_transpose_f64(B_tgt, n_orb, n_fc, n_aux, n_orb_act, BtT64, N, T,
                                           (int64_t)n_aux * n_orb, (int64_t)n_orb_act * N, s), 1);
    CHECK_LAUNCH(ctx, launch_to_f32_transposed(B_tgt, n_orb, n_fc, n_aux, n_orb_act, BtT32, KpN, n_orb_act, T,
                                               (int64_t)n_aux * n_orb, (int64_t)n_orb_act * KpN, s), 1);
    if (rowsTp > rowsT)
      LTGW_CUDA(ctx, cudaMemsetAsync(BtT32 + rowsT * KpN, 0, (size_t)(rowsTp - rowsT) * KpN * sizeof(float), s));
    return LTGW_OK;
  }
  const int Kpa = (n_aux + 63) / 64 * 64;
  const int nI_ov = (int)((n_ov + 127) / 128);
  const int MpT = (n_orb_act + 127) / 128 * 128;
  float *UtF, *BactT, *BtgT, *ones;
  __nv_bfloat16 *Bh, *Bl, *Uh = nullptr, *Ul = nullptr;   // B operands pre-split for the TMA-fed kernel
  const bool pre = Bh_in != nullptr;
  auto layout = [&](Arena &A) {
    UtF = A.take<float>((size_t)MpN * Kpa);
    BactT = (B_act && !pre) ? A.take<float>((size_t)nI_ov * 128 * Kpa) : nullptr;
    BtgT = window ? nullptr : A.take<float>((size_t)T * MpT * Kpa);
    ones = A.take<float>((size_t)std::max(T, 1) * Kpa);
    Bh = (B_act && !pre) ? A.take<__nv_bfloat16>((size_t)nI_ov * 128 * Kpa) : nullptr;
    Bl = (B_act && !pre) ? A.take<__nv_bfloat16>((size_t)nI_ov * 128 * Kpa) : nullptr;
    if (!window) {
      Uh = A.take<__nv_bfloat16>((size_t)MpN * Kpa);
      Ul = A.take<__nv_bfloat16>((size_t)MpN * Kpa);
    }
  };
  ctx->a5.begin_sizing();
  layout(ctx->a5);
  if (ctx->a5.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "tensor-core operand allocation failed"); return ctx->status(); }
  layout(ctx->a5);
  CHECK_LAUNCH(ctx, launch_to_f32_padded(Ut, n_aux, N, n_aux, UtF, MpN, Kpa, s), 1);
  if (B_act && !pre)
    CHECK_LAUNCH(ctx, launch_to_f32_transposed(B_act, ld_act, 0, n_aux, (int)n_ov, BactT, Kpa, nI_ov * 128, 1, 0, 0, s),
                 1);
  if (!window)
    CHECK_LAUNCH(ctx, launch_to_f32_transposed(B_tgt, n_orb, n_fc, n_aux, n_orb_act, BtgT, Kpa, MpT, T,
                                               (int64_t)n_aux * n_orb, (int64_t)MpT * Kpa, s), 1);
  CHECK_LAUNCH(ctx, launch_scale_table(nullptr, n_aux, Kpa, std::max(T, 1), nullptr, nullptr, SCALE_NONE, ones, s), 1);
  // R~_ov = U^T R_ov: rows N (A = U^T), columns n_ov (B rows = R_ov^T)
  if (B_act || pre) {
    if (!pre) CHECK_LAUNCH(ctx, launch_split_bf16(BactT, Bh, Bl, (int64_t)nI_ov * 128 * Kpa, s), 1);
    TcGemmArgs g;
    g.A = UtF; g.B = BactT; g.scale = ones; g.Kp = Kpa; g.n_t = 1; g.nt_group = 1;
    g.B_hi = pre ? Bh_in : Bh; g.B_lo = pre ? Bl_in : Bl; g.rows_a = MpN; g.rows_b = (int64_t)nI_ov * 128;
    TcRun run;
    const int nI = (N + 127) / 128;
    if (tc_run(ctx, ctx->a4, g, full_tiles(nI, nI_ov), 0, &run, s) != LTGW_OK) return ctx->status();
    if (window) {
      CHECK_LAUNCH(ctx, launch_tc_reduce_full(run.partial, run.partial32, run.splits, run.groups, run.n_tiles, nI_ov,
                                              N, (int)n_ov, 1.0, nullptr, 0, 0, Bf + window->col0, window->ld_bf,
                                              MpN, 0, s, n_ov), 1);
      return LTGW_OK;
    }
    CHECK_LAUNCH(ctx, launch_tc_reduce_full(run.partial, run.partial32, run.splits, run.groups, run.n_tiles, nI_ov, N,
                                            (int)n_ov, 1.0, nullptr, 0, 0, Bf, Kp_ov, MpN, 0, s), 1);
  }
  // R~_tgt[t]^T = R_tgt[t]^T U: per target t, rows n_orb_act (A), columns N (B rows = U^T)
  {
    CHECK_LAUNCH(ctx, launch_split_bf16(UtF, Uh, Ul, (int64_t)MpN * Kpa, s), 1);
    TcGemmArgs g;
    g.A = BtgT; g.a_group_stride = (int64_t)MpT * Kpa; g.B = UtF; g.scale = ones; g.Kp = Kpa;
    g.n_t = T; g.nt_group = 1;
    g.B_hi = Uh; g.B_lo = Ul; g.rows_a = MpT; g.rows_b = MpN;
    TcRun run;
    const int nJ = (N + 127) / 128;
    if (tc_run(ctx, ctx->a4, g, full_tiles(MpT / 128, nJ), 0, &run, s) != LTGW_OK) return ctx->status();
    CHECK_LAUNCH(ctx, launch_tc_reduce_full(run.partial, run.partial32, run.splits, run.groups, run.n_tiles, nJ,
                                            n_orb_act, N, 1.0, BtT64, N, (int64_t)n_orb_act * N, BtT32, KpN,
                                            n_orb_act, (int64_t)n_orb_act * KpN, s), 1);
    if (rowsTp > rowsT)
      LTGW_CUDA(ctx, cudaMemsetAsync(BtT32 + rowsT * KpN, 0, (size_t)(rowsTp - rowsT) * KpN * sizeof(float), s));
  }
  return LTGW_OK;
}

// W_nm(i w_j) (Eq. ScreenedCoulombOrbital) on the tensor cores: Y_j = C_j R~_tgt
// with the column dot against R~_tgt fused into the epilogue; split BF16, or
// (fp8) FP8 E4M3 codes of C_j's and R~_tgt^T's rows, each row with its own
// scale (C_j's rows are auxiliary functions).
ltgw_status wnm_tc(ltgw_ctx *ctx, int N, int n_omega, const double *C, int T, int n_orb_act, const double *BtT64,
                   const float *BtT32, double *W, cudaStream_t s, bool fp8) {
  const int KpN = (N + 63) / 64 * 64, MpN = (N + 127) / 128 * 128, nI = MpN / 128, Kq = (N + 127) / 128 * 128;
  const int ncols = T * n_orb_act, nJ = (ncols + 127) / 128, rowsTp = nJ * 128;
  float *Cf, *ones = nullptr, *dsC = nullptr, *dsR = nullptr;
  uint8_t *qC = nullptr, *qR = nullptr;
  __nv_bfloat16 *Rh = nullptr, *Rl = nullptr;   // R~_tgt^T pre-split for the TMA-fed kernel
  auto layout = [&](Arena &A) {
    Cf = A.take<float>((size_t)n_omega * MpN * KpN);
    if (fp8) {
      qC = A.take<uint8_t>((size_t)n_omega * MpN * 3 * Kq);
      qR = A.take<uint8_t>((size_t)rowsTp * 3 * Kq);
      dsC = A.take<float>((size_t)n_omega * MpN);
      dsR = A.take<float>((size_t)rowsTp);
    } else {
      ones = A.take<float>((size_t)n_omega * KpN);
      Rh = A.take<__nv_bfloat16>((size_t)rowsTp * KpN);
      Rl = A.take<__nv_bfloat16>((size_t)rowsTp * KpN);
    }
  };
  ctx->a5.begin_sizing();
  layout(ctx->a5);
  if (ctx->a5.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "tensor-core operand allocation failed"); return ctx->status(); }
  layout(ctx->a5);
  // C_j is symmetric, so its transpose is its padded copy
  CHECK_LAUNCH(ctx, launch_to_f32_transposed(C, N, 0, N, N, Cf, KpN, MpN, n_omega, (int64_t)N * N,
                                             (int64_t)MpN * KpN, s), 1);
  TcGemmArgs g;
  if (fp8) {
    // two-term E4M3 expansions: C_j's rows as A operands, R~_tgt^T's as B
    CHECK_LAUNCH(ctx, launch_fp8_quantize_a(Cf, KpN, Kq, n_omega * MpN, qC, dsC, s, 1), 1);
    CHECK_LAUNCH(ctx, launch_fp8_quantize(BtT32, KpN, Kq, nullptr, 0, rowsTp, nullptr, qR, nullptr, dsR, s, 1), 1);
    g.A8 = qC; g.B8 = qR; g.ds_a = dsC; g.ds_b = dsR; g.Kp = 3 * Kq; g.rows_a = MpN; g.rows_b = rowsTp;
  } else {
    CHECK_LAUNCH(ctx, launch_scale_table(nullptr, N, KpN, n_omega, nullptr, nullptr, SCALE_NONE, ones, s), 1);
    CHECK_LAUNCH(ctx, launch_split_bf16(BtT32, Rh, Rl, (int64_t)rowsTp * KpN, s), 1);
    g.A = Cf; g.a_group_stride = (int64_t)MpN * KpN; g.B = BtT32; g.scale = ones; g.Kp = KpN;
    g.B_hi = Rh; g.B_lo = Rl; g.rows_a = MpN; g.rows_b = rowsTp;   // C_j stacked by frequency
  }
  g.n_t = n_omega; g.nt_group = 1;
  g.out_mode = TC_OUT_COLDOT;
  g.cd_B = BtT64; g.cd_ld = N; g.cd_rows = N; g.cd_cols = ncols; g.cd_cols_p = nJ * 128;
  TcRun run;
  if (tc_run(ctx, ctx->a4, g, full_tiles(nI, nJ), nI, &run, s) != LTGW_OK) return ctx->status();
  CHECK_LAUNCH(ctx, launch_tc_reduce_coldot(run.cd_out, run.splits, run.groups, nI, nJ * 128, ncols, W, ncols, s), 1);
  return LTGW_OK;
}

ltgw_status validate(ltgw_ctx *ctx, const ltgw_params *p) {
  REQUIRE(ctx, p != nullptr, "params is NULL");
  REQUIRE(ctx, p->n_occ >= 1 && p->n_virt >= 1 && p->n_aux >= 1, "n_occ, n_virt, n_aux must be >= 1");
  REQUIRE(ctx, p->n_frozen >= 0 && p->n_frozen < p->n_occ, "need 0 <= n_frozen < n_occ");
  REQUIRE(ctx, p->n_omega >= 1 && p->n_omega <= 256, "n_omega must be in [1, 256]");
  REQUIRE(ctx, p->omega0 > 0.0 && isfinite(p->omega0), "omega0 must be positive");
  REQUIRE(ctx, p->spin == 1 || p->spin == 2, "spin must be 1 or 2");
  REQUIRE(ctx, p->use_laplace >= 0 && p->use_laplace <= 2, "use_laplace must be 0, 1 or 2");
  REQUIRE(ctx, !p->use_laplace || (p->n_tau >= 1 && p->n_tau <= 32), "n_tau must be in [1, 32]");
  REQUIRE(ctx, p->precision >= LTGW_FP64 && p->precision <= LTGW_FP64_EMU,
          "precision must be LTGW_FP64, LTGW_BF16X3, LTGW_FP8, LTGW_FP8_PI or LTGW_FP64_EMU");
  REQUIRE(ctx, p->reserved == 0, "reserved must be 0");
  REQUIRE(ctx, isfinite(p->naf_thresh), "naf_thresh must be finite");
  return LTGW_OK;
}

}  // namespace

extern "C" {

const char *ltgw_status_string(ltgw_status s) {
  switch (s) {
    case LTGW_OK: return "ok";
    case LTGW_ERR_BAD_ARG: return "bad argument";
    case LTGW_ERR_NOMEM: return "out of memory";
    case LTGW_ERR_NOT_SPD: return "1 - Pi not positive definite";
    case LTGW_ERR_NO_CONVERGE: return "quasi-particle solve did not converge";
    case LTGW_ERR_DEVICE: return "CUDA error";
    case LTGW_ERR_EIG: return "eigensolver failure";
    case LTGW_ERR_NO_NAF: return "no natural auxiliary function kept";
    case LTGW_ERR_TIMEOUT: return "timed out";
  }
  return "unknown status";
}

ltgw_status ltgw_create(ltgw_ctx **out, int device) {
  if (!out) return LTGW_ERR_BAD_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return LTGW_ERR_DEVICE;
  }
  if (cudaSetDevice(device) != cudaSuccess) return LTGW_ERR_DEVICE;
  ltgw_ctx *c = new ltgw_ctx();
  c->device = device;
  if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->n_sm < 1) {
    cudaGetLastError();
    c->n_sm = 148;
  }
  if (cudaMalloc(&c->flags, FLAG_COUNT * sizeof(int)) != cudaSuccess) {
    delete c;
    return LTGW_ERR_NOMEM;
  }
  for (auto &e : c->ev) cudaEventCreate(&e);
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->fill_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->blk_ready[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->blk_ready[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->blk_done[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->blk_done[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ltgw_destroy(c);
    return LTGW_ERR_DEVICE;
  }
  *out = c;
  return LTGW_OK;
}

void ltgw_destroy(ltgw_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  ctx->a1.release();
  ctx->a2.release();
  ctx->a3.release();
  ctx->a4.release();
  ctx->a5.release();
  if (ctx->flags) cudaFree(ctx->flags);
  for (auto &e : ctx->ev) if (e) cudaEventDestroy(e);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  if (ctx->fill_stream) cudaStreamDestroy(ctx->fill_stream);
  for (int b = 0; b < 2; ++b) {
    if (ctx->blk_ready[b]) cudaEventDestroy(ctx->blk_ready[b]);
    if (ctx->blk_done[b]) cudaEventDestroy(ctx->blk_done[b]);
  }
  delete ctx;
}

const char *ltgw_last_error(const ltgw_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

ltgw_status ltgw_set_timing(ltgw_ctx *ctx, int on) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->timing = (on != 0);
  return LTGW_OK;
}

size_t ltgw_workspace_bytes(const ltgw_ctx *ctx) {
  if (!ctx) return 0;
  return ctx->a1.cap + ctx->a2.cap + ctx->a3.cap + ctx->a4.cap + ctx->a5.cap;
}

ltgw_status ltgw_trim(ltgw_ctx *ctx) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  LTGW_CUDA(ctx, cudaSetDevice(ctx->device));
  ctx->a1.release();
  ctx->a2.release();
  ctx->a3.release();
  ctx->a4.release();
  ctx->a5.release();
  return LTGW_OK;
}

ltgw_status ltgw_set_autotune(ltgw_ctx *ctx, int on) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->autotune = (on != 0);
  return LTGW_OK;
}

ltgw_status ltgw_get_stats(const ltgw_ctx *ctx, ltgw_stats *out) {
  if (!ctx || !out) return LTGW_ERR_BAD_ARG;
  *out = ctx->stats;
  return LTGW_OK;
}

}  // extern "C"

namespace {

// One solve; with `fill` set, B_ov is not given and the occupied blocks are
// requested from the caller twice (NAF metric, then projection).
// One solve; ev_cycles > 0 adds evGW cycles (Sec. 3): Pi, W and Sigma rebuilt
// from the previous quasi-particle energies (targets) and the scissor shift of
// the nearest target (other active orbitals), the NAF basis and the projected
// tensors kept, until the HOMO/LUMO quasi-particle gap changes by less than
// ev_gap_tol (> 0; both states among the targets) or ev_cycles cycles ran.
ltgw_status solve_impl(ltgw_ctx *ctx, const ltgw_params *p, const double *eps, const double *B_ov,
                       ltgw_block_fn fill, void *user, int occ_block, const double *B_tgt, const int *targets,
                       int n_tgt, const double *shift, const double *tau_x, const double *tau_w,
                       double *sigma_iw, double *e_qp, int *qp_status, void *stream, int ev_cycles = 0,
                       double ev_gap_tol = 0.0, int *ev_done = nullptr) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->reset();
  if (validate(ctx, p) != LTGW_OK) return ctx->status();
  const bool streamed = fill != nullptr;
  REQUIRE(ctx, eps && (B_ov || streamed) && B_tgt && targets && shift && sigma_iw && e_qp && qp_status,
          "a required pointer is NULL");
  REQUIRE(ctx, !streamed || (p->naf_thresh >= 0.0 && occ_block >= 1),
          "the streamed solve needs NAF (naf_thresh >= 0) and occ_block >= 1");
  REQUIRE(ctx, n_tgt >= 1, "n_tgt must be >= 1");
  REQUIRE(ctx, (tau_x == nullptr) == (tau_w == nullptr), "tau_x and tau_w must both be given or both NULL");
  REQUIRE(ctx, ev_cycles >= 0 && ev_cycles <= 100 && ev_gap_tol >= 0.0, "need 0 <= ev_cycles <= 100, ev_gap_tol >= 0");
  LTGW_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int n_occ = p->n_occ, n_virt = p->n_virt, n_fc = p->n_frozen, n_aux = p->n_aux;
  const int n_orb = n_occ + n_virt, n_act = n_occ - n_fc, n_orb_act = n_orb - n_fc;
  const int64_t n_ov_all = (int64_t)n_occ * n_virt, n_ov = (int64_t)n_act * n_virt;
  const int n_omega = p->n_omega, T = n_tgt;
  const int n_tau = p->use_laplace ? p->n_tau : 0;
  const bool naf = p->naf_thresh >= 0.0;
  // emulated FP64 form: the FP64 form's data flow with K, the projections, Pi
  // and W_nm FP64-accurate from integer slices on the tensor cores
  const bool emu = p->precision == LTGW_FP64_EMU;
  const int n_sl = kEmuSlices;
  const bool mixed = p->precision != LTGW_FP64 && !emu;   // split-BF16 / FP8 contractions
  const bool fp8 = p->precision == LTGW_FP8 || p->precision == LTGW_FP8_PI;   // Pi build in FP8 E4M3
  const bool fp8_w = p->precision == LTGW_FP8;                                // W_nm in FP8 E4M3
  ctx->stats = ltgw_stats{};
  ctx->mark(EV_START, s);

  // small inputs on the host
  std::vector<double> h_eps(n_orb), h_shift(T);
  std::vector<int> h_tg(T);
  if (read_small(ctx, h_eps.data(), eps, n_orb * sizeof(double), s) != LTGW_OK) return ctx->status();
  if (read_small(ctx, h_tg.data(), targets, T * sizeof(int), s) != LTGW_OK) return ctx->status();
  if (read_small(ctx, h_shift.data(), shift, T * sizeof(double), s) != LTGW_OK) return ctx->status();
  for (int i = 0; i < n_orb; ++i) REQUIRE(ctx, isfinite(h_eps[i]), "eps has a non-finite entry");
  for (int i = 1; i < n_orb; ++i) REQUIRE(ctx, h_eps[i] >= h_eps[i - 1], "eps must be ascending");
  REQUIRE(ctx, h_eps[n_occ] > h_eps[n_occ - 1], "need eps_LUMO > eps_HOMO");
  for (int t = 0; t < T; ++t)
    REQUIRE(ctx, h_tg[t] >= n_fc && h_tg[t] < n_orb, "target outside the active orbitals");
  double eF = 0.5 * (h_eps[n_occ - 1] + h_eps[n_occ]);
  std::vector<double> h_om(n_omega), h_wt(n_omega);
  if (ltgw_gl_grid(n_omega, p->omega0, h_om.data(), h_wt.data()) != LTGW_OK) {
    ctx->fail(LTGW_ERR_BAD_ARG, "GL grid");
    return ctx->status();
  }
  std::vector<double> h_x(n_tau), h_w(n_tau), h_E((size_t)n_omega * std::max(n_tau, 1));
  ctx->stats.lt_max_rel_err = NAN;
  // The library's grid for orbital energies e: Eq. LT's bounds of Sec. 3
  // (a = gap^2 + w_min^2, b = max(span^2, 1e4)), or the imaginary-time fit on
  // [gap, span] (the tensor-core forms carry ~1e-5 relative error in M^k: a
  // larger ridge keeps the recombination from magnifying it).
  auto fit_grid = [&](const std::vector<double> &e) -> ltgw_status {
    const double gap = e[n_occ] - e[n_occ - 1];
    const double span = *std::max_element(e.begin() + n_fc, e.end()) - *std::min_element(e.begin() + n_fc, e.end());
    double err = 0.0;
    if (p->use_laplace == 2) {
      if (ltgw_cosine_grid(n_tau, gap, span, n_omega, h_om.data(), mixed ? 1e-10 : 1e-14, h_x.data(), h_E.data(),
                           &err, nullptr) != LTGW_OK) {
        ctx->fail(LTGW_ERR_BAD_ARG, "imaginary-time grid fit");
        return ctx->status();
      }
    } else {
      if (ltgw_laplace_grid(n_tau, gap * gap + h_om[0] * h_om[0], std::max(span * span, 1e4), h_x.data(), h_w.data(),
                            &err) != LTGW_OK) {
        ctx->fail(LTGW_ERR_BAD_ARG, "Laplace grid fit");
        return ctx->status();
      }
      for (int j = 0; j < n_omega; ++j)
        for (int k = 0; k < n_tau; ++k) h_E[(size_t)j * n_tau + k] = exp(-h_om[j] * h_om[j] * h_x[k]);
    }
    ctx->stats.lt_max_rel_err = err;
    return LTGW_OK;
  };
  if (n_tau && tau_x) {
    // caller's grid: Eq. LT (x, w), or imaginary time (tau_k, gamma [n_omega][n_tau])
    if (read_small(ctx, h_x.data(), tau_x, n_tau * sizeof(double), s) != LTGW_OK) return ctx->status();
    if (p->use_laplace == 2) {
      if (read_small(ctx, h_E.data(), tau_w, h_E.size() * sizeof(double), s) != LTGW_OK) return ctx->status();
    } else {
      if (read_small(ctx, h_w.data(), tau_w, n_tau * sizeof(double), s) != LTGW_OK) return ctx->status();
      for (int j = 0; j < n_omega; ++j)
        for (int k = 0; k < n_tau; ++k) h_E[(size_t)j * n_tau + k] = exp(-h_om[j] * h_om[j] * h_x[k]);
    }
  } else if (n_tau && fit_grid(h_eps) != LTGW_OK) {
    return ctx->status();
  }
  std::vector<double> h_epsn(T);
  for (int t = 0; t < T; ++t) h_epsn[t] = h_eps[h_tg[t]];

  const bool bov_dev = streamed || is_device_ptr(B_ov), btg_dev = is_device_ptr(B_tgt);
  // a streamed solve that fails leaves no callback work in flight behind it
  struct FillDrain {
    ltgw_ctx *ctx;
    bool on;
    ~FillDrain() {
      if (on) cudaStreamSynchronize(ctx->fill_stream);
    }
  } fill_drain{ctx, streamed};
  const int blk = streamed ? std::min(occ_block, n_act) : 0;
  double *d_blk[2] = {nullptr, nullptr};
  // streamed tensor-core forms: every block, transposed and split into BF16
  // hi / lo as the projection's operand, is kept from the metric's pass, so
  // that the callback is asked for each block once
  const bool keep_split = streamed && mixed;
  const int64_t n_ov_p = (n_ov + 127) / 128 * 128, Kpa_aux = (n_aux + 63) / 64 * 64;
  __nv_bfloat16 *d_Rh = nullptr, *d_Rl = nullptr;
  float *d_Rt = nullptr;   // one block, transposed, FP32
  ctx->gen_ms = 0.0;
  // ---- phase-1 workspace: inputs, grids, NAF
  double *d_eps, *d_delta, *d_om, *d_wt, *d_x, *d_w, *d_E, *d_epsn, *d_shift, *d_Bov, *d_Btg, *d_Ut, *d_lam;
  auto layout1 = [&](Arena &A) {
    d_eps = A.take<double>(n_orb);
    d_delta = A.take<double>(n_ov);
    d_om = A.take<double>(n_omega);
    d_wt = A.take<double>(n_omega);
    d_x = A.take<double>(std::max(n_tau, 1));
    d_w = A.take<double>(std::max(n_tau, 1));
    d_E = A.take<double>(h_E.size());
    d_epsn = A.take<double>(T);
    d_shift = A.take<double>(T);
    d_Bov = bov_dev ? const_cast<double *>(B_ov) : A.take<double>((size_t)n_aux * n_ov_all);
    d_blk[0] = streamed ? A.take<double>((size_t)n_aux * blk * n_virt) : nullptr;
    d_blk[1] = streamed ? A.take<double>((size_t)n_aux * blk * n_virt) : nullptr;
    d_Rh = keep_split ? A.take<__nv_bfloat16>((size_t)n_ov_p * Kpa_aux) : nullptr;
    d_Rl = keep_split ? A.take<__nv_bfloat16>((size_t)n_ov_p * Kpa_aux) : nullptr;
    d_Rt = keep_split ? A.take<float>((size_t)blk * n_virt * Kpa_aux) : nullptr;
    d_Btg = btg_dev ? const_cast<double *>(B_tgt) : A.take<double>((size_t)T * n_aux * n_orb);
    d_Ut = naf ? A.take<double>((size_t)n_aux * n_aux) : nullptr;
    d_lam = naf ? A.take<double>(n_aux) : nullptr;
  };
  ctx->a1.begin_sizing();
  layout1(ctx->a1);
  if (ctx->a1.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "input workspace allocation failed"); return ctx->status(); }
  layout1(ctx->a1);
  LTGW_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
  copy_in(ctx, d_eps, h_eps.data(), n_orb * sizeof(double), s);
  copy_in(ctx, d_om, h_om.data(), n_omega * sizeof(double), s);
  copy_in(ctx, d_wt, h_wt.data(), n_omega * sizeof(double), s);
  if (n_tau) {
    copy_in(ctx, d_x, h_x.data(), n_tau * sizeof(double), s);
    copy_in(ctx, d_w, h_w.data(), n_tau * sizeof(double), s);
    copy_in(ctx, d_E, h_E.data(), h_E.size() * sizeof(double), s);
  }
  copy_in(ctx, d_epsn, h_epsn.data(), T * sizeof(double), s);
  copy_in(ctx, d_shift, h_shift.data(), T * sizeof(double), s);
  // a solve that fails from here on waits for its stream before it returns,
  // so that no copy from the caller's (possibly pinned) B_ov or B_tgt is
  // still in flight when the call returns
  struct SyncOnError {
    ltgw_ctx *ctx;
    cudaStream_t s;
    bool active;
    ~SyncOnError() {
      if (active && ctx->status() != LTGW_OK) cudaStreamSynchronize(s);
    }
  } sync_on_error{ctx, s, !bov_dev || !btg_dev};
  // host B_ov: only the active pairs' columns cross the link (the frozen
  // columns are never read)
  if (!bov_dev && n_fc == 0) copy_in(ctx, d_Bov, B_ov, (size_t)n_aux * n_ov_all * sizeof(double), s);
  if (!bov_dev && n_fc > 0)
    LTGW_CUDA(ctx, cudaMemcpy2DAsync(d_Bov + (int64_t)n_fc * n_virt, (size_t)n_ov_all * sizeof(double),
                                     B_ov + (int64_t)n_fc * n_virt, (size_t)n_ov_all * sizeof(double),
                                     (size_t)n_ov * sizeof(double), (size_t)n_aux, cudaMemcpyDefault, s));
  // host B_tgt is first read by the projections, after the NAF: its copy runs
  // on the side stream meanwhile.  A solve that fails before the join waits
  // for the copy, so the caller may release B_tgt when the call returns.
  struct SideJoin {
    ltgw_ctx *ctx = nullptr;
    bool pending = false;
    ltgw_status join(cudaStream_t s) {
      if (!pending) return LTGW_OK;
      pending = false;
      LTGW_CUDA(ctx, cudaStreamWaitEvent(s, ctx->join_ev, 0));
      return LTGW_OK;
    }
    ~SideJoin() {
      if (pending) cudaStreamSynchronize(ctx->side);
    }
  } btg_join;
  btg_join.ctx = ctx;
  if (!btg_dev) {
    LTGW_CUDA(ctx, cudaEventRecord(ctx->fork_ev, s));
    LTGW_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0));
    LTGW_CUDA(ctx, cudaMemcpyAsync(d_Btg, B_tgt, (size_t)T * n_aux * n_orb * sizeof(double), cudaMemcpyDefault,
                                   ctx->side));
    btg_join.pending = true;
    LTGW_CUDA(ctx, cudaEventRecord(ctx->join_ev, ctx->side));
  }
  if (ctx->status() != LTGW_OK) return ctx->status();
  CHECK_LAUNCH(ctx, launch_pair_gaps(d_eps, n_occ, n_virt, n_fc, d_delta, s), 1);

  // ---- frozen-core slice: the active pairs are the trailing columns
  const double *B_act = streamed ? nullptr : d_Bov + (int64_t)n_fc * n_virt;
  const int64_t ld_act = n_ov_all;
  // streamed: ask the caller for occupied block [i0, i1) into the next of the
  // two block buffers (*dst).  The buffer's previous consumers are waited for
  // on the host first, so the callback may write it by any means; its work,
  // issued on the fill stream, then overlaps the consumers of the other
  // buffer on `s`, which waits for the block's arrival.  block_done() marks
  // the block's consumers issued.
  int blk_next = 0;
  auto get_block = [&](int i0, int i1, double **dst) -> ltgw_status {
    const int b = blk_next;
    LTGW_CUDA(ctx, cudaEventSynchronize(ctx->blk_done[b]));
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = fill(user, i0, i1, d_blk[b], (void *)ctx->fill_stream);
    ctx->gen_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc != 0) {
      cudaStreamSynchronize(ctx->fill_stream);
      ctx->fail(LTGW_ERR_BAD_ARG, "the block callback reported an error");
      return ctx->status();
    }
    LTGW_CUDA(ctx, cudaEventRecord(ctx->blk_ready[b], ctx->fill_stream));
    LTGW_CUDA(ctx, cudaStreamWaitEvent(s, ctx->blk_ready[b], 0));
    *dst = d_blk[b];
    return LTGW_OK;
  };
  auto block_done = [&]() -> ltgw_status {
    LTGW_CUDA(ctx, cudaEventRecord(ctx->blk_done[blk_next], s));
    blk_next ^= 1;
    return LTGW_OK;
  };
  KBuilder build_K = [&](double *K) -> ltgw_status {
    LTGW_CUDA(ctx, cudaMemsetAsync(K, 0, (size_t)n_aux * n_aux * sizeof(double), s));
    for (int i0 = n_fc; i0 < n_occ; i0 += blk) {
      const int i1 = std::min(n_occ, i0 + blk);
      const int64_t cols = (int64_t)(i1 - i0) * n_virt;
      double *B_blk = nullptr;
      if (get_block(i0, i1, &B_blk) != LTGW_OK) return ctx->status();
      if (mixed) {
        if (naf_metric_tc(ctx, n_aux, cols, B_blk, cols, K, s, 1.0) != LTGW_OK) return ctx->status();
        // the projection's operand rows (i0 - n_fc) n_virt .. + cols, transposed and split
        const int64_t off = (int64_t)(i0 - n_fc) * n_virt * Kpa_aux;
        CHECK_LAUNCH(ctx, launch_to_f32_transposed(B_blk, cols, 0, n_aux, (int)cols, d_Rt, (int)Kpa_aux, (int)cols,
                                                   1, 0, 0, s), 1);
        CHECK_LAUNCH(ctx, launch_split_bf16(d_Rt, d_Rh + off, d_Rl + off, cols * Kpa_aux, s), 1);
      } else if (emu) {
        EmuPlan ep;   // K += B_blk B_blk^T from slices
        if (emu_prepare(ctx, n_aux, n_aux, cols, n_sl, true, 0, &ep, s, true) != LTGW_OK) return ctx->status();
        if (emu_syrk(ctx, ep, B_blk, cols, K, 1.0, s) != LTGW_OK) return ctx->status();
      } else {
        GemmF64Args g;  // K += B_blk B_blk^T
        g.M = n_aux; g.N = n_aux; g.K = cols;
        g.A = B_blk; g.lda = cols; g.B = B_blk; g.ldb = cols;
        g.C = K; g.ldc = n_aux; g.syrk = 1; g.beta = 1.0;
        CHECK_LAUNCH(ctx, launch_gemm_f64(g, 1, true, true, s), 1);
      }
      if (block_done() != LTGW_OK) return ctx->status();
    }
    if (keep_split && n_ov_p > n_ov) {
      LTGW_CUDA(ctx, cudaMemsetAsync(d_Rh + n_ov * Kpa_aux, 0, (size_t)(n_ov_p - n_ov) * Kpa_aux * 2, s));
      LTGW_CUDA(ctx, cudaMemsetAsync(d_Rl + n_ov * Kpa_aux, 0, (size_t)(n_ov_p - n_ov) * Kpa_aux * 2, s));
    }
    return LTGW_OK;
  };

  // ---- NAF (Eqs. nafeq, naftrafo) on a separate arena for its scratch
  int N = n_aux, near = 0;
  if (naf) {
    if (naf_basis_dev(ctx, ctx->a3, n_aux, n_ov, B_act, ld_act, p->naf_thresh, d_Ut, d_lam, &N, &near, s,
                      mixed, streamed ? &build_K : nullptr, emu ? n_sl : 0) != LTGW_OK)
      return ctx->status();
  }
  ctx->stats.n_naf = N;
  ctx->stats.naf_near_threshold = near;
  if (btg_join.join(s) != LTGW_OK) return ctx->status();   // B_tgt is read from here on

  // ---- phase-2 workspace
  double *d_Bt = nullptr, *d_Btt = nullptr, *d_M = nullptr, *d_Pi, *d_X0, *d_X1, *d_C, *d_W, *d_sig, *d_eqp;
  int *d_st;
  float *d_Bf = nullptr, *d_BtT32 = nullptr;
  double *d_BtT64 = nullptr;
  const int64_t Kp_ov = (n_ov + 63) / 64 * 64;
  auto layout2 = [&](Arena &A) {
    d_Bt = (naf && !mixed) ? A.take<double>((size_t)N * n_ov) : nullptr;
    d_Btt = (naf && !mixed) ? A.take<double>((size_t)T * N * n_orb_act) : nullptr;
    if (mixed) {
      d_Bf = A.take<float>((size_t)((N + 127) / 128 * 128) * Kp_ov);
      d_BtT64 = A.take<double>((size_t)T * n_orb_act * N);
      d_BtT32 = A.take<float>((size_t)(((int64_t)T * n_orb_act + 127) / 128 * 128) * ((N + 63) / 64 * 64));
    }
    d_M = n_tau ? A.take<double>((size_t)n_tau * N * N) : nullptr;
    d_Pi = A.take<double>((size_t)n_omega * N * N);
    d_X0 = A.take<double>(screen_blocked_scratch(N, n_omega));
    d_X1 = nullptr;
    d_C = A.take<double>((size_t)n_omega * N * N);
    d_W = A.take<double>((size_t)n_omega * T * n_orb_act);
    d_sig = A.take<double>((size_t)T * n_omega * 2);
    d_eqp = A.take<double>(T);
    d_st = A.take<int>(T);
  };
  ctx->a2.begin_sizing();
  layout2(ctx->a2);
  if (ctx->a2.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "solve workspace allocation failed"); return ctx->status(); }
  layout2(ctx->a2);

  const double *Bt = B_act;
  int64_t ld_bt = ld_act;
  const double *Btt = d_Btg + n_fc;
  int64_t ld_btt = n_orb, stride_btt = (int64_t)n_aux * n_orb;
  if (mixed && streamed) {
    // one projection over every block's kept operand: no second pass of the callback
    if (naf_project_tc(ctx, N, n_aux, d_Ut, nullptr, 0, n_ov, d_Btg, n_orb, n_fc, T, n_orb_act, d_Bf, d_BtT64,
                       d_BtT32, s, nullptr, d_Rh, d_Rl) != LTGW_OK)
      return ctx->status();
  } else if (mixed) {
    if (naf_project_tc(ctx, N, n_aux, naf ? d_Ut : nullptr, B_act, ld_act, n_ov, d_Btg, n_orb, n_fc, T, n_orb_act,
                       d_Bf, d_BtT64, d_BtT32, s) != LTGW_OK)
      return ctx->status();
  } else if (naf) {
    if (streamed) {
      for (int i0 = n_fc; i0 < n_occ; i0 += blk) {
        const int i1 = std::min(n_occ, i0 + blk);
        const int64_t cols = (int64_t)(i1 - i0) * n_virt;
        double *B_blk = nullptr;
        if (get_block(i0, i1, &B_blk) != LTGW_OK) return ctx->status();
        if (emu) {
          if (project_emu(ctx, N, n_aux, d_Ut, B_blk, cols, (int)cols, d_Bt + (int64_t)(i0 - n_fc) * n_virt, n_ov,
                          n_sl, s) != LTGW_OK)
            return ctx->status();
        } else {
          GemmF64Args g;  // R~_ov[:, block] = U^T R_blk
          g.M = N; g.N = (int)cols; g.K = n_aux;
          g.A = d_Ut; g.lda = n_aux;
          g.B = B_blk; g.ldb = cols;
          g.C = d_Bt + (int64_t)(i0 - n_fc) * n_virt; g.ldc = n_ov;
          CHECK_LAUNCH(ctx, launch_gemm_f64(g, 1, true, false, s), 1);
        }
        if (block_done() != LTGW_OK) return ctx->status();
      }
    } else if (emu) {
      REQUIRE(ctx, n_ov <= INT32_MAX, "too many pairs for one emulated projection");
      if (project_emu(ctx, N, n_aux, d_Ut, B_act, ld_act, (int)n_ov, d_Bt, n_ov, n_sl, s) != LTGW_OK)
        return ctx->status();
    } else {
      GemmF64Args g;  // R~_ov = U^T R_ov
      g.M = N; g.N = (int)std::min<int64_t>(n_ov, INT32_MAX); g.K = n_aux;
      g.A = d_Ut; g.lda = n_aux;
      g.B = B_act; g.ldb = ld_act;
      g.C = d_Bt; g.ldc = n_ov;
      CHECK_LAUNCH(ctx, launch_gemm_f64(g, 1, true, false, s), 1);
    }
    if (emu) {
      for (int t = 0; t < T; ++t)   // R~_tgt[t] = U^T R_tgt[t][:, active]
        if (project_emu(ctx, N, n_aux, d_Ut, d_Btg + (int64_t)t * n_aux * n_orb + n_fc, n_orb, n_orb_act,
                        d_Btt + (int64_t)t * N * n_orb_act, n_orb_act, n_sl, s) != LTGW_OK)
          return ctx->status();
    } else {
      GemmF64Args h;  // R~_tgt[t] = U^T R_tgt[t][:, active]
      h.M = N; h.N = n_orb_act; h.K = n_aux;
      h.A = d_Ut; h.lda = n_aux; h.strideA = 0;
      h.B = d_Btg + n_fc; h.ldb = n_orb; h.strideB = (int64_t)n_aux * n_orb;
      h.C = d_Btt; h.ldc = n_orb_act; h.strideC = (int64_t)N * n_orb_act;
      CHECK_LAUNCH(ctx, launch_gemm_f64(h, T, true, false, s), 1);
    }
    Bt = d_Bt; ld_bt = n_ov;
    Btt = d_Btt; ld_btt = n_orb_act; stride_btt = (int64_t)N * n_orb_act;
  }
  ctx->mark(EV_NAF, s);

  // evGW: the quasi-particle energies of the previous cycle (targets) and the
  // scissor shift of the nearest target by orbital index (other active orbitals)
  auto ev_energies = [&](const std::vector<double> &hq) {
    std::vector<double> e = h_eps;
    std::vector<std::pair<int, double>> ts(T);
    for (int t = 0; t < T; ++t) ts[t] = {h_tg[t], hq[t] - h_eps[h_tg[t]]};
    std::sort(ts.begin(), ts.end());
    for (int q = n_fc; q < n_orb; ++q) {
      int best = 0;
      for (int t = 1; t < T; ++t)
        if (abs(ts[t].first - q) < abs(ts[best].first - q)) best = t;   // ties keep the lower target
      e[q] = h_eps[q] + ts[best].second;
    }
    return e;
  };
  int ih = -1, il = -1;
  for (int t = 0; t < T; ++t) {
    if (h_tg[t] == n_occ - 1) ih = t;
    if (h_tg[t] == n_occ) il = t;
  }
  std::vector<double> hq_prev;
  int cycles = 0;
  for (int cyc = 0;; ++cyc) {
    // ---- Pi (Eq. Pi or the Laplace form)
    if (mixed) {
      if (polarizability_tc(ctx, N, n_ov, nullptr, 0, d_Bf, d_delta, n_omega, d_om, n_tau, d_x, d_w, d_E,
                            d_M, p->spin, d_Pi, s, fp8, p->use_laplace) != LTGW_OK)
        return ctx->status();
    } else if (emu) {
      if (polarizability_emu(ctx, N, n_ov, Bt, ld_bt, d_delta, n_omega, d_om, n_tau, d_x, d_w, d_E, d_M, p->spin,
                             d_Pi, s, p->use_laplace, n_sl) != LTGW_OK)
        return ctx->status();
    } else if (polarizability_dev(ctx, N, n_ov, Bt, ld_bt, d_delta, n_omega, d_om, n_tau, d_x, d_w, d_E, d_M,
                                  p->spin, d_Pi, s, p->use_laplace) != LTGW_OK) {
      return ctx->status();
    }
    ctx->mark(EV_PI, s);

    // ---- screening
    int nl = 0;
    cudaError_t e = launch_screen_blocked(d_Pi, N, n_omega, d_X0, d_C, ctx->flags, s, &nl);
    ctx->launches += nl;
    if (e != cudaSuccess) { ctx->fail(LTGW_ERR_DEVICE, std::string("screen: ") + cudaGetErrorString(e)); return ctx->status(); }
    ctx->mark(EV_SCREEN, s);

    // ---- W_nm(i w_j)
    if (mixed) {
      if (wnm_tc(ctx, N, n_omega, d_C, T, n_orb_act, d_BtT64, d_BtT32, d_W, s, fp8_w) != LTGW_OK) return ctx->status();
    } else if (emu) {
      if (wnm_emu(ctx, N, n_omega, d_C, T, n_orb_act, Btt, ld_btt, stride_btt, d_W, n_sl, s) != LTGW_OK)
        return ctx->status();
    } else {
      ColDotArgs cd;
      cd.N = N; cd.ncols = n_orb_act; cd.n_tgt = T;
      cd.C = d_C; cd.ldc = N; cd.strideC = (int64_t)N * N;
      cd.Bt = Btt; cd.ldb = ld_btt; cd.strideBt = stride_btt;
      cd.W = d_W; cd.ldw = n_orb_act;
      CHECK_LAUNCH(ctx, launch_gemm_coldot(cd, n_omega, s), 1);
    }
    ctx->mark(EV_WNM, s);

    // ---- Sigma(i w), Pade, Newton
    SigmaArgs sa;
    sa.n_tgt = T; sa.n_omega = n_omega; sa.n_orb = n_orb_act;
    sa.W = d_W; sa.eps_m = d_eps + n_fc; sa.omega = d_om; sa.weight = d_wt;
    sa.eps_F = eF; sa.sigma = d_sig;
    CHECK_LAUNCH(ctx, launch_sigma(sa, s), 1);
    QpArgs q;
    q.n_tgt = T; q.n_omega = n_omega; q.pade_stride = 2;
    q.sigma = d_sig; q.omega = d_om; q.eps_n = d_epsn; q.shift = d_shift;
    q.eps_F = eF; q.eta = 0.0; q.tol = 1e-12; q.max_iter = 100;
    q.e_qp = d_eqp; q.status = d_st;
    CHECK_LAUNCH(ctx, launch_qp(q, s), 1);
    ctx->mark(EV_SIGQP, s);

    if (cyc == ev_cycles) break;
    // ---- next evGW cycle
    std::vector<double> hq(T);
    if (read_small(ctx, hq.data(), d_eqp, T * sizeof(double), s) != LTGW_OK) return ctx->status();
    if (cyc > 0 && ev_gap_tol > 0.0 && ih >= 0 && il >= 0 &&
        fabs((hq[il] - hq[ih]) - (hq_prev[il] - hq_prev[ih])) < ev_gap_tol)
      break;
    const std::vector<double> e_next = ev_energies(hq);
    REQUIRE(ctx, e_next[n_occ] > e_next[n_occ - 1], "evGW: the quasi-particle HOMO/LUMO gap closed");
    eF = 0.5 * (e_next[n_occ - 1] + e_next[n_occ]);
    copy_in(ctx, d_eps, e_next.data(), n_orb * sizeof(double), s);
    CHECK_LAUNCH(ctx, launch_pair_gaps(d_eps, n_occ, n_virt, n_fc, d_delta, s), 1);
    if (n_tau && !tau_x) {
      if (fit_grid(e_next) != LTGW_OK) return ctx->status();
      copy_in(ctx, d_x, h_x.data(), n_tau * sizeof(double), s);
      copy_in(ctx, d_w, h_w.data(), n_tau * sizeof(double), s);
      copy_in(ctx, d_E, h_E.data(), h_E.size() * sizeof(double), s);
    }
    if (ctx->status() != LTGW_OK) return ctx->status();
    hq_prev = hq;
    ++cycles;
  }
  if (ev_done) *ev_done = cycles;

  // ---- outputs
  LTGW_CUDA(ctx, cudaMemcpyAsync(sigma_iw, d_sig, (size_t)T * n_omega * 2 * sizeof(double), cudaMemcpyDefault, s));
  LTGW_CUDA(ctx, cudaMemcpyAsync(e_qp, d_eqp, (size_t)T * sizeof(double), cudaMemcpyDefault, s));
  LTGW_CUDA(ctx, cudaMemcpyAsync(qp_status, d_st, (size_t)T * sizeof(int), cudaMemcpyDefault, s));
  ctx->mark(EV_END, s);
  LTGW_CUDA(ctx, cudaStreamSynchronize(s));
  if (check_flags(ctx, s) != LTGW_OK) return ctx->status();

  ltgw_stats &st = ctx->stats;
  st.n_pade = (n_omega + 1) / 2;
  st.n_tau = n_tau;
  st.kernel_launches = ctx->launches;
  st.pi_kernel_launches = 1;
  st.ms_naf = ctx->ms(EV_START, EV_NAF);
  st.ms_pi = ctx->ms(EV_NAF, EV_PI);
  st.ms_pi_kernel = ctx->ms(EV_PI0, EV_PI1);
  st.ms_screen = ctx->ms(EV_PI, EV_SCREEN);
  st.ms_wnm = ctx->ms(EV_SCREEN, EV_WNM);
  st.ms_sigma_qp = ctx->ms(EV_WNM, EV_SIGQP);
  st.ms_total = ctx->ms(EV_START, EV_END);
  st.ms_tridiag = naf ? ctx->ms(EV_TRI0, EV_TRI1) : 0.0;
  st.ms_naf_metric = naf ? ctx->ms(EV_K0, EV_TRI0) : 0.0;
  st.ms_eig_vectors = naf ? ctx->ms(EV_TRI1, EV_VEC1) : 0.0;
  st.ms_naf_project = naf ? ctx->ms(EV_VEC1, EV_NAF) : 0.0;

  st.ms_generate = ctx->gen_ms;
  std::vector<int> hs(T);
  if (read_small(ctx, hs.data(), qp_status, T * sizeof(int), s) != LTGW_OK) return ctx->status();
  for (int t = 0; t < T; ++t)
    if (hs[t] != 0) ctx->fail(LTGW_ERR_NO_CONVERGE, "a quasi-particle Newton solve did not converge");
  return ctx->status();
}

ltgw_status polarizability_dev_api(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt, const double *delta,
                                   int n_omega, const double *omegas, int n_tau, const double *x, const double *w,
                                   int spin, double *Pi, void *stream, int lt_form, const double *gamma) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->reset();
  REQUIRE(ctx, N >= 1 && n_pairs >= 1 && n_omega >= 1 && n_omega <= 256, "bad sizes");
  REQUIRE(ctx, n_tau >= 0 && n_tau <= 32, "n_tau must be in [0, 32]");
  REQUIRE(ctx, spin == 1 || spin == 2, "spin must be 1 or 2");
  REQUIRE(ctx, Bt && delta && omegas && Pi && (n_tau == 0 || (x && (lt_form == 2 ? gamma : w) != nullptr)),
          "a required pointer is NULL");
  REQUIRE(ctx, is_device_ptr(Bt) && is_device_ptr(delta) && is_device_ptr(Pi), "Bt, delta, Pi must be device pointers");
  LTGW_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<double> h_om(omegas, omegas + n_omega), h_E((size_t)n_omega * std::max(n_tau, 1));
  for (int j = 0; j < n_omega; ++j)
    for (int k = 0; k < n_tau; ++k)
      h_E[(size_t)j * n_tau + k] = lt_form == 2 ? gamma[(size_t)j * n_tau + k] : exp(-h_om[j] * h_om[j] * x[k]);
  double *d_om, *d_x, *d_w, *d_E, *d_M;
  auto layout = [&](Arena &A) {
    d_om = A.take<double>(n_omega);
    d_x = A.take<double>(std::max(n_tau, 1));
    d_w = A.take<double>(std::max(n_tau, 1));
    d_E = A.take<double>(h_E.size());
    d_M = n_tau ? A.take<double>((size_t)n_tau * N * N) : nullptr;
  };
  ctx->a2.begin_sizing();
  layout(ctx->a2);
  if (ctx->a2.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "workspace allocation failed"); return ctx->status(); }
  layout(ctx->a2);
  copy_in(ctx, d_om, h_om.data(), n_omega * sizeof(double), s);
  if (n_tau) {
    copy_in(ctx, d_x, x, n_tau * sizeof(double), s);
    if (lt_form != 2) copy_in(ctx, d_w, w, n_tau * sizeof(double), s);
    copy_in(ctx, d_E, h_E.data(), h_E.size() * sizeof(double), s);
  }
  if (ctx->status() != LTGW_OK) return ctx->status();
  if (polarizability_dev(ctx, N, n_pairs, Bt, n_pairs, delta, n_omega, d_om, n_tau, d_x, d_w, d_E, d_M,
                         spin, Pi, s, lt_form) != LTGW_OK)
    return ctx->status();
  LTGW_CUDA(ctx, cudaStreamSynchronize(s));  // the staged grid lives in the workspace
  return LTGW_OK;
}

// lt_form 1: x, w are the Laplace grid of Eq. LT; 2: x holds tau_k and gamma
// [n_omega][n_tau] the imaginary-time recombination (w unused).
ltgw_status polarizability_tc_api(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt, const double *delta,
                                  int n_omega, const double *omegas, int n_tau, const double *x, const double *w,
                                  int spin, double *Pi, void *stream, bool fp8, int lt_form = 1,
                                  const double *gamma = nullptr) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->reset();
  REQUIRE(ctx, N >= 1 && n_pairs >= 1 && n_omega >= 1 && n_omega <= 256, "bad sizes");
  REQUIRE(ctx, n_tau >= 0 && n_tau <= 32, "n_tau must be in [0, 32]");
  REQUIRE(ctx, spin == 1 || spin == 2, "spin must be 1 or 2");
  REQUIRE(ctx, Bt && delta && omegas && Pi && (n_tau == 0 || (x && (lt_form == 2 ? gamma : w) != nullptr)),
          "a required pointer is NULL");
  REQUIRE(ctx, is_device_ptr(Bt) && is_device_ptr(delta) && is_device_ptr(Pi), "Bt, delta, Pi must be device pointers");
  LTGW_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<double> h_om(omegas, omegas + n_omega), h_E((size_t)n_omega * std::max(n_tau, 1));
  for (int j = 0; j < n_omega; ++j)
    for (int k = 0; k < n_tau; ++k)
      h_E[(size_t)j * n_tau + k] = lt_form == 2 ? gamma[(size_t)j * n_tau + k] : exp(-h_om[j] * h_om[j] * x[k]);
  double *d_om, *d_x, *d_w, *d_E, *d_M;
  auto layout = [&](Arena &A) {
    d_om = A.take<double>(n_omega);
    d_x = A.take<double>(std::max(n_tau, 1));
    d_w = A.take<double>(std::max(n_tau, 1));
    d_E = A.take<double>(h_E.size());
    d_M = n_tau ? A.take<double>((size_t)n_tau * N * N) : nullptr;
  };
  ctx->a2.begin_sizing();
  layout(ctx->a2);
  if (ctx->a2.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "workspace allocation failed"); return ctx->status(); }
  layout(ctx->a2);
  LTGW_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
  copy_in(ctx, d_om, h_om.data(), n_omega * sizeof(double), s);
  if (n_tau) {
    copy_in(ctx, d_x, x, n_tau * sizeof(double), s);
    if (lt_form != 2) copy_in(ctx, d_w, w, n_tau * sizeof(double), s);
    copy_in(ctx, d_E, h_E.data(), h_E.size() * sizeof(double), s);
  }
  if (ctx->status() != LTGW_OK) return ctx->status();
  if (polarizability_tc(ctx, N, n_pairs, Bt, n_pairs, nullptr, delta, n_omega, d_om, n_tau, d_x, d_w, d_E, d_M,
                        spin, Pi, s, fp8, lt_form) != LTGW_OK)
    return ctx->status();
  LTGW_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->stats.ms_pi_kernel = ctx->ms(EV_PI0, EV_PI1);
  ctx->stats.pi_kernel_launches = 1;
  return check_flags(ctx, s);
}

}  // namespace

extern "C" {

ltgw_status ltgw_solve(ltgw_ctx *ctx, const ltgw_params *p, const double *eps, const double *B_ov,
                       const double *B_tgt, const int *targets, int n_tgt, const double *shift,
                       const double *tau_x, const double *tau_w, double *sigma_iw, double *e_qp,
                       int *qp_status, void *stream) {
  return solve_impl(ctx, p, eps, B_ov, nullptr, nullptr, 0, B_tgt, targets, n_tgt, shift, tau_x, tau_w, sigma_iw,
                    e_qp, qp_status, stream);
}

ltgw_status ltgw_solve_ev(ltgw_ctx *ctx, const ltgw_params *p, const double *eps, const double *B_ov,
                          const double *B_tgt, const int *targets, int n_tgt, const double *shift,
                          const double *tau_x, const double *tau_w, int n_cycles, double gap_tol,
                          double *sigma_iw, double *e_qp, int *qp_status, int *cycles_done, void *stream) {
  return solve_impl(ctx, p, eps, B_ov, nullptr, nullptr, 0, B_tgt, targets, n_tgt, shift, tau_x, tau_w, sigma_iw,
                    e_qp, qp_status, stream, n_cycles, gap_tol, cycles_done);
}

ltgw_status ltgw_solve_streamed(ltgw_ctx *ctx, const ltgw_params *p, const double *eps, ltgw_block_fn fill,
                                void *user, int occ_block, const double *B_tgt, const int *targets, int n_tgt,
                                const double *shift, const double *tau_x, const double *tau_w, double *sigma_iw,
                                double *e_qp, int *qp_status, void *stream) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  if (!fill) {
    ctx->reset();
    ctx->fail(LTGW_ERR_BAD_ARG, "fill callback is NULL");
    return ctx->status();
  }
  return solve_impl(ctx, p, eps, nullptr, fill, user, occ_block, B_tgt, targets, n_tgt, shift, tau_x, tau_w,
                    sigma_iw, e_qp, qp_status, stream);
}

static ltgw_status naf_basis_api(ltgw_ctx *ctx, int n_aux, int64_t n_pairs, const double *B, int64_t ld,
                                 double thresh, double *Ut, double *lambda, int *n_naf, void *stream, bool mixed) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->reset();
  REQUIRE(ctx, n_aux >= 1 && n_pairs >= 1 && ld >= n_pairs, "bad sizes");
  REQUIRE(ctx, B && Ut && lambda && n_naf, "a required pointer is NULL");
  REQUIRE(ctx, is_device_ptr(B) && is_device_ptr(Ut) && is_device_ptr(lambda), "B, Ut, lambda must be device pointers");
  REQUIRE(ctx, isfinite(thresh), "thresh must be finite");
  LTGW_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  LTGW_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
  int k = 0, near = 0;
  if (naf_basis_dev(ctx, ctx->a3, n_aux, n_pairs, B, ld, thresh, Ut, lambda, &k, &near, s, mixed) != LTGW_OK)
    return ctx->status();
  *n_naf = k;
  ctx->stats = ltgw_stats{};
  ctx->stats.n_naf = k;
  ctx->stats.naf_near_threshold = near;
  LTGW_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->stats.ms_naf_metric = ctx->ms(EV_K0, EV_TRI0);
  ctx->stats.ms_tridiag = ctx->ms(EV_TRI0, EV_TRI1);
  ctx->stats.ms_eig_vectors = ctx->ms(EV_TRI1, EV_VEC1);
  ctx->stats.kernel_launches = ctx->launches;
  return check_flags(ctx, s);
}

ltgw_status ltgw_naf_basis(ltgw_ctx *ctx, int n_aux, int64_t n_pairs, const double *B, int64_t ld,
                           double thresh, double *Ut, double *lambda, int *n_naf, void *stream) {
  return naf_basis_api(ctx, n_aux, n_pairs, B, ld, thresh, Ut, lambda, n_naf, stream, false);
}

ltgw_status ltgw_naf_basis_mixed(ltgw_ctx *ctx, int n_aux, int64_t n_pairs, const double *B, int64_t ld,
                                 double thresh, double *Ut, double *lambda, int *n_naf, void *stream) {
  return naf_basis_api(ctx, n_aux, n_pairs, B, ld, thresh, Ut, lambda, n_naf, stream, true);
}

ltgw_status ltgw_polarizability(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                const double *delta, int n_omega, const double *omegas, int n_tau,
                                const double *x, const double *w, int spin, double *Pi, void *stream) {
  return polarizability_dev_api(ctx, N, n_pairs, Bt, delta, n_omega, omegas, n_tau, x, w, spin, Pi, stream, 1,
                                nullptr);
}

ltgw_status ltgw_polarizability_tau(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt, const double *delta,
                                    int n_omega, const double *omegas, int n_tau, const double *tau,
                                    const double *gamma, int spin, int precision, double *Pi, void *stream) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  if (n_tau < 1) { ctx->reset(); ctx->fail(LTGW_ERR_BAD_ARG, "n_tau must be >= 1"); return ctx->status(); }
  if (precision == LTGW_FP64)
    return polarizability_dev_api(ctx, N, n_pairs, Bt, delta, n_omega, omegas, n_tau, tau, nullptr, spin, Pi,
                                  stream, 2, gamma);
  if (precision < LTGW_FP64 || precision > LTGW_FP8_PI) {
    ctx->reset();
    ctx->fail(LTGW_ERR_BAD_ARG, "unknown precision");
    return ctx->status();
  }
  return polarizability_tc_api(ctx, N, n_pairs, Bt, delta, n_omega, omegas, n_tau, tau, nullptr, spin, Pi, stream,
                               precision == LTGW_FP8 || precision == LTGW_FP8_PI, 2, gamma);
}

ltgw_status ltgw_polarizability_mixed(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                      const double *delta, int n_omega, const double *omegas, int n_tau,
                                      const double *x, const double *w, int spin, double *Pi,
                                      void *stream) {
  return polarizability_tc_api(ctx, N, n_pairs, Bt, delta, n_omega, omegas, n_tau, x, w, spin, Pi, stream, false);
}

ltgw_status ltgw_polarizability_fp8(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                    const double *delta, int n_omega, const double *omegas, int n_tau,
                                    const double *x, const double *w, int spin, double *Pi, void *stream) {
  return polarizability_tc_api(ctx, N, n_pairs, Bt, delta, n_omega, omegas, n_tau, x, w, spin, Pi, stream, true);
}

ltgw_status ltgw_gemm_emulated(ltgw_ctx *ctx, int m, int n, int64_t k, const double *A, int64_t lda,
                               const double *B, int64_t ldb, double *C, int64_t ldc, int sym, int n_slices,
                               void *stream) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->reset();
  REQUIRE(ctx, m >= 1 && n >= 1 && k >= 1 && lda >= k && ldb >= k && ldc >= n, "bad sizes");
  REQUIRE(ctx, n_slices >= 2 && n_slices <= 8, "n_slices must be in [2, 8]");
  REQUIRE(ctx, A && C && (sym || B), "a required pointer is NULL");
  REQUIRE(ctx, !sym || (m == n && ldc == n), "sym needs m == n and ldc == n");
  REQUIRE(ctx, m <= 65535, "m must be <= 65535");
  REQUIRE(ctx, is_device_ptr(A) && is_device_ptr(C) && (sym || is_device_ptr(B)), "A, B, C must be device pointers");
  LTGW_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  LTGW_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
  ctx->stats = ltgw_stats{};
  ctx->mark(EV_START, s);
  if (emu_gemm(ctx, m, n, k, A, lda, sym ? A : B, sym ? lda : ldb, C, ldc, sym != 0, n_slices, s) != LTGW_OK)
    return ctx->status();
  ctx->mark(EV_END, s);
  LTGW_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->stats.ms_total = ctx->ms(EV_START, EV_END);
  ctx->stats.kernel_launches = ctx->launches;
  return check_flags(ctx, s);
}

ltgw_status ltgw_polarizability_emulated(ltgw_ctx *ctx, int N, int64_t n_pairs, const double *Bt,
                                         const double *delta, int n_omega, const double *omegas, int n_tau,
                                         const double *x, const double *w, int spin, int n_slices, double *Pi,
                                         void *stream) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->reset();
  REQUIRE(ctx, N >= 1 && n_pairs >= 1 && n_omega >= 1 && n_omega <= 256, "bad sizes");
  REQUIRE(ctx, n_tau >= 0 && n_tau <= 32, "n_tau must be in [0, 32]");
  REQUIRE(ctx, spin == 1 || spin == 2, "spin must be 1 or 2");
  REQUIRE(ctx, n_slices >= 2 && n_slices <= 8, "n_slices must be in [2, 8]");
  REQUIRE(ctx, Bt && delta && omegas && Pi && (n_tau == 0 || (x && w)), "a required pointer is NULL");
  REQUIRE(ctx, is_device_ptr(Bt) && is_device_ptr(delta) && is_device_ptr(Pi), "Bt, delta, Pi must be device pointers");
  LTGW_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  LTGW_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
  ctx->stats = ltgw_stats{};
  ctx->mark(EV_START, s);
  std::vector<double> h_om(omegas, omegas + n_omega), h_E((size_t)n_omega * std::max(n_tau, 1));
  for (int j = 0; j < n_omega; ++j)
    for (int k = 0; k < n_tau; ++k) h_E[(size_t)j * n_tau + k] = exp(-h_om[j] * h_om[j] * x[k]);
  double *d_om, *d_x, *d_w, *d_E, *d_M;
  auto layout = [&](Arena &A) {
    d_om = A.take<double>(n_omega);
    d_x = A.take<double>(std::max(n_tau, 1));
    d_w = A.take<double>(std::max(n_tau, 1));
    d_E = A.take<double>(h_E.size());
    d_M = n_tau ? A.take<double>((size_t)n_tau * N * N) : nullptr;
  };
  ctx->a2.begin_sizing();
  layout(ctx->a2);
  if (ctx->a2.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "workspace allocation failed"); return ctx->status(); }
  layout(ctx->a2);
  copy_in(ctx, d_om, h_om.data(), n_omega * sizeof(double), s);
  if (n_tau) {
    copy_in(ctx, d_x, x, n_tau * sizeof(double), s);
    copy_in(ctx, d_w, w, n_tau * sizeof(double), s);
    copy_in(ctx, d_E, h_E.data(), h_E.size() * sizeof(double), s);
  }
  if (ctx->status() != LTGW_OK) return ctx->status();
  if (polarizability_emu(ctx, N, n_pairs, Bt, n_pairs, delta, n_omega, d_om, n_tau, d_x, d_w, d_E, d_M, spin, Pi, s,
                         1, n_slices) != LTGW_OK)
    return ctx->status();
  ctx->mark(EV_END, s);
  LTGW_CUDA(ctx, cudaStreamSynchronize(s));   // the staged grid lives in the workspace
  ctx->stats.ms_total = ctx->ms(EV_START, EV_END);
  ctx->stats.ms_pi_kernel = ctx->ms(EV_PI0, EV_PI1);
  ctx->stats.kernel_launches = ctx->launches;
  return check_flags(ctx, s);
}

ltgw_status ltgw_screen(ltgw_ctx *ctx, int N, int n_omega, const double *Pi, double *C, void *stream) {
  if (!ctx) return LTGW_ERR_BAD_ARG;
  ctx->reset();
  REQUIRE(ctx, N >= 1 && n_omega >= 1, "bad sizes");
  REQUIRE(ctx, Pi && C && Pi != C, "Pi and C must be distinct non-NULL pointers");
  REQUIRE(ctx, is_device_ptr(Pi) && is_device_ptr(C), "Pi and C must be device pointers");
  LTGW_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  double *X0;
  auto layout = [&](Arena &A) { X0 = A.take<double>(screen_blocked_scratch(N, n_omega)); };
  ctx->a2.begin_sizing();
  layout(ctx->a2);
  if (ctx->a2.commit() != cudaSuccess) { ctx->fail(LTGW_ERR_NOMEM, "workspace allocation failed"); return ctx->status(); }
  layout(ctx->a2);
  LTGW_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
  int nl = 0;
  cudaError_t e = launch_screen_blocked(Pi, N, n_omega, X0, C, ctx->flags, s, &nl);
  if (e != cudaSuccess) { ctx->fail(LTGW_ERR_DEVICE, std::string("screen: ") + cudaGetErrorString(e)); return ctx->status(); }
  LTGW_CUDA(ctx, cudaStreamSynchronize(s));
  return check_flags(ctx, s);
}

}  // extern "C"
