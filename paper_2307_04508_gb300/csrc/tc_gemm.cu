// Tensor-core contractions on sm_103a (tcgen05 + TMEM, operands by TMA):
//
//   D_t[i][j] = sum_k A[i][k] s_t[k] B[j][k],   t = 0..n_t-1
//
// the scaled rank-k products of the LT-GW path (Pi(tau_k) moments, Eq. LT
// and the M^m form; the NAF metric, Eq. nafeq; projections and the W_nm
// contraction, Eqs. naftrafo and ScreenedCoulombOrbital) in the mixed
// precision forms.
//
// Split BF16 (tc_tma_ts_kernel): each operand value x is split into
// x_hi = bf16(x) and x_lo = bf16(x - x_hi), and D accumulates hi*hi + hi*lo +
// lo*hi with FP32 accumulation in tensor memory, drained into FP64 every
// `drain_k` pairs.  The drain length bounds the FP32 accumulation error: each
// MMA adds its products into D with an FP32 rounding that loses about half an
// ulp on average, all in the same direction for sums of one sign, so the
// relative bias grows with the number of MMAs into one accumulator (about
// 1.7e-5 after 2048 pairs of three products).  B arrives pre-split; the scale
// s_t is applied to A by converter warps that write the scaled split of A into
// tensor memory (the per-pair scale is fused into the operand load).
//
// FP8 E4M3 (tc_fp8_kernel): codes of both operands with per-row scales,
// kind::f8f6f4, de-scaled in the epilogue.
//
// Operands are zero-padded to multiples of the tile (rows to 128, K to 64 or
// 128) so the kernels need no bounds checks.  CTA = one 128 x 128 output tile
// for its scales, one K-split range.  Every mbarrier wait is bounded (about two
// seconds of wall time); on expiry the CTA records an error flag and unwinds.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stddef.h>

#include <algorithm>
#include <mutex>

#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ltgw {
namespace {

constexpr int TM = 128, TN = 128, TK = 64;    // tile rows (A), cols (B), K chunk
constexpr int MAXT = 4;                       // scales per CTA at most (TMEM: 4 x 128 columns)
constexpr int CONV_WARPS = 16, EPI_WARPS = 4;
constexpr uint32_t B_BYTES = TN * TK * 2;      // one bf16 tile, 16 KB
constexpr uint32_t B_STAGE = 2 * B_BYTES;      // hi + lo

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b))
               : "memory");
}

// Bounded wait for the phase with the given parity; false on time-out (or, when
// honor_abort, as soon as another role of the CTA has given up).
__device__ __forceinline__ uint32_t mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return done;
}

// Bounded wait for the phase with the given parity; false on time-out (or, when
// honor_abort, as soon as another role of the CTA has given up).  A phase that
// has already completed costs one try_wait: the MMA issue thread waits once per
// stage, and anything it executes between MMAs leaves the tensor pipe idle.
__device__ __forceinline__ bool mbar_wait_slow(uint64_t *b, uint32_t parity, int *abort, int *err, bool honor_abort) {
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 1023) == 0) {
      if (honor_abort && *(volatile int *)abort) return false;
      if (globaltimer() - t0 > 2000000000ull) {
        atomicExch(&err[FLAG_TC_TIMEOUT], 1);
        *(volatile int *)abort = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int *abort, int *err,
                                          bool honor_abort = true) {
  if (mbar_try(b, parity)) return true;
  return mbar_wait_slow(b, parity, abort, err, honor_abort);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);        // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused, swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// kind::f16, D = FP32, A = B = BF16, both K-major, M = 128, N = 64.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);


__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}


// Epilogue (EPI_WARPS warps): tcgen05.ld of the accumulators after each drain
// window (set dr % nbuf), into FP64 / FP32 partial tiles or the column-dot reduction.
__device__ __forceinline__ void epilogue_drain(const TcGemmArgs &g, uint32_t tmem, uint64_t *acc_full, uint64_t *acc_empty,
                               int *abort, int ndrains, int nt, int nbuf, int tile, int grp, int split, int ti,
                               int tj, float (*cd_red)[TN], int n_tiles, int n_groups) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ew = warp & 3;                   // TMEM lane quarter this warp may read
  const int row = ew * 32 + lane;
  const int64_t tile_elems = (int64_t)TM * TN;
  const int64_t base = (((int64_t)split * n_groups + grp) * g.nt_group * n_tiles + tile) * tile_elems;
  const int64_t tstride = (int64_t)n_tiles * tile_elems;   // between scales
  for (int dr = 0; dr < ndrains; ++dr) {
    const int buf = dr % nbuf;
    if (!mbar_wait(&acc_full[buf], (dr / nbuf) & 1, abort, g.err)) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    for (int t = 0; t < nt; ++t) {
      for (int h = 0; h < TN / 32; ++h) {
        uint32_t r[32];
        const uint32_t a = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)((buf * nt + t) * TN + h * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
              "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
              "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
              "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(a));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (g.ds_a) {   // FP8 form: per-row de-scales of both operands
          const float ra = g.ds_a[(int64_t)(grp * g.nt_group + t) * g.rows_a + ti * TM + row];
          const float *cb = g.ds_b + tj * TN + h * 32;
#pragma unroll
          for (int q = 0; q < 32; ++q) r[q] = __float_as_uint(__uint_as_float(r[q]) * (ra * __ldg(cb + q)));
        }
        if (g.out_colmajor && g.out_mode != TC_OUT_COLDOT) {
          // [col][row]: for each column the warp's 32 rows are one contiguous store
          const int64_t o = base + t * tstride + (int64_t)(h * 32) * TM + row;
          if (g.out_mode == TC_OUT_F32) {
#pragma unroll
            for (int q = 0; q < 32; ++q) g.partial32[o + (int64_t)q * TM] = __uint_as_float(r[q]);
          } else if (dr == 0) {
#pragma unroll
            for (int q = 0; q < 32; ++q) g.partial[o + (int64_t)q * TM] = (double)__uint_as_float(r[q]);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q) g.partial[o + (int64_t)q * TM] += (double)__uint_as_float(r[q]);
          }
        } else if (g.out_mode == TC_OUT_F64) {
          double *oh = g.partial + base + t * tstride + (int64_t)row * TN + h * 32;
          if (dr == 0) {
#pragma unroll
            for (int q = 0; q < 32; q += 2)
              *reinterpret_cast<double2 *>(oh + q) =
                  make_double2((double)__uint_as_float(r[q]), (double)__uint_as_float(r[q + 1]));
          } else {
#pragma unroll
            for (int q = 0; q < 32; q += 2) {
              double2 v = *reinterpret_cast<double2 *>(oh + q);
              v.x += (double)__uint_as_float(r[q]);
              v.y += (double)__uint_as_float(r[q + 1]);
              *reinterpret_cast<double2 *>(oh + q) = v;
            }
          }
        } else if (g.out_mode == TC_OUT_F32) {
          float *oh = g.partial32 + base + t * tstride + (int64_t)row * TN + h * 32;
#pragma unroll
          for (int q = 0; q < 32; q += 4)
            *reinterpret_cast<uint4 *>(oh + q) = make_uint4(r[q], r[q + 1], r[q + 2], r[q + 3]);
        } else {
          // column dot: D[row][col] * cd_B[col][row], summed over the 128 rows
          const int grow = ti * TM + row;
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int col = tj * TN + h * 32 + q;
            float prod = 0.0f;
            if (grow < g.cd_rows && col < g.cd_cols)
              prod = __uint_as_float(r[q]) * (float)g.cd_B[(int64_t)col * g.cd_ld + grow];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) prod += __shfl_xor_sync(0xffffffffu, prod, o);
            if (lane == 0) cd_red[ew][h * 32 + q] = prod;
          }
        }
      }
    }
    if (g.out_mode == TC_OUT_COLDOT) {
      asm volatile("bar.sync 2, %0;" ::"n"(32 * EPI_WARPS) : "memory");   // epilogue warps only
      if (row < TN) {
        const float v = cd_red[0][row] + cd_red[1][row] + cd_red[2][row] + cd_red[3][row];
        g.cd_out[(((int64_t)split * n_groups + grp) * g.n_tile_rows + ti) * g.cd_cols_p + tj * TN + row] = v;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    mbar_arrive(&acc_empty[buf]);
  }
}

// ---- split BF16 with A in tensor memory, operands brought in by TMA ----
// B arrives pre-split (BF16 hi and lo arrays, row-major [rows][Kp]) as two
// tiled TMA copies per chunk with the 128-byte swizzle the tensor core reads,
// so no thread touches it.  A arrives as an FP32 tile (two 128B-swizzled
// boxes of 32 k, so a warp reading 32 consecutive rows at one k offset is
// free of bank conflicts) plus the chunk's scale rows in a staging ring.  The
// converter warps scale and split A and write hi / lo straight into tensor
// memory (tcgen05.st), and the MMA takes A from there: shared memory carries
// only the TMA copies, the staging reads and the B operand reads of the
// tensor core.  TMEM columns: nt accumulators of 128, then a ring of A
// stages of 64 columns (hi: 32 columns of packed k pairs, lo: 32).
// Warp roles (23 warps): 0 TMEM allocation and MMA issue for scale 0, 1 TMA
// producer, 2-17 converters (lane quarter warp % 4, k slice (warp - 2) / 4 of
// 16 values), 18-21 epilogue, 22 MMA issue for scale 1.  One issuing thread
// per accumulator: a thread's MMAs reach the tensor pipe at full rate only when
// they are issued back to back, so each stage's twelve MMAs form one
// instruction block and the per-stage waits of the two issuers overlap.  Each
// A stage belongs to one issuer (the stage count is a multiple of the scales
// per CTA), so an issuer never waits on a phase more than one ahead of its
// stage's barrier, where the parity test would alias.
constexpr int T3_SF = 3, T3_SB = 3;
constexpr int T3_MAXT = 2;                                // scales per CTA
constexpr int T3_MAXSA = (512 - 128) / (TK);              // A stages when nt = 1
constexpr int T3_ISSUE1 = 2 + CONV_WARPS + EPI_WARPS;     // issuer warp of scale 1
constexpr int T3_THREADS = 32 * (T3_ISSUE1 + T3_MAXT - 1);
static_assert(((512 - 128 * 1) / TK) % 1 == 0 && ((512 - 128 * 2) / TK) % 2 == 0,
              "every A stage must belong to one issuer");
constexpr uint32_t F_BYTES = TM * TK * 4;                 // FP32 A tile, 32 KB
constexpr uint32_t F_BOX = TM * 32 * 4;                   // one 32-k box, 16 KB
constexpr uint32_t F_STAGE = F_BYTES + 1024;              // + the chunk's scale rows (nt x 256 B)
constexpr uint32_t T3_SMEM = T3_SF * F_STAGE + T3_SB * B_STAGE + 1024;
static_assert(F_STAGE % 1024 == 0, "stages must stay 1024-byte aligned for the 128-byte swizzle");
static_assert(T3_MAXT * TK * 4 <= 1024, "scale rows must fit the staging slot");
static_assert(TK == 64, "the stage MMA block covers four K = 16 steps and A_lo 32 columns after A_hi");

struct Bars3 {
  uint64_t f_full[T3_SF], f_empty[T3_SF], b_full[T3_SB], b_empty[T3_SB];
  uint64_t a_full[T3_MAXSA], a_empty[T3_MAXSA];
  uint64_t acc_full[1], acc_empty[1], fin;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// A operand in tensor memory: M = 128 rows on the 128 lanes, k pairs packed
// per 32-bit column.  One stage of one scale: D += A_hi B_hi + A_hi B_lo + A_lo B_hi over the 64 k
// of a chunk as four K = 16 steps.  a: TMEM column of A_hi (A_lo 32 columns
// on); bh / bl: descriptors of B_hi / B_lo (a 32-byte k step adds 2 to the
// start-address field).  acc0 = 0 overwrites D with the first product.
__device__ __forceinline__ void mma_stage_ts(uint32_t d, uint32_t a, uint64_t bh, uint64_t bl, uint32_t acc0) {
  asm volatile(
      "{\n.reg .pred p;\n.reg .b32 a1, a2, a3, l0, l1, l2, l3;\n.reg .b64 h1, h2, h3, m1, m2, m3;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "add.u32 a1, %1, 8;\nadd.u32 a2, %1, 16;\nadd.u32 a3, %1, 24;\n"
      "add.u32 l0, %1, 32;\nadd.u32 l1, %1, 40;\nadd.u32 l2, %1, 48;\nadd.u32 l3, %1, 56;\n"
      "add.u64 h1, %2, 2;\nadd.u64 h2, %2, 4;\nadd.u64 h3, %2, 6;\n"
      "add.u64 m1, %3, 2;\nadd.u64 m2, %3, 4;\nadd.u64 m3, %3, 6;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %5, p;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %3, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [l0], %2, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], h1, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], m1, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [l1], h1, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], h2, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], m2, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [l2], h2, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], h3, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], m3, %5, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [l3], h3, %5, 1;\n"
      "}\n" ::"r"(d),
      "r"(a), "l"(bh), "l"(bl), "r"(acc0), "r"(IDESC)
      : "memory");
}

// The same stage with one product per step, D += A_hi B_hi (operands exact in BF16).
__device__ __forceinline__ void mma_stage_single(uint32_t d, uint32_t a, uint64_t bh, uint32_t acc0) {
  asm volatile(
      "{\n.reg .pred p;\n.reg .b32 a1, a2, a3;\n.reg .b64 h1, h2, h3;\n"
      "setp.ne.b32 p, %3, 0;\n"
      "add.u32 a1, %1, 8;\nadd.u32 a2, %1, 16;\nadd.u32 a3, %1, 24;\n"
      "add.u64 h1, %2, 2;\nadd.u64 h2, %2, 4;\nadd.u64 h3, %2, 6;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %4, p;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], h1, %4, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], h2, %4, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], h3, %4, 1;\n"
      "}\n" ::"r"(d),
      "r"(a), "l"(bh), "r"(acc0), "r"(IDESC)
      : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t v[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

__global__ void __launch_bounds__(T3_THREADS, 1)
    tc_tma_ts_kernel(TcGemmArgs g, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                     const __grid_constant__ CUtensorMap tmBlo) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sF = smem;                                 // T3_SF staging slots: FP32 A tile + scales
  uint8_t *sB = sF + T3_SF * F_STAGE;                 // T3_SB stages of [hi | lo]
  __shared__ __align__(16) Bars3 bars;
  __shared__ float cd_red[EPI_WARPS][TN];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grid (groups, tiles, splits) for many tiles: the groups of one tile, which
  // read the same A and B panels, are adjacent in launch order and resident
  // together; else (tiles, groups, splits)
  const bool gfirst = g.groups_fastest != 0;
  const int grp = gfirst ? blockIdx.x : blockIdx.y, tile = gfirst ? blockIdx.y : blockIdx.x, split = blockIdx.z;
  const int n_groups = gfirst ? gridDim.x : gridDim.y, n_tiles = gfirst ? gridDim.y : gridDim.x;
  const int ti = g.tiles[2 * tile], tj = g.tiles[2 * tile + 1];
  const int t0 = grp * g.nt_group;
  const int nt = min(g.nt_group, g.n_t - t0);
  const int nsa = (512 - TN * g.nt_group) / TK;       // A stages in TMEM after the accumulators
  const uint32_t acol0 = (uint32_t)(TN * g.nt_group); // first A column
  const int64_t kb = g.k_begin + (int64_t)split * g.k_per_split;
  const int64_t ke = min(g.k_end ? g.k_end : g.Kp, kb + g.k_per_split);
  const int nchunks = (int)((ke - kb) / TK);
  const int chunks_per_drain = (int)(g.drain_k / TK);
  const int ndrains = (nchunks + chunks_per_drain - 1) / chunks_per_drain;

  if (threadIdx.x == 0) {
    // b_empty, acc_full and fin collect one commit from each of the nt issuers
    for (int s = 0; s < T3_SF; ++s) { mbar_init(&bars.f_full[s], 1); mbar_init(&bars.f_empty[s], CONV_WARPS); }
    for (int s = 0; s < T3_SB; ++s) { mbar_init(&bars.b_full[s], 1); mbar_init(&bars.b_empty[s], nt); }
    for (int s = 0; s < T3_MAXSA; ++s) { mbar_init(&bars.a_full[s], CONV_WARPS); mbar_init(&bars.a_empty[s], 1); }
    mbar_init(&bars.acc_full[0], nt);
    mbar_init(&bars.acc_empty[0], 32 * EPI_WARPS);
    mbar_init(&bars.fin, nt);
    bars.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(&bars.tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = bars.tmem_base;

  const int issue_t = warp == 0 ? 0 : (warp >= T3_ISSUE1 ? warp - T3_ISSUE1 + 1 : -1);
  if (issue_t >= 0) {
    // ---------------------------------------------------------------- MMA issue, scale issue_t
    // Stages of A come in the order (chunk, scale): this scale's stage of
    // chunk c is (c nt + issue_t) mod nsa.
    if (lane == 0 && issue_t < nt) {
      const uint64_t db0 = make_desc(smem_u32(sB));
      const uint32_t d = tmem + (uint32_t)(issue_t * TN);
      int ia = issue_t, ib = 0;
      uint32_t pa = 0, pb = 0;
      while (ia >= nsa) { ia -= nsa; pa ^= 1; }
      bool ok = true;
      for (int dr = 0; dr < ndrains && ok; ++dr) {
        ok = mbar_wait(&bars.acc_empty[0], (dr & 1) ^ 1, &bars.abort, g.err);
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int c_end = min(nchunks, (dr + 1) * chunks_per_drain);
        for (int c = dr * chunks_per_drain; c < c_end && ok; ++c) {
          ok = mbar_wait(&bars.b_full[ib], pb, &bars.abort, g.err) && mbar_wait(&bars.a_full[ia], pa, &bars.abort, g.err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t bh = db0 + (uint64_t)((ib * B_STAGE) >> 4);
          if (g.single)
            mma_stage_single(d, tmem + acol0 + (uint32_t)(ia * TK), bh, c == dr * chunks_per_drain ? 0u : 1u);
          else
            mma_stage_ts(d, tmem + acol0 + (uint32_t)(ia * TK), bh, bh + (B_BYTES >> 4),
                         c == dr * chunks_per_drain ? 0u : 1u);
          mma_commit(&bars.a_empty[ia]);
          mma_commit(&bars.b_empty[ib]);
          for (ia += nt; ia >= nsa;) { ia -= nsa; pa ^= 1; }
          if (++ib == T3_SB) { ib = 0; pb ^= 1; }
        }
        if (ok) mma_commit(&bars.acc_full[0]);
      }
      // all issued MMAs complete before the CTA tears down
      mma_commit(&bars.fin);
      mbar_wait(&bars.fin, 0, &bars.abort, g.err, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      // stacked A groups (a_group_stride = rows_a Kp): group grp's rows follow grp * rows_a
      const int arow0 = (g.a_group_stride ? grp * (int)g.rows_a : 0) + ti * TM;
      int jf = 0, jb = 0;
      uint32_t pf = 0, pb = 0;
      for (int c = 0; c < nchunks; ++c) {
        const int k0 = (int)(kb + (int64_t)c * TK);   // multiple of 64: x stays 16-byte aligned for both types
        if (!mbar_wait(&bars.f_empty[jf], pf ^ 1, &bars.abort, g.err)) break;
        uint8_t *slot = sF + jf * F_STAGE;
        mbar_expect_tx(&bars.f_full[jf], F_BYTES + (uint32_t)nt * TK * 4);
        tma_load_2d(slot, &tmA, k0, arow0, &bars.f_full[jf]);
        tma_load_2d(slot + F_BOX, &tmA, k0 + 32, arow0, &bars.f_full[jf]);
        for (int t = 0; t < nt; ++t)
          bulk_load(slot + F_BYTES + t * TK * 4, g.scale + (int64_t)(t0 + t) * g.Kp + k0, TK * 4, &bars.f_full[jf]);
        if (++jf == T3_SF) { jf = 0; pf ^= 1; }
        if (!mbar_wait(&bars.b_empty[jb], pb ^ 1, &bars.abort, g.err)) break;
        uint8_t *bs = sB + jb * B_STAGE;
        mbar_expect_tx(&bars.b_full[jb], g.single ? B_BYTES : B_STAGE);
        tma_load_2d(bs, &tmBhi, k0, tj * TN, &bars.b_full[jb]);
        if (!g.single) tma_load_2d(bs + B_BYTES, &tmBlo, k0, tj * TN, &bars.b_full[jb]);
        if (++jb == T3_SB) { jb = 0; pb ^= 1; }
      }
    }
    __syncwarp();
  } else if (warp < 2 + CONV_WARPS) {
    // ---------------------------------------------------------------- converters
    // Thread = tile row r (its TMEM lane) x 16 k values of the chunk: 4 reads
    // of 16 bytes from the swizzled staging box, then per scale 16 products,
    // their hi / lo split and two 8-column TMEM stores.
    const int wq = warp & 3;
    const int sub = (warp - 2) >> 2;
    const int r = wq * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(wq * 32) << 16;
    const uint32_t roff = (uint32_t)(sub >> 1) * F_BOX + (uint32_t)r * 128;
    const int c0 = (sub & 1) * 4;
    int jf = 0, ia = 0;
    uint32_t pf = 0, pa = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      if (!mbar_wait(&bars.f_full[jf], pf, &bars.abort, g.err)) break;
      const uint8_t *slot = sF + jf * F_STAGE;
      float a[16];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 x = *reinterpret_cast<const float4 *>(slot + roff + (((c0 + j) ^ (r & 7)) << 4));
        a[4 * j] = x.x; a[4 * j + 1] = x.y; a[4 * j + 2] = x.z; a[4 * j + 3] = x.w;
      }
      for (int t = 0; t < nt && ok; ++t) {
        const float4 *ps = reinterpret_cast<const float4 *>(slot + F_BYTES + t * TK * 4 + sub * 64);
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 s4 = ps[j];   // the same address in every lane: one broadcast
          const float v0 = a[4 * j] * s4.x, v1 = a[4 * j + 1] * s4.y, v2 = a[4 * j + 2] * s4.z,
                      v3 = a[4 * j + 3] * s4.w;
          __nv_bfloat162 h0 = __floats2bfloat162_rn(v0, v1), h1 = __floats2bfloat162_rn(v2, v3);
          const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
          __nv_bfloat162 l0 = __floats2bfloat162_rn(v0 - f0.x, v1 - f0.y), l1 = __floats2bfloat162_rn(v2 - f1.x, v3 - f1.y);
          hi[2 * j] = *reinterpret_cast<uint32_t *>(&h0);
          hi[2 * j + 1] = *reinterpret_cast<uint32_t *>(&h1);
          lo[2 * j] = *reinterpret_cast<uint32_t *>(&l0);
          lo[2 * j + 1] = *reinterpret_cast<uint32_t *>(&l1);
        }
        if (!mbar_wait(&bars.a_empty[ia], pa ^ 1, &bars.abort, g.err)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ta = tmem + lane_addr + acol0 + (uint32_t)(ia * TK + sub * 8);
        tmem_st8(ta, hi);
        if (!g.single) tmem_st8(ta + TK / 2, lo);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars.a_full[ia]);
        if (++ia == nsa) { ia = 0; pa ^= 1; }
      }
      // the slot is refilled by TMA (the async proxy): order these reads before it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.f_empty[jf]);
      if (++jf == T3_SF) { jf = 0; pf ^= 1; }
    }
  } else {
    epilogue_drain(g, tmem, bars.acc_full, bars.acc_empty, &bars.abort, ndrains, nt, 1, tile, grp, split, ti, tj,
                   cd_red, n_tiles, n_groups);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ---- FP8 E4M3 form: both operands quantised per row, brought in by TMA ----
// D_t = qa_t qb^T on tcgen05 kind::f8f6f4 (E4M3 x E4M3, FP32 accumulation),
// K = 32 per MMA; the per-row de-scales of both operands are applied in the
// epilogue.  A chunk is 128 pairs (one 128-byte swizzled row per tile row); a
// stage holds the A tiles of the CTA's nt_group scales and the B tile, and as
// many stages as fit (2 with four scales, 4 with two, up to 4) keep the
// loads of later chunks in flight behind the MMAs.  Warp roles
// (9 warps): 0 TMEM allocation and MMA issue for scale 0, 1 TMA producer,
// 2-5 epilogue, 6-8 MMA issue for scales 1-3 (one issuing thread per
// accumulator, each stage's four MMAs back to back).
constexpr int F8_K = 128;
constexpr int F8_MAXSTAGES = 4;
constexpr int F8_MAXT = 4;
constexpr uint32_t F8_TILE = TM * F8_K;                      // 16 KB
constexpr uint32_t F8_RING = 12 * F8_TILE;                   // 192 KB of stages
constexpr int F8_ISSUE1 = 2 + EPI_WARPS;                     // issuer warp of scale 1
constexpr int F8_THREADS = 32 * (F8_ISSUE1 + F8_MAXT - 1);
constexpr uint32_t F8_SMEM = F8_RING + 1024;
// stages of (nt + 1) tiles that fit the ring
__host__ __device__ constexpr int f8_stages(int nt) {
  return (int)(F8_RING / ((uint32_t)(nt + 1) * F8_TILE)) < F8_MAXSTAGES ? (int)(F8_RING / ((uint32_t)(nt + 1) * F8_TILE))
                                                                       : F8_MAXSTAGES;
}
static_assert(f8_stages(F8_MAXT) >= 2, "two stages of four scales must fit");
// kind::f8f6f4: D = FP32 (bit 4), A = B = E4M3 (format code 0), both K-major, N = 128, M = 128
constexpr uint32_t IDESC8 = (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
static_assert(F8_TILE % 1024 == 0, "swizzled tiles must stay 1024-byte aligned");

struct Bars8 {
  uint64_t full[F8_MAXSTAGES], empty[F8_MAXSTAGES], acc_full[1], acc_empty[1], fin;
  uint32_t tmem_base;
  int abort;
};

// D += A B^T over one 128-pair chunk: four K = 32 steps (32 bytes: +2 in the
// descriptors' start-address field).  acc0 = 0 overwrites D first.
__device__ __forceinline__ void mma_stage_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t acc0) {
  asm volatile(
      "{\n.reg .pred p;\n.reg .b64 a1, a2, a3, b1, b2, b3;\n"
      "setp.ne.b32 p, %3, 0;\n"
      "add.u64 a1, %1, 2;\nadd.u64 a2, %1, 4;\nadd.u64 a3, %1, 6;\n"
      "add.u64 b1, %2, 2;\nadd.u64 b2, %2, 4;\nadd.u64 b3, %2, 6;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %4, p;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], a1, b1, %4, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], a2, b2, %4, 1;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], a3, b3, %4, 1;\n"
      "}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(acc0), "r"(IDESC8)
      : "memory");
}

__global__ void __launch_bounds__(F8_THREADS, 1)
    tc_fp8_kernel(TcGemmArgs g, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sS = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(16) Bars8 bars;
  __shared__ float cd_red[EPI_WARPS][TN];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, grp = blockIdx.y, split = blockIdx.z;
  const int ti = g.tiles[2 * tile], tj = g.tiles[2 * tile + 1];
  const int t0 = grp * g.nt_group;
  const int nt = min(g.nt_group, g.n_t - t0);
  const int64_t kb = g.k_begin + (int64_t)split * g.k_per_split;
  const int64_t ke = min(g.k_end ? g.k_end : g.Kp, kb + g.k_per_split);
  const int nchunks = (int)((ke - kb) / F8_K);
  const int chunks_per_drain = (int)(g.drain_k / F8_K);
  const int ndrains = (nchunks + chunks_per_drain - 1) / chunks_per_drain;
  const int nst = f8_stages(g.nt_group);                              // stages in the ring
  const uint32_t stage_bytes = (uint32_t)(g.nt_group + 1) * F8_TILE;  // A tiles, then B

  if (threadIdx.x == 0) {
    // empty, acc_full and fin collect one commit from each of the nt issuers
    for (int s = 0; s < F8_MAXSTAGES; ++s) { mbar_init(&bars.full[s], 1); mbar_init(&bars.empty[s], nt); }
    mbar_init(&bars.acc_full[0], nt);
    mbar_init(&bars.acc_empty[0], 32 * EPI_WARPS);
    mbar_init(&bars.fin, nt);
    bars.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(&bars.tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = bars.tmem_base;

  const int issue_t = warp == 0 ? 0 : (warp >= F8_ISSUE1 ? warp - F8_ISSUE1 + 1 : -1);
  if (issue_t >= 0) {
    // ---------------------------------------------------------------- MMA issue, scale issue_t
    if (lane == 0 && issue_t < nt) {
      const uint64_t db0 = make_desc(smem_u32(sS));
      const uint32_t d = tmem + (uint32_t)(issue_t * TN);
      int js = 0;
      uint32_t ps = 0;
      bool ok = true;
      for (int dr = 0; dr < ndrains && ok; ++dr) {
        ok = mbar_wait(&bars.acc_empty[0], (dr & 1) ^ 1, &bars.abort, g.err);
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int c_end = min(nchunks, (dr + 1) * chunks_per_drain);
        for (int c = dr * chunks_per_drain; c < c_end && ok; ++c) {
          ok = mbar_wait(&bars.full[js], ps, &bars.abort, g.err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t st = (uint32_t)js * stage_bytes;
          mma_stage_f8(d, db0 + ((st + (uint32_t)issue_t * F8_TILE) >> 4),
                       db0 + ((st + (uint32_t)g.nt_group * F8_TILE) >> 4), c == dr * chunks_per_drain ? 0u : 1u);
          mma_commit(&bars.empty[js]);
          if (++js == nst) { js = 0; ps ^= 1; }
        }
        if (ok) mma_commit(&bars.acc_full[0]);
      }
      // all issued MMAs complete before the CTA tears down
      mma_commit(&bars.fin);
      mbar_wait(&bars.fin, 0, &bars.abort, g.err, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int js = 0;
      uint32_t ps = 0;
      for (int c = 0; c < nchunks; ++c) {
        const int k0 = (int)(kb + (int64_t)c * F8_K);   // multiple of 128 bytes
        if (!mbar_wait(&bars.empty[js], ps ^ 1, &bars.abort, g.err)) break;
        uint8_t *st = sS + js * stage_bytes;
        mbar_expect_tx(&bars.full[js], (uint32_t)(nt + 1) * F8_TILE);
        for (int t = 0; t < nt; ++t)
          tma_load_2d(st + t * F8_TILE, &tmA, k0, (int)((t0 + t) * g.rows_a + ti * TM), &bars.full[js]);
        tma_load_2d(st + g.nt_group * F8_TILE, &tmB, k0, tj * TN, &bars.full[js]);
        if (++js == nst) { js = 0; ps ^= 1; }
      }
    }
    __syncwarp();
  } else {
    epilogue_drain(g, tmem, bars.acc_full, bars.acc_empty, &bars.abort, ndrains, nt, 1, tile, grp, split, ti, tj,
                   cd_red, (int)gridDim.x, (int)gridDim.y);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
using TmapEncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TmapEncodeFn tmap_encoder() {
  static TmapEncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmapEncodeFn>(p);
    cudaGetLastError();
  });
  return fn;
}

// 2-D row-major [rows][cols] map with a [box_rows][box_cols] box.
bool encode_2d(CUtensorMap *m, CUtensorMapDataType dt, size_t esize, const void *base, int64_t cols, int64_t rows,
               uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle sw) {
  const TmapEncodeFn f = tmap_encoder();
  if (!f || ((uintptr_t)base & 15) || (cols * (int64_t)esize) % 16) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(cols * (int64_t)esize)};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estride[2] = {1, 1};
  return f(m, dt, 2, const_cast<void *>(base), dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t tc_gemm_smem_bytes() { return std::max<size_t>(T3_SMEM, F8_SMEM); }

cudaError_t launch_tc_fp8_gemm(const TcGemmArgs &g, int n_tiles, cudaStream_t s) {
  if (n_tiles <= 0 || g.n_t <= 0) return cudaSuccess;
  if (!g.A8 || !g.B8 || !g.ds_a || !g.ds_b || g.Kp % F8_K || g.k_per_split % F8_K || g.drain_k % F8_K ||
      g.k_per_split <= 0 || g.drain_k <= 0 || g.nt_group < 1 || g.nt_group > F8_MAXT ||
      (g.out_mode == TC_OUT_COLDOT ? (g.nt_group != 1 || g.k_per_split > g.drain_k) : !g.out_colmajor) ||
      (g.out_mode == TC_OUT_F32 && g.k_per_split > g.drain_k) || g.rows_a < TM || g.rows_b < TN ||
      g.rows_a % TM || g.rows_b % TN || (int64_t)g.n_t * g.rows_a > INT32_MAX)
    return cudaErrorInvalidValue;
  const int groups = (g.n_t + g.nt_group - 1) / g.nt_group;
  const int64_t k_len = (g.k_end ? g.k_end : g.Kp) - g.k_begin;
  if (g.k_begin < 0 || g.k_begin % F8_K || k_len <= 0 || g.k_begin + k_len > g.Kp) return cudaErrorInvalidValue;
  const int splits = (int)((k_len + g.k_per_split - 1) / g.k_per_split);
  CUtensorMap ta, tb;
  if (!encode_2d(&ta, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, g.A8, g.Kp, (int64_t)g.n_t * g.rows_a, F8_K, TM,
                 CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_2d(&tb, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, g.B8, g.Kp, g.rows_b, F8_K, TN, CU_TENSOR_MAP_SWIZZLE_128B))
    return cudaErrorNotSupported;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(tc_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F8_SMEM);
  });
  if (attr_err != cudaSuccess) return attr_err;
  tc_fp8_kernel<<<dim3(n_tiles, groups, splits), F8_THREADS, F8_SMEM, s>>>(g, ta, tb);
  return cudaGetLastError();
}

cudaError_t launch_tc_split_gemm(const TcGemmArgs &g, int n_tiles, cudaStream_t s) {
  if (n_tiles <= 0 || g.n_t <= 0) return cudaSuccess;
  if (g.Kp % TK || g.k_per_split % TK || g.drain_k % TK || g.k_per_split <= 0 || g.drain_k <= 0)
    return cudaErrorInvalidValue;
  if (g.nt_group < 1 || g.nt_group > MAXT) return cudaErrorInvalidValue;
  if (g.out_mode == TC_OUT_F32 && g.k_per_split > g.drain_k) return cudaErrorInvalidValue;
  if (g.out_mode == TC_OUT_COLDOT && (g.nt_group != 1 || g.k_per_split > g.drain_k)) return cudaErrorInvalidValue;
  const int groups = (g.n_t + g.nt_group - 1) / g.nt_group;
  const int64_t k_len = (g.k_end ? g.k_end : g.Kp) - g.k_begin;
  if (g.k_begin < 0 || g.k_begin % TK || k_len <= 0 || g.k_begin + k_len > g.Kp) return cudaErrorInvalidValue;
  const int splits = (int)((k_len + g.k_per_split - 1) / g.k_per_split);
  if (!g.B_hi || (!g.B_lo && !g.single)) return cudaErrorInvalidValue;   // the kernel takes B pre-split
  {
    if ((g.a_group_stride != 0 && g.a_group_stride != g.rows_a * g.Kp) ||
        (g.a_group_stride != 0 && g.nt_group != 1) || g.nt_group > T3_MAXT || g.rows_a < TM || g.rows_b < TN ||
        g.rows_a % TM || g.rows_b % TN)
      return cudaErrorInvalidValue;
    CUtensorMap ta, tbh, tbl;
    const int64_t a_rows = g.a_group_stride ? (int64_t)groups * g.rows_a : g.rows_a;   // stacked groups
    if (!encode_2d(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g.A, g.Kp, a_rows, 32, TM,
                   CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_2d(&tbh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.B_hi, g.Kp, g.rows_b, TK, TN,
                   CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_2d(&tbl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.single ? g.B_hi : g.B_lo, g.Kp, g.rows_b, TK, TN,
                   CU_TENSOR_MAP_SWIZZLE_128B))
      return cudaErrorNotSupported;
    static std::once_flag once2;
    static cudaError_t attr_err2 = cudaSuccess;
    std::call_once(once2, [] {
      attr_err2 = cudaFuncSetAttribute(tc_tma_ts_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)T3_SMEM);
    });
    if (attr_err2 != cudaSuccess) return attr_err2;
    TcGemmArgs h = g;
    // groups first when they share A (Pi's scales) and there are many tiles, or
    // when the tiles are very many (W_nm's frequencies share only B); measured:
    // large Pi and W_nm faster, the mid W_nm (188 tiles) slower that way
    h.groups_fastest = n_tiles <= 65535 && (g.a_group_stride == 0 ? n_tiles >= 64 : n_tiles >= 4096);
    const dim3 grid = h.groups_fastest ? dim3(groups, n_tiles, splits) : dim3(n_tiles, groups, splits);
    tc_tma_ts_kernel<<<grid, T3_THREADS, T3_SMEM, s>>>(h, ta, tbh, tbl);
    return cudaGetLastError();
  }
}

}  // namespace ltgw
