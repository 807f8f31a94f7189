// Tensor-core path (FD_PREC_BF16X3): Gram and rotate on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in TMEM, operands staged by TMA).
//
// Split precision. Every FP32 value x of the buffer is held as two bfloat16
// numbers hi = bf16(x), lo = bf16(x - hi), so x = hi + lo to about 2^-17.
// A product x*y is taken as hi_x*hi_y + hi_x*lo_y + lo_x*hi_y (the lo*lo term,
// about 2^-16 of the product, is dropped) and accumulated in FP32: each K step
// of 16 in a fresh TMEM accumulator, the steps added in registers. The Gram's
// diagonal, where lo*lo is a sum of squares, is replaced by the eigensolve
// with FP64 squared norms of the stored rows.
//
// Buffer layout in HBM (one sketch of width d, buffer of L rows, L = 2*ell by default):
//   rm_hi, rm_lo2: row-major  L x ldb  (ldb = d rounded up to 64), lo2 = 2*lo
//   cm_hi, cm_lo:  column-major (d x L stored as ldb rows of ldl, ldl = L up
//                  to a multiple of 64)
// The Gram G = B B^T reads the row-major planes (K = d contiguous); the rotate
// B'^T = B^T W^T reads the column-major planes (K = L contiguous); both are
// K-major tcgen05 operands in the 128-byte swizzled layout TMA writes.
//
// Gram: Z = Bh Bh^T + Bh (2 Bl)^T in one accumulator; G = (Z + Z^T) / 2 =
// Bh Bh^T + Bh Bl^T + Bl Bh^T (the eigensolve symmetrises when it loads G).
// A cluster of up to 8 CTAs splits K = d; the partial tiles are summed in a
// fixed order through distributed shared memory, so G is deterministic.
//
// Rotate: D (128 rows of d x N = ell-1 padded to 16) = B^T W^T with three
// MMAs per K step (hi*hi, hi*lo, lo*hi); the epilogue splits D = B'^T again
// and writes it into both layouts (or to FP32 rows for a non-destructive
// flush). One CTA owns 128 values of d and all of K, so writing in place is
// safe once its MMAs have completed.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "fd_internal.cuh"

namespace cg = cooperative_groups;

namespace fdk {

cudaError_t launch_eig_shrink_f32(const EigArgs& a, cudaStream_t st);

namespace {

constexpr int TILE_BYTES = 128 * 128;  // 128 rows x 64 bf16
constexpr long long WAIT_LIMIT = 1ll << 20;

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and raises the error flag) after WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D (TMEM) [+]= A (smem desc) * B (smem desc)^T, bf16 inputs, fp32 accumulate.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major tile, 128-byte swizzle, rows of
// 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr & 0x3FFFFull) >> 4;       // start address
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset: 8-row atoms
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::f16, A = B = bf16, D = f32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// ---------------------------------------------------------------------------
// Accumulation. The tensor core adds the products of one MMA into its FP32
// accumulator with truncation, so a long chain of MMAs into one accumulator
// drifts toward zero by about half an ulp per MMA; over the thousands of
// reductions of a stream that bias removes mass from every retained row.
// Each K = 16 step therefore goes into a fresh TMEM accumulator (two,
// alternating), and four epilogue warps add it into a running sum held in
// registers with FP32 round-to-nearest adds while the next step runs.
// Warp roles: 0 = TMA producer, 1 = MMA issuer (and TMEM owner), 2..5 =
// epilogue (warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31).
// ---------------------------------------------------------------------------
constexpr int TC_WARPS = 6;
constexpr int TC_NT = 32 * TC_WARPS;
constexpr uint32_t TC_TMEM_COLS = 256;  // two accumulators of up to 128 columns

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait of every lane of a warp; true only if all lanes saw the phase.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* err) {
  const bool ok = mbar_wait(bar, parity, err);
  return __all_sync(0xffffffffu, ok) != 0;
}

// Epilogue: drain accumulator b (columns b*128 .. b*128 + 32*nch - 1 of this
// warp's 32 lanes) into acc with round-to-nearest adds.
// A tcgen05.mma result rounds toward zero: each step's value is short of the
// exact sum of its products by part of an ulp, always on the side of zero,
// and over the K steps of a product, and over the reductions of a stream,
// those shortfalls add up (uncorrected, the sketch lost about 1e-6 of each
// row's mass at every rotate at 2*ell = 200). The correction is
// proportional to each step's value, so the corrections of all steps sum to
// one factor times the accumulated sum, applied once at the end: kTcRound
// per rounding in a step. Half an ulp (a uniformly distributed discarded
// fraction) would be 2^-24 / (2 ln 2) of a value with log-uniform mantissa;
// the shortfall measured through the rotate's row masses on the Random
// Noisy stream (d = 2,000, ell = 100) is smaller, about 2^-25 of the value
// (many step sums need no rounding at all), and that is the factor used.
constexpr float kTcRound = 2.9802322e-08f;  // 2^-25

template <int NCH>
__device__ __forceinline__ void drain_add(uint32_t taddr, int q, int b, int nch, float* acc) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    if (c < nch) {
      float v[32];
      tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 128 + c * 32), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[c * 32 + i] += v[i];
    }
  }
}

// The same for two accumulators per step: the large products (columns
// b*128..) and the small cross products (columns 256 + b*128..).
template <int NCH>
__device__ __forceinline__ void drain_add2(uint32_t taddr, int q, int b, int nch, float* acc) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    if (c < nch) {
      float v[32], w[32];
      tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 128 + c * 32), v);
      tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(256 + b * 128 + c * 32), w);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[c * 32 + i] += v[i] + w[i];
    }
  }
}

// ---------------------------------------------------------------------------
// Gram kernel. Grid = tiles * ks (cluster of ks CTAs along x per 128x128 tile).
// Each CTA sums its share of K; the ks partial tiles are added in a fixed
// order through distributed shared memory.
// ---------------------------------------------------------------------------
constexpr int GRAM_STAGES = 4;
constexpr int GRAM_STAGE_BYTES = 3 * TILE_BYTES;  // A (hi), B (hi), B (2 lo)
constexpr int GRAM_PLD = 129;                     // partial tile row stride (floats)

__global__ void __launch_bounds__(TC_NT, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap map_hi,
                   const __grid_constant__ CUtensorMap map_lo2, float* __restrict__ G, int ldg,
                   int nrows, int kblocks, int ks, int ntiles_side, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + GRAM_STAGES * GRAM_STAGE_BYTES);
  uint64_t* empty = full + GRAM_STAGES;
  uint64_t* accfull = empty + GRAM_STAGES;
  uint64_t* accfree = accfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accfree + 2);
  float* part = reinterpret_cast<float*>(stages);  // reused after the MMAs complete

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tile = blockIdx.x / ks;
  const int ti = tile / ntiles_side, tj = tile % ntiles_side;
  const int i0 = ti * 128, j0 = tj * 128;
  const int per = (kblocks + ks - 1) / ks;
  const int kb0 = min(kblocks, rank * per), kb1 = min(kblocks, kb0 + per);
  const int nk = kb1 - kb0;
  const int nsteps = 4 * nk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < GRAM_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accfull[b], 1); mbar_init(&accfree[b], 4); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tslot, TC_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      for (int it = 0; it < nk && ok; ++it) {
        const int s = it % GRAM_STAGES;
        if (it >= GRAM_STAGES) ok = mbar_wait(&empty[s], ((it / GRAM_STAGES) - 1) & 1, err);
        if (!ok) break;
        uint8_t* st = stages + s * GRAM_STAGE_BYTES;
        mbar_expect_tx(&full[s], GRAM_STAGE_BYTES);
        const int kc = (kb0 + it) * 64;
        tma_load_2d(st, &map_hi, &full[s], kc, i0);
        tma_load_2d(st + TILE_BYTES, &map_hi, &full[s], kc, j0);
        tma_load_2d(st + 2 * TILE_BYTES, &map_lo2, &full[s], kc, j0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, 128);
      bool ok = true;
      for (int it = 0; it < nk && ok; ++it) {
        const int s = it % GRAM_STAGES;
        ok = mbar_wait(&full[s], (it / GRAM_STAGES) & 1, err);
        if (!ok) break;
        tc_fence_after();
        uint8_t* st = stages + s * GRAM_STAGE_BYTES;
#pragma unroll 1
        for (int kk = 0; kk < 4 && ok; ++kk) {
          const int step = it * 4 + kk, b = step & 1;
          if (step >= 2) {
            ok = mbar_wait(&accfree[b], ((step >> 1) - 1) & 1, err);
            if (!ok) break;
            tc_fence_after();
          }
          const uint32_t dt = taddr + (uint32_t)(b * 128);
          const uint64_t a = smem_desc_sw128(st + kk * 32);
          const uint64_t b1 = smem_desc_sw128(st + TILE_BYTES + kk * 32);
          const uint64_t b2 = smem_desc_sw128(st + 2 * TILE_BYTES + kk * 32);
          mma_bf16(dt, a, b1, idesc, 0u);
          mma_bf16(dt, a, b2, idesc, 1u);
          mma_commit(&accfull[b]);
        }
        mma_commit(&empty[s]);
      }
    }
  } else {
    // epilogue: running sum of row r = 32 q + lane over the 128 columns
    const int q = warp & 3, r = q * 32 + lane;
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
    for (int step = 0; step < nsteps; ++step) {
      const int b = step & 1;
      if (!warp_wait(&accfull[b], (step >> 1) & 1, err)) break;
      tc_fence_after();
      drain_add<4>(taddr, q, b, 4, acc);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[b]);
    }
#pragma unroll
    for (int i = 0; i < 128; ++i) part[r * GRAM_PLD + i] = fmaf(acc[i], 2.f * kTcRound, acc[i]);  // two roundings a step
  }
  __syncwarp();  // the producer and MMA lanes rejoin their warps
  tc_fence_before();
  cluster.sync();
  // fixed-order sum of the ks partial tiles; this CTA writes its row slice
  {
    const int rows_per = (128 + ks - 1) / ks;
    const int rs0 = rank * rows_per, rs1 = min(128, rs0 + rows_per);
    for (int idx = threadIdx.x; idx < (rs1 - rs0) * 128; idx += TC_NT) {
      const int r = rs0 + idx / 128, c = idx % 128;
      float s = 0.0f;
      for (int q = 0; q < ks; ++q) {
        const float* rp = cluster.map_shared_rank(part, q);
        s += rp[r * GRAM_PLD + c];
      }
      const int gi = i0 + r, gj = j0 + c;
      if (gi < nrows && gj < nrows) G[(int64_t)gi * ldg + gj] = s;
    }
  }
  cluster.sync();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(taddr, TC_TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Rotate kernel. Grid = (ceil(d / 128), nsplit): CTA (x, y) computes the
// 128 values m0 .. m0+127 of d for output rows y*NC .. y*NC + NC - 1
// (NC <= 128, a multiple of 16; nsplit * NC >= ell - 1). The hi*hi products
// of a step have an accumulator of their own (the truncation of one MMA is
// relative to its result, and the retained row's own term makes that result
// as large as the output); the small cross products share a second one.
// ---------------------------------------------------------------------------
constexpr int ROT_STAGES = 2;

__global__ void __launch_bounds__(TC_NT, 1)
    rotate_tc_kernel(const __grid_constant__ CUtensorMap map_cm_hi,
                     const __grid_constant__ CUtensorMap map_cm_lo,
                     const __grid_constant__ CUtensorMap map_w_hi,
                     const __grid_constant__ CUtensorMap map_w_lo, int kblocks, int NC, int nout,
                     int64_t d, __nv_bfloat16* rm_hi, __nv_bfloat16* rm_lo2, int64_t ld_rm,
                     __nv_bfloat16* cm_hi, __nv_bfloat16* cm_lo, int64_t ld_cm,
                     float* out_rows, int64_t ldo, double* rot_part, int rot_ld, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  const int wbytes = NC * 128;
  const int stage_bytes = 2 * TILE_BYTES + 2 * wbytes;
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ROT_STAGES * stage_bytes);
  uint64_t* empty = full + ROT_STAGES;
  uint64_t* accfull = empty + ROT_STAGES;
  uint64_t* accfree = accfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accfree + 2);
  const int m0 = blockIdx.x * 128;
  const int n0 = blockIdx.y * NC;
  const int nsteps = 4 * kblocks;
  const int nch = (NC + 31) / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ROT_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accfull[b], 1); mbar_init(&accfree[b], 4); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tslot, 2 * TC_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tslot;

  float acc[128];
#pragma unroll
  for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
  bool drained = true;
  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      for (int it = 0; it < kblocks && ok; ++it) {
        const int s = it % ROT_STAGES;
        if (it >= ROT_STAGES) ok = mbar_wait(&empty[s], ((it / ROT_STAGES) - 1) & 1, err);
        if (!ok) break;
        uint8_t* st = stages + s * stage_bytes;
        mbar_expect_tx(&full[s], (uint32_t)stage_bytes);
        const int kc = it * 64;
        tma_load_2d(st, &map_cm_hi, &full[s], kc, m0);
        tma_load_2d(st + TILE_BYTES, &map_cm_lo, &full[s], kc, m0);
        tma_load_2d(st + 2 * TILE_BYTES, &map_w_hi, &full[s], kc, n0);
        tma_load_2d(st + 2 * TILE_BYTES + wbytes, &map_w_lo, &full[s], kc, n0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, NC);
      bool ok = true;
      for (int it = 0; it < kblocks && ok; ++it) {
        const int s = it % ROT_STAGES;
        ok = mbar_wait(&full[s], (it / ROT_STAGES) & 1, err);
        if (!ok) break;
        tc_fence_after();
        uint8_t* st = stages + s * stage_bytes;
#pragma unroll 1
        for (int kk = 0; kk < 4 && ok; ++kk) {
          const int step = it * 4 + kk, b = step & 1;
          if (step >= 2) {
            ok = mbar_wait(&accfree[b], ((step >> 1) - 1) & 1, err);
            if (!ok) break;
            tc_fence_after();
          }
          const uint32_t dt = taddr + (uint32_t)(b * 128);
          const uint32_t dx = taddr + (uint32_t)(256 + b * 128);
          const uint64_t ah = smem_desc_sw128(st + kk * 32);
          const uint64_t al = smem_desc_sw128(st + TILE_BYTES + kk * 32);
          const uint64_t wh = smem_desc_sw128(st + 2 * TILE_BYTES + kk * 32);
          const uint64_t wl = smem_desc_sw128(st + 2 * TILE_BYTES + wbytes + kk * 32);
          mma_bf16(dt, ah, wh, idesc, 0u);
          mma_bf16(dx, ah, wl, idesc, 0u);
          mma_bf16(dx, al, wh, idesc, 1u);
          mma_commit(&accfull[b]);
        }
        mma_commit(&empty[s]);
      }
    }
  } else {
    const int q = warp & 3;
    for (int step = 0; step < nsteps; ++step) {
      const int b = step & 1;
      if (!warp_wait(&accfull[b], (step >> 1) & 1, err)) { drained = false; break; }
      tc_fence_after();
      drain_add2<4>(taddr, q, b, nch, acc);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[b]);
    }
  }
  // Every MMA has completed and every stage was consumed once the epilogue
  // saw the last step, so the stage memory is free for the row sums.
  __syncwarp();  // the producer and MMA lanes rejoin their warps
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  float* wsum = reinterpret_cast<float*>(stages);  // 4 x 128 partial squared norms
  if (warp >= 2) {
    const int q = warp & 3;
    const int64_t m = m0 + q * 32 + lane;  // this thread's d index
    const bool live = (m < d) && drained;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c >= nch) break;  // warp-uniform
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int jl = c * 32 + i, j = n0 + jl;
        const float x0 = acc[c * 32 + i];
        float sq = 0.0f;
        if (live && jl < NC && j < nout) {
          if (out_rows) {
            out_rows[(int64_t)j * ldo + m] = fmaf(x0, kTcRound, x0);  // one rounding a step (hi.hi)
          } else {
            // the correction goes into the low part, where it is far above
            // the rounding unit (x0 - hi is exact)
            const __nv_bfloat16 hi = __float2bfloat16_rn(x0);
            const __nv_bfloat16 lo =
                __float2bfloat16_rn(fmaf(x0, kTcRound, x0 - __bfloat162float(hi)));
            cm_hi[m * ld_cm + j] = hi;
            cm_lo[m * ld_cm + j] = lo;
            rm_hi[(int64_t)j * ld_rm + m] = hi;
            rm_lo2[(int64_t)j * ld_rm + m] = __float2bfloat16_rn(2.0f * __bfloat162float(lo));
            const float y = __bfloat162float(hi) + __bfloat162float(lo);
            sq = y * y;
          }
        }
        v[i] = sq;
      }
      if (rot_part != nullptr) {
        // transpose-reduce: after the step with offset o each lane keeps the
        // half of its values selected by its bit o, added to its partner's;
        // lane i ends with row c*32+i summed over the warp's 32 columns
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
          const bool up = (lane & o) != 0;
#pragma unroll
          for (int k = 0; k < o; ++k) {
            const float send = up ? v[k] : v[k + o];
            const float keep = up ? v[k + o] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
        }
        wsum[q * 128 + c * 32 + lane] = v[0];
      }
    }
  }
  if (rot_part != nullptr) {
    __syncthreads();
    for (int j = threadIdx.x; j < NC; j += TC_NT) {
      const double t = ((double)wsum[j] + (double)wsum[128 + j]) +
                       ((double)wsum[256 + j] + (double)wsum[384 + j]);
      rot_part[(int64_t)blockIdx.x * rot_ld + n0 + j] = t;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(taddr, 2 * TC_TMEM_COLS);
}

// hi + lo of the first `rows` buffer rows as FP32 (row-major planes).
__global__ void export_rows_kernel(const __nv_bfloat16* __restrict__ rm_hi,
                                   const __nv_bfloat16* __restrict__ rm_lo2, int64_t ld_rm,
                                   int rows, int64_t d, float* __restrict__ out, int64_t ldo) {
  const int r = blockIdx.x;
  if (r >= rows) return;
  for (int64_t k = threadIdx.x; k < d; k += blockDim.x)
    out[(int64_t)r * ldo + k] = __bfloat162float(rm_hi[r * ld_rm + k]) +
                                0.5f * __bfloat162float(rm_lo2[r * ld_rm + k]);
}

// ---- host side ----------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D bf16 map over a row-major [rows][ld] array, box = 64 x box_rows, 128B swizzle.
bool make_map(CUtensorMap* map, void* base, uint64_t ld, uint64_t rows, uint32_t box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {ld, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

struct TcCtx {
  int64_t d = 0, ldb = 0;
  int ell = 0, L = 0, ldl = 0;
  int NC = 0, nsplit = 1;  // rotate output rows per CTA, CTAs along them
  cudaStream_t st = nullptr;
  __nv_bfloat16 *rm_hi = nullptr, *rm_lo2 = nullptr, *cm_hi = nullptr, *cm_lo = nullptr;
  __nv_bfloat16 *w_hi = nullptr, *w_lo = nullptr;
  float* G = nullptr;
  float* wrot32 = nullptr;
  int* err = nullptr;
  // exact Gram diagonal (see EigArgs): FP64 squared norms of the stored new
  // rows, the rotate's per-CTA partial squared norms of the rows it wrote,
  // and the per-reduction diagonal
  double* slot_n2 = nullptr;
  double* rot_part = nullptr;
  double* diag64 = nullptr;
  int rot_grid = 0, rot_ld = 0;
  int keep = 0;   // rows a reduction leaves
  int nret = 0;   // leading buffer rows written by the last committed rotate
  CUtensorMap m_rm_hi, m_rm_lo2, m_cm_hi, m_cm_lo, m_w_hi, m_w_lo;
  int ks = 1;
  size_t gram_smem = 0, rot_smem = 0;
};

int tc_available() { return get_encode() != nullptr ? 1 : 0; }

void tc_destroy(TcCtx* t) {
  if (!t) return;
  cudaFree(t->rm_hi); cudaFree(t->rm_lo2); cudaFree(t->cm_hi); cudaFree(t->cm_lo);
  cudaFree(t->w_hi); cudaFree(t->w_lo); cudaFree(t->G); cudaFree(t->wrot32); cudaFree(t->err);
  cudaFree(t->slot_n2); cudaFree(t->rot_part); cudaFree(t->diag64);
  delete t;
}

int tc_create(TcCtx** out, int64_t d, int ell, int L, int keep, cudaStream_t st) {
  *out = nullptr;
  TcCtx* t = new (std::nothrow) TcCtx();
  if (!t) return FD_ENOMEM;
  t->d = d;
  t->ldb = (d + 63) / 64 * 64;
  t->ell = ell;
  t->L = L;
  t->ldl = (t->L + 63) / 64 * 64;
  {
    int np = ((ell - 1) + 15) / 16 * 16;
    if (np < 16) np = 16;
    t->nsplit = (np + 127) / 128;
    t->NC = ((np + t->nsplit - 1) / t->nsplit + 15) / 16 * 16;
  }
  t->rot_ld = t->nsplit * t->NC;
  t->st = st;
  t->keep = keep;
  t->rot_grid = (int)((d + 127) / 128);
  const size_t plane_rm = (size_t)t->L * t->ldb * 2;
  const size_t plane_cm = (size_t)t->ldb * t->ldl * 2;
  const size_t wplane = (size_t)t->rot_ld * t->ldl * 2;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t b) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(p, b);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, b, st);
  };
  alloc((void**)&t->rm_hi, plane_rm);
  alloc((void**)&t->rm_lo2, plane_rm);
  alloc((void**)&t->cm_hi, plane_cm);
  alloc((void**)&t->cm_lo, plane_cm);
  alloc((void**)&t->w_hi, wplane);
  alloc((void**)&t->w_lo, wplane);
  alloc((void**)&t->G, (size_t)t->L * t->L * 4);
  alloc((void**)&t->wrot32, (size_t)ell * t->ldl * 4);
  alloc((void**)&t->err, sizeof(int));
  alloc((void**)&t->slot_n2, (size_t)t->L * 8);
  alloc((void**)&t->rot_part, (size_t)t->rot_grid * t->rot_ld * 8);
  alloc((void**)&t->diag64, (size_t)t->L * 8);
  if (e != cudaSuccess) {
    set_cuda_error(e, "tc_create alloc");
    tc_destroy(t);
    return FD_ENOMEM;
  }
  bool ok = make_map(&t->m_rm_hi, t->rm_hi, t->ldb, t->L, 128) &&
            make_map(&t->m_rm_lo2, t->rm_lo2, t->ldb, t->L, 128) &&
            make_map(&t->m_cm_hi, t->cm_hi, t->ldl, t->ldb, 128) &&
            make_map(&t->m_cm_lo, t->cm_lo, t->ldl, t->ldb, 128) &&
            make_map(&t->m_w_hi, t->w_hi, t->ldl, t->rot_ld, t->NC) &&
            make_map(&t->m_w_lo, t->w_lo, t->ldl, t->rot_ld, t->NC);
  if (!ok) {
    tc_destroy(t);
    return FD_EINVAL;
  }
  const int kblocks = (int)(t->ldb / 64);
  t->ks = kblocks < 8 ? kblocks : 8;
  if (t->ks < 1) t->ks = 1;
  t->gram_smem = 1024 + GRAM_STAGES * GRAM_STAGE_BYTES + 256;
  t->rot_smem = 1024 + ROT_STAGES * (2 * TILE_BYTES + 2 * t->NC * 128) + 256;
  e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)t->gram_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rotate_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)t->rot_smem);
  if (e != cudaSuccess) {
    set_cuda_error(e, "tc_create attributes");
    tc_destroy(t);
    return FD_ECUDA;
  }
  *out = t;
  return FD_OK;
}

int tc_ingest(TcCtx* t, const void* src, int64_t n, int64_t ld, int dtype, int row0,
              double* rownorm, DevCounters* ctr, double* part) {
  cudaError_t e = launch_ingest_tiles(src, n, ld, dtype, nullptr, 0, t->d, row0, t->rm_hi,
                                      t->rm_lo2, t->ldb, t->cm_hi, t->cm_lo, t->ldl, part,
                                      rownorm, t->slot_n2, ctr, &ctr->ingest_ticket, t->err,
                                      t->st);
  if (e != cudaSuccess) { set_cuda_error(e, "tc_ingest"); return FD_ECUDA; }
  return FD_OK;
}

// One reduction in three launches (Gram, eigensolve + shrink, rotate), split
// so that the caller can time each.
int tc_gram(TcCtx* t, int nrows) {
  cudaError_t e;
  if (nrows < t->L) {
    // a flush of fewer rows: rows nrows..L-1 hold earlier input, free slots
    // that must read as zero
    e = cudaMemsetAsync(t->rm_hi + (size_t)nrows * t->ldb, 0, (size_t)(t->L - nrows) * t->ldb * 2, t->st);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(t->rm_lo2 + (size_t)nrows * t->ldb, 0, (size_t)(t->L - nrows) * t->ldb * 2, t->st);
    if (e == cudaSuccess)
      e = cudaMemset2DAsync(t->cm_hi + nrows, (size_t)t->ldl * 2, 0, (size_t)(t->L - nrows) * 2, (size_t)t->ldb, t->st);
    if (e == cudaSuccess)
      e = cudaMemset2DAsync(t->cm_lo + nrows, (size_t)t->ldl * 2, 0, (size_t)(t->L - nrows) * 2, (size_t)t->ldb, t->st);
    if (e != cudaSuccess) { set_cuda_error(e, "tc flush zero"); return FD_ECUDA; }
  }
  // Gram
  const int side = (nrows + 127) / 128;
  const int kblocks = (int)(t->ldb / 64);
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)t->ks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(side * side * t->ks), 1, 1);
  cfg.blockDim = dim3(TC_NT, 1, 1);
  cfg.dynamicSmemBytes = t->gram_smem;
  cfg.stream = t->st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, gram_tc_kernel, t->m_rm_hi, t->m_rm_lo2, t->G, t->L, nrows, kblocks,
                         t->ks, side, t->err);
  if (e != cudaSuccess) { set_cuda_error(e, "gram_tc_kernel"); return FD_ECUDA; }
  return FD_OK;
}

int tc_eig(TcCtx* t, const EigArgs& tmpl, int commit) {
  cudaError_t e;
  EigArgs a = tmpl;
  a.nret = t->nret;
  a.rot_part = t->rot_part;
  a.rot_nparts = t->rot_grid;
  a.rot_ld = t->rot_ld;
  a.slot_n2 = t->slot_n2;
  a.diag64 = t->diag64;
  (void)commit;
  a.parts = t->G;
  a.nparts = 1;
  a.ldp = t->L;
  a.part_stride = 0;
  a.symmetrize = 1;
  a.wrot = t->wrot32;
  a.ldr = t->ldl;
  a.wrot_hi = t->w_hi;
  a.wrot_lo = t->w_lo;
  a.ldr16 = t->ldl;
  e = launch_eig_shrink_f32(a, t->st);
  if (e != cudaSuccess) { set_cuda_error(e, "eig_shrink (tc)"); return FD_ECUDA; }
  return FD_OK;
}

int tc_rotate(TcCtx* t, int nrows, int write_sketch, float* sketch_out, int64_t ldo) {
  cudaError_t e;
  const int kb_rot = (nrows + 63) / 64;
  const dim3 grid((unsigned)t->rot_grid, (unsigned)t->nsplit, 1);
  rotate_tc_kernel<<<grid, TC_NT, t->rot_smem, t->st>>>(
      t->m_cm_hi, t->m_cm_lo, t->m_w_hi, t->m_w_lo, kb_rot, t->NC, t->ell - 1, t->d, t->rm_hi,
      t->rm_lo2, t->ldb, t->cm_hi, t->cm_lo, t->ldl, write_sketch ? sketch_out : nullptr, ldo,
      write_sketch ? nullptr : t->rot_part, t->rot_ld, t->err);
  e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e, "rotate_tc_kernel"); return FD_ECUDA; }
  if (!write_sketch) t->nret = t->keep;
  return FD_OK;
}

// Zero the buffer planes (a fresh, empty sketch).
int tc_reset(TcCtx* t) {
  const size_t plane_rm = (size_t)t->L * t->ldb * 2;
  const size_t plane_cm = (size_t)t->ldb * t->ldl * 2;
  cudaError_t e = cudaMemsetAsync(t->rm_hi, 0, plane_rm, t->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->rm_lo2, 0, plane_rm, t->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->cm_hi, 0, plane_cm, t->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->cm_lo, 0, plane_cm, t->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->err, 0, sizeof(int), t->st);
  if (e != cudaSuccess) { set_cuda_error(e, "tc_reset"); return FD_ECUDA; }
  t->nret = 0;
  return FD_OK;
}

// Nonzero when a bounded wait of a tensor-core kernel gave up (synchronises).
int tc_error(TcCtx* t) {
  int h = 0;
  if (cudaMemcpyAsync(&h, t->err, sizeof(int), cudaMemcpyDeviceToHost, t->st) != cudaSuccess) return 1;
  if (cudaStreamSynchronize(t->st) != cudaSuccess) return 1;
  return h;
}

int tc_export_rows(TcCtx* t, int rows, float* out, int64_t ldo) {
  if (rows <= 0) return FD_OK;
  export_rows_kernel<<<rows, 256, 0, t->st>>>(t->rm_hi, t->rm_lo2, t->ldb, rows, t->d, out, ldo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e, "export_rows"); return FD_ECUDA; }
  return FD_OK;
}

}  // namespace fdk
