// Row ingest (Algorithm 1, "insert a_i into a zero valued row of B"; the
// squared Frobenius norm ||A||_F^2 of Sec. 1.1 kept in FP64).
//
// One CTA moves a tile of 32 rows x 128 columns of the incoming rows into
// the free rows of the buffer. FP32 rows whose row stride and base are
// 16-byte aligned are staged into shared memory by one TMA load
// (cp.async.bulk.tensor, a 2-D tensor map encoded per call; rows or columns
// past the end are filled with zeros by the copy engine); other input
// (bfloat16, FP64, unaligned FP32) is read by the threads, coalesced. From
// the tile each thread writes 16 consecutive values of one row (vector
// stores), and for the tensor-core buffer the transposed (column-major)
// planes are written from a padded copy of the tile, 32 rows of one column
// per warp instruction, so that both layouts are written coalesced.
// Squared row norms are summed in FP64 per tile; the last CTA of the launch
// adds each row's tiles in a fixed order and then the rows in order, so
// ||A||_F^2 does not depend on the schedule.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "fd_internal.cuh"

namespace fdk {

namespace {

constexpr int IG_ROWS = 32;
constexpr int IG_COLS = 128;
constexpr int IG_THREADS = 256;
constexpr long long IG_WAIT_LIMIT = 1ll << 22;

__device__ __forceinline__ uint32_t ig_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

struct IngestArgs {
  const void* src;
  int64_t ld;
  int dtype;
  int nrows;        // rows of this launch
  int64_t d;
  int row0;         // first buffer row written
  float* dst;       // FP32 row-major buffer (row stride ldd), or null
  int64_t ldd;
  __nv_bfloat16* rm_hi;  // tensor-core planes, or null
  __nv_bfloat16* rm_lo2;
  int64_t ld_rm;
  __nv_bfloat16* cm_hi;
  __nv_bfloat16* cm_lo;
  int64_t ld_cm;
  double* part;     // coltiles x 2 x nrows partial squared norms (input, stored)
  double* rownorm;  // per row of this launch: squared norm of the input row
  double* slot_n2;  // per buffer row: squared norm of the stored hi + lo (or null)
  DevCounters* ctr;
  unsigned int* ticket;
  int* err;
};

__global__ void __launch_bounds__(IG_THREADS)
    ingest_tile_kernel(const __grid_constant__ CUtensorMap map, int use_tma, IngestArgs a) {
  __shared__ __align__(128) float tile[IG_ROWS * IG_COLS];
  __shared__ float tpad[IG_ROWS * (IG_COLS + 1)];
  __shared__ __align__(8) uint64_t bar;
  __shared__ double rsum[IG_ROWS][2];
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  const int rt = blockIdx.x, ct = blockIdx.y;
  const int r0 = rt * IG_ROWS;
  const int64_t k0 = (int64_t)ct * IG_COLS;

  // 1. the tile (zeros past the last row or column)
  bool ok = true;
  if (use_tma) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ig_smem_u32(&bar)));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                       ig_smem_u32(&bar)),
                   "r"((uint32_t)(IG_ROWS * IG_COLS * 4))
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%3, %4}], [%2];" ::"r"(ig_smem_u32(tile)),
          "l"((uint64_t)&map), "r"(ig_smem_u32(&bar)), "r"((int)k0), "r"(r0)
          : "memory");
    }
    // bounded wait by every thread; a timeout raises the error flag and the
    // tile is taken as zeros
    uint32_t done = 0;
    for (long long it = 0; it < IG_WAIT_LIMIT && !done; ++it) {
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(ig_smem_u32(&bar))
          : "memory");
    }
    if (!done) {
      ok = false;
      atomicExch(a.err, 1);
    }
    ok = __syncthreads_and(ok);
    if (!ok)
      for (int i = tid; i < IG_ROWS * IG_COLS; i += IG_THREADS) tile[i] = 0.f;
  } else {
    for (int i = tid; i < IG_ROWS * IG_COLS; i += IG_THREADS) {
      const int r = i / IG_COLS, c = i - r * IG_COLS;
      const int64_t k = k0 + c;
      float v = 0.f;
      if (r0 + r < a.nrows && k < a.d) {
        const int64_t idx = (int64_t)(r0 + r) * a.ld + k;
        if (a.dtype == FD_F32) {
          v = reinterpret_cast<const float*>(a.src)[idx];
        } else if (a.dtype == FD_F64) {
          v = (float)reinterpret_cast<const double*>(a.src)[idx];
        } else {
          const unsigned short raw = reinterpret_cast<const unsigned short*>(a.src)[idx];
          v = __uint_as_float(((unsigned int)raw) << 16);
        }
      }
      tile[i] = v;
    }
  }
  if (tid < IG_ROWS) { rsum[tid][0] = 0.0; rsum[tid][1] = 0.0; }
  __syncthreads();

  // 2. row-major outputs: thread t takes row t / 8 and 16 consecutive columns
  {
    const int r = tid >> 3, c0 = (tid & 7) * 16;
    const bool row_live = r0 + r < a.nrows;
    double sa = 0.0;  // input values, squared
    float sb = 0.f;   // stored hi + lo, squared
    if (row_live) {
      const int64_t brow = a.row0 + r0 + r;
      if (a.dtype == FD_F64) {
        const double* s = reinterpret_cast<const double*>(a.src) + (int64_t)(r0 + r) * a.ld;
        for (int j = 0; j < 16; ++j) {
          const int64_t k = k0 + c0 + j;
          if (k < a.d) sa = fma(s[k], s[k], sa);
        }
      }
#pragma unroll
      for (int j4 = 0; j4 < 16; j4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(&tile[r * IG_COLS + c0 + j4]);
        const float x[4] = {v.x, v.y, v.z, v.w};
        const int64_t kb = k0 + c0 + j4;
        if (a.dtype != FD_F64)
#pragma unroll
          for (int u = 0; u < 4; ++u) sa = fma((double)x[u], (double)x[u], sa);
        if (a.dst != nullptr) {
          float* drow = a.dst + brow * a.ldd;
          if (kb + 3 < a.d && ((a.ldd & 3) == 0)) {
            *reinterpret_cast<float4*>(drow + kb) = v;
          } else {
            for (int u = 0; u < 4; ++u)
              if (kb + u < a.d) drow[kb + u] = x[u];
          }
        }
        if (a.rm_hi != nullptr) {
#pragma unroll
          for (int u = 0; u < 4; u += 2) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x[u]);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(x[u + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x[u] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x[u + 1] - __bfloat162float(h1));
            const float y0 = __bfloat162float(h0) + __bfloat162float(l0);
            const float y1 = __bfloat162float(h1) + __bfloat162float(l1);
            sb = fmaf(y0, y0, fmaf(y1, y1, sb));
            const int64_t k = kb + u;
            if (k + 1 < a.d) {
              __nv_bfloat162 hh, ll;
              hh.x = h0; hh.y = h1;
              ll.x = __float2bfloat16_rn(2.f * __bfloat162float(l0));
              ll.y = __float2bfloat16_rn(2.f * __bfloat162float(l1));
              *reinterpret_cast<__nv_bfloat162*>(a.rm_hi + brow * a.ld_rm + k) = hh;
              *reinterpret_cast<__nv_bfloat162*>(a.rm_lo2 + brow * a.ld_rm + k) = ll;
            } else if (k < a.d) {
              a.rm_hi[brow * a.ld_rm + k] = h0;
              a.rm_lo2[brow * a.ld_rm + k] = __float2bfloat16_rn(2.f * __bfloat162float(l0));
            }
          }
        }
      }
    }
    // the 8 threads of a row: a fixed-order tree
    double sbd = (double)sb;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sbd += __shfl_xor_sync(0xffffffffu, sbd, o);
    }
    if ((tid & 7) == 0) { rsum[r][0] = sa; rsum[r][1] = sbd; }
  }

  // 3. column-major planes (tensor-core buffer) through a padded copy
  if (a.cm_hi != nullptr) {
    for (int i = tid; i < IG_ROWS * IG_COLS; i += IG_THREADS) {
      const int r = i / IG_COLS, c = i - r * IG_COLS;
      tpad[r * (IG_COLS + 1) + c] = tile[i];
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    const bool live = r0 + lane < a.nrows;
    for (int c = warp; c < IG_COLS; c += IG_THREADS / 32) {
      const int64_t k = k0 + c;
      if (k >= a.d) break;  // warp-uniform
      const float x = tpad[lane * (IG_COLS + 1) + c];
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
      if (live) {
        a.cm_hi[k * a.ld_cm + a.row0 + r0 + lane] = h;
        a.cm_lo[k * a.ld_cm + a.row0 + r0 + lane] = l;
      }
    }
  }
  __syncthreads();

  // 4. partial squared norms of this tile; the last CTA adds them in order
  const int ncol = gridDim.y;
  if (tid < IG_ROWS && r0 + tid < a.nrows) {
    a.part[((int64_t)ct * 2 + 0) * a.nrows + r0 + tid] = rsum[tid][0];
    a.part[((int64_t)ct * 2 + 1) * a.nrows + r0 + tid] = rsum[tid][1];
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned int total = gridDim.x * gridDim.y;
    s_last = (atomicAdd(a.ticket, 1u) == total - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int r = tid; r < a.nrows; r += IG_THREADS) {
    double s0 = 0.0, s1 = 0.0;
    for (int c = 0; c < ncol; ++c) {
      s0 += ((volatile double*)a.part)[((int64_t)c * 2 + 0) * a.nrows + r];
      s1 += ((volatile double*)a.part)[((int64_t)c * 2 + 1) * a.nrows + r];
    }
    a.rownorm[r] = s0;
    if (a.slot_n2 != nullptr) a.slot_n2[a.row0 + r] = s1;
  }
  __syncthreads();
  if (tid == 0) {
    double tot = a.ctr->norm_a2;
    for (int r = 0; r < a.nrows; ++r) tot += a.rownorm[r];
    a.ctr->norm_a2 = tot;
    *a.ticket = 0u;
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point.
typedef CUresult (*IgEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                               const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                               const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

IgEncodeFn ig_encode() {
  static IgEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<IgEncodeFn>(p);
  }
  return fn;
}

}  // namespace

size_t ingest_part_bytes(int64_t d, int max_rows) {
  return (size_t)((d + IG_COLS - 1) / IG_COLS) * 2 * (size_t)max_rows * sizeof(double);
}

cudaError_t launch_ingest_tiles(const void* src, int64_t n, int64_t ld, int dtype, float* dst,
                                int64_t ldd, int64_t d, int row0, __nv_bfloat16* rm_hi,
                                __nv_bfloat16* rm_lo2, int64_t ld_rm, __nv_bfloat16* cm_hi,
                                __nv_bfloat16* cm_lo, int64_t ld_cm, double* part,
                                double* rownorm, double* slot_n2, DevCounters* ctr,
                                unsigned int* ticket, int* err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  IngestArgs a;
  a.src = src; a.ld = ld; a.dtype = dtype; a.nrows = (int)n; a.d = d; a.row0 = row0;
  a.dst = dst; a.ldd = ldd;
  a.rm_hi = rm_hi; a.rm_lo2 = rm_lo2; a.ld_rm = ld_rm;
  a.cm_hi = cm_hi; a.cm_lo = cm_lo; a.ld_cm = ld_cm;
  a.part = part; a.rownorm = rownorm; a.slot_n2 = slot_n2; a.ctr = ctr; a.ticket = ticket;
  a.err = err;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  int use_tma = 0;
  // TMA needs a 16-byte aligned base and row stride; the box starts at
  // column multiples of 128 (x * 4 bytes, a multiple of 16)
  IgEncodeFn enc = ig_encode();
  if (enc != nullptr && dtype == FD_F32 && ((uintptr_t)src & 15) == 0 && (ld & 3) == 0) {
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {IG_COLS, IG_ROWS};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(src), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      use_tma = 1;
  }
  const dim3 grid((unsigned)((n + IG_ROWS - 1) / IG_ROWS), (unsigned)((d + IG_COLS - 1) / IG_COLS));
  ingest_tile_kernel<<<grid, IG_THREADS, 0, st>>>(map, use_tma, a);
  return cudaGetLastError();
}

}  // namespace fdk
