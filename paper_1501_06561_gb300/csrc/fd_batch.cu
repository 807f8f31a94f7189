// Batched update of many independent sketches in one persistent launch.
//
// Every sketch keeps its own 2*ell x d FP32 buffer and FP64 counters in HBM.
// A fixed grid of CTAs (two per SM) pulls work items -- (sketch, block of
// rows) -- from a device queue ordered longest-first; the CTA that takes an
// item runs the whole row block through Algorithm 1 (Sec. 2.3) for that
// sketch: ingest, and at every full buffer one reduction done entirely inside
// the CTA (Gram into shared memory; the tridiagonal eigensolve of a full
// buffer, or block Jacobi for a partial one at a flush, both in shared memory;
// FP64 ReduceRank; rotate back into the buffer). No inter-CTA
// synchronisation is needed because a sketch is owned by one CTA at a time.
// Each append is one item-table copy, one counter reset and one launch on the
// batch's stream; the tile sizes below are compile-time constants.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fd_internal.cuh"
#include "fd_eig.cuh"
#include "fd_jacobi.cuh"
#include "fd_tridiag.cuh"

namespace fdk {

namespace {

constexpr int BT = 256;           // threads per CTA
constexpr int GB = (528 + BT - 1) / BT;  // Gram 4x4 blocks per thread (<= 528 blocks)
constexpr int BMAX_L = 128;       // largest buffer (2*ell) a batched sketch may have
constexpr int KCH = 32;           // Gram K chunk
constexpr int RCH = 64;           // rotate column chunk
// Global workspace of one CTA for the Rayleigh-Ritz refinement of a full
// buffer: the scaled Gram (BMAX_L rows, stride BMAX_L) and the vectors /
// G U products ((BMAX_L / 2 + 4) x BMAX_L floats).
constexpr size_t BATCH_WS_FLOATS = (size_t)BMAX_L * BMAX_L + (size_t)(BMAX_L / 2 + 4) * BMAX_L;

struct BatchSketch {
  long long d, ldb;
  int ell, L, m, pad;
  float* buf;          // L x ldb, FP32
  DevCounters* ctr;
};

struct BatchItem {
  int id, dtype;
  const void* rows;
  long long n, ld;
};

__device__ __forceinline__ float load_as_f32(const void* p, long long idx, int dtype) {
  if (dtype == FD_F32) return reinterpret_cast<const float*>(p)[idx];
  if (dtype == FD_F64) return (float)reinterpret_cast<const double*>(p)[idx];
  const unsigned short raw = reinterpret_cast<const unsigned short*>(p)[idx];
  return __uint_as_float(((unsigned int)raw) << 16);
}

__device__ __forceinline__ double load_as_f64(const void* p, long long idx, int dtype) {
  if (dtype == FD_F64) return reinterpret_cast<const double*>(p)[idx];
  return (double)load_as_f32(p, idx, dtype);
}

// Shared memory map (bytes): region A 64 KB (Jacobi matrix / rotate staging),
// region B 32 KB (Gram staging / rotate matrix), scalars.
constexpr int TRI_NB = 16;        // inverse-iteration vectors per batch
static_assert(BT / 32 * 32 * TRI_CPT >= BMAX_L, "step 1 of the solve covers 2*ell - 1 columns");
constexpr size_t REG_A = ((size_t)BMAX_L * (BMAX_L | 1) * 4 + 15) / 16 * 16;
constexpr size_t REG_B = (size_t)BMAX_L * RCH * 4;
constexpr size_t SCAL = (size_t)BMAX_L * (4 * sizeof(double) + 2 * sizeof(int)) + BMAX_L * 4 + 256;
constexpr size_t REST = (REG_B + SCAL > tri_rest_bytes(BMAX_L, TRI_NB)) ? REG_B + SCAL
                                                                       : tri_rest_bytes(BMAX_L, TRI_NB);
constexpr size_t BATCH_SMEM = REG_A + REST;

// One reduction of the first `nrows` rows of S.buf; new rows 0..ell-2 go to
// `out` (stride ldo; may be S.buf itself), counters from cin to cout.
__device__ void batch_reduce(const BatchSketch& S, int nrows, float* out, long long ldo,
                             const DevCounters* cin, DevCounters* cout, int variant,
                             double alpha, int max_sweeps, double tol, unsigned char* smem,
                             float* ws = nullptr) {
  const int tid = threadIdx.x;
  float* A = reinterpret_cast<float*>(smem);
  float* Bst = reinterpret_cast<float*>(smem + REG_A);
  __shared__ double s_mass[BMAX_L / 2];       // sigma'^2 of each output row
  unsigned char* sc = smem + REG_A + REG_B;
  const int np = nrows + (nrows & 1);
  const int npb = (np + 7) & ~7;  // block Jacobi pads to whole 4-column block pairs
  // full buffers take the tridiagonal eigensolve (odd stride), flushes Jacobi
  const bool tri = (nrows == 2 * S.ell) && nrows >= 4;
  const int ld = tri ? (nrows | 1) : npb;
  const int nz = tri ? nrows : npb;  // rows of A in use
  const long long d = S.d, ldb = S.ldb;
  const float* buf = S.buf;

  // ---- Gram G = B B^T (upper 4x4 blocks, K in chunks of KCH staged in Bst) ----
  const int nb4 = (np + 3) / 4;
  const int nblk = nb4 * (nb4 + 1) / 2;
  float acc[GB][16];
#pragma unroll
  for (int u = 0; u < GB; ++u)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[u][e] = 0.f;
  int bi[GB], bj[GB];
#pragma unroll
  for (int u = 0; u < GB; ++u) {
    int b = tid + u * BT;
    bi[u] = -1;
    bj[u] = -1;
    if (b < nblk) {
      // unrank b -> (i, j) with i <= j in row-major upper triangle
      int i = 0, rem = b;
      while (rem >= nb4 - i) { rem -= nb4 - i; ++i; }
      bi[u] = i;
      bj[u] = i + rem;
    }
  }
  for (long long k0 = 0; k0 < d; k0 += KCH) {
    __syncthreads();
    for (int idx = tid; idx < np * KCH; idx += BT) {
      const int r = idx / KCH, k = idx % KCH;
      Bst[k * (BMAX_L + 4) + r] =
          (r < nrows && k0 + k < d) ? buf[(long long)r * ldb + k0 + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      if (bi[u] < 0) continue;
      const int i0 = bi[u] * 4, j0 = bj[u] * 4;
#pragma unroll 8
      for (int k = 0; k < KCH; ++k) {
        const float4 a4 = *reinterpret_cast<const float4*>(&Bst[k * (BMAX_L + 4) + i0]);
        const float4 b4 = *reinterpret_cast<const float4*>(&Bst[k * (BMAX_L + 4) + j0]);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w};
        const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[u][x * 4 + y] = fmaf(av[x], bv[y], acc[u][x * 4 + y]);
      }
    }
  }
  __syncthreads();
  // write G (both triangles) into A with stride ld, zero padding
  for (int idx = tid; idx < nz * ld; idx += BT) A[idx] = 0.f;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < GB; ++u) {
    if (bi[u] < 0) continue;
    const int i0 = bi[u] * 4, j0 = bj[u] * 4;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int i = i0 + x, j = j0 + y;
        if (i < nrows && j < nrows) {
          A[i * ld + j] = acc[u][x * 4 + y];
          A[j * ld + i] = acc[u][x * 4 + y];
        }
      }
  }
  __syncthreads();

  // ---- eigensolve (scaled by the largest diagonal entry) ----
  __shared__ float s_max;
  if (tid == 0) s_max = 0.f;
  __syncthreads();
  float dm = 0.f;
  for (int i = tid; i < nrows; i += BT) dm = fmaxf(dm, fabsf(A[i * ld + i]));
  for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((tid & 31) == 0) atomicMax(reinterpret_cast<int*>(&s_max), __float_as_int(dm));
  __syncthreads();
  const float smax = eig_pow2_scale(s_max);
  const float inv = 1.f / smax;  // exact: smax is a power of two
  for (int idx = tid; idx < nz * ld; idx += BT) A[idx] *= inv;
  __syncthreads();
  if (tri) {
    EigArgs a;
    memset(&a, 0, sizeof(a));
    a.n = nrows;
    a.ell = S.ell;
    a.variant = variant;
    a.alpha = alpha;
    a.ctr_in = cin;
    a.ctr_out = cout;
    a.wrot = Bst;  // written last, over the solve's dead scratch area
    a.ldr = np;
    a.max_sweeps = max_sweeps;
    a.row_mass = s_mass;
    if (ws != nullptr) {
      // Rayleigh-Ritz refinement with the scaled G (as for a single sketch)
      const int ldg = (nrows + 3) & ~3;
      float* gsave = ws;
      for (int idx = tid; idx < nrows * ldg; idx += BT) {
        const int i = idx / ldg, j = idx - i * ldg;
        gsave[idx] = (j < nrows) ? A[i * ld + j] : 0.f;
      }
      __syncthreads();
      a.gsave = gsave;
      a.ldgsave = ldg;
      a.uvec = ws + (size_t)BMAX_L * BMAX_L;
    }
    // step 1 of the solve works in the scratch area (272 n >= tri_rw_bytes(n, 8) bytes)
    tri_eig_shrink<TRI_NB, 4, 32, 1>(a, A, ld, nrows, smax > 0.f ? (double)smax : 1.0, smem + REG_A,
                                     smem + REG_A + tri_scratch_bytes(nrows, TRI_NB), smem + REG_A);
  } else {
  float* nrm = reinterpret_cast<float*>(sc);
  double* lam = reinterpret_cast<double*>(sc + BMAX_L * 4);
  double* mu = lam + BMAX_L;
  double* mup = mu + BMAX_L;
  double* scl = mup + BMAX_L;
  int* ord = reinterpret_cast<int*>(scl + BMAX_L);
  int* rrank = ord + BMAX_L;
  __syncthreads();
  int capped = 0;
  // block Jacobi: 16-lane groups hold two 4-column blocks in registers per
  // round (np <= 128: 16 groups, 2 float4 chunks per lane per column)
  const int sweeps = jacobi_blocks4_f32<16, 2>(A, ld, npb, nrm, max_sweeps, (float)tol, &capped);

  // ---- shrink + rotate matrix (rows 0..ell-2, stride np) into Bst ----
  EigArgs a;
  memset(&a, 0, sizeof(a));
  a.n = nrows;
  a.ell = S.ell;
  a.variant = variant;
  a.alpha = alpha;
  a.ctr_in = cin;
  a.ctr_out = cout;
  a.wrot = Bst;
  a.ldr = np;
  a.max_sweeps = max_sweeps;
  a.row_mass = s_mass;
  __syncthreads();
  eig_finish<float>(a, A, ld, nrows, np, sweeps, capped, smax > 0.f ? (double)smax : 1.0, lam,
                    mu, mup, scl, ord, rrank);
  }
  __syncthreads();

  // ---- rotate: out[r][c] = sum_i W[r][i] B[i][c], column chunks staged in A ----
  // The squares of every output are summed per (row, chunk column) in shared
  // memory behind the staging area (each slot has one owner: a fixed order).
  const int nout = S.ell - 1;
  float* W = Bst;
  float* sq = A + BMAX_L * RCH;  // nout x RCH sums of squares
  static_assert((size_t)(BMAX_L + BMAX_L / 2) * RCH * 4 <= REG_A, "rotate staging");
  for (int idx = tid; idx < nout * RCH; idx += BT) sq[idx] = 0.f;
  for (long long c0 = 0; c0 < d; c0 += RCH) {
    __syncthreads();
    for (int idx = tid; idx < nrows * RCH; idx += BT) {
      const int r = idx / RCH, c = idx % RCH;
      A[r * RCH + c] = (c0 + c < d) ? buf[(long long)r * ldb + c0 + c] : 0.f;
    }
    __syncthreads();
    for (int idx = tid; idx < nout * RCH; idx += BT) {
      const int r = idx / RCH, c = idx % RCH;
      float s0 = 0.f, s1 = 0.f;
      const float* wr = W + r * np;
      int i = 0;
      for (; i + 1 < nrows; i += 2) {
        s0 = fmaf(wr[i], A[i * RCH + c], s0);
        s1 = fmaf(wr[i + 1], A[(i + 1) * RCH + c], s1);
      }
      if (i < nrows) s0 = fmaf(wr[i], A[i * RCH + c], s0);
      if (c0 + c < d) {
        const float v = s0 + s1;
        out[(long long)r * ldo + c0 + c] = v;
        sq[idx] = fmaf(v, v, sq[idx]);
      }
    }
  }
  __syncthreads();
  // A row of S'V^T has norm sigma' exactly (Alg. 1): rescale each output row
  // to its FP64 target sigma'^2. This removes the error that the ratio
  // sigma'^2 / sigma^2 would otherwise amplify (large for SS merges into a
  // small direction).
  __shared__ float s_rscale[BMAX_L / 2];
  {
    const int lane = tid & 31, warp = tid >> 5;
    for (int r = warp; r < nout; r += BT / 32) {
      float t = 0.f;
      for (int c = lane; c < RCH; c += 32) t += sq[r * RCH + c];
      t = warp_sum(t);
      if (lane == 0) s_rscale[r] = (t > 0.f) ? (float)sqrt(s_mass[r] / (double)t) : 1.f;
    }
  }
  __syncthreads();
  for (long long idx = tid; idx < (long long)nout * d; idx += BT) {
    const int r = (int)(idx / d);
    const long long c = idx - (long long)r * d;
    out[(long long)r * ldo + c] *= s_rscale[r];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(BT, 2)
    batch_kernel(BatchSketch* __restrict__ sk, const BatchItem* __restrict__ items, int nitems,
                 int* __restrict__ next, int variant, double alpha, int max_sweeps,
                 double tol, float* ws_all, const int* __restrict__ nitems_dev) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ double s_rn[BMAX_L];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= (nitems_dev ? *nitems_dev : nitems)) break;
    const BatchItem item = items[it];
    BatchSketch S = sk[item.id];
    int m = S.m;
    long long i = 0;
    while (i < item.n) {
      const int c = (int)min((long long)(S.L - m), item.n - i);
      // ingest c rows: warp per row, FP64 row norms summed in row order
      for (int r = warp; r < c; r += BT / 32) {
        const long long src = (i + r) * item.ld;
        float* dst = S.buf + (long long)(m + r) * S.ldb;
        double acc = 0.0;
        for (long long k = lane; k < S.d; k += 32) {
          const double x = load_as_f64(item.rows, src + k, item.dtype);
          dst[k] = (float)x;
          acc = fma(x, x, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_rn[r] = acc;
      }
      __syncthreads();
      if (tid == 0) {
        double tot = S.ctr->norm_a2;
        for (int r = 0; r < c; ++r) tot += s_rn[r];
        S.ctr->norm_a2 = tot;
      }
      m += c;
      i += c;
      if (m == S.L) {
        __syncthreads();
        batch_reduce(S, S.L, S.buf, S.ldb, S.ctr, S.ctr, variant, alpha, max_sweeps, tol, smem,
                     ws_all ? ws_all + (size_t)blockIdx.x * BATCH_WS_FLOATS : nullptr);
        m = S.ell - 1;
      }
      __syncthreads();
    }
    if (tid == 0) sk[item.id].m = m;
  }
}

// Flush one sketch on a copy: rows 0..ell-2 of the reduction of its m pending
// rows go to out; counters to cout. One CTA.
__global__ void __launch_bounds__(BT, 1)
    batch_flush_kernel(const BatchSketch* __restrict__ sk, int id, float* out, long long ldo,
                       DevCounters* cout, int variant, double alpha, int max_sweeps, double tol) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BatchSketch S = sk[id];
  batch_reduce(S, S.m, out, ldo, S.ctr, cout, variant, alpha, max_sweeps, tol, smem);
}

// Every sketch of the batch, flushed on a copy like fd_sketch, into one
// device arena: sketch id at out + offs[id] as ell_id x d_id rows.
__global__ void __launch_bounds__(BT, 1)
    batch_flush_all_kernel(const BatchSketch* __restrict__ sk, int count, float* out,
                           const long long* __restrict__ offs, DevCounters* fctr, int variant,
                           double alpha, int max_sweeps, double tol) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (int id = blockIdx.x; id < count; id += gridDim.x) {
    const BatchSketch S = sk[id];
    float* o = out + offs[id];
    int valid;
    if (S.m > S.ell - 1) {
      batch_reduce(S, S.m, o, S.d, S.ctr, fctr + id, variant, alpha, max_sweeps, tol, smem);
      valid = S.ell - 1;
    } else {
      for (long long idx = threadIdx.x; idx < (long long)S.m * S.d; idx += BT) {
        const long long r = idx / S.d, c = idx % S.d;
        o[idx] = S.buf[r * S.ldb + c];
      }
      if (threadIdx.x == 0) fctr[id] = *S.ctr;
      valid = S.m;
    }
    for (long long idx = (long long)valid * S.d + threadIdx.x; idx < (long long)S.ell * S.d; idx += BT)
      o[idx] = 0.f;
    __syncthreads();
  }
}

}  // namespace

}  // namespace fdk

using namespace fdk;

struct fd_batch_state {
  int count = 0, variant = 0, prec = 0;
  double alpha = 1.0;
  cudaStream_t st = nullptr;
  std::vector<int64_t> d;
  std::vector<int32_t> ell;
  std::vector<int> m;          // pending rows per sketch (host mirror)
  std::vector<int64_t> nseen;
  std::vector<BatchSketch> hs;
  BatchSketch* dsk = nullptr;
  float* arena = nullptr;      // all buffers
  DevCounters* ctrs = nullptr;
  DevCounters* ctr_flush = nullptr;
  float* flush_out = nullptr;  // largest ell x ldb
  BatchItem* ditems = nullptr;
  int items_cap = 0;
  int* next = nullptr;
  int nsm = 0;
  int max_sweeps = 30;
  long long* doffs = nullptr;     // device copy of the sketch_all offsets
  DevCounters* fctr_all = nullptr;
  float* ws = nullptr;            // 2 * nsm CTA workspaces (BATCH_WS_FLOATS each)
  // The CUDA graph of an append: the queue-counter reset and the persistent
  // launch (2 x SMs CTAs; those beyond the work exit at once), with the item
  // table and its length read from fixed device buffers. Captured once, on
  // the first append, and relaunched for every append; the items are copied
  // in from pinned host memory before each launch.
  cudaStream_t cap_st = nullptr;
  cudaGraphExec_t gexec = nullptr;
  BatchItem* gitems = nullptr;    // device, count entries
  BatchItem* hitems = nullptr;    // pinned, count entries
  int* dcount = nullptr;          // device item count
  int* hcount = nullptr;          // pinned
  cudaEvent_t ev_copy = nullptr;  // the last append's copies have been read
  bool copy_pending = false;
  bool graph_off = false;
  long long graph_launches = 0;
};

static int batch_fail(cudaError_t e, const char* w) {
  set_cuda_error(e, w);
  return e == cudaErrorMemoryAllocation ? FD_ENOMEM : FD_ECUDA;
}

extern "C" int fd_batch_destroy(fd_batch_state* b);

extern "C" int fd_batch_create(int32_t count, const int64_t* d, const int32_t* ell, int32_t variant,
                               double alpha, int32_t prec, void* stream, fd_batch_state** out) {
  if (!out || count < 1 || !d || !ell) return FD_EINVAL;
  *out = nullptr;
  if (variant < FD_VAR_FD || variant > FD_VAR_ISVD) return FD_EINVAL;
  if (variant == FD_VAR_PFD && !(alpha > 0.0 && alpha <= 1.0)) return FD_EINVAL;
  if (prec != FD_PREC_FP32) return FD_EINVAL;
  for (int i = 0; i < count; ++i)
    if (d[i] < 1 || ell[i] < 2 || 2 * ell[i] > BMAX_L) return FD_EINVAL;
  fd_batch_state* b = new (std::nothrow) fd_batch_state();
  if (!b) return FD_ENOMEM;
  b->count = count;
  b->variant = variant;
  b->alpha = variant == FD_VAR_PFD ? alpha : 1.0;
  b->prec = prec;
  b->st = reinterpret_cast<cudaStream_t>(stream);
  b->d.assign(d, d + count);
  b->ell.assign(ell, ell + count);
  b->m.assign(count, 0);
  b->nseen.assign(count, 0);
  size_t total = 0, maxsk = 0;
  std::vector<size_t> off(count);
  for (int i = 0; i < count; ++i) {
    const int64_t ldb = (d[i] + 3) / 4 * 4;
    off[i] = total;
    total += (size_t)2 * ell[i] * ldb;
    maxsk = std::max(maxsk, (size_t)ell[i] * ldb);
  }
  cudaError_t e = cudaMalloc(&b->arena, total * sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->arena, 0, total * sizeof(float), b->st);
  if (e == cudaSuccess) e = cudaMalloc(&b->ctrs, (size_t)count * sizeof(DevCounters));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ctrs, 0, (size_t)count * sizeof(DevCounters), b->st);
  if (e == cudaSuccess) e = cudaMalloc(&b->ctr_flush, sizeof(DevCounters));
  if (e == cudaSuccess) e = cudaMalloc(&b->flush_out, maxsk * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b->dsk, (size_t)count * sizeof(BatchSketch));
  if (e == cudaSuccess) e = cudaMalloc(&b->next, sizeof(int));
  if (e != cudaSuccess) {
    fd_batch_destroy(b);
    return batch_fail(e, "fd_batch_create alloc");
  }
  b->hs.resize(count);
  for (int i = 0; i < count; ++i) {
    BatchSketch& s = b->hs[i];
    s.d = d[i];
    s.ldb = (d[i] + 3) / 4 * 4;
    s.ell = ell[i];
    s.L = 2 * ell[i];
    s.m = 0;
    s.pad = 0;
    s.buf = b->arena + off[i];
    s.ctr = b->ctrs + i;
  }
  e = cudaMemcpyAsync(b->dsk, b->hs.data(), (size_t)count * sizeof(BatchSketch),
                      cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BATCH_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_flush_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BATCH_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_flush_all_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BATCH_SMEM);
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaMalloc(&b->ws, (size_t)2 * b->nsm * BATCH_WS_FLOATS * sizeof(float));
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) {
    fd_batch_destroy(b);
    return batch_fail(e, "fd_batch_create setup");
  }
  *out = b;
  return FD_OK;
}

// Capture the append graph (once per batch). False if any step fails; the
// caller then launches directly.
static bool batch_graph_build(fd_batch_state* b) {
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->gitems, (size_t)b->count * sizeof(BatchItem));
  if (e == cudaSuccess) e = cudaMalloc(&b->dcount, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->hitems, (size_t)b->count * sizeof(BatchItem));
  if (e == cudaSuccess) e = cudaMallocHost(&b->hcount, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_copy, cudaEventDisableTiming);
  if (e != cudaSuccess) return false;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return false;
  const double eps = 1.1920928955078125e-07;
  cudaError_t e1 = cudaMemsetAsync(b->next, 0, sizeof(int), b->cap_st);
  if (e1 == cudaSuccess) {
    batch_kernel<<<2 * b->nsm, BT, BATCH_SMEM, b->cap_st>>>(
        b->dsk, b->gitems, 0, b->next, b->variant, b->alpha, b->max_sweeps,
        4.0 * eps * std::sqrt((double)BMAX_L), b->ws, b->dcount);
    e1 = cudaGetLastError();
  }
  e = cudaStreamEndCapture(b->cap_st, &g);
  if (e1 != cudaSuccess || e != cudaSuccess || g == nullptr) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  e = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->gexec = nullptr;
    cudaGetLastError();
    return false;
  }
  return true;
}

extern "C" int fd_batch_uses_graph(fd_batch_state* b, int64_t* launches) {
  if (!b) return FD_EINVAL;
  if (launches) *launches = b->graph_launches;
  return (b->gexec != nullptr && !b->graph_off) ? 1 : 0;
}

extern "C" int fd_batch_append(fd_batch_state* b, const fd_work_t* items, int32_t n_items) {
  if (!b || (n_items > 0 && !items) || n_items < 0) return FD_EINVAL;
  if (n_items == 0) return FD_OK;
  std::vector<int> seen(b->count, 0);
  std::vector<BatchItem> hi(n_items);
  std::vector<double> cost(n_items);
  for (int i = 0; i < n_items; ++i) {
    const fd_work_t& w = items[i];
    if (w.id < 0 || w.id >= b->count || seen[w.id] || w.n < 0 || !w.rows ||
        w.ld < b->d[w.id] || (w.dtype != FD_F32 && w.dtype != FD_BF16 && w.dtype != FD_F64))
      return FD_EINVAL;
    seen[w.id] = 1;
    hi[i] = BatchItem{w.id, w.dtype, w.rows, w.n, w.ld};
    const double L = 2.0 * b->ell[w.id];
    // reductions x (eigensolve ~ L^3 + Gram and rotate ~ L^2 d)
    cost[i] = (double)w.n / (b->ell[w.id] + 1) * (L * L * L * 2.0 + L * L * b->d[w.id]);
  }
  // longest first
  std::vector<int> order(n_items);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<BatchItem> sorted(n_items);
  for (int i = 0; i < n_items; ++i) sorted[i] = hi[order[i]];
  if (!b->graph_off && b->gexec == nullptr && !batch_graph_build(b)) b->graph_off = true;
  if (!b->graph_off) {
    // the previous append's item copy must have been read before the pinned
    // table is refilled
    cudaError_t e = b->copy_pending ? cudaEventSynchronize(b->ev_copy) : cudaSuccess;
    if (e != cudaSuccess) return batch_fail(e, "batch item copy wait");
    std::memcpy(b->hitems, sorted.data(), (size_t)n_items * sizeof(BatchItem));
    *b->hcount = n_items;
    e = cudaMemcpyAsync(b->gitems, b->hitems, (size_t)n_items * sizeof(BatchItem),
                        cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->dcount, b->hcount, sizeof(int), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_copy, b->st);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->gexec, b->st);
    if (e != cudaSuccess) return batch_fail(e, "batch graph launch");
    b->copy_pending = true;
    ++b->graph_launches;
  } else {
    if (n_items > b->items_cap) {
      cudaFree(b->ditems);
      b->ditems = nullptr;
      cudaError_t e = cudaMalloc(&b->ditems, (size_t)n_items * sizeof(BatchItem));
      if (e != cudaSuccess) return batch_fail(e, "batch items");
      b->items_cap = n_items;
    }
    cudaError_t e = cudaMemcpyAsync(b->ditems, sorted.data(), (size_t)n_items * sizeof(BatchItem),
                                    cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->next, 0, sizeof(int), b->st);
    if (e != cudaSuccess) return batch_fail(e, "batch items copy");
    const int grid = std::min(n_items, 2 * b->nsm);
    const double eps = 1.1920928955078125e-07;
    batch_kernel<<<grid, BT, BATCH_SMEM, b->st>>>(b->dsk, b->ditems, n_items, b->next, b->variant,
                                                  b->alpha, b->max_sweeps,
                                                  4.0 * eps * std::sqrt((double)BMAX_L), b->ws,
                                                  nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return batch_fail(e, "batch_kernel");
  }
  for (int i = 0; i < n_items; ++i) {
    const int id = items[i].id;
    const int L = 2 * b->ell[id];
    int64_t m = b->m[id] + items[i].n;
    if (m >= L) m = (b->ell[id] - 1) + (m - L) % (b->ell[id] + 1);
    b->m[id] = (int)m;
    b->nseen[id] += items[i].n;
  }
  return FD_OK;
}

extern "C" int fd_batch_sketch(fd_batch_state* b, int32_t id, void* out, int32_t dtype,
                               int32_t out_on_device) {
  if (!b || id < 0 || id >= b->count || !out || (dtype != FD_F32 && dtype != FD_F64))
    return FD_EINVAL;
  const BatchSketch& s = b->hs[id];
  const int ell = s.ell;
  const void* src;
  int valid;
  cudaError_t e;
  if (b->m[id] > ell - 1) {
    const double eps = 1.1920928955078125e-07;
    batch_flush_kernel<<<1, BT, BATCH_SMEM, b->st>>>(b->dsk, id, b->flush_out, s.ldb,
                                                     b->ctr_flush, b->variant, b->alpha,
                                                     b->max_sweeps,
                                                     4.0 * eps * std::sqrt((double)BMAX_L));
    e = cudaGetLastError();
    if (e != cudaSuccess) return batch_fail(e, "batch_flush_kernel");
    src = b->flush_out;
    valid = ell - 1;
  } else {
    e = cudaMemcpyAsync(b->ctr_flush, b->ctrs + id, sizeof(DevCounters), cudaMemcpyDeviceToDevice,
                        b->st);
    if (e != cudaSuccess) return batch_fail(e, "batch counters");
    src = s.buf;
    valid = b->m[id];
  }
  void* dst = out;
  void* tmp = nullptr;
  const size_t ob = (size_t)ell * s.d * (dtype == FD_F64 ? 8 : 4);
  if (!out_on_device) {
    e = cudaMalloc(&tmp, ob);
    if (e != cudaSuccess) return batch_fail(e, "batch sketch tmp");
    dst = tmp;
  }
  e = launch_norm_b2(src, 0, s.ldb, valid, s.d, b->ctr_flush, b->st);
  if (e == cudaSuccess)
    e = launch_convert_out(src, 0, s.ldb, ell, s.d, dst, dtype == FD_F64, s.d, valid, b->st);
  if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(out, tmp, ob, cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess && tmp) e = cudaStreamSynchronize(b->st);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return batch_fail(e, "batch sketch out");
  return FD_OK;
}

extern "C" int fd_batch_sketch_all(fd_batch_state* b, float* out, const int64_t* offsets) {
  if (!b || !out || !offsets) return FD_EINVAL;
  cudaError_t e = cudaSuccess;
  if (!b->doffs) {
    e = cudaMalloc(&b->doffs, (size_t)b->count * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->fctr_all, (size_t)b->count * sizeof(DevCounters));
    if (e != cudaSuccess) return batch_fail(e, "sketch_all alloc");
  }
  e = cudaMemcpyAsync(b->doffs, offsets, (size_t)b->count * sizeof(long long),
                      cudaMemcpyHostToDevice, b->st);
  if (e != cudaSuccess) return batch_fail(e, "sketch_all offsets");
  const double eps = 1.1920928955078125e-07;
  const int grid = std::min(b->count, 2 * b->nsm);
  batch_flush_all_kernel<<<grid, BT, BATCH_SMEM, b->st>>>(b->dsk, b->count, out, b->doffs,
                                                          b->fctr_all, b->variant, b->alpha,
                                                          b->max_sweeps,
                                                          4.0 * eps * std::sqrt((double)BMAX_L));
  e = cudaGetLastError();
  if (e != cudaSuccess) return batch_fail(e, "batch_flush_all_kernel");
  return FD_OK;
}

extern "C" int fd_batch_stats(fd_batch_state* b, int32_t id, fd_stats_t* s) {
  if (!b || id < 0 || id >= b->count || !s) return FD_EINVAL;
  DevCounters c[2];
  cudaError_t e = cudaMemcpyAsync(&c[0], b->ctrs + id, sizeof(DevCounters), cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&c[1], b->ctr_flush, sizeof(DevCounters), cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return batch_fail(e, "batch stats");
  std::memset(s, 0, sizeof(*s));
  s->d = b->d[id];
  s->ell = b->ell[id];
  s->variant = b->variant;
  s->alpha = b->alpha;
  s->prec = b->prec;
  s->pending = b->m[id];
  s->n_seen = b->nseen[id];
  s->reductions = c[0].reductions;
  s->noconv = c[0].noconv;
  s->eig_fallbacks = c[0].fallbacks;
  s->norm_a2 = c[0].norm_a2;
  s->sum_delta = c[0].sum_delta;
  s->last_delta = c[0].last_delta;
  s->removed = c[0].removed;
  s->max_sweeps = c[0].max_sweeps;
  // flush totals refer to the latest fd_batch_sketch call
  s->sketch_sum_delta = c[1].sum_delta;
  s->sketch_removed = c[1].removed;
  s->sketch_norm_b2 = c[1].norm_b2;
  return FD_OK;
}

extern "C" int fd_batch_reset(fd_batch_state* b) {
  if (!b) return FD_EINVAL;
  size_t total = 0;
  for (int i = 0; i < b->count; ++i) total += (size_t)2 * b->ell[i] * ((b->d[i] + 3) / 4 * 4);
  cudaError_t e = cudaMemsetAsync(b->arena, 0, total * sizeof(float), b->st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->ctrs, 0, (size_t)b->count * sizeof(DevCounters), b->st);
  for (auto& s : b->hs) s.m = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->dsk, b->hs.data(), (size_t)b->count * sizeof(BatchSketch),
                        cudaMemcpyHostToDevice, b->st);
  if (e != cudaSuccess) return batch_fail(e, "batch reset");
  std::fill(b->m.begin(), b->m.end(), 0);
  std::fill(b->nseen.begin(), b->nseen.end(), 0);
  return FD_OK;
}

extern "C" int fd_batch_destroy(fd_batch_state* b) {
  if (!b) return FD_EINVAL;
  if (b->st) cudaStreamSynchronize(b->st);
  cudaFree(b->arena);
  cudaFree(b->ctrs);
  cudaFree(b->ctr_flush);
  cudaFree(b->flush_out);
  cudaFree(b->dsk);
  cudaFree(b->ditems);
  cudaFree(b->next);
  cudaFree(b->doffs);
  cudaFree(b->fctr_all);
  cudaFree(b->ws);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  cudaFree(b->gitems);
  cudaFree(b->dcount);
  if (b->hitems) cudaFreeHost(b->hitems);
  if (b->hcount) cudaFreeHost(b->hcount);
  if (b->ev_copy) cudaEventDestroy(b->ev_copy);
  delete b;
  return FD_OK;
}

// ===========================================================================
// Serving: continuous batching of append requests over many live sketches.
//
// Requests (sketch id, a block of rows) are admitted into a pinned host ring
// and a device ring of the same size -- the device-memory budget. A native
// engine thread repeatedly takes every admitted request whose sketch is not
// already on the GPU (at most one per sketch per launch), copies their rows
// to the device ring, and launches one batched update over all of them on the
// next of several streams, so launches overlap on the device while sketches
// stay consistent (a sketch is in at most one launch at a time). A launch's
// completion releases its ring space and completes its requests; latency is
// arrival (submit) to completion.
// ===========================================================================
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

namespace {

struct ServeReq {
  int64_t ticket;
  int id;
  int64_t n;
  size_t off;      // byte offset in the rings
  size_t bytes;
  double t_submit;
};

struct ServeLaunch {
  cudaEvent_t ev;
  std::vector<ServeReq> reqs;
  int stream;
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct fd_server_state {
  fd_batch_state* b = nullptr;
  int64_t d = 0;
  int ell = 0;
  size_t cap = 0;           // ring bytes
  char* hring = nullptr;    // pinned
  char* dring = nullptr;
  size_t head = 0;          // next free byte; the oldest live allocation marks the tail
  std::deque<std::pair<size_t, size_t>> allocs;  // (offset, bytes) in allocation order
  std::vector<char> released;                    // per outstanding allocation: done?
  int nstreams = 2;
  std::vector<cudaStream_t> streams;
  std::vector<BatchItem*> ditems;   // per stream
  std::vector<BatchItem*> hitems;   // pinned, per stream
  std::vector<int*> dnext;          // per stream
  std::vector<float*> ws;           // per stream: 2 * nsm CTA workspaces
  std::vector<char> busy_stream;
  int next_stream = 0;
  std::vector<char> inflight;       // per sketch
  int in_transit = 0;               // requests taken from pending, not yet in launches
  std::deque<ServeReq> pending;
  std::deque<ServeLaunch> launches;
  std::vector<std::pair<int64_t, double>> done;  // (ticket, latency s)
  std::mutex mu;
  std::condition_variable cv;
  std::thread engine;
  std::atomic<bool> stop{false};
  int64_t next_ticket = 1;
  int64_t admitted = 0, busy = 0, launched = 0, rows_done = 0;
  int err = 0;
};

static void serve_release_locked(fd_server_state* s) {
  // free ring space from the front, in allocation order
  while (!s->allocs.empty() && s->released.front()) {
    s->allocs.pop_front();
    s->released.erase(s->released.begin());
  }
  if (s->allocs.empty()) s->head = 0;
}

// Contiguous space of `bytes` in the ring, FIFO order; false when full.
static bool serve_ring_alloc_locked(fd_server_state* s, size_t bytes, size_t* off) {
  if (s->allocs.empty()) {
    if (bytes > s->cap) return false;
    *off = 0;
    s->head = bytes;
    return true;
  }
  const size_t tail = s->allocs.front().first;
  if (s->head > tail) {            // live bytes in [tail, head)
    if (s->cap - s->head >= bytes) { *off = s->head; s->head += bytes; return true; }
    if (tail >= bytes) { *off = 0; s->head = bytes; return true; }
    return false;
  }
  if (s->head < tail) {            // live bytes in [tail, cap) and [0, head)
    if (tail - s->head >= bytes) { *off = s->head; s->head += bytes; return true; }
    return false;
  }
  return false;                    // head == tail with live allocations: full
}

static void serve_engine(fd_server_state* s) {
  const double eps = 1.1920928955078125e-07;
  while (!s->stop.load()) {
    std::vector<ServeReq> take;
    int st = -1;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // completions
      for (auto it = s->launches.begin(); it != s->launches.end();) {
        if (cudaEventQuery(it->ev) == cudaSuccess) {
          const double t = now_s();
          for (auto& r : it->reqs) {
            s->done.emplace_back(r.ticket, t - r.t_submit);
            s->inflight[r.id] = 0;
            s->rows_done += r.n;
            for (size_t k = 0; k < s->allocs.size(); ++k)
              if (s->allocs[k].first == r.off && s->allocs[k].second == r.bytes) { s->released[k] = 1; break; }
          }
          s->busy_stream[it->stream] = 0;
          cudaEventDestroy(it->ev);
          it = s->launches.erase(it);
        } else {
          ++it;
        }
      }
      serve_release_locked(s);
      // a free stream?
      for (int k = 0; k < s->nstreams; ++k) {
        const int c = (s->next_stream + k) % s->nstreams;
        if (!s->busy_stream[c]) { st = c; break; }
      }
      if (st >= 0) {
        std::vector<char> picked(s->inflight.size(), 0);
        for (auto it = s->pending.begin(); it != s->pending.end();) {
          if (!s->inflight[it->id] && !picked[it->id]) {
            picked[it->id] = 1;
            take.push_back(*it);
            it = s->pending.erase(it);
          } else {
            ++it;
          }
        }
        for (auto& r : take) s->inflight[r.id] = 1;
        if (!take.empty()) {
          s->busy_stream[st] = 1;
          s->next_stream = (st + 1) % s->nstreams;
          s->in_transit += (int)take.size();
        }
      }
      if (take.empty()) {
        s->cv.wait_for(lk, std::chrono::microseconds(20));
        continue;
      }
    }
    // launch outside the lock
    cudaStream_t stream = s->streams[st];
    BatchItem* hi = s->hitems[st];
    const int ns = (int)take.size();
    for (int i = 0; i < ns; ++i) {
      const ServeReq& r = take[i];
      cudaMemcpyAsync(s->dring + r.off, s->hring + r.off, r.bytes, cudaMemcpyHostToDevice, stream);
      hi[i] = BatchItem{r.id, FD_F32, s->dring + r.off, r.n, s->d};
    }
    cudaMemcpyAsync(s->ditems[st], hi, (size_t)ns * sizeof(BatchItem), cudaMemcpyHostToDevice, stream);
    cudaMemsetAsync(s->dnext[st], 0, sizeof(int), stream);
    const int grid = std::min(ns, 2 * s->b->nsm);
    batch_kernel<<<grid, BT, BATCH_SMEM, stream>>>(s->b->dsk, s->ditems[st], ns, s->dnext[st],
                                                   s->b->variant, s->b->alpha, s->b->max_sweeps,
                                                   4.0 * eps * std::sqrt((double)BMAX_L), s->ws[st],
                                                   nullptr);
    ServeLaunch L;
    cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
    cudaEventRecord(L.ev, stream);
    L.reqs = std::move(take);
    L.stream = st;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& r : L.reqs) {
        int64_t m = s->b->m[r.id] + r.n;
        const int Lr = 2 * s->b->ell[r.id];
        if (m >= Lr) m = (s->b->ell[r.id] - 1) + (m - Lr) % (s->b->ell[r.id] + 1);
        s->b->m[r.id] = (int)m;
        s->b->nseen[r.id] += r.n;
      }
      s->launched += 1;
      s->in_transit -= (int)L.reqs.size();
      s->launches.push_back(std::move(L));
    }
    if (cudaGetLastError() != cudaSuccess) s->err = 1;
  }
}

extern "C" int fd_serve_destroy(fd_server_state* s);

extern "C" int fd_serve_create(int32_t count, int64_t d, int32_t ell, int32_t variant,
                               double alpha, int64_t budget_bytes, int32_t nstreams,
                               fd_server_state** out) {
  if (!out || count < 1 || d < 1 || budget_bytes < d * 4 || nstreams < 1 || nstreams > 8)
    return FD_EINVAL;
  *out = nullptr;
  std::vector<int64_t> ds(count, d);
  std::vector<int32_t> es(count, ell);
  fd_server_state* s = new (std::nothrow) fd_server_state();
  if (!s) return FD_ENOMEM;
  int rc = fd_batch_create(count, ds.data(), es.data(), variant, alpha, FD_PREC_FP32, nullptr, &s->b);
  if (rc != FD_OK) { delete s; return rc; }
  s->d = d;
  s->ell = ell;
  s->cap = (size_t)budget_bytes;
  s->nstreams = nstreams;
  cudaError_t e = cudaMallocHost(&s->hring, s->cap);
  if (e == cudaSuccess) e = cudaMalloc(&s->dring, s->cap);
  s->streams.resize(nstreams);
  s->ditems.resize(nstreams);
  s->hitems.resize(nstreams);
  s->dnext.resize(nstreams);
  s->ws.assign(nstreams, nullptr);
  s->busy_stream.assign(nstreams, 0);
  for (int k = 0; k < nstreams && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->ditems[k], (size_t)count * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMallocHost(&s->hitems[k], (size_t)count * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMalloc(&s->dnext[k], sizeof(int));
    if (e == cudaSuccess)
      e = cudaMalloc(&s->ws[k], (size_t)2 * s->b->nsm * BATCH_WS_FLOATS * sizeof(float));
  }
  if (e != cudaSuccess) {
    set_cuda_error(e, "fd_serve_create");
    fd_serve_destroy(s);
    return FD_ENOMEM;
  }
  s->inflight.assign(count, 0);
  s->engine = std::thread(serve_engine, s);
  *out = s;
  return FD_OK;
}

extern "C" int fd_serve_submit(fd_server_state* s, int32_t id, const float* rows, int64_t n,
                               int64_t* ticket) {
  if (!s || !rows || n < 1 || !ticket || id < 0 || id >= s->b->count) return FD_EINVAL;
  const size_t bytes = (size_t)n * s->d * 4;
  if (bytes > s->cap) return FD_EINVAL;
  size_t off = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!serve_ring_alloc_locked(s, bytes, &off)) { s->busy += 1; return FD_EBUSY; }
    s->allocs.emplace_back(off, bytes);
    s->released.push_back(0);
    *ticket = s->next_ticket++;
    s->admitted += 1;
  }
  std::memcpy(s->hring + off, rows, bytes);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending.push_back(ServeReq{*ticket, id, n, off, bytes, now_s()});
  }
  s->cv.notify_one();
  return FD_OK;
}

extern "C" int fd_serve_poll(fd_server_state* s, int64_t* tickets, double* latency_s, int32_t max,
                             int32_t* count) {
  if (!s || !count || max < 0 || (max > 0 && (!tickets || !latency_s))) return FD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  const int k = (int)std::min<size_t>((size_t)max, s->done.size());
  for (int i = 0; i < k; ++i) {
    tickets[i] = s->done[i].first;
    latency_s[i] = s->done[i].second;
  }
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *count = k;
  return s->err ? FD_ECUDA : FD_OK;
}

extern "C" int fd_serve_drain(fd_server_state* s) {
  if (!s) return FD_EINVAL;
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->pending.empty() && s->launches.empty() && s->in_transit == 0) break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  return s->err ? FD_ECUDA : FD_OK;
}

extern "C" int fd_serve_sketch(fd_server_state* s, int32_t id, void* out, int32_t dtype) {
  if (!s) return FD_EINVAL;
  int rc = fd_serve_drain(s);
  if (rc != FD_OK) return rc;
  cudaDeviceSynchronize();
  return fd_batch_sketch(s->b, id, out, dtype, 0);
}

extern "C" int fd_serve_counters(fd_server_state* s, int64_t* admitted, int64_t* busy,
                                 int64_t* launches, int64_t* rows_done) {
  if (!s) return FD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (admitted) *admitted = s->admitted;
  if (busy) *busy = s->busy;
  if (launches) *launches = s->launched;
  if (rows_done) *rows_done = s->rows_done;
  return FD_OK;
}

extern "C" int fd_serve_destroy(fd_server_state* s) {
  if (!s) return FD_EINVAL;
  if (s->engine.joinable()) {
    fd_serve_drain(s);
    s->stop.store(true);
    s->cv.notify_all();
    s->engine.join();
  }
  for (auto& L : s->launches) cudaEventDestroy(L.ev);
  for (int k = 0; k < (int)s->streams.size(); ++k) {
    if (s->streams[k]) { cudaStreamSynchronize(s->streams[k]); cudaStreamDestroy(s->streams[k]); }
    cudaFree(s->ditems[k]);
    if (s->hitems[k]) cudaFreeHost(s->hitems[k]);
    cudaFree(s->dnext[k]);
    cudaFree(s->ws[k]);
  }
  if (s->hring) cudaFreeHost(s->hring);
  cudaFree(s->dring);
  if (s->b) fd_batch_destroy(s->b);
  delete s;
  return FD_OK;
}
