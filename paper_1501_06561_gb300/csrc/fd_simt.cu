// CUDA-core kernels of the buffered FD reduction: row ingest, the plain
// FP32/FP64 Gram and rotate, and the fused one-CTA eigensolve + shrink.
//
// One reduction of Algorithm 1 (Sec. 2.3) on a buffer B of n rows is
//   G = B B^T                         (gram_simt_kernel or the tcgen05 Gram)
//   G = U diag(sigma^2) U^T           (eig_tri_kernel: FP32 tridiagonal solve of
//                                      a full buffer; eig_fast_kernel and
//                                      eig_shrink_kernel: one-sided Jacobi for
//                                      a flush and for FP64)
//   sigma' = ReduceRank(sigma)        (same kernel, FP64)
//   B' = diag(sigma'/sigma) U^T B     (rotate_simt_kernel or the tcgen05 rotate)
// which equals B' = S' V^T because U^T B = S V^T for the SVD B = U S V^T.
#include <cfloat>
#include <cmath>
#include <cstdio>

#include "fd_internal.cuh"
#include "fd_jacobi.cuh"
#include "fd_eig.cuh"
#include "fd_tridiag.cuh"

namespace fdk {

// ---------------------------------------------------------------------------
// Row ingest: copy rows into the buffer (Algorithm 1, "insert a_i into a zero
// valued row") and add sum ||a_i||^2 (Sec. 1.1) to ||A||_F^2 in FP64.
// One block per row; the last block to finish sums the per-row norms in row
// order, so the FP64 total is deterministic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double load_elem(const void* p, int64_t idx, int dtype) {
  if (dtype == FD_F32) return (double)reinterpret_cast<const float*>(p)[idx];
  if (dtype == FD_F64) return reinterpret_cast<const double*>(p)[idx];
  const unsigned short raw = reinterpret_cast<const unsigned short*>(p)[idx];
  return (double)__uint_as_float(((unsigned int)raw) << 16);
}

__global__ void ingest_kernel(const void* __restrict__ src, int64_t ld, int dtype,
                              void* __restrict__ dst, int64_t ldd, int dst_f64, int64_t d,
                              double* __restrict__ rownorm, DevCounters* __restrict__ ctr,
                              __nv_bfloat16* rm_hi, __nv_bfloat16* rm_lo2, int64_t ld_rm,
                              __nv_bfloat16* cm_hi, __nv_bfloat16* cm_lo, int64_t ld_cm,
                              int row0, int nrows, double* __restrict__ slot_n2) {
  const int r = blockIdx.x;
  const void* srow = src;
  double acc = 0.0;
  float acc2 = 0.0f;  // squared norm of the stored hi + lo pair
  for (int64_t k = threadIdx.x; k < d; k += blockDim.x) {
    const double x = load_elem(srow, (int64_t)r * ld + k, dtype);
    acc += x * x;
    if (dst != nullptr) {
      if (dst_f64) reinterpret_cast<double*>(dst)[(int64_t)r * ldd + k] = x;
      else reinterpret_cast<float*>(dst)[(int64_t)r * ldd + k] = (float)x;
    }
    if (rm_hi != nullptr) {
      const float xf = (float)x;
      const __nv_bfloat16 hi = __float2bfloat16_rn(xf);
      const float rem = xf - __bfloat162float(hi);   // exact in FP32
      const __nv_bfloat16 lo = __float2bfloat16_rn(rem);
      const int64_t row = row0 + r;
      rm_hi[row * ld_rm + k] = hi;
      rm_lo2[row * ld_rm + k] = __float2bfloat16_rn(2.0f * __bfloat162float(lo));
      cm_hi[k * ld_cm + row] = hi;
      cm_lo[k * ld_cm + row] = lo;
      const float y = __bfloat162float(hi) + __bfloat162float(lo);
      acc2 = fmaf(y, y, acc2);
    }
  }
  __shared__ double red[32], red2[32];
  double a2 = (double)acc2;
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = acc; red2[threadIdx.x >> 5] = a2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, s2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s += red[w]; s2 += red2[w]; }
    if (slot_n2 != nullptr) slot_n2[row0 + r] = s2;
    rownorm[r] = s;
    __threadfence();
    const unsigned int t = atomicAdd(&ctr->ingest_ticket, 1u);
    if (t == (unsigned int)nrows - 1) {
      __threadfence();
      double tot = ctr->norm_a2;
      for (int i = 0; i < nrows; ++i) tot += ((volatile double*)rownorm)[i];
      ctr->norm_a2 = tot;
      ctr->ingest_ticket = 0u;
    }
  }
}

cudaError_t launch_ingest(const void* src, int64_t n, int64_t ld, int dtype, void* dst,
                          int64_t ldd, int dst_is_f64, int64_t d, double* rownorm,
                          DevCounters* ctr, __nv_bfloat16* rm_hi, __nv_bfloat16* rm_lo2,
                          int64_t ld_rm, __nv_bfloat16* cm_hi, __nv_bfloat16* cm_lo,
                          int64_t ld_cm, int row0, cudaStream_t st, double* slot_n2) {
  if (n <= 0) return cudaSuccess;
  ingest_kernel<<<(unsigned)n, 256, 0, st>>>(src, ld, dtype, dst, ldd, dst_is_f64, d, rownorm,
                                             ctr, rm_hi, rm_lo2, ld_rm, cm_hi, cm_lo, ld_cm,
                                             row0, (int)n, slot_n2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plain CUDA-core Gram G = B B^T over the first n rows, split along d into
// `ksplit` partial sums (summed in fixed order by the eigensolve's load).
// 64 x 64 output tile per block, 256 threads, 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) gram_simt_kernel(const T* __restrict__ B, int64_t ldb,
                                                        int n, int64_t d, T* __restrict__ parts,
                                                        int ldp, int64_t kchunk,
                                                        int64_t part_stride) {
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64, ks = blockIdx.z;
  const int64_t k0 = (int64_t)ks * kchunk;
  const int64_t k1 = min(d, k0 + kchunk);
  __shared__ T As[16][64 + 4];
  __shared__ T Bs[16][64 + 4];
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int64_t kk = k0; kk < k1; kk += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int r = e >> 4, k = e & 15;
      const int64_t kg = kk + k;
      As[k][r] = (i0 + r < n && kg < k1) ? B[(int64_t)(i0 + r) * ldb + kg] : T(0);
      Bs[k][r] = (j0 + r < n && kg < k1) ? B[(int64_t)(j0 + r) * ldb + kg] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  T* out = parts + (int64_t)ks * part_stride;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
    if (i >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx * 4 + b;
      if (j < n) out[(int64_t)i * ldp + j] = acc[a][b];
    }
  }
}

template <typename T>
cudaError_t launch_gram_simt(const T* B, int64_t ldb, int n, int64_t d, T* parts, int ldp,
                             int ksplit, cudaStream_t st) {
  const int tiles = (n + 63) / 64;
  int64_t kchunk = (d + ksplit - 1) / ksplit;
  kchunk = ((kchunk + 15) / 16) * 16;
  const int ks = (int)((d + kchunk - 1) / kchunk);
  dim3 grid(tiles, tiles, ks);
  gram_simt_kernel<T><<<grid, 256, 0, st>>>(B, ldb, n, d, parts, ldp, kchunk,
                                            (int64_t)ldp * ldp);
  return cudaGetLastError();
}

template cudaError_t launch_gram_simt<float>(const float*, int64_t, int, int64_t, float*, int,
                                             int, cudaStream_t);
template cudaError_t launch_gram_simt<double>(const double*, int64_t, int, int64_t, double*,
                                              int, int, cudaStream_t);

// G = (Z + Z^T) / 2 with Z the sum of the Gram's partial slices (fixed
// order), over the whole grid, so that the one-CTA eigensolve loads a single
// matrix (summing the slices there took longer than the solve's first phase).
template <typename T>
__global__ void __launch_bounds__(256) gram_sum_parts_kernel(const T* __restrict__ parts,
                                                             int nparts, int ldp,
                                                             int64_t part_stride, int n,
                                                             T* __restrict__ out, int ldo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
  T sij = T(0), sji = T(0);
  for (int p = 0; p < nparts; ++p) {
    sij += parts[(int64_t)p * part_stride + (int64_t)i * ldp + j];
    sji += parts[(int64_t)p * part_stride + (int64_t)j * ldp + i];
  }
  out[(int64_t)i * ldo + j] = T(0.5) * (sij + sji);
}

template <typename T>
cudaError_t launch_gram_sum_parts(const T* parts, int nparts, int ldp, int n, T* out, int ldo,
                                  cudaStream_t st) {
  const int64_t tot = (int64_t)n * n;
  gram_sum_parts_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      parts, nparts, ldp, (int64_t)ldp * ldp, n, out, ldo);
  return cudaGetLastError();
}

template cudaError_t launch_gram_sum_parts<float>(const float*, int, int, int, float*, int,
                                                  cudaStream_t);
template cudaError_t launch_gram_sum_parts<double>(const double*, int, int, int, double*, int,
                                                   cudaStream_t);

// Number of partial slices the Gram launch above produces for (d, ksplit).
int gram_simt_slices(int64_t d, int ksplit) {
  int64_t kchunk = (d + ksplit - 1) / ksplit;
  kchunk = ((kchunk + 15) / 16) * 16;
  return (int)((d + kchunk - 1) / kchunk);
}

// ---------------------------------------------------------------------------
// Eigensolve + shrink, one CTA per reduction.
//
// One-sided (Hestenes) Jacobi on the columns of the symmetric positive
// semidefinite G: W = G V with V a product of plane rotations, iterated until
// the columns of W are mutually orthogonal. Then W^T W = V^T G^2 V is
// diagonal, so V holds eigenvectors of G and column j of W equals
// lambda_j u_j: the eigenvector comes out of W itself and V is never stored.
// Pairs are visited in round-robin (tournament) order: np/2 disjoint pairs per
// round, one warp per pair, np-1 rounds per sweep, one barrier per round.
// Eigenvalues lambda_j = ||w_j|| are formed in FP64 and the ReduceRank rule
// of the variant runs in FP64 (Sec. 2.3, Algorithms 2 and 3).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(EIG_THREADS) eig_shrink_kernel(EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n;
  const int np = n + (n & 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const bool in_smem = (a.work == nullptr);
  const int ld = in_smem ? np : a.ldw_work;
  T* Wm = in_smem ? reinterpret_cast<T*>(smem_raw) : reinterpret_cast<T*>(a.work);
  size_t off = in_smem ? (((size_t)np * np * sizeof(T) + 15) & ~(size_t)15) : 0;
  double* lam = reinterpret_cast<double*>(smem_raw + off);
  double* mu = lam + np;
  double* mup = mu + np;
  double* scl = mup + np;
  int* ord = reinterpret_cast<int*>(scl + np);
  int* rrank = ord + np;
  __shared__ int s_rot;

  eig_prepare_diag(a, n);
  eig_load<T>(a, Wm, ld, n, np);
  if (tid == 0) s_rot = 0;
  __syncthreads();

  // 2. Jacobi sweeps.
  const int npairs = np / 2;
  const int nrounds = np - 1;
  const int epl = (np + 31) / 32;
  const T tol = (T)a.tol;
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    int local_rot = 0;
    for (int r = 0; r < nrounds; ++r) {
      for (int k = warp; k < npairs; k += nwarps) {
        const int p = rr_index(k, r, np);
        const int q = rr_index(np - 1 - k, r, np);
        T* wp = Wm + (int64_t)p * ld;
        T* wq = Wm + (int64_t)q * ld;
        T xp[EIG_MAX_EPL], xq[EIG_MAX_EPL];
        T al = T(0), be = T(0), ga = T(0);
#pragma unroll
        for (int e = 0; e < EIG_MAX_EPL; ++e) {
          const int i = lane + 32 * e;
          if (e < epl && i < np) { xp[e] = wp[i]; xq[e] = wq[i]; }
          else { xp[e] = T(0); xq[e] = T(0); }
          al = fma(xp[e], xp[e], al);
          be = fma(xq[e], xq[e], be);
          ga = fma(xp[e], xq[e], ga);
        }
        al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
        if (ga != T(0) && fabs(ga) > tol * sqrt(al * be)) {
          const T zeta = (be - al) / (T(2) * ga);
          const T az = fabs(zeta);
          T t = (az > T(1e15)) ? T(0.5) / zeta
                               : copysign(T(1), zeta) / (az + sqrt(T(1) + zeta * zeta));
          const T c = T(1) / sqrt(T(1) + t * t);
          const T s = c * t;
#pragma unroll
          for (int e = 0; e < EIG_MAX_EPL; ++e) {
            const int i = lane + 32 * e;
            if (e < epl && i < np) {
              const T np_ = c * xp[e] - s * xq[e];
              const T nq_ = s * xp[e] + c * xq[e];
              wp[i] = np_;
              wq[i] = nq_;
            }
          }
          ++local_rot;
        }
      }
      __syncthreads();
    }
    if (lane == 0 && local_rot) atomicAdd(&s_rot, local_rot);
    __syncthreads();
    const int total = s_rot;
    __syncthreads();
    if (tid == 0) s_rot = 0;
    __syncthreads();
    if (total == 0) break;
  }
  // sweeps run: the last one found no pair to rotate, unless the cap was hit
  const int sweeps_run = (sweep < a.max_sweeps) ? sweep + 1 : a.max_sweeps;

  eig_finish<T>(a, Wm, ld, n, np, sweeps_run, sweep >= a.max_sweeps, 1.0, lam, mu, mup, scl,
                ord, rrank);
}

// FP32 eigensolve with G in shared memory (one-sided Jacobi of fd_jacobi.cuh),
// G scaled by its largest diagonal entry so that every column norm is at most
// np whatever the scale of the rows.
template <int GS, int MAXV, int MAXP, int NT>
__global__ void __launch_bounds__(NT) eig_fast_kernel(EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n;
  const int np = n + (n & 1);
  const int ld = (np + 3) & ~3;
  const int tid = threadIdx.x;
  float* Wm = reinterpret_cast<float*>(smem_raw);
  size_t off = (((size_t)np * ld * sizeof(float) + 15) & ~(size_t)15);
  float* nrm = reinterpret_cast<float*>(smem_raw + off);
  off += (((size_t)np * sizeof(float) + 15) & ~(size_t)15);
  double* lam = reinterpret_cast<double*>(smem_raw + off);
  double* mu = lam + np;
  double* mup = mu + np;
  double* scl = mup + np;
  int* ord = reinterpret_cast<int*>(scl + np);
  int* rrank = ord + np;
  __shared__ float s_max;

  eig_prepare_diag(a, n);
  eig_load<float>(a, Wm, ld, n, np);
  if (tid == 0) s_max = 0.f;
  __syncthreads();
  float dm = 0.f;
  for (int i = tid; i < n; i += blockDim.x) dm = fmaxf(dm, fabsf(Wm[(size_t)i * ld + i]));
  for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((tid & 31) == 0) atomicMax(reinterpret_cast<int*>(&s_max), __float_as_int(dm));
  __syncthreads();
  const float smax = eig_pow2_scale(s_max);
  const float inv = 1.f / smax;  // exact: smax is a power of two
  for (int idx = tid; idx < np * ld; idx += blockDim.x) Wm[idx] *= inv;
  __syncthreads();
  int capped = 0;
  const int sweeps = jacobi_sweeps_f32<GS, MAXV, MAXP>(Wm, ld, np, nrm, a.max_sweeps,
                                                        (float)a.tol, &capped);
  eig_finish<float>(a, Wm, ld, n, np, sweeps, capped, (smax > 0.f) ? (double)smax : 1.0, lam,
                    mu, mup, scl, ord, rrank);
}

// Full-buffer FP32 reductions: Householder tridiagonalisation, bisection and
// inverse iteration (fd_tridiag.cuh), G scaled by its largest diagonal entry.
template <int NB, int R, int MAXJ, int VPT, bool GLOBAL>
__global__ void __launch_bounds__(512, 1) eig_tri_kernel(EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n;
  const int ld = n | 1;
  const int tid = threadIdx.x;
  // A and the scratch area in shared memory, or (large buffers) in the
  // global workspace a.work
  float* A = GLOBAL ? reinterpret_cast<float*>(a.work) : reinterpret_cast<float*>(smem_raw);
  unsigned char* scr = GLOBAL ? reinterpret_cast<unsigned char*>(a.work) + tri_al16((size_t)n * ld * 4)
                              : smem_raw + tri_al16((size_t)n * ld * 4);
  unsigned char* small = GLOBAL ? smem_raw : scr + tri_scratch_bytes(n, NB);
  // step-1 workspace: the scratch area while that is in shared memory
  // (tri_config checks that it is large enough), else after `small`
  unsigned char* rw = GLOBAL ? smem_raw + tri_small_bytes(n) : scr;
  __shared__ float s_max;
  if (tid == 0) s_max = 0.f;
  eig_prepare_diag(a, n);
  eig_load_sym<float>(a, A, ld, n);
  float dm = 0.f;
  for (int i = tid; i < n; i += blockDim.x) dm = fmaxf(dm, fabsf(A[(size_t)i * ld + i]));
  for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((tid & 31) == 0) atomicMax(reinterpret_cast<int*>(&s_max), __float_as_int(dm));
  __syncthreads();
  const float smax = eig_pow2_scale(s_max);
  const float inv = 1.f / smax;  // exact: smax is a power of two
  {
    // scale; the scaled G is also kept (gsave) for the Rayleigh quotients
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int wcols = (a.gsave != nullptr && a.ldgsave > ld) ? a.ldgsave : ld;
    for (int i = warp; i < n; i += nw) {
      for (int j = lane; j < wcols; j += 32) {
        float v = 0.f;
        if (j < ld) {
          v = A[(size_t)i * ld + j] * inv;
          A[(size_t)i * ld + j] = v;
        }
        if (a.gsave != nullptr && j < a.ldgsave)
          a.gsave[(size_t)i * a.ldgsave + j] = (j < n) ? v : 0.f;
      }
    }
    __syncthreads();
  }
  tri_eig_shrink<NB, R, MAXJ, VPT>(a, A, ld, n, (smax > 0.f) ? (double)smax : 1.0, scr, small, rw);
}

template <int NB, int R, int MAXJ, int VPT, bool GLOBAL>
cudaError_t launch_tri(const EigArgs& a, size_t smem, cudaStream_t st) {
  static size_t attr_set = 0;
  if (smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(eig_tri_kernel<NB, R, MAXJ, VPT, GLOBAL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = smem;
  }
  eig_tri_kernel<NB, R, MAXJ, VPT, GLOBAL><<<1, 512, smem, st>>>(a);
  return cudaGetLastError();
}

// Whether a reduction of n rows takes the tridiagonal eigensolve: buffers of
// at least 2*ell rows (a flush of a partial buffer is solved at the full
// buffer size, its missing rows zero). 1: n <= 128 in
// shared memory; 2, 3: up to 206 rows in shared memory (LU batches of 16 or 8
// vectors for the fallback path); 4: up to 512 rows with A and the scratch
// area in a global workspace of tri_global_bytes(n, 16) bytes.
int tri_config(int n, int ell) {
  if (n < 2 * ell || n < 4) return 0;  // retained vectors <= n/2
  const size_t rw = tri_rw_bytes(n, 16);  // 512 threads
  if (n <= 128 && tri_smem_bytes(n, 32) <= 226 * 1024 && tri_scratch_bytes(n, 32) >= rw) return 1;
  if (n <= 208 && tri_smem_bytes(n, 16) <= 226 * 1024 && tri_scratch_bytes(n, 16) >= rw) return 2;
  if (n <= 208 && tri_smem_bytes(n, 8) <= 226 * 1024 && tri_scratch_bytes(n, 8) >= rw) return 3;
  if (n <= 512) return 4;
  return 0;
}

size_t tri_global_workspace(int n) { return tri_global_bytes(n, 16); }

size_t eig_fast_smem(int np) {
  const int ld = (np + 3) & ~3;
  return (((size_t)np * ld * 4 + 15) & ~(size_t)15) + (((size_t)np * 4 + 15) & ~(size_t)15) +
         eig_scalar_bytes(np);
}

template <int GS, int MAXV, int MAXP, int NT>
cudaError_t launch_fast(const EigArgs& a, size_t smem, cudaStream_t st) {
  static size_t attr_set = 0;  // largest dynamic size granted so far for this instantiation
  if (smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(eig_fast_kernel<GS, MAXV, MAXP, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = smem;
  }
  const int np = a.n + (a.n & 1);
  int threads = ((np / 2) * GS + 31) / 32 * 32;
  if (threads > NT) threads = NT;
  if (threads < 64) threads = 64;
  eig_fast_kernel<GS, MAXV, MAXP, NT><<<1, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// FP32 reductions of up to 224 rows keep G in shared memory and use the
// grouped kernel; larger (or FP64) reductions use the warp-per-pair kernel.
template <typename T>
cudaError_t launch_eig_shrink(const EigArgs& a, cudaStream_t st) {
  const int np = a.n + (a.n & 1);
  if (sizeof(T) == 4 && a.use_tri) {
    const int cfg = tri_config(a.n, a.ell);
    if (cfg == 1) return launch_tri<32, 8, 16, 1, false>(a, tri_smem_bytes(a.n, 32), st);
    if (cfg == 2) return launch_tri<16, 8, 26, 2, false>(a, tri_smem_bytes(a.n, 16), st);
    if (cfg == 3) return launch_tri<8, 8, 26, 2, false>(a, tri_smem_bytes(a.n, 8), st);
    if (cfg == 4 && a.work != nullptr && a.work_bytes >= tri_global_bytes(a.n, 16))
      return launch_tri<16, 16, 32, 2, true>(a, tri_small_bytes(a.n) + tri_rw_bytes(a.n, 16), st);
  }
  if (sizeof(T) == 4 && a.work == nullptr && np <= 224 && eig_fast_smem(np) <= 226 * 1024) {
    const size_t smem = eig_fast_smem(np);
    if (np <= 64) return launch_fast<8, 2, 1, 256>(a, smem, st);
    if (np <= 128) return launch_fast<8, 4, 1, 512>(a, smem, st);
    return launch_fast<16, 4, 2, 1024>(a, smem, st);
  }
  size_t smem = eig_scalar_bytes(np);
  if (a.work == nullptr) smem += (((size_t)np * np * sizeof(T) + 15) & ~(size_t)15);
  cudaError_t e = cudaFuncSetAttribute(eig_shrink_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eig_shrink_kernel<T><<<1, EIG_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_eig_shrink<float>(const EigArgs&, cudaStream_t);
template cudaError_t launch_eig_shrink<double>(const EigArgs&, cudaStream_t);

// Whether the eigensolve of an n-row reduction keeps G in shared memory.
bool eig_fits_smem(int n, size_t elem) {
  const int np = n + (n & 1);
  if (elem == 4 && np <= 224 && eig_fast_smem(np) <= 226 * 1024) return true;
  const size_t need = eig_scalar_bytes(np) + (((size_t)np * np * elem + 15) & ~(size_t)15);
  return need <= 226 * 1024;
}

// ---------------------------------------------------------------------------
// Plain CUDA-core rotate B' = Wrot B (Sec. 2.3, B <- S' V^T): rows 0..nout-1.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) rotate_simt_kernel(const T* __restrict__ W, int ldw,
                                                          int nout, int n,
                                                          const T* __restrict__ Bin,
                                                          int64_t ldb, T* __restrict__ Bout,
                                                          int64_t ldo, int64_t d) {
  const int r0 = blockIdx.y * 64;
  const int64_t c0 = (int64_t)blockIdx.x * 64;
  __shared__ T Ws[16][64 + 4];
  __shared__ T Bs[16][64 + 4];
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int kk = 0; kk < n; kk += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int r = e >> 4, k = e & 15;
      Ws[k][r] = (r0 + r < nout && kk + k < n) ? W[(int64_t)(r0 + r) * ldw + kk + k] : T(0);
      const int kb = e >> 6, cb = e & 63;
      Bs[kb][cb] = (kk + kb < n && c0 + cb < d) ? Bin[(int64_t)(kk + kb) * ldb + c0 + cb] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Ws[k][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
    if (r >= nout) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t c = c0 + tx * 4 + b;
      if (c < d) Bout[(int64_t)r * ldo + c] = acc[a][b];
    }
  }
}

template <typename T>
cudaError_t launch_rotate_simt(const T* W, int ldw, int nout, int n, const T* Bin, int64_t ldb,
                               T* Bout, int64_t ldo, int64_t d, cudaStream_t st) {
  dim3 grid((unsigned)((d + 63) / 64), (unsigned)((nout + 63) / 64));
  rotate_simt_kernel<T><<<grid, 256, 0, st>>>(W, ldw, nout, n, Bin, ldb, Bout, ldo, d);
  return cudaGetLastError();
}

template cudaError_t launch_rotate_simt<float>(const float*, int, int, int, const float*,
                                               int64_t, float*, int64_t, int64_t,
                                               cudaStream_t);
template cudaError_t launch_rotate_simt<double>(const double*, int, int, int, const double*,
                                                int64_t, double*, int64_t, int64_t,
                                                cudaStream_t);

// ---------------------------------------------------------------------------
// Output conversion and ||B||_F^2.
// ---------------------------------------------------------------------------
__global__ void convert_out_kernel(const void* __restrict__ src, int src_f64, int64_t lds,
                                   int rows, int64_t d, void* __restrict__ dst, int dst_f64,
                                   int64_t ldd, int zero_from) {
  const int r = blockIdx.x;
  for (int64_t k = threadIdx.x; k < d; k += blockDim.x) {
    double v = 0.0;
    if (r < zero_from) {
      v = src_f64 ? reinterpret_cast<const double*>(src)[(int64_t)r * lds + k]
                  : (double)reinterpret_cast<const float*>(src)[(int64_t)r * lds + k];
    }
    if (dst_f64) reinterpret_cast<double*>(dst)[(int64_t)r * ldd + k] = v;
    else reinterpret_cast<float*>(dst)[(int64_t)r * ldd + k] = (float)v;
  }
}

cudaError_t launch_convert_out(const void* src, int src_f64, int64_t lds, int rows, int64_t d,
                               void* dst, int dst_f64, int64_t ldd, int zero_from_row,
                               cudaStream_t st) {
  convert_out_kernel<<<rows, 256, 0, st>>>(src, src_f64, lds, rows, d, dst, dst_f64, ldd,
                                           zero_from_row);
  return cudaGetLastError();
}

__global__ void norm_b2_kernel(const void* __restrict__ src, int src_f64, int64_t lds,
                               int rows, int64_t d, DevCounters* ctr) {
  double acc = 0.0;
  for (int r = 0; r < rows; ++r)
    for (int64_t k = threadIdx.x; k < d; k += blockDim.x) {
      const double v = src_f64 ? reinterpret_cast<const double*>(src)[(int64_t)r * lds + k]
                               : (double)reinterpret_cast<const float*>(src)[(int64_t)r * lds + k];
      acc = fma(v, v, acc);
    }
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    ctr->norm_b2 = s;
  }
}

cudaError_t launch_norm_b2(const void* src, int src_f64, int64_t lds, int rows, int64_t d,
                           DevCounters* ctr, cudaStream_t st) {
  norm_b2_kernel<<<1, 256, 0, st>>>(src, src_f64, lds, rows, d, ctr);
  return cudaGetLastError();
}

// Compensative FD (Sec. 3.1): row r of a sketch with orthogonal rows, norm
// sigma'_r, is scaled by sqrt((sigma'_r^2 + Delta) / sigma'_r^2); zero rows stay
// zero. One block per row, the squared norm in FP64.
__global__ void compensate_rows_kernel(void* __restrict__ B, int b_f64, int64_t ld, int64_t d,
                                       const DevCounters* __restrict__ ctr) {
  const int64_t r = blockIdx.x;
  __shared__ double red[32];
  __shared__ double s_f;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < d; k += blockDim.x) {
    const double v = b_f64 ? reinterpret_cast<const double*>(B)[r * ld + k]
                           : (double)reinterpret_cast<const float*>(B)[r * ld + k];
    acc = fma(v, v, acc);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    s_f = (s > 0.0) ? sqrt((s + ctr->sum_delta) / s) : 1.0;
  }
  __syncthreads();
  const double f = s_f;
  for (int64_t k = threadIdx.x; k < d; k += blockDim.x) {
    if (b_f64) {
      double* x = reinterpret_cast<double*>(B) + r * ld + k;
      *x *= f;
    } else {
      float* x = reinterpret_cast<float*>(B) + r * ld + k;
      *x = (float)((double)*x * f);
    }
  }
}

cudaError_t launch_compensate_rows(void* B, int b_f64, int64_t ld, int rows, int64_t d,
                                   const DevCounters* ctr, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  compensate_rows_kernel<<<rows, 256, 0, st>>>(B, b_f64, ld, d, ctr);
  return cudaGetLastError();
}

// Rows of a sketch up to its last nonzero one (1 + index, 0 if all zero):
// one warp per row, block-wide maximum.
__global__ void last_nonzero_row_kernel(const void* __restrict__ src, int src_f64, int64_t lds,
                                        int rows, int64_t d, int* out) {
  __shared__ int s_last;
  if (threadIdx.x == 0) s_last = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < rows; r += nw) {
    int nz = 0;
    for (int64_t k = lane; k < d && !nz; k += 32) {
      const double v = src_f64 ? reinterpret_cast<const double*>(src)[(int64_t)r * lds + k]
                               : (double)reinterpret_cast<const float*>(src)[(int64_t)r * lds + k];
      nz = (v != 0.0);
    }
    if (__any_sync(0xffffffffu, nz) && lane == 0) atomicMax(&s_last, r + 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *out = s_last;
}

cudaError_t launch_last_nonzero_row(const void* src, int src_f64, int64_t lds, int rows, int64_t d,
                                    int* out, cudaStream_t st) {
  last_nonzero_row_kernel<<<1, 256, 0, st>>>(src, src_f64, lds, rows, d, out);
  return cudaGetLastError();
}

// Counters of a merge: dst takes src's stream mass in place of the appended
// sketch rows' mass (ingest already added ||B_src||_F^2), and src's deltas,
// removed mass and reductions (src: the counters of its latest sketch).
__global__ void merge_counters_kernel(DevCounters* dst, const DevCounters* src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    dst->norm_a2 += src->norm_a2 - src->norm_b2;
    dst->sum_delta += src->sum_delta;
    dst->removed += src->removed;
    dst->reductions += src->reductions;
  }
}

// fd_merge_sketch: ||A||_F^2 = its value before the rows were appended plus
// the source stream's; the source's deltas, removed mass and reductions added.
__global__ void merge_counters_values_kernel(DevCounters* dst, const double* norm_before,
                                             double norm_a2, double sum_delta, double removed,
                                             long long reductions) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    dst->norm_a2 = *norm_before + norm_a2;
    dst->sum_delta += sum_delta;
    dst->removed += removed;
    dst->reductions += reductions;
  }
}

cudaError_t launch_merge_counters_values(DevCounters* dst, const double* norm_before,
                                         double norm_a2, double sum_delta, double removed,
                                         long long reductions, cudaStream_t st) {
  merge_counters_values_kernel<<<1, 32, 0, st>>>(dst, norm_before, norm_a2, sum_delta, removed,
                                                 reductions);
  return cudaGetLastError();
}

cudaError_t launch_merge_counters(DevCounters* dst, const DevCounters* src, cudaStream_t st) {
  merge_counters_kernel<<<1, 32, 0, st>>>(dst, src);
  return cudaGetLastError();
}

}  // namespace fdk

namespace fdk {
cudaError_t launch_eig_shrink_f32(const EigArgs& a, cudaStream_t st) {
  return launch_eig_shrink<float>(a, st);
}
}  // namespace fdk
