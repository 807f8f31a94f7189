// CUDA-core kernels of the buffered FD reduction: row ingest, the plain
// FP32/FP64 Gram and rotate, and the fused one-CTA eigensolve + shrink.
//
// One reduction of Algorithm 1 (Sec. 2.3) on a buffer B of n rows is
//   G = B B^T                         (gram_simt_kernel or the tcgen05 Gram)
//   G = U diag(sigma^2) U^T           (eig_shrink_kernel, one-sided Jacobi)
//   sigma' = ReduceRank(sigma)        (eig_shrink_kernel, FP64)
//   B' = diag(sigma'/sigma) U^T B     (rotate_simt_kernel or the tcgen05 rotate)
// which equals B' = S' V^T because U^T B = S V^T for the SVD B = U S V^T.
#include <cfloat>
#include <cmath>
#include <cstdio>

#include "fd_internal.cuh"

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
                              int row0, int nrows) {
  const int r = blockIdx.x;
  const void* srow = src;
  double acc = 0.0;
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
    }
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
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
                          int64_t ld_cm, int row0, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ingest_kernel<<<(unsigned)n, 256, 0, st>>>(src, ld, dtype, dst, ldd, dst_is_f64, d, rownorm,
                                             ctr, rm_hi, rm_lo2, ld_rm, cm_hi, cm_lo, ld_cm,
                                             row0, (int)n);
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
__device__ __forceinline__ int rr_index(int pos, int r, int np) {
  // position 0 is fixed, the others rotate by one place per round
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (np - 1);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

constexpr int EIG_THREADS = 512;
constexpr int EIG_MAX_EPL = 16;  // elements per lane per column: n <= 512

size_t eig_scalar_bytes(int np) {
  return (size_t)np * (4 * sizeof(double) + 2 * sizeof(int)) + 256;
}

// Load G = sum of the partial slices (fixed order), symmetrised, into Wm
// (column j = row j of the symmetric G, stride ld, zero padding to np).
template <typename T>
__device__ void eig_load(const EigArgs& a, T* Wm, int ld, int n, int np) {
  const T* parts = reinterpret_cast<const T*>(a.parts);
  for (int idx = threadIdx.x; idx < np * ld; idx += blockDim.x) {
    const int i = idx / ld, j = idx - (idx / ld) * ld;
    T v = T(0);
    if (i < n && j < n) {
      T sij = T(0), sji = T(0);
      for (int p = 0; p < a.nparts; ++p) {
        sij += parts[(int64_t)p * a.part_stride + (int64_t)i * a.ldp + j];
        sji += parts[(int64_t)p * a.part_stride + (int64_t)j * a.ldp + i];
      }
      v = T(0.5) * (sij + sji);
    }
    Wm[(int64_t)i * ld + j] = v;
  }
}

// Steps after the Jacobi sweeps: eigenvalues, sort, ReduceRank (FP64),
// rotate matrix, counters. `sweep` = sweeps run (== max_sweeps if capped).
template <typename T>
__device__ void eig_finish(const EigArgs& a, const T* Wm, int ld, int n, int np, int sweep,
                           int capped, double* lam, double* mu, double* mup, double* scl,
                           int* ord, int* rrank) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  __shared__ int s_count;
  __shared__ double s_dsum, s_dlast;
  const int s_sweeps = sweep;
  // lambda_j = ||w_j|| in FP64 (one warp per column).
  for (int j = warp; j < np; j += nwarps) {
    double s = 0.0;
    for (int i = lane; i < np; i += 32) {
      const double v = (double)Wm[(int64_t)j * ld + i];
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) lam[j] = (j < n) ? sqrt(s) : -1.0;  // padding column sorts last
  }
  __syncthreads();

  // 4. Sort descending, ties by column index.
  for (int j = tid; j < np; j += blockDim.x) {
    const double lj = lam[j];
    int rank = 0;
    for (int i = 0; i < np; ++i) {
      const double li = lam[i];
      rank += (li > lj) || (li == lj && i < j);
    }
    ord[rank] = j;
  }
  __syncthreads();
  for (int k = tid; k < np; k += blockDim.x) {
    const double v = lam[ord[k]];
    mu[k] = v > 0.0 ? v : 0.0;
  }
  if (tid == 0) { s_dsum = 0.0; s_dlast = 0.0; }
  __syncthreads();

  // 5. ReduceRank in FP64 on the masses mu_k = sigma_k^2 (k = 0..n-1 sorted).
  const int ell = a.ell;
  if (a.variant != FD_VAR_SS) {
    const double delta = (n >= ell) ? mu[ell - 1] : 0.0;
    int keep = 0;
    if (a.variant == FD_VAR_PFD) {
      // Algorithm 2 keeps floor((1-alpha)*ell) values; alpha > 0 shrinks at least one
      keep = (int)floor((1.0 - a.alpha) * ell + 1e-9);
      keep = keep < 0 ? 0 : (keep > ell - 1 ? ell - 1 : keep);
    }
    for (int k = tid; k < np; k += blockDim.x) {
      const double m0 = mu[k];
      double mp = 0.0;
      if (k < n) {
        if (a.variant == FD_VAR_FD) mp = fmax(m0 - delta, 0.0);
        else if (a.variant == FD_VAR_ISVD) mp = (k < ell - 1) ? m0 : 0.0;
        else mp = (k < keep) ? m0 : ((k < ell) ? fmax(m0 - delta, 0.0) : 0.0);
      }
      mup[k] = mp;
    }
    if (tid == 0) { s_dsum = delta; s_dlast = delta; }
  } else if (warp == 0) {
    // SS (Algorithm 3, repeated): masses at or below the numerical-rank floor
    // are empty; then merge the second-smallest into the smallest until ell-1
    // directions remain. Ties: the larger sorted position counts as smaller.
    const double flo = mu[0] * (double)np * Eps<T>::v;
    for (int k = lane; k < np; k += 32) mup[k] = (k < n && mu[k] > flo) ? mu[k] : 0.0;
    __syncwarp();
    int alive = 0;
    for (int k = lane; k < np; k += 32) alive += (mup[k] > 0.0);
    alive = warp_sum(alive);
    double dsum = 0.0, dlast = 0.0;
    while (alive > ell - 1) {
      // per lane: two smallest alive (mass asc, position desc)
      double m1 = INFINITY, m2 = INFINITY;
      int i1 = -1, i2 = -1;
      for (int k = lane; k < np; k += 32) {
        const double v = mup[k];
        if (v <= 0.0) continue;
        const bool lt1 = (v < m1) || (v == m1 && k > i1);
        if (lt1) { m2 = m1; i2 = i1; m1 = v; i1 = k; }
        else {
          const bool lt2 = (v < m2) || (v == m2 && k > i2);
          if (lt2) { m2 = v; i2 = k; }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double om1 = __shfl_xor_sync(0xffffffffu, m1, o);
        const double om2 = __shfl_xor_sync(0xffffffffu, m2, o);
        const int oi1 = __shfl_xor_sync(0xffffffffu, i1, o);
        const int oi2 = __shfl_xor_sync(0xffffffffu, i2, o);
        // merge two sorted pairs (m1,i1),(m2,i2) and (om1,oi1),(om2,oi2)
        double c[4] = {m1, m2, om1, om2};
        int ci[4] = {i1, i2, oi1, oi2};
        double b1 = INFINITY, b2 = INFINITY;
        int j1 = -1, j2 = -1;
        for (int t = 0; t < 4; ++t) {
          const double v = c[t];
          const int k = ci[t];
          if (k < 0 || k == j1) continue;
          const bool lt1 = (v < b1) || (v == b1 && k > j1);
          if (lt1) { b2 = b1; j2 = j1; b1 = v; j1 = k; }
          else if (k != j1) {
            const bool lt2 = (v < b2) || (v == b2 && k > j2);
            if (lt2) { b2 = v; j2 = k; }
          }
        }
        m1 = b1; i1 = j1; m2 = b2; i2 = j2;
      }
      // i1 = q (smallest), i2 = p (second smallest)
      if (lane == 0) {
        const double dp = mup[i2];
        mup[i1] = mup[i1] + dp;
        mup[i2] = 0.0;
        dsum += dp;
        dlast = dp;
      }
      __syncwarp();
      --alive;
    }
    if (lane == 0) { s_dsum = dsum; s_dlast = dlast; }
  }
  __syncthreads();

  // 6. Output order: retained positions by sigma'^2 descending, ties by position.
  for (int k = tid; k < np; k += blockDim.x) {
    const double v = mup[k];
    int rank = -1;
    if (v > 0.0) {
      rank = 0;
      for (int i = 0; i < np; ++i) {
        const double w = mup[i];
        rank += (w > v) || (w == v && i < k);
      }
    }
    rrank[k] = rank;
    // scale of column w_j: sigma'/sigma / lambda = sqrt(mu'/mu) / mu
    scl[k] = (v > 0.0 && mu[k] > 0.0) ? sqrt(v / mu[k]) / mu[k] : 0.0;
  }
  if (tid == 0) {
    int cnt = 0;
    for (int k = 0; k < np; ++k) cnt += (mup[k] > 0.0);
    s_count = cnt;
  }
  __syncthreads();

  // 7. Rotate matrix rows 0..ell-2: row r = scale * w_j (zero rows past the count).
  const int nout = ell - 1;
  T* wr = reinterpret_cast<T*>(a.wrot);
  for (int idx = tid; idx < nout * n; idx += blockDim.x) {
    const int r = idx / n, i = idx - (idx / n) * n;
    if (r >= s_count) {
      wr[(int64_t)r * a.ldr + i] = T(0);
      if (a.wrot_hi) {
        a.wrot_hi[(int64_t)r * a.ldr16 + i] = __float2bfloat16_rn(0.0f);
        a.wrot_lo[(int64_t)r * a.ldr16 + i] = __float2bfloat16_rn(0.0f);
      }
    }
  }
  for (int k = warp; k < np; k += nwarps) {
    const int r = rrank[k];
    if (r < 0 || r >= nout) continue;
    const int j = ord[k];
    const double sc = scl[k];
    for (int i = lane; i < n; i += 32) {
      const double v = sc * (double)Wm[(int64_t)j * ld + i];
      wr[(int64_t)r * a.ldr + i] = (T)v;
      if (a.wrot_hi) {
        const float vf = (float)v;
        const __nv_bfloat16 hi = __float2bfloat16_rn(vf);
        a.wrot_hi[(int64_t)r * a.ldr16 + i] = hi;
        a.wrot_lo[(int64_t)r * a.ldr16 + i] = __float2bfloat16_rn(vf - __bfloat162float(hi));
      }
    }
  }

  // 8. FP64 bookkeeping and diagnostics.
  if (a.sig2_out) for (int k = tid; k < n; k += blockDim.x) { a.sig2_out[k] = mu[k]; a.sigp2_out[k] = mup[k]; }
  if (tid == 0) {
    DevCounters c = *a.ctr_in;
    double rem = 0.0, nb = 0.0;
    for (int k = 0; k < n; ++k) { rem += mu[k] - mup[k]; nb += mup[k]; }
    c.sum_delta += s_dsum;
    c.last_delta = s_dlast;
    c.removed += rem;
    c.norm_b2 = nb;
    c.reductions += 1;
    c.noconv += capped ? 1 : 0;
    c.max_sweeps = fmax(c.max_sweeps, (double)s_sweeps);
    c.retained = s_count < nout ? s_count : nout;
    *a.ctr_out = c;
  }
}

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

  eig_finish<T>(a, Wm, ld, n, np, sweeps_run, sweep >= a.max_sweeps, lam, mu, mup, scl, ord,
                rrank);
}

// FP32 Jacobi with GS lanes per column pair, float4 column access, column
// norms carried through the sweep by the exact update
//   ||w_p'||^2 = ||w_p||^2 - t*gamma,  ||w_q'||^2 = ||w_q||^2 + t*gamma
// (recomputed from the data at every sweep start, and at once when the update
// cancels more than three quarters of a norm).
template <int GS, int MAXV, int NT>
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

  eig_load<float>(a, Wm, ld, n, np);
  __syncthreads();

  const int g = tid / GS, gl = tid % GS;
  const int ngroups = NT / GS;
  const unsigned gmask = (GS == 32) ? 0xffffffffu
                                    : (((1u << GS) - 1u) << ((tid & 31) & ~(GS - 1)));
  const int nv = (np + 3) >> 2;  // float4 chunks per column
  const int npairs = np / 2, nrounds = np - 1;
  const float tol = (float)a.tol;

  auto col_sq = [&](const float* w) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < MAXV; ++c) {
      const int v = c * GS + gl;
      if (v < nv) {
        const float4 x = reinterpret_cast<const float4*>(w)[v];
        s = fmaf(x.x, x.x, s); s = fmaf(x.y, x.y, s); s = fmaf(x.z, x.z, s); s = fmaf(x.w, x.w, s);
      }
    }
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, GS);
    return s;
  };

  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    // exact norms at the start of the sweep
    for (int j = g; j < np; j += ngroups) {
      const float s = col_sq(Wm + (int64_t)j * ld);
      if (gl == 0) nrm[j] = s;
    }
    __syncthreads();
    int rotated = 0;
    for (int r = 0; r < nrounds; ++r) {
      for (int k = g; k < npairs; k += ngroups) {
        const int p = rr_index(k, r, np);
        const int q = rr_index(np - 1 - k, r, np);
        float4* wp = reinterpret_cast<float4*>(Wm + (int64_t)p * ld);
        float4* wq = reinterpret_cast<float4*>(Wm + (int64_t)q * ld);
        float4 xp[MAXV], xq[MAXV];
        float ga = 0.f;
#pragma unroll
        for (int c = 0; c < MAXV; ++c) {
          const int v = c * GS + gl;
          if (v < nv) { xp[c] = wp[v]; xq[c] = wq[v]; }
          else { xp[c] = make_float4(0.f, 0.f, 0.f, 0.f); xq[c] = xp[c]; }
          ga = fmaf(xp[c].x, xq[c].x, ga); ga = fmaf(xp[c].y, xq[c].y, ga);
          ga = fmaf(xp[c].z, xq[c].z, ga); ga = fmaf(xp[c].w, xq[c].w, ga);
        }
#pragma unroll
        for (int o = GS / 2; o > 0; o >>= 1) ga += __shfl_xor_sync(gmask, ga, o, GS);
        const float al = nrm[p], be = nrm[q];
        if (ga != 0.f && fabsf(ga) > tol * sqrtf(al * be)) {
          const float zeta = (be - al) / (2.f * ga);
          const float az = fabsf(zeta);
          const float t = (az > 1e15f) ? 0.5f / zeta : copysignf(1.f, zeta) / (az + sqrtf(1.f + zeta * zeta));
          const float cs = rsqrtf(1.f + t * t);
          const float sn = cs * t;
#pragma unroll
          for (int c = 0; c < MAXV; ++c) {
            const int v = c * GS + gl;
            if (v < nv) {
              float4 a4, b4;
              a4.x = cs * xp[c].x - sn * xq[c].x; b4.x = sn * xp[c].x + cs * xq[c].x;
              a4.y = cs * xp[c].y - sn * xq[c].y; b4.y = sn * xp[c].y + cs * xq[c].y;
              a4.z = cs * xp[c].z - sn * xq[c].z; b4.z = sn * xp[c].z + cs * xq[c].z;
              a4.w = cs * xp[c].w - sn * xq[c].w; b4.w = sn * xp[c].w + cs * xq[c].w;
              wp[v] = a4;
              wq[v] = b4;
            }
          }
          float na = al - t * ga, nb = be + t * ga;
          if (na < 0.25f * al) na = col_sq(reinterpret_cast<float*>(wp));
          if (nb < 0.25f * be) nb = col_sq(reinterpret_cast<float*>(wq));
          if (gl == 0) { nrm[p] = na; nrm[q] = nb; }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;
  }
  const int sweeps_run = (sweep < a.max_sweeps) ? sweep + 1 : a.max_sweeps;
  eig_finish<float>(a, Wm, ld, n, np, sweeps_run, sweep >= a.max_sweeps, lam, mu, mup, scl, ord,
                    rrank);
}

size_t eig_fast_smem(int np) {
  const int ld = (np + 3) & ~3;
  return (((size_t)np * ld * 4 + 15) & ~(size_t)15) + (((size_t)np * 4 + 15) & ~(size_t)15) +
         eig_scalar_bytes(np);
}

template <int GS, int MAXV, int NT>
cudaError_t launch_fast(const EigArgs& a, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(eig_fast_kernel<GS, MAXV, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eig_fast_kernel<GS, MAXV, NT><<<1, NT, smem, st>>>(a);
  return cudaGetLastError();
}

// FP32 reductions of up to 224 rows keep G in shared memory and use the
// grouped kernel; larger (or FP64) reductions use the warp-per-pair kernel.
template <typename T>
cudaError_t launch_eig_shrink(const EigArgs& a, cudaStream_t st) {
  const int np = a.n + (a.n & 1);
  if (sizeof(T) == 4 && a.work == nullptr && np <= 224 && eig_fast_smem(np) <= 227 * 1024) {
    const size_t smem = eig_fast_smem(np);
    if (np <= 64) return launch_fast<8, 2, 256>(a, smem, st);
    if (np <= 128) return launch_fast<8, 4, 512>(a, smem, st);
    return launch_fast<16, 4, 1024>(a, smem, st);
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
  if (elem == 4 && np <= 224 && eig_fast_smem(np) <= 227 * 1024) return true;
  const size_t need = eig_scalar_bytes(np) + (((size_t)np * np * elem + 15) & ~(size_t)15);
  return need <= 227 * 1024;
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

}  // namespace fdk

namespace fdk {
cudaError_t launch_eig_shrink_f32(const EigArgs& a, cudaStream_t st) {
  return launch_eig_shrink<float>(a, st);
}
}  // namespace fdk
