// Symmetric eigensolve of the 2*ell x 2*ell Gram by Householder reduction to
// tridiagonal form, bisection for the eigenvalues and inverse iteration for
// the eigenvectors that the ReduceRank step keeps (FP32, one CTA, shared
// memory). It replaces the Jacobi sweeps for full-buffer reductions: about
// (4/3) n^3 + n^2 * (kept vectors) operations instead of ~25 n^3.
//
//   1. A = Q T Q^T: n-2 Householder steps. Step k reflects the trailing
//      column with v_k (unit, length n-k-1) and updates the trailing block by
//      the rank-2 correction A22 -= v q^T + q v^T, q = 2 (A22 v - (v^T A22 v) v).
//      v_k is kept in A's strictly lower part (column k below the diagonal).
//   2. Eigenvalues of T by bisection on Sturm counts, one thread per
//      eigenvalue, sorted descending by construction.
//   3. After ReduceRank decides which positions are kept, one eigenvector of
//      T per kept position by inverse iteration: (T - lambda I) z = z solved by
//      LU with partial pivoting, three times. Vectors are then made
//      orthonormal (classical Gram-Schmidt, twice) and mapped back, u = Q z.
//
// Storage: A is n x ld (ld >= n). After step 1 its strictly upper part is
// free; kept vector c (0 <= c <= n/2-2) lives there, split over two row tails
// of total length n: entries [0, n-1-c) in row c (columns c+1..n-1) and the
// rest in row n-2-c (columns n-1-c..n-1).
#pragma once

#include "fd_eig.cuh"
#include "fd_internal.cuh"

namespace fdk {

__device__ __forceinline__ float tri_block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// Address of entry i of kept vector c in the split layout.
__device__ __forceinline__ float* zslot(float* A, int ld, int n, int c, int i) {
  return (i < n - 1 - c) ? (A + (size_t)c * ld + (c + 1 + i)) : (A + (size_t)(n - 2 - c) * ld + i);
}

// Step 1. d (n) and e (n-1) receive the tridiagonal; vb, pb: n floats.
static __device__ void tri_reduce(float* A, int ld, int n, float* d, float* e, float* vb, float* pb,
                           float* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    float* colk = A + (size_t)(k + 1) * ld + k;  // colk[i * ld] = A[k+1+i][k]
    float s = 0.f;
    for (int i = tid; i < m; i += nt) {
      const float x = colk[(size_t)i * ld];
      s = fmaf(x, x, s);
    }
    const float ss = tri_block_sum(s, red);
    const float x0 = colk[0];
    float alpha = 0.f, scale = 0.f;
    if (ss > 0.f) {
      const float nx = sqrtf(ss);
      alpha = (x0 >= 0.f) ? -nx : nx;
      scale = rsqrtf(2.f * (ss - x0 * alpha));  // 1 / ||x - alpha e_1||
    }
    for (int i = tid; i < m; i += nt)
      vb[i] = ((i == 0) ? (x0 - alpha) : colk[(size_t)i * ld]) * scale;
    if (tid == 0) {
      d[k] = A[(size_t)k * ld + k];
      e[k] = alpha;
    }
    __syncthreads();
    // p = A22 v, one thread per row (rows are ld apart: conflict-free for odd ld)
    const float* A22 = A + (size_t)(k + 1) * ld + (k + 1);
    for (int i = tid; i < m; i += nt) {
      const float* row = A22 + (size_t)i * ld;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      int j = 0;
      for (; j + 3 < m; j += 4) {
        a0 = fmaf(row[j], vb[j], a0);
        a1 = fmaf(row[j + 1], vb[j + 1], a1);
        a2 = fmaf(row[j + 2], vb[j + 2], a2);
        a3 = fmaf(row[j + 3], vb[j + 3], a3);
      }
      for (; j < m; ++j) a0 = fmaf(row[j], vb[j], a0);
      pb[i] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    float kp = 0.f;
    for (int i = tid; i < m; i += nt) kp = fmaf(vb[i], pb[i], kp);
    const float K = tri_block_sum(kp, red);
    for (int i = tid; i < m; i += nt) pb[i] = 2.f * fmaf(-K, vb[i], pb[i]);
    __syncthreads();
    // A22 -= v q^T + q v^T (one warp per row); keep v in column k
    for (int i = warp; i < m; i += nwarps) {
      float* row = A + (size_t)(k + 1 + i) * ld + (k + 1);
      const float vi = vb[i], qi = pb[i];
      for (int j = lane; j < m; j += 32) row[j] = fmaf(-vi, pb[j], fmaf(-qi, vb[j], row[j]));
    }
    for (int i = tid; i < m; i += nt) colk[(size_t)i * ld] = vb[i];
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(size_t)(n - 2) * ld + (n - 2)];
      e[n - 2] = A[(size_t)(n - 1) * ld + (n - 2)];
    }
    d[n - 1] = A[(size_t)(n - 1) * ld + (n - 1)];
  }
  __syncthreads();
}

// Number of eigenvalues of T below x (Sturm sequence of the LDL^T pivots).
__device__ __forceinline__ int tri_sturm(const float* d, const float* e2, int n, float x,
                                         float pivmin) {
  float q = d[0] - x;
  int cnt = (q < 0.f);
  for (int i = 1; i < n; ++i) {
    if (fabsf(q) < pivmin) q = -pivmin;
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    cnt += (q < 0.f);
  }
  return cnt;
}

// Step 2. lam[j] = j-th largest eigenvalue of T (one thread per eigenvalue).
// Returns the Gershgorin bound of ||T|| through *tnorm_out (shared).
static __device__ void tri_bisect(const float* d, const float* e, float* e2, int n, float* lam,
                           float* tnorm_out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ float s_lo, s_hi;
  for (int i = tid; i < n - 1; i += nt) e2[i] = e[i] * e[i];
  if (tid == 0) {
    float lo = 3.4e38f, hi = -3.4e38f;
    for (int i = 0; i < n; ++i) {
      const float r = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i < n - 1 ? fabsf(e[i]) : 0.f);
      lo = fminf(lo, d[i] - r);
      hi = fmaxf(hi, d[i] + r);
    }
    s_lo = lo;
    s_hi = hi;
    *tnorm_out = fmaxf(fabsf(lo), fabsf(hi));
  }
  __syncthreads();
  const float tnorm = fmaxf(fabsf(s_lo), fabsf(s_hi));
  const float eps = 1.1920929e-07f;
  const float pivmin = fmaxf(tnorm, 1e-30f) * 1e-30f;
  const float atol = 2.f * eps * tnorm;
  const float span = s_hi - s_lo;
  for (int j = tid; j < n; j += nt) {
    const int target = n - 1 - j;  // 0-based index from the smallest
    float lo = s_lo - 0.01f * span - atol, hi = s_hi + 0.01f * span + atol;
    for (int it = 0; it < 80; ++it) {
      if (hi - lo <= atol + 2.f * eps * fmaxf(fabsf(lo), fabsf(hi))) break;
      const float mid = 0.5f * (lo + hi);
      if (tri_sturm(d, e2, n, mid, pivmin) > target) hi = mid; else lo = mid;
    }
    lam[j] = 0.5f * (lo + hi);
  }
  __syncthreads();
}

// Step 3a. Inverse iteration for kept vectors c = c0 + t (t < NB, c < cend):
// eigenvalue lam[pos[c]]; the vector is written to its slot. Scratch holds
// NB interleaved copies of the four LU bands plus NB x n pivot bytes.
template <int NB>
__device__ void tri_invit_batch(float* A, int ld, int n, const float* d, const float* e,
                                const float* lam, const int* pos, int c0, int cend, float tnorm,
                                float* scr, unsigned char* piv) {
  const int t = threadIdx.x;
  const int c = c0 + t;
  if (t >= NB || c >= cend) return;
  float* dd = scr;
  float* du = scr + (size_t)NB * n;
  float* du2 = scr + (size_t)2 * NB * n;
  float* dl = scr + (size_t)3 * NB * n;
#define DD(i) dd[(size_t)(i) * NB + t]
#define DU(i) du[(size_t)(i) * NB + t]
#define DU2(i) du2[(size_t)(i) * NB + t]
#define DL(i) dl[(size_t)(i) * NB + t]
#define PV(i) piv[(size_t)(i) * NB + t]
  const float eps = 1.1920929e-07f;
  const float tiny = eps * fmaxf(tnorm, 1e-30f);
  const float lmb = lam[pos[c]];
  for (int i = 0; i < n; ++i) {
    DD(i) = d[i] - lmb;
    if (i < n - 1) { DU(i) = e[i]; DL(i) = e[i]; DU2(i) = 0.f; }
  }
  for (int i = 0; i + 1 < n; ++i) {
    const float di = DD(i), li = DL(i);
    if (fabsf(di) >= fabsf(li)) {
      const float dv = (di == 0.f) ? tiny : di;
      DD(i) = dv;
      const float f = li / dv;
      DL(i) = f;
      DD(i + 1) = DD(i + 1) - f * DU(i);
      PV(i) = 0;
    } else {
      const float f = di / li;
      DD(i) = li;
      DL(i) = f;
      const float tmp = DU(i);
      const float dn = DD(i + 1);
      DU(i) = dn;
      DD(i + 1) = tmp - f * dn;
      if (i + 2 < n) {
        DU2(i) = DU(i + 1);
        DU(i + 1) = -f * DU(i + 1);
      }
      PV(i) = 1;
    }
  }
  if (DD(n - 1) == 0.f) DD(n - 1) = tiny;
  // start vector: ones with a small deterministic perturbation
  for (int i = 0; i < n; ++i) {
    unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)(c * 40503u + 0x9e3779b9u);
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    *zslot(A, ld, n, c, i) = 1.f + 0.25f * ((float)(h & 0xffff) / 65536.f - 0.5f);
  }
  for (int rep = 0; rep < 3; ++rep) {
    // forward (row interchanges as recorded)
    for (int i = 0; i + 1 < n; ++i) {
      float* bi = zslot(A, ld, n, c, i);
      float* bj = zslot(A, ld, n, c, i + 1);
      if (!PV(i)) {
        *bj = *bj - DL(i) * *bi;
      } else {
        const float tmp = *bi;
        *bi = *bj;
        *bj = tmp - DL(i) * *bi;
      }
    }
    // backward
    float x2 = 0.f, x1 = 0.f;  // z[i+2], z[i+1]
    for (int i = n - 1; i >= 0; --i) {
      float* bi = zslot(A, ld, n, c, i);
      float v = *bi;
      if (i + 1 < n) v -= DU(i) * x1;
      if (i + 2 < n) v -= DU2(i) * x2;
      v /= DD(i);
      *bi = v;
      x2 = x1;
      x1 = v;
    }
    // normalise (max-norm first to stay in range)
    float mx = 0.f;
    for (int i = 0; i < n; ++i) mx = fmaxf(mx, fabsf(*zslot(A, ld, n, c, i)));
    const float inv = (mx > 0.f) ? 1.f / mx : 1.f;
    float s2 = 0.f;
    for (int i = 0; i < n; ++i) {
      float* bi = zslot(A, ld, n, c, i);
      const float v = *bi * inv;
      *bi = v;
      s2 = fmaf(v, v, s2);
    }
    const float r = rsqrtf(fmaxf(s2, 1e-30f));
    for (int i = 0; i < n; ++i) *zslot(A, ld, n, c, i) *= r;
  }
#undef DD
#undef DU
#undef DU2
#undef DL
#undef PV
}

// Step 3b. Kept vectors 0..count-1 orthonormal (classical Gram-Schmidt twice).
static __device__ void tri_orthonormalize(float* A, int ld, int n, int count, float* hbuf, float* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int c = 0; c < count; ++c) {
    for (int pass = 0; pass < 2 && c > 0; ++pass) {
      for (int cp = warp; cp < c; cp += nwarps) {
        float s = 0.f;
        for (int i = lane; i < n; i += 32) s = fmaf(*zslot(A, ld, n, cp, i), *zslot(A, ld, n, c, i), s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) hbuf[cp] = s;
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) {
        float s = 0.f;
        for (int cp = 0; cp < c; ++cp) s = fmaf(hbuf[cp], *zslot(A, ld, n, cp, i), s);
        *zslot(A, ld, n, c, i) -= s;
      }
      __syncthreads();
    }
    float s = 0.f;
    for (int i = tid; i < n; i += nt) {
      const float v = *zslot(A, ld, n, c, i);
      s = fmaf(v, v, s);
    }
    const float ss = tri_block_sum(s, red);
    const float r = rsqrtf(fmaxf(ss, 1e-30f));
    for (int i = tid; i < n; i += nt) *zslot(A, ld, n, c, i) *= r;
    __syncthreads();
  }
}

// Step 3c. u_c = Q z_c = H_0 H_1 ... H_{n-3} z_c for every kept vector; each
// warp takes its own vectors through all reflectors (no barrier inside).
template <int VPW>
__device__ void tri_back_transform(float* A, int ld, int n, int count) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int k = n - 3; k >= 0; --k) {
    const int m = n - k - 1;
    const float* colk = A + (size_t)(k + 1) * ld + k;
    float g[VPW];
#pragma unroll
    for (int q = 0; q < VPW; ++q) g[q] = 0.f;
    for (int i = lane; i < m; i += 32) {
      const float v = colk[(size_t)i * ld];
#pragma unroll
      for (int q = 0; q < VPW; ++q) {
        const int c = warp + q * nwarps;
        if (c < count) g[q] = fmaf(v, *zslot(A, ld, n, c, k + 1 + i), g[q]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < VPW; ++q) g[q] += __shfl_xor_sync(0xffffffffu, g[q], o);
    for (int i = lane; i < m; i += 32) {
      const float v2 = 2.f * colk[(size_t)i * ld];
#pragma unroll
      for (int q = 0; q < VPW; ++q) {
        const int c = warp + q * nwarps;
        if (c < count) {
          float* zp = zslot(A, ld, n, c, k + 1 + i);
          *zp = fmaf(-v2, g[q], *zp);
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// Shared-memory layout after A (bytes, 16-aligned pieces).
__host__ __device__ constexpr size_t tri_al16(size_t b) { return (b + 15) / 16 * 16; }
__host__ __device__ constexpr size_t tri_rest_bytes(int n, int NB) {
  return tri_al16((size_t)NB * n * 16) + tri_al16((size_t)NB * n)  // LU bands, pivots
         + tri_al16((size_t)n * 4 * 7 + 64 * 4)                    // d e e2 lam vb pb hbuf, red
         + tri_al16((size_t)n * 16) + tri_al16((size_t)n * 8);       // mu mup, rrank pos
}
// Shared-memory bytes the tridiagonal eigensolve needs for n = 2*ell rows
// with NB vectors per inverse-iteration batch (A has stride n | 1).
__host__ __device__ constexpr size_t tri_smem_bytes(int n, int NB) {
  return tri_al16((size_t)n * (size_t)(n | 1) * 4) + tri_rest_bytes(n, NB);
}

// The whole eigensolve + shrink + rotate-matrix write for a full buffer of
// n = 2*ell rows whose Gram is already in A (n x ld, scaled by 1/smax).
template <int NB, int VPW>
__device__ void tri_eig_shrink(const EigArgs& a, float* A, int ld, int n, double smax,
                               unsigned char* rest) {
  const int tid = threadIdx.x, nt = blockDim.x;
  float* scr = reinterpret_cast<float*>(rest);
  unsigned char* piv = rest + tri_al16((size_t)NB * n * 16);
  float* fv = reinterpret_cast<float*>(piv + tri_al16((size_t)NB * n));
  float* d = fv;
  float* e = d + n;
  float* e2 = e + n;
  float* lam = e2 + n;
  float* vb = lam + n;
  float* pb = vb + n;
  float* hbuf = pb + n;
  float* red = hbuf + n;  // 64 floats
  double* mu = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(fv) +
                                         tri_al16((size_t)n * 4 * 7 + 64 * 4));
  double* mup = mu + n;
  int* rrank = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(mu) + tri_al16((size_t)n * 16));
  int* pos = rrank + n;
  __shared__ float s_tnorm;
  __shared__ int s_count;
  __shared__ double s_dsum, s_dlast;

  tri_reduce(A, ld, n, d, e, vb, pb, red);
  tri_bisect(d, e, e2, n, lam, &s_tnorm);
  for (int k = tid; k < n; k += nt) mu[k] = fmax((double)lam[k], 0.0) * smax;
  __syncthreads();
  shrink_sorted(a, n, n, 1.1920928955078125e-07, mu, mup, rrank, &s_count, &s_dsum, &s_dlast);
  const int nout = a.ell - 1;
  const int count = s_count < nout ? s_count : nout;
  for (int k = tid; k < n; k += nt) {
    const int r = rrank[k];
    if (r >= 0 && r < nout) pos[r] = k;
  }
  __syncthreads();
  const float tnorm = s_tnorm;
  for (int c0 = 0; c0 < count; c0 += NB) {
    tri_invit_batch<NB>(A, ld, n, d, e, lam, pos, c0, count, tnorm, scr, piv);
    __syncthreads();
  }
  tri_orthonormalize(A, ld, n, count, hbuf, red);
  tri_back_transform<VPW>(A, ld, n, count);
  // rotate-matrix rows: row r = sqrt(mu'/mu) u_r, zero rows past the count
  float* wr = reinterpret_cast<float*>(a.wrot);
  for (int idx = tid; idx < nout * n; idx += nt) {
    const int r = idx / n, i = idx - r * n;
    float v = 0.f;
    if (r < count) {
      const int k = pos[r];
      const double sc = (mu[k] > 0.0) ? sqrt(mup[k] / mu[k]) : 0.0;
      v = (float)(sc * (double)*zslot(A, ld, n, r, i));
    }
    wr[(size_t)r * a.ldr + i] = v;
    if (a.wrot_hi) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      a.wrot_hi[(size_t)r * a.ldr16 + i] = hi;
      a.wrot_lo[(size_t)r * a.ldr16 + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  }
  __syncthreads();
  write_counters(a, n, mu, mup, s_count, s_dsum, s_dlast, 0, 1);
}

}  // namespace fdk
