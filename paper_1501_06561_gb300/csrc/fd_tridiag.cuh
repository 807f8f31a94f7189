// Symmetric eigensolve of the n x n buffer Gram (a full buffer, n >= 2*ell) in
// FP32 on one CTA, for the ReduceRank step of Sec. 2.3. Only the retained
// directions need eigenvectors, so the solve is split:
//
//   1. Householder reduction T = Q^T G Q (n-2 reflectors). Step s computes
//      p = A22 v, K = v^T p, q = 2 (p - K v) and A22 <- A22 - v q^T - q v^T.
//      The update of step s and the product A33 v_{s+1} of step s+1 share one
//      pass over the trailing block (the next reflector is formed from the
//      updated column first), so each step costs one read and one write of
//      the trailing block and two barriers. Reflector vectors are packed, in
//      step order, into the finished leading rows of the same buffer. The
//      last 32 steps run on one warp with the block in registers.
//   2. Eigenvalues of T from Sturm counts of T - x I (LDL^T pivots): one
//      count per thread on an even grid brackets every eigenvalue, then
//      groups of lanes refine each bracket by multisection to a width of
//      2 eps |lambda| (relative accuracy). Only the ell+1 largest are solved
//      unless SS or a recorded spectrum needs all of them. Values at or below
//      2 eps lambda_1 count as zero.
//   3. For each retained position r, an eigenvector of T from a twisted
//      factorisation of T - lambda_r I (forward and backward LDL^T pivots,
//      twist index at the smallest |gamma|): one thread per vector, O(n).
//   4. One Cholesky-QR pass (C = Z^T Z = L L^T, Z <- Z L^-T) makes the
//      vectors orthonormal. If C has a pivot below 1/4 (vectors too close to
//      dependent, e.g. a multiple eigenvalue), the members of each tight
//      group of eigenvalues are recomputed by two rounds of block inverse
//      iteration from independent starts and made orthonormal within the
//      group, and Cholesky-QR runs again; if a twisted vector failed or that
//      fails too, every vector is recomputed by inverse iteration and
//      orthonormalised by classical Gram-Schmidt twice.
//   5. u_r = Q z_r = H_0 ... H_{n-3} z_r with each thread holding a strided
//      slice of one vector in registers; the rotate matrix rows
//      sqrt(mu'_r / mu_r) u_r go straight to their destination, or (step 6)
//      the raw vectors go to a global scratch.
//   6. Rayleigh-Ritz with the saved original G for positions 0..ell (FD,
//      PFD, iSVD): H = U^T G U with compensated sums, Jacobi rotations on H,
//      the Ritz values in place of T's eigenvalues for the shrink, and the
//      rotate matrix from the rotated vectors. SS instead scales its rows by
//      the Rayleigh quotients of its vectors.
//
// Memory: A (n x ld floats, ld >= n) holds G on entry; afterwards its front
// holds the packed reflectors (n(n-1)/2 floats) and, from tri_zoff(n), the
// eigenvector block Zt (n x ldz, column r = vector r). The `rest` region
// holds a scratch area first (LU bands, the Cholesky matrix, bisection
// counts; dead when the rotate matrix is written, so a caller may point the
// rotate output at it), then the spectra and small vectors.
#pragma once

#include "fd_eig.cuh"
#include "fd_internal.cuh"

namespace fdk {

constexpr int TRI_CPT = 4;  // trailing-block columns per thread in step 1

__host__ __device__ constexpr size_t tri_al16(size_t b) { return (b + 15) / 16 * 16; }
// offset (floats) of reflector s (length n-1-s) in the packed store
__host__ __device__ constexpr int tri_voff(int n, int s) { return s * (n - 1) - (s * (s - 1)) / 2; }
// offset (floats) of the eigenvector block inside the A region
__host__ __device__ constexpr int tri_zoff(int n) { return (n * (n - 1) / 2 + 3) & ~3; }
__host__ __device__ constexpr int tri_ldz(int count) { return count | 1; }

// rest-region pieces (bytes)
__host__ __device__ constexpr size_t tri_scratch_bytes(int n, int NB) {
  // max of: LU bands + pivots (NB vectors); Cholesky matrix + inverse diagonal
  // (count <= n/2) and the Sturm counts of the grid pass (<= 1024 threads)
  // (count <= n/2 + 1: the retained vectors and the one at the cut)
  return (tri_al16((size_t)NB * n * 16) + tri_al16((size_t)NB * n)) >
                 tri_al16((size_t)(n / 2 + 1) * ((n / 2 + 1) | 1) * 4) +
                     tri_al16((size_t)(n / 2 + 1) * 4) + 4096
             ? tri_al16((size_t)NB * n * 16) + tri_al16((size_t)NB * n)
             : tri_al16((size_t)(n / 2 + 1) * ((n / 2 + 1) | 1) * 4) +
                   tri_al16((size_t)(n / 2 + 1) * 4) + 4096;
}
// floats of the small-vector region: red (64), five vectors of 8*ceil(n/8)
// (xb, vb0, vb1, qb, pb), d, e, e2, lam (n each)
__host__ __device__ constexpr size_t tri_fv_floats(int n) {
  return 64 + 5 * (size_t)((n + 7) & ~7) + 4 * (size_t)n;
}
// the small-vector region (always in shared memory)
__host__ __device__ constexpr size_t tri_small_bytes(int n) {
  return tri_al16((size_t)n * 16)              // mu, mup
         + tri_al16(tri_fv_floats(n) * 4)      // small vectors
         + tri_al16((size_t)(2 * n + 16) * 4); // rrank pos
}
__host__ __device__ constexpr size_t tri_rest_bytes(int n, int NB) {
  return tri_scratch_bytes(n, NB) + tri_small_bytes(n);
}
// Global-memory workspace of the solve when A and the scratch area do not fit
// in shared memory (n x (n|1) floats, then the scratch area).
__host__ __device__ constexpr size_t tri_global_bytes(int n, int NB) {
  return tri_al16((size_t)n * (size_t)(n | 1) * 4) + tri_scratch_bytes(n, NB);
}
// Step-1 workspace in shared memory: two packed (v, q, x) arrays of n float4
// and the row groups' partial products (at most nw * min(n, 32 TRI_CPT)
// floats). It is dead once step 1 ends, so it may share the scratch area.
__host__ __device__ constexpr size_t tri_rw_bytes(int n, int nw) {
  return 2 * tri_al16((size_t)n * 16) +
         tri_al16((size_t)nw * (size_t)(n < 32 * TRI_CPT ? n : 32 * TRI_CPT) * 4);
}
// Shared-memory bytes of the whole solve for n rows (A with stride n | 1).
__host__ __device__ constexpr size_t tri_smem_bytes(int n, int NB) {
  return tri_al16((size_t)n * (size_t)(n | 1) * 4) + tri_rest_bytes(n, NB);
}

// ---------------------------------------------------------------------------
// Step 1. d (n) and e (n-1) receive T; red: 64 floats (16-byte aligned);
// rw: tri_rw_bytes(n, warps) bytes of shared memory (16-byte aligned).
// ---------------------------------------------------------------------------
// Sum of the first nw (<= 32) floats of a 16-byte aligned shared array:
// four-wide loads and a tree, so the result waits on one load latency
// instead of nw dependent ones.
__device__ __forceinline__ float tri_sum_parts(const float* p, int nw) {
  float s[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (4 * q < nw) {
      const float4 v = reinterpret_cast<const float4*>(p)[q];
      s[q] = (4 * q + 3 < nw) ? (v.x + v.y) + (v.z + v.w)
                              : v.x + (4 * q + 1 < nw ? v.y : 0.f) + (4 * q + 2 < nw ? v.z : 0.f);
    } else {
      s[q] = 0.f;
    }
  }
  return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// One pass over the trailing block T (m x m, row stride ld) by the warps of
// row group g (rows g, g + G, ...): apply the previous step's update
// a_rc -= v_r q_c + q_r v_c and accumulate the column sums sum_r a_rc xh_r
// of the updated block for U columns per thread (c0 + cs u). Pc[r] holds
// (v_r, q_r, x_r) of the previous reflector and the current column; row 0
// weighs xh0 instead of x_0. The symmetric block gives p = A v from column
// sums, so no lane-to-lane reduction is needed. Writes the group's partial
// p_c to pp[g m + c] and returns this thread's share of v^T p.
template <int U>
__device__ __forceinline__ float tri_pass(float* T, int ld, int m, const float4* Pc, float* pp,
                                          int g, int G, int c0, int cs, float xh0, float scale) {
  float vc[U], qc[U], wc[U], acc[U];
  int col[U];
  bool live[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = c0 + cs * u;
    live[u] = c < m;
    col[u] = live[u] ? c : m - 1;
    const float4 pc = Pc[col[u]];
    vc[u] = live[u] ? pc.x : 0.f;
    qc[u] = live[u] ? pc.y : 0.f;
    wc[u] = (c == 0) ? xh0 : pc.z;
    acc[u] = 0.f;
  }
  int r = g;
  if (g == 0) {  // row 0 weighs x_0 - alpha
    const float4 pr = Pc[0];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float a = T[col[u]];
      a = fmaf(-pr.x, qc[u], fmaf(-pr.y, vc[u], a));
      if (live[u]) T[col[u]] = a;
      acc[u] = fmaf(a, xh0, acc[u]);
    }
    r = G;
  }
  for (; r + G < m; r += 2 * G) {  // two rows at a time: all loads first
    const float4 p0 = Pc[r], p1 = Pc[r + G];
    float* row0 = T + (size_t)r * ld;
    float* row1 = row0 + (size_t)G * ld;
    float a0[U], a1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a0[u] = row0[col[u]];
      a1[u] = row1[col[u]];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a0[u] = fmaf(-p0.x, qc[u], fmaf(-p0.y, vc[u], a0[u]));
      a1[u] = fmaf(-p1.x, qc[u], fmaf(-p1.y, vc[u], a1[u]));
      if (live[u]) {
        row0[col[u]] = a0[u];
        row1[col[u]] = a1[u];
      }
      acc[u] = fmaf(a1[u], p1.z, fmaf(a0[u], p0.z, acc[u]));
    }
  }
  if (r < m) {
    const float4 pr = Pc[r];
    float* row = T + (size_t)r * ld;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float a = row[col[u]];
      a = fmaf(-pr.x, qc[u], fmaf(-pr.y, vc[u], a));
      if (live[u]) row[col[u]] = a;
      acc[u] = fmaf(a, pr.z, acc[u]);
    }
  }
  float kp = 0.f;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (live[u]) {
      const float p = acc[u] * scale;
      pp[g * m + col[u]] = p;
      kp = fmaf(wc[u] * scale, p, kp);
    }
  }
  return kp;
}

// sum_g pp[g m + i] over the G (<= 16) row groups: independent loads, tree sum
__device__ __forceinline__ float tri_group_sum(const float* pp, int m, int i, int G) {
  float t[16];
#pragma unroll
  for (int g = 0; g < 16; ++g) t[g] = (g < G) ? pp[g * m + i] : 0.f;
#pragma unroll
  for (int h = 8; h > 0; h >>= 1)
#pragma unroll
    for (int g = 0; g < h; ++g) t[g] += t[g + h];
  return t[0];
}

// a / b for b in 1..4 without a division instruction
__device__ __forceinline__ int tri_div14(int a, int b) {
  return (b == 1) ? a : (b == 2) ? (a >> 1) : (b == 4) ? (a >> 2) : a / 3;
}

// The last steps (trailing block of m0 <= 32) on warp 0 alone, with no block
// barriers. Lane j holds column s0+1+j of the block in registers (a[i] = row
// s0+1+i). Entry state is that of the block-wide loop at the top of step s0:
// the block still lacks step s0-1's update, which Pc carries as (v, q) per
// row, and Pc[r].z is x_{s0}. At step s0+k the column x_s is, by symmetry,
// row s of the block: register a[k-1] of every lane. v_i and q_i of other
// rows come by shuffle from lane i. Writes e, d (from s0+1) and the packed
// reflectors; the shared-memory copy of the block is left stale.
__device__ __forceinline__ void tri_reduce_tail(float* A, int ld, int n, int s0, const float4* Pc,
                                                float* d, float* e) {
  constexpr unsigned FULL = 0xffffffffu;
  const int j = threadIdx.x & 31;
  const int m0 = n - 1 - s0;
  const bool lj = j < m0;
  const float4 pj = Pc[lj ? j : 0];
  const float vj = lj ? pj.x : 0.f, qj = lj ? pj.y : 0.f;
  float x = lj ? pj.z : 0.f;
  const float* T = A + (size_t)(s0 + 1) * ld + (s0 + 1);
  float a[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float v = 0.f;
    if (i < m0 && lj) {
      const float4 pi = Pc[i];
      v = fmaf(-pi.x, qj, fmaf(-pi.y, vj, T[(size_t)i * ld + j]));
    }
    a[i] = v;
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k >= m0) break;
    const int s = s0 + k, m = m0 - k;
    if (k > 0) x = a[k - 1];
    if (j < k) x = 0.f;
    const float x0 = __shfl_sync(FULL, x, k);
    const float ss = warp_sum(x * x);
    float alpha = x0, scale = 0.f;  // a length-1 (or zero) column needs no reflection
    if (m > 1 && ss > 0.f) {
      const float nx = sqrtf(ss);
      alpha = (x0 >= 0.f) ? -nx : nx;
      scale = 1.f / sqrtf(2.f * (ss - x0 * alpha));
    }
    if (j == 0) e[s] = alpha;
    const float v = (j >= k) ? ((j == k) ? x - alpha : x) * scale : 0.f;
    if (m > 1 && j >= k) A[tri_voff(n, s) + (j - k)] = v;
    float p = 0.f;
#pragma unroll
    for (int i = k; i < 32; ++i) p = fmaf(a[i], __shfl_sync(FULL, v, i), p);
    const float K = warp_sum(v * p);
    const float q = (j >= k) ? 2.f * fmaf(-K, v, p) : 0.f;
#pragma unroll
    for (int i = k; i < 32; ++i) {
      const float vi = __shfl_sync(FULL, v, i), qi = __shfl_sync(FULL, q, i);
      a[i] = fmaf(-vi, q, fmaf(-qi, v, a[i]));
    }
    if (j == k) d[s + 1] = a[k];
  }
}

// Reflector of a column x with ||x||^2 = ss and first entry x0 (length m):
// alpha = -sign(x0) ||x||, scale = 1 / ||x - alpha e_1||; a length-1 (or
// zero) column needs no reflection (alpha = x0, scale = 0).
__device__ __forceinline__ float4 tri_reflector(float ss, float x0, int m) {
  float alpha = x0, scale = 0.f;
  if (m > 1 && ss > 0.f) {
    const float nx = sqrtf(ss);
    alpha = (x0 >= 0.f) ? -nx : nx;
    scale = 1.f / sqrtf(2.f * (ss - x0 * alpha));
  }
  return make_float4(alpha, scale, x0 - alpha, 0.f);
}

static __device__ void tri_reduce(float* A, int ld, int n, float* d, float* e, unsigned char* rw,
                                  float* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  float4* P0 = reinterpret_cast<float4*>(rw);
  float4* P1 = reinterpret_cast<float4*>(rw + tri_al16((size_t)n * 16));
  float* pp = reinterpret_cast<float*>(rw + 2 * tri_al16((size_t)n * 16));
  float* kpart = red;                                  // per-warp parts of K = v^T p
  float4* scal = reinterpret_cast<float4*>(red + 32);  // (alpha, scale, x0 - alpha) of the step
  if (tid == 0) d[0] = A[0];
  for (int i = tid; i < n - 1; i += nt)
    P0[i] = make_float4(0.f, 0.f, A[(size_t)(i + 1) * ld], 0.f);  // no previous step to apply
  __syncthreads();
  if (warp == 0 && n - 1 > 32) {
    float sq = 0.f;
    for (int i = lane; i < n - 1; i += 32) sq = fmaf(P0[i].z, P0[i].z, sq);
    const float4 r = tri_reflector(warp_sum(sq), P0[0].z, n - 1);
    if (lane == 0) *scal = r;
  }
  __syncthreads();
  for (int s = 0; s + 1 < n; ++s) {
    const int m = n - 1 - s;  // length of x_s = size of the trailing block
    const float4* Pc = (s & 1) ? P1 : P0;
    float4* Pn = (s & 1) ? P0 : P1;
    if (m <= 32) {  // the rest on one warp, in registers
      if (warp == 0) tri_reduce_tail(A, ld, n, s, Pc, d, e);
      __syncthreads();
      return;
    }
    // reflector s: v = (x - alpha e_1) * scale, from the scalars warp 0 wrote
    const float4 sc = *scal;
    const float alpha = sc.x, scale = sc.y, xh0 = sc.z;
    if (tid == 0) e[s] = alpha;
    {
      float* vpk = A + tri_voff(n, s);  // inside rows 0..s, which are finished
      for (int i = tid; i < m; i += nt) vpk[i] = ((i == 0) ? xh0 : Pc[i].z) * scale;
    }
    // trailing block rows/cols s+1..n-1: CW warps cover its columns (TRI_CPT
    // per thread), G groups of CW warps split its rows
    static_assert(TRI_CPT == 4, "the group arithmetic assumes 1 <= CW <= 4");
    const int CW = (m + 32 * TRI_CPT - 1) / (32 * TRI_CPT);
    const int G = tri_div14(nw, CW);
    {
      const int g = tri_div14(warp, CW), cb = warp - g * CW;
      float kp = 0.f;
      if (g < G) {
        const int cs = 32 * CW, c0 = 32 * cb + lane;
        int nu = 0;  // live column chunks of this warp: warp-uniform, >= 1
#pragma unroll
        for (int u = 0; u < TRI_CPT; ++u) nu += (32 * cb + cs * u < m);
        float* T = A + (size_t)(s + 1) * ld + (s + 1);
        if (nu == 4)      kp = tri_pass<4>(T, ld, m, Pc, pp, g, G, c0, cs, xh0, scale);
        else if (nu == 3) kp = tri_pass<3>(T, ld, m, Pc, pp, g, G, c0, cs, xh0, scale);
        else if (nu == 2) kp = tri_pass<2>(T, ld, m, Pc, pp, g, G, c0, cs, xh0, scale);
        else              kp = tri_pass<1>(T, ld, m, Pc, pp, g, G, c0, cs, xh0, scale);
      }
      kp = warp_sum(kp);
      if (lane == 0) kpart[warp] = kp;
    }
    __syncthreads();
    // warp 0: q_s = 2 (p - K v), column s+1 updated by step s (its diagonal is
    // d[s+1], the rest is x_{s+1}; (v_s, q_s, x_{s+1}) go to Pn shifted by
    // one), and the scalars of reflector s+1. One warp does it so that the
    // norm needs no block-wide reduction and the scalars are computed once.
    if (warp == 0) {
      const float K = tri_sum_parts(kpart, nw);
      const float v0 = xh0 * scale;
      const float q0 = 2.f * fmaf(-K, v0, tri_group_sum(pp, m, 0, G));
      float sq = 0.f, x1 = 0.f;
#pragma unroll 4
      for (int i = lane; i < m; i += 32) {
        const float pi = tri_group_sum(pp, m, i, G);
        const float vi = (i == 0) ? v0 : Pc[i].z * scale;
        const float qi = 2.f * fmaf(-K, vi, pi);
        float a = A[(size_t)(s + 1 + i) * ld + (s + 1)];
        a = fmaf(-vi, q0, fmaf(-qi, v0, a));
        if (i == 0) {
          d[s + 1] = a;
        } else {
          Pn[i - 1] = make_float4(vi, qi, a, 0.f);
          sq = fmaf(a, a, sq);
          if (i == 1) x1 = a;
        }
      }
      const float ss = warp_sum(sq);
      x1 = __shfl_sync(0xffffffffu, x1, 1);  // m > 32: lane 1 holds i = 1
      const float4 r = tri_reflector(ss, x1, m - 1);
      if (lane == 0) *scal = r;
    }
    __syncthreads();
  }
  if (tid == 0) d[n - 1] = A[(size_t)(n - 1) * ld + (n - 1)];  // n == 1 only
  __syncthreads();
}

// Number of eigenvalues of T below x (signs of the LDL^T pivots of T - x I).
// A pivot smaller than pivmin in magnitude is replaced by -pivmin before its
// sign is counted, so that the count and the rest of the recurrence see the
// same pivot (counting a zero pivot as non-negative while dividing by
// -pivmin made the count drop by one where x equals a diagonal entry).
__device__ __forceinline__ int tri_sturm(const float* d, const float* e2, int n, float x,
                                         float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = (q < 0.f);
  int i = 1;
  for (; i + 7 < n; i += 8) {  // loads of a chunk first, then the pivot chain
    float dx[8], ee[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      dx[u] = d[i + u] - x;
      ee[u] = e2[i - 1 + u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      q = dx[u] - __fdividef(ee[u], q);
      if (fabsf(q) < pivmin) q = -pivmin;
      cnt += (q < 0.f);
    }
  }
  for (; i < n; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += (q < 0.f);
  }
  return cnt;
}

// ---------------------------------------------------------------------------
// Step 2. lam[j] = j-th largest eigenvalue of T for j < nl (0 for the rest).
// cnt: blockDim.x ints of scratch. Returns the Gershgorin bound of ||T||
// through *tnorm_out (shared).
// ---------------------------------------------------------------------------
static __device__ void tri_bisect(const float* d, const float* e, float* e2, int n, float* lam,
                                  float* tnorm_out, int* cnt, int nl) {
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
  const float glo = s_lo, ghi = s_hi;
  const float tnorm = fmaxf(fabsf(glo), fabsf(ghi));
  const float eps = 1.1920929e-07f;
  const float pivmin = fmaxf(tnorm, 1e-30f) * 1e-30f;
  const float atol = 2.f * eps * tnorm;
  const float lo0 = glo - 0.01f * (ghi - glo) - atol;
  const float hi0 = ghi + 0.01f * (ghi - glo) + atol;
  // Intervals are refined to a width of 2 eps |lambda| (relative), down to
  // pivmin-level absolute widths: the eigenvalues near the cut are small
  // against ||T||, and a twisted vector taken at a shift that is off by
  // eps ||T|| mixes in its neighbours at that scale, which the Rayleigh-Ritz
  // step cannot undo for neighbours outside its subspace. The FP32 Sturm
  // counts of T resolve those eigenvalues to relative accuracy. Widths of
  // eps^2 ||T|| end the refinement (values that small count as zero later).
  const float rtol_abs = fmaxf(eps * eps * tnorm, 1e3f * pivmin);
  const float h = (hi0 - lo0) / (float)(nt + 1);
  // grid pass: counts at lo0 + (p + 1) h, p = 0..nt-1 (non-decreasing in p)
  cnt[tid] = tri_sturm(d, e2, n, lo0 + (float)(tid + 1) * h, pivmin);
  __syncthreads();
  int G = 1;  // lanes per eigenvalue (power of two, <= 8)
  while (G < 8 && 2 * G * nl <= nt) G <<= 1;
  const int sub = tid & (G - 1);
  const int per = nt / G;
  for (int j = nl + tid; j < n; j += nt) lam[j] = 0.f;  // not needed by the caller
  for (int j0 = 0; j0 < nl; j0 += per) {
    const int j = j0 + tid / G;
    const bool act = j < nl;
    const int target = n - 1 - j;  // lambda_j is the target-th smallest (0-based)
    float lo = lo0, hi = hi0;
    if (act) {
      int a = -1, b = nt;  // count(x_a) <= target < count(x_b)
      while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (cnt[mid] <= target) a = mid; else b = mid;
      }
      if (a >= 0) lo = lo0 + (float)(a + 1) * h;
      if (b < nt) hi = lo0 + (float)(b + 1) * h;
    }
    for (int it = 0; it < 64; ++it) {
      const bool done = !act || (hi - lo <= rtol_abs + 2.f * eps * fmaxf(fabsf(lo), fabsf(hi)));
      if (__all_sync(0xffffffffu, done)) break;
      const float x = lo + (hi - lo) * (float)(sub + 1) / (float)(G + 1);
      const int c = act ? tri_sturm(d, e2, n, x, pivmin) : 0;
      float nlo = (c <= target) ? x : lo;
      float nhi = (c > target) ? x : hi;
      for (int o = 1; o < G; o <<= 1) {
        nlo = fmaxf(nlo, __shfl_xor_sync(0xffffffffu, nlo, o));
        nhi = fminf(nhi, __shfl_xor_sync(0xffffffffu, nhi, o));
      }
      if (!done) {
        lo = nlo;
        hi = nhi;
      }
    }
    if (act && sub == 0) lam[j] = 0.5f * (lo + hi);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Step 3. Eigenvector of T for eigenvalue lmb from the twisted factorisation
// of T - lmb I (one thread). z: n entries with stride ldz. Returns false if
// the vector came out zero or not finite.
//   forward pivots  D+_0 = d_0 - lmb,     D+_i = d_i - lmb - e_{i-1}^2 / D+_{i-1}
//   backward pivots D-_{n-1} = d_{n-1} - lmb, D-_i = d_i - lmb - e_i^2 / D-_{i+1}
//   gamma_r = D+_r - e_r^2 / D-_{r+1};  z_r = 1,
//   z_i = -e_i z_{i+1} / D+_i (i < r),  z_{i+1} = -e_i z_i / D-_{i+1} (i >= r)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tri_clamp_piv(float q, float pivmin) {
  return (fabsf(q) < pivmin) ? -pivmin : q;
}

static __device__ bool tri_twisted(const float* d, const float* e, const float* e2, int n,
                                   float lmb, float pivmin, float* z, int ldz) {
  // (each pass loads a chunk of 8 entries ahead of its recurrence)
  float dp = tri_clamp_piv(d[0] - lmb, pivmin);
  z[0] = dp;
  int i = 1;
  for (; i + 7 < n; i += 8) {
    float dx[8], ee[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      dx[u] = d[i + u] - lmb;
      ee[u] = e2[i - 1 + u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      dp = tri_clamp_piv(dx[u] - __fdividef(ee[u], dp), pivmin);
      z[(size_t)(i + u) * ldz] = dp;
    }
  }
  for (; i < n; ++i) {
    dp = tri_clamp_piv((d[i] - lmb) - __fdividef(e2[i - 1], dp), pivmin);
    z[(size_t)i * ldz] = dp;
  }
  float dm = tri_clamp_piv(d[n - 1] - lmb, pivmin);
  int r = n - 1;
  float best = fabsf(dp);
  i = n - 2;
  for (; i >= 7; i -= 8) {
    float dx[8], ee[8], zp[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      dx[u] = d[i - u] - lmb;
      ee[u] = e2[i - u];
      zp[u] = z[(size_t)(i - u) * ldz];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float q = __fdividef(ee[u], dm);
      const float g = fabsf(zp[u] - q);
      if (g < best) {
        best = g;
        r = i - u;
      }
      dm = tri_clamp_piv(dx[u] - q, pivmin);
    }
  }
  for (; i >= 0; --i) {
    const float q = __fdividef(e2[i], dm);
    const float g = fabsf(z[(size_t)i * ldz] - q);
    if (g < best) {
      best = g;
      r = i;
    }
    dm = tri_clamp_piv((d[i] - lmb) - q, pivmin);
  }
  // D-_i for i > r replace D+_i (no longer needed there)
  dm = tri_clamp_piv(d[n - 1] - lmb, pivmin);
  i = n - 1;
  for (; i - 7 > r; i -= 8) {
    float dx[8], ee[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      dx[u] = d[i - 1 - u] - lmb;
      ee[u] = e2[i - 1 - u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      z[(size_t)(i - u) * ldz] = dm;
      dm = tri_clamp_piv(dx[u] - __fdividef(ee[u], dm), pivmin);
    }
  }
  for (; i > r; --i) {
    z[(size_t)i * ldz] = dm;
    dm = tri_clamp_piv((d[i - 1] - lmb) - __fdividef(e2[i - 1], dm), pivmin);
  }
  z[(size_t)r * ldz] = 1.f;
  float s2 = 1.f, zz = 1.f;
  i = r - 1;
  for (; i >= 7; i -= 8) {
    float ee[8], dd[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ee[u] = e[i - u];
      dd[u] = z[(size_t)(i - u) * ldz];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      zz = -__fdividef(ee[u] * zz, dd[u]);
      z[(size_t)(i - u) * ldz] = zz;
      s2 = fmaf(zz, zz, s2);
    }
  }
  for (; i >= 0; --i) {
    zz = -__fdividef(e[i] * zz, z[(size_t)i * ldz]);
    z[(size_t)i * ldz] = zz;
    s2 = fmaf(zz, zz, s2);
  }
  zz = 1.f;
  i = r;
  for (; i + 8 < n; i += 8) {
    float ee[8], dd[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ee[u] = e[i + u];
      dd[u] = z[(size_t)(i + u + 1) * ldz];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      zz = -__fdividef(ee[u] * zz, dd[u]);
      z[(size_t)(i + u + 1) * ldz] = zz;
      s2 = fmaf(zz, zz, s2);
    }
  }
  for (; i + 1 < n; ++i) {
    zz = -__fdividef(e[i] * zz, z[(size_t)(i + 1) * ldz]);
    z[(size_t)(i + 1) * ldz] = zz;
    s2 = fmaf(zz, zz, s2);
  }
  if (!(s2 < 3.0e38f)) return false;
  const float inv = rsqrtf(s2);
  for (int k = 0; k < n; ++k) z[(size_t)k * ldz] *= inv;
  return true;
}

// ---------------------------------------------------------------------------
// Step 4. One Cholesky-QR pass over the columns of Zt (n x count, stride
// ldz): C = Zt^T Zt = L L^T (C: count x ldc, lower triangle; dinv: count),
// Zt <- Zt L^-T. Returns false, with Zt unchanged, if a pivot of C is below
// tau (uniform across the block).
// ---------------------------------------------------------------------------
template <int U>  // panel rows per lane: count <= 32 U
__device__ bool tri_cholqr(float* Zt, int ldz, int n, int count, float* C, int ldc, float* dinv,
                           float tau) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nb = (count + 3) >> 2;
  const int ntile = nb * (nb + 1) / 2;
  for (int t = tid; t < ntile; t += nt) {
    int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int a0 = 4 * ti, b0 = 4 * tj;
    float acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
#pragma unroll 4
    for (int i = 0; i < n; ++i) {
      const float* zr = Zt + (size_t)i * ldz;
      float za[4], zb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        za[q] = (a0 + q < count) ? zr[a0 + q] : 0.f;
        zb[q] = (b0 + q < count) ? zr[b0 + q] : 0.f;
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(za[p], zb[q], acc[p][q]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (a0 + p < count && b0 + q <= a0 + p) C[(size_t)(a0 + p) * ldc + b0 + q] = acc[p][q];
  }
  __syncthreads();
  // Right-looking Cholesky by panels of 8 columns. Warp 0 factors a panel in
  // registers (lane l holds rows j0 + l + 32 u), then all threads update the
  // trailing lower triangle with 4x4 tiles.
  __shared__ int s_ok;
  const int lane = tid & 31, warp = tid >> 5;
  for (int j0 = 0; j0 < count; j0 += 8) {
    const int jb = min(8, count - j0);
    if (warp == 0) {
      float P[U][8];
      int ok = 1;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = j0 + lane + 32 * u;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          P[u][jj] = (i < count && jj < jb && i >= j0 + jj) ? C[(size_t)i * ldc + j0 + jj] : 0.f;
      }
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        if (jj < jb) {
          const float piv = __shfl_sync(0xffffffffu, P[0][jj], jj);
          if (!(piv >= tau)) ok = 0;
          const float rinv = ok ? 1.f / sqrtf(piv) : 0.f;
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (lane + 32 * u > jj) P[u][jj] *= rinv;
          if (lane == 0) dinv[j0 + jj] = rinv;
#pragma unroll
          for (int kk = jj + 1; kk < 8; ++kk) {
            const float lk = __shfl_sync(0xffffffffu, P[0][jj], kk);  // l_{j0+kk, jj}
            if (kk < jb)
#pragma unroll
              for (int u = 0; u < U; ++u)
                if (lane + 32 * u >= kk) P[u][kk] = fmaf(-P[u][jj], lk, P[u][kk]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = j0 + lane + 32 * u;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (i < count && jj < jb && i > j0 + jj) C[(size_t)i * ldc + j0 + jj] = P[u][jj];
      }
      if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return false;  // same value in every thread
    // trailing update: C[i][k] -= sum_jj L[i][j0+jj] L[k][j0+jj], j0+jb <= k <= i < count
    const int t0 = j0 + jb;
    const int nb4 = (count - t0 + 3) >> 2;
    const int ntl = nb4 * (nb4 + 1) / 2;
    for (int t = tid; t < ntl; t += nt) {
      int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
      while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
      while (ti * (ti + 1) / 2 > t) --ti;
      const int tk = t - ti * (ti + 1) / 2;
      const int i0 = t0 + 4 * ti, k0 = t0 + 4 * tk;
      float acc16[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc16[p][q] = 0.f;
#pragma unroll
      for (int h = 0; h < 8; h += 4) {
        float li[4][4], lk[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            li[p][jj] = (i0 + p < count && h + jj < jb) ? C[(size_t)(i0 + p) * ldc + j0 + h + jj] : 0.f;
            lk[p][jj] = (k0 + p < count && h + jj < jb) ? C[(size_t)(k0 + p) * ldc + j0 + h + jj] : 0.f;
          }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc16[p][q] = fmaf(li[p][jj], lk[q][jj], acc16[p][q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = i0 + p, k = k0 + q;
          if (i < count && k <= i) C[(size_t)i * ldc + k] -= acc16[p][q];
        }
    }
    __syncthreads();
  }
  // Z <- Z L^{-T}, a forward substitution per row: q_c = (z_c - sum_{b<c}
  // q_b L_cb) / L_cc. T consecutive lanes share a row (T n <= nt). Columns go
  // in blocks of 8: the sum over earlier blocks is split between the T lanes
  // (each z_b loaded once for the 8 columns) and added by shuffles; every lane
  // then solves the block's 8 x 8 triangle alike and lane h = 0 writes it.
  // With fewer than four lanes per row the blocked form measured slower than
  // one thread per row (2*ell = 200: 71 vs 50 us), so it is used from four up.
  int T = 1;
  while (T < 8 && 2 * T * n <= nt) T <<= 1;
  if (T < 4) {
    for (int i = tid; i < n; i += nt) {
      float* zr = Zt + (size_t)i * ldz;
      for (int c = 0; c < count; ++c) {
        const float* Lc = C + (size_t)c * ldc;
        float a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = 0.f;
        a[0] = zr[c];
        int b = 0;
        for (; b + 7 < c; b += 8) {
          float zq[8], lq[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            zq[u] = zr[b + u];
            lq[u] = Lc[b + u];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) a[u] = fmaf(-zq[u], lq[u], a[u]);
        }
        for (; b < c; ++b) a[0] = fmaf(-zr[b], Lc[b], a[0]);
        zr[c] = (((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]))) * dinv[c];
      }
    }
    __syncthreads();
    return true;
  }
  const int rpp = nt / T;  // rows per pass
  for (int i0 = 0; i0 < n; i0 += rpp) {
    const int i = i0 + tid / T, h = tid % T;
    const bool act = i < n;
    float* zr = Zt + (size_t)(act ? i : 0) * ldz;
    for (int j0 = 0; j0 < count; j0 += 8) {
      const int jb = min(8, count - j0);
      float acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.f;
      if (act) {
        for (int b = h; b < j0; b += T) {
          const float zb = zr[b];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (u < jb) acc[u] = fmaf(zb, C[(size_t)(j0 + u) * ldc + b], acc[u]);
        }
      }
      for (int o = 1; o < T; o <<= 1)
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
      float zc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        zc[u] = 0.f;
        if (u < jb) {
          float v = (act ? zr[j0 + u] : 0.f) - acc[u];
#pragma unroll
          for (int w = 0; w < u; ++w) v = fmaf(-zc[w], C[(size_t)(j0 + u) * ldc + j0 + w], v);
          zc[u] = v * dinv[j0 + u];
        }
      }
      __syncwarp();  // every lane of the row has read z before it is overwritten
      if (act && h == 0)
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < jb) zr[j0 + u] = zc[u];
      __syncwarp();
    }
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Fallback of steps 3-4: inverse iteration from a random start for vectors
// list[c0 .. min(c0+NB, cend)-1] (c0 + t itself without a list; thread
// t < NB takes one): eigenvalue lam[pos[c]], (T - lambda I) z = z0 solved
// once by LU with partial pivoting, z0 eliminated during the factorisation.
// Divisions use the fast reciprocal: the solve only has to amplify the
// eigenvector direction. scr holds NB interleaved copies of the three bands
// of U (1/U_ii stored).
// ---------------------------------------------------------------------------
template <int NB>
__device__ void tri_invit_batch(float* Zt, int ldz, int n, const float* d, const float* e,
                                const float* lam, const int* pos, const int* list, int c0,
                                int cend, float tnorm, float* scr) {
  const int t = threadIdx.x;
  if (t >= NB || c0 + t >= cend) return;
  const int c = list ? list[c0 + t] : c0 + t;
  float* ru = scr;                      // 1 / U_ii
  float* du = scr + (size_t)NB * n;     // U_{i,i+1}
  float* du2 = scr + (size_t)2 * NB * n;  // U_{i,i+2} (fill from row swaps)
  float* z = Zt + c;
#define RU(i) ru[(size_t)(i) * NB + t]
#define DU(i) du[(size_t)(i) * NB + t]
#define DU2(i) du2[(size_t)(i) * NB + t]
#define Z(i) z[(size_t)(i) * ldz]
  const float eps = 1.1920929e-07f;
  const float tiny = eps * fmaxf(tnorm, 1e-30f);
  const float lmb = lam[pos[c]];
  // start vector: ones with a small deterministic perturbation (a hash of i, c)
  auto start = [c](int i) {
    unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)(c * 40503u + 0x9e3779b9u);
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    return 1.f + 0.25f * ((float)(h & 0xffff) / 65536.f - 0.5f);
  };
  // LU with partial pivoting of T - lmb I, the start vector eliminated along:
  // (dc, uc, u2c | zc) is the current row restricted to columns i, i+1, i+2
  float dc = d[0] - lmb, uc = (n > 1) ? e[0] : 0.f, u2c = 0.f, zc = start(0);
  for (int i = 0; i + 1 < n; ++i) {
    const float li = e[i];  // row i+1, column i
    const float dn = d[i + 1] - lmb, un = (i + 2 < n) ? e[i + 1] : 0.f, zn = start(i + 1);
    if (fabsf(dc) >= fabsf(li)) {
      const float dv = (dc == 0.f) ? tiny : dc;
      const float f = __fdividef(li, dv);
      RU(i) = __fdividef(1.f, dv);
      DU(i) = uc;
      DU2(i) = u2c;
      Z(i) = zc;
      dc = fmaf(-f, uc, dn);
      uc = fmaf(-f, u2c, un);
      zc = fmaf(-f, zc, zn);
    } else {  // row i+1 becomes the pivot row
      const float f = __fdividef(dc, li);
      RU(i) = __fdividef(1.f, li);
      DU(i) = dn;
      DU2(i) = un;
      Z(i) = zn;
      dc = fmaf(-f, dn, uc);
      uc = fmaf(-f, un, u2c);
      zc = fmaf(-f, zn, zc);
    }
    u2c = 0.f;
  }
  // back substitution, tracking the largest entry
  float x = zc * __fdividef(1.f, (dc == 0.f) ? tiny : dc), x2 = 0.f, mx = fabsf(x);
  Z(n - 1) = x;
  for (int i = n - 2; i >= 0; --i) {
    const float v = fmaf(-DU2(i), x2, fmaf(-DU(i), x, Z(i))) * RU(i);
    Z(i) = v;
    x2 = x;
    x = v;
    mx = fmaxf(mx, fabsf(v));
  }
  const float inv = (mx > 0.f) ? 1.f / mx : 1.f;
  float s2 = 0.f;
  for (int i = 0; i < n; ++i) {
    const float v = Z(i) * inv;
    Z(i) = v;
    s2 = fmaf(v, v, s2);
  }
  const float r = rsqrtf(fmaxf(s2, 1e-30f));
  for (int i = 0; i < n; ++i) Z(i) *= r;
#undef RU
#undef DU
#undef DU2
#undef Z
}

// Members of clusters for the fallback: the retained positions ordered by
// eigenvalue are split where neighbours are more than gtol apart; the members
// of every group of two or more go to list (thread 0; returns their number
// through *nlist, shared).
static __device__ void tri_cluster_members(const float* lam, const int* pos, int n, int count,
                                           float gtol, int* ord, int* list, int* nlist) {
  // ord: retained vectors by their position in the spectrum (the positions
  // pos[r] are distinct), one rank per thread
  for (int r = threadIdx.x; r < count; r += blockDim.x) {
    const int pr = pos[r];
    int rank = 0;
    for (int q = 0; q < count; ++q) rank += (pos[q] < pr);
    ord[rank] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nl = 0;
    for (int a = 0; a < count;) {
      int b = a + 1;
      while (b < count && lam[pos[ord[b - 1]]] - lam[pos[ord[b]]] <= gtol) ++b;
      if (b - a >= 2)
        for (int j = a; j < b; ++j) list[nl++] = ord[j];
      a = b;
    }
    *nlist = nl;
  }
  __syncthreads();
}

__device__ __forceinline__ float tri_block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// Fallback of step 4 for eigenvalues that bisection cannot tell apart.
// Columns are taken in order of their position in the spectrum; a group is a
// run of consecutive ones whose eigenvalues differ by at most gt. The group's
// first column keeps its twisted vector, the others start from pseudo-random
// vectors; then two rounds of block inverse iteration: every member takes one
// solve of (T - lambda I) z = z (LU with partial pivoting, one thread per
// member, NB at a time), and each group is made orthonormal again by two
// passes of classical Gram-Schmidt in its order. The group's columns then span
// its invariant subspace instead of repeating one vector.
// scr: NB x 3n floats; ord, gstart, mlist: count ints each; hbuf: count
// floats; red: block-sum scratch.
template <int NB>
__device__ void tri_tight_repair(float* Zt, int ldz, int n, const float* d, const float* e,
                                 const float* lam, const int* pos, int count, float gt,
                                 float tnorm, float* scr, int* ord, int* gstart, int* mlist,
                                 float* hbuf, float* red, int* s_ng) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int r = tid; r < count; r += nt) {
    const int pr = pos[r];
    int rank = 0;
    for (int q = 0; q < count; ++q) rank += (pos[q] < pr);
    ord[rank] = r;
  }
  __syncthreads();
  __shared__ int s_nm;
  if (tid == 0) {
    int ng = 0, nm = 0;
    for (int a = 0; a < count;) {
      int b = a + 1;
      while (b < count && lam[pos[ord[b - 1]]] - lam[pos[ord[b]]] <= gt) ++b;
      if (b - a >= 2) {
        gstart[2 * ng] = a;
        gstart[2 * ng + 1] = b;
        ++ng;
        for (int m = a; m < b; ++m) mlist[nm++] = ord[m];
      }
      a = b;
    }
    *s_ng = ng;
    s_nm = nm;
  }
  __syncthreads();
  const int ng = *s_ng, nm = s_nm;
  // pseudo-random starts for all but each group's first member
  for (int g = 0; g < ng; ++g) {
    const int a = gstart[2 * g], b = gstart[2 * g + 1];
    for (int idx = tid; idx < (b - a - 1) * n; idx += nt) {
      const int c = ord[a + 1 + idx / n], i = idx % n;
      unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)(c * 40503u + 0x7f4a7c15u);
      h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
      Zt[(size_t)i * ldz + c] = (float)(h & 0xffff) / 65536.f - 0.5f;
    }
  }
  __syncthreads();
  const float eps = 1.1920929e-07f;
  const float tiny = eps * fmaxf(tnorm, 1e-30f);
  for (int round = 0; round < 2; ++round) {
    for (int c0 = 0; c0 < nm; c0 += NB) {
      const int t = tid;
      if (t < NB && c0 + t < nm) {
        const int c = mlist[c0 + t];
        float* z = Zt + c;
        float* ru = scr;
        float* du = scr + (size_t)NB * n;
        float* du2 = scr + (size_t)2 * NB * n;
#define RU(i) ru[(size_t)(i) * NB + t]
#define DU(i) du[(size_t)(i) * NB + t]
#define DU2(i) du2[(size_t)(i) * NB + t]
        const float lmb = lam[pos[c]];
        float dc = d[0] - lmb, uc = (n > 1) ? e[0] : 0.f, u2c = 0.f, zc = z[0];
        for (int i = 0; i + 1 < n; ++i) {
          const float li = e[i];
          const float dn = d[i + 1] - lmb, un = (i + 2 < n) ? e[i + 1] : 0.f;
          const float zn = z[(size_t)(i + 1) * ldz];
          if (fabsf(dc) >= fabsf(li)) {
            const float dv = (dc == 0.f) ? tiny : dc;
            const float f = __fdividef(li, dv);
            RU(i) = __fdividef(1.f, dv); DU(i) = uc; DU2(i) = u2c; z[(size_t)i * ldz] = zc;
            dc = fmaf(-f, uc, dn); uc = fmaf(-f, u2c, un); zc = fmaf(-f, zc, zn);
          } else {
            const float f = __fdividef(dc, li);
            RU(i) = __fdividef(1.f, li); DU(i) = dn; DU2(i) = un; z[(size_t)i * ldz] = zn;
            dc = fmaf(-f, dn, uc); uc = fmaf(-f, un, u2c); zc = fmaf(-f, zn, zc);
          }
          u2c = 0.f;
        }
        float x = zc * __fdividef(1.f, (dc == 0.f) ? tiny : dc), x2 = 0.f, mx = fabsf(x);
        z[(size_t)(n - 1) * ldz] = x;
        for (int i = n - 2; i >= 0; --i) {
          const float v = fmaf(-DU2(i), x2, fmaf(-DU(i), x, z[(size_t)i * ldz])) * RU(i);
          z[(size_t)i * ldz] = v;
          x2 = x; x = v;
          mx = fmaxf(mx, fabsf(v));
        }
        const float inv = (mx > 0.f) ? 1.f / mx : 1.f;
        for (int i = 0; i < n; ++i) z[(size_t)i * ldz] *= inv;
#undef RU
#undef DU
#undef DU2
      }
      __syncthreads();
    }
    // each group orthonormal again, in its order (CGS, two passes)
    for (int g = 0; g < ng; ++g) {
      const int a = gstart[2 * g], b = gstart[2 * g + 1];
      for (int m = a; m < b; ++m) {
        const int c = ord[m];
        for (int pass = 0; pass < 2 && m > a; ++pass) {
          for (int q = a + warp; q < m; q += nw) {
            const int cp = ord[q];
            float sdot = 0.f;
            for (int i = lane; i < n; i += 32)
              sdot = fmaf(Zt[(size_t)i * ldz + cp], Zt[(size_t)i * ldz + c], sdot);
            sdot = warp_sum(sdot);
            if (lane == 0) hbuf[q - a] = sdot;
          }
          __syncthreads();
          for (int i = tid; i < n; i += nt) {
            float sacc = 0.f;
            for (int q = a; q < m; ++q) sacc = fmaf(hbuf[q - a], Zt[(size_t)i * ldz + ord[q]], sacc);
            Zt[(size_t)i * ldz + c] -= sacc;
          }
          __syncthreads();
        }
        float s2 = 0.f;
        for (int i = tid; i < n; i += nt) {
          const float v = Zt[(size_t)i * ldz + c];
          s2 = fmaf(v, v, s2);
        }
        const float ss = tri_block_sum(s2, red);
        const float rr = 1.f / sqrtf(fmaxf(ss, 1e-30f));
        for (int i = tid; i < n; i += nt) Zt[(size_t)i * ldz + c] *= rr;
        __syncthreads();
      }
    }
  }
}


// Fallback of step 4: columns 0..count-1 of Zt orthonormal by classical
// Gram-Schmidt, twice per column.
static __device__ void tri_cgs2(float* Zt, int ldz, int n, int count, float* hbuf, float* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int c = 0; c < count; ++c) {
    for (int pass = 0; pass < 2 && c > 0; ++pass) {
      for (int cp = warp; cp < c; cp += nw) {
        float s = 0.f;
        for (int i = lane; i < n; i += 32) s = fmaf(Zt[(size_t)i * ldz + cp], Zt[(size_t)i * ldz + c], s);
        s = warp_sum(s);
        if (lane == 0) hbuf[cp] = s;
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) {
        float s = 0.f;
        for (int cp = 0; cp < c; ++cp) s = fmaf(hbuf[cp], Zt[(size_t)i * ldz + cp], s);
        Zt[(size_t)i * ldz + c] -= s;
      }
      __syncthreads();
    }
    float s = 0.f;
    for (int i = tid; i < n; i += nt) {
      const float v = Zt[(size_t)i * ldz + c];
      s = fmaf(v, v, s);
    }
    const float ss = tri_block_sum(s, red);
    const float r = 1.f / sqrtf(fmaxf(ss, 1e-30f));
    for (int i = tid; i < n; i += nt) Zt[(size_t)i * ldz + c] *= r;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Step 5. u_c = H_0 H_1 ... H_{n-3} z_c and the rotate-matrix rows
// sqrt(mu'/mu) u_c. Thread (c, g) = (tid / R, tid % R) holds rows
// i = n-1-(g + R j), j < MAXJ, of vector c, so that the rows a reflector
// touches (i > s) are a prefix in j. Reflectors go four at a time: for the
// block H_{s-3} H_{s-2} H_{s-1} H_s z with a_k = v_{s-k},
//   h_k = a_k . z,  g_k = h_k - 2 sum_{j<k} g_j (a_k . a_j),  z -= 2 sum_k g_k a_k,
// the six products a_k . a_j of every block being formed first (mw: 6 per
// block). VPT: vectors per thread (1 or 2; with 2, each reflector load
// feeds both). Rows count..ell-2 of the output are zero.
// ---------------------------------------------------------------------------
template <int R, int MAXJ, int VPT>
__device__ void tri_back_write(const EigArgs& a, const float* V, int n, const float* Zt, int ldz,
                               int count, const double* mu, const double* mup, const int* pos,
                               float* mw, float* raw = nullptr, int ldraw = 0) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int nout = a.ell - 1;
  float* wr = reinterpret_cast<float*>(a.wrot);
  const int nblk = (n - 2 + 3) >> 2;  // reflectors 0..n-3, block b tops at n-3-4b
  for (int w = warp; w < nblk * 6; w += nw) {
    const int b = w / 6, p = w - 6 * (w / 6);
    const int k = (p == 0) ? 1 : (p < 3 ? 2 : 3);
    const int j = (p == 0) ? 0 : (p == 1 ? 0 : (p == 2 ? 1 : p - 3));
    const int sb = n - 3 - 4 * b;
    float sum = 0.f;
    if (sb - k >= 0) {
      const float* ak = V + tri_voff(n, sb - k) - (sb - k + 1);
      const float* aj = V + tri_voff(n, sb - j) - (sb - j + 1);
      for (int i = sb - j + 1 + lane; i < n; i += 32) sum = fmaf(ak[i], aj[i], sum);
    }
    sum = warp_sum(sum);
    if (lane == 0) mw[w] = sum;
  }
  __syncthreads();
  if constexpr (VPT == 1) {
  const int per = nt / R;
  for (int cb = 0; cb < count; cb += per) {  // uniform across the block
    const int c = cb + tid / R, g = tid % R;
    const bool act = c < count;
    float z[MAXJ];
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      const int i = n - 1 - (g + R * j);
      z[j] = (act && i >= 0) ? Zt[(size_t)i * ldz + c] : 0.f;
    }
    for (int b = 0; b < nblk; ++b) {
      const int sb = n - 3 - 4 * b;
      int je[4];
      const float* ap[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int sk = sb - k;
        je[k] = (sk >= 0) ? (n - 1 - sk - g + R - 1) / R : 0;  // rows i > sk: j < je[k]
        const int sc = sk >= 0 ? sk : 0;
        ap[k] = V + tri_voff(n, sc) - (sc + 1) + (n - 1 - g);  // a_k[i_j] = ap[k][-R j]
      }
      const int jmx = max(max(je[0], je[1]), max(je[2], je[3]));
      float h[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j0 = 0; j0 < MAXJ; j0 += 4) {
        if (j0 >= jmx) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          if (j < MAXJ) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float av = (j < je[k]) ? ap[k][-R * j] : 0.f;
              h[k] = fmaf(av, z[j], h[k]);
            }
          }
        }
      }
#pragma unroll
      for (int o = 1; o < R; o <<= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] += __shfl_xor_sync(0xffffffffu, h[k], o);
      const float* m6 = mw + 6 * b;
      const float g0 = h[0];
      const float g1 = h[1] - 2.f * g0 * m6[0];
      const float g2 = h[2] - 2.f * (g0 * m6[1] + g1 * m6[2]);
      const float g3 = h[3] - 2.f * (g0 * m6[3] + g1 * m6[4] + g2 * m6[5]);
      const float t[4] = {2.f * g0, 2.f * g1, 2.f * g2, 2.f * g3};
#pragma unroll
      for (int j0 = 0; j0 < MAXJ; j0 += 4) {
        if (j0 >= jmx) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          if (j < MAXJ) {
            float upd = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float av = (j < je[k]) ? ap[k][-R * j] : 0.f;
              upd = fmaf(t[k], av, upd);
            }
            z[j] -= upd;
          }
        }
      }
    }
    if (act && raw != nullptr) {
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        const int i = n - 1 - (g + R * j);
        if (i >= 0) raw[(size_t)c * ldraw + i] = z[j];
      }
    } else if (act) {
      const int k = pos[c];
      // sqrt(mu'/mu) in FP32: the rotate matrix itself is FP32
      const float sc = (mu[k] > 0.0) ? sqrtf((float)mup[k] / (float)mu[k]) : 0.f;
      if (a.row_mass && g == 0) a.row_mass[c] = mup[k];
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        const int i = n - 1 - (g + R * j);
        if (i >= 0) {
          const float val = sc * z[j];
          wr[(size_t)c * a.ldr + i] = val;
          if (a.wrot_hi) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(val);
            a.wrot_hi[(size_t)c * a.ldr16 + i] = hi;
            a.wrot_lo[(size_t)c * a.ldr16 + i] = __float2bfloat16_rn(val - __bfloat162float(hi));
          }
        }
      }
    }
  }
  } else {
  // thread (pair p, g): vectors 2p and 2p+1, rows i = n-1-(g + R j)
  const int per = nt / R;  // vector pairs per pass
  for (int cb = 0; cb < count; cb += 2 * per) {  // uniform across the block
    const int c0 = cb + 2 * (tid / R), g = tid % R;
    const bool act0 = c0 < count, act1 = c0 + 1 < count;
    float z0[MAXJ], z1[MAXJ];
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      const int i = n - 1 - (g + R * j);
      z0[j] = (act0 && i >= 0) ? Zt[(size_t)i * ldz + c0] : 0.f;
      z1[j] = (act1 && i >= 0) ? Zt[(size_t)i * ldz + c0 + 1] : 0.f;
    }
    for (int b = 0; b < nblk; ++b) {
      const int sb = n - 3 - 4 * b;
      int je[4];
      const float* ap[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int sk = sb - k;
        je[k] = (sk >= 0) ? (n - 1 - sk - g + R - 1) / R : 0;  // rows i > sk: j < je[k]
        const int sc = sk >= 0 ? sk : 0;
        ap[k] = V + tri_voff(n, sc) - (sc + 1) + (n - 1 - g);  // a_k[i_j] = ap[k][-R j]
      }
      // rows j < jall are touched by all four reflectors (none in a partial block)
      const int jall = (sb - 3 >= 0) ? je[0] : 0;
      const int jmx = max(max(je[0], je[1]), max(je[2], je[3]));
      float h0[4] = {0.f, 0.f, 0.f, 0.f}, h1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int jc = 0; jc < MAXJ; jc += 4) {
        if (jc >= jmx) break;
        if (jc + 4 <= jall) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = jc + u;
            if (j < MAXJ) {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float av = ap[k][-R * j];
                h0[k] = fmaf(av, z0[j], h0[k]);
                h1[k] = fmaf(av, z1[j], h1[k]);
              }
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = jc + u;
            if (j < MAXJ) {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float av = (j < je[k]) ? ap[k][-R * j] : 0.f;
                h0[k] = fmaf(av, z0[j], h0[k]);
                h1[k] = fmaf(av, z1[j], h1[k]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int o = 1; o < R; o <<= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          h0[k] += __shfl_xor_sync(0xffffffffu, h0[k], o);
          h1[k] += __shfl_xor_sync(0xffffffffu, h1[k], o);
        }
      const float* m6 = mw + 6 * b;
      float t0[4], t1[4];
      {
        const float g0 = h0[0];
        const float g1 = h0[1] - 2.f * g0 * m6[0];
        const float g2 = h0[2] - 2.f * (g0 * m6[1] + g1 * m6[2]);
        const float g3 = h0[3] - 2.f * (g0 * m6[3] + g1 * m6[4] + g2 * m6[5]);
        t0[0] = 2.f * g0; t0[1] = 2.f * g1; t0[2] = 2.f * g2; t0[3] = 2.f * g3;
      }
      {
        const float g0 = h1[0];
        const float g1 = h1[1] - 2.f * g0 * m6[0];
        const float g2 = h1[2] - 2.f * (g0 * m6[1] + g1 * m6[2]);
        const float g3 = h1[3] - 2.f * (g0 * m6[3] + g1 * m6[4] + g2 * m6[5]);
        t1[0] = 2.f * g0; t1[1] = 2.f * g1; t1[2] = 2.f * g2; t1[3] = 2.f * g3;
      }
#pragma unroll
      for (int jc = 0; jc < MAXJ; jc += 4) {
        if (jc >= jmx) break;
        if (jc + 4 <= jall) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = jc + u;
            if (j < MAXJ) {
              float u0 = 0.f, u1 = 0.f;
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float av = ap[k][-R * j];
                u0 = fmaf(t0[k], av, u0);
                u1 = fmaf(t1[k], av, u1);
              }
              z0[j] -= u0;
              z1[j] -= u1;
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = jc + u;
            if (j < MAXJ) {
              float u0 = 0.f, u1 = 0.f;
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float av = (j < je[k]) ? ap[k][-R * j] : 0.f;
                u0 = fmaf(t0[k], av, u0);
                u1 = fmaf(t1[k], av, u1);
              }
              z0[j] -= u0;
              z1[j] -= u1;
            }
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = c0 + h;
      if (c < count && raw != nullptr) {
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) {
          const int i = n - 1 - (g + R * j);
          if (i >= 0) raw[(size_t)c * ldraw + i] = h ? z1[j] : z0[j];
        }
      } else if (c < count) {
        const int k = pos[c];
        const float sc = (mu[k] > 0.0) ? sqrtf((float)mup[k] / (float)mu[k]) : 0.f;
        if (a.row_mass && g == 0) a.row_mass[c] = mup[k];
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) {
          const int i = n - 1 - (g + R * j);
          if (i >= 0) {
            const float val = sc * (h ? z1[j] : z0[j]);
            wr[(size_t)c * a.ldr + i] = val;
            if (a.wrot_hi) {
              const __nv_bfloat16 hi = __float2bfloat16_rn(val);
              a.wrot_hi[(size_t)c * a.ldr16 + i] = hi;
              a.wrot_lo[(size_t)c * a.ldr16 + i] = __float2bfloat16_rn(val - __bfloat162float(hi));
            }
          }
        }
      }
    }
  }
  }
  if (raw != nullptr) {
    __syncthreads();
    return;
  }
  if (a.row_mass)
    for (int r = count + tid; r < nout; r += nt) a.row_mass[r] = 0.0;
  for (int idx = tid; idx < (nout - count) * n; idx += nt) {
    const int r = count + idx / n, i = idx % n;
    wr[(size_t)r * a.ldr + i] = 0.f;
    if (a.wrot_hi) {
      a.wrot_hi[(size_t)r * a.ldr16 + i] = __float2bfloat16_rn(0.f);
      a.wrot_lo[(size_t)r * a.ldr16 + i] = __float2bfloat16_rn(0.f);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Step 6 (refinement): Rayleigh-Ritz with the original G. The reflectors of
// step 1 carry rounding errors of about eps ||G||, so the eigenvalues of T near
// the cut, small against ||G||, are off by that much, and the vectors of
// eigenvalues closer than that mix (the fallback of step 4 only makes such
// groups orthonormal). The shrink sigma'^2 = sigma^2 - delta takes the
// difference of two of these eigenvalues. In the basis U of the P vectors
// the projected matrix H = U^T G U is diagonal up to those mixings; its
// entries are sums of products of G with the vectors, rounded relative to the
// terms they add, which are small where a vector is small along the large
// rows of G. H is diagonalised by Jacobi rotations (U rotated alongside), and
// its diagonal gives the eigenvalues.
//   Us: n x ldu floats (shared or global; ldu = P rounded up to 4), the
//   vectors transposed (Us[k * ldu + c] = u_c[k]); H: P x ldh floats after it;
//   Y: n x ldu floats of global scratch (G U); G: the scaled Gram as loaded,
//   row stride ldg (a multiple of 4); uvec: P rows of n floats (global).
// G U and U^T (G U) are formed from 32-term FP32 chunks added by a
// compensated (two-sum) FP32 accumulation. Rotation (p, q), for columns at
// most 32 apart in spectral order, is taken when |H_pq| > 1e-2 |H_pp - H_qq|
// and above the FP32 resolution of the diagonal; a coupling below that
// shifts an eigenvalue by at most 1e-4 of the gap.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tri_twosum_add(float& hi, float& lo, float b) {
  const float t = hi + b, bb = t - hi;
  lo += (hi - (t - bb)) + (b - bb);
  hi = t;
}

// Stage the P vectors of uvec (P rows of n floats, global) transposed into
// Us (Us[k * ldu + c] = u_c[k], each scaled to unit norm, columns P..ldu-1
// zero) and form Y = G U (n x ldu floats, global) from 32-term FP32 chunks
// added by a compensated (two-sum) FP32 accumulation. Ends with a barrier.
__device__ inline void tri_stage_gu(const float* G, int ldg, const float* uvec, int n, int P,
                                    float* Us, int ldu, float* Y) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  // vectors, transposed, each scaled to unit norm (FP32 chunks, FP64 total)
  for (int c = warp; c < P; c += nt >> 5) {
    double s2 = 0.0;
    for (int k0 = 0; k0 < n; k0 += 32) {
      const float v = (k0 + lane < n) ? uvec[(size_t)c * n + k0 + lane] : 0.f;
      s2 += (double)warp_sum(v * v);
    }
    const float inv = (s2 > 0.0) ? (float)(1.0 / sqrt(s2)) : 0.f;
    for (int k = lane; k < n; k += 32) Us[(size_t)k * ldu + c] = uvec[(size_t)c * n + k] * inv;
  }
  for (int idx = tid; idx < n * (ldu - P); idx += nt) {
    const int k = idx / (ldu - P), c = P + idx - k * (ldu - P);
    Us[(size_t)k * ldu + c] = 0.f;
  }
  __syncthreads();
  // Y = G U, 4 x 4 blocks per thread
  const int nrb = (n + 3) / 4, ncb = ldu / 4;
  for (int blk = tid; blk < nrb * ncb; blk += nt) {
    const int cb = blk % ncb, rb = blk / ncb;
    const int i0 = 4 * rb, c0 = 4 * cb;
    float hs[4][4], ls[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) { hs[p][q] = 0.f; ls[p][q] = 0.f; }
    // G is symmetric: rows i0..i0+3 at column k are row k at columns
    // i0..i0+3, one four-wide load (columns n..ldg-1 hold zeros)
    const float* gk = G + i0;
    for (int k0 = 0; k0 < n; k0 += 32) {
      float ch[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) ch[p][q] = 0.f;
      const int k1 = min(n, k0 + 32);
      for (int k = k0; k < k1; ++k) {
        const float4 g4 = *reinterpret_cast<const float4*>(gk + (size_t)k * ldg);
        const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
        const float4 u = *reinterpret_cast<const float4*>(Us + (size_t)k * ldu + c0);
        const float uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) ch[p][q] = fmaf(gv[p], uv[q], ch[p][q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) tri_twosum_add(hs[p][q], ls[p][q], ch[p][q]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (i0 + p >= n) break;
      *reinterpret_cast<float4*>(Y + (size_t)(i0 + p) * ldu + c0) =
          make_float4(hs[p][0] + ls[p][0], hs[p][1] + ls[p][1], hs[p][2] + ls[p][2],
                      hs[p][3] + ls[p][3]);
    }
  }
  __syncthreads();
}

__device__ inline void tri_ritz(const float* G, int ldg, const float* uvec, int n,
                                int P, float* Us, int ldu, float* H, int ldh, float* Y) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  tri_stage_gu(G, ldg, uvec, n, P, Us, ldu, Y);
  const int ncb = ldu / 4;
  // H = U^T Y, 4 x 4 blocks per thread: the blocks on and above the
  // diagonal, each mirrored below it
  const int nhb = ncb * (ncb + 1) / 2;
  for (int blk = tid; blk < nhb; blk += nt) {
    // blk -> (ab, bb), ab <= bb; block row ab starts at ab * ncb - ab (ab - 1) / 2
    int ab = (int)((2.f * ncb + 1.f - sqrtf((2.f * ncb + 1.f) * (2.f * ncb + 1.f) - 8.f * blk)) * 0.5f);
    ab = max(0, min(ab, ncb - 1));
    while (ab > 0 && ab * ncb - ab * (ab - 1) / 2 > blk) --ab;
    while (ab + 1 < ncb && (ab + 1) * ncb - (ab + 1) * ab / 2 <= blk) ++ab;
    const int bb = ab + (blk - (ab * ncb - ab * (ab - 1) / 2));
    const int a0 = 4 * ab, b0 = 4 * bb;
    float hs[4][4], ls[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) { hs[p][q] = 0.f; ls[p][q] = 0.f; }
    for (int k0 = 0; k0 < n; k0 += 32) {
      float ch[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) ch[p][q] = 0.f;
      const int k1 = min(n, k0 + 32);
      for (int k = k0; k < k1; ++k) {
        const float4 u = *reinterpret_cast<const float4*>(Us + (size_t)k * ldu + a0);
        const float4 y = *reinterpret_cast<const float4*>(Y + (size_t)k * ldu + b0);
        const float uv[4] = {u.x, u.y, u.z, u.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) ch[p][q] = fmaf(uv[p], yv[q], ch[p][q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) tri_twosum_add(hs[p][q], ls[p][q], ch[p][q]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (a0 + p < P && b0 + q < P) {
          const float v = hs[p][q] + ls[p][q];
          H[(size_t)(a0 + p) * ldh + b0 + q] = v;
          if (a0 != b0) H[(size_t)(b0 + q) * ldh + a0 + p] = v;
        }
  }
  __syncthreads();
  // symmetrise: H_ab = (H_ab + H_ba) / 2
  for (int idx = tid; idx < P * P; idx += nt) {
    const int a = idx / P, b = idx - a * P;
    if (a < b) {
      const float v = 0.5f * (H[(size_t)a * ldh + b] + H[(size_t)b * ldh + a]);
      H[(size_t)a * ldh + b] = v;
      H[(size_t)b * ldh + a] = v;
    }
  }
  __syncthreads();
  // Jacobi on H by warp 0: sweeps over the pairs, 32 pairs tested at a time,
  // the significant ones rotated one after another
  if (warp == 0) {
    const float eps = 1.1920929e-07f;
    for (int sweep = 0; sweep < 6; ++sweep) {
      bool any = false;
      // pairs (p, q) with q - p <= 32: the columns are in spectral order,
      // and a coupling H_pq above 1e-2 |H_pp - H_qq| joins near neighbours
      for (int pr = 0; pr + 1 < P; ++pr)
      for (int q0 = pr + 1; q0 < min(P, pr + 33); q0 += 32) {
        // pairs (pr, q0 + lane)
        int p = -1, q = -1;
        if (q0 + lane < P) {
          p = pr;
          q = q0 + lane;
        }
        bool sig = false;
        if (p >= 0) {
          const float app = H[(size_t)p * ldh + p], aqq = H[(size_t)q * ldh + q];
          const float apq = H[(size_t)p * ldh + q];
          sig = fabsf(apq) > 1e-2f * fabsf(app - aqq) &&
                fabsf(apq) > 4.f * eps * sqrtf(fabsf(app) * fabsf(aqq));
        }
        unsigned m = __ballot_sync(0xffffffffu, sig);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const int pp = __shfl_sync(0xffffffffu, p, src);
          const int qq = __shfl_sync(0xffffffffu, q, src);
          const float app = H[(size_t)pp * ldh + pp], aqq = H[(size_t)qq * ldh + qq];
          const float apq = H[(size_t)pp * ldh + qq];
          // recheck: earlier rotations of this batch may have changed the pair
          if (!(fabsf(apq) > 1e-2f * fabsf(app - aqq) &&
                fabsf(apq) > 4.f * eps * sqrtf(fabsf(app) * fabsf(aqq))))
            continue;
          any = true;
          const float zeta = (aqq - app) / (2.f * apq);
          const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = 1.f / sqrtf(1.f + tt * tt), s = c * tt;
          __syncwarp();
          // rows p, q (then columns by symmetry)
          for (int j = lane; j < P; j += 32) {
            if (j == pp || j == qq) continue;
            const float hp = H[(size_t)pp * ldh + j], hq = H[(size_t)qq * ldh + j];
            const float np_ = c * hp - s * hq, nq_ = s * hp + c * hq;
            H[(size_t)pp * ldh + j] = np_;
            H[(size_t)qq * ldh + j] = nq_;
            H[(size_t)j * ldh + pp] = np_;
            H[(size_t)j * ldh + qq] = nq_;
          }
          if (lane == 0) {
            H[(size_t)pp * ldh + pp] = app - tt * apq;
            H[(size_t)qq * ldh + qq] = aqq + tt * apq;
            H[(size_t)pp * ldh + qq] = 0.f;
            H[(size_t)qq * ldh + pp] = 0.f;
          }
          for (int k = lane; k < n; k += 32) {
            const float up = Us[(size_t)k * ldu + pp], uq = Us[(size_t)k * ldu + qq];
            Us[(size_t)k * ldu + pp] = c * up - s * uq;
            Us[(size_t)k * ldu + qq] = s * up + c * uq;
          }
          __syncwarp();
        }
      }
      if (!any) break;
    }
  }
  __syncthreads();
}

// Rayleigh quotients rho_c = u_c^T G u_c of the P unit vectors staged by
// tri_stage_gu (Us, and Y = G U), in FP64 from the FP32 products; one warp
// per vector. Ends with a barrier.
__device__ inline void tri_rq_diag(const float* Us, int ldu, const float* Y, int n, int P,
                                   double* rho) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < P; c += nw) {
    double s = 0.0;
    for (int k = lane; k < n; k += 32)
      s = fma((double)Us[(size_t)k * ldu + c], (double)Y[(size_t)k * ldu + c], s);
    s = warp_sum(s);
    if (lane == 0) rho[c] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The whole eigensolve + ReduceRank shrink + rotate-matrix write for a full
// buffer of n = 2*ell rows whose Gram is in A (n x ld, scaled by 1/smax).
// NB: vectors per fallback inverse-iteration batch; R, MAXJ, VPT: step-5
// layout (n <= R * MAXJ). scr_raw: tri_scratch_bytes(n, NB) bytes; small:
// tri_small_bytes(n) bytes of shared memory; rw: tri_rw_bytes(n, warps)
// bytes of shared memory for step 1 (may be scr_raw when that is in shared
// memory). A and scr_raw may be in shared or in global memory. Needs
// n - 1 <= 32 TRI_CPT warps.
// ---------------------------------------------------------------------------
template <int NB, int R, int MAXJ, int VPT>
__device__ void tri_eig_shrink(const EigArgs& a, float* A, int ld, int n, double smax,
                               unsigned char* scr_raw, unsigned char* small, unsigned char* rw) {
  constexpr int TRI_CU = (R * MAXJ / 2 + 32) / 32;  // vectors <= n / 2 + 1 <= 32 TRI_CU
  const int tid = threadIdx.x, nt = blockDim.x;
  double* mu = reinterpret_cast<double*>(small);
  double* mup = mu + n;
  float* fv = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(mu) + tri_al16((size_t)n * 16));
  const int np8 = (n + 7) & ~7;
  float* red = fv;  // 64 floats, 16-byte aligned (read four at a time)
  float* xb = red + 64;
  float* vb0 = xb + np8;
  float* vb1 = vb0 + np8;
  float* qb = vb1 + np8;
  float* pb = qb + np8;
  float* d = pb + np8;
  float* e = d + n;
  float* e2 = e + n;
  float* lam = e2 + n;
  int* rrank = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(fv) +
                                      tri_al16(tri_fv_floats(n) * 4));
  int* pos = rrank + n;
  __shared__ float s_tnorm;
  __shared__ int s_count, s_ok;
  __shared__ double s_dsum, s_dlast;

  // Values past the (ell+1)-th are zeroed by every rule but SS, so only SS and
  // a recorded spectrum need them; without them the removed mass comes from
  // the trace of G (FP64, taken before step 1 changes the diagonal).
  const int nl = (a.variant == FD_VAR_SS || a.sig2_out) ? n : min(n, a.ell + 1);
  __shared__ double s_trace;
  if (threadIdx.x < 32) {
    const double t = eig_trace(a, A, ld, n, smax);
    if (threadIdx.x == 0) s_trace = t;
  }
  tri_reduce(A, ld, n, d, e, rw, red);
  tri_bisect(d, e, e2, n, lam, &s_tnorm, reinterpret_cast<int*>(scr_raw), nl);
  {
    // eigenvalues at or below the bisection's resolution (2 eps lambda_1)
    // are zero: their sign and size are rounding noise
    const float zfloor = 2.f * 1.1920929e-07f * fmaxf(lam[0], 0.f);
    for (int k = tid; k < n; k += nt) mu[k] = (lam[k] > zfloor) ? (double)lam[k] * smax : 0.0;
  }
  __syncthreads();
  // n <= blockDim.x (512 threads for n <= 512; the batched kernel: n <= 128, 256 threads)
  shrink_sorted(a, n, n, 1.1920928955078125e-07, mu, mup, rrank, &s_count, &s_dsum, &s_dlast);
  const int nout = a.ell - 1;
  // Refinement (step 6) for the rules that keep or shrink by position (FD,
  // PFD, iSVD): vectors for positions 0..ell, the retained ones, the one at
  // the cut (delta) and the next, whose Ritz values replace the eigenvalues
  // of T (also when delta = 0: the kept values are then sigma^2 itself).
  // Needs room for ell+1 vectors and the saved G.
  const int nref = a.ell + 1;
  const bool refine = a.gsave != nullptr && a.uvec != nullptr &&
                      (a.variant == FD_VAR_FD || a.variant == FD_VAR_PFD ||
                       a.variant == FD_VAR_ISVD) &&
                      nref <= n / 2 + 1 && mu[0] > 0.0 &&
                      (size_t)tri_zoff(n) + (size_t)n * nref <= (size_t)n * ld &&
                      (size_t)n * ((nref + 3) & ~3) + (size_t)nref * (nref + 1) <= (size_t)n * ld;
  const int count = refine ? nref : (s_count < nout ? s_count : nout);
  if (refine) {
    for (int k = tid; k < nref; k += nt) pos[k] = k;
  } else {
    for (int k = tid; k < n; k += nt) {
      const int r = rrank[k];
      if (r >= 0 && r < nout) pos[r] = k;
    }
  }
  if (tid == 0) s_ok = 1;
  __syncthreads();
  const float tnorm = s_tnorm;
  const float pivmin = fmaxf(tnorm, 1e-30f) * 1e-30f;
  float* Zt = A + tri_zoff(n);
  // odd stride (fewer bank conflicts) where it fits after the reflectors
  const int ldz = ((size_t)tri_zoff(n) + (size_t)n * tri_ldz(count) <= (size_t)n * ld)
                      ? tri_ldz(count) : count;
  for (int r = tid; r < count; r += nt)
    if (!tri_twisted(d, e, e2, n, lam[pos[r]], pivmin, Zt + r, ldz)) s_ok = 0;
  __syncthreads();
  bool ok = s_ok != 0;
  bool fell_back = false;
  if (ok) {
    const int ldc = tri_ldz(count);
    float* C = reinterpret_cast<float*>(scr_raw);
    float* dinv = reinterpret_cast<float*>(scr_raw + tri_al16((size_t)count * ldc * 4));
    ok = tri_cholqr<TRI_CU>(Zt, ldz, n, count, C, ldc, dinv, 0.25f);
  }
  if (!ok) {
    fell_back = true;
    // Vectors of close eigenvalues came out nearly dependent. Within a window
    // of a few eps ||T|| any orthonormal basis of the invariant subspace is
    // as good, so the members of such clusters are replaced by one
    // inverse-iteration solve from a random start each (generic, independent
    // combinations inside the subspace); then Cholesky-QR again. If a twisted
    // vector failed, or that still fails, every vector is recomputed that way
    // and orthonormalised by classical Gram-Schmidt (twice).
    __shared__ int s_nl;
    __syncthreads();
    float* scr = reinterpret_cast<float*>(scr_raw);
    int* ord = reinterpret_cast<int*>(vb0);   // vb0, vb1: np8 >= count entries each,
    int* list = reinterpret_cast<int*>(vb1);  // dead after step 1
    bool redo = s_ok == 0;
    if (!redo) {
      tri_tight_repair<NB>(Zt, ldz, n, d, e, lam, pos, count, 16.f * 1.1920929e-07f * tnorm,
                           tnorm, scr, ord, list, reinterpret_cast<int*>(qb), xb, red, &s_nl);
      const int ldc = tri_ldz(count);
      float* C = reinterpret_cast<float*>(scr_raw);
      float* dinv = reinterpret_cast<float*>(scr_raw + tri_al16((size_t)count * ldc * 4));
      redo = !tri_cholqr<TRI_CU>(Zt, ldz, n, count, C, ldc, dinv, 0.25f);
    }
    if (redo) {
      __syncthreads();
      for (int c0 = 0; c0 < count; c0 += NB) {
        tri_invit_batch<NB>(Zt, ldz, n, d, e, lam, pos, nullptr, c0, count, tnorm, scr);
        __syncthreads();
      }
      tri_cgs2(Zt, ldz, n, count, xb, red);
    }
  }
  // SS: the merged masses go to the smallest kept directions, whose
  // eigenvalues of T are small against ||G||; a row scaled by
  // sqrt(mu'/lambda) then carries mu' * (u^T G u) / lambda, off by the error
  // of lambda relative to the row's own Rayleigh quotient. The rows are
  // scaled by sqrt(mu' / (u^T G u)) instead, with the quotient formed from
  // the saved G, so that each row carries mu' (SS conserves ||B||_F^2).
  const bool rqscale = !refine && a.variant == FD_VAR_SS && a.gsave != nullptr &&
                       a.uvec != nullptr && count > 0 &&
                       (size_t)n * ((count + 3) & ~3) <= (size_t)n * ld;
  if (rqscale) {
    tri_back_write<R, MAXJ, VPT>(a, A, n, Zt, ldz, count, mu, mup, pos, vb0, a.uvec, n);
    const int ldu = (count + 3) & ~3;
    float* Us = A;  // A, Zt and the scratch area are dead now
    double* rq = reinterpret_cast<double*>(d);  // d, e: 2n floats >= count doubles
    tri_stage_gu(a.gsave, a.ldgsave, a.uvec, n, count, Us, ldu, a.uvec);
    tri_rq_diag(Us, ldu, a.uvec, n, count, rq);
    float* wr = reinterpret_cast<float*>(a.wrot);
    float* rscale = vb1;
    for (int r = tid; r < nout; r += nt) {
      const double m1 = (r < count) ? mup[pos[r]] : 0.0;
      const double q = (r < count) ? rq[r] * smax : 0.0;
      rscale[r] = (q > 0.0 && m1 > 0.0) ? (float)sqrt(m1 / q) : 0.f;
      if (a.row_mass) a.row_mass[r] = m1;
    }
    __syncthreads();
    for (int idx = tid; idx < nout * n; idx += nt) {
      const int r = idx / n, i = idx - r * n;
      const float val = (r < count) ? rscale[r] * Us[(size_t)i * ldu + r] : 0.f;
      wr[(size_t)r * a.ldr + i] = val;
      if (a.wrot_hi) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(val);
        a.wrot_hi[(size_t)r * a.ldr16 + i] = hi;
        a.wrot_lo[(size_t)r * a.ldr16 + i] = __float2bfloat16_rn(val - __bfloat162float(hi));
      }
    }
    __syncthreads();
    write_counters(a, n, mu, mup, s_count, s_dsum, s_dlast, 0, 1, nl < n ? s_trace : -1.0,
                   fell_back ? 1 : 0);
    return;
  }
  if (!refine) {
    tri_back_write<R, MAXJ, VPT>(a, A, n, Zt, ldz, count, mu, mup, pos, vb0);  // vb0..pb: 4 np8 floats
    write_counters(a, n, mu, mup, s_count, s_dsum, s_dlast, 0, 1, nl < n ? s_trace : -1.0,
                   fell_back ? 1 : 0);
    return;
  }
  // unscaled vectors u_0..u_ell (original basis) to the global scratch
  tri_back_write<R, MAXJ, VPT>(a, A, n, Zt, ldz, count, mu, mup, pos, vb0, a.uvec, n);
  // Rayleigh-Ritz; A, Zt and the scratch area are dead now: the vectors are
  // staged (transposed) in the front of A, H after them, G U in the vectors'
  // global scratch (read into Us first)
  const int ldu = (nref + 3) & ~3;
  const int ldh = nref + 1;
  double* rho = reinterpret_cast<double*>(d);  // d, e: 2n floats >= nref doubles
  float* Us = A;
  float* Hm = A + (size_t)n * ldu;
  tri_ritz(a.gsave, a.ldgsave, a.uvec, n, nref, Us, ldu, Hm, ldh, a.uvec);
  for (int c = tid; c < nref; c += nt) rho[c] = (double)Hm[(size_t)c * ldh + c];
  __syncthreads();
  // refined masses in descending order (ties by position); positions past
  // the refined block keep the bisection values, capped by the last refined one
  int* ordv = reinterpret_cast<int*>(e2);  // sorted index -> vector column
  for (int c = tid; c < nref; c += nt) {
    const double v = rho[c];
    int rk = 0;
    for (int q = 0; q < nref; ++q) {
      const double w = rho[q];
      rk += (w > v) || (w == v && q < c);
    }
    ordv[rk] = c;
  }
  __syncthreads();
  {
    // the same floor as for the eigenvalues of T: Ritz values at or below
    // 2 eps of the largest are rounding noise of the FP32 Gram (a rank-
    // deficient buffer), taken as zero
    const double zf = 2.0 * 1.1920928955078125e-07 * fmax(rho[ordv[0]], 0.0);
    for (int k = tid; k < nref; k += nt) {
      const double v = rho[ordv[k]];
      mu[k] = (v > zf) ? v * smax : 0.0;
    }
  }
  __syncthreads();
  for (int k = nref + tid; k < n; k += nt) mu[k] = fmin(mu[k], mu[nref - 1]);
  __syncthreads();
  shrink_sorted(a, n, n, 1.1920928955078125e-07, mu, mup, rrank, &s_count, &s_dsum, &s_dlast);
  // rotate matrix rows: rank r <- sorted position k <- vector column ordv[k],
  // scaled by sqrt(mu'/mu); rows past the retained count are zero
  const int cnt = s_count < nout ? s_count : nout;
  float* wr = reinterpret_cast<float*>(a.wrot);
  for (int k = tid; k < nref; k += nt) {
    const int r = rrank[k];
    if (r >= 0 && r < nout) pos[r] = k;
  }
  __syncthreads();
  // per output row: its scale sqrt(mu'/mu) (one FP64 square root a row) and
  // the column of Us it takes
  float* rscale = vb1;
  int* rcol = reinterpret_cast<int*>(xb);
  for (int r = tid; r < nout; r += nt) {
    const int k = (r < cnt) ? pos[r] : 0;
    rscale[r] = (r < cnt && mu[k] > 0.0) ? (float)sqrt(mup[k] / mu[k]) : 0.f;
    rcol[r] = (r < cnt) ? ordv[k] : 0;
  }
  __syncthreads();
  for (int idx = tid; idx < nout * n; idx += nt) {
    const int r = idx / n, i = idx - r * n;
    const float val = rscale[r] * Us[(size_t)i * ldu + rcol[r]];
    wr[(size_t)r * a.ldr + i] = val;
    if (a.wrot_hi) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(val);
      a.wrot_hi[(size_t)r * a.ldr16 + i] = hi;
      a.wrot_lo[(size_t)r * a.ldr16 + i] = __float2bfloat16_rn(val - __bfloat162float(hi));
    }
  }
  if (a.row_mass)
    for (int r = tid; r < nout; r += nt) a.row_mass[r] = (r < cnt) ? mup[pos[r]] : 0.0;
  __syncthreads();
  write_counters(a, n, mu, mup, s_count, s_dsum, s_dlast, 0, 1, nl < n ? s_trace : -1.0,
                 fell_back ? 1 : 0);
}

}  // namespace fdk
