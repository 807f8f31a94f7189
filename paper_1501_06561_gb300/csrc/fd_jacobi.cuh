// One-sided (Hestenes) Jacobi sweeps in FP32 on a symmetric matrix held in
// shared memory, shared by the single-sketch and the batched kernels.
//
// The columns w_j of W (initially W = G, column j stored contiguously with
// stride ld) are rotated in pairs until they are mutually orthogonal. Then
// W = G V with V orthogonal and W^T W = V^T G^2 V diagonal, so column j of W
// is lambda_j u_j for an eigenpair (lambda_j, u_j) of the positive
// semidefinite G; V is never formed.
//
// Schedule: round-robin (tournament) order, np/2 disjoint pairs per round and
// np-1 rounds per sweep; a group of GS lanes owns a pair, reads its two
// columns as float4 chunks, reduces the inner product across the group, and
// writes the rotated columns back; one barrier per round. Column norms are
// carried through a sweep with the exact update ||w_p'||^2 = ||w_p||^2 - t g,
// ||w_q'||^2 = ||w_q||^2 + t g (g = <w_p, w_q>), recomputed from the data at
// every sweep start and at once when the update cancels more than three
// quarters of a norm.
#pragma once

#include <cuda_runtime.h>

namespace fdk {

template <int GS>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
  for (int o = GS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, GS);
  return v;
}

template <int GS, int MAXV>
__device__ __forceinline__ float col_sq_f32(const float* w, int nv, int gl, unsigned mask) {
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int c = 0; c < MAXV; ++c) {
    const int v = c * GS + gl;
    if (v < nv) {
      const float4 x = reinterpret_cast<const float4*>(w)[v];
      s0 = fmaf(x.x, x.x, s0);
      s1 = fmaf(x.y, x.y, s1);
      s0 = fmaf(x.z, x.z, s0);
      s1 = fmaf(x.w, x.w, s1);
    }
  }
  return group_sum<GS>(s0 + s1, mask);
}

// Runs sweeps until one performs no rotation or `max_sweeps` is reached.
// Wm: np columns of stride ld (ld % 4 == 0, padding zero); nrm: np floats of
// shared scratch. All threads of the block (blockDim.x a multiple of GS)
// must call it. Returns the number of sweeps run; *capped = hit the cap.
template <int GS, int MAXV, int MAXP>
__device__ int jacobi_sweeps_f32(float* Wm, int ld, int np, float* nrm, int max_sweeps,
                                 float tol, int* capped) {
  const int tid = threadIdx.x;
  const int g = tid / GS, gl = tid % GS;
  const int ngroups = blockDim.x / GS;
  const unsigned gmask =
      (GS == 32) ? 0xffffffffu : (((1u << GS) - 1u) << ((tid & 31) & ~(GS - 1)));
  const int nv = (np + 3) >> 2;
  const int npairs = np / 2, nrounds = np - 1;
  const float tol2 = tol * tol;

  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int j = g; j < np; j += ngroups) {
      const float s = col_sq_f32<GS, MAXV>(Wm + (size_t)j * ld, nv, gl, gmask);
      if (gl == 0) nrm[j] = s;
    }
    __syncthreads();
    // round-0 positions of this group's pairs; each round moves every index
    // except 0 forward by one, wrapping np-1 -> 1
    int P[MAXP], Q[MAXP];
#pragma unroll
    for (int s = 0; s < MAXP; ++s) {
      const int k = g + s * ngroups;
      P[s] = k;
      Q[s] = np - 1 - k;
    }
    int rotated = 0;
    for (int r = 0; r < nrounds; ++r) {
#pragma unroll
      for (int s = 0; s < MAXP; ++s) {
        const int k = g + s * ngroups;
        if (k < npairs) {
          const int p = P[s], q = Q[s];
          float4* wp = reinterpret_cast<float4*>(Wm + (size_t)p * ld);
          float4* wq = reinterpret_cast<float4*>(Wm + (size_t)q * ld);
          const float al = nrm[p], be = nrm[q];
          float4 xp[MAXV], xq[MAXV];
          float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
          for (int c = 0; c < MAXV; ++c) {
            const int v = c * GS + gl;
            if (v < nv) {
              xp[c] = wp[v];
              xq[c] = wq[v];
            } else {
              xp[c] = make_float4(0.f, 0.f, 0.f, 0.f);
              xq[c] = xp[c];
            }
            g0 = fmaf(xp[c].x, xq[c].x, g0);
            g1 = fmaf(xp[c].y, xq[c].y, g1);
            g2 = fmaf(xp[c].z, xq[c].z, g2);
            g3 = fmaf(xp[c].w, xq[c].w, g3);
          }
          const float ga = group_sum<GS>((g0 + g1) + (g2 + g3), gmask);
          if (ga != 0.f && ga * ga > tol2 * al * be) {
            // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (be - al) / (2 ga),
            // written with one division
            const float num = be - al, den = 2.f * ga;
            const float hyp = sqrtf(fmaf(num, num, den * den));
            float t = __fdividef(fabsf(den), fabsf(num) + hyp);
            if ((num < 0.f) != (den < 0.f)) t = -t;
            const float cs = 1.f / sqrtf(fmaf(t, t, 1.f));  // correctly rounded: cs^2 + sn^2 = 1 unbiased
            const float sn = cs * t;
#pragma unroll
            for (int c = 0; c < MAXV; ++c) {
              const int v = c * GS + gl;
              if (v < nv) {
                float4 a4, b4;
                a4.x = fmaf(cs, xp[c].x, -sn * xq[c].x);
                b4.x = fmaf(sn, xp[c].x, cs * xq[c].x);
                a4.y = fmaf(cs, xp[c].y, -sn * xq[c].y);
                b4.y = fmaf(sn, xp[c].y, cs * xq[c].y);
                a4.z = fmaf(cs, xp[c].z, -sn * xq[c].z);
                b4.z = fmaf(sn, xp[c].z, cs * xq[c].z);
                a4.w = fmaf(cs, xp[c].w, -sn * xq[c].w);
                b4.w = fmaf(sn, xp[c].w, cs * xq[c].w);
                wp[v] = a4;
                wq[v] = b4;
              }
            }
            float na = fmaf(-t, ga, al), nb = fmaf(t, ga, be);
            if (na < 0.25f * al) na = col_sq_f32<GS, MAXV>(reinterpret_cast<float*>(wp), nv, gl, gmask);
            if (nb < 0.25f * be) nb = col_sq_f32<GS, MAXV>(reinterpret_cast<float*>(wq), nv, gl, gmask);
            if (gl == 0) {
              nrm[p] = na;
              nrm[q] = nb;
            }
            rotated = 1;
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < MAXP; ++s) {
        if (P[s] != 0) P[s] = (P[s] + 1 == np) ? 1 : P[s] + 1;
        Q[s] = (Q[s] + 1 == np) ? 1 : Q[s] + 1;
      }
    }
    if (!__syncthreads_or(rotated)) break;
  }
  *capped = (sweep >= max_sweeps) ? 1 : 0;
  return (sweep < max_sweeps) ? sweep + 1 : max_sweeps;
}

}  // namespace fdk

namespace fdk {

// ---------------------------------------------------------------------------
// Block variant of the same sweeps: the np columns form nb = np/BS blocks of
// BS columns; blocks meet in round-robin order (nb-1 rounds per sweep), and a
// group of GS lanes holds its two blocks (2*BS columns) in registers for the
// whole round. In round 0 of a sweep every block is first orthogonalised
// internally (BS-1 sub-rounds); then the BS*BS cross pairs are rotated in BS
// sub-rounds of BS disjoint pairs, i.e. BS independent rotations at a time.
// Every column pair is rotated once per sweep, as in the scalar schedule, but
// shared memory sees each column twice per round instead of twice per pair.
// ---------------------------------------------------------------------------
template <int GS, int MAXV, int NC>
struct BlockCols {
  float4 v[NC][MAXV];
  float nn[NC];
};

// Pair patterns over the 8 columns of a block pair (0-3 top block, 4-7
// bottom block). PAT 0-2: the three rounds of disjoint pairs inside each
// block; PAT 3-6: cross pairs (i, 4 + (i + PAT - 3) mod 4).
template <int PAT>
__device__ __forceinline__ constexpr int pat_p(int i) {
  return PAT == 0 ? 2 * i : (PAT <= 2 ? (i < 2 ? i : i + 2) : i);
}
template <int PAT>
__device__ __forceinline__ constexpr int pat_q(int i) {
  return PAT == 0 ? 2 * i + 1
                  : (PAT == 1 ? (i < 2 ? i + 2 : i + 4)
                              : (PAT == 2 ? (i < 2 ? 3 - i : 9 - i) : 4 + ((i + PAT - 3) & 3)));
}

// Rotates the 4 disjoint column pairs of pattern PAT of `b`. Branch-free:
// a pair below the tolerance gets the identity rotation (t = 0, c = 1,
// s = 0), so the four independent rotations can be interleaved.
template <int GS, int MAXV, int NC, int PAT>
__device__ __forceinline__ void rotate_set(BlockCols<GS, MAXV, NC>& b, float tol2,
                                           unsigned gmask, int& rotated) {
  constexpr int K = 4;
  float g[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int c = 0; c < MAXV; ++c) {
      const float4 x = b.v[pat_p<PAT>(i)][c], y = b.v[pat_q<PAT>(i)][c];
      a0 = fmaf(x.x, y.x, a0);
      a1 = fmaf(x.y, y.y, a1);
      a0 = fmaf(x.z, y.z, a0);
      a1 = fmaf(x.w, y.w, a1);
    }
    g[i] = a0 + a1;
  }
#pragma unroll
  for (int o = GS / 2; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < K; ++i) g[i] += __shfl_xor_sync(gmask, g[i], o, GS);
  float cs[K], sn[K];
  bool recompute = false;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int P = pat_p<PAT>(i), Q = pat_q<PAT>(i);
    const float al = b.nn[P], be = b.nn[Q], ga = g[i];
    const bool doit = (ga != 0.f) && (ga * ga > tol2 * al * be);
    const float num = be - al, den = 2.f * ga;
    const float hyp = sqrtf(fmaf(num, num, den * den));
    float t = __fdividef(fabsf(den), fabsf(num) + hyp);
    if ((num < 0.f) != (den < 0.f)) t = -t;
    t = doit ? t : 0.f;
    cs[i] = 1.f / sqrtf(fmaf(t, t, 1.f));  // correctly rounded: cs^2 + sn^2 = 1 unbiased
    sn[i] = cs[i] * t;
    const float na = fmaf(-t, ga, al), nb = fmaf(t, ga, be);
    recompute |= doit && (na < 0.25f * al || nb < 0.25f * be);
    b.nn[P] = na;
    b.nn[Q] = nb;
    rotated |= doit ? 1 : 0;
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int P = pat_p<PAT>(i), Q = pat_q<PAT>(i);
#pragma unroll
    for (int c = 0; c < MAXV; ++c) {
      const float4 x = b.v[P][c], y = b.v[Q][c];
      float4 xn, yn;
      xn.x = fmaf(cs[i], x.x, -sn[i] * y.x); yn.x = fmaf(sn[i], x.x, cs[i] * y.x);
      xn.y = fmaf(cs[i], x.y, -sn[i] * y.y); yn.y = fmaf(sn[i], x.y, cs[i] * y.y);
      xn.z = fmaf(cs[i], x.z, -sn[i] * y.z); yn.z = fmaf(sn[i], x.z, cs[i] * y.z);
      xn.w = fmaf(cs[i], x.w, -sn[i] * y.w); yn.w = fmaf(sn[i], x.w, cs[i] * y.w);
      b.v[P][c] = xn;
      b.v[Q][c] = yn;
    }
  }
  if (recompute) {  // uniform within the group: every lane holds the same norms
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int P = pat_p<PAT>(i), Q = pat_q<PAT>(i);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int c = 0; c < MAXV; ++c) {
        const float4 x = b.v[P][c], y = b.v[Q][c];
        s0 = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, s0))));
        s1 = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, s1))));
      }
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(gmask, s0, o, GS);
        s1 += __shfl_xor_sync(gmask, s1, o, GS);
      }
      b.nn[P] = s0;
      b.nn[Q] = s1;
    }
  }
}

// Block sweeps with BS = 4 columns per block. Wm holds npb = round_up(np, 8)
// columns of stride ld (columns past np zero; ld % 4 == 0). Threads: at least
// (npb / 8) * GS (one group per block pair); extra threads idle at barriers.
template <int GS, int MAXV>
__device__ int jacobi_blocks4_f32(float* Wm, int ld, int np, float* nrm, int max_sweeps,
                                  float tol, int* capped) {
  constexpr int BS = 4;
  const int tid = threadIdx.x;
  const int g = tid / GS, gl = tid % GS;
  const unsigned gmask =
      (GS == 32) ? 0xffffffffu : (((1u << GS) - 1u) << ((tid & 31) & ~(GS - 1)));
  const int npb = (np + 2 * BS - 1) / (2 * BS) * (2 * BS);
  const int nb = npb / BS;
  const int nv = (npb + 3) >> 2;
  const int ngroups_needed = nb / 2;
  const float tol2 = tol * tol;

  const int ngroups = blockDim.x / GS;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // exact column norms at the start of every sweep
    for (int j = g; j < npb; j += ngroups) {
      const float s = col_sq_f32<GS, MAXV>(Wm + (size_t)j * ld, nv, gl, gmask);
      if (gl == 0) nrm[j] = s;
    }
    __syncthreads();
    int rotated = 0;
    for (int r = 0; r < nb - 1; ++r) {
      // block pairs k = g, g + ngroups, ...: block indices in round r follow the
      // round-robin rule (index 0 fixed, the others advance by one per round)
      for (int k = g; k < ngroups_needed; k += ngroups) {
        const int bt = (k == 0) ? 0 : 1 + (k - 1 + r) % (nb - 1);
        const int bb = 1 + (nb - 2 - k + r) % (nb - 1);
        BlockCols<GS, MAXV, 2 * BS> b;
#pragma unroll
        for (int j = 0; j < 2 * BS; ++j) {
          const int col = (j < BS ? bt * BS + j : bb * BS + (j - BS));
          const float4* w = reinterpret_cast<const float4*>(Wm + (size_t)col * ld);
#pragma unroll
          for (int c = 0; c < MAXV; ++c) {
            const int v = c * GS + gl;
            b.v[j][c] = (v < nv) ? w[v] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          b.nn[j] = nrm[col];
        }
        if (r == 0) {
          rotate_set<GS, MAXV, 2 * BS, 0>(b, tol2, gmask, rotated);
          rotate_set<GS, MAXV, 2 * BS, 1>(b, tol2, gmask, rotated);
          rotate_set<GS, MAXV, 2 * BS, 2>(b, tol2, gmask, rotated);
        }
        rotate_set<GS, MAXV, 2 * BS, 3>(b, tol2, gmask, rotated);
        rotate_set<GS, MAXV, 2 * BS, 4>(b, tol2, gmask, rotated);
        rotate_set<GS, MAXV, 2 * BS, 5>(b, tol2, gmask, rotated);
        rotate_set<GS, MAXV, 2 * BS, 6>(b, tol2, gmask, rotated);
#pragma unroll
        for (int j = 0; j < 2 * BS; ++j) {
          const int col = (j < BS ? bt * BS + j : bb * BS + (j - BS));
          float4* w = reinterpret_cast<float4*>(Wm + (size_t)col * ld);
#pragma unroll
          for (int c = 0; c < MAXV; ++c) {
            const int v = c * GS + gl;
            if (v < nv) w[v] = b.v[j][c];
          }
          if (gl == 0) nrm[col] = b.nn[j];
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;
  }
  *capped = (sweep >= max_sweeps) ? 1 : 0;
  return (sweep < max_sweeps) ? sweep + 1 : max_sweeps;
}

}  // namespace fdk
