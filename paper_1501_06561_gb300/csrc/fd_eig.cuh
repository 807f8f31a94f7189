// Eigensolve building blocks shared by the single-sketch and batched kernels:
// loading G, and everything after the Jacobi sweeps (eigenvalues, sort, the
// FP64 ReduceRank rules of Sec. 2.3 / Algorithms 2-3, the rotate matrix and
// the FP64 counters).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "fd_internal.cuh"

namespace fdk {

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

inline size_t eig_scalar_bytes(int np) {
  return (size_t)np * (4 * sizeof(double) + 2 * sizeof(int)) + 256;
}

// The exact diagonal of a tensor-core buffer (EigArgs.diag64 set): FP64
// squared norms of the stored rows, the rotate's partial sums added in a
// fixed order for rows 0..nret-1. Ends with a block barrier.
__device__ inline void eig_prepare_diag(const EigArgs& a, int n) {
  if (a.diag64 != nullptr) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double dg;
      if (a.nvalid > 0 && i >= a.nvalid) {
        dg = 0.0;  // padding rows of a flush
      } else if (i < a.nret) {
        dg = 0.0;
        for (int p = 0; p < a.rot_nparts; ++p) dg += a.rot_part[(int64_t)p * a.rot_ld + i];
      } else {
        dg = a.slot_n2[i];
      }
      a.diag64[i] = dg;
    }
  }
  __syncthreads();
}

// Load G = sum of the partial slices (fixed order), symmetrised, into Wm
// (column j = row j of the symmetric G, stride ld, zero padding to np),
// with the exact diagonal when eig_prepare_diag supplied one.
template <typename T>
__device__ void eig_load(const EigArgs& a, T* Wm, int ld, int n, int np) {
  const T* parts = reinterpret_cast<const T*>(a.parts);
  const int nv = (a.nvalid > 0 && a.nvalid < n) ? a.nvalid : n;  // rows holding data
  for (int idx = threadIdx.x; idx < np * ld; idx += blockDim.x) {
    const int i = idx / ld, j = idx - (idx / ld) * ld;
    T v = T(0);
    if (i < nv && j < nv) {
      if (a.diag64 != nullptr && i == j) {
        v = (T)a.diag64[i];
      } else {
        T sij = T(0), sji = T(0);
        for (int p = 0; p < a.nparts; ++p) {
          sij += parts[(int64_t)p * a.part_stride + (int64_t)i * a.ldp + j];
          sji += parts[(int64_t)p * a.part_stride + (int64_t)j * a.ldp + i];
        }
        v = T(0.5) * (sij + sji);
      }
    }
    Wm[(int64_t)i * ld + j] = v;
  }
}

// eig_load for a row-major G in shared memory (stride ld >= n): the partial
// slices summed row by row with coalesced loads, several in flight per lane,
// then symmetrised in place, G_ij = (Z_ij + Z_ji) / 2 (the values eig_load
// gives), and the exact diagonal put in when eig_prepare_diag supplied one.
// Columns n..ld-1 are zeroed. Ends with a block barrier.
template <typename T>
__device__ void eig_load_sym(const EigArgs& a, T* Wm, int ld, int n) {
  const T* parts = reinterpret_cast<const T*>(a.parts);
  const int nv = (a.nvalid > 0 && a.nvalid < n) ? a.nvalid : n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int U = 8;
  for (int i = warp; i < n; i += nw) {
    T* row = Wm + (size_t)i * ld;
    for (int j0 = 0; j0 < ld; j0 += 32 * U) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = T(0);
      if (i < nv) {
        for (int p = 0; p < a.nparts; ++p) {
          const T* src = parts + (int64_t)p * a.part_stride + (int64_t)i * a.ldp;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int j = j0 + lane + 32 * u;
            if (j < nv) v[u] += src[j];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + lane + 32 * u;
        if (j < ld) row[j] = v[u];
      }
    }
  }
  __syncthreads();
  for (int i = warp; i < n; i += nw) {
    for (int j = i + 1 + lane; j < n; j += 32) {
      const T v = T(0.5) * (Wm[(size_t)i * ld + j] + Wm[(size_t)j * ld + i]);
      Wm[(size_t)i * ld + j] = v;
      Wm[(size_t)j * ld + i] = v;
    }
  }
  if (a.diag64 != nullptr)
    for (int i = threadIdx.x; i < nv; i += blockDim.x) Wm[(size_t)i * ld + i] = (T)a.diag64[i];
  __syncthreads();
}

// Scale of the Gram before an FP32 eigensolve: the power of two at or above
// its largest diagonal entry smax (1 for an empty Gram). Multiplying by a
// power of two is exact; a factor fl(1/smax) would move every eigenvalue by
// the same relative amount (up to 2^-24), and since FD subtracts delta at
// every reduction, that shift would add up along a stream.
__device__ __forceinline__ float eig_pow2_scale(float smax) {
  if (!(smax > 0.f)) return 1.f;
  int e;
  (void)frexpf(smax, &e);  // smax = f 2^e, f in [0.5, 1)
  return ldexpf(1.f, e);
}

// FP64 trace of the loaded G: the exact diagonal when it is known, else the
// diagonal of Wm (scaled back by wscale). One warp (threads 0..31); the
// result is valid in lane 0.
template <typename T>
__device__ double eig_trace(const EigArgs& a, const T* Wm, int ld, int n, double wscale) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 32)
    t += (a.diag64 != nullptr) ? a.diag64[i] : (double)Wm[(size_t)i * ld + i] * wscale;
  return warp_sum(t);
}

// Steps after the Jacobi sweeps: eigenvalues, sort, ReduceRank (FP64),
// rotate matrix, counters. `sweep` = sweeps run (== max_sweeps if capped).
// ReduceRank in FP64 on the masses mu_k = sigma_k^2 sorted descending
// (k = 0..n-1; entries n..np-1 are padding): writes sigma'^2 to mup and the
// output rank of every retained position (-1 if freed) to rrank; returns the
// number of retained positions and the deltas subtracted through dsum_out /
// dlast_out (shared). `eps_arith` is the unit of the eigensolve's arithmetic
// (SS treats masses at or below np * eps_arith * mu_0 as empty).
// MAXK: positions per thread in the ranking, np <= MAXK * blockDim.x (every
// eigensolve launch has at least np threads).
template <int MAXK = 1>
static __device__ void shrink_sorted(const EigArgs& a, int n, int np, double eps_arith, const double* mu,
                              double* mup, int* rrank, int* count_out, double* dsum_out,
                              double* dlast_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ double s_dsum, s_dlast;
  __shared__ int s_count;
  if (tid == 0) { s_dsum = 0.0; s_dlast = 0.0; }
  __syncthreads();
  // 5. ReduceRank in FP64 on the masses mu_k = sigma_k^2 (k = 0..n-1 sorted).
  const int ell = a.ell;
  if (a.variant != FD_VAR_SS) {
    double delta = (n >= ell) ? mu[ell - 1] : 0.0;
    int keep = 0;
    if (a.variant == FD_VAR_PFD) {
      // Algorithm 2 keeps floor((1-alpha)*ell) values; alpha > 0 shrinks at least one
      keep = (int)floor((1.0 - a.alpha) * ell + 1e-9);
      keep = keep < 0 ? 0 : (keep > ell - 1 ? ell - 1 : keep);
    } else if (a.variant == FD_VAR_FAST_PFD) {
      // Fast alpha-FD: delta = sigma_t^2, t = ell - ell*alpha/2 (at least one
      // value past t); floor((1-alpha)*ell) values kept, at most t-1
      const int t = fast_pfd_t(ell, a.alpha);
      keep = (int)floor((1.0 - a.alpha) * ell + 1e-9);
      keep = keep < 0 ? 0 : (keep > t - 1 ? t - 1 : keep);
      delta = (n >= t) ? mu[t - 1] : 0.0;
    }
    for (int k = tid; k < np; k += blockDim.x) {
      const double m0 = mu[k];
      double mp = 0.0;
      if (k < n) {
        if (a.variant == FD_VAR_FD) mp = fmax(m0 - delta, 0.0);
        else if (a.variant == FD_VAR_ISVD) mp = (k < ell - 1) ? m0 : 0.0;
        // PFD and Fast alpha-FD: keep, then clip at zero up to ell, zero past it
        else mp = (k < keep) ? m0 : ((k < ell) ? fmax(m0 - delta, 0.0) : 0.0);
      }
      mup[k] = mp;
    }
    if (tid == 0) { s_dsum = delta; s_dlast = delta; }
  } else if (warp == 0) {
    // SS (Algorithm 3, repeated): masses at or below the numerical-rank floor
    // are empty and freed first; then merge the second-smallest into the
    // smallest until ell-1 directions remain. Ties: the larger sorted position
    // counts as smaller.
    // Their total is added to the smallest retained direction at the end, so
    // the sketch keeps the mass of the stream (SS conserves ||B||_F^2).
    const double flo = mu[0] * (double)np * eps_arith;
    double freed = 0.0;
    for (int k = lane; k < np; k += 32) {
      const double v = (k < n) ? mu[k] : 0.0;
      mup[k] = (v > flo) ? v : 0.0;
      if (!(v > flo)) freed += v;
    }
    freed = warp_sum(freed);
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
    if (freed > 0.0 && alive > 0) {
      // smallest alive (mass asc, position desc), as in the merges
      double m1 = INFINITY;
      int i1 = -1;
      for (int k = lane; k < np; k += 32) {
        const double v = mup[k];
        if (v > 0.0 && ((v < m1) || (v == m1 && k > i1))) { m1 = v; i1 = k; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, m1, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i1, o);
        if (oi >= 0 && (i1 < 0 || om < m1 || (om == m1 && oi > i1))) { m1 = om; i1 = oi; }
      }
      if (lane == 0) {
        mup[i1] += freed;
        dsum += freed;
        dlast = freed;
      }
      __syncwarp();
    }
    if (lane == 0) { s_dsum = dsum; s_dlast = dlast; }
  }
  __syncthreads();

  // 6. Output order: retained positions by sigma'^2 descending, ties by
  // position. The keys are compared in FP32 (the order only places rows; a
  // positive mass stays positive): FP64 runs at a small fraction of the FP32
  // rate here. The keys sit in rrank until the ranks replace them.
  float* key = reinterpret_cast<float*>(rrank);
  if (tid == 0) s_count = 0;
  for (int k = tid; k < np; k += blockDim.x)
    key[k] = (mup[k] > 0.0) ? fmaxf((float)mup[k], 1.17549435e-38f) : 0.f;
  __syncthreads();
  int rk[MAXK];
  int mine = 0;
#pragma unroll
  for (int u = 0; u < MAXK; ++u) {
    const int k = tid + u * (int)blockDim.x;
    rk[u] = -1;
    if (k < np) {
      const float v = key[k];
      if (v > 0.f) {
        int r = 0;
        for (int i = 0; i < np; ++i) {
          const float w = key[i];
          r += (w > v) || (w == v && i < k);
        }
        rk[u] = r;
        ++mine;
      }
    }
  }
  if (mine) atomicAdd(&s_count, mine);
  __syncthreads();
#pragma unroll
  for (int u = 0; u < MAXK; ++u) {
    const int k = tid + u * (int)blockDim.x;
    if (k < np) rrank[k] = rk[u];
  }
  __syncthreads();

  if (tid == 0) { *count_out = s_count; *dsum_out = s_dsum; *dlast_out = s_dlast; }
  __syncthreads();
}

// FP64 bookkeeping of one reduction (thread 0) and the spectrum diagnostics.
// total_mass >= 0: sum of all sigma^2 (the trace of G) when mu holds only the
// leading values; otherwise the sum of mu.
static __device__ void write_counters(const EigArgs& a, int n, const double* mu, const double* mup,
                               int count, double dsum, double dlast, int capped, int sweeps,
                               double total_mass = -1.0, int fallback = 0) {
  const int tid = threadIdx.x;
  const int nout = a.ell - 1;
  if (a.sig2_out) for (int k = tid; k < n; k += blockDim.x) { a.sig2_out[k] = mu[k]; a.sigp2_out[k] = mup[k]; }
  if (tid < 32) {  // one warp: the sums in FP64
    double rem = 0.0, nb = 0.0;
    for (int k = tid; k < n; k += 32) { rem += mu[k] - mup[k]; nb += mup[k]; }
    rem = warp_sum(rem);
    nb = warp_sum(nb);
    if (total_mass >= 0.0) rem = total_mass - nb;
    if (tid != 0) return;
    DevCounters c = *a.ctr_in;
    c.sum_delta += dsum;
    c.last_delta = dlast;
    c.removed += rem;
    c.norm_b2 = nb;
    c.reductions += 1;
    c.noconv += capped ? 1 : 0;
    c.fallbacks += fallback ? 1 : 0;
    c.max_sweeps = fmax(c.max_sweeps, (double)sweeps);
    c.retained = count < nout ? count : nout;
    *a.ctr_out = c;
  }
}

template <typename T>
__device__ void eig_finish(const EigArgs& a, const T* Wm, int ld, int n, int np, int sweep,
                           int capped, double wscale, double* lam, double* mu, double* mup,
                           double* scl, int* ord, int* rrank) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  // lambda_j = ||w_j|| in FP64 (one warp per column).
  for (int j = warp; j < np; j += nwarps) {
    double s = 0.0;
    for (int i = lane; i < np; i += 32) {
      const double v = (double)Wm[(int64_t)j * ld + i];
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) lam[j] = (j < n) ? sqrt(s) * wscale : -1.0;  // padding column sorts last
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
  __syncthreads();

  __shared__ int s_cnt;
  __shared__ double s_ds, s_dl;
  shrink_sorted(a, n, np, Eps<T>::v, mu, mup, rrank, &s_cnt, &s_ds, &s_dl);
  for (int k = tid; k < np; k += blockDim.x) {
    const double v = mup[k];
    // scale of column w_j: sigma'/sigma / lambda = sqrt(mu'/mu) / mu
    scl[k] = (v > 0.0 && mu[k] > 0.0) ? sqrt(v / mu[k]) / mu[k] : 0.0;
  }
  const int s_count = s_cnt;
  __syncthreads();

  // 7. Rotate matrix rows 0..ell-2: row r = scale * w_j (zero rows past the count).
  const int nout = a.ell - 1;
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
  if (a.row_mass)
    for (int k = tid; k < np; k += blockDim.x) {
      const int r = rrank[k];
      if (r >= 0 && r < nout) a.row_mass[r] = mup[k];
      if (k < nout && k >= s_count) a.row_mass[k] = 0.0;
    }
  for (int k = warp; k < np; k += nwarps) {
    const int r = rrank[k];
    if (r < 0 || r >= nout) continue;
    const int j = ord[k];
    const double sc = scl[k] * wscale;
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

  double tr = -1.0;
  if (a.diag64 != nullptr) {
    __shared__ double s_tr;
    if (tid < 32) {
      const double t = eig_trace(a, Wm, ld, n, wscale);
      if (tid == 0) s_tr = t;
    }
    __syncthreads();
    tr = s_tr;
  }
  write_counters(a, n, mu, mup, s_count, s_ds, s_dl, capped, sweep, tr);
}


}  // namespace fdk
