// Covariance-error evaluator: cov-err(A, B) = ||A^T A - B^T B||_2 / ||A||_F^2
// (Sec. 1.1), with ||M||_2 = max |eigenvalue| of the symmetric M.
//
// Lanczos with full reorthogonalisation on M = A^T A - B^T B. Each product
// M x streams A twice from HBM (t = A x, then A^T t) and never forms the d x d
// matrix; the small tridiagonal problem is solved on the device by Sturm
// bisection (extreme Ritz values) and inverse iteration (their residual
// bounds beta_k |s_k|). Iteration stops once both extreme Ritz values carry a
// residual bound below 1e-10 ||A||_F^2, or the Krylov space is exhausted.
//
// Projection-error evaluator: proj-err(A, B) = ||A - pi_{B_k}(A)||_F^2 /
// ||A - A_k||_F^2 (Sec. 1.1). The same Lanczos on M = A^T A gives the k
// largest eigenvalues (stopped once each carries a residual bound below
// 1e-10 ||A||_F^2), so ||A - A_k||_F^2 = ||A||_F^2 - sum of them; one more
// pass over A gives sum_j ||A v_j||^2 for the top right singular vectors v_j
// of B, so the numerator is ||A||_F^2 minus that sum.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fd_internal.cuh"

namespace fdk {

namespace {

constexpr int CE_THREADS = 256;

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// t_i = a_i . x for every row (one warp per row), FP32 products in groups of 8
// added into FP64; optionally also ||a_i||^2 into rownorm.
template <typename TA>
__global__ void rows_dot_kernel(const TA* __restrict__ A, int64_t n, int64_t d, int64_t lda,
                                const double* __restrict__ x, double* __restrict__ t,
                                double* __restrict__ rownorm) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n; i += nw) {
    const TA* a = A + i * lda;
    double acc = 0.0, nrm = 0.0;
    TA part = TA(0);
    int cnt = 0;
    for (int64_t k = lane; k < d; k += 32) {
      const TA av = a[k];
      part = fma(av, (TA)x[k], part);
      if (rownorm) nrm = fma((double)av, (double)av, nrm);
      if (++cnt == 8) { acc += (double)part; part = TA(0); cnt = 0; }
    }
    acc += (double)part;
    acc = warp_sum_t(acc);
    if (rownorm) nrm = warp_sum_t(nrm);
    if (lane == 0) {
      t[i] = acc;
      if (rownorm) rownorm[i] = nrm;
    }
  }
}

// partial[c][k] = sum over rows of chunk c of a_ik t_i (column per thread).
template <typename TA>
__global__ void cols_acc_kernel(const TA* __restrict__ A, int64_t n, int64_t d, int64_t lda,
                                const double* __restrict__ t, int64_t rows_per_chunk,
                                double* __restrict__ partial) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  if (k >= d) return;
  double acc = 0.0;
  TA part = TA(0);
  int cnt = 0;
  for (int64_t i = r0; i < r1; ++i) {
    part = fma(A[i * lda + k], (TA)t[i], part);
    if (++cnt == 16) { acc += (double)part; part = TA(0); cnt = 0; }
  }
  acc += (double)part;
  partial[(int64_t)blockIdx.y * d + k] = acc;
}

// y_k = sum_c partial[c][k] - sum_r b_rk (B x)_r, fixed order.
template <typename TB>
__global__ void finish_matvec_kernel(const double* __restrict__ partial, int nchunks, int64_t d,
                                     const TB* __restrict__ B, int64_t rows, int64_t ldb,
                                     const double* __restrict__ tb, double* __restrict__ y) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[(int64_t)c * d + k];
  double sb = 0.0;
  for (int64_t r = 0; r < rows; ++r) sb = fma((double)B[r * ldb + k], tb[r], sb);
  y[k] = s - sb;
}

// tb_r = b_r . x in FP64 (B is tiny).
template <typename TB>
__global__ void b_dot_kernel(const TB* __restrict__ B, int64_t rows, int64_t d, int64_t ldb,
                             const double* __restrict__ x, double* __restrict__ tb) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= rows) return;
  double acc = 0.0;
  for (int64_t k = lane; k < d; k += 32) acc = fma((double)B[w * ldb + k], x[k], acc);
  acc = warp_sum_t(acc);
  if (lane == 0) tb[w] = acc;
}

// c_v = V_v . w for v < nv (one warp per vector).
__global__ void vdots_kernel(const double* __restrict__ V, int nv, int64_t d,
                             const double* __restrict__ w, double* __restrict__ c) {
  const int lane = threadIdx.x & 31;
  const int v = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (v >= nv) return;
  double acc = 0.0;
  for (int64_t k = lane; k < d; k += 32) acc = fma(V[(int64_t)v * d + k], w[k], acc);
  acc = warp_sum_t(acc);
  if (lane == 0) c[v] = acc;
}

// w_k -= sum_v c_v V_vk
__global__ void vaxpy_kernel(const double* __restrict__ V, int nv, int64_t d,
                             const double* __restrict__ c, double* __restrict__ w) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double s = 0.0;
  for (int v = 0; v < nv; ++v) s = fma(c[v], V[(int64_t)v * d + k], s);
  w[k] -= s;
}

// Single-block reductions: sum of squares / dot into out[0].
__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) acc = fma(a[k], b[k], acc);
  __shared__ double red[32];
  acc = warp_sum_t(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    out[0] = s;
  }
}

__global__ void sum_kernel(const double* __restrict__ a, int64_t n, double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) acc += a[k];
  __shared__ double red[32];
  acc = warp_sum_t(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    out[0] = s;
  }
}

// Lanczos three-term step on w = M v_j:
//   alpha_j = v_j . w;  w -= alpha_j v_j + beta_{j-1} v_{j-1}
__global__ void three_term_kernel(double* __restrict__ w, const double* __restrict__ vj,
                                  const double* __restrict__ vjm1, const double* __restrict__ alpha,
                                  const double* __restrict__ beta_prev, int64_t d) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double v = w[k] - alpha[0] * vj[k];
  if (vjm1) v -= beta_prev[0] * vjm1[k];
  w[k] = v;
}

// v_{j+1} = w / beta (beta = sqrt(ww)); beta written to beta_out.
__global__ void normalize_kernel(const double* __restrict__ w, const double* __restrict__ ww,
                                 double* __restrict__ vnext, double* __restrict__ beta_out,
                                 int64_t d) {
  const double b = sqrt(fmax(ww[0], 0.0));
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) beta_out[0] = b;
  if (k >= d) return;
  vnext[k] = (b > 0.0) ? w[k] / b : 0.0;
}

// Deterministic start vector (a fixed integer hash per coordinate), unit norm
// applied by normalize_kernel.
__global__ void start_kernel(double* __restrict__ w, int64_t d) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  uint64_t z = (uint64_t)k * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  w[k] = ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 0.5;
}

// Number of eigenvalues of the tridiagonal (a, b) below x (Sturm sequence).
__device__ int sturm_count(const double* a, const double* b, int k, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < k; ++i) {
    if (fabs(q) < 1e-300) q = (q < 0 ? -1e-300 : 1e-300);
    q = a[i] - x - b[i - 1] * b[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Eigenvalue number `idx` (0 = smallest) of the tridiagonal by bisection.
__device__ double tri_eig(const double* a, const double* b, int k, int idx, double lo, double hi) {
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, k, mid) > idx) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// |last component| of the unit eigenvector of the tridiagonal at theta, by
// inverse iteration (three solves of (T - theta I) z = z_prev, Thomas).
__device__ double tri_last_component(const double* a, const double* b, int k, double theta,
                                     double* cp, double* z, double shift_eps) {
  for (int i = 0; i < k; ++i) z[i] = 1.0;
  for (int rep = 0; rep < 3; ++rep) {
    // forward sweep
    double den = a[0] - theta;
    if (fabs(den) < shift_eps) den = shift_eps;
    cp[0] = (k > 1) ? b[0] / den : 0.0;
    z[0] = z[0] / den;
    for (int i = 1; i < k; ++i) {
      den = (a[i] - theta) - b[i - 1] * cp[i - 1];
      if (fabs(den) < shift_eps) den = (den < 0 ? -shift_eps : shift_eps);
      cp[i] = (i < k - 1) ? b[i] / den : 0.0;
      z[i] = (z[i] - b[i - 1] * z[i - 1]) / den;
    }
    for (int i = k - 2; i >= 0; --i) z[i] -= cp[i] * z[i + 1];
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm = fmax(nrm, fabs(z[i]));
    if (!(nrm > 0.0)) return 1.0;
    for (int i = 0; i < k; ++i) z[i] /= nrm;
  }
  double s2 = 0.0;
  for (int i = 0; i < k; ++i) s2 += z[i] * z[i];
  return fabs(z[k - 1]) / sqrt(s2);
}

// out: [theta_min, theta_max, resid_min, resid_max]
__global__ void tri_check_kernel(const double* __restrict__ alpha, const double* __restrict__ beta,
                                 int k, double* __restrict__ scratch, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i < k - 1 ? fabs(beta[i]) : 0.0);
    lo = fmin(lo, alpha[i] - r);
    hi = fmax(hi, alpha[i] + r);
  }
  const double span = fmax(hi - lo, 1e-300);
  lo -= 1e-12 * span;
  hi += 1e-12 * span;
  const double tmin = tri_eig(alpha, beta, k, 0, lo, hi);
  const double tmax = tri_eig(alpha, beta, k, k - 1, lo, hi);
  const double eps = 1e-14 * span;
  double* cp = scratch;
  double* z = scratch + k;
  const double smin = tri_last_component(alpha, beta, k, tmin, cp, z, eps);
  const double smax = tri_last_component(alpha, beta, k, tmax, cp, z, eps);
  const double bk = fabs(beta[k - 1]);
  out[0] = tmin;
  out[1] = tmax;
  out[2] = bk * smin;
  out[3] = bk * smax;
}

// The topk largest Ritz values (descending) and their residual bounds
// beta_k |s_k|: out[i] = theta_i, out[topk + i] = bound_i (zero past k).
// One thread per value; scratch: 2 k doubles per thread.
__global__ void tri_topk_kernel(const double* __restrict__ alpha, const double* __restrict__ beta,
                                int k, int topk, double* __restrict__ scratch,
                                double* __restrict__ out) {
  const int i = threadIdx.x;
  if (i >= topk) return;
  if (i >= k) {
    out[i] = 0.0;
    out[topk + i] = 0.0;
    return;
  }
  double lo = 1e300, hi = -1e300;
  for (int q = 0; q < k; ++q) {
    const double r = (q > 0 ? fabs(beta[q - 1]) : 0.0) + (q < k - 1 ? fabs(beta[q]) : 0.0);
    lo = fmin(lo, alpha[q] - r);
    hi = fmax(hi, alpha[q] + r);
  }
  const double span = fmax(hi - lo, 1e-300);
  lo -= 1e-12 * span;
  hi += 1e-12 * span;
  const double th = tri_eig(alpha, beta, k, k - 1 - i, lo, hi);
  const double sk = tri_last_component(alpha, beta, k, th, scratch + (size_t)2 * k * i,
                                       scratch + (size_t)2 * k * i + k, 1e-14 * span);
  out[i] = th;
  out[topk + i] = fabs(beta[k - 1]) * sk;
}

// topk = 0: extreme eigenvalues of M (cov-err). topk > 0: the topk largest
// eigenvalues into top_out (descending). norm_out (optional): ||A||_F^2.
template <typename TA, typename TB>
int run_lanczos(const TA* A, int64_t n, int64_t d, int64_t lda, const TB* B, int64_t rows,
                int64_t ldb, cudaStream_t st, double* cov, double* lmin, double* lmax,
                int topk = 0, double* top_out = nullptr, double* norm_out = nullptr) {
  const int kmax = (int)std::min<int64_t>(d, 1200);
  const int ct = (int)((d + 127) / 128);
  const int nchunks = std::max(1, std::min<int>((int)((n + 255) / 256), 608 / std::max(1, ct)));
  const int64_t rpc = (n + nchunks - 1) / nchunks;
  double *V = nullptr, *t = nullptr, *rn = nullptr, *part = nullptr, *w = nullptr, *c = nullptr,
         *tb = nullptr, *al = nullptr, *be = nullptr, *sc = nullptr, *res = nullptr, *na = nullptr;
  auto cleanup = [&]() {
    cudaFree(V); cudaFree(t); cudaFree(rn); cudaFree(part); cudaFree(w); cudaFree(c);
    cudaFree(tb); cudaFree(al); cudaFree(be); cudaFree(sc); cudaFree(res); cudaFree(na);
  };
#define CE_ALLOC(p, cnt)                                              \
  if (cudaMalloc(&(p), sizeof(double) * (size_t)(cnt)) != cudaSuccess) { \
    cleanup();                                                        \
    set_cuda_error(cudaErrorMemoryAllocation, "cov-err workspace");  \
    return FD_ENOMEM;                                                 \
  }
  CE_ALLOC(V, (size_t)(kmax + 1) * d);
  CE_ALLOC(t, n);
  CE_ALLOC(rn, n);
  CE_ALLOC(part, (size_t)nchunks * d);
  CE_ALLOC(w, d);
  CE_ALLOC(c, kmax + 2);
  CE_ALLOC(tb, std::max<int64_t>(rows, 1));
  CE_ALLOC(al, kmax + 1);
  CE_ALLOC(be, kmax + 1);
  CE_ALLOC(sc, 2 * (size_t)(kmax + 1) * std::max(1, topk));
  CE_ALLOC(res, std::max(4, 2 * topk));
  CE_ALLOC(na, 1);
#undef CE_ALLOC
  const int rows_blocks = 608;
  const unsigned dblocks = (unsigned)((d + CE_THREADS - 1) / CE_THREADS);
  auto matvec = [&](const double* x, bool want_norm) {
    rows_dot_kernel<TA><<<rows_blocks, CE_THREADS, 0, st>>>(A, n, d, lda, x, t,
                                                            want_norm ? rn : nullptr);
    dim3 g((unsigned)ct, (unsigned)nchunks);
    cols_acc_kernel<TA><<<g, 128, 0, st>>>(A, n, d, lda, t, rpc, part);
    if (rows > 0)
      b_dot_kernel<TB><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(B, rows, d, ldb, x, tb);
    finish_matvec_kernel<TB><<<dblocks, CE_THREADS, 0, st>>>(part, nchunks, d, B, rows, ldb, tb, w);
  };
  // v_0
  start_kernel<<<dblocks, CE_THREADS, 0, st>>>(w, d);
  dot_kernel<<<1, 1024, 0, st>>>(w, w, d, c);
  normalize_kernel<<<dblocks, CE_THREADS, 0, st>>>(w, c, V, c + 1, d);
  std::vector<double> h(std::max(4, 2 * topk));
  double h_norm = 0.0;
  int k = 0;
  for (int j = 0; j < kmax; ++j) {
    const double* vj = V + (size_t)j * d;
    matvec(vj, j == 0);
    if (j == 0) {
      sum_kernel<<<1, 1024, 0, st>>>(rn, n, na);
    }
    dot_kernel<<<1, 1024, 0, st>>>(vj, w, d, al + j);
    three_term_kernel<<<dblocks, CE_THREADS, 0, st>>>(w, vj, j > 0 ? V + (size_t)(j - 1) * d : nullptr,
                                                      al + j, j > 0 ? be + (j - 1) : nullptr, d);
    for (int pass = 0; pass < 2; ++pass) {
      vdots_kernel<<<(unsigned)(((j + 1) * 32 + 255) / 256), 256, 0, st>>>(V, j + 1, d, w, c);
      vaxpy_kernel<<<dblocks, CE_THREADS, 0, st>>>(V, j + 1, d, c, w);
    }
    dot_kernel<<<1, 1024, 0, st>>>(w, w, d, c);
    normalize_kernel<<<dblocks, CE_THREADS, 0, st>>>(w, c, V + (size_t)(j + 1) * d, be + j, d);
    k = j + 1;
    const bool last = (k == kmax);
    if ((k >= 4 && (k % 8) == 0) || last) {  // always check at the last step (d < 4 too)
      const int nres = topk > 0 ? 2 * topk : 4;
      if (topk > 0)
        tri_topk_kernel<<<1, ((topk + 31) / 32) * 32, 0, st>>>(al, be, k, topk, sc, res);
      else
        tri_check_kernel<<<1, 32, 0, st>>>(al, be, k, sc, res);
      cudaError_t e = cudaMemcpyAsync(h.data(), res, nres * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h_norm, na, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { set_cuda_error(e, "cov-err lanczos"); cleanup(); return FD_ECUDA; }
      const double tol = 1e-10 * std::max(h_norm, 1e-300);
      bool conv = true;
      if (topk > 0) {
        for (int i = 0; i < topk; ++i) conv = conv && (h[topk + i] <= tol);
      } else {
        conv = (h[2] <= tol && h[3] <= tol);
      }
      if (conv || last) break;
    }
  }
  cudaError_t e = cudaGetLastError();
  cleanup();
  if (e != cudaSuccess) { set_cuda_error(e, "cov-err kernels"); return FD_ECUDA; }
  if (norm_out) *norm_out = h_norm;
  if (topk > 0) {
    for (int i = 0; i < topk; ++i) top_out[i] = h[i];
    return FD_OK;
  }
  *lmin = h[0];
  *lmax = h[1];
  *cov = (h_norm > 0.0) ? std::max(std::fabs(h[0]), std::fabs(h[1])) / h_norm : 0.0;
  return FD_OK;
}

// rinv2[j] = 1 / ||r_j||^2 (0 for a zero row), one warp per row of R (k x d).
__global__ void row_inv_norm2_kernel(const double* __restrict__ R, int k, int64_t d,
                                     double* __restrict__ rinv2) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = w; j < k; j += blockDim.x >> 5) {
    double acc = 0.0;
    for (int64_t c = lane; c < d; c += 32) acc = fma(R[(int64_t)j * d + c], R[(int64_t)j * d + c], acc);
    acc = warp_sum_t(acc);
    if (lane == 0) rinv2[j] = (acc > 0.0) ? 1.0 / acc : 0.0;
  }
}

template <typename TA>
__global__ void cast_rows_kernel(const double* __restrict__ R, int64_t cnt, TA* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TA)R[i];
}

// partial[block] = sum over the block's rows a_i of sum_j (a_i . r_j)^2 / ||r_j||^2:
// one warp per row, eight vectors at a time, FP32 products in groups of 8
// added into FP64 (as rows_dot_kernel).
template <typename TA>
__global__ void proj_rows_kernel(const TA* __restrict__ A, int64_t n, int64_t d, int64_t lda,
                                 const TA* __restrict__ R, const double* __restrict__ rinv2,
                                 int k, double* __restrict__ partial) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double mine = 0.0;
  for (int64_t i = gw; i < n; i += nw) {
    const TA* a = A + i * lda;
    double rowsum = 0.0;
    for (int j0 = 0; j0 < k; j0 += 8) {
      double acc[8];
      TA part[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) { acc[u] = 0.0; part[u] = TA(0); }
      int cnt = 0;
      for (int64_t c = lane; c < d; c += 32) {
        const TA av = a[c];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j0 + u < k) part[u] = fma(av, R[(int64_t)(j0 + u) * d + c], part[u]);
        if (++cnt == 8) {
#pragma unroll
          for (int u = 0; u < 8; ++u) { acc[u] += (double)part[u]; part[u] = TA(0); }
          cnt = 0;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const double t = warp_sum_t(acc[u] + (double)part[u]);
        if (j0 + u < k) rowsum += t * t * rinv2[j0 + u];
      }
    }
    mine += rowsum;  // identical in every lane
  }
  __shared__ double red[32];
  if (lane == 0) red[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

template <typename TA>
int run_proj(const TA* A, int64_t n, int64_t d, int64_t lda, const double* R, int k,
             cudaStream_t st, double* pe, double* num_out, double* den_out) {
  std::vector<double> top(k);
  double na2 = 0.0, dummy = 0.0;
  int rc = run_lanczos<TA, double>(A, n, d, lda, nullptr, 0, d, st, &dummy, &dummy, &dummy, k,
                                   top.data(), &na2);
  if (rc != FD_OK) return rc;
  const int blocks = 608;
  double *rinv2 = nullptr, *part = nullptr, *out = nullptr;
  TA* Rt = nullptr;
  auto cleanup = [&]() { cudaFree(rinv2); cudaFree(part); cudaFree(out); cudaFree(Rt); };
  if (cudaMalloc(&rinv2, sizeof(double) * k) != cudaSuccess ||
      cudaMalloc(&part, sizeof(double) * blocks) != cudaSuccess ||
      cudaMalloc(&out, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&Rt, sizeof(TA) * (size_t)k * d) != cudaSuccess) {
    cleanup();
    set_cuda_error(cudaErrorMemoryAllocation, "proj-err workspace");
    return FD_ENOMEM;
  }
  row_inv_norm2_kernel<<<1, 256, 0, st>>>(R, k, d, rinv2);
  cast_rows_kernel<TA><<<256, 256, 0, st>>>(R, (int64_t)k * d, Rt);
  proj_rows_kernel<TA><<<blocks, CE_THREADS, 0, st>>>(A, n, d, lda, Rt, rinv2, k, part);
  sum_kernel<<<1, 1024, 0, st>>>(part, blocks, out);
  double cap = 0.0;
  cudaError_t e = cudaMemcpyAsync(&cap, out, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) { set_cuda_error(e, "proj-err kernels"); return FD_ECUDA; }
  double topsum = 0.0;
  for (int i = 0; i < k; ++i) topsum += top[i];
  // A of rank at most k (k >= d, or a denominator at the Lanczos run's
  // resolution of 1e-10 ||A||_F^2 per value) has ||A - A_k||_F^2 = 0; the
  // ratio is then 1 when B_k captures A as well (a numerator at the
  // resolution of the FP32 products), and unbounded otherwise
  double num = na2 - cap, den = (k >= d) ? 0.0 : na2 - topsum;
  if (den <= 10.0 * k * 1e-10 * na2) den = 0.0;
  if (den == 0.0 && num <= 1e-6 * na2) num = 0.0;
  if (num_out) *num_out = num;
  if (den_out) *den_out = den;
  if (den <= 0.0) *pe = (num <= 0.0) ? 1.0 : INFINITY;
  else *pe = num / den;
  return FD_OK;
}

}  // namespace

int proj_err_device(const void* A, int64_t n, int64_t d, int64_t lda, int a_f64, const double* R,
                    int k, cudaStream_t st, double* pe, double* num, double* den) {
  if (a_f64) return run_proj<double>((const double*)A, n, d, lda, R, k, st, pe, num, den);
  return run_proj<float>((const float*)A, n, d, lda, R, k, st, pe, num, den);
}

int cov_err_device(const void* A, int64_t n, int64_t d, int64_t lda, int a_f64, const void* B,
                   int64_t rows, int64_t ldb, int b_f64, cudaStream_t st, double* cov,
                   double* lmin, double* lmax) {
  if (a_f64 && b_f64)
    return run_lanczos<double, double>((const double*)A, n, d, lda, (const double*)B, rows, ldb,
                                       st, cov, lmin, lmax);
  if (a_f64)
    return run_lanczos<double, float>((const double*)A, n, d, lda, (const float*)B, rows, ldb, st,
                                      cov, lmin, lmax);
  if (b_f64)
    return run_lanczos<float, double>((const float*)A, n, d, lda, (const double*)B, rows, ldb, st,
                                      cov, lmin, lmax);
  return run_lanczos<float, float>((const float*)A, n, d, lda, (const float*)B, rows, ldb, st,
                                   cov, lmin, lmax);
}

}  // namespace fdk
