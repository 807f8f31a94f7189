// Covariance-error evaluator that allocates nothing.
//
// For callers that cannot call cudaMalloc: code running inside a custom
// device allocator or a memory-pool callback (where a nested allocation would
// re-enter the allocator), runtimes that account for every byte of device
// memory themselves, and inference servers that forbid allocation after
// start-up. The caller passes A and B in device memory and receives the value
// on the host; all intermediate vectors live in one file-scope device array of
// fixed size, which every GPU that loads the library keeps until the process
// exits.
//
// The evaluation is the Lanczos process of fd_coverr.cu written against that
// fixed workspace: one product M x = A^T (A x) - B^T (B x) is a single pass
// over A (each CTA forms row dots for its rows and accumulates a_i * (a_i . x)
// into a per-CTA partial vector), followed by a fixed-order sum of the
// partials, so no buffer grows with the number of rows.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "fd_internal.cuh"

namespace fdk {

namespace {

constexpr int NA_MAX_D = 1024;      // widest A and B
constexpr int NA_MAX_ROWS_B = 512;  // most sketch rows
constexpr int NA_KMAX = 256;        // most Lanczos steps
constexpr int NA_NCH = 304;         // CTAs of one product (partial vectors)
constexpr int NA_THREADS = 256;

// Workspace layout (doubles).
constexpr size_t OFF_V = 0;                                          // (KMAX+1) x MAX_D
constexpr size_t OFF_PART = OFF_V + (size_t)(NA_KMAX + 1) * NA_MAX_D;  // NCH x MAX_D
constexpr size_t OFF_W = OFF_PART + (size_t)NA_NCH * NA_MAX_D;       // MAX_D
constexpr size_t OFF_C = OFF_W + NA_MAX_D;                           // KMAX + 2
constexpr size_t OFF_TB = OFF_C + NA_KMAX + 2;                       // MAX_ROWS_B
constexpr size_t OFF_AL = OFF_TB + NA_MAX_ROWS_B;                    // KMAX + 1
constexpr size_t OFF_BE = OFF_AL + NA_KMAX + 1;                      // KMAX + 1
constexpr size_t OFF_SC = OFF_BE + NA_KMAX + 1;                      // 2 (KMAX + 1)
constexpr size_t OFF_RES = OFF_SC + 2 * (NA_KMAX + 1);               // 4
constexpr size_t OFF_NRM = OFF_RES + 4;                              // NCH (row norms)
constexpr size_t OFF_NA = OFF_NRM + NA_NCH;                          // 1
constexpr size_t NA_WORDS = OFF_NA + 8;

// The workspace: about 4.6 MB.
static __device__ __align__(256) double g_noalloc_ws[NA_WORDS];

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One pass over A: partial[c][k] = sum over this CTA's rows of a_ik (a_i . x)
// (FP64 accumulation); with want_norm, also this CTA's sum of ||a_i||^2.
template <typename TA>
__global__ void __launch_bounds__(NA_THREADS) na_matvec_kernel(const TA* __restrict__ A,
                                                               int64_t n, int d, int64_t lda,
                                                               const double* __restrict__ x,
                                                               double* __restrict__ partial,
                                                               double* __restrict__ nrm_part,
                                                               int want_norm) {
  __shared__ double ys[NA_MAX_D];
  __shared__ double xs[NA_MAX_D];
  __shared__ double red[NA_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = NA_THREADS / 32;
  for (int k = threadIdx.x; k < d; k += NA_THREADS) { ys[k] = 0.0; xs[k] = x[k]; }
  __syncthreads();
  const int64_t rpc = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = min(n, r0 + rpc);
  double yl[NA_MAX_D / 32];
#pragma unroll
  for (int j = 0; j < NA_MAX_D / 32; ++j) yl[j] = 0.0;
  double nsum = 0.0;
  for (int64_t i = r0 + warp; i < r1; i += nwarps) {
    const TA* a = A + i * lda;
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < NA_MAX_D / 32; ++j) {
      const int k = lane + 32 * j;
      if (k < d) {
        const double av = (double)a[k];
        t = fma(av, xs[k], t);
        if (want_norm) nsum = fma(av, av, nsum);
      }
    }
    t = wsum(t);
#pragma unroll
    for (int j = 0; j < NA_MAX_D / 32; ++j) {
      const int k = lane + 32 * j;
      if (k < d) yl[j] = fma((double)a[k], t, yl[j]);
    }
  }
  // warps add their partial vectors in a fixed order
  for (int w = 0; w < nwarps; ++w) {
    if (warp == w) {
#pragma unroll
      for (int j = 0; j < NA_MAX_D / 32; ++j) {
        const int k = lane + 32 * j;
        if (k < d) ys[k] += yl[j];
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < d; k += NA_THREADS) partial[(int64_t)blockIdx.x * NA_MAX_D + k] = ys[k];
  if (want_norm) {
    nsum = wsum(nsum);
    if (lane == 0) red[warp] = nsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[w];
      nrm_part[blockIdx.x] = s;
    }
  }
}

template <typename TB>
__global__ void na_bdot_kernel(const TB* __restrict__ B, int64_t rows, int d,
                               const double* __restrict__ x, double* __restrict__ tb) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= rows) return;
  double acc = 0.0;
  for (int k = lane; k < d; k += 32) acc = fma((double)B[w * d + k], x[k], acc);
  acc = wsum(acc);
  if (lane == 0) tb[w] = acc;
}

// y_k = sum_c partial[c][k] - sum_r b_rk tb_r
template <typename TB>
__global__ void na_finish_kernel(const double* __restrict__ partial, int nch, int d,
                                 const TB* __restrict__ B, int64_t rows,
                                 const double* __restrict__ tb, double* __restrict__ y) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double s = 0.0;
  for (int c = 0; c < nch; ++c) s += partial[(int64_t)c * NA_MAX_D + k];
  double sb = 0.0;
  for (int64_t r = 0; r < rows; ++r) sb = fma((double)B[r * d + k], tb[r], sb);
  y[k] = s - sb;
}

__global__ void na_sum_kernel(const double* __restrict__ a, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i];
    out[0] = s;
  }
}

__global__ void na_dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int n,
                              double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc = fma(a[k], b[k], acc);
  acc = wsum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    out[0] = s;
  }
}

__global__ void na_three_term_kernel(double* __restrict__ w, const double* __restrict__ vj,
                                     const double* __restrict__ vjm1,
                                     const double* __restrict__ alpha,
                                     const double* __restrict__ beta_prev, int d) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double v = w[k] - alpha[0] * vj[k];
  if (vjm1) v -= beta_prev[0] * vjm1[k];
  w[k] = v;
}

__global__ void na_vdots_kernel(const double* __restrict__ V, int nv, int d,
                                const double* __restrict__ w, double* __restrict__ c) {
  const int lane = threadIdx.x & 31;
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (v >= nv) return;
  double acc = 0.0;
  for (int k = lane; k < d; k += 32) acc = fma(V[(int64_t)v * NA_MAX_D + k], w[k], acc);
  acc = wsum(acc);
  if (lane == 0) c[v] = acc;
}

__global__ void na_vaxpy_kernel(const double* __restrict__ V, int nv, int d,
                                const double* __restrict__ c, double* __restrict__ w) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double s = 0.0;
  for (int v = 0; v < nv; ++v) s = fma(c[v], V[(int64_t)v * NA_MAX_D + k], s);
  w[k] -= s;
}

__global__ void na_normalize_kernel(const double* __restrict__ w, const double* __restrict__ ww,
                                    double* __restrict__ vnext, double* __restrict__ beta_out,
                                    int d) {
  const double b = sqrt(fmax(ww[0], 0.0));
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) beta_out[0] = b;
  if (k >= d) return;
  vnext[k] = (b > 0.0) ? w[k] / b : 0.0;
}

__global__ void na_start_kernel(double* __restrict__ w, int d) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  uint64_t z = (uint64_t)k * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  w[k] = ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 0.5;
}

__device__ int na_sturm(const double* a, const double* b, int k, double x) {
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

__device__ double na_eig(const double* a, const double* b, int k, int idx, double lo, double hi) {
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (na_sturm(a, b, k, mid) > idx) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

__device__ double na_last_comp(const double* a, const double* b, int k, double theta, double* cp,
                               double* z, double eps) {
  for (int i = 0; i < k; ++i) z[i] = 1.0;
  for (int rep = 0; rep < 3; ++rep) {
    double den = a[0] - theta;
    if (fabs(den) < eps) den = eps;
    cp[0] = (k > 1) ? b[0] / den : 0.0;
    z[0] = z[0] / den;
    for (int i = 1; i < k; ++i) {
      den = (a[i] - theta) - b[i - 1] * cp[i - 1];
      if (fabs(den) < eps) den = (den < 0 ? -eps : eps);
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

__global__ void na_tri_check_kernel(const double* __restrict__ alpha,
                                    const double* __restrict__ beta, int k,
                                    double* __restrict__ scratch, double* __restrict__ out) {
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
  const double tmin = na_eig(alpha, beta, k, 0, lo, hi);
  const double tmax = na_eig(alpha, beta, k, k - 1, lo, hi);
  const double eps = 1e-14 * span;
  const double smin = na_last_comp(alpha, beta, k, tmin, scratch, scratch + k, eps);
  const double smax = na_last_comp(alpha, beta, k, tmax, scratch, scratch + k, eps);
  const double bk = fabs(beta[k - 1]);
  out[0] = tmin;
  out[1] = tmax;
  out[2] = bk * smin;
  out[3] = bk * smax;
}

// Device address of the workspace, looked up once per device.
constexpr int NA_MAX_DEVICES = 64;
double* g_ws_ptr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_ws_mu;

int workspace(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_cuda_error(e, "cudaGetDevice"); return FD_ECUDA; }
  if (dev < 0 || dev >= NA_MAX_DEVICES) return FD_EINVAL;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  if (!g_ws_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess) { set_cuda_error(e, "cudaGetSymbolAddress"); return FD_ECUDA; }
    g_ws_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ws_ptr[dev];
  return FD_OK;
}

template <typename TA, typename TB>
int na_lanczos(const TA* A, int64_t n, int d, int64_t lda, const TB* B, int64_t rows,
               cudaStream_t st, double* ws, double* cov) {
  double* V = ws + OFF_V;
  double* part = ws + OFF_PART;
  double* w = ws + OFF_W;
  double* c = ws + OFF_C;
  double* tb = ws + OFF_TB;
  double* al = ws + OFF_AL;
  double* be = ws + OFF_BE;
  double* sc = ws + OFF_SC;
  double* res = ws + OFF_RES;
  double* nrm = ws + OFF_NRM;
  double* na = ws + OFF_NA;
  const int kmax = std::min(d, NA_KMAX);
  const int nch = (int)std::max<int64_t>(1, std::min<int64_t>(NA_NCH, (n + 31) / 32));
  const unsigned dblocks = (unsigned)((d + 255) / 256);
  // every call starts from a cleared workspace (results of an earlier call
  // must not leak into this one)
  cudaError_t e = cudaMemsetAsync(ws, 0, NA_WORDS * sizeof(double), st);
  if (e != cudaSuccess) { set_cuda_error(e, "noalloc clear"); return FD_ECUDA; }
  auto matvec = [&](const double* x, int want_norm) {
    na_matvec_kernel<TA><<<nch, NA_THREADS, 0, st>>>(A, n, d, lda, x, part, nrm, want_norm);
    if (rows > 0)
      na_bdot_kernel<TB><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(B, rows, d, x, tb);
    na_finish_kernel<TB><<<dblocks, 256, 0, st>>>(part, nch, d, B, rows, tb, w);
  };
  na_start_kernel<<<dblocks, 256, 0, st>>>(w, d);
  na_dot_kernel<<<1, 1024, 0, st>>>(w, w, d, c);
  na_normalize_kernel<<<dblocks, 256, 0, st>>>(w, c, V, c + 1, d);
  double h[4] = {0, 0, 0, 0};
  double h_norm = 0.0;
  for (int j = 0; j < kmax; ++j) {
    const double* vj = V + (size_t)j * NA_MAX_D;
    matvec(vj, j == 0 ? 1 : 0);
    if (j == 0) na_sum_kernel<<<1, 32, 0, st>>>(nrm, nch, na);
    na_dot_kernel<<<1, 1024, 0, st>>>(vj, w, d, al + j);
    na_three_term_kernel<<<dblocks, 256, 0, st>>>(
        w, vj, j > 0 ? V + (size_t)(j - 1) * NA_MAX_D : nullptr, al + j,
        j > 0 ? be + (j - 1) : nullptr, d);
    for (int pass = 0; pass < 2; ++pass) {
      na_vdots_kernel<<<(unsigned)(((j + 1) * 32 + 255) / 256), 256, 0, st>>>(V, j + 1, d, w, c);
      na_vaxpy_kernel<<<dblocks, 256, 0, st>>>(V, j + 1, d, c, w);
    }
    na_dot_kernel<<<1, 1024, 0, st>>>(w, w, d, c);
    na_normalize_kernel<<<dblocks, 256, 0, st>>>(w, c, V + (size_t)(j + 1) * NA_MAX_D, be + j, d);
    const int k = j + 1;
    const bool last = (k == kmax);
    if ((k >= 4 && (k % 8) == 0) || last) {  // always check at the last step (d < 4 too)
      na_tri_check_kernel<<<1, 32, 0, st>>>(al, be, k, sc, res);
      e = cudaMemcpyAsync(h, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h_norm, na, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { set_cuda_error(e, "noalloc lanczos"); return FD_ECUDA; }
      const double tol = 1e-10 * std::max(h_norm, 1e-300);
      if ((h[2] <= tol && h[3] <= tol) || last) break;
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e, "noalloc kernels"); return FD_ECUDA; }
  *cov = (h_norm > 0.0) ? std::max(std::fabs(h[0]), std::fabs(h[1])) / h_norm : 0.0;
  return FD_OK;
}

}  // namespace

}  // namespace fdk

using namespace fdk;

extern "C" int fd_cov_err_noalloc(const void* A, int64_t n, int64_t d, int64_t lda,
                                  int32_t a_dtype, const void* B, int64_t rows, int32_t b_dtype,
                                  void* cuda_stream, double* cov_err) {
  if (!A || !cov_err || n < 1 || d < 1 || lda < d || rows < 0 || (rows > 0 && !B))
    return FD_EINVAL;
  if ((a_dtype != FD_F32 && a_dtype != FD_F64) || (b_dtype != FD_F32 && b_dtype != FD_F64))
    return FD_EINVAL;
  if (d > NA_MAX_D || rows > NA_MAX_ROWS_B) return FD_ETOOBIG;
  double* ws = nullptr;
  int rc = workspace(&ws);
  if (rc != FD_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int di = (int)d;
  if (a_dtype == FD_F64 && b_dtype == FD_F64)
    return na_lanczos<double, double>((const double*)A, n, di, lda, (const double*)B, rows, st, ws, cov_err);
  if (a_dtype == FD_F64)
    return na_lanczos<double, float>((const double*)A, n, di, lda, (const float*)B, rows, st, ws, cov_err);
  if (b_dtype == FD_F64)
    return na_lanczos<float, double>((const float*)A, n, di, lda, (const double*)B, rows, st, ws, cov_err);
  return na_lanczos<float, float>((const float*)A, n, di, lda, (const float*)B, rows, st, ws, cov_err);
}
