// Internal declarations shared by the translation units of libfdsketch.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <math.h>

#include "fdsketch.h"

namespace fdk {

// FP64 bookkeeping of one sketch, kept on the device so that a whole
// reduction (Gram -> eigensolve -> shrink -> rotate) needs no host round trip.
struct DevCounters {
  double norm_a2;      // ||A||_F^2 of the rows ingested so far
  double sum_delta;    // Delta (Sec. 3.1): every delta subtracted
  double last_delta;
  double removed;      // sum_j (sigma_j^2 - sigma'_j^2) over reductions
  double norm_b2;      // ||B||_F^2 after the latest reduction
  double max_sweeps;
  long long reductions;
  long long noconv;
  long long fallbacks;  // eigensolves whose eigenvectors needed the fallback path
  unsigned int ingest_ticket;  // last-block-done counter of the ingest kernel
  int retained;                // rows with sigma' > 0 after the latest reduction
};

// Parameters of the fused eigensolve + shrink kernel (one CTA per reduction).
struct EigArgs {
  const void* parts;   // Gram partial sums: nparts slices of ldp x ldp (T)
  int nparts;
  int ldp;
  long long part_stride;  // elements between slices
  int symmetrize;      // informational: the load always takes G = (Z + Z^T) / 2
  int n;               // rows being reduced (2*ell, or fewer at a flush)
  int ell;
  int variant;
  double alpha;
  void* work;          // global G when it does not fit in shared memory (n x ldw)
  int ldw_work;
  size_t work_bytes;   // size of work
  const DevCounters* ctr_in;
  DevCounters* ctr_out;
  double* sig2_out;    // sorted sigma^2 (n) or null
  double* sigp2_out;   // sigma'^2 aligned with it, or null
  void* wrot;          // rotate matrix rows 0..ell-2 (T), ld = ldr
  int ldr;
  __nv_bfloat16* wrot_hi;  // optional split copies (BF16 hi / lo) for tcgen05
  __nv_bfloat16* wrot_lo;
  int ldr16;
  int max_sweeps;
  double tol;          // rotate when |gamma| > tol * sqrt(alpha * beta)
  int use_tri;         // 1: tridiagonal eigensolve where it applies (FP32)
  double* row_mass;    // optional: sigma'^2 of each output row r (ell-1 entries)
  // Exact Gram diagonal of a tensor-core buffer (FD_PREC_BF16X3), optional
  // (diag64 != null enables it). The split products drop lo*lo, which on the
  // diagonal is a sum of squares and so a bias (about 2^-19.6 of each squared
  // norm); the diagonal is replaced by the FP64 squared norms of the rows as
  // stored: rows 0..nret-1 (written by the previous rotate) from the rotate's
  // per-CTA partial sums, added in a fixed order; the others from slot_n2,
  // written at ingest.
  int nret;
  const double* rot_part;     // rot_nparts x rot_ld partial squared norms of rows 0..nret-1
  int rot_nparts, rot_ld;
  const double* slot_n2;      // FP64 squared norm of every stored new row
  double* diag64;             // out: the exact diagonal, n entries
  // Rayleigh-quotient refinement of the tridiagonal solve (optional, both
  // null disables it): the loaded, scaled G is saved to gsave (n rows, row
  // stride ldgsave, a multiple of 4) and the unscaled vectors u_0..u_ell to
  // uvec ((ell+1) x n; at least n x ((ell+1) rounded up to 4) floats, since
  // it then holds G U).
  float* gsave;
  int ldgsave;
  float* uvec;
  // Rows of the buffer that hold data; rows nvalid..n-1 of G are taken as
  // zero (a flush of a partial buffer solved at the full size n). 0: all n.
  int nvalid;
};

// t of Fast alpha-FD (Sec. 3.1): delta = sigma_t^2, t = ell - ell*alpha/2 with
// ell*alpha/2 rounded down and at least 1.
__host__ __device__ inline int fast_pfd_t(int ell, double alpha) {
  int half = (int)floor(alpha * ell / 2.0 + 1e-9);
  if (half < 1) half = 1;
  return ell - half;
}

// --- launchers (fd_simt.cu) -------------------------------------------------
cudaError_t launch_ingest(const void* src, int64_t n, int64_t ld, int dtype,
                          void* dst, int64_t ldd, int dst_is_f64, int64_t d,
                          double* rownorm_scratch, DevCounters* ctr,
                          __nv_bfloat16* rm_hi, __nv_bfloat16* rm_lo2, int64_t ld_rm,
                          __nv_bfloat16* cm_hi, __nv_bfloat16* cm_lo, int64_t ld_cm,
                          int row0, cudaStream_t st, double* slot_n2 = nullptr);

// Tile ingest (fd_ingest.cu): FP32 buffer rows (dst) and/or the tensor-core
// planes, squared norms summed per tile in FP64 and added in a fixed order.
// part: ingest_part_bytes(d, rows) bytes of scratch; ticket: a zeroed counter.
size_t ingest_part_bytes(int64_t d, int max_rows);
cudaError_t launch_ingest_tiles(const void* src, int64_t n, int64_t ld, int dtype, float* dst,
                                int64_t ldd, int64_t d, int row0, __nv_bfloat16* rm_hi,
                                __nv_bfloat16* rm_lo2, int64_t ld_rm, __nv_bfloat16* cm_hi,
                                __nv_bfloat16* cm_lo, int64_t ld_cm, double* part,
                                double* rownorm, double* slot_n2, DevCounters* ctr,
                                unsigned int* ticket, int* err, cudaStream_t st);

template <typename T>
cudaError_t launch_gram_simt(const T* B, int64_t ldb, int n, int64_t d, T* parts,
                             int ldp, int ksplit, cudaStream_t st);

template <typename T>
cudaError_t launch_gram_sum_parts(const T* parts, int nparts, int ldp, int n, T* out, int ldo,
                                  cudaStream_t st);

template <typename T>
cudaError_t launch_eig_shrink(const EigArgs& a, cudaStream_t st);

template <typename T>
cudaError_t launch_rotate_simt(const T* W, int ldw, int nout, int n, const T* Bin,
                               int64_t ldb, T* Bout, int64_t ldo, int64_t d,
                               cudaStream_t st);

cudaError_t launch_convert_out(const void* src, int src_f64, int64_t lds, int rows,
                               int64_t d, void* dst, int dst_f64, int64_t ldd,
                               int zero_from_row, cudaStream_t st);

cudaError_t launch_norm_b2(const void* src, int src_f64, int64_t lds, int rows,
                           int64_t d, DevCounters* ctr, cudaStream_t st);

cudaError_t launch_last_nonzero_row(const void* src, int src_f64, int64_t lds, int rows, int64_t d,
                                    int* out, cudaStream_t st);

cudaError_t launch_merge_counters(DevCounters* dst, const DevCounters* src, cudaStream_t st);

cudaError_t launch_merge_counters_values(DevCounters* dst, const double* norm_before,
                                         double norm_a2, double sum_delta, double removed,
                                         long long reductions, cudaStream_t st);

cudaError_t launch_compensate_rows(void* B, int b_f64, int64_t ld, int rows, int64_t d,
                                   const DevCounters* ctr, cudaStream_t st);

// --- tensor-core path (fd_tc.cu) ---------------------------------------------
struct TcPlanes;  // opaque, defined in fd_tc.cu
int tc_available();

// --- cov-err evaluator (fd_coverr.cu) ---------------------------------------
int cov_err_device(const void* A, int64_t n, int64_t d, int64_t lda, int a_f64,
                   const void* B, int64_t rows, int64_t ldb, int b_f64,
                   cudaStream_t st, double* cov, double* lmin, double* lmax);

// proj-err evaluator (fd_coverr.cu): R holds k rows sigma_j v_j (FP64, k x d,
// zero rows allowed) spanning B_k; num and den (optional) receive the two
// squared Frobenius norms.
int proj_err_device(const void* A, int64_t n, int64_t d, int64_t lda, int a_f64, const double* R,
                    int k, cudaStream_t st, double* pe, double* num, double* den);

// Records the text of the last failing CUDA call (for fd_strerror).
void set_cuda_error(cudaError_t e, const char* where);

}  // namespace fdk
