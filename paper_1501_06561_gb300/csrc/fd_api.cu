// C ABI of libfdsketch: handle management and the host side of the buffered
// FD stream (Algorithm 1, Sec. 2.3). The host only tracks how many rows the
// device buffer holds and launches kernels; every arithmetic step of a
// reduction runs on the GPU, ordered on the handle's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fd_internal.cuh"

namespace fdk {

static std::mutex g_err_mu;
static std::string g_err_text = "no CUDA error recorded";

void set_cuda_error(cudaError_t e, const char* where) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err_text = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

const char* cuda_error_text() {
  std::lock_guard<std::mutex> lk(g_err_mu);
  static thread_local std::string copy;
  copy = g_err_text;
  return copy.c_str();
}

int gram_simt_slices(int64_t d, int ksplit);
bool eig_fits_smem(int n, size_t elem);
int tri_config(int n, int ell);
size_t tri_global_workspace(int n);

// tensor-core path (fd_tc.cu)
struct TcCtx;
int tc_create(TcCtx** out, int64_t d, int ell, int L, int keep, cudaStream_t st);
void tc_destroy(TcCtx* t);
int tc_ingest(TcCtx* t, const void* src, int64_t n, int64_t ld, int dtype, int row0,
              double* rownorm, DevCounters* ctr, double* part);
int tc_gram(TcCtx* t, int nrows);
int tc_eig(TcCtx* t, const EigArgs& eig_template, int commit);
int tc_rotate(TcCtx* t, int nrows, int write_sketch, float* sketch_out, int64_t ldo);
int tc_export_rows(TcCtx* t, int rows, float* out, int64_t ldo);
int tc_error(TcCtx* t);
int tc_reset(TcCtx* t);

}  // namespace fdk

using namespace fdk;

#define FD_CK(call)                                     \
  do {                                                  \
    cudaError_t e__ = (call);                           \
    if (e__ != cudaSuccess) {                           \
      set_cuda_error(e__, #call);                       \
      return (e__ == cudaErrorMemoryAllocation) ? FD_ENOMEM : FD_ECUDA; \
    }                                                   \
  } while (0)

struct fd_state {
  int64_t d = 0;
  int64_t ldb = 0;        // buffer leading dimension (d rounded up to 64)
  int ell = 0, L = 0;     // L = 2*ell buffer rows
  int variant = 0, prec = 0;
  double alpha = 1.0;
  cudaStream_t st = nullptr;
  size_t es = 4;          // bytes per buffer element (FP32 / FP64)

  void* buf[2] = {nullptr, nullptr};  // ping-pong buffers, L x ldb
  int cur = 0;
  int m = 0;              // rows held in buf[cur]
  int64_t n_seen = 0;

  void* parts = nullptr;  // Gram partial slices
  void* gsum = nullptr;   // their sum, symmetrised (L x L)
  int ldp = 0;
  int ksplit = 1;
  int keep = 0;  // rows a reduction leaves in the buffer
  bool record_spectrum = false;  // fd_record_spectrum
  void* work = nullptr;   // eigensolve matrix in global memory when it does not fit smem
  size_t work_bytes = 0;
  void* wrot = nullptr;   // rotate matrix (ell-1) x ldr
  int ldr = 0;
  void* sk = nullptr;     // flush output, ell x ldb
  void* outdev = nullptr; // conversion scratch for host output, ell x d doubles

  float* gsave = nullptr;  // eigensolve refinement: the scaled Gram (L x ldg)
  int ldg = 0;
  float* uvec = nullptr;   // and the unscaled vectors ((ell+1) x L)

  DevCounters* ctr = nullptr;
  DevCounters* ctr_flush = nullptr;
  double* rownorm = nullptr;
  double* ing_part = nullptr;  // tile ingest: partial squared norms
  int* ing_err = nullptr;      // tile ingest: a bounded TMA wait gave up
  double* sig2 = nullptr;
  double* sigp2 = nullptr;
  bool flushed = false;

  // host-input staging (double buffered)
  void* pin[2] = {nullptr, nullptr};
  void* dstage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  int stage_next = 0;
  DevCounters* hctr = nullptr;  // pinned copy for fd_stats
  int* dint = nullptr;          // device int (merge: rows of the sketch)
  double* merge_tmp = nullptr;  // device double (fd_merge_sketch: ||A||_F^2 before the rows)
  int* hint = nullptr;          // pinned copy

  TcCtx* tc = nullptr;    // tensor-core planes (FD_PREC_BF16X3)
  int max_sweeps = 30;
  double tol = 0.0;

  // kernel timing (fd_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_marks;  // (class, index of start event)
  int64_t kcount[FD_KCLASSES] = {0, 0, 0, 0};
  double kms[FD_KCLASSES] = {0, 0, 0, 0};
};

// Bracket a launch of kernel class `cls` with events when profiling is on.
struct ProfScope {
  fd_state* h;
  int cls;
  int idx = -1;
  ProfScope(fd_state* hh, int c) : h(hh), cls(c) {
    if (!h->prof) return;
    const size_t need = h->ev_marks.size() * 2 + 2;
    while (h->ev_pool.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      h->ev_pool.push_back(e);
    }
    idx = (int)h->ev_marks.size() * 2;
    cudaEventRecord(h->ev_pool[idx], h->st);
  }
  ~ProfScope() {
    if (idx < 0) return;
    cudaEventRecord(h->ev_pool[idx + 1], h->st);
    h->ev_marks.emplace_back(cls, idx);
  }
};

static void prof_collect(fd_state* h) {
  if (h->ev_marks.empty()) return;
  cudaStreamSynchronize(h->st);
  for (auto& m : h->ev_marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[m.second], h->ev_pool[m.second + 1]) == cudaSuccess) {
      h->kcount[m.first] += 1;
      h->kms[m.first] += ms;
    }
  }
  h->ev_marks.clear();
}

static size_t dtype_size(int dt) {
  return dt == FD_F32 ? 4 : (dt == FD_BF16 ? 2 : (dt == FD_F64 ? 8 : 0));
}

static void free_state(fd_state* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->buf[i]);
    cudaFree(h->dstage[i]);
    if (h->pin[i]) cudaFreeHost(h->pin[i]);
    if (h->stage_ev[i]) cudaEventDestroy(h->stage_ev[i]);
  }
  cudaFree(h->parts);
  cudaFree(h->gsum);
  cudaFree(h->work);
  cudaFree(h->gsave);
  cudaFree(h->uvec);
  cudaFree(h->wrot);
  cudaFree(h->sk);
  cudaFree(h->outdev);
  cudaFree(h->ctr);
  cudaFree(h->ctr_flush);
  cudaFree(h->rownorm);
  cudaFree(h->ing_part);
  cudaFree(h->ing_err);
  cudaFree(h->sig2);
  cudaFree(h->sigp2);
  if (h->hctr) cudaFreeHost(h->hctr);
  cudaFree(h->dint);
  cudaFree(h->merge_tmp);
  if (h->hint) cudaFreeHost(h->hint);
  if (h->tc) tc_destroy(h->tc);
  delete h;
}

extern "C" int fd_create(int64_t d, int32_t ell, int32_t variant, double alpha, int32_t prec,
                         void* cuda_stream, fd_handle* out) {
  if (!out) return FD_EINVAL;
  *out = nullptr;
  if (ell < 2 || 2 * (int64_t)ell > FD_MAX_BUFFER_ROWS) return FD_EINVAL;
  return fd_create_buffered(d, ell, variant, alpha, prec,
                            variant == FD_VAR_FAST_PFD ? ell : 2 * ell, cuda_stream, out);
}

extern "C" int fd_create_buffered(int64_t d, int32_t ell, int32_t variant, double alpha,
                                  int32_t prec, int32_t buffer_rows, void* cuda_stream,
                                  fd_handle* out) {
  if (!out) return FD_EINVAL;
  *out = nullptr;
  if (d < 1 || ell < 2 || buffer_rows > FD_MAX_BUFFER_ROWS) return FD_EINVAL;
  if (variant < FD_VAR_FD || variant > FD_VAR_FAST_PFD) return FD_EINVAL;
  if (prec < FD_PREC_FP32 || prec > FD_PREC_FP64) return FD_EINVAL;
  if ((variant == FD_VAR_PFD || variant == FD_VAR_FAST_PFD) && !(alpha > 0.0 && alpha <= 1.0))
    return FD_EINVAL;
  if (variant == FD_VAR_FAST_PFD) {
    if (buffer_rows != ell || fast_pfd_t(ell, alpha) < 2) return FD_EINVAL;
  } else if (buffer_rows != ell && buffer_rows < 2 * ell) {
    // buffer_rows == ell: the literal Algorithms 1-3 (a reduction whenever the
    // ell-row sketch has no zero row left)
    return FD_EINVAL;
  }
  if (prec == FD_PREC_BF16X3 && !tc_available()) return FD_EINVAL;

  fd_state* h = new (std::nothrow) fd_state();
  if (!h) return FD_ENOMEM;
  h->d = d;
  h->ldb = (d + 63) / 64 * 64;
  h->ell = ell;
  h->L = buffer_rows;
  // rows a reduction leaves: ell-1, or t-1 for Fast alpha-FD (its values
  // t..ell are zeroed, so the next t-1.. slots are free)
  h->keep = (variant == FD_VAR_FAST_PFD) ? fast_pfd_t(ell, alpha) - 1 : ell - 1;
  h->variant = variant;
  h->alpha = (variant == FD_VAR_PFD || variant == FD_VAR_FAST_PFD) ? alpha : 1.0;
  h->prec = prec;
  h->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->es = (prec == FD_PREC_FP64) ? 8 : 4;
  const int np = h->L;
  h->max_sweeps = (prec == FD_PREC_FP64) ? 40 : 30;
  const double eps = (prec == FD_PREC_FP64) ? 2.220446049250313e-16 : 1.1920928955078125e-07;
  h->tol = 4.0 * eps * std::sqrt((double)np);

  auto fail = [&](cudaError_t e, const char* w) {
    set_cuda_error(e, w);
    free_state(h);
    return e == cudaErrorMemoryAllocation ? FD_ENOMEM : FD_ECUDA;
  };
  cudaError_t e;
#define FD_ALLOC(ptr, bytes)                                   \
  do {                                                         \
    e = cudaMalloc(reinterpret_cast<void**>(&(ptr)), (bytes)); \
    if (e != cudaSuccess) return fail(e, "cudaMalloc " #ptr);  \
    e = cudaMemsetAsync((ptr), 0, (bytes), h->st);             \
    if (e != cudaSuccess) return fail(e, "cudaMemset " #ptr);  \
  } while (0)

  const size_t bufbytes = (size_t)h->L * h->ldb * h->es;
  if (prec != FD_PREC_BF16X3) {
    FD_ALLOC(h->buf[0], bufbytes);
    FD_ALLOC(h->buf[1], bufbytes);
    h->ldp = h->L;
    const int tiles = (h->L + 63) / 64;
    const int64_t kt = (d + 63) / 64;
    h->ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(kt, 304 / (tiles * tiles)));
    const int slices = gram_simt_slices(d, h->ksplit);
    FD_ALLOC(h->parts, (size_t)slices * h->ldp * h->ldp * h->es);
    FD_ALLOC(h->gsum, (size_t)h->ldp * h->ldp * h->es);
    size_t wb = eig_fits_smem(h->L, h->es) ? 0 : (size_t)(np + 1) * (np + 1) * h->es;
    if (prec == FD_PREC_FP32 && tri_config(h->L, ell) == 4)
      wb = std::max(wb, tri_global_workspace(h->L));
    if (wb) { FD_ALLOC(h->work, wb); h->work_bytes = wb; }
  } else {
    int rc = tc_create(&h->tc, d, ell, h->L, h->keep, h->st);
    if (rc != FD_OK) { free_state(h); return rc; }
    size_t wb = eig_fits_smem(h->L, 4) ? 0 : (size_t)(np + 1) * (np + 1) * 4;
    if (tri_config(h->L, ell) == 4) wb = std::max(wb, tri_global_workspace(h->L));
    if (wb) { FD_ALLOC(h->work, wb); h->work_bytes = wb; }
  }
  if (prec != FD_PREC_FP64 && tri_config(h->L, ell) != 0) {
    h->ldg = (h->L + 3) & ~3;
    FD_ALLOC(h->gsave, (size_t)h->L * h->ldg * 4);
    FD_ALLOC(h->uvec, (size_t)(ell + 4) * h->L * 4);  // also G U, L x ((ell+1) rounded to 4)
  }
  h->ldr = (h->L + 63) / 64 * 64;
  FD_ALLOC(h->wrot, (size_t)ell * h->ldr * h->es);
  FD_ALLOC(h->sk, (size_t)ell * h->ldb * h->es);
  FD_ALLOC(h->outdev, (size_t)ell * d * 8);
  FD_ALLOC(h->ctr, sizeof(DevCounters));
  FD_ALLOC(h->ctr_flush, sizeof(DevCounters));
  FD_ALLOC(h->rownorm, (size_t)FD_MAX_BUFFER_ROWS * 8);
  FD_ALLOC(h->ing_part, ingest_part_bytes(d, h->L));
  FD_ALLOC(h->ing_err, sizeof(int));
  FD_ALLOC(h->dint, 16);
  FD_ALLOC(h->merge_tmp, 8);
  FD_ALLOC(h->sig2, (size_t)FD_MAX_BUFFER_ROWS * 8);
  FD_ALLOC(h->sigp2, (size_t)FD_MAX_BUFFER_ROWS * 8);
#undef FD_ALLOC
  h->stage_bytes = std::max<size_t>((size_t)16 << 20, (size_t)h->L * d * 8);
  for (int i = 0; i < 2; ++i) {
    e = cudaMallocHost(&h->pin[i], h->stage_bytes);
    if (e != cudaSuccess) return fail(e, "cudaMallocHost staging");
    e = cudaMalloc(&h->dstage[i], h->stage_bytes);
    if (e != cudaSuccess) return fail(e, "cudaMalloc staging");
    e = cudaEventCreateWithFlags(&h->stage_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(e, "cudaEventCreate");
  }
  e = cudaMallocHost(reinterpret_cast<void**>(&h->hctr), 2 * sizeof(DevCounters));
  if (e != cudaSuccess) return fail(e, "cudaMallocHost counters");
  e = cudaMallocHost(reinterpret_cast<void**>(&h->hint), 16);
  if (e != cudaSuccess) return fail(e, "cudaMallocHost hint");
  e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(e, "cudaStreamSynchronize");
  *out = h;
  return FD_OK;
}

// One reduction of the first `nrows` rows of buf[cur]. Writes the ell-1 new
// rows to `out` (leading dimension ldo) and the counters to ctr_out.
static int reduce_rows(fd_state* h, int nrows, void* out, int64_t ldo, DevCounters* ctr_out,
                       bool diag) {
  EigArgs a;
  std::memset(&a, 0, sizeof(a));
  // A flush of a partial buffer is solved at the full buffer size, its
  // missing rows taken as zero, so that it gets the same eigensolve (and
  // refinement) as a full reduction; FP64 and buffers the tridiagonal solve
  // does not take keep the one-sided Jacobi on the rows present.
  const bool tri = h->prec != FD_PREC_FP64 && tri_config(h->L, h->ell) != 0;
  a.n = tri ? h->L : nrows;
  a.nvalid = nrows;
  a.ell = h->ell;
  a.variant = h->variant;
  a.alpha = h->alpha;
  a.work = h->work;
  a.work_bytes = h->work_bytes;
  a.ldw_work = a.n + (a.n & 1);
  a.gsave = h->gsave;
  a.ldgsave = h->ldg;
  a.uvec = h->uvec;
  a.ctr_in = h->ctr;
  a.ctr_out = ctr_out;
  a.sig2_out = (diag && h->record_spectrum) ? h->sig2 : nullptr;
  a.sigp2_out = (diag && h->record_spectrum) ? h->sigp2 : nullptr;
  a.wrot = h->wrot;
  a.ldr = h->ldr;
  a.max_sweeps = h->max_sweeps;
  a.tol = h->tol;
  a.symmetrize = 1;
  a.use_tri = tri ? 1 : 0;
  if (h->prec == FD_PREC_BF16X3) {
    int rc;
    { ProfScope ps(h, FD_K_GRAM); rc = tc_gram(h->tc, nrows); }
    if (rc != FD_OK) return rc;
    { ProfScope ps(h, FD_K_EIG); rc = tc_eig(h->tc, a, out == nullptr ? 1 : 0); }
    if (rc != FD_OK) return rc;
    { ProfScope ps(h, FD_K_ROTATE);
      rc = tc_rotate(h->tc, nrows, out != nullptr ? 1 : 0, reinterpret_cast<float*>(out), ldo); }
    return rc;
  }
  const int slices = gram_simt_slices(h->d, h->ksplit);
  a.parts = h->gsum;
  a.nparts = 1;
  a.ldp = h->ldp;
  a.part_stride = (long long)h->ldp * h->ldp;
  if (h->prec == FD_PREC_FP64) {
    const double* B = reinterpret_cast<const double*>(h->buf[h->cur]);
    { ProfScope ps(h, FD_K_GRAM);
      FD_CK((launch_gram_simt<double>(B, h->ldb, nrows, h->d, reinterpret_cast<double*>(h->parts),
                                      h->ldp, h->ksplit, h->st)));
      FD_CK((launch_gram_sum_parts<double>(reinterpret_cast<const double*>(h->parts), slices,
                                           h->ldp, nrows, reinterpret_cast<double*>(h->gsum),
                                           h->ldp, h->st))); }
    { ProfScope ps(h, FD_K_EIG);
      FD_CK(launch_eig_shrink<double>(a, h->st)); }
    { ProfScope ps(h, FD_K_ROTATE);
      FD_CK((launch_rotate_simt<double>(reinterpret_cast<const double*>(h->wrot), h->ldr,
                                        h->ell - 1, nrows, B, h->ldb,
                                        reinterpret_cast<double*>(out), ldo, h->d, h->st))); }
  } else {
    const float* B = reinterpret_cast<const float*>(h->buf[h->cur]);
    { ProfScope ps(h, FD_K_GRAM);
      FD_CK((launch_gram_simt<float>(B, h->ldb, nrows, h->d, reinterpret_cast<float*>(h->parts),
                                     h->ldp, h->ksplit, h->st)));
      FD_CK((launch_gram_sum_parts<float>(reinterpret_cast<const float*>(h->parts), slices,
                                          h->ldp, nrows, reinterpret_cast<float*>(h->gsum),
                                          h->ldp, h->st))); }
    { ProfScope ps(h, FD_K_EIG);
      FD_CK(launch_eig_shrink<float>(a, h->st)); }
    { ProfScope ps(h, FD_K_ROTATE);
      FD_CK((launch_rotate_simt<float>(reinterpret_cast<const float*>(h->wrot), h->ldr,
                                       h->ell - 1, nrows, B, h->ldb,
                                       reinterpret_cast<float*>(out), ldo, h->d, h->st))); }
  }
  return FD_OK;
}

// Append n device rows (row-major, ld, dtype): ingest into the free rows and
// reduce whenever the 2*ell buffer is full.
static int append_device(fd_state* h, const char* src, int64_t n, int64_t ld, int dtype) {
  const size_t rb = (size_t)ld * dtype_size(dtype);
  int64_t i = 0;
  while (i < n) {
    const int c = (int)std::min<int64_t>(n - i, h->L - h->m);
    ProfScope* ps = new ProfScope(h, FD_K_INGEST);
    if (h->prec == FD_PREC_BF16X3) {
      int rc = tc_ingest(h->tc, src + i * rb, c, ld, dtype, h->m, h->rownorm, h->ctr,
                         h->ing_part);
      if (rc != FD_OK) return rc;
    } else if (h->prec == FD_PREC_FP32) {
      FD_CK(launch_ingest_tiles(src + i * rb, c, ld, dtype,
                                reinterpret_cast<float*>(h->buf[h->cur]), h->ldb, h->d, h->m,
                                nullptr, nullptr, 0, nullptr, nullptr, 0, h->ing_part,
                                h->rownorm, nullptr, h->ctr, &h->ctr->ingest_ticket, h->ing_err,
                                h->st));
    } else {
      char* dst = reinterpret_cast<char*>(h->buf[h->cur]) + (size_t)h->m * h->ldb * h->es;
      FD_CK(launch_ingest(src + i * rb, c, ld, dtype, dst, h->ldb, 1, h->d, h->rownorm, h->ctr,
                          nullptr, nullptr, 0, nullptr, nullptr, 0, h->m, h->st));
    }
    delete ps;
    h->m += c;
    h->n_seen += c;
    i += c;
    if (h->m == h->L) {
      int rc;
      if (h->prec == FD_PREC_BF16X3) {
        rc = reduce_rows(h, h->L, nullptr, 0, h->ctr, true);
      } else {
        const int nxt = h->cur ^ 1;
        rc = reduce_rows(h, h->L, h->buf[nxt], h->ldb, h->ctr, true);
        h->cur = nxt;
      }
      if (rc != FD_OK) return rc;
      h->m = h->keep;
    }
  }
  return FD_OK;
}

extern "C" int fd_append(fd_handle h, const void* rows, int64_t n, int64_t ld, int32_t dtype,
                         int32_t on_device) {
  if (!h) return FD_EINVAL;
  if (n < 0) return FD_EINVAL;
  if (n == 0) return FD_OK;
  if (!rows || ld < h->d || dtype_size(dtype) == 0) return FD_EINVAL;
  h->flushed = false;
  if (on_device) return append_device(h, reinterpret_cast<const char*>(rows), n, ld, dtype);
  // host rows: pack into pinned staging, copy, then run the device path
  const size_t es = dtype_size(dtype);
  const size_t row_bytes = (size_t)h->d * es;
  const int64_t per_slot = std::max<int64_t>(1, (int64_t)(h->stage_bytes / row_bytes));
  const char* src = reinterpret_cast<const char*>(rows);
  for (int64_t i = 0; i < n; i += per_slot) {
    const int64_t c = std::min<int64_t>(per_slot, n - i);
    const int slot = h->stage_next;
    h->stage_next ^= 1;
    FD_CK(cudaEventSynchronize(h->stage_ev[slot]));
    char* pin = reinterpret_cast<char*>(h->pin[slot]);
    if (ld == h->d) {
      std::memcpy(pin, src + (size_t)i * row_bytes, (size_t)c * row_bytes);
    } else {
      for (int64_t r = 0; r < c; ++r)
        std::memcpy(pin + (size_t)r * row_bytes, src + (size_t)(i + r) * ld * es, row_bytes);
    }
    FD_CK(cudaMemcpyAsync(h->dstage[slot], pin, (size_t)c * row_bytes, cudaMemcpyHostToDevice,
                          h->st));
    int rc = append_device(h, reinterpret_cast<const char*>(h->dstage[slot]), c, h->d, dtype);
    if (rc != FD_OK) return rc;
    FD_CK(cudaEventRecord(h->stage_ev[slot], h->st));
  }
  return FD_OK;
}

extern "C" int fd_sketch(fd_handle h, void* out, int32_t dtype, int32_t out_on_device) {
  if (!h || !out || (dtype != FD_F32 && dtype != FD_F64)) return FD_EINVAL;
  const int dst_f64 = (dtype == FD_F64);
  const void* src;
  int64_t lds;
  int valid;
  int src_f64 = (h->prec == FD_PREC_FP64);
  if (h->m > h->ell - 1) {
    int rc = reduce_rows(h, h->m, h->sk, h->ldb, h->ctr_flush, false);
    if (rc != FD_OK) return rc;
    src = h->sk;
    lds = h->ldb;
    valid = h->ell - 1;
    if (h->prec == FD_PREC_BF16X3) src_f64 = 0;
  } else {
    FD_CK(cudaMemcpyAsync(h->ctr_flush, h->ctr, sizeof(DevCounters), cudaMemcpyDeviceToDevice,
                          h->st));
    if (h->prec == FD_PREC_BF16X3) {
      int rc = tc_export_rows(h->tc, h->m, reinterpret_cast<float*>(h->sk), h->ldb);
      if (rc != FD_OK) return rc;
      src = h->sk;
      src_f64 = 0;
    } else {
      src = h->buf[h->cur];
    }
    lds = h->ldb;
    valid = h->m;
  }
  FD_CK(launch_norm_b2(src, src_f64, lds, valid, h->d, h->ctr_flush, h->st));
  h->flushed = true;
  if (out_on_device) {
    FD_CK(launch_convert_out(src, src_f64, lds, h->ell, h->d, out, dst_f64, h->d, valid, h->st));
    return FD_OK;
  }
  FD_CK(launch_convert_out(src, src_f64, lds, h->ell, h->d, h->outdev, dst_f64, h->d, valid,
                           h->st));
  FD_CK(cudaMemcpyAsync(out, h->outdev, (size_t)h->ell * h->d * (dst_f64 ? 8 : 4),
                        cudaMemcpyDeviceToHost, h->st));
  FD_CK(cudaStreamSynchronize(h->st));
  return FD_OK;
}

// Compensative FD: the sketch, then each nonzero row rescaled (see fdsketch.h).
extern "C" int fd_sketch_compensated(fd_handle h, void* out, int32_t dtype, int32_t out_on_device) {
  if (!h || !out || (dtype != FD_F32 && dtype != FD_F64)) return FD_EINVAL;
  if (h->variant != FD_VAR_FD && h->variant != FD_VAR_PFD) return FD_EINVAL;
  const int dst_f64 = (dtype == FD_F64);
  void* dev = out_on_device ? out : h->outdev;
  int rc = fd_sketch(h, dev, dtype, 1);
  if (rc != FD_OK) return rc;
  FD_CK(launch_compensate_rows(dev, dst_f64, h->d, h->ell, h->d, h->ctr_flush, h->st));
  if (out_on_device) return FD_OK;
  FD_CK(cudaMemcpyAsync(out, h->outdev, (size_t)h->ell * h->d * (dst_f64 ? 8 : 4),
                        cudaMemcpyDeviceToHost, h->st));
  FD_CK(cudaStreamSynchronize(h->st));
  return FD_OK;
}

// Merge: src's sketch rows become stream rows of dst (see fdsketch.h).
extern "C" int fd_merge(fd_handle dst, fd_handle src) {
  if (!dst || !src || dst == src || dst->d != src->d) return FD_EINVAL;
  const int32_t dt = (dst->prec == FD_PREC_FP64) ? FD_F64 : FD_F32;
  int rc = fd_sketch(src, src->outdev, dt, 1);  // on a copy: src is unchanged
  if (rc != FD_OK) return rc;
  FD_CK(launch_last_nonzero_row(src->outdev, dt == FD_F64, src->d, src->ell, src->d, src->dint,
                                src->st));
  FD_CK(cudaMemcpyAsync(src->hint, src->dint, sizeof(int), cudaMemcpyDeviceToHost, src->st));
  FD_CK(cudaStreamSynchronize(src->st));
  const int rows = *src->hint;
  dst->flushed = false;
  if (rows > 0) {
    rc = append_device(dst, reinterpret_cast<const char*>(src->outdev), rows, src->d, dt);
    if (rc != FD_OK) return rc;
  }
  FD_CK(launch_merge_counters(dst->ctr, src->ctr_flush, dst->st));
  dst->n_seen += src->n_seen - rows;
  // src's buffers feed dst's stream: finish before src can reuse them
  FD_CK(cudaStreamSynchronize(dst->st));
  return FD_OK;
}

extern "C" int fd_merge_sketch(fd_handle dst, const void* B, int64_t rows, int64_t ld,
                               int32_t dtype, int32_t on_device, const fd_stats_t* src) {
  if (!dst || !src || rows < 0 || (rows > 0 && (!B || ld < dst->d)) || dtype_size(dtype) == 0)
    return FD_EINVAL;
  if (rows > dst->ell) return FD_EINVAL;  // a sketch has at most ell rows
  if (src->n_seen < rows || src->d != dst->d) return FD_EINVAL;
  FD_CK(cudaMemcpyAsync(dst->merge_tmp, &dst->ctr->norm_a2, sizeof(double),
                        cudaMemcpyDeviceToDevice, dst->st));
  dst->flushed = false;
  if (rows > 0) {
    // the sketch rows enter dst's stream as ordinary rows (as in fd_merge)
    int rc = fd_append(dst, B, rows, ld, dtype, on_device);
    if (rc != FD_OK) return rc;
  }
  FD_CK(launch_merge_counters_values(dst->ctr, dst->merge_tmp, src->norm_a2,
                                     src->sketch_sum_delta, src->sketch_removed,
                                     src->reductions, dst->st));
  dst->n_seen += src->n_seen - rows;
  FD_CK(cudaStreamSynchronize(dst->st));
  return FD_OK;
}

extern "C" int fd_stats(fd_handle h, fd_stats_t* s) {
  if (!h || !s) return FD_EINVAL;
  FD_CK(cudaMemcpyAsync(h->hctr, h->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, h->st));
  FD_CK(cudaMemcpyAsync(h->hctr + 1, h->ctr_flush, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                        h->st));
  FD_CK(cudaStreamSynchronize(h->st));
  if (h->tc && tc_error(h->tc)) {
    set_cuda_error(cudaErrorLaunchTimeout, "tensor-core pipeline wait gave up");
    return FD_ECUDA;
  }
  {
    int ie = 0;
    FD_CK(cudaMemcpy(&ie, h->ing_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (ie) {
      set_cuda_error(cudaErrorLaunchTimeout, "ingest TMA wait gave up");
      return FD_ECUDA;
    }
  }
  const DevCounters& c = h->hctr[0];
  const DevCounters& f = h->hctr[1];
  std::memset(s, 0, sizeof(*s));
  s->d = h->d;
  s->ell = h->ell;
  s->variant = h->variant;
  s->alpha = h->alpha;
  s->prec = h->prec;
  s->pending = h->m;
  s->n_seen = h->n_seen;
  s->reductions = c.reductions;
  s->noconv = c.noconv;
  s->eig_fallbacks = c.fallbacks;
  s->norm_a2 = c.norm_a2;
  s->sum_delta = c.sum_delta;
  s->last_delta = c.last_delta;
  s->removed = c.removed;
  s->max_sweeps = std::max(c.max_sweeps, h->flushed ? f.max_sweeps : 0.0);
  if (h->flushed) {
    s->sketch_sum_delta = f.sum_delta;
    s->sketch_removed = f.removed;
    s->sketch_norm_b2 = f.norm_b2;
  } else {
    s->sketch_sum_delta = c.sum_delta;
    s->sketch_removed = c.removed;
    s->sketch_norm_b2 = c.norm_b2;
  }
  return FD_OK;
}

extern "C" int fd_record_spectrum(fd_handle h, int32_t on) {
  if (!h) return FD_EINVAL;
  h->record_spectrum = (on != 0);
  return FD_OK;
}

extern "C" int fd_last_spectrum(fd_handle h, double* sigma2, double* sigma_prime2) {
  if (!h || !sigma2 || !sigma_prime2 || !h->record_spectrum) return FD_EINVAL;
  FD_CK(cudaMemcpyAsync(sigma2, h->sig2, (size_t)h->L * 8, cudaMemcpyDeviceToHost, h->st));
  FD_CK(cudaMemcpyAsync(sigma_prime2, h->sigp2, (size_t)h->L * 8, cudaMemcpyDeviceToHost, h->st));
  FD_CK(cudaStreamSynchronize(h->st));
  return FD_OK;
}

extern "C" int fd_reset(fd_handle h) {
  if (!h) return FD_EINVAL;
  const size_t bufbytes = (size_t)h->L * h->ldb * h->es;
  for (int i = 0; i < 2; ++i)
    if (h->buf[i]) FD_CK(cudaMemsetAsync(h->buf[i], 0, bufbytes, h->st));
  if (h->tc) {
    int rc = tc_reset(h->tc);
    if (rc != FD_OK) return rc;
  }
  FD_CK(cudaMemsetAsync(h->ctr, 0, sizeof(DevCounters), h->st));
  FD_CK(cudaMemsetAsync(h->ctr_flush, 0, sizeof(DevCounters), h->st));
  FD_CK(cudaMemsetAsync(h->sig2, 0, (size_t)FD_MAX_BUFFER_ROWS * 8, h->st));
  FD_CK(cudaMemsetAsync(h->sigp2, 0, (size_t)FD_MAX_BUFFER_ROWS * 8, h->st));
  h->cur = 0;
  h->m = 0;
  h->n_seen = 0;
  h->flushed = false;
  return FD_OK;
}

extern "C" int fd_profile(fd_handle h, int32_t enable) {
  if (!h) return FD_EINVAL;
  prof_collect(h);
  h->prof = enable != 0;
  if (h->prof)
    for (int c = 0; c < FD_KCLASSES; ++c) { h->kcount[c] = 0; h->kms[c] = 0.0; }
  return FD_OK;
}

extern "C" int fd_kernel_times(fd_handle h, int64_t* counts, double* ms) {
  if (!h || !counts || !ms) return FD_EINVAL;
  prof_collect(h);
  for (int c = 0; c < FD_KCLASSES; ++c) { counts[c] = h->kcount[c]; ms[c] = h->kms[c]; }
  return FD_OK;
}

extern "C" int fd_destroy(fd_handle h) {
  if (!h) return FD_EINVAL;
  free_state(h);
  return FD_OK;
}

extern "C" int fd_cov_err(fd_handle h, const void* A, int64_t n, int64_t ld, int32_t dtype,
                          int32_t on_device, double* cov_err) {
  if (!h || !A || !cov_err || ld < h->d || n < 1) return FD_EINVAL;
  if (dtype != FD_F32 && dtype != FD_F64) return FD_EINVAL;
  // the sketch as fd_sketch returns it, kept on the device in FP64
  double* B = nullptr;
  FD_CK(cudaMalloc(&B, (size_t)h->ell * h->d * 8));
  int rc = fd_sketch(h, B, FD_F64, 1);
  if (rc != FD_OK) { cudaFree(B); return rc; }
  const void* Ad = A;
  void* tmp = nullptr;
  if (!on_device) {
    const size_t bytes = (size_t)n * ld * dtype_size(dtype);
    cudaError_t e = cudaMalloc(&tmp, bytes);
    if (e != cudaSuccess) { cudaFree(B); set_cuda_error(e, "cudaMalloc A"); return FD_ENOMEM; }
    e = cudaMemcpyAsync(tmp, A, bytes, cudaMemcpyHostToDevice, h->st);
    if (e != cudaSuccess) { cudaFree(B); cudaFree(tmp); set_cuda_error(e, "copy A"); return FD_ECUDA; }
    Ad = tmp;
  }
  double lmin, lmax;
  rc = cov_err_device(Ad, n, h->d, ld, dtype == FD_F64, B, h->ell, h->d, 1, h->st, cov_err,
                      &lmin, &lmax);
  cudaStreamSynchronize(h->st);
  cudaFree(B);
  if (tmp) cudaFree(tmp);
  return rc;
}

// proj-err of the current sketch against the rows A (see fdsketch.h).
extern "C" int fd_proj_err(fd_handle h, const void* A, int64_t n, int64_t ld, int32_t dtype,
                           int32_t on_device, int32_t k, double* proj_err) {
  if (!h || !A || !proj_err || ld < h->d || n < 1 || k < 1 || k >= h->ell) return FD_EINVAL;
  if (dtype != FD_F32 && dtype != FD_F64) return FD_EINVAL;
  const int ell = h->ell;
  const int64_t d = h->d;
  const int np = ell + (ell & 1);
  const int slices = gram_simt_slices(d, 1);
  double *B = nullptr, *parts = nullptr, *work = nullptr, *wrot = nullptr, *R = nullptr;
  DevCounters* ctr = nullptr;
  void* tmp = nullptr;
  auto cleanup = [&]() {
    cudaFree(B); cudaFree(parts); cudaFree(work); cudaFree(wrot); cudaFree(R); cudaFree(ctr);
    cudaFree(tmp);
  };
  const bool big = !eig_fits_smem(ell, 8);
  if (cudaMalloc(&B, sizeof(double) * (size_t)ell * d) != cudaSuccess ||
      cudaMalloc(&parts, sizeof(double) * (size_t)slices * np * np) != cudaSuccess ||
      (big && cudaMalloc(&work, sizeof(double) * (size_t)np * np) != cudaSuccess) ||
      cudaMalloc(&wrot, sizeof(double) * (size_t)k * ell) != cudaSuccess ||
      cudaMalloc(&R, sizeof(double) * (size_t)k * d) != cudaSuccess ||
      cudaMalloc(&ctr, 2 * sizeof(DevCounters)) != cudaSuccess) {
    cleanup();
    set_cuda_error(cudaErrorMemoryAllocation, "proj-err workspace");
    return FD_ENOMEM;
  }
  // the sketch as fd_sketch returns it, in FP64 on the device
  int rc = fd_sketch(h, B, FD_F64, 1);
  if (rc != FD_OK) { cleanup(); return rc; }
  // top k right singular vectors of B: an eigensolve of B B^T whose
  // ReduceRank is the iSVD rule with ell' = k + 1 (the k largest values kept,
  // the rest zeroed), then the rotate gives the rows sigma_j v_j
  EigArgs a;
  std::memset(&a, 0, sizeof(a));
  a.parts = parts;
  a.nparts = slices;
  a.ldp = np;
  a.part_stride = (long long)np * np;
  a.symmetrize = 1;
  a.n = ell;
  a.ell = k + 1;
  a.variant = FD_VAR_ISVD;
  a.alpha = 1.0;
  a.work = work;
  a.ldw_work = np;
  a.work_bytes = big ? sizeof(double) * (size_t)np * np : 0;
  a.ctr_in = ctr;
  a.ctr_out = ctr + 1;
  a.wrot = wrot;
  a.ldr = ell;
  a.max_sweeps = 40;
  a.tol = 4.0 * 1.1102230246251565e-16 * std::sqrt((double)np);
  a.use_tri = 0;
  FD_CK(cudaMemsetAsync(ctr, 0, 2 * sizeof(DevCounters), h->st));
  FD_CK((launch_gram_simt<double>(B, d, ell, d, parts, np, 1, h->st)));
  FD_CK(launch_eig_shrink<double>(a, h->st));
  FD_CK((launch_rotate_simt<double>(wrot, ell, k, ell, B, d, R, d, d, h->st)));
  const void* Ad = A;
  if (!on_device) {
    const size_t bytes = (size_t)n * ld * dtype_size(dtype);
    cudaError_t e = cudaMalloc(&tmp, bytes);
    if (e != cudaSuccess) { cleanup(); set_cuda_error(e, "cudaMalloc A"); return FD_ENOMEM; }
    e = cudaMemcpyAsync(tmp, A, bytes, cudaMemcpyHostToDevice, h->st);
    if (e != cudaSuccess) { cleanup(); set_cuda_error(e, "copy A"); return FD_ECUDA; }
    Ad = tmp;
  }
  rc = proj_err_device(Ad, n, d, ld, dtype == FD_F64, R, k, h->st, proj_err, nullptr, nullptr);
  cudaStreamSynchronize(h->st);
  cleanup();
  return rc;
}

extern "C" int fd_cov_err_pair(const void* A, int64_t n, int64_t d, int64_t lda, int32_t a_dtype,
                               const void* B, int64_t rows, int32_t b_dtype, int32_t on_device,
                               void* cuda_stream, double* cov_err, double* lambda_min,
                               double* lambda_max) {
  if (!A || !B || !cov_err || n < 1 || d < 1 || rows < 0 || lda < d) return FD_EINVAL;
  if ((a_dtype != FD_F32 && a_dtype != FD_F64) || (b_dtype != FD_F32 && b_dtype != FD_F64))
    return FD_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const void* Ad = A;
  const void* Bd = B;
  void* ta = nullptr;
  void* tb = nullptr;
  if (!on_device) {
    const size_t ab = (size_t)n * lda * dtype_size(a_dtype);
    const size_t bb = (size_t)std::max<int64_t>(rows, 1) * d * dtype_size(b_dtype);
    FD_CK(cudaMalloc(&ta, ab));
    cudaError_t e = cudaMalloc(&tb, bb);
    if (e != cudaSuccess) { cudaFree(ta); set_cuda_error(e, "cudaMalloc B"); return FD_ENOMEM; }
    cudaMemcpyAsync(ta, A, ab, cudaMemcpyHostToDevice, st);
    if (rows > 0) cudaMemcpyAsync(tb, B, (size_t)rows * d * dtype_size(b_dtype), cudaMemcpyHostToDevice, st);
    Ad = ta;
    Bd = tb;
  }
  double lmin = 0, lmax = 0;
  int rc = cov_err_device(Ad, n, d, lda, a_dtype == FD_F64, Bd, rows, d, b_dtype == FD_F64, st,
                          cov_err, &lmin, &lmax);
  cudaStreamSynchronize(st);
  if (ta) cudaFree(ta);
  if (tb) cudaFree(tb);
  if (lambda_min) *lambda_min = lmin;
  if (lambda_max) *lambda_max = lmax;
  return rc;
}

extern "C" const char* fd_strerror(int32_t code) {
  switch (code) {
    case FD_OK: return "ok";
    case FD_EINVAL: return "invalid argument";
    case FD_ENOMEM: return "out of memory";
    case FD_ECUDA: return cuda_error_text();
    case FD_ENOCONV: return "eigensolve reached its sweep cap";
    case FD_EBUSY: return "no room to admit the request";
    case FD_ETOOBIG: return "size exceeds the fixed workspace of the no-allocation evaluator";
    default: return "unknown error code";
  }
}

extern "C" const char* fd_version(void) { return "fdsketch 0.1 (sm_103a)"; }
