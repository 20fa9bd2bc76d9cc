// C ABI of libensemble_solve.so: matrix lifetime, GSpMV entry points and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ens_internal.cuh"
#include "rowprod.cuh"

namespace ens {

static thread_local std::string g_last_error;
static thread_local uint64_t g_last_ws_bytes = 0;
static thread_local bool g_last_ws_overflow = false;

void record_workspace(size_t bytes, bool overflow) {
  g_last_ws_bytes = bytes;
  g_last_ws_overflow = overflow;
}
bool last_workspace_overflow() { return g_last_ws_overflow; }

ens_status fail(ens_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

ens_status cuda_fail(cudaError_t e, const char *what) {
  const ens_status st = (e == cudaErrorMemoryAllocation) ? ENS_ERR_OOM : ENS_ERR_CUDA;
  return fail(st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void clear_error() { g_last_error.clear(); }

namespace {

// Per-row set-up: inverse diagonal (Jacobi scaling) and the float32 / split copies of val.
// flags[0] |= 1 if some nonzero value lies outside the split product range,
// flags[0] |= 2 if some row has no nonzero diagonal entry.
__global__ void k_matrix_aux(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ va, float *__restrict__ v32, float2 *__restrict__ vs,
                             double *__restrict__ dinv, float *__restrict__ dinv32, unsigned *flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned local = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d = 0.0;
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j) {
      const double v = va[j];
      if (ci[j] == i) d = v;
      v32[j] = (float)v;
      const float hi = (float)v;
      const float lo = (float)(v - (double)hi);
      vs[j] = make_float2(hi, lo);
      const double a = fabs(v);
      // split range of the product path: 2^-40 <= |v| < 2^60, or v == 0
      if (v != 0.0 && !(a >= 0x1p-40 && a < 0x1p60)) local |= 1u;
    }
    if (d == 0.0) local |= 2u;
    dinv[i] = d != 0.0 ? 1.0 / d : 0.0;
    dinv32[i] = d != 0.0 ? (float)(1.0 / d) : 0.f;
  }
  if (local) atomicOr(flags, local);
}

template <typename T>
cudaError_t dmalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void **)p, count * sizeof(T));
}

void free_matrix(ens_matrix *A) {
  free_amg(A->amg);
  cudaFree(A->row);
  cudaFree(A->col);
  cudaFree(A->val);
  cudaFree(A->val32);
  cudaFree(A->valsplit);
  cudaFree(A->dinv);
  cudaFree(A->dinv32);
  cudaFree(A->stage_x);
  cudaFree(A->stage_y);
  for (cudaEvent_t ev : A->pipe_ev)
    if (ev) cudaEventDestroy(ev);
  if (A->pipe_h2d) cudaStreamDestroy(A->pipe_h2d);
  if (A->pipe_d2h) cudaStreamDestroy(A->pipe_d2h);
  delete A;
}

ens_status check_gspmv_args(const ens_matrix *A, int32_t m, int32_t dtype, const void *X, const void *Y) {
  if (!A) return fail(ENS_ERR_INVALID, "gspmv: matrix is NULL");
  if (m < 1) return fail(ENS_ERR_INVALID, "gspmv: m must be >= 1 (got %d)", m);
  if (dtype != ENS_F64 && dtype != ENS_F32) return fail(ENS_ERR_INVALID, "gspmv: unknown dtype %d", dtype);
  if ((int64_t)m * A->n > ((int64_t)1 << 62) / 8) return fail(ENS_ERR_INVALID, "gspmv: n*m too large");
  if (A->n > 0 && (!X || !Y)) return fail(ENS_ERR_INVALID, "gspmv: X or Y is NULL");
  const size_t es = dtype == ENS_F64 ? 8 : 4;
  if ((uintptr_t)X % es || (uintptr_t)Y % es) return fail(ENS_ERR_INVALID, "gspmv: X/Y not aligned to the element size");
  const size_t xbytes = (size_t)A->ncols * m * es, ybytes = (size_t)A->n * m * es;
  const char *x = (const char *)X, *y = (const char *)Y;
  if (A->n > 0 && x < y + ybytes && y < x + xbytes) return fail(ENS_ERR_INVALID, "gspmv: X and Y overlap");
  return ENS_OK;
}

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" {

const char *ens_last_error(void) { return g_last_error.c_str(); }

uint64_t ens_last_workspace_bytes(void) { return g_last_ws_bytes; }

const char *ens_version(void) { return "ensemble_solve 0.1 (sm_103a)"; }

ens_status ens_create_matrix(int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                             const double *val, uint32_t flags, void *stream, ens_matrix **out) {
  clear_error();
  return create_matrix(n, n, nnz, row_ptr, col_idx, val, flags, stream, out);
}

}  // extern "C"

ens_status ens::create_matrix(int64_t n, int64_t ncols, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                              const double *val, uint32_t flags, void *stream, ens_matrix **out) {
  if (!out) return fail(ENS_ERR_INVALID, "create_matrix: out is NULL");
  *out = nullptr;
  if (n < 1 || n > INT32_MAX) return fail(ENS_ERR_INVALID, "create_matrix: n = %lld outside [1, 2^31-1]", (long long)n);
  if (ncols < 1 || ncols > INT32_MAX)
    return fail(ENS_ERR_INVALID, "create_matrix: ncols = %lld outside [1, 2^31-1]", (long long)ncols);
  if (ncols != n && (flags & ENS_MATRIX_SINGULAR))
    return fail(ENS_ERR_INVALID, "create_matrix: ENS_MATRIX_SINGULAR needs a square matrix");
  if (nnz < 0 || nnz > INT32_MAX) return fail(ENS_ERR_INVALID, "create_matrix: nnz = %lld outside [0, 2^31-1]", (long long)nnz);
  if (!row_ptr || (nnz > 0 && (!col_idx || !val))) return fail(ENS_ERR_INVALID, "create_matrix: NULL array");
  if (flags & ~ENS_MATRIX_SINGULAR) return fail(ENS_ERR_INVALID, "create_matrix: unknown flags 0x%x", flags);
  // Host-side validation of the CSR structure.
  if (row_ptr[0] != 0) return fail(ENS_ERR_INVALID, "create_matrix: row_ptr[0] = %d, expected 0", row_ptr[0]);
  int32_t max_len = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t len = row_ptr[i + 1] - row_ptr[i];
    if (row_ptr[i + 1] < row_ptr[i]) return fail(ENS_ERR_INVALID, "create_matrix: row_ptr decreases at row %lld", (long long)i);
    if (len > max_len) max_len = len;
  }
  if (row_ptr[n] != nnz) return fail(ENS_ERR_INVALID, "create_matrix: row_ptr[n] = %d != nnz = %lld", row_ptr[n], (long long)nnz);
  for (int64_t j = 0; j < nnz; ++j)
    if (col_idx[j] < 0 || col_idx[j] >= ncols)
      return fail(ENS_ERR_INVALID, "create_matrix: col_idx[%lld] = %d outside [0, %lld)", (long long)j, col_idx[j],
                  (long long)ncols);

  cudaStream_t s = (cudaStream_t)stream;
  ens_matrix *A = new ens_matrix();
  A->n = n;
  A->ncols = ncols;
  A->nnz = nnz;
  A->max_row_len = max_len;
  A->flags = flags;
  cudaError_t e = cudaGetDevice(&A->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&A->num_sms, cudaDevAttrMultiProcessorCount, A->device);
  unsigned *dflags = nullptr;
  // CSR arrays carry kCsrPad zeroed elements at the end: tiles stage 16-byte rounded segments.
  if (e == cudaSuccess) e = dmalloc(&A->row, n + 1 + kCsrPad);
  if (e == cudaSuccess) e = dmalloc(&A->col, nnz + kCsrPad);
  if (e == cudaSuccess) e = dmalloc(&A->val, nnz + kCsrPad);
  if (e == cudaSuccess) e = dmalloc(&A->val32, nnz + kCsrPad);
  if (e == cudaSuccess) e = dmalloc(&A->valsplit, nnz + kCsrPad);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->row + n + 1, 0, kCsrPad * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->col + nnz, 0, kCsrPad * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->val + nnz, 0, kCsrPad * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->val32 + nnz, 0, kCsrPad * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->valsplit + nnz, 0, kCsrPad * sizeof(float2), s);
  if (e == cudaSuccess) e = dmalloc(&A->dinv, n);
  if (e == cudaSuccess) e = dmalloc(&A->dinv32, n);
  if (e == cudaSuccess) e = dmalloc(&dflags, 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A->row, row_ptr, (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(A->col, col_idx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(A->val, val, nnz * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dflags, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)A->num_sms * 8);
    k_matrix_aux<<<grid, 256, 0, s>>>((int32_t)n, A->row, A->col, A->val, A->val32, A->valsplit, A->dinv, A->dinv32, dflags);
    e = cudaGetLastError();
  }
  unsigned hflags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, dflags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dflags);
  if (e != cudaSuccess) {
    free_matrix(A);
    return cuda_fail(e, "create_matrix");
  }
  A->split_ok = (hflags & 1u) == 0;
  A->full_diag = (hflags & 2u) == 0;
  // Row chunks of the pipelined host-buffer product: up to kPipeChunks chunks of whole tiles, each
  // with the set of X row blocks its column indices reach.
  {
    const int64_t tiles = (n + kPipeAlignRows - 1) / kPipeAlignRows;
    const int64_t chunks = std::min<int64_t>(kPipeChunks, tiles);
    const int64_t per = (tiles + chunks - 1) / chunks * kPipeAlignRows;
    A->pipe_block_rows = std::max<int64_t>(1, (ncols + kPipeBlocks - 1) / kPipeBlocks);
    for (int64_t r0 = 0; r0 < n; r0 += per) {
      const int64_t r1 = std::min<int64_t>(n, r0 + per);
      uint64_t mask[kPipeMaskWords] = {};
      for (int64_t j = row_ptr[r0]; j < row_ptr[r1]; ++j) {
        const int64_t b = (int64_t)col_idx[j] / A->pipe_block_rows;
        mask[b / 64] |= 1ull << (b % 64);
      }
      A->pipe_row.push_back(r0);
      A->pipe_mask.insert(A->pipe_mask.end(), mask, mask + kPipeMaskWords);
    }
    A->pipe_row.push_back(n);
  }
  *out = A;
  return ENS_OK;
}

extern "C" {

ens_status ens_destroy_matrix(ens_matrix *A) {
  clear_error();
  if (!A) return ENS_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_matrix(A);
  if (e != cudaSuccess) return cuda_fail(e, "destroy_matrix");
  return ENS_OK;
}

ens_status ens_matrix_info(const ens_matrix *A, int64_t *n, int64_t *nnz, int32_t *max_row_len) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "matrix_info: matrix is NULL");
  if (n) *n = A->n;
  if (nnz) *nnz = A->nnz;
  if (max_row_len) *max_row_len = A->max_row_len;
  return ENS_OK;
}

ens_status ens_set_f64_mode(ens_matrix *A, int32_t mode) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "set_f64_mode: matrix is NULL");
  if (mode < ENS_F64_AUTO || mode > ENS_F64_HYBRID) return fail(ENS_ERR_INVALID, "set_f64_mode: unknown mode %d", mode);
  A->f64_mode = mode;
  return ENS_OK;
}

ens_status ens_set_native_share(ens_matrix *A, int32_t share) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "set_native_share: matrix is NULL");
  if (share < -1 || share > 32) return fail(ENS_ERR_INVALID, "set_native_share: share %d outside [-1, 32]", share);
  A->native_share = share;
  return ENS_OK;
}

ens_status ens_autotune(ens_matrix *A, int32_t m, int32_t dtype, void *stream, int32_t *lanes, int32_t *share,
                        double *best_us) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "autotune: matrix is NULL");
  if (m < 1 || m > kTuneMaxM) return fail(ENS_ERR_INVALID, "autotune: m = %d outside [1, %d]", m, kTuneMaxM);
  if (dtype != ENS_F64 && dtype != ENS_F32) return fail(ENS_ERR_INVALID, "autotune: unknown dtype %d", dtype);
  return autotune(A, m, dtype, (cudaStream_t)stream, lanes, share, best_us);
}

ens_status ens_set_untiled(ens_matrix *A, int32_t mode) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "set_untiled: matrix is NULL");
  if (mode < -1 || mode > 1) return fail(ENS_ERR_INVALID, "set_untiled: mode %d outside [-1, 1]", mode);
  A->untiled = mode;
  return ENS_OK;
}

ens_status ens_tuned_variant(const ens_matrix *A, int32_t m, int32_t dtype, int32_t *lanes, int32_t *share,
                             int32_t *untiled) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "tuned_variant: matrix is NULL");
  if (m < 1 || m > kTuneMaxM) return fail(ENS_ERR_INVALID, "tuned_variant: m = %d outside [1, %d]", m, kTuneMaxM);
  if (dtype != ENS_F64 && dtype != ENS_F32) return fail(ENS_ERR_INVALID, "tuned_variant: unknown dtype %d", dtype);
  const int di = dtype == ENS_F32 ? 1 : 0;
  if (lanes) *lanes = A->tuned_lanes[di][m];
  if (share) *share = dtype == ENS_F32 ? 0 : A->tuned_share[m];
  if (untiled) *untiled = A->tuned_direct[di][m];
  return ENS_OK;
}

ens_status ens_gspmv(const ens_matrix *A, int32_t m, int32_t dtype, const void *X, void *Y, void *stream) {
  clear_error();
  ens_status st = check_gspmv_args(A, m, dtype, X, Y);
  if (st != ENS_OK) return st;
  return launch_gspmv(A, m, dtype, X, Y, (cudaStream_t)stream);
}

ens_status ens_gspmv_host(ens_matrix *A, int32_t m, int32_t dtype, const void *X, void *Y, void *stream) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "gspmv_host: matrix is NULL");
  if (A->ncols != A->n) return fail(ENS_ERR_INVALID, "gspmv_host: needs a square matrix");
  if (m < 1) return fail(ENS_ERR_INVALID, "gspmv_host: m must be >= 1 (got %d)", m);
  if (dtype != ENS_F64 && dtype != ENS_F32) return fail(ENS_ERR_INVALID, "gspmv_host: unknown dtype %d", dtype);
  if (!X || !Y) return fail(ENS_ERR_INVALID, "gspmv_host: X or Y is NULL");
  const size_t bytes = (size_t)A->n * m * (dtype == ENS_F64 ? 8 : 4);
  cudaStream_t s = (cudaStream_t)stream;
  if (bytes > A->stage_bytes) {
    ENS_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(A->stage_x);
    cudaFree(A->stage_y);
    A->stage_x = A->stage_y = nullptr;
    A->stage_bytes = 0;
    ENS_CUDA_TRY(cudaMalloc(&A->stage_x, bytes));
    cudaError_t e = cudaMalloc(&A->stage_y, bytes);
    if (e != cudaSuccess) {
      cudaFree(A->stage_x);
      A->stage_x = nullptr;
      return cuda_fail(e, "gspmv_host staging");
    }
    A->stage_bytes = bytes;
  }
  const int64_t chunks = (int64_t)A->pipe_row.size() - 1;
  // X and Y may be the same host array (an in-place product): then all of X is copied in before
  // any row of Y is copied out
  const char *xb = (const char *)X, *yb = (const char *)Y;
  const bool overlap = xb < yb + bytes && yb < xb + bytes;
  if (chunks < 2 || overlap) {
    ENS_CUDA_TRY(cudaMemcpyAsync(A->stage_x, X, bytes, cudaMemcpyHostToDevice, s));
    // every exit after the first copy waits for the stream: a later call may free and regrow
    // the staging buffers, which must not happen under a copy or kernel still in flight
    ens_status st = launch_gspmv(A, m, dtype, A->stage_x, A->stage_y, s);
    cudaError_t e = cudaSuccess;
    if (st == ENS_OK) e = cudaMemcpyAsync(Y, A->stage_y, bytes, cudaMemcpyDeviceToHost, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (st != ENS_OK) return st;
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) return cuda_fail(e, "gspmv_host");
    return ENS_OK;
  }
  // Pipelined: X arrives in row blocks on one copy stream, each row chunk runs on `s` once the
  // blocks it reads are in, and its Y rows leave on a second copy stream (both copy directions and
  // the kernels overlap).
  cudaError_t e = cudaSuccess;
  if (!A->pipe_h2d) {
    e = cudaStreamCreateWithFlags(&A->pipe_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&A->pipe_d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) A->pipe_ev.assign(2 * chunks + 1, nullptr);
    for (cudaEvent_t &ev : A->pipe_ev)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {  // leave no half-made pipeline behind: the next call starts over
      for (cudaEvent_t ev : A->pipe_ev)
        if (ev) cudaEventDestroy(ev);
      A->pipe_ev.clear();
      if (A->pipe_h2d) cudaStreamDestroy(A->pipe_h2d);
      if (A->pipe_d2h) cudaStreamDestroy(A->pipe_d2h);
      A->pipe_h2d = A->pipe_d2h = nullptr;
      return cuda_fail(e, "gspmv_host pipeline set-up");
    }
  }
  const size_t row_bytes = (size_t)m * (dtype == ENS_F64 ? 8 : 4);
  const char *hx = (const char *)X;
  char *hy = (char *)Y, *dx = (char *)A->stage_x, *dy = (char *)A->stage_y;
  cudaEvent_t *ev_x = A->pipe_ev.data(), *ev_y = ev_x + chunks, ev_start = ev_x[2 * chunks];
  e = cudaEventRecord(ev_start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(A->pipe_h2d, ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(A->pipe_d2h, ev_start, 0);
  // X blocks in the order the chunks first need them, each maximal run of new blocks as one copy
  uint64_t have[kPipeMaskWords] = {};
  const int64_t brows = A->pipe_block_rows, nblocks = (A->n + brows - 1) / brows;
  for (int64_t k = 0; k < chunks && e == cudaSuccess; ++k) {
    const uint64_t *need = A->pipe_mask.data() + k * kPipeMaskWords;
    int64_t b = 0;
    while (b < nblocks && e == cudaSuccess) {
      const bool want = ((need[b / 64] & ~have[b / 64]) >> (b % 64)) & 1ull;
      if (!want) {
        ++b;
        continue;
      }
      int64_t b1 = b;
      while (b1 < nblocks && (((need[b1 / 64] & ~have[b1 / 64]) >> (b1 % 64)) & 1ull)) ++b1;
      const int64_t r0 = b * brows, r1 = std::min<int64_t>(A->n, b1 * brows);
      e = cudaMemcpyAsync(dx + r0 * row_bytes, hx + r0 * row_bytes, (r1 - r0) * row_bytes, cudaMemcpyHostToDevice,
                          A->pipe_h2d);
      b = b1;
    }
    for (int w = 0; w < kPipeMaskWords; ++w) have[w] |= need[w];
    if (e == cudaSuccess) e = cudaEventRecord(ev_x[k], A->pipe_h2d);
  }
  // All chunk kernels are queued before any device-to-host copy: with pageable Y a copy call
  // returns only when it is done, which would otherwise hold back the next chunk's launch.
  ens_status st = ENS_OK;
  int64_t launched = 0;
  for (int64_t k = 0; k < chunks && e == cudaSuccess && st == ENS_OK; ++k) {
    const int64_t r0 = A->pipe_row[k], r1 = A->pipe_row[k + 1];
    e = cudaStreamWaitEvent(s, ev_x[k], 0);
    if (e == cudaSuccess) st = launch_gspmv_rows(A, m, dtype, A->stage_x, A->stage_y, r0, r1, s);
    if (e == cudaSuccess && st == ENS_OK) e = cudaEventRecord(ev_y[k], s);
    if (e == cudaSuccess && st == ENS_OK) launched = k + 1;
  }
  for (int64_t k = 0; k < launched && e == cudaSuccess; ++k) {
    const int64_t r0 = A->pipe_row[k], r1 = A->pipe_row[k + 1];
    e = cudaStreamWaitEvent(A->pipe_d2h, ev_y[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hy + r0 * row_bytes, dy + r0 * row_bytes, (r1 - r0) * row_bytes, cudaMemcpyDeviceToHost,
                          A->pipe_d2h);
  }
  // wait for every copy that was issued (also on failure: they read and write the caller's buffers)
  const cudaError_t e1 = cudaStreamSynchronize(A->pipe_h2d);
  const cudaError_t e2 = cudaStreamSynchronize(A->pipe_d2h);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (st != ENS_OK) return st;
  if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
  if (e != cudaSuccess) return cuda_fail(e, "gspmv_host");
  return ENS_OK;
}

}  // extern "C"
