// Device work of one rank in the row-split (domain-decomposed) solve: row blocks of the matrix,
// per-column partial dots, block linear combinations and the halo row gather (ensemble_dist.h).
// All kernels are streaming kernels over n x m row-interleaved blocks: each thread keeps one column
// (the grid stride over the flat index is a multiple of m), so its per-column scalars stay in
// registers and consecutive threads touch consecutive addresses.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ens_internal.cuh"
#include "ensemble_dist.h"
#include "partials.cuh"

namespace ens {
namespace {

constexpr int kDistMaxM = 256;
constexpr int kMaxPairs = 4;
constexpr int kMaxTerms = 4;

struct Ptrs4 {
  const double *p[4];
};

// Threads of the grid and the flat-index stride: the largest multiple of m that is <= the thread
// count, so thread t always visits column t % m. Threads with t >= stride stay idle.
inline int64_t flat_stride(int64_t threads, int32_t m) { return threads / m * m; }

int grid_for_elems(int64_t elems, int sms) {
  const int64_t want = (elems + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
}

// Pass 1: per block, per pair and column, the sum of X*Y over the elements this block's threads
// visit, accumulated per thread in flat-index order and then over the block's threads in thread
// order (fixed order: deterministic). partials[b][k*m + l]. NP pairs; the loads of four strided
// elements are issued before their products, which are then added in the same order as one at a
// time (the same bits, more loads in flight).
template <int NP>
__global__ void __launch_bounds__(kThreads)
    k_dots_partial(int64_t total, int32_t m, Ptrs4 X, Ptrs4 Y, int64_t stride, double *partials) {
  constexpr int U = 4;
  __shared__ double sm[NP][kThreads];
  const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  double acc[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) acc[k] = 0.0;
  if (t < stride) {
    int64_t e = t;
    for (; e + (U - 1) * stride < total; e += U * stride) {
      double x[U][NP], y[U][NP];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          x[u][k] = __ldg(X.p[k] + e + u * stride);
          y[u][k] = __ldg(Y.p[k] + e + u * stride);
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < NP; ++k) acc[k] = fma(x[u][k], y[u][k], acc[k]);
    }
    for (; e < total; e += stride) {
#pragma unroll
      for (int k = 0; k < NP; ++k) acc[k] = fma(__ldg(X.p[k] + e), __ldg(Y.p[k] + e), acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  // thread j < NP*m sums column l = j % m of pair k = j / m over the threads of this block that
  // own column l, in thread order
  const int64_t base = (int64_t)blockIdx.x * kThreads;
  for (int j = threadIdx.x; j < NP * m; j += kThreads) {
    const int k = j / m, l = j % m;
    // first thread of this block whose global index is congruent to l modulo m
    int first = (int)((l - base % m + m) % m);
    double s = 0.0;
    for (int u = first; u < kThreads; u += m)
      if (base + u < stride) s += sm[k][u];
    partials[(int64_t)blockIdx.x * NP * m + j] = s;
  }
}

__global__ void __launch_bounds__(kThreads)
    k_lincomb(int64_t total, int32_t m, int32_t nterms, Ptrs4 coef, Ptrs4 vec, double *out, int64_t stride) {
  const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (t >= stride) return;
  const int l = (int)(t % m);
  double c[kMaxTerms];
#pragma unroll
  for (int k = 0; k < kMaxTerms; ++k) c[k] = (k < nterms) ? (coef.p[k] ? coef.p[k][l] : 1.0) : 0.0;
  for (int64_t e = t; e < total; e += stride) {
    double s = c[0] * vec.p[0][e];
#pragma unroll
    for (int k = 1; k < kMaxTerms; ++k)
      if (k < nterms) s = fma(c[k], vec.p[k][e], s);
    out[e] = s;
  }
}

__global__ void __launch_bounds__(kThreads)
    k_gather_rows(int64_t count, int32_t m, const int32_t *__restrict__ idx, const double *__restrict__ X,
                  double *__restrict__ out) {
  const int64_t total = count * m;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < total; e += (int64_t)gridDim.x * kThreads) {
    const int64_t k = e / m;
    const int l = (int)(e - k * m);
    out[e] = __ldg(X + (int64_t)__ldg(idx + k) * m + l);
  }
}

int device_sms() {
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" {

ens_status ens_create_matrix_rect(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *row_ptr,
                                  const int32_t *col_idx, const double *val, void *stream, ens_matrix **out) {
  clear_error();
  return create_matrix(n_rows, n_cols, nnz, row_ptr, col_idx, val, 0u, stream, out);
}

ens_status ens_matrix_shape(const ens_matrix *A, int64_t *n_rows, int64_t *n_cols) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "matrix_shape: matrix is NULL");
  if (n_rows) *n_rows = A->n;
  if (n_cols) *n_cols = A->ncols;
  return ENS_OK;
}

ens_status ens_block_dots(int64_t n, int32_t m, int32_t npairs, const double *const *X, const double *const *Y,
                          double *out, void *stream) {
  clear_error();
  if (n < 0) return fail(ENS_ERR_INVALID, "block_dots: n < 0");
  if (m < 1 || m > kDistMaxM) return fail(ENS_ERR_INVALID, "block_dots: m = %d outside [1, %d]", m, kDistMaxM);
  if (npairs < 1 || npairs > kMaxPairs) return fail(ENS_ERR_INVALID, "block_dots: npairs = %d outside [1, 4]", npairs);
  if (!X || !Y || !out) return fail(ENS_ERR_INVALID, "block_dots: NULL argument");
  Ptrs4 px{}, py{};
  for (int k = 0; k < npairs; ++k) {
    if (n > 0 && (!X[k] || !Y[k])) return fail(ENS_ERR_INVALID, "block_dots: pair %d has a NULL block", k);
    px.p[k] = X[k];
    py.p[k] = Y[k];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t total = n * m;
  const int grid = grid_for_elems(total, device_sms());
  const int64_t stride = flat_stride((int64_t)grid * kThreads, m);
  double *partials = nullptr;
  ENS_CUDA_TRY(cudaMallocAsync(&partials, (size_t)grid * npairs * m * sizeof(double), s));
  switch (npairs) {
    case 1: k_dots_partial<1><<<grid, kThreads, 0, s>>>(total, m, px, py, stride, partials); break;
    case 2: k_dots_partial<2><<<grid, kThreads, 0, s>>>(total, m, px, py, stride, partials); break;
    case 3: k_dots_partial<3><<<grid, kThreads, 0, s>>>(total, m, px, py, stride, partials); break;
    default: k_dots_partial<4><<<grid, kThreads, 0, s>>>(total, m, px, py, stride, partials); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_partials_final<<<partials_final_grid(npairs * m), 256, 0, s>>>(grid, npairs * m, partials, out);
    e = cudaGetLastError();
  }
  const cudaError_t ef = cudaFreeAsync(partials, s);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return cuda_fail(e, "block_dots");
  return ENS_OK;
}

ens_status ens_block_lincomb(int64_t n, int32_t m, int32_t nterms, const double *const *coef, const double *const *vec,
                             double *out, void *stream) {
  clear_error();
  if (n < 0) return fail(ENS_ERR_INVALID, "block_lincomb: n < 0");
  if (m < 1 || m > kDistMaxM) return fail(ENS_ERR_INVALID, "block_lincomb: m = %d outside [1, %d]", m, kDistMaxM);
  if (nterms < 1 || nterms > kMaxTerms) return fail(ENS_ERR_INVALID, "block_lincomb: nterms = %d outside [1, 4]", nterms);
  if (!coef || !vec || (n > 0 && !out)) return fail(ENS_ERR_INVALID, "block_lincomb: NULL argument");
  if (n == 0) return ENS_OK;
  Ptrs4 pc{}, pv{};
  for (int k = 0; k < nterms; ++k) {
    if (!vec[k]) return fail(ENS_ERR_INVALID, "block_lincomb: term %d has a NULL block", k);
    pc.p[k] = coef[k];
    pv.p[k] = vec[k];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t total = n * m;
  const int grid = grid_for_elems(total, device_sms());
  k_lincomb<<<grid, kThreads, 0, s>>>(total, m, nterms, pc, pv, out, flat_stride((int64_t)grid * kThreads, m));
  ENS_CUDA_TRY(cudaGetLastError());
  return ENS_OK;
}

ens_status ens_gather_rows(int64_t count, int32_t m, const int32_t *idx, const double *X, double *out, void *stream) {
  clear_error();
  if (count < 0 || m < 1) return fail(ENS_ERR_INVALID, "gather_rows: count < 0 or m < 1");
  if (count == 0) return ENS_OK;
  if (!idx || !X || !out) return fail(ENS_ERR_INVALID, "gather_rows: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = grid_for_elems(count * m, device_sms());
  k_gather_rows<<<grid, kThreads, 0, s>>>(count, m, idx, X, out);
  ENS_CUDA_TRY(cudaGetLastError());
  return ENS_OK;
}

}  // extern "C"
