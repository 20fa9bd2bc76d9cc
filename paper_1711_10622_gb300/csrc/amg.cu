// Aggregation multigrid hierarchy (the set-up half of ENS_PRECOND_AMG): strength of connection,
// three-phase plain aggregation, Galerkin coarse operators P^T A P with piecewise-constant P, and
// the upload of every coarse level as a matrix of its own (so its products use the same GSpMV
// kernels as the fine level). The set-up runs on the host once per matrix; the V-cycle itself is
// in solver_impl.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "ens_internal.cuh"

namespace ens {
namespace {

struct HostCsr {
  int64_t n = 0;
  std::vector<int32_t> row, col;
  std::vector<double> val;
};

// Aggregate (next-level row) of every row; returns the aggregate count.
int64_t aggregate_rows(const HostCsr &L, double theta, std::vector<int32_t> &agg) {
  const int64_t n = L.n;
  std::vector<double> diag(n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t k = L.row[i]; k < L.row[i + 1]; ++k)
      if (L.col[k] == i) diag[i] = L.val[k];
  auto strong = [&](int64_t i, int32_t k) {
    const int32_t j = L.col[k];
    return j != i && std::fabs(L.val[k]) >= theta * std::sqrt(std::fabs(diag[i]) * std::fabs(diag[j]));
  };
  agg.assign(n, -1);
  int64_t count = 0;
  // phase 1: a row whose strong neighbours are all free starts an aggregate with them
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free_nbrs = true;
    for (int32_t k = L.row[i]; k < L.row[i + 1] && free_nbrs; ++k)
      if (strong(i, k) && agg[L.col[k]] >= 0) free_nbrs = false;
    if (!free_nbrs) continue;
    agg[i] = (int32_t)count;
    for (int32_t k = L.row[i]; k < L.row[i + 1]; ++k)
      if (strong(i, k)) agg[L.col[k]] = (int32_t)count;
    ++count;
  }
  // phase 2: join the phase-1 aggregate of the strongest aggregated strong neighbour
  const std::vector<int32_t> first = agg;
  for (int64_t i = 0; i < n; ++i) {
    if (first[i] >= 0) continue;
    double best = -1.0;
    int32_t pick = -1;
    for (int32_t k = L.row[i]; k < L.row[i + 1]; ++k) {
      const int32_t j = L.col[k];
      if (!strong(i, k) || first[j] < 0) continue;
      const double a = std::fabs(L.val[k]);
      if (a > best || (a == best && j < pick)) {
        best = a;
        pick = j;
      }
    }
    if (pick >= 0) agg[i] = first[pick];
  }
  // phase 3: rows still free start aggregates with their free strong neighbours
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = (int32_t)count;
    for (int32_t k = L.row[i]; k < L.row[i + 1]; ++k)
      if (strong(i, k) && agg[L.col[k]] < 0) agg[L.col[k]] = (int32_t)count;
    ++count;
  }
  return count;
}

// Rows of each aggregate in ascending order (counting sort): ptr [nc + 1], members [n].
void group_rows(const std::vector<int32_t> &agg, int64_t nc, std::vector<int32_t> &ptr, std::vector<int32_t> &mem) {
  ptr.assign(nc + 1, 0);
  for (int32_t a : agg) ptr[a + 1]++;
  for (int64_t I = 0; I < nc; ++I) ptr[I + 1] += ptr[I];
  mem.resize(agg.size());
  std::vector<int32_t> next(ptr.begin(), ptr.end() - 1);
  for (int64_t i = 0; i < (int64_t)agg.size(); ++i) mem[next[agg[i]]++] = (int32_t)i;
}

// A_c = P^T A P: coarse row I sums the rows of aggregate I (in ascending row order, each row in CSR
// order) into the columns agg(j); a position table per coarse column keeps every structural entry.
HostCsr galerkin(const HostCsr &L, const std::vector<int32_t> &agg, int64_t nc, const std::vector<int32_t> &ptr,
                 const std::vector<int32_t> &mem) {
  HostCsr C;
  C.n = nc;
  C.row.assign(nc + 1, 0);
  std::vector<int32_t> slot(nc, -1);
  std::vector<std::pair<int32_t, double>> line;
  for (int64_t I = 0; I < nc; ++I) {
    line.clear();
    for (int32_t t = ptr[I]; t < ptr[I + 1]; ++t) {
      const int32_t i = mem[t];
      for (int32_t k = L.row[i]; k < L.row[i + 1]; ++k) {
        const int32_t J = agg[L.col[k]];
        if (slot[J] < 0) {
          slot[J] = (int32_t)line.size();
          line.emplace_back(J, 0.0);
        }
        line[slot[J]].second += L.val[k];
      }
    }
    for (auto &e : line) slot[e.first] = -1;
    std::sort(line.begin(), line.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    for (auto &e : line) {
      C.col.push_back(e.first);
      C.val.push_back(e.second);
    }
    C.row[I + 1] = (int32_t)C.col.size();
  }
  return C;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src, cudaStream_t s) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), std::max<size_t>(src.size(), 1) * sizeof(T));
  if (e != cudaSuccess || src.empty()) return e;
  return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

ens_status check_opts(const ens_amg_opts &o) {
  if (!(o.theta >= 0.0) || !(o.theta < 1.0)) return fail(ENS_ERR_INVALID, "amg_setup: theta must lie in [0, 1)");
  if (o.max_levels < 2 || o.max_levels > 16) return fail(ENS_ERR_INVALID, "amg_setup: max_levels must lie in [2, 16]");
  if (o.coarse_size < 1) return fail(ENS_ERR_INVALID, "amg_setup: coarse_size must be >= 1");
  if (o.smooth_steps < 1 || o.coarse_steps < 1) return fail(ENS_ERR_INVALID, "amg_setup: smoothing steps must be >= 1");
  if (!(o.cheb_lo > 0.0) || !(o.cheb_hi > o.cheb_lo) || !std::isfinite(o.cheb_hi))
    return fail(ENS_ERR_INVALID, "amg_setup: need 0 < cheb_lo < cheb_hi");
  return ENS_OK;
}

}  // namespace

void free_amg(ens_amg *H) {
  if (!H) return;
  for (ens_amg_lev &l : H->lev) {
    if (l.owned) ens_destroy_matrix(l.A);
    ens_destroy_matrix(l.As);
    cudaFree(l.agg);
    cudaFree(l.agg_ptr);
    cudaFree(l.members);
  }
  delete H;
}

}  // namespace ens

using namespace ens;

extern "C" void ens_default_amg_opts(ens_amg_opts *o) {
  if (!o) return;
  o->theta = 0.08;
  o->max_levels = 8;
  o->coarse_size = 512;
  o->smooth_steps = 2;
  o->coarse_steps = 16;
  o->cheb_lo = 2.0 / 30.0;
  o->cheb_hi = 2.0;
}

static ens_status amg_setup_impl(ens_matrix *A, const ens_amg_opts *opts, void *stream);

extern "C" ens_status ens_amg_setup(ens_matrix *A, const ens_amg_opts *opts, void *stream) {
  clear_error();
  try {
    return amg_setup_impl(A, opts, stream);
  } catch (const std::bad_alloc &) {
    return fail(ENS_ERR_OOM, "amg_setup: host allocation failed");
  }
}

static ens_status amg_setup_impl(ens_matrix *A, const ens_amg_opts *opts, void *stream) {
  if (!A) return fail(ENS_ERR_INVALID, "amg_setup: matrix is NULL");
  if (A->ncols != A->n) return fail(ENS_ERR_INVALID, "amg_setup: needs a square matrix");
  ens_amg_opts o;
  ens_default_amg_opts(&o);
  if (opts) o = *opts;
  ens_status st = check_opts(o);
  if (st != ENS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the fine matrix, back on the host
  HostCsr L;
  L.n = A->n;
  L.row.resize(A->n + 1);
  L.col.resize(A->nnz);
  L.val.resize(A->nnz);
  ENS_CUDA_TRY(cudaMemcpyAsync(L.row.data(), A->row, (A->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (A->nnz) {
    ENS_CUDA_TRY(cudaMemcpyAsync(L.col.data(), A->col, A->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ENS_CUDA_TRY(cudaMemcpyAsync(L.val.data(), A->val, A->nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  ENS_CUDA_TRY(cudaStreamSynchronize(s));

  ens_amg *H = new ens_amg();
  H->opts = o;
  H->lev.push_back(ens_amg_lev{A, false});
  cudaError_t e = cudaSuccess;
  while ((int)H->lev.size() < o.max_levels && L.n > o.coarse_size) {
    std::vector<int32_t> agg, ptr, mem;
    const int64_t nc = aggregate_rows(L, o.theta, agg);
    if ((double)nc > (double)L.n / 1.5) break;
    group_rows(agg, nc, ptr, mem);
    HostCsr C = galerkin(L, agg, nc, ptr, mem);
    ens_amg_lev &f = H->lev.back();
    f.nc = nc;
    // the column-scaled copy A D^-1 of this (smoothed) level: the first smoothing update needs
    // A D^-1 src, one product of this copy instead of a scaled intermediate block
    {
      std::vector<double> dinv(L.n, 0.0), vs(L.val.size());
      for (int64_t i = 0; i < L.n; ++i)
        for (int32_t k = L.row[i]; k < L.row[i + 1]; ++k)
          if (L.col[k] == i && L.val[k] != 0.0) dinv[i] = 1.0 / L.val[k];
      for (int64_t i = 0; i < L.n; ++i)
        for (int32_t k = L.row[i]; k < L.row[i + 1]; ++k) vs[k] = L.val[k] * dinv[L.col[k]];
      st = ens_create_matrix(L.n, (int64_t)vs.size(), L.row.data(), L.col.data(), vs.data(), 0, stream, &f.As);
      if (st != ENS_OK) {
        free_amg(H);
        return st;
      }
    }
    e = upload(&f.agg, agg, s);
    if (e == cudaSuccess) e = upload(&f.agg_ptr, ptr, s);
    if (e == cudaSuccess) e = upload(&f.members, mem, s);
    if (e != cudaSuccess) break;
    ens_matrix *Mc = nullptr;
    st = ens_create_matrix(C.n, (int64_t)C.col.size(), C.row.data(), C.col.data(), C.val.data(),
                           A->flags & ENS_MATRIX_SINGULAR, stream, &Mc);
    if (st != ENS_OK) {
      free_amg(H);
      return st;
    }
    H->lev.push_back(ens_amg_lev{Mc, true});
    L = std::move(C);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_amg(H);
    return cuda_fail(e, "amg_setup");
  }
  free_amg(A->amg);
  A->amg = H;
  return ENS_OK;
}

extern "C" ens_status ens_amg_info(const ens_matrix *A, int32_t *levels, int64_t *rows, int64_t *nnz) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "amg_info: matrix is NULL");
  const int32_t nl = A->amg ? (int32_t)A->amg->lev.size() : 0;
  if (levels) *levels = nl;
  for (int32_t l = 0; l < nl; ++l) {
    if (rows) rows[l] = A->amg->lev[l].A->n;
    if (nnz) nnz[l] = A->amg->lev[l].A->nnz;
  }
  return ENS_OK;
}

extern "C" ens_status ens_amg_level(const ens_matrix *A, int32_t level, int32_t *row_ptr, int32_t *col_idx, double *val,
                                    int32_t *agg) {
  clear_error();
  if (!A || !A->amg) return fail(ENS_ERR_INVALID, "amg_level: matrix has no hierarchy");
  if (level < 0 || level >= (int32_t)A->amg->lev.size())
    return fail(ENS_ERR_INVALID, "amg_level: level %d outside [0, %zu)", level, A->amg->lev.size());
  const ens_amg_lev &l = A->amg->lev[level];
  const ens_matrix *M = l.A;
  if (row_ptr) ENS_CUDA_TRY(cudaMemcpy(row_ptr, M->row, (M->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (col_idx && M->nnz) ENS_CUDA_TRY(cudaMemcpy(col_idx, M->col, M->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (val && M->nnz) ENS_CUDA_TRY(cudaMemcpy(val, M->val, M->nnz * sizeof(double), cudaMemcpyDeviceToHost));
  if (agg && l.agg) ENS_CUDA_TRY(cudaMemcpy(agg, l.agg, M->n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  return ENS_OK;
}
