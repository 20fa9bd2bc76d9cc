// C ABI of the multi-RHS solve: option defaults, validation and dispatch on the FP64 arithmetic.
// The solver itself is in solver_impl.cuh (instantiated in solver_{f32,split,native}.cu).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include <memory>
#include <type_traits>
#include <vector>

#include "ens_internal.cuh"
#include "solver_impl.cuh"

namespace ens {

bool use_split(const ens_matrix *A);

namespace solver {
ens_status solve_f64_split(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                           const ens_solve_opts &o, ens_solve_stats *st, cudaStream_t s);
ens_status solve_f64_native(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                            const ens_solve_opts &o, ens_solve_stats *st, cudaStream_t s);
ens_status solve_f64_hybrid(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                            const ens_solve_opts &o, ens_solve_stats *st, cudaStream_t s);
}  // namespace solver

// FP64 arithmetic of the solver's products for block width m (padded to even): native, split with
// a native share, or the column hybrid (0, 1, 2).
static int solver_arith(const ens_matrix *A, int32_t m) {
  if (!use_split(A)) return 0;
  const int mp = m == 1 ? 1 : (m + 1) / 2 * 2;
  const int share = native_share(A, mp);
  if (share == kShareHybrid) return mp % 2 == 0 ? 2 : 0;
  return share >= 32 ? 0 : 1;
}

namespace {

ens_status validate_solve(const ens_matrix *A, int32_t m, const double *B, double *X, const double *tol,
                          const ens_solve_opts &o) {
  if (!A) return fail(ENS_ERR_INVALID, "solve_block: matrix is NULL");
  if (A->ncols != A->n) return fail(ENS_ERR_INVALID, "solve_block: needs a square matrix");
  if (m < 1 || m > kMaxSolveM) return fail(ENS_ERR_INVALID, "solve_block: m = %d outside [1, %d]", m, kMaxSolveM);
  if (!B || !X) return fail(ENS_ERR_INVALID, "solve_block: B or X is NULL");
  if (!tol) return fail(ENS_ERR_INVALID, "solve_block: tol is NULL");
  for (int l = 0; l < m; ++l)
    if (!(tol[l] >= 0.0) || !std::isfinite(tol[l]))
      return fail(ENS_ERR_INVALID, "solve_block: tol[%d] must be finite and >= 0", l);
  if ((uintptr_t)B % 8 || (uintptr_t)X % 8) return fail(ENS_ERR_INVALID, "solve_block: B/X not 8-byte aligned");
  if (o.max_iter < 0) return fail(ENS_ERR_INVALID, "solve_block: max_iter < 0");
  if (o.precond != ENS_PRECOND_NONE && o.precond != ENS_PRECOND_CHEBYSHEV && o.precond != ENS_PRECOND_AMG)
    return fail(ENS_ERR_INVALID, "solve_block: unknown preconditioner %d", o.precond);
  if (o.precond == ENS_PRECOND_AMG) {
    if (!A->amg) return fail(ENS_ERR_INVALID, "solve_block: ENS_PRECOND_AMG needs ens_amg_setup on the matrix");
    if (!A->full_diag) return fail(ENS_ERR_INVALID, "solve_block: AMG smoothing needs a nonzero diagonal in every row");
  }
  if (o.precond == ENS_PRECOND_CHEBYSHEV) {
    if (o.cheb_steps < 1 || o.cheb_steps > 64) return fail(ENS_ERR_INVALID, "solve_block: cheb_steps outside [1, 64]");
    if (!(o.cheb_lo > 0.0) || !(o.cheb_hi > o.cheb_lo) || !std::isfinite(o.cheb_hi))
      return fail(ENS_ERR_INVALID, "solve_block: need 0 < cheb_lo < cheb_hi");
    if (!A->full_diag) return fail(ENS_ERR_INVALID, "solve_block: Chebyshev needs a nonzero diagonal in every row");
  }
  if (o.precision != ENS_PREC_F64 && o.precision != ENS_PREC_MIXED)
    return fail(ENS_ERR_INVALID, "solve_block: unknown precision %d", o.precision);
  if (o.precision == ENS_PREC_MIXED && (!(o.inner_tol > 0.0) || !(o.inner_tol < 1.0) || o.max_outer < 1 || o.inner_max_iter < 0))
    return fail(ENS_ERR_INVALID, "solve_block: mixed mode needs 0 < inner_tol < 1, max_outer >= 1, inner_max_iter >= 0");
  if (o.check_every < 1) return fail(ENS_ERR_INVALID, "solve_block: check_every < 1");
  if (o.workspace && ((uintptr_t)o.workspace % 256))
    return fail(ENS_ERR_INVALID, "solve_block: workspace must be 256-byte aligned");
  return ENS_OK;
}

// A solve that ran out of its caller-provided workspace reports ENS_ERR_BUDGET with the size.
ens_status workspace_status(ens_status st, const ens_solve_opts &o, const char *who) {
  if (st != ENS_OK && o.workspace && last_workspace_overflow())
    return fail(ENS_ERR_BUDGET, "%s: the %llu-byte workspace is too small (the call needs at least %llu bytes)", who,
                (unsigned long long)o.workspace_bytes, (unsigned long long)ens_last_workspace_bytes());
  return st;
}

}  // namespace
}  // namespace ens

using namespace ens;
extern "C" {

void ens_default_solve_opts(ens_solve_opts *o) {
  if (!o) return;
  o->max_iter = 10000;
  o->precond = ENS_PRECOND_NONE;
  o->cheb_steps = 4;
  o->cheb_lo = 2.0 / 30.0;
  o->cheb_hi = 2.0;
  o->precision = ENS_PREC_F64;
  o->inner_tol = 1e-3;
  o->max_outer = 50;
  o->inner_max_iter = 100;
  o->check_every = 1;
  o->x0_zero = 0;
  o->use_graph = 1;
  o->workspace = nullptr;
  o->workspace_bytes = 0;
}

ens_status ens_solve_batch(int32_t nsys, const ens_batch_item *items, const ens_solve_opts *opts, void *stream) {
  clear_error();
  if (nsys < 1 || !items) return fail(ENS_ERR_INVALID, "solve_batch: need nsys >= 1 items");
  ens_solve_opts o;
  ens_default_solve_opts(&o);
  if (opts) o = *opts;
  for (int32_t i = 0; i < nsys; ++i) {
    const ens_batch_item &it = items[i];
    ens_status st = validate_solve(it.A, it.m, it.B, it.X, it.tol, o);
    if (st != ENS_OK) {
      const std::string msg = ens_last_error();
      return fail(st, "solve_batch: item %d: %s", i, msg.c_str());
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<std::unique_ptr<solver::SysBase>> sys;
  for (int32_t i = 0; i < nsys; ++i) {
    const ens_batch_item &it = items[i];
    const int ar = solver_arith(it.A, it.m);
    sys.emplace_back(ar == 2   ? solver::make_system_hybrid(it.A, it.m, it.B, it.X, it.tol, o, s)
                     : ar == 1 ? solver::make_system_split(it.A, it.m, it.B, it.X, it.tol, o, s)
                               : solver::make_system_native(it.A, it.m, it.B, it.X, it.tol, o, s));
  }
  cudaError_t e = cudaSuccess;
  {
    solver::Scratch sc(s, o);
    for (auto &p : sys)
      if (e == cudaSuccess) e = p->setup(sc);
    // one graph: a branch per system forked from and joined into a private capture stream
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> br(nsys, nullptr);
    std::vector<cudaEvent_t> ev(nsys + 1, nullptr);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    for (int32_t i = 0; i < nsys && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
    for (int32_t i = 0; i <= nsys && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t ek = cudaEventRecord(ev[nsys], cap);
      for (int32_t i = 0; i < nsys && ek == cudaSuccess; ++i) {
        ek = cudaStreamWaitEvent(br[i], ev[nsys], 0);
        if (ek == cudaSuccess) ek = sys[i]->record(br[i]);
        if (ek == cudaSuccess) ek = cudaEventRecord(ev[i], br[i]);
        if (ek == cudaSuccess) ek = cudaStreamWaitEvent(cap, ev[i], 0);
      }
      e = cudaStreamEndCapture(cap, &g);
      if (e == cudaSuccess) e = ek;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
    for (auto &p : sys)
      if (e == cudaSuccess) e = p->fetch();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    for (cudaStream_t x : br)
      if (x) cudaStreamDestroy(x);
    if (cap) cudaStreamDestroy(cap);
  }
  const cudaError_t esync = cudaStreamSynchronize(s);  // also on failure (queued work may use the scratch)
  if (e == cudaSuccess) e = esync;
  if (e != cudaSuccess) return workspace_status(cuda_fail(e, "solve_batch"), o, "solve_batch");
  for (int32_t i = 0; i < nsys; ++i) sys[i]->write(items[i].stats);
  return ENS_OK;
}

ens_status ens_solve_block(const ens_matrix *A, int32_t m, const double *B, double *X, const double *tol,
                           const ens_solve_opts *opts, ens_solve_stats *stats, void *stream) {
  clear_error();
  ens_solve_opts o;
  ens_default_solve_opts(&o);
  if (opts) o = *opts;
  ens_status st = validate_solve(A, m, B, X, tol, o);
  if (st != ENS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int ar = solver_arith(A, m);
  if (ar == 2) st = solver::solve_f64_hybrid(A, m, B, X, tol, o, stats, s);
  else if (ar == 1) st = solver::solve_f64_split(A, m, B, X, tol, o, stats, s);
  else st = solver::solve_f64_native(A, m, B, X, tol, o, stats, s);
  return workspace_status(st, o, "solve_block");
}

}  // extern "C"

// ----------------------------------------------------------------------------- AMG apply
namespace ens {
namespace {

template <typename T>
__global__ void k_amg_pad(int64_t n, int32_t m, int32_t mp, const T *__restrict__ src, T *__restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * mp; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / mp;
    const int32_t l = (int32_t)(t - i * mp);
    dst[t] = l < m ? src[i * m + l] : T(0);
  }
}
template <typename T>
__global__ void k_amg_unpad(int64_t n, int32_t m, int32_t mp, const T *__restrict__ src, T *__restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * m; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / m;
    dst[t] = src[i * mp + (t - i * m)];
  }
}

template <typename Arith>
ens_status amg_apply_impl(const ens_matrix *A, int32_t m, const void *R, void *Z, cudaStream_t s) {
  using T = typename Arith::T;
  const int32_t mp = m == 1 ? 1 : (m + 1) & ~1;
  // the solver's column mapping: four float32 columns per lane where the width and (for unpadded
  // blocks, which are used in place) the 16-byte alignment allow, two otherwise
  const bool al16 = mp != m || ((uintptr_t)R % 16 == 0 && (uintptr_t)Z % 16 == 0);
  const int vec = mp == 1 ? 1 : (std::is_same<Arith, ArithF32>::value && mp % 4 == 0 && al16) ? 4 : 2;
  int lanes = 1;
  while (lanes * vec < mp) lanes <<= 1;
  const int64_t n = A->n;
  cudaError_t e = cudaSuccess;
  {
    solver::Scratch sc(s);
    const T *r = (const T *)R;
    T *z = (T *)Z;
    T *rp = nullptr, *zp = nullptr;
    const int pgrid = (int)std::max<int64_t>(1, std::min<int64_t>((n * mp + 255) / 256, (int64_t)A->num_sms * 8));
    if (mp != m) {
      e = sc.get(&rp, (size_t)n * mp);
      if (e == cudaSuccess) e = sc.get(&zp, (size_t)n * mp);
      if (e == cudaSuccess) {
        k_amg_pad<T><<<pgrid, 256, 0, s>>>(n, m, mp, r, rp);
        e = cudaGetLastError();
      }
      r = rp;
    }
    solver::AmgCycle<Arith> cyc;
    if (e == cudaSuccess) e = cyc.setup(sc, A->amg, mp, vec, lanes);
    if (e == cudaSuccess) e = cyc.apply(r, mp != m ? zp : z, s);
    if (e == cudaSuccess && mp != m) {
      k_amg_unpad<T><<<pgrid, 256, 0, s>>>(n, m, mp, zp, z);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "amg_apply");
  return ENS_OK;
}

}  // namespace
}  // namespace ens

extern "C" ens_status ens_amg_apply(const ens_matrix *A, int32_t m, int32_t dtype, const void *R, void *Z, void *stream) {
  clear_error();
  if (!A || !A->amg) return fail(ENS_ERR_INVALID, "amg_apply: matrix has no hierarchy (ens_amg_setup)");
  if (A->ncols != A->n) return fail(ENS_ERR_INVALID, "amg_apply: needs a square matrix");
  if (m < 1 || m > kMaxSolveM) return fail(ENS_ERR_INVALID, "amg_apply: m = %d outside [1, %d]", m, kMaxSolveM);
  if (!R || !Z) return fail(ENS_ERR_INVALID, "amg_apply: R or Z is NULL");
  if (dtype != ENS_F64 && dtype != ENS_F32) return fail(ENS_ERR_INVALID, "amg_apply: unknown dtype %d", dtype);
  if (!A->full_diag) return fail(ENS_ERR_INVALID, "amg_apply: smoothing needs a nonzero diagonal in every row");
  const size_t es = dtype == ENS_F64 ? 8 : 4;
  const uintptr_t r = (uintptr_t)R, z = (uintptr_t)Z, bytes = (uintptr_t)A->n * m * es;
  if (r < z + bytes && z < r + bytes) return fail(ENS_ERR_INVALID, "amg_apply: R and Z overlap");
  if (r % (2 * es) || z % (2 * es)) return fail(ENS_ERR_INVALID, "amg_apply: R/Z must be %zu-byte aligned", 2 * es);
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == ENS_F32) return amg_apply_impl<ArithF32>(A, m, R, Z, s);
  return use_split(A) ? amg_apply_impl<ArithF64Split>(A, m, R, Z, s) : amg_apply_impl<ArithF64Native>(A, m, R, Z, s);
}
