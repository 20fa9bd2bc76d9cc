// Instantiation of the float64 solver on column-hybrid GSpMV arithmetic (one column per lane on
// native DFMA, one on split-float arithmetic).
#include "solver_impl.cuh"

namespace ens {
namespace solver {
template struct Bicg<ArithF64Hybrid>;

ens_status solve_f64_hybrid(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                            const ens_solve_opts &o, ens_solve_stats *st, cudaStream_t s) {
  return solve_f64<ArithF64Hybrid>(M, m, B, X, tol, o, st, s);
}
SysBase *make_system_hybrid(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                            const ens_solve_opts &o, cudaStream_t s) {
  return new SysImpl<ArithF64Hybrid>(M, m, B, X, tol, o, s);
}
}  // namespace solver
}  // namespace ens
