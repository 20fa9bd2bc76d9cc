// Instantiation of the float64 solver on split-float GSpMV arithmetic.
#include "solver_impl.cuh"

namespace ens {
namespace solver {
template struct Bicg<ArithF64Split>;

ens_status solve_f64_split(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                           const ens_solve_opts &o, ens_solve_stats *st, cudaStream_t s) {
  return solve_f64<ArithF64Split>(M, m, B, X, tol, o, st, s);
}
SysBase *make_system_split(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                           const ens_solve_opts &o, cudaStream_t s) {
  return new SysImpl<ArithF64Split>(M, m, B, X, tol, o, s);
}
}  // namespace solver
}  // namespace ens
