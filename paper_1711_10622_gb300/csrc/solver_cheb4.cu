// Four-column Chebyshev steps of the split float64 solver (launch_cheb4_split, solver_impl.cuh), in
// a translation unit of their own so that they compile in parallel with the solver instances.
#include "solver_impl.cuh"

namespace ens {
namespace solver {

namespace {
template <int L>
void cheb4(bool first, bool last, const MatView &A, int32_t m, const double *din, double *dout, const double *src,
           double *res, double *z, double c1, double c2, uint32_t mask, int grid, cudaStream_t st) {
  if (first && last)
    k_cheb<ArithF64Split, 4, L, true, true><<<grid, kThreads, 0, st>>>(A, m, din, dout, src, res, z, c1, c2, mask);
  else if (first)
    k_cheb<ArithF64Split, 4, L, true, false><<<grid, kThreads, 0, st>>>(A, m, din, dout, src, res, z, c1, c2, mask);
  else if (last)
    k_cheb<ArithF64Split, 4, L, false, true><<<grid, kThreads, 0, st>>>(A, m, din, dout, src, res, z, c1, c2, mask);
  else
    k_cheb<ArithF64Split, 4, L, false, false><<<grid, kThreads, 0, st>>>(A, m, din, dout, src, res, z, c1, c2, mask);
}
}  // namespace

bool launch_cheb4_split(int lanes4, bool first, bool last, const MatView &A, int32_t m, const double *din,
                        double *dout, const double *src, double *res, double *z, double c1, double c2,
                        uint32_t mask, int num_sms, int64_t grid_cap, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(grid_cap, (int64_t)num_sms * ChebBlocks<ArithF64Split, 4>::value));
  switch (lanes4) {  // one lane per row (m = 4) spills at 48 registers: the two-column form runs it
    case 2: cheb4<2>(first, last, A, m, din, dout, src, res, z, c1, c2, mask, grid, st); return true;
    case 4: cheb4<4>(first, last, A, m, din, dout, src, res, z, c1, c2, mask, grid, st); return true;
    case 8: cheb4<8>(first, last, A, m, din, dout, src, res, z, c1, c2, mask, grid, st); return true;
    default: return false;
  }
}

}  // namespace solver
}  // namespace ens
