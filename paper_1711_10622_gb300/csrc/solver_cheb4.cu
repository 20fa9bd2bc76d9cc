// Four-column forms of the split float64 solver's heaviest GSpMV kernels (the Chebyshev step, the
// V-cycle's residual and two-update smoothing; launchers declared in solver_impl.cuh), in a
// translation unit of their own so that they compile in parallel with the solver instances.
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

namespace {
int grid4(int num_sms, int64_t grid_cap) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(grid_cap, (int64_t)num_sms * ChebBlocks<ArithF64Split, 4>::value));
}
template <int L>
void resid4(const MatView &A, int32_t m, const double *z, const double *r, double *res, uint32_t mask, int grid,
            cudaStream_t st) {
  k_amg_resid<ArithF64Split, 4, L><<<grid, kThreads, 0, st>>>(A, m, z, r, res, mask);
}
template <int L>
void smooth4(bool add, const MatView &As, const MatView &A, int32_t m, const double *src, double *z, double it, double c1,
             double c2, uint32_t mask, int grid, cudaStream_t st) {
  if (add)
    k_amg_smooth2<ArithF64Split, 4, L, true><<<grid, kThreads, 0, st>>>(As, A, m, src, z, it, c1, c2, mask);
  else
    k_amg_smooth2<ArithF64Split, 4, L, false><<<grid, kThreads, 0, st>>>(As, A, m, src, z, it, c1, c2, mask);
}
}  // namespace

bool launch_amg_resid4_split(int lanes4, const MatView &A, int32_t m, const double *z, const double *r, double *res,
                             uint32_t mask, int num_sms, int64_t grid_cap, cudaStream_t st) {
  const int grid = grid4(num_sms, grid_cap);
  switch (lanes4) {
    case 2: resid4<2>(A, m, z, r, res, mask, grid, st); return true;
    case 4: resid4<4>(A, m, z, r, res, mask, grid, st); return true;
    case 8: resid4<8>(A, m, z, r, res, mask, grid, st); return true;
    default: return false;
  }
}

bool launch_amg_smooth2_4_split(int lanes4, bool add, const MatView &As, const MatView &A, int32_t m, const double *src,
                                double *z, double inv_theta, double c1, double c2, uint32_t mask, int num_sms,
                                int64_t grid_cap, cudaStream_t st) {
  const int grid = grid4(num_sms, grid_cap);
  switch (lanes4) {
    case 2: smooth4<2>(add, As, A, m, src, z, inv_theta, c1, c2, mask, grid, st); return true;
    case 4: smooth4<4>(add, As, A, m, src, z, inv_theta, c1, c2, mask, grid, st); return true;
    case 8: smooth4<8>(add, As, A, m, src, z, inv_theta, c1, c2, mask, grid, st); return true;
    default: return false;
  }
}

}  // namespace solver
}  // namespace ens
