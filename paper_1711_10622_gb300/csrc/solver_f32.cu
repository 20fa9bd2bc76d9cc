// Instantiation of the float32 BiCGStab (inner solver of the mixed-precision mode).
#include "solver_impl.cuh"

namespace ens {
namespace solver {
template struct Bicg<ArithF32>;
}  // namespace solver
}  // namespace ens
