// Per-column block reductions with a deterministic cross-block pass.
//
// A kernel whose threads own (row, column-chunk) pairs accumulates ND per-column sums in
// registers; reduce_cols() combines them inside the block (warp shuffles in a fixed butterfly,
// then a fixed-order sum over warps), writes one partial per block and column, and the last
// block to finish (ticket from an atomic counter) sums the partials in block order and runs a
// per-column finalisation (the scalar step of the solver). No value is ever accumulated with an
// atomic, so results do not depend on block scheduling and are bitwise reproducible.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ens_internal.cuh"

namespace ens {

constexpr int kMaxSolveM = 64;  // columns handled by the solver kernels (one chunk per lane)

template <typename T, int ND>
struct ColTotals {
  T v[ND][kMaxSolveM];
};

// acc[d][q]: this thread's sum for dot d and column lane*VEC + q (zero for idle lanes).
// partials: gridDim.x * ND * m scratch values; counter: zero before the launch, reset to zero by
// the last block. fin(l, totals) runs on threads l < m of the last block.
struct NoAfter {
  __device__ void operator()() const {}
};

// after(): runs once, on thread 0 of the last block, when every column's fin() has finished.
template <typename T, int ND, int VEC, int LANES, typename Fin, typename After = NoAfter>
__device__ __forceinline__ void reduce_cols(T (&acc)[ND][VEC], int32_t m, T *__restrict__ partials,
                                            unsigned *__restrict__ counter, Fin &&fin, After &&after = After()) {
  constexpr int kWarps = kThreads / 32;
  __shared__ ColTotals<T, ND> blk;  // block sums, accumulated warp by warp in a fixed order
  __shared__ ColTotals<T, ND> tot;
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = LANES; off < 32; off <<= 1)
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[d][q] += __shfl_xor_sync(0xffffffffu, acc[d][q], off);
  for (int w = 0; w < kWarps; ++w) {
    if (warp == w && lane < LANES) {
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        const int c = lane * VEC + q;
        if (c < m)
#pragma unroll
          for (int d = 0; d < ND; ++d) blk.v[d][c] = w == 0 ? acc[d][q] : blk.v[d][c] + acc[d][q];
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < ND * m; t += kThreads) partials[(size_t)blockIdx.x * ND * m + t] = blk.v[t / m][t % m];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int t = warp; t < ND * m; t += kWarps) {
    T s = T(0);
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partials + (size_t)b * ND * m + t);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) tot.v[t / m][t % m] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x < m) fin((int)threadIdx.x, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    after();
    *counter = 0u;
  }
}

}  // namespace ens
