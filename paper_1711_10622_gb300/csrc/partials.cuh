// Deterministic second pass of the per-block column reductions (block dots, Gram products, column
// statistics): out[j] = sum over b < nblocks of partials[b * width + j].
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ens {
namespace {

// One block of 256 threads per output j (grid-stride over j): thread t sums the partials of blocks
// t, t + 256, t + 512, ... in that order, then the 256 thread sums are added by a fixed binary tree.
// The same nblocks and width always give the same bits.
__global__ void __launch_bounds__(256)
    k_partials_final(int32_t nblocks, int32_t width, const double *__restrict__ partials, double *__restrict__ out) {
  __shared__ double sm[256];
  for (int32_t j = blockIdx.x; j < width; j += gridDim.x) {
    double s = 0.0;
    for (int32_t b = threadIdx.x; b < nblocks; b += 256) s += partials[(int64_t)b * width + j];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = sm[0];
    __syncthreads();
  }
}

inline int partials_final_grid(int32_t width) { return width < 1024 ? (width > 0 ? width : 1) : 1024; }

}  // namespace
}  // namespace ens
