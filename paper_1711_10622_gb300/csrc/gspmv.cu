// GSpMV Y = A X for a CSR matrix and an n x m row-interleaved block (Section 2.3, Fig. GSpMV).
//
// Work mapping: a "row group" of LANES consecutive threads owns one row at a time; each lane
// owns VEC consecutive columns of that row and reads them from X with one VEC-wide load
// (128-bit for double2 / float4), so a row of X (m contiguous values) is read by the group as
// one contiguous segment. Every val[j] and col_idx[j] is loaded once per lane group and reused
// for all the lane's columns; with LANES = m / VEC there is exactly one pass per row. The grid
// is sized to fill the GPU once and strides over the rows.
//
// Three arithmetic variants:
//   * float32 (ENS_F32): float products and sums (inner solver of the mixed-precision mode).
//   * native float64: one DFMA per product.
//   * split float64: FP64-accurate products on the FP32 pipe. GB300's FP64 rate is a small
//     fraction of its FP32 rate, so native DFMA makes the FP64 product ALU-bound for m >= 2;
//     here each value is carried as an unevaluated sum hi + lo of two floats (about 47
//     significant bits) and each row sum is accumulated error-free in (hi, lo) form. Segments
//     whose X values fall outside the split range are recomputed with native DFMA.
#include <cuda_runtime.h>

#include <cstdint>

#include "ens_internal.cuh"
#include "rowprod.cuh"

namespace ens {
namespace {

MatView view_of(const ens_matrix *A) {
  return MatView{(int32_t)A->n, A->row, A->col, A->val, A->val32, A->valsplit, A->dinv, A->dinv32};
}

// Tiled GSpMV: CSR segments staged in shared memory (tile_rows), Y written with streaming stores.
template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    gspmv_kernel(MatView A, int32_t m, const typename Arith::T *__restrict__ X, typename Arith::T *__restrict__ Y,
                 uint32_t native_mask) {
  using T = typename Arith::T;
  tile_rows<Arith, VEC, LANES>(A, m, X, native_mask,
                               [&](int64_t i, int32_t c, const T (&y)[VEC]) { store_vec_cs<T, VEC>(Y + i * m + c, y); });
}

int grid_for(const ens_matrix *A, const void *kernel) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (A->n + kTileRows - 1) / kTileRows;
  const int64_t full = (int64_t)A->num_sms * per_sm;
  return (int)(need < full ? need : full);
}

template <typename Arith, int VEC, int LANES>
cudaError_t run(const ens_matrix *A, int m, const void *X, void *Y, uint32_t mask, cudaStream_t s) {
  using T = typename Arith::T;
  auto k = gspmv_kernel<Arith, VEC, LANES>;
  const int grid = grid_for(A, (const void *)k);
  k<<<grid, kThreads, 0, s>>>(view_of(A), m, (const T *)X, (T *)Y, mask);
  return cudaGetLastError();
}

int pow2_at_least(int v, int cap) {
  int p = 1;
  while (p < v && p < cap) p <<= 1;
  return p;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Dispatch on LANES, a power of two in [1, 32].
template <typename Arith, int VEC>
cudaError_t dispatch(const ens_matrix *A, int m, const void *X, void *Y, int lanes, uint32_t mask, cudaStream_t s) {
  switch (lanes) {
    case 1: return run<Arith, VEC, 1>(A, m, X, Y, mask, s);
    case 2: return run<Arith, VEC, 2>(A, m, X, Y, mask, s);
    case 4: return run<Arith, VEC, 4>(A, m, X, Y, mask, s);
    case 8: return run<Arith, VEC, 8>(A, m, X, Y, mask, s);
    case 16: return run<Arith, VEC, 16>(A, m, X, Y, mask, s);
    default: return run<Arith, VEC, 32>(A, m, X, Y, mask, s);
  }
}

}  // namespace

bool use_split(const ens_matrix *A) {
  return A->f64_mode != ENS_F64_NATIVE && A->split_ok && A->max_row_len <= kSplitMaxRow;
}

// Share (in 32nds) of row sweeps given to native DFMA in split mode, by block width m: the FP64
// pipe is otherwise idle, so hybrid tiles add its throughput to that of the split path. A value
// set with ens_set_native_share overrides the table.
int native_share(const ens_matrix *A, int m) {
  if (A->native_share >= 0) return A->native_share;
  if (A->f64_mode == ENS_F64_SPLIT) return 0;
  // Measured on GB300 (channel 256 x 128 x 128): native DFMA is fastest up to m = 2; beyond, half
  // of the row sweeps on the FP64 pipe and half split is fastest (m = 32: 1213 us against 1444 us
  // all split and 1710 us all native).
  if (m <= 2) return 32;
  return 16;
}

// Bit s set for about share/32 of the sweep indices s = 0..31, spread evenly.
uint32_t share_mask(int share) {
  uint32_t mask = 0;
  for (int s = 0; s < 32; ++s)
    if (((s + 1) * share) / 32 > (s * share) / 32) mask |= 1u << s;
  return mask;
}

ens_status launch_gspmv(const ens_matrix *A, int m, int dtype, const void *X, void *Y, cudaStream_t s) {
  if (A->n == 0) return ENS_OK;
  cudaError_t e;
  if (dtype == ENS_F32) {
    if (m % 4 == 0 && aligned(X, 16) && aligned(Y, 16))
      e = dispatch<ArithF32, 4>(A, m, X, Y, pow2_at_least(m / 4, 8), 0u, s);
    else if (m % 2 == 0 && aligned(X, 8) && aligned(Y, 8))
      e = dispatch<ArithF32, 2>(A, m, X, Y, pow2_at_least(m / 2, 16), 0u, s);
    else
      e = dispatch<ArithF32, 1>(A, m, X, Y, pow2_at_least(m, 32), 0u, s);
  } else {
    const bool vec2 = (m % 2 == 0) && aligned(X, 16) && aligned(Y, 16);
    const int lanes = vec2 ? pow2_at_least(m / 2, 16) : pow2_at_least(m, 32);
    const int share = use_split(A) ? native_share(A, m) : 32;
    if (share < 32) {
      const uint32_t mask = share_mask(share);
      e = vec2 ? dispatch<ArithF64Split, 2>(A, m, X, Y, lanes, mask, s)
               : dispatch<ArithF64Split, 1>(A, m, X, Y, lanes, mask, s);
    } else {
      e = vec2 ? dispatch<ArithF64Native, 2>(A, m, X, Y, lanes, 0u, s)
               : dispatch<ArithF64Native, 1>(A, m, X, Y, lanes, 0u, s);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "gspmv launch");
  return ENS_OK;
}

}  // namespace ens
