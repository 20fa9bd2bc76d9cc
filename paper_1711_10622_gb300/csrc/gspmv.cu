// GSpMV Y = A X for a CSR matrix and an n x m row-interleaved block (Section 2.3, Fig. GSpMV).
//
// Work mapping: a "row group" of LANES consecutive threads owns one row at a time; each lane
// owns VEC consecutive columns of that row and reads them from X with 16-byte loads (one double2
// or float4; four doubles as two double2), so a row of X (m contiguous values) is read by the
// group as one contiguous segment. Every val[j] and col_idx[j] is loaded once per lane group and
// reused for all the lane's columns; with LANES = m / VEC there is exactly one pass per row. The
// grid is sized to fill the GPU once and strides over tiles of rows; a launch may also cover a
// row range only (the pipelined host-buffer product).
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

#include <type_traits>

#include <cstdint>
#include <vector>

#include "ens_internal.cuh"
#include "rowprod.cuh"

namespace ens {
namespace {

MatView view_of(const ens_matrix *A) {
  return MatView{(int32_t)A->n, A->row, A->col, A->val, A->val32, A->valsplit, A->dinv, A->dinv32};
}

// Tiled GSpMV: CSR segments staged in shared memory (tile_rows), Y written with streaming stores.
template <typename Arith, int VEC, int LANES>
__device__ __forceinline__ void gspmv_body(const MatView &A, int32_t m, const typename Arith::T *__restrict__ X,
                                           typename Arith::T *__restrict__ Y, uint32_t native_mask) {
  using T = typename Arith::T;
  tile_rows<Arith, VEC, LANES>(A, m, X, native_mask,
                               [&](int64_t i, int32_t c, const T (&y)[VEC]) { store_vec_cs<T, VEC>(Y + i * m + c, y); });
}

template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    gspmv_kernel(MatView A, int32_t m, const typename Arith::T *__restrict__ X, typename Arith::T *__restrict__ Y,
                 uint32_t native_mask) {
  gspmv_body<Arith, VEC, LANES>(A, m, X, Y, native_mask);
}

// Register caps (minimum resident blocks per SM) for the gather-latency-bound kernels, which need
// resident warps more than registers. Measured on GB300, channel 256 x 128 x 128:
//   * split float64, two columns per lane: 6 blocks, 40 registers (6 beat 5 by 1-10 % over
//     m = 2..32; 7 or 8 blocks spill and lose 1-10 %);
//   * split float64, four columns per lane: 5 blocks, 48 registers (6 spill 164-212 bytes; 4 blocks
//     with 64 registers lose 2-12 %);
//   * float32: 8 blocks, 32 registers (10-12 % faster than the compiler's own 40 registers over
//     m = 8..32).
// Native float64 keeps the compiler's own choice (no minimum): a minimum of one block, which asks
// for no occupancy at all, let the compiler take far more registers and halved the launches (split
// kernels: 125-140 registers; native m = 32: 3.3 ms against 1.7 ms).
template <typename Arith, int VEC>
struct MinBlocks {
  static constexpr int value = std::is_same<Arith, ArithF32>::value ? 8 : VEC == 4 ? 5 : 6;
};
template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads, MinBlocks<Arith, VEC>::value)
    gspmv_kernel_capped(MatView A, int32_t m, const typename Arith::T *__restrict__ X,
                        typename Arith::T *__restrict__ Y, uint32_t native_mask) {
  gspmv_body<Arith, VEC, LANES>(A, m, X, Y, native_mask);
}

// Untiled variant (direct_rows): an autotuner candidate beside the tiled kernels.
template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads, MinBlocks<Arith, VEC>::value)
    gspmv_kernel_direct(MatView A, int32_t m, const typename Arith::T *__restrict__ X,
                        typename Arith::T *__restrict__ Y, uint32_t native_mask) {
  using T = typename Arith::T;
  direct_rows<Arith, VEC, LANES>(A, m, X, native_mask,
                                 [&](int64_t i, int32_t c, const T (&y)[VEC]) { store_vec_cs<T, VEC>(Y + i * m + c, y); });
}
template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    gspmv_kernel_direct_free(MatView A, int32_t m, const typename Arith::T *__restrict__ X,
                             typename Arith::T *__restrict__ Y, uint32_t native_mask) {
  using T = typename Arith::T;
  direct_rows<Arith, VEC, LANES>(A, m, X, native_mask,
                                 [&](int64_t i, int32_t c, const T (&y)[VEC]) { store_vec_cs<T, VEC>(Y + i * m + c, y); });
}

// A contiguous range of rows [r0, r1) of the product (r0 a multiple of kTileRows, so the shifted
// row-pointer array keeps its 16-byte alignment).
struct Rows {
  int64_t r0, r1;
};
static_assert(kPipeAlignRows % kTileRows == 0, "row chunks must be whole tiles");

int grid_for(const ens_matrix *A, int64_t rows, const void *kernel, int64_t rows_per_block = kTileRows) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (rows + rows_per_block - 1) / rows_per_block;
  const int64_t full = (int64_t)A->num_sms * per_sm;
  return (int)(need < full ? need : full);
}

template <typename Arith, int VEC, int LANES>
cudaError_t run(const ens_matrix *A, int m, const void *X, void *Y, uint32_t mask, const Rows &rows, cudaStream_t s,
                bool direct) {
  using T = typename Arith::T;
  MatView v = view_of(A);
  v.n = (int32_t)(rows.r1 - rows.r0);
  v.rp = A->row + rows.r0;
  T *y = (T *)Y + rows.r0 * m;
  constexpr bool capped = std::is_same<Arith, ArithF64Split>::value || std::is_same<Arith, ArithF32>::value;
  if constexpr (!std::is_same<Arith, ArithF64Hybrid>::value) {
    if (direct) {
      auto k = capped ? gspmv_kernel_direct<Arith, VEC, LANES> : gspmv_kernel_direct_free<Arith, VEC, LANES>;
      k<<<grid_for(A, v.n, (const void *)k, kThreads / LANES), kThreads, 0, s>>>(v, m, (const T *)X, y, mask);
      return cudaGetLastError();
    }
  }
  if constexpr (capped) {
    auto k = gspmv_kernel_capped<Arith, VEC, LANES>;
    k<<<grid_for(A, v.n, (const void *)k), kThreads, 0, s>>>(v, m, (const T *)X, y, mask);
  } else {
    auto k = gspmv_kernel<Arith, VEC, LANES>;
    k<<<grid_for(A, v.n, (const void *)k), kThreads, 0, s>>>(v, m, (const T *)X, y, mask);
  }
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
cudaError_t dispatch(const ens_matrix *A, int m, const void *X, void *Y, int lanes, uint32_t mask, const Rows &rows,
                     cudaStream_t s, bool direct = false) {
  switch (lanes) {
    case 1: return run<Arith, VEC, 1>(A, m, X, Y, mask, rows, s, direct);
    case 2: return run<Arith, VEC, 2>(A, m, X, Y, mask, rows, s, direct);
    case 4: return run<Arith, VEC, 4>(A, m, X, Y, mask, rows, s, direct);
    case 8: return run<Arith, VEC, 8>(A, m, X, Y, mask, rows, s, direct);
    case 16: return run<Arith, VEC, 16>(A, m, X, Y, mask, rows, s, direct);
    default: return run<Arith, VEC, 32>(A, m, X, Y, mask, rows, s, direct);
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
  if (A->f64_mode == ENS_F64_HYBRID) return kShareHybrid;
  if (A->native_share >= 0) return A->native_share;
  if (A->f64_mode == ENS_F64_SPLIT) return 0;
  if (m >= 1 && m <= kTuneMaxM && A->tuned_share[m] >= 0) return A->tuned_share[m];
  // Measured on GB300 (channel 256 x 128 x 128): native DFMA is fastest up to m = 2; at m = 4 nearly
  // all split (4/32: 180 us, against 195 us with 12/32); from m = 8 about 12/32 of the row sweeps
  // on the FP64 pipe and the rest split (m = 32: 928 us against 1077 us all split and 1695 us all
  // native).
  if (m <= 2) return 32;
  if (m < 8) return 4;
  return 12;
}

// Bit s set for about share/32 of the sweep indices s = 0..31, spread evenly.
uint32_t share_mask(int share) {
  uint32_t mask = 0;
  for (int s = 0; s < 32; ++s)
    if (((s + 1) * share) / 32 > (s * share) / 32) mask |= 1u << s;
  return mask;
}

namespace {

// Launch configuration of one product: VEC from m and alignment; lanes per row (rows per warp =
// 32 / lanes, column tile = VEC * lanes); share of native-DFMA sweeps (FP64 only).
struct Cfg {
  int vec, lanes, share;
  bool direct = false;  // untiled rows (direct_rows) instead of shared-memory tiles
};

// VEC and full-width lanes of a float64 launch with native share `share`: split-float products take
// four columns per lane when m allows (two packed float pairs share each nonzero's index and
// matrix pair; measured on GB300, channel 256 x 128 x 128, m = 8..32: 9-11 % faster than two),
// native DFMA and the column hybrid two.
void f64_shape(int m, int share, bool al16, int &vec, int &lanes) {
  if (share < 32 && m % 4 == 0 && al16) {
    vec = 4;
    lanes = pow2_at_least(m / 4, 8);
  } else if (m % 2 == 0 && al16) {
    vec = 2;
    lanes = pow2_at_least(m / 2, 16);
  } else {
    vec = 1;
    lanes = pow2_at_least(m, 32);
  }
}

Cfg default_cfg(const ens_matrix *A, int m, int dtype, const void *X, const void *Y) {
  Cfg c{};
  if (dtype == ENS_F32) {
    if (m % 4 == 0 && aligned(X, 16) && aligned(Y, 16)) {
      c.vec = 4;
      c.lanes = pow2_at_least(m / 4, 8);
    } else if (m % 2 == 0 && aligned(X, 8) && aligned(Y, 8)) {
      c.vec = 2;
      c.lanes = pow2_at_least(m / 2, 16);
    } else {
      c.vec = 1;
      c.lanes = pow2_at_least(m, 32);
    }
    c.share = 0;
  } else {
    c.share = use_split(A) ? native_share(A, m) : 32;
    f64_shape(m, c.share, aligned(X, 16) && aligned(Y, 16), c.vec, c.lanes);
  }
  if (m >= 1 && m <= kTuneMaxM) {
    const int tl = A->tuned_lanes[dtype == ENS_F32 ? 1 : 0][m];
    if (tl > 0 && tl <= c.lanes) c.lanes = tl;  // tuned for the same share, hence VEC (alignment permitting)
    c.direct = A->tuned_direct[dtype == ENS_F32 ? 1 : 0][m] == 1 && c.share != kShareHybrid;
  }
  if (A->untiled >= 0) c.direct = A->untiled == 1 && c.share != kShareHybrid;
  return c;
}

cudaError_t launch_cfg(const ens_matrix *A, int m, int dtype, const void *X, void *Y, const Cfg &c, const Rows &rows,
                       cudaStream_t s) {
  const bool d = c.direct;
  if (dtype == ENS_F32) {
    if (c.vec == 4) return dispatch<ArithF32, 4>(A, m, X, Y, c.lanes, 0u, rows, s, d);
    if (c.vec == 2) return dispatch<ArithF32, 2>(A, m, X, Y, c.lanes, 0u, rows, s, d);
    return dispatch<ArithF32, 1>(A, m, X, Y, c.lanes, 0u, rows, s, d);
  }
  if (c.share == kShareHybrid) {  // column hybrid needs two columns per lane
    return c.vec == 2 ? dispatch<ArithF64Hybrid, 2>(A, m, X, Y, c.lanes, 0u, rows, s)
                      : dispatch<ArithF64Native, 1>(A, m, X, Y, c.lanes, 0u, rows, s);
  }
  if (c.share < 32) {
    const uint32_t mask = share_mask(c.share);
    if (c.vec == 4) return dispatch<ArithF64Split, 4>(A, m, X, Y, c.lanes, mask, rows, s, d);
    return c.vec == 2 ? dispatch<ArithF64Split, 2>(A, m, X, Y, c.lanes, mask, rows, s, d)
                      : dispatch<ArithF64Split, 1>(A, m, X, Y, c.lanes, mask, rows, s, d);
  }
  return c.vec == 2 ? dispatch<ArithF64Native, 2>(A, m, X, Y, c.lanes, 0u, rows, s, d)
                    : dispatch<ArithF64Native, 1>(A, m, X, Y, c.lanes, 0u, rows, s, d);
}

// Deterministic N(0,1)-like fill of the tuning block (values in the split range, no zeros).
__global__ void k_tune_fill(int64_t count, double *x, float *x32) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)(e * 2654435761ull) ^ 0x9E3779B9u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    const float v = 0.25f + (float)(h & 0xFFFFFF) * (1.0f / 16777216.0f);  // [0.25, 1.25)
    const float sgn = (h & 0x80000000u) ? -1.f : 1.f;
    if (x) x[e] = (double)(sgn * v);
    if (x32) x32[e] = sgn * v;
  }
}

}  // namespace

ens_status launch_gspmv(const ens_matrix *A, int m, int dtype, const void *X, void *Y, cudaStream_t s) {
  if (A->n == 0) return ENS_OK;
  const Cfg c = default_cfg(A, m, dtype, X, Y);
  cudaError_t e = launch_cfg(A, m, dtype, X, Y, c, Rows{0, A->n}, s);
  if (e != cudaSuccess) return cuda_fail(e, "gspmv launch");
  return ENS_OK;
}

ens_status launch_gspmv_rows(const ens_matrix *A, int m, int dtype, const void *X, void *Y, int64_t r0, int64_t r1,
                             cudaStream_t s) {
  if (r1 <= r0) return ENS_OK;
  const Cfg c = default_cfg(A, m, dtype, X, Y);
  cudaError_t e = launch_cfg(A, m, dtype, X, Y, c, Rows{r0, r1}, s);
  if (e != cudaSuccess) return cuda_fail(e, "gspmv launch");
  return ENS_OK;
}

// Autotuner: time every candidate (FP64 arithmetic: native DFMA, split with native shares 0, 8, 12,
// 16, 24 and the column hybrid; for each, lanes per row giving the full, half and quarter column
// tile of its VEC) on this matrix for block width m with CUDA events, keep the fastest in the
// matrix's table.
ens_status autotune(ens_matrix *A, int m, int dtype, cudaStream_t s, int32_t *lanes_out, int32_t *share_out,
                    double *best_us_out) {
  const size_t count = (size_t)A->n * m, xcount = (size_t)A->ncols * m;  // Y rows, X rows (= n if square)
  void *X = nullptr, *Y = nullptr;
  const size_t es = dtype == ENS_F32 ? 4 : 8;
  cudaError_t e = cudaMallocAsync(&X, xcount * es, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&Y, count * es, s);
  if (e == cudaSuccess) {
    const int grid = A->num_sms * 8;
    k_tune_fill<<<grid, 256, 0, s>>>((int64_t)xcount, dtype == ENS_F32 ? nullptr : (double *)X,
                                     dtype == ENS_F32 ? (float *)X : nullptr);
    e = cudaGetLastError();
  }
  // the defaults without any previous tuning
  const int di = dtype == ENS_F32 ? 1 : 0;
  const int keep_lanes = A->tuned_lanes[di][m], keep_share = A->tuned_share[m], keep_direct = A->tuned_direct[di][m];
  A->tuned_lanes[di][m] = -1;
  A->tuned_direct[di][m] = -1;
  if (dtype != ENS_F32) A->tuned_share[m] = -1;
  const Cfg base = default_cfg(A, m, dtype, X, Y);
  std::vector<Cfg> cand;
  auto add_widths = [&](int vec, int full, int share) {
    for (int div = 1; div <= 4 && full / div >= 1; div *= 2) {
      cand.push_back(Cfg{vec, full / div, share, false});
      if (share != kShareHybrid) cand.push_back(Cfg{vec, full / div, share, true});
    }
  };
  if (dtype == ENS_F32) {
    add_widths(base.vec, base.lanes, 0);
  } else {
    std::vector<int> shares{32};
    if (use_split(A)) shares.insert(shares.end(), {0, 8, 12, 16, 24, kShareHybrid});
    for (int sh : shares) {
      int vec = 1, full = 1;
      f64_shape(m, sh, true, vec, full);  // the tuning blocks are 256-byte aligned
      if (sh == kShareHybrid && vec != 2) continue;
      add_widths(vec, full, sh);
    }
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 1e30f;
  Cfg bestc = base;
  for (const Cfg &c : cand) {
    if (e != cudaSuccess) break;
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_cfg(A, m, dtype, X, Y, c, Rows{0, A->n}, s);
    if (e == cudaSuccess) e = cudaEventRecord(t0, s);
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = launch_cfg(A, m, dtype, X, Y, c, Rows{0, A->n}, s);
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      bestc = c;
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (X) cudaFreeAsync(X, s);
  if (Y) cudaFreeAsync(Y, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    A->tuned_lanes[di][m] = keep_lanes;
    A->tuned_share[m] = keep_share;
    A->tuned_direct[di][m] = keep_direct;
    return cuda_fail(e, "autotune");
  }
  A->tuned_lanes[di][m] = bestc.lanes;
  A->tuned_direct[di][m] = bestc.direct ? 1 : 0;
  if (dtype != ENS_F32) A->tuned_share[m] = bestc.share;
  if (lanes_out) *lanes_out = bestc.lanes;
  if (share_out) *share_out = bestc.share;
  if (best_us_out) *best_us_out = best * 1e3 / 5.0;
  return ENS_OK;
}

}  // namespace ens
