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

namespace ens {
namespace {

template <typename T, int VEC>
struct Vec;
template <>
struct Vec<double, 1> { using type = double; };
template <>
struct Vec<double, 2> { using type = double2; };
template <>
struct Vec<float, 1> { using type = float; };
template <>
struct Vec<float, 2> { using type = float2; };
template <>
struct Vec<float, 4> { using type = float4; };

template <typename T, int VEC>
__device__ __forceinline__ void load_x(const T *__restrict__ p, T (&v)[VEC]) {
  using V = typename Vec<T, VEC>::type;
  const V t = __ldg(reinterpret_cast<const V *>(p));
  const T *e = reinterpret_cast<const T *>(&t);
#pragma unroll
  for (int q = 0; q < VEC; ++q) v[q] = e[q];
}

template <typename T, int VEC>
__device__ __forceinline__ void store_y(T *__restrict__ p, const T (&v)[VEC]) {
  using V = typename Vec<T, VEC>::type;
  V t;
  T *e = reinterpret_cast<T *>(&t);
#pragma unroll
  for (int q = 0; q < VEC; ++q) e[q] = v[q];
  __stcs(reinterpret_cast<V *>(p), t);  // streaming store: Y is written once
}

constexpr int kUnroll = 4;

// ------------------------------------------------------------------ float32 / native float64
template <typename T, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    gspmv_plain(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                const T *__restrict__ va, int32_t m, const T *__restrict__ X, T *__restrict__ Y) {
  const int lane = threadIdx.x % LANES;
  const int64_t G = (int64_t)gridDim.x * (kThreads / LANES);
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / LANES) + threadIdx.x / LANES; i < n; i += G) {
    const int32_t j0 = __ldg(rp + i), j1 = __ldg(rp + i + 1);
    for (int32_t c = lane * VEC; c < m; c += LANES * VEC) {
      T acc[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] = T(0);
      int32_t j = j0;
      for (; j + kUnroll <= j1; j += kUnroll) {
        int32_t k[kUnroll];
        T a[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          k[u] = __ldcs(ci + j + u);
          a[u] = __ldcs(va + j + u);
        }
        T x[kUnroll][VEC];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) load_x<T, VEC>(X + (int64_t)k[u] * m + c, x[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[q] = fma(a[u], x[u][q], acc[q]);
      }
      for (; j < j1; ++j) {
        const int32_t k = __ldcs(ci + j);
        const T a = __ldcs(va + j);
        T x[VEC];
        load_x<T, VEC>(X + (int64_t)k * m + c, x);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = fma(a, x[q], acc[q]);
      }
      store_y<T, VEC>(Y + i * m + c, acc);
    }
  }
}

// ------------------------------------------------------------------ split float64
// x = hi + lo with hi = x rounded toward zero to a float and lo holding the next 23 mantissa
// bits of x exactly (bits 5..0 of the 52-bit mantissa are dropped: |x - hi - lo| < 2^-46 |x|).
// Built from the bit pattern: the exponent of lo's leading bit is that of hi minus 23, so
// lo = F - P where P = sign(x) 2^(e-23) and F = P with the 23 kept bits as its mantissa (the
// subtraction is exact). Valid while hi is a normal float with biased exponent >= 24; the caller
// checks the range.
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo) {
  hi = __double2float_rz(x);
  const uint32_t hb = __float_as_uint(hi);
  const uint32_t lw = (uint32_t)__double_as_longlong(x);
  const uint32_t pb = (hb & 0xFF800000u) - (23u << 23);
  lo = __fsub_rn(__uint_as_float(pb | ((lw >> 6) & 0x7FFFFFu)), __uint_as_float(pb));
}

// The split product path is used for |x| in [2^-50, 2^61) (float biased exponents 77..187) and
// |val| in the same range (checked once per matrix, zeros allowed): every nonzero product then
// lies in [2^-100, 2^122), so the absolute error of a row is at most about 2^-46 of its
// sum_j |val||x| (low parts that turn subnormal carry errors below 2^-149, i.e. 2^-49 of the
// smallest product), and sums of up to kSplitMaxRow products do not overflow. Exact zeros in X
// take the native path (their exponent field is 0).
constexpr uint32_t kSplitExpLo = 77u, kSplitExpHi = 187u;

__device__ __forceinline__ bool split_out_of_range(float hi) {
  return ((__float_as_uint(hi) & 0x7F800000u) - (kSplitExpLo << 23)) > ((kSplitExpHi - kSplitExpLo) << 23);
}

// (s, e) = TwoSum(a, b): s = fl(a + b), s + e = a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc_hi + acc_lo += (ah + al) * (xh + xl); the al*xl term (~2^-48 relative) is dropped.
__device__ __forceinline__ void split_fma(float ah, float al, float xh, float xl, float &acc_hi, float &acc_lo) {
  const float ph = __fmul_rn(ah, xh);
  float pl = __fmaf_rn(ah, xh, -ph);  // exact rounding error of ah*xh
  pl = __fmaf_rn(ah, xl, pl);
  pl = __fmaf_rn(al, xh, pl);
  float s, e;
  two_sum(acc_hi, ph, s, e);
  acc_hi = s;
  acc_lo = __fadd_rn(acc_lo, __fadd_rn(e, pl));
}

// Both floats widen exactly; one double rounding of their sum.
__device__ __forceinline__ double split_to_double(float hi, float lo) { return (double)hi + (double)lo; }

template <int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    gspmv_split(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                const float2 *__restrict__ vs, const double *__restrict__ va, int32_t m,
                const double *__restrict__ X, double *__restrict__ Y) {
  const int lane = threadIdx.x % LANES;
  const int64_t G = (int64_t)gridDim.x * (kThreads / LANES);
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / LANES) + threadIdx.x / LANES; i < n; i += G) {
    const int32_t j0 = __ldg(rp + i), j1 = __ldg(rp + i + 1);
    for (int32_t c = lane * VEC; c < m; c += LANES * VEC) {
      float sh[VEC], sl[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) sh[q] = sl[q] = 0.f;
      bool bad = false;
      int32_t j = j0;
      for (; j + kUnroll <= j1; j += kUnroll) {
        int32_t k[kUnroll];
        float2 a[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          k[u] = __ldcs(ci + j + u);
          a[u] = __ldcs(vs + j + u);
        }
        double x[kUnroll][VEC];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) load_x<double, VEC>(X + (int64_t)k[u] * m + c, x[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            float xh, xl;
            split_f64(x[u][q], xh, xl);
            bad |= split_out_of_range(xh);
            split_fma(a[u].x, a[u].y, xh, xl, sh[q], sl[q]);
          }
      }
      for (; j < j1; ++j) {
        const int32_t k = __ldcs(ci + j);
        const float2 a = __ldcs(vs + j);
        double x[VEC];
        load_x<double, VEC>(X + (int64_t)k * m + c, x);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          float xh, xl;
          split_f64(x[q], xh, xl);
          bad |= split_out_of_range(xh);
          split_fma(a.x, a.y, xh, xl, sh[q], sl[q]);
        }
      }
      double y[VEC];
      if (!bad) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) y[q] = split_to_double(sh[q], sl[q]);
      } else {  // values outside the split range: native FP64 for this row segment
#pragma unroll
        for (int q = 0; q < VEC; ++q) y[q] = 0.0;
        for (int32_t jj = j0; jj < j1; ++jj) {
          const double av = __ldg(va + jj);
          double x[VEC];
          load_x<double, VEC>(X + (int64_t)__ldg(ci + jj) * m + c, x);
#pragma unroll
          for (int q = 0; q < VEC; ++q) y[q] = fma(av, x[q], y[q]);
        }
      }
      store_y<double, VEC>(Y + i * m + c, y);
    }
  }
}

int grid_for(const ens_matrix *A, int64_t groups_per_block_rows, const void *kernel) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (A->n + groups_per_block_rows - 1) / groups_per_block_rows;
  const int64_t full = (int64_t)A->num_sms * per_sm;
  return (int)(need < full ? need : full);
}

template <typename T, int VEC, int LANES>
cudaError_t run_plain(const ens_matrix *A, const T *val, int m, const T *X, T *Y, cudaStream_t s) {
  auto k = gspmv_plain<T, VEC, LANES>;
  const int grid = grid_for(A, kThreads / LANES, (const void *)k);
  k<<<grid, kThreads, 0, s>>>((int32_t)A->n, A->row, A->col, val, m, X, Y);
  return cudaGetLastError();
}

template <int VEC, int LANES>
cudaError_t run_split(const ens_matrix *A, int m, const double *X, double *Y, cudaStream_t s) {
  auto k = gspmv_split<VEC, LANES>;
  const int grid = grid_for(A, kThreads / LANES, (const void *)k);
  k<<<grid, kThreads, 0, s>>>((int32_t)A->n, A->row, A->col, A->valsplit, A->val, m, X, Y);
  return cudaGetLastError();
}

int pow2_at_least(int v, int cap) {
  int p = 1;
  while (p < v && p < cap) p <<= 1;
  return p;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Dispatch on (VEC, LANES). LANES is a power of two in [1, 32].
template <typename T, int VEC>
cudaError_t dispatch_plain(const ens_matrix *A, const T *val, int m, const T *X, T *Y, int lanes, cudaStream_t s) {
  switch (lanes) {
    case 1: return run_plain<T, VEC, 1>(A, val, m, X, Y, s);
    case 2: return run_plain<T, VEC, 2>(A, val, m, X, Y, s);
    case 4: return run_plain<T, VEC, 4>(A, val, m, X, Y, s);
    case 8: return run_plain<T, VEC, 8>(A, val, m, X, Y, s);
    case 16: return run_plain<T, VEC, 16>(A, val, m, X, Y, s);
    default: return run_plain<T, VEC, 32>(A, val, m, X, Y, s);
  }
}

template <int VEC>
cudaError_t dispatch_split(const ens_matrix *A, int m, const double *X, double *Y, int lanes, cudaStream_t s) {
  switch (lanes) {
    case 1: return run_split<VEC, 1>(A, m, X, Y, s);
    case 2: return run_split<VEC, 2>(A, m, X, Y, s);
    case 4: return run_split<VEC, 4>(A, m, X, Y, s);
    case 8: return run_split<VEC, 8>(A, m, X, Y, s);
    case 16: return run_split<VEC, 16>(A, m, X, Y, s);
    default: return run_split<VEC, 32>(A, m, X, Y, s);
  }
}

}  // namespace

// Rows longer than this use native FP64 (sums of split products must not overflow).
constexpr int32_t kSplitMaxRow = 64;

ens_status launch_gspmv(const ens_matrix *A, int m, int dtype, const void *X, void *Y, cudaStream_t s) {
  if (A->n == 0) return ENS_OK;
  cudaError_t e;
  if (dtype == ENS_F32) {
    const float *x = (const float *)X;
    float *y = (float *)Y;
    if (m % 4 == 0 && aligned(X, 16) && aligned(Y, 16))
      e = dispatch_plain<float, 4>(A, A->val32, m, x, y, pow2_at_least(m / 4, 8), s);
    else if (m % 2 == 0 && aligned(X, 8) && aligned(Y, 8))
      e = dispatch_plain<float, 2>(A, A->val32, m, x, y, pow2_at_least(m / 2, 16), s);
    else
      e = dispatch_plain<float, 1>(A, A->val32, m, x, y, pow2_at_least(m, 32), s);
  } else {
    const double *x = (const double *)X;
    double *y = (double *)Y;
    const bool vec2 = (m % 2 == 0) && aligned(X, 16) && aligned(Y, 16);
    const int lanes = vec2 ? pow2_at_least(m / 2, 16) : pow2_at_least(m, 32);
    const bool split = A->f64_mode != ENS_F64_NATIVE && A->split_ok && A->max_row_len <= kSplitMaxRow;
    if (split)
      e = vec2 ? dispatch_split<2>(A, m, x, y, lanes, s) : dispatch_split<1>(A, m, x, y, lanes, s);
    else
      e = vec2 ? dispatch_plain<double, 2>(A, A->val, m, x, y, lanes, s)
               : dispatch_plain<double, 1>(A, A->val, m, x, y, lanes, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "gspmv launch");
  return ENS_OK;
}

}  // namespace ens
