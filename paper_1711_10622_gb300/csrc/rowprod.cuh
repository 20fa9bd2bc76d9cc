// Device building blocks of the GSpMV family: block-row loads/stores and the per-row product
//   y[q] = sum_{j = row_ptr[i]}^{row_ptr[i+1]-1} val[j] * X[col_idx[j]*m + c + q],  q < VEC
// (Section 2.3, Fig. GSpMV) in three arithmetics: float32, native float64 and split float64.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ens {

// Read-only view of a device CSR matrix and its derived arrays, passed to kernels by value.
struct MatView {
  int32_t n;
  const int32_t *__restrict__ rp;
  const int32_t *__restrict__ ci;
  const double *__restrict__ val;
  const float *__restrict__ val32;
  const float2 *__restrict__ vs;
  const double *__restrict__ dinv;
  const float *__restrict__ dinv32;
};

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

// VEC consecutive elements starting at p (p aligned to VEC * sizeof(T)).
template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T *__restrict__ p, T (&v)[VEC]) {
  using V = typename Vec<T, VEC>::type;
  const V t = __ldg(reinterpret_cast<const V *>(p));
  const T *e = reinterpret_cast<const T *>(&t);
#pragma unroll
  for (int q = 0; q < VEC; ++q) v[q] = e[q];
}

// Same, for data written earlier in the same kernel launch by this thread (no read-only path).
template <typename T, int VEC>
__device__ __forceinline__ void load_vec_rw(const T *p, T (&v)[VEC]) {
  using V = typename Vec<T, VEC>::type;
  const V t = *reinterpret_cast<const V *>(p);
  const T *e = reinterpret_cast<const T *>(&t);
#pragma unroll
  for (int q = 0; q < VEC; ++q) v[q] = e[q];
}

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[VEC]) {
  using V = typename Vec<T, VEC>::type;
  V t;
  T *e = reinterpret_cast<T *>(&t);
#pragma unroll
  for (int q = 0; q < VEC; ++q) e[q] = v[q];
  *reinterpret_cast<V *>(p) = t;
}

// Streaming store (evict-first): for outputs written once and not re-read soon.
template <typename T, int VEC>
__device__ __forceinline__ void store_vec_cs(T *p, const T (&v)[VEC]) {
  using V = typename Vec<T, VEC>::type;
  V t;
  T *e = reinterpret_cast<T *>(&t);
#pragma unroll
  for (int q = 0; q < VEC; ++q) e[q] = v[q];
  __stcs(reinterpret_cast<V *>(p), t);
}

constexpr int kUnroll = 4;

// ------------------------------------------------------------------ float32 / native float64
template <typename T, int VEC>
__device__ __forceinline__ void row_plain(int32_t j0, int32_t j1, const int32_t *__restrict__ ci,
                                          const T *__restrict__ va, int32_t m, int32_t c,
                                          const T *__restrict__ X, T (&acc)[VEC]) {
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
    for (int u = 0; u < kUnroll; ++u) load_vec<T, VEC>(X + (int64_t)k[u] * m + c, x[u]);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] = fma(a[u], x[u][q], acc[q]);
  }
  for (; j < j1; ++j) {
    const int32_t k = __ldcs(ci + j);
    const T a = __ldcs(va + j);
    T x[VEC];
    load_vec<T, VEC>(X + (int64_t)k * m + c, x);
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = fma(a, x[q], acc[q]);
  }
}

// ------------------------------------------------------------------ split float64
// GB300 executes FP64 arithmetic AND every float<->double conversion on a narrow FP64 pipe
// (a few operations per clock per SM against ~250 FP32 FMAs), so the split path touches no
// FP64 instruction per product: the double is cut into floats with integer operations only.
//
// x = hi + lo: hi takes the sign, the exponent and mantissa bits 51..29 of x (truncation), lo the
// next 23 bits exactly (bits 5..0 of the 52-bit mantissa are dropped: |x - hi - lo| < 2^-46 |x|).
//   hi: the funnel shift (hw:lw) << 3 puts mantissa bits 51..29 in place and the low 8 bits of
//       the 11-bit exponent E in bits 30..23; E - 896 (the float bias shift) equals those 8 bits
//       with bit 7 flipped for E in [896, 1151]; the sign is copied.
//   lo: lo = F - P with P = sign(x) 2^(e-23) (float exponent of hi minus 23) and F = P carrying
//       mantissa bits 28..6 of x; the subtraction is exact.
// Valid for +-0 and for biased exponents E in [kSplitELo, kSplitEHi] (|x| in [2^-40, 2^60)); the
// function returns false outside that range (tiny, huge, Inf, NaN) and the caller recomputes the
// row segment with native DFMA. Zero gets hi = 0 explicitly (the exponent rebias would otherwise
// turn it into 2.0); its lo is then F - P = 0 by construction.
constexpr uint32_t kSplitELo = 983u, kSplitEHi = 1082u;
constexpr int32_t kSplitMaxRow = 64;

__device__ __forceinline__ bool split_f64(double x, float &hi, float &lo) {
  const uint32_t hw = (uint32_t)__double2hiint(x);
  const uint32_t lw = (uint32_t)__double2loint(x);
  const bool zero = ((hw & 0x7FFFFFFFu) | lw) == 0u;
  const uint32_t fb = __funnelshift_l(lw, hw, 3);
  const uint32_t hb = zero ? 0u : (((fb & 0x7FFFFFFFu) ^ 0x40000000u) | (hw & 0x80000000u));
  const uint32_t pb = (hb & 0xFF800000u) - (23u << 23);
  hi = __uint_as_float(hb);
  lo = __fsub_rn(__uint_as_float(pb | ((lw >> 6) & 0x7FFFFFu)), __uint_as_float(pb));
  return zero || ((hw & 0x7FF00000u) - (kSplitELo << 20)) <= ((kSplitEHi - kSplitELo) << 20);
}

// With |x| and |val| in [2^-40, 2^60) (val checked once per matrix, zeros allowed) every nonzero
// product lies in [2^-80, 2^120): its low parts stay normal floats (or fall below 2^-126, i.e.
// 2^-46 of the smallest product, where flushing them is harmless), and a sum of at most
// kSplitMaxRow products stays below 2^127.

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

// Exact float -> double widening with integer operations (zero and subnormal floats give 0).
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t mag = b & 0x7FFFFFFFu;
  const bool normal = mag >= 0x00800000u;
  const uint32_t hi = (b & 0x80000000u) | (normal ? (mag >> 3) + (896u << 20) : 0u);
  const uint32_t lo = normal ? (mag << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}

// One double addition of the exactly widened parts (the only FP64 instruction per output).
__device__ __forceinline__ double split_to_double(float hi, float lo) { return widen_f32(hi) + widen_f32(lo); }

// Each column decides on its own whether its split result is valid, so the value of one column
// never depends on the values of the others (a column solved alone or inside a block gives the
// same bits).
template <int VEC>
__device__ __forceinline__ void row_split(int32_t j0, int32_t j1, const int32_t *__restrict__ ci,
                                          const float2 *__restrict__ vs, const double *__restrict__ va,
                                          int32_t m, int32_t c, const double *__restrict__ X,
                                          double (&y)[VEC]) {
  float sh[VEC], sl[VEC];
  bool ok[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    sh[q] = sl[q] = 0.f;
    ok[q] = true;
  }
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
    for (int u = 0; u < kUnroll; ++u) load_vec<double, VEC>(X + (int64_t)k[u] * m + c, x[u]);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        float xh, xl;
        ok[q] &= split_f64(x[u][q], xh, xl);
        split_fma(a[u].x, a[u].y, xh, xl, sh[q], sl[q]);
      }
  }
  for (; j < j1; ++j) {
    const int32_t k = __ldcs(ci + j);
    const float2 a = __ldcs(vs + j);
    double x[VEC];
    load_vec<double, VEC>(X + (int64_t)k * m + c, x);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      float xh, xl;
      ok[q] &= split_f64(x[q], xh, xl);
      split_fma(a.x, a.y, xh, xl, sh[q], sl[q]);
    }
  }
  bool all_ok = true;
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    y[q] = split_to_double(sh[q], sl[q]);
    all_ok &= ok[q];
  }
  if (!all_ok) {  // values outside the split range: native FP64 for the affected columns
    double z[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) z[q] = 0.0;
    for (int32_t jj = j0; jj < j1; ++jj) {
      const double av = __ldg(va + jj);
      double x[VEC];
      load_vec<double, VEC>(X + (int64_t)__ldg(ci + jj) * m + c, x);
#pragma unroll
      for (int q = 0; q < VEC; ++q) z[q] = fma(av, x[q], z[q]);
    }
#pragma unroll
    for (int q = 0; q < VEC; ++q) y[q] = ok[q] ? y[q] : z[q];
  }
}

// Arithmetic selectors for kernels templated on the product variant.
struct ArithF32 {
  using T = float;
  template <int VEC>
  __device__ __forceinline__ static void row(const MatView &A, int64_t i, int32_t m, int32_t c, const float *X, float (&y)[VEC]) {
    row_plain<float, VEC>(__ldg(A.rp + i), __ldg(A.rp + i + 1), A.ci, A.val32, m, c, X, y);
  }
  __device__ __forceinline__ static float dinv(const MatView &A, int64_t i) { return __ldg(A.dinv32 + i); }
};
struct ArithF64Native {
  using T = double;
  template <int VEC>
  __device__ __forceinline__ static void row(const MatView &A, int64_t i, int32_t m, int32_t c, const double *X, double (&y)[VEC]) {
    row_plain<double, VEC>(__ldg(A.rp + i), __ldg(A.rp + i + 1), A.ci, A.val, m, c, X, y);
  }
  __device__ __forceinline__ static double dinv(const MatView &A, int64_t i) { return __ldg(A.dinv + i); }
};
struct ArithF64Split {
  using T = double;
  template <int VEC>
  __device__ __forceinline__ static void row(const MatView &A, int64_t i, int32_t m, int32_t c, const double *X, double (&y)[VEC]) {
    row_split<VEC>(__ldg(A.rp + i), __ldg(A.rp + i + 1), A.ci, A.vs, A.val, m, c, X, y);
  }
  __device__ __forceinline__ static double dinv(const MatView &A, int64_t i) { return __ldg(A.dinv + i); }
};

}  // namespace ens
