// Device building blocks of the GSpMV family: block-row loads/stores and the per-row product
//   y[q] = sum_{j = row_ptr[i]}^{row_ptr[i+1]-1} val[j] * X[col_idx[j]*m + c + q],  q < VEC
// (Section 2.3, Fig. GSpMV) in three arithmetics: float32, native float64 and split float64.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

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

// One access of a VEC-element vector: a single load or store of VEC elements, except for float64
// vectors wider than two, which move as VEC / 2 16-byte halves.
template <typename T, int VEC>
struct Access {
  using type = typename Vec<T, VEC>::type;
  static constexpr int n = VEC;
};
template <int VEC>
struct Access<double, VEC> {
  using type = typename Vec<double, (VEC > 1 ? 2 : 1)>::type;
  static constexpr int n = VEC > 1 ? 2 : 1;
};

// VEC consecutive elements starting at p (p aligned to the access width: VEC * sizeof(T), 16 bytes
// for float64 vectors of two or more).
template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T *__restrict__ p, T (&v)[VEC]) {
  using A = Access<T, VEC>;
  using V = typename A::type;
#pragma unroll
  for (int h = 0; h < VEC / A::n; ++h) {
    const V t = __ldg(reinterpret_cast<const V *>(p) + h);
    const T *e = reinterpret_cast<const T *>(&t);
#pragma unroll
    for (int q = 0; q < A::n; ++q) v[h * A::n + q] = e[q];
  }
}

// Same, for data written earlier in the same kernel launch by this thread (no read-only path).
template <typename T, int VEC>
__device__ __forceinline__ void load_vec_rw(const T *p, T (&v)[VEC]) {
  using A = Access<T, VEC>;
  using V = typename A::type;
#pragma unroll
  for (int h = 0; h < VEC / A::n; ++h) {
    const V t = reinterpret_cast<const V *>(p)[h];
    const T *e = reinterpret_cast<const T *>(&t);
#pragma unroll
    for (int q = 0; q < A::n; ++q) v[h * A::n + q] = e[q];
  }
}

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[VEC]) {
  using A = Access<T, VEC>;
  using V = typename A::type;
#pragma unroll
  for (int h = 0; h < VEC / A::n; ++h) {
    V t;
    T *e = reinterpret_cast<T *>(&t);
#pragma unroll
    for (int q = 0; q < A::n; ++q) e[q] = v[h * A::n + q];
    reinterpret_cast<V *>(p)[h] = t;
  }
}

// Streaming store (evict-first): for outputs written once and not re-read soon.
template <typename T, int VEC>
__device__ __forceinline__ void store_vec_cs(T *p, const T (&v)[VEC]) {
  using A = Access<T, VEC>;
  using V = typename A::type;
#pragma unroll
  for (int h = 0; h < VEC / A::n; ++h) {
    V t;
    T *e = reinterpret_cast<T *>(&t);
#pragma unroll
    for (int q = 0; q < A::n; ++q) e[q] = v[h * A::n + q];
    __stcs(reinterpret_cast<V *>(p) + h, t);
  }
}

constexpr int kUnroll = 4;

// ------------------------------------------------------------------ float32 / native float64
// ci/va point either into a shared-memory tile or into global memory; j0, j1 index them.
// Nonzeros are processed kUnroll at a time (all X loads of a group in flight together). For float
// data the last partial group is issued as one predicated group (a 7-nonzero row costs two L2
// round trips instead of four); for double data the extra registers of that form cost more
// occupancy than they save (measured on GB300: native m = 2, 129 us against 159 us), so the tail
// is processed one nonzero at a time.
template <typename T, typename V, int VEC>
__device__ __forceinline__ void row_plain(int32_t j0, int32_t j1, const int32_t *ci, const V *va, int32_t m,
                                          int32_t c, const T *__restrict__ X, T (&acc)[VEC]) {
  constexpr bool kGroupTail = sizeof(T) == 4;
  constexpr int U = kUnroll;
#pragma unroll
  for (int q = 0; q < VEC; ++q) acc[q] = T(0);
  int32_t j = j0;
  for (; j + U <= j1; j += U) {
    int32_t k[U];
    T a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      k[u] = ci[j + u];
      a[u] = (T)va[j + u];
    }
    T x[U][VEC];
#pragma unroll
    for (int u = 0; u < U; ++u) load_vec<T, VEC>(X + (int64_t)k[u] * m + c, x[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] = fma(a[u], x[u][q], acc[q]);
  }
  if (kGroupTail) {
    if (j < j1) {
      const int32_t len = j1 - j;
      int32_t k[U];
      T a[U];
      T x[U][VEC];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool v = u < len;
        k[u] = v ? ci[j + u] : 0;
        a[u] = v ? (T)va[j + u] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < len) {
          load_vec<T, VEC>(X + (int64_t)k[u] * m + c, x[u]);
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q) x[u][q] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < VEC; ++q)
          if (u < len) acc[q] = fma(a[u], x[u][q], acc[q]);
    }
  } else {
    for (; j < j1; ++j) {
      const int32_t k = ci[j];
      const T a = (T)va[j];
      T x[VEC];
      load_vec<T, VEC>(X + (int64_t)k * m + c, x);
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] = fma(a, x[q], acc[q]);
    }
  }
}

// ------------------------------------------------------------------ split float64
// GB300 executes FP64 arithmetic AND every float<->double conversion on a narrow FP64 pipe
// (2 DFMA per clock per SM against 128 FP32 lanes), so the split path issues no FP64 instruction
// per product: each double is cut into two floats with integer operations and one FP32 step.
//
// x = hi + lo + r with |r| < 2^-46 |x| (E = biased exponent of x):
//   hi: sign, exponent E - 896 and mantissa bits 51..29 of x (truncation). The funnel shift
//       (hw:lw) << 3 puts mantissa bits 51..29 in bits 22..0 and exponent bits 7..0 in bits
//       30..23. Bit 31 must be the sign and bit 30 the top bit of E - 896, which for E in
//       [896, 1151] is exponent bit 10 of x, i.e. bit 30 of hw: one bit select takes bits 31..30
//       from hw and bits 29..0 from the shifted word. x = +-0 gives hi = +-0.
//   lo: mantissa bits 28..6 of x, worth m_lo 2^(E-1069). G = 2^-23 (1 + m_lo 2^-23) is those
//       bits under a constant exponent, and lo = (G - 2^-23) P with P = sign(x) 2^(E-1023), the
//       sign and exponent bits of hi. The subtraction is exact (Sterbenz) and so is the scaling
//       by a power of two (no underflow inside the window below). x = +-0 gives lo = 0.
// The construction holds for E in [896, 1151]. A row segment takes the split path for a column
// when every x it reads has E in [kSplitELo, kSplitELo + 127] (|x| in [2^-40, 2^88)):
// split_range(x) is below kSplitWindow exactly for those, so one OR per element accumulates the
// test. Zeros, tiny, huge and non-finite values fail it and the segment is recomputed with native
// DFMA for that column.
constexpr uint32_t kSplitELo = 983u;
constexpr uint32_t kSplitWindow = 128u << 21;
constexpr int32_t kSplitMaxRow = 64;
constexpr uint32_t kSplitG = 0x34000000u;  // 2^-23

__device__ __forceinline__ uint32_t split_hi_bits(uint32_t hw, uint32_t lw) {
  return (__funnelshift_l(lw, hw, 3) & 0x3FFFFFFFu) | (hw & 0xC0000000u);
}
__device__ __forceinline__ uint32_t split_g_bits(uint32_t lw) { return ((lw >> 6) & 0x007FFFFFu) | kSplitG; }

__device__ __forceinline__ void split_f64(double x, float &hi, float &lo) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const uint32_t hb = split_hi_bits(hw, lw);
  hi = __uint_as_float(hb);
  lo = __fmul_rn(__fsub_rn(__uint_as_float(split_g_bits(lw)), __uint_as_float(kSplitG)),
                 __uint_as_float(hb & 0xFF800000u));
}

// (E - kSplitELo) << 21 plus the high mantissa bits, modulo 2^32 (the sign drops out).
__device__ __forceinline__ uint32_t split_range(double x) {
  return (uint32_t)__double2hiint(x) * 2u - (kSplitELo << 21);
}

// The matrix values are checked once (2^-40 <= |a| < 2^60, or a = 0), so every nonzero product
// has magnitude >= 2^-80 and its low part stays a normal float. Products of up to 2^148 can
// overflow the float range: the accumulators then hold Inf or NaN, which split_ok() catches.
__device__ __forceinline__ bool split_finite(float f) { return (__float_as_uint(f) & 0x7F800000u) != 0x7F800000u; }
__device__ __forceinline__ bool split_ok(uint32_t range_or, float hi, float lo) {
  return range_or < kSplitWindow && split_finite(hi) && split_finite(lo);
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

// Packed pairs of floats (f32x2): sm_100-class SMs execute FP32 add/mul/fma on two lanes per
// instruction, so the two columns a lane owns share every FP32 instruction of the split path.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Native DFMA row product (the split path's fallback and the FP64 share of hybrid tiles).
template <int VEC>
__device__ __forceinline__ void row_native_f64(int32_t j0, int32_t j1, const int32_t *ci, const double *__restrict__ vn,
                                               int32_t m, int32_t c, const double *__restrict__ X, double (&z)[VEC]) {
  row_plain<double, double, VEC>(j0, j1, ci, vn, m, c, X, z);
}

// Split-float row product. ci / vs (hi, lo pairs) are indexed by j in [j0, j1) and point into a
// shared-memory tile or into global memory; vn is the float64 value array under the same index
// (global), used when a column's X values leave the split range. Each column decides on its own,
// so one column's values never change another column's result.
template <int VEC>
__device__ __forceinline__ void row_split(int32_t j0, int32_t j1, const int32_t *ci, const float2 *vs,
                                          const double *__restrict__ vn, int32_t m, int32_t c,
                                          const double *__restrict__ X, double (&y)[VEC]) {
  float sh[VEC], sl[VEC];
  uint32_t rng[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    sh[q] = sl[q] = 0.f;
    rng[q] = 0u;
  }
  for (int32_t j = j0; j < j1; j += kUnroll) {
    const int32_t len = j1 - j;
    double x[kUnroll][VEC];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int32_t k = ci[u < len ? j + u : j];
      load_vec<double, VEC>(X + (int64_t)k * m + c, x[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (u < len) {
        const float2 a = vs[j + u];
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          float xh, xl;
          rng[q] |= split_range(x[u][q]);
          split_f64(x[u][q], xh, xl);
          split_fma(a.x, a.y, xh, xl, sh[q], sl[q]);
        }
      }
    }
  }
  bool ok[VEC], all_ok = true;
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    ok[q] = split_ok(rng[q], sh[q], sl[q]);
    y[q] = split_to_double(sh[q], sl[q]);
    all_ok &= ok[q];
  }
  if (!all_ok) {
    double z[VEC];
    row_native_f64<VEC>(j0, j1, ci, vn, m, c, X, z);
#pragma unroll
    for (int q = 0; q < VEC; ++q) y[q] = ok[q] ? y[q] : z[q];
  }
}

// Two columns per lane, packed f32x2 arithmetic. A nonzero's matrix value enters as the pairs
// AH = (ah, ah) and AL = (al, al), the X values as XH = (xh0, xh1) and XL = (xl0, xl1). Per nonzero:
//   PH = AH * XH (rounded), PL = AH*XH - PH (exact, one FMA against -PH) + AH*XL + AL*XH,
//   (SH, E) = TwoSum(SH, PH), SL += E + PL.
// Full groups of kUnroll nonzeros run without any predicate; the last 1..kUnroll-1 nonzeros run
// as one group whose missing entries re-read the group's first X row and carry a zero matrix
// value (an exact no-op: 0 * x adds +-0 to both accumulators; a non-finite x there is also in
// slot 0 and already fails the range test).
struct SplitPair {
  uint64_t ah, al;
};
__device__ __forceinline__ SplitPair split_pair(const float4 &v) { return {f2_pack(v.x, v.y), f2_pack(v.z, v.w)}; }
__device__ __forceinline__ SplitPair split_pair(const float2 &v) { return {f2_pack(v.x, v.x), f2_pack(v.y, v.y)}; }

__device__ __forceinline__ void split_acc2(const SplitPair &a, double x0, double x1, uint64_t g23, uint64_t &sh,
                                           uint64_t &sl, uint32_t &rng0, uint32_t &rng1) {
  const uint32_t hw0 = (uint32_t)__double2hiint(x0), lw0 = (uint32_t)__double2loint(x0);
  const uint32_t hw1 = (uint32_t)__double2hiint(x1), lw1 = (uint32_t)__double2loint(x1);
  rng0 |= split_range(x0);
  rng1 |= split_range(x1);
  const uint32_t hb0 = split_hi_bits(hw0, lw0), hb1 = split_hi_bits(hw1, lw1);
  const uint64_t xh = f2_pack(__uint_as_float(hb0), __uint_as_float(hb1));
  const uint64_t g = f2_pack(__uint_as_float(split_g_bits(lw0)), __uint_as_float(split_g_bits(lw1)));
  const uint64_t pw = f2_pack(__uint_as_float(hb0 & 0xFF800000u), __uint_as_float(hb1 & 0xFF800000u));
  const uint64_t xl = f2_mul(f2_sub(g, g23), pw);
  const uint64_t ph = f2_mul(a.ah, xh);
  // exact rounding error of ah*xh: fma(ah, xh, -ph), with -ph formed by flipping both sign bits.
  // (Forming -ph as the packed difference 0 - ph lost this error term on sm_103a in a GPU check
  // against the scalar form; the bit flip is exact and the result matches the scalar form.)
  uint64_t pl = f2_fma(a.ah, xh, ph ^ 0x8000000080000000ull);
  pl = f2_fma(a.ah, xl, pl);
  pl = f2_fma(a.al, xh, pl);
  const uint64_t s = f2_add(sh, ph);
  const uint64_t bb = f2_sub(s, sh);
  const uint64_t e = f2_add(f2_sub(sh, f2_sub(s, bb)), f2_sub(ph, bb));
  sh = s;
  sl = f2_add(sl, f2_add(e, pl));
}

// X row k at the lane's column offset: one wide multiply-add on byte offsets.
__device__ __forceinline__ const double2 *xrow(const char *xc, int32_t k, uint32_t row_bytes) {
  return reinterpret_cast<const double2 *>(xc + (uint64_t)(uint32_t)k * row_bytes);
}

template <typename AV>
__device__ __forceinline__ void row_split2(int32_t j0, int32_t j1, const int32_t *ci, const AV *va,
                                           const double *__restrict__ vn, int32_t m, int32_t c,
                                           const double *__restrict__ X, double (&y)[2]) {
  uint64_t sh = 0ull, sl = 0ull;
  uint32_t rng0 = 0u, rng1 = 0u;
  const uint64_t g23 = f2_pack(__uint_as_float(kSplitG), __uint_as_float(kSplitG));
  const char *xc = reinterpret_cast<const char *>(X + c);
  const uint32_t rb = (uint32_t)m * 8u;
  int32_t j = j0;
  for (; j + kUnroll <= j1; j += kUnroll) {
    double2 x[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) x[u] = __ldg(xrow(xc, ci[j + u], rb));
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) split_acc2(split_pair(va[j + u]), x[u].x, x[u].y, g23, sh, sl, rng0, rng1);
  }
  if (j < j1) {
    const int32_t len = j1 - j;
    double2 x[kUnroll - 1];
    SplitPair a[kUnroll - 1];
#pragma unroll
    for (int u = 0; u < kUnroll - 1; ++u) {
      const bool v = u < len;
      const int32_t jj = v ? j + u : j;
      x[u] = __ldg(xrow(xc, ci[jj], rb));
      a[u] = split_pair(va[jj]);
      if (!v) a[u] = SplitPair{0ull, 0ull};
    }
#pragma unroll
    for (int u = 0; u < kUnroll - 1; ++u) split_acc2(a[u], x[u].x, x[u].y, g23, sh, sl, rng0, rng1);
  }
  float h0, h1, l0, l1;
  f2_unpack(sh, h0, h1);
  f2_unpack(sl, l0, l1);
  const bool ok0 = split_ok(rng0, h0, l0), ok1 = split_ok(rng1, h1, l1);
  y[0] = split_to_double(h0, l0);
  y[1] = split_to_double(h1, l1);
  if (!(ok0 && ok1)) {
    double z[2];
    row_native_f64<2>(j0, j1, ci, vn, m, c, X, z);
    y[0] = ok0 ? y[0] : z[0];
    y[1] = ok1 ? y[1] : z[1];
  }
}

// Four or more columns per lane: NP packed pairs of row_split2 share each nonzero's column index
// and matrix pair; gathers of kUnroll / NP nonzeros (NP 16-byte pieces each) are issued together.
// The kernels use NP = 2 (eight columns per lane, NP = 4, needs 64-80 registers, spills, and was
// 15-20 % slower on GB300).
template <int NP, typename AV>
__device__ __forceinline__ void row_split_pairs(int32_t j0, int32_t j1, const int32_t *ci, const AV *va,
                                                const double *__restrict__ vn, int32_t m, int32_t c,
                                                const double *__restrict__ X, double (&y)[2 * NP]) {
  constexpr int G = kUnroll / NP > 1 ? kUnroll / NP : 1;
  uint64_t sh[NP], sl[NP];
  uint32_t rng[2 * NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    sh[p] = sl[p] = 0ull;
    rng[2 * p] = rng[2 * p + 1] = 0u;
  }
  const uint64_t g23 = f2_pack(__uint_as_float(kSplitG), __uint_as_float(kSplitG));
  const char *xc = reinterpret_cast<const char *>(X + c);
  const uint32_t rb = (uint32_t)m * 8u;
  int32_t j = j0;
  for (; j + G <= j1; j += G) {
    double2 x[G][NP];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const double2 *px = xrow(xc, ci[j + u], rb);
#pragma unroll
      for (int p = 0; p < NP; ++p) x[u][p] = __ldg(px + p);
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const SplitPair a = split_pair(va[j + u]);
#pragma unroll
      for (int p = 0; p < NP; ++p) split_acc2(a, x[u][p].x, x[u][p].y, g23, sh[p], sl[p], rng[2 * p], rng[2 * p + 1]);
    }
  }
  auto one = [&](int32_t jj) {
    const double2 *px = xrow(xc, ci[jj], rb);
    double2 x[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) x[p] = __ldg(px + p);
    const SplitPair a = split_pair(va[jj]);
#pragma unroll
    for (int p = 0; p < NP; ++p) split_acc2(a, x[p].x, x[p].y, g23, sh[p], sl[p], rng[2 * p], rng[2 * p + 1]);
  };
  if constexpr (G == 2) {  // the last 1..G-1 nonzeros
    if (j < j1) one(j);
  } else if constexpr (G > 2) {
    for (; j < j1; ++j) one(j);
  }
  float h[2 * NP], l[2 * NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    f2_unpack(sh[p], h[2 * p], h[2 * p + 1]);
    f2_unpack(sl[p], l[2 * p], l[2 * p + 1]);
  }
  bool ok[2 * NP], all_ok = true;
#pragma unroll
  for (int q = 0; q < 2 * NP; ++q) {
    ok[q] = split_ok(rng[q], h[q], l[q]);
    y[q] = split_to_double(h[q], l[q]);
    all_ok &= ok[q];
  }
  if (!all_ok) {
    double z[2 * NP];
    row_native_f64<2 * NP>(j0, j1, ci, vn, m, c, X, z);
#pragma unroll
    for (int q = 0; q < 2 * NP; ++q) y[q] = ok[q] ? y[q] : z[q];
  }
}

// ------------------------------------------------------------------ row tiles (shared memory)
constexpr int kTileRows = 256;
constexpr int kTileNnz = 2048;
constexpr int kCsrPad = 4;  // extra elements allocated after row_ptr, col_idx and every value array

template <typename V>
struct TileSmem {
  int32_t ci[kTileNnz];
  V va[kTileNnz];
};

// Asynchronous 16-byte global -> shared copies (per thread, completion by cp.async.wait_all, which
// waits only for this thread's own copies: no spin loop is involved).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename E>
__device__ __forceinline__ void stage16_async(E *dst, const E *src, int32_t count) {
  // count elements, count * sizeof(E) a multiple of 16, src and dst 16-byte aligned
  const int32_t n16 = count * (int32_t)sizeof(E) / 16;
  for (int32_t t = threadIdx.x; t < n16; t += blockDim.x)
    cp_async16(reinterpret_cast<int4 *>(dst) + t, reinterpret_cast<const int4 *>(src) + t);
}

template <typename E>
__device__ __forceinline__ void stage16(E *dst, const E *__restrict__ src, int32_t count) {
  // count elements, count * sizeof(E) a multiple of 16, src and dst 16-byte aligned
  const int32_t n16 = count * (int32_t)sizeof(E) / 16;
  const int4 *s = reinterpret_cast<const int4 *>(src);
  int4 *d = reinterpret_cast<int4 *>(dst);
  for (int32_t t = threadIdx.x; t < n16; t += blockDim.x) d[t] = __ldcs(s + t);
}

// ------------------------------------------------------------------ column-hybrid float64
// Each lane owns two columns: the first is computed with native DFMA, the second with split-float
// arithmetic, in the same instruction stream. The FP64 pipe and the FP32/integer pipes then work
// at the same time on every warp instead of taking turns. Column 1 falls back to DFMA when its X
// values leave the split range (decided for that column alone).
template <int VEC>
__device__ __forceinline__ void row_hybrid(int32_t j0, int32_t j1, const int32_t *ci, const double *vd,
                                           const float2 *vs, int32_t m, int32_t c, const double *__restrict__ X,
                                           double (&y)[VEC]);
template <>
__device__ __forceinline__ void row_hybrid<2>(int32_t j0, int32_t j1, const int32_t *ci, const double *vd,
                                              const float2 *vs, int32_t m, int32_t c, const double *__restrict__ X,
                                              double (&y)[2]) {
  double acc = 0.0;
  float sh = 0.f, sl = 0.f;
  uint32_t rng = 0u;
  for (int32_t j = j0; j < j1; j += kUnroll) {
    const int32_t len = j1 - j;
    double x[kUnroll][2];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int32_t k = ci[u < len ? j + u : j];
      load_vec<double, 2>(X + (int64_t)k * m + c, x[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (u < len) {
        acc = fma(vd[j + u], x[u][0], acc);
        float xh, xl;
        rng |= split_range(x[u][1]);
        split_f64(x[u][1], xh, xl);
        const float2 a = vs[j + u];
        split_fma(a.x, a.y, xh, xl, sh, sl);
      }
    }
  }
  y[0] = acc;
  y[1] = split_to_double(sh, sl);
  if (!split_ok(rng, sh, sl)) {
    double z = 0.0;
    for (int32_t jj = j0; jj < j1; ++jj) z = fma(vd[jj], __ldg(X + (int64_t)ci[jj] * m + c + 1), z);
    y[1] = z;
  }
}
template <>
__device__ __forceinline__ void row_hybrid<1>(int32_t j0, int32_t j1, const int32_t *ci, const double *vd,
                                              const float2 *, int32_t m, int32_t c, const double *__restrict__ X,
                                              double (&y)[1]) {
  row_plain<double, double, 1>(j0, j1, ci, vd, m, c, X, y);
}

// ------------------------------------------------------------------ arithmetic policies
// T: element type of X and Y. Tile: the shared-memory layout of a staged row tile. stage() copies
// the tile's CSR segment [ab, ae) (16-byte rounded) into it; row_s() computes one row segment
// from the tile, row_g() from global memory (tiles whose segment does not fit). `native` forces
// DFMA for the sweep (split arithmetic with a native share).
struct ArithF32 {
  using T = float;
  using Tile = TileSmem<float>;
  __device__ __forceinline__ static void stage(Tile &sm, const MatView &A, int32_t ab, int32_t ae) {
    stage16<int32_t>(sm.ci, A.ci + ab, ae - ab);
    stage16<float>(sm.va, A.val32 + ab, ae - ab);
  }
  template <int VEC>
  __device__ __forceinline__ static void row_s(const Tile &sm, const MatView &, int32_t, int32_t j0, int32_t j1,
                                               int32_t m, int32_t c, const float *X, float (&y)[VEC], bool) {
    row_plain<float, float, VEC>(j0, j1, sm.ci, sm.va, m, c, X, y);
  }
  template <int VEC>
  __device__ __forceinline__ static void row_g(const MatView &A, int32_t ab, int32_t j0, int32_t j1, int32_t m,
                                               int32_t c, const float *X, float (&y)[VEC], bool) {
    row_plain<float, float, VEC>(j0, j1, A.ci + ab, A.val32 + ab, m, c, X, y);
  }
  __device__ __forceinline__ static float dinv(const MatView &A, int64_t i) { return __ldg(A.dinv32 + i); }
};
struct ArithF64Native {
  using T = double;
  using Tile = TileSmem<double>;
  __device__ __forceinline__ static void stage(Tile &sm, const MatView &A, int32_t ab, int32_t ae) {
    stage16<int32_t>(sm.ci, A.ci + ab, ae - ab);
    stage16<double>(sm.va, A.val + ab, ae - ab);
  }
  template <int VEC>
  __device__ __forceinline__ static void row_s(const Tile &sm, const MatView &, int32_t, int32_t j0, int32_t j1,
                                               int32_t m, int32_t c, const double *X, double (&y)[VEC], bool) {
    row_plain<double, double, VEC>(j0, j1, sm.ci, sm.va, m, c, X, y);
  }
  template <int VEC>
  __device__ __forceinline__ static void row_g(const MatView &A, int32_t ab, int32_t j0, int32_t j1, int32_t m,
                                               int32_t c, const double *X, double (&y)[VEC], bool) {
    row_plain<double, double, VEC>(j0, j1, A.ci + ab, A.val + ab, m, c, X, y);
  }
  __device__ __forceinline__ static double dinv(const MatView &A, int64_t i) { return __ldg(A.dinv + i); }
};
// The split tile keeps the (ah, al) pairs (8 bytes per value); the packed operand pairs are formed
// in registers. A tile of (ah, ah, al, al) entries saves those moves but doubles the tile's shared
// memory, and the occupancy it costs is worth more (measured on GB300: 1042 against 1030 us at
// m = 32, 314 against 290 us at m = 8).
struct ArithF64Split {
  using T = double;
  using Tile = TileSmem<float2>;
  __device__ __forceinline__ static void stage(Tile &sm, const MatView &A, int32_t ab, int32_t ae) {
    stage16<int32_t>(sm.ci, A.ci + ab, ae - ab);
    stage16<float2>(sm.va, A.vs + ab, ae - ab);
  }
  template <int VEC>
  __device__ __forceinline__ static void row_s(const Tile &sm, const MatView &A, int32_t ab, int32_t j0, int32_t j1,
                                               int32_t m, int32_t c, const double *X, double (&y)[VEC], bool native) {
    if (native) {
      row_native_f64<VEC>(j0, j1, sm.ci, A.val + ab, m, c, X, y);
    } else if constexpr (VEC == 2) {
      row_split2<float2>(j0, j1, sm.ci, sm.va, A.val + ab, m, c, X, y);
    } else if constexpr (VEC == 4) {
      row_split_pairs<2, float2>(j0, j1, sm.ci, sm.va, A.val + ab, m, c, X, y);
    } else {
      row_split<VEC>(j0, j1, sm.ci, A.vs + ab, A.val + ab, m, c, X, y);
    }
  }
  template <int VEC>
  __device__ __forceinline__ static void row_g(const MatView &A, int32_t ab, int32_t j0, int32_t j1, int32_t m,
                                               int32_t c, const double *X, double (&y)[VEC], bool native) {
    if (native) {
      row_native_f64<VEC>(j0, j1, A.ci + ab, A.val + ab, m, c, X, y);
    } else if constexpr (VEC == 2) {
      row_split2<float2>(j0, j1, A.ci + ab, A.vs + ab, A.val + ab, m, c, X, y);
    } else if constexpr (VEC == 4) {
      row_split_pairs<2, float2>(j0, j1, A.ci + ab, A.vs + ab, A.val + ab, m, c, X, y);
    } else {
      row_split<VEC>(j0, j1, A.ci + ab, A.vs + ab, A.val + ab, m, c, X, y);
    }
  }
  __device__ __forceinline__ static double dinv(const MatView &A, int64_t i) { return __ldg(A.dinv + i); }
};
// Column hybrid: the tile holds the float64 values and their (hi, lo) split, computed once per
// staged value (amortised over all lanes of the tile); only the float64 array is read from HBM.
struct HybridTile {
  int32_t ci[kTileNnz];
  double vd[kTileNnz];
  float2 vs[kTileNnz];
};
struct ArithF64Hybrid {
  using T = double;
  using Tile = HybridTile;
  __device__ __forceinline__ static void stage(Tile &sm, const MatView &A, int32_t ab, int32_t ae) {
    stage16<int32_t>(sm.ci, A.ci + ab, ae - ab);
    const int32_t n16 = (ae - ab) / 2;  // two doubles per 16 bytes
    const int4 *src = reinterpret_cast<const int4 *>(A.val + ab);
    for (int32_t t = threadIdx.x; t < n16; t += blockDim.x) {
      const int4 q = __ldcs(src + t);
      reinterpret_cast<int4 *>(sm.vd)[t] = q;
      const double v0 = __hiloint2double(q.y, q.x), v1 = __hiloint2double(q.w, q.z);
      float h0, l0, h1, l1;
      split_f64(v0, h0, l0);  // matrix values are inside the split range (checked at creation)
      split_f64(v1, h1, l1);
      reinterpret_cast<float4 *>(sm.vs)[t] = make_float4(h0, l0, h1, l1);
    }
  }
  template <int VEC>
  __device__ __forceinline__ static void row_s(const Tile &sm, const MatView &, int32_t, int32_t j0, int32_t j1,
                                               int32_t m, int32_t c, const double *X, double (&y)[VEC], bool) {
    row_hybrid<VEC>(j0, j1, sm.ci, sm.vd, sm.vs, m, c, X, y);
  }
  template <int VEC>
  __device__ __forceinline__ static void row_g(const MatView &A, int32_t ab, int32_t j0, int32_t j1, int32_t m,
                                               int32_t c, const double *X, double (&y)[VEC], bool) {
    row_native_f64<VEC>(j0, j1, A.ci + ab, A.val + ab, m, c, X, y);
  }
  __device__ __forceinline__ static double dinv(const MatView &A, int64_t i) { return __ldg(A.dinv + i); }
};

// A block walks tiles of kTileRows consecutive rows (grid-stride). For each tile it stages the
// row pointers and the tile's contiguous CSR segment (column indices and values) in shared
// memory with 16-byte coalesced loads (the arrays are padded so the rounded-out segment stays
// inside them), then each row group of LANES threads computes rows g, g + G, g + 2G, ... of the
// tile from shared memory and hands each (row, column chunk) result to the epilogue. A tile
// whose segment exceeds kTileNnz is computed from global memory instead. native_mask bit
// (s & 31) sends row sweep s (counted over all tiles) to native DFMA (split arithmetic only), so the
// FP64 pipe takes a share of the products while the FP32/integer pipes take the rest.

// Visits the (row, column chunk) pairs of this thread in exactly the order tile_rows does, without
// any product: kernels that skip the GSpMV (a zero initial guess) reduce in the same order as the
// kernels that perform it, so both give the same bits.
template <int VEC, int LANES, typename Fn>
__device__ __forceinline__ void tile_order_rows(int64_t n, int32_t m, Fn &&fn) {
  constexpr int G = 256 / LANES;
  constexpr int RPG = kTileRows / G;
  const int lane = threadIdx.x % LANES, grp = threadIdx.x / LANES;
  for (int64_t r0 = (int64_t)blockIdx.x * kTileRows; r0 < n; r0 += (int64_t)gridDim.x * kTileRows) {
    const int rows = (int)min((int64_t)kTileRows, n - r0);
    for (int rr = 0; rr < RPG; ++rr) {
      const int lr = rr * G + grp;
      if (lr >= rows) break;
      for (int32_t c = lane * VEC; c < m; c += LANES * VEC) fn(r0 + lr, c);
    }
  }
}

template <typename Arith, int VEC, int LANES, typename Epi>
__device__ __forceinline__ void tile_rows(const MatView &A, int32_t m, const typename Arith::T *__restrict__ X,
                                          uint32_t native_mask, Epi &&epi) {
  using T = typename Arith::T;
  constexpr int kThr = 256;
  constexpr int G = kThr / LANES;
  constexpr int RPG = kTileRows / G;
  // Row pointers of the current tile and of the next one: the next tile's are copied asynchronously
  // while the current tile is computed, so each tile waits for one memory round trip (its CSR
  // segment) instead of two (row pointers, then the segment they delimit). Measured on GB300:
  // m = 1 91 us against 101, split m = 8 260 against 268, float32 m = 4 77 against 83. The float32
  // four-column kernels with 4 or more lanes per row run at 32 registers, where the prefetch's loop
  // state spills (m = 32: 350 against 298 us); they stage the row pointers in the loop instead.
  constexpr bool kPrefetch = !(std::is_same<Arith, ArithF32>::value && VEC == 4 && LANES >= 4);
  __shared__ __align__(16) typename Arith::Tile sm;
  __shared__ __align__(16) int32_t rpb[kPrefetch ? 2 : 1][kTileRows + 4];
  const int lane = threadIdx.x % LANES, grp = threadIdx.x / LANES;
  int64_t r0 = (int64_t)blockIdx.x * kTileRows;
  if constexpr (kPrefetch) {
    if (r0 < A.n) stage16<int32_t>(rpb[0], A.rp + r0, ((int)min((int64_t)kTileRows, (int64_t)A.n - r0) + 1 + 3) & ~3);
    __syncthreads();
  }
  for (int cur = 0; r0 < A.n; r0 += (int64_t)gridDim.x * kTileRows, cur ^= kPrefetch ? 1 : 0) {
    const int rows = (int)min((int64_t)kTileRows, (int64_t)A.n - r0);
    const int32_t *rp = rpb[cur];
    if constexpr (!kPrefetch) {
      stage16<int32_t>(rpb[0], A.rp + r0, (rows + 1 + 3) & ~3);
      __syncthreads();
    }
    const int32_t ab = rp[0] & ~3, ae = (rp[rows] + 3) & ~3;
    const bool staged = ae - ab <= kTileNnz;
    if (staged) Arith::stage(sm, A, ab, ae);
    if constexpr (kPrefetch) {
      const int64_t r1 = r0 + (int64_t)gridDim.x * kTileRows;
      if (r1 < A.n) {
        stage16_async<int32_t>(rpb[cur ^ 1], A.rp + r1, ((int)min((int64_t)kTileRows, (int64_t)A.n - r1) + 1 + 3) & ~3);
        cp_async_commit();
      }
    }
    __syncthreads();
    // sweep counter: spreads native_mask over tiles; the per-warp rotation keeps warps of one SM in
    // different phases so the FP64 pipe (native sweeps) and the FP32/integer pipes (split sweeps)
    // work at the same time
    const uint32_t sweep0 = (uint32_t)(r0 / kTileRows) * RPG + (threadIdx.x >> 5) * 5u + blockIdx.x;
    if (staged) {
#pragma unroll 1
      for (int rr = 0; rr < RPG; ++rr) {
        const int lr = rr * G + grp;
        if (lr >= rows) break;
        const int32_t j0 = rp[lr] - ab, j1 = rp[lr + 1] - ab;
        const bool nat = (native_mask >> ((sweep0 + rr) & 31)) & 1u;
        for (int32_t c = lane * VEC; c < m; c += LANES * VEC) {
          T y[VEC];
          Arith::template row_s<VEC>(sm, A, ab, j0, j1, m, c, X, y, nat);
          epi(r0 + lr, c, y);
        }
      }
    } else {
#pragma unroll 1
      for (int rr = 0; rr < RPG; ++rr) {
        const int lr = rr * G + grp;
        if (lr >= rows) break;
        const int32_t j0 = rp[lr] - ab, j1 = rp[lr + 1] - ab;
        const bool nat = (native_mask >> ((sweep0 + rr) & 31)) & 1u;
        for (int32_t c = lane * VEC; c < m; c += LANES * VEC) {
          T y[VEC];
          Arith::template row_g<VEC>(A, ab, j0, j1, m, c, X, y, nat);
          epi(r0 + lr, c, y);
        }
      }
    }
    if constexpr (kPrefetch) cp_async_wait_all();
    __syncthreads();
  }
}

// Rows straight from global memory, without a shared-memory tile and without block barriers: row
// group g of the grid takes rows g, g + groups, g + 2 groups, ... (consecutive groups, consecutive
// rows); the lanes of a group read the row's column indices and values through L1 at the same
// addresses. The native-DFMA rows of the split arithmetic are spread by the row index as the
// tiled kernel spreads its sweeps.
template <typename Arith, int VEC, int LANES, typename Epi>
__device__ __forceinline__ void direct_rows(const MatView &A, int32_t m, const typename Arith::T *__restrict__ X,
                                            uint32_t native_mask, Epi &&epi) {
  using T = typename Arith::T;
  constexpr int G = 256 / LANES;
  const int lane = threadIdx.x % LANES;
  const int64_t groups = (int64_t)gridDim.x * G;
  const uint32_t rot = (threadIdx.x >> 5) * 5u + blockIdx.x;
  for (int64_t i = (int64_t)blockIdx.x * G + threadIdx.x / LANES; i < A.n; i += groups) {
    const int32_t j0 = __ldg(A.rp + i), j1 = __ldg(A.rp + i + 1);
    const bool nat = (native_mask >> (((uint32_t)i + rot) & 31u)) & 1u;
    for (int32_t c = lane * VEC; c < m; c += LANES * VEC) {
      T y[VEC];
      Arith::template row_g<VEC>(A, 0, j0, j1, m, c, X, y, nat);
      epi(i, c, y);
    }
  }
}

}  // namespace ens
