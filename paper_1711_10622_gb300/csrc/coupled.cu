// Coupled block-Krylov solve: block BiCGStab on all m columns at once (ens_solve_block_coupled).
//
// The solver of solver_impl.cuh runs m independent recurrences that share each GSpMV. This one
// builds a single Krylov space from the m columns (Guennouni, Jbilou and Sadok 2003): the step
// lengths alpha and beta are m x m matrices and every column's update mixes all columns, with one
// Frobenius step omega per block. Per iteration, with right preconditioning:
//   P^ = M^-1 P, V = A P^; G = R~^T V, H = R~^T R      -> alpha = G^-1 H   (host LU, m x m)
//   S = R - V alpha; S^ = M^-1 S, T = A S^; ||S_l||^2, <T, S>_F, <T, T>_F -> omega
//   X += P^ alpha + omega S^;  R = S - omega T;  ||R_l||^2, F = R~^T T     -> beta = -G^-1 F
//   P = R + P beta - omega V beta
// Device work: the GSpMV and the preconditioner (Chebyshev polynomial or the aggregation V-cycle)
// of the main solver on every column of the block, a block Gram kernel (U^T [W1 W2], fixed
// summation order), a block update kernel (Y = Z0 + sum_t Z_t M_t with m x m matrices M_t) and the
// per-column dots. The m x m factorisations run on the host (three small synchronisations per
// iteration). Gram products and updates cost O(n m^2) multiply-adds per iteration; on the split path
// they run as split-float products on the FP32 pipe (GB300's FP64 pipe is narrow), otherwise as
// native DFMA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "ensemble_dist.h"
#include "partials.cuh"
#include "solver_impl.cuh"

namespace ens {
namespace coupled {

using solver::Scratch;

constexpr int kMaxCoupledM = 32;
constexpr int kGramRows = 16;  // rows of U and W staged per step of the Gram kernel

// Pass 1 of C (k x q) = U^T [W1 | W2] (q = q1 + q2): each block sums its rows in order, staged in
// shared memory kGramRows at a time; thread t owns entries t, t + 256, ... (row-major i * q + j).
__global__ void __launch_bounds__(256)
    k_gram(int64_t n, int32_t ld, int32_t k, const double *__restrict__ U, const double *__restrict__ W1, int32_t q1,
           const double *__restrict__ W2, int32_t q2, double *__restrict__ partials) {
  __shared__ double su[kGramRows][kMaxCoupledM];
  __shared__ double sw[kGramRows][2 * kMaxCoupledM];
  const int q = q1 + q2;
  const int ne = k * q;
  double acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.0;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
  for (int64_t base = r0; base < r1; base += kGramRows) {
    const int rows = (int)min((int64_t)kGramRows, r1 - base);
    __syncthreads();
    for (int t = threadIdx.x; t < rows * k; t += blockDim.x) su[t / k][t % k] = U[(base + t / k) * ld + t % k];
    for (int t = threadIdx.x; t < rows * q; t += blockDim.x) {
      const int r = t / q, j = t % q;
      sw[r][j] = j < q1 ? W1[(base + r) * ld + j] : W2[(base + r) * ld + (j - q1)];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = threadIdx.x + u * 256;
      if (e < ne) {
        const int i = e / q, j = e % q;
        for (int r = 0; r < rows; ++r) acc[u] = fma(su[r][i], sw[r][j], acc[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int e = threadIdx.x + u * 256;
    if (e < ne) partials[(int64_t)blockIdx.x * ne + e] = acc[u];
  }
}

// Per-column reductions over an n x m block (column statistics, sums, residual norms): f(e, v) gives
// the NV values of flat element e; thread t owns column t % m (the grid stride is a multiple of m),
// sums its elements in order, and the block adds its threads' sums per column in thread order.
// partials[b][q * m + l]; the second pass is k_partials_final.
template <int NV, typename F>
__global__ void __launch_bounds__(256) k_colred(int64_t total, int32_t m, int64_t stride, F f, double *partials) {
  __shared__ double sm[NV][256];
  const int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  if (t < stride)
    for (int64_t e = t; e < total; e += stride) {
      double v[NV];
      f(e, v);
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] += v[q];
    }
#pragma unroll
  for (int q = 0; q < NV; ++q) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * 256;
  for (int j = threadIdx.x; j < NV * m; j += 256) {
    const int q = j / m, l = j % m;
    const int first = (int)((l - base % m + m) % m);
    double s = 0.0;
    for (int u = first; u < 256; u += m)
      if (base + u < stride) s += sm[q][u];
    partials[(int64_t)blockIdx.x * NV * m + j] = s;
  }
}

// ||b||^2, sum(b) and the count of non-finite entries of b (and of x0 when given), per column.
struct StatsF {
  const double *B, *X;
  __device__ void operator()(int64_t e, double (&v)[3]) const {
    const double b = B[e];
    v[0] = b * b;
    v[1] = b;
    v[2] = (!isfinite(b) || (X && !isfinite(X[e]))) ? 1.0 : 0.0;
  }
};
struct SumF {
  const double *X;
  __device__ void operator()(int64_t e, double (&v)[1]) const { v[0] = X[e]; }
};
struct ResidF {
  const double *B, *AX;
  __device__ void operator()(int64_t e, double (&v)[1]) const {
    const double r = B[e] - AX[e];
    v[0] = r * r;
  }
};

// X[e] = zero[l] ? 0 : X[e] - shift[l] for column l = e % m (zero-b columns, zero-mean solutions).
__global__ void k_fix_cols(int64_t total, int32_t m, int64_t stride, double *X, const double *__restrict__ shift,
                           const int32_t *__restrict__ zero) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= stride) return;
  const int l = (int)(t % m);
  const double sh = shift[l];
  const bool z = zero[l] != 0;
  for (int64_t e = t; e < total; e += stride) X[e] = z ? 0.0 : X[e] - sh;
}

struct Terms {
  const double *Z[3];
  const double *M[3];  // k x k, row-major (M[p * k + q]); device
};

// Y[i, q] = Z0[i, q] + sum_t sum_p Z_t[i, p] M_t[p, q] for q < k (columns k..ld-1 untouched).
// A group of G = pow2 >= k lanes owns one row: lane p loads Z_t[i, p], the products are formed by
// broadcasting within the group, and the row is written only after all its reads (Y may be Z0 or a
// Z_t).
template <int G>
__global__ void __launch_bounds__(256)
    k_bupdate(int64_t n, int32_t ld, int32_t k, const double *Z0, Terms tm, int32_t nt, double *Y) {
  __shared__ double sm[3][kMaxCoupledM * kMaxCoupledM];
  for (int t = 0; t < nt; ++t)
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) sm[t][e] = tm.M[t][e];
  __syncthreads();
  const int lane = threadIdx.x % G;
  const unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << ((threadIdx.x % 32) / G * G));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; i < n; i += groups) {
    double y = lane < k ? Z0[i * ld + lane] : 0.0;
    for (int t = 0; t < nt; ++t) {
      const double z = lane < k ? tm.Z[t][i * ld + lane] : 0.0;
      const double *M = sm[t];
      for (int p = 0; p < k; ++p) {
        const double zp = __shfl_sync(gmask, z, p, G);
        if (lane < k) y = fma(zp, M[p * k + lane], y);
      }
    }
    __syncwarp(gmask);
    if (lane < k) Y[i * ld + lane] = y;
  }
}

// ---------------------------------------------------------------- split-float block kernels
// On the split path the Gram products and block updates run on the FP32 pipe like the GSpMV: each
// double is cut into (hi, lo) floats (split_f64), products are formed as ah*bh (rounded) plus its
// exact rounding error plus ah*bl + al*bh, and sums are carried as float pairs through TwoSum, two
// columns per packed f32x2 instruction. Relative to sum |a||b| the error is about 2^-44 (the
// truncation of x, the dropped al*bl, the float rounding of the low sums).
//
// An element takes the split form when it is zero or 2^-40 <= |x| < 2^44: then every nonzero
// product of two such elements lies in [2^-80, 2^88), its error terms stay normal floats, and a sum
// of up to 2^31 of them cannot overflow. A row (update) or tile (Gram) that holds any other value is
// computed with native DFMA instead.
__device__ __forceinline__ bool blk_split_ok(double x) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  return (((hw >> 20) & 0x7FFu) - 983u < 84u) || (((hw & 0x7FFFFFFFu) | lw) == 0u);
}

// (sh, sl) += (ah + al) * (bh + bl) on two packed float lanes.
__device__ __forceinline__ void acc_pair(uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl, uint64_t &sh,
                                         uint64_t &sl) {
  const uint64_t ph = f2_mul(ah, bh);
  uint64_t pl = f2_fma(ah, bh, ph ^ 0x8000000080000000ull);  // exact error of ah*bh (-ph by sign flip)
  pl = f2_fma(ah, bl, pl);
  pl = f2_fma(al, bh, pl);
  const uint64_t t = f2_add(sh, ph);
  const uint64_t bb = f2_sub(t, sh);
  const uint64_t e = f2_add(f2_sub(sh, f2_sub(t, bb)), f2_sub(ph, bb));
  sh = t;
  sl = f2_add(sl, f2_add(e, pl));
}

__device__ __forceinline__ bool pair_finite(uint64_t v) {
  float a, b;
  f2_unpack(v, a, b);
  return split_finite(a) && split_finite(b);
}

// (hi + lo) of lane c of a packed pair, widened exactly.
__device__ __forceinline__ double pair_value(uint64_t sh, uint64_t sl, int c) {
  float h0, h1, l0, l1;
  f2_unpack(sh, h0, h1);
  f2_unpack(sl, l0, l1);
  return c == 0 ? widen_f32(h0) + widen_f32(l0) : widen_f32(h1) + widen_f32(l1);
}

struct SplitTerms {
  const double *Z[3];
  const float4 *Ms[3];  // [p][j], p < ld, j < ld / 2: {hi M[p][2j], hi M[p][2j+1], lo M[p][2j], lo M[p][2j+1]}
  const double *Md[3];  // k x k row-major (the native fallback)
};

// Y[i, q] = Z0[i, q] + sum_t sum_p Z_t[i, p] M_t[p, q], ld even (ld = k or k + 1 with a zero padding
// column; M_t is zero-padded to ld x ld, so the padding column keeps Z0's zero). A group of G lanes
// owns one row, lane j the columns 2j and 2j + 1 (j < ld / 2): it splits its two Z_t values, and
// every lane takes each pair in turn from its owner by shuffle. Each lane reads its own elements
// before it writes them (Y may be Z0 or a Z_t).
template <int G>
__global__ void __launch_bounds__(256)
    k_bupdate_split(int64_t n, int32_t ld, int32_t k, const double *Z0, SplitTerms tm, int32_t nt, double *Y) {
  __shared__ float4 sm[3][kMaxCoupledM * kMaxCoupledM / 2];
  const int half = ld / 2;
#pragma unroll
  for (int t = 0; t < 3; ++t)
    if (t < nt)
      for (int e = threadIdx.x; e < ld * half; e += blockDim.x) sm[t][e] = tm.Ms[t][e];
  __syncthreads();
  const int lane = threadIdx.x % G;
  const bool own = lane < half;
  const int lc = own ? lane : 0;
  const unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << ((threadIdx.x % 32) / G * G));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; i < n; i += groups) {
    const int64_t off = i * ld + 2 * lc;
    double2 y0 = make_double2(0.0, 0.0), z[3];
    if (own) y0 = *reinterpret_cast<const double2 *>(Z0 + off);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      z[t] = make_double2(0.0, 0.0);
      if (t < nt && own) z[t] = *reinterpret_cast<const double2 *>(tm.Z[t] + off);
    }
    uint64_t sh = 0, sl = 0;
    bool bad = false;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (t >= nt) break;
      bad = bad || !blk_split_ok(z[t].x) || !blk_split_ok(z[t].y);
      float h0, l0, h1, l1;
      split_f64(z[t].x, h0, l0);
      split_f64(z[t].y, h1, l1);
      const float4 *M = sm[t];
      for (int j = 0; j < half; ++j) {
        const float a0 = __shfl_sync(gmask, h0, j, G), b0 = __shfl_sync(gmask, l0, j, G);
        const float a1 = __shfl_sync(gmask, h1, j, G), b1 = __shfl_sync(gmask, l1, j, G);
        const float4 m0 = M[(2 * j) * half + lc], m1 = M[(2 * j + 1) * half + lc];
        acc_pair(f2_pack(a0, a0), f2_pack(b0, b0), f2_pack(m0.x, m0.y), f2_pack(m0.z, m0.w), sh, sl);
        acc_pair(f2_pack(a1, a1), f2_pack(b1, b1), f2_pack(m1.x, m1.y), f2_pack(m1.z, m1.w), sh, sl);
      }
    }
    bad = bad || !pair_finite(sh) || !pair_finite(sl);
    double2 y;
    if (__any_sync(gmask, bad)) {  // the whole group recomputes the row with native DFMA
      y = y0;
      const int q0 = 2 * lc, q1 = 2 * lc + 1;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        if (t >= nt) break;
        for (int p = 0; p < k; ++p) {
          const double zp = __shfl_sync(gmask, (p & 1) ? z[t].y : z[t].x, p >> 1, G);
          if (own && q0 < k) y.x = fma(zp, __ldg(tm.Md[t] + p * k + q0), y.x);
          if (own && q1 < k) y.y = fma(zp, __ldg(tm.Md[t] + p * k + q1), y.y);
        }
      }
    } else {
      y.x = y0.x + pair_value(sh, sl, 0);
      y.y = y0.y + pair_value(sh, sl, 1);
    }
    if (own) *reinterpret_cast<double2 *>(Y + off) = y;
  }
}

constexpr int kGramStage = 768;  // staged elements per tile (3 per thread)

// Column jj of the padded Gram layout [W1 (ld) | W2 (ld)] as a column of C (-1: a padding column).
__device__ __forceinline__ int gram_real_col(int jj, int ld, int q1, int q2) {
  const int q1p = q1 > 0 ? ld : 0;
  return jj < q1p ? (jj < q1 ? jj : -1) : (jj - q1p < q2 ? q1 + jj - q1p : -1);
}

// Pass 1 of C (k x q) = U^T [W1 | W2] on the split path.
// Tiles of R rows (R even, R w <= 768 with w = ld + qp, qp = ld or 2 ld, ld even) of the row layout
// [U (ld) | W1 (ld) | W2 (ld)] are staged as split (hi, lo) floats, transposed: column c, rows
// (2 rp, 2 rp + 1) form one packed pair at c * RPs + rp (RPs odd, so consecutive columns fall in
// different banks), and one 64-bit shared load gives a packed operand for two rows at once. Each
// thread loads its three elements of the next tile into registers while the current one is
// computed. Thread t owns the entries (i, j) and (i, j + qp / 2) for e = t % np (np = k qp / 2; i =
// e / (qp / 2), j = e % (qp / 2); with np > 256, e = t, t + 256, ...), the two sharing the U loads,
// and with np <= 128 the row pairs rp = s, s + S, ... of each tile (slice s = t / np, S = 256 / np).
// The two packed lanes (even and odd rows) and then the slices are added in order at the end;
// partials[b][i * q + j] for the real columns. A tile holding a value outside the split window is
// computed with native DFMA.
// EPT: entry pairs per thread the kernel is compiled for (1 when np <= 256, else 4).
template <int EPT>
__global__ void __launch_bounds__(256, EPT == 1 ? 4 : 2)
    k_gram_split(int64_t n, int32_t ld, int32_t k, const double *__restrict__ U, const double *__restrict__ W1,
                 int32_t q1, const double *__restrict__ W2, int32_t q2, double *__restrict__ partials) {
  __shared__ uint64_t st_hi[kGramStage / 2 + 96], st_lo[kGramStage / 2 + 96];
  __shared__ double red[512];
  const int q1p = q1 > 0 ? ld : 0, qp = q1p + (q2 > 0 ? ld : 0), hp = qp / 2;
  const int w = ld + qp, R = (kGramStage / w) & ~1, RPs = (R / 2) | 1;
  const int np = k * hp;
  const int S = np >= 256 ? 1 : 256 / np;
  const int ept = np > 256 ? (np + 255) / 256 : 1;  // <= EPT (k <= 32, qp <= 64)
  const int slice = np >= 256 ? 0 : (int)threadIdx.x / np;
  const bool active = slice < S;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
  // this thread's three staged elements: source pointer (advanced by one tile per step), tile row,
  // float slot in the stage
  const double *src[3];
  int srow[3], sslot[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int v = (int)threadIdx.x + u * 256;
    const int r = v / w, c = v % w;
    srow[u] = v < R * w ? r : R;  // R: no element
    const double *col = c < ld ? U + c : (c < ld + q1p ? W1 + (c - ld) : W2 + (c - ld - q1p));
    src[u] = col + (r0 + (srow[u] < R ? r : 0)) * ld;
    sslot[u] = (c * RPs + r / 2) * 2 + (r & 1);
  }
  const int64_t tile_step = (int64_t)R * ld;
  // this thread's entry pairs: stage offsets of its U column and its two W columns
  int eoff_u[EPT], eoff_a[EPT], eoff_b[EPT], ei[EPT], ej[EPT];
  bool eon[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int e = (np >= 256 ? (int)threadIdx.x + u * 256 : (int)threadIdx.x % np);
    eon[u] = active && u < ept && e < np;
    ei[u] = eon[u] ? e / hp : 0;
    ej[u] = eon[u] ? e % hp : 0;
    eoff_u[u] = ei[u] * RPs;
    eoff_a[u] = (ld + ej[u]) * RPs;
    eoff_b[u] = (ld + ej[u] + hp) * RPs;
  }
  uint64_t ah[EPT], al[EPT], bh[EPT], bl[EPT];
  double nat[EPT][2];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    ah[u] = al[u] = bh[u] = bl[u] = 0;
    nat[u][0] = nat[u][1] = 0.0;
  }
  double x[3];
  auto fetch = [&](int rows) {
#pragma unroll
    for (int u = 0; u < 3; ++u) x[u] = srow[u] < rows ? *src[u] : 0.0;
  };
  if (r0 < r1) fetch((int)min((int64_t)R, r1 - r0));
  float *fh = reinterpret_cast<float *>(st_hi), *fl = reinterpret_cast<float *>(st_lo);
  for (int64_t base = r0; base < r1; base += R) {
    const int rows = (int)min((int64_t)R, r1 - base);
    __syncthreads();  // the previous tile's products are done with the stage
    bool bad = false;
#pragma unroll
    for (int u = 0; u < 3; ++u)
      if (srow[u] < R) {  // rows past the end of the block's range are staged as zeros
        bad = bad || !blk_split_ok(x[u]);
        split_f64(x[u], fh[sslot[u]], fl[sslot[u]]);
      }
    const bool tile_bad = __syncthreads_or(bad) != 0;
    if (base + R < r1) {
#pragma unroll
      for (int u = 0; u < 3; ++u) src[u] += tile_step;
      fetch((int)min((int64_t)R, r1 - base - R));
    }
    const int rps = (rows + 1) / 2;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      if (!eon[u]) break;
      if (!tile_bad) {
        const uint64_t *uh = st_hi + eoff_u[u], *ul = st_lo + eoff_u[u];
        const uint64_t *wah = st_hi + eoff_a[u], *wal = st_lo + eoff_a[u];
        const uint64_t *wbh = st_hi + eoff_b[u], *wbl = st_lo + eoff_b[u];
        for (int rp = slice; rp < rps; rp += S) {
          const uint64_t xh = uh[rp], xl = ul[rp];
          acc_pair(xh, xl, wah[rp], wal[rp], ah[u], al[u]);
          acc_pair(xh, xl, wbh[rp], wbl[rp], bh[u], bl[u]);
        }
      } else {
        const int ja = ej[u], jb = ej[u] + hp, i = ei[u];
        const double *Wa = ja < q1p ? W1 + ja : W2 + (ja - q1p);
        const double *Wb = jb < q1p ? W1 + jb : W2 + (jb - q1p);
        for (int rp = slice; rp < rps; rp += S)
          for (int h = 0; h < 2; ++h) {
            const int r = 2 * rp + h;
            if (r >= rows) break;
            const int64_t o = (base + r) * ld;
            const double uv = U[o + i];
            nat[u][0] = fma(uv, Wa[o], nat[u][0]);
            nat[u][1] = fma(uv, Wb[o], nat[u][1]);
          }
      }
    }
  }
  __syncthreads();
  // per owned entry pair: even rows + odd rows + the native tiles; then the slices in order
  const int q = q1 + q2;
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    if (!eon[u]) break;
    const double va = (pair_value(ah[u], al[u], 0) + pair_value(ah[u], al[u], 1)) + nat[u][0];
    const double vb = (pair_value(bh[u], bl[u], 0) + pair_value(bh[u], bl[u], 1)) + nat[u][1];
    if (S == 1) {
      const int ca = gram_real_col(ej[u], ld, q1, q2), cb = gram_real_col(ej[u] + hp, ld, q1, q2);
      if (ca >= 0) partials[(int64_t)blockIdx.x * k * q + ei[u] * q + ca] = va;
      if (cb >= 0) partials[(int64_t)blockIdx.x * k * q + ei[u] * q + cb] = vb;
    } else {
      red[2 * threadIdx.x] = va;
      red[2 * threadIdx.x + 1] = vb;
    }
  }
  if (S == 1) return;
  __syncthreads();
  if ((int)threadIdx.x < np) {
    const int e = threadIdx.x, i = e / hp, j = e % hp;
    double va = 0.0, vb = 0.0;
    for (int sidx = 0; sidx < S; ++sidx) {
      va += red[2 * (sidx * np + e)];
      vb += red[2 * (sidx * np + e) + 1];
    }
    const int ca = gram_real_col(j, ld, q1, q2), cb = gram_real_col(j + hp, ld, q1, q2);
    if (ca >= 0) partials[(int64_t)blockIdx.x * k * q + i * q + ca] = va;
    if (cb >= 0) partials[(int64_t)blockIdx.x * k * q + i * q + cb] = vb;
  }
}

// ---------------------------------------------------------------- host helpers
// Solve G Y = F (k x k, row-major) by LU with partial pivoting; false on a zero pivot or a
// non-finite result. G is not modified.
bool lu_solve_multi(int k, const std::vector<double> &G, const std::vector<double> &F, std::vector<double> &Y) {
  std::vector<double> a(G);
  std::vector<int> piv(k);
  for (int c = 0; c < k; ++c) {
    int p = c;
    for (int r = c + 1; r < k; ++r)
      if (std::fabs(a[r * k + c]) > std::fabs(a[p * k + c])) p = r;
    if (a[p * k + c] == 0.0) return false;
    piv[c] = p;
    if (p != c)
      for (int j = 0; j < k; ++j) std::swap(a[c * k + j], a[p * k + j]);
    for (int r = c + 1; r < k; ++r) {
      const double f = a[r * k + c] / a[c * k + c];
      a[r * k + c] = f;
      for (int j = c + 1; j < k; ++j) a[r * k + j] -= f * a[c * k + j];
    }
  }
  Y.assign(k * k, 0.0);
  std::vector<double> b(k);
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < k; ++i) b[i] = F[i * k + j];
    for (int c = 0; c < k; ++c)
      if (piv[c] != c) std::swap(b[c], b[piv[c]]);
    for (int i = 1; i < k; ++i)
      for (int c = 0; c < i; ++c) b[i] -= a[i * k + c] * b[c];
    for (int i = k - 1; i >= 0; --i) {
      double s = b[i];
      for (int c = i + 1; c < k; ++c) s -= a[i * k + c] * b[c];
      b[i] = s / a[i * k + i];
    }
    for (int i = 0; i < k; ++i) {
      if (!std::isfinite(b[i])) return false;
      Y[i * k + j] = b[i];
    }
  }
  return true;
}

__global__ void k_gather_cols(int64_t n, int32_t m, int32_t mp, int32_t k, const int32_t *__restrict__ idx,
                              const double *__restrict__ src, double *__restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * mp; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / mp;
    const int32_t q = (int32_t)(e - i * mp);
    dst[e] = q < k ? src[i * m + idx[q]] : 0.0;
  }
}
__global__ void k_scatter_cols(int64_t n, int32_t m, int32_t mp, int32_t k, const int32_t *__restrict__ idx,
                               const double *__restrict__ src, double *__restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    const int32_t q = (int32_t)(e - i * k);
    dst[i * m + idx[q]] = src[i * mp + q];
  }
}

template <typename Arith>
struct Coupled {
  const ens_matrix *M;
  int64_t n;
  int m, mp, k, vec, lanes, grid, ggrid;
  ens_solve_opts o;
  cudaStream_t s;
  Scratch &sc;
  ens_amg single;  // one-level "hierarchy" = the Chebyshev polynomial preconditioner
  solver::AmgCycle<Arith> pre;
  bool use_pre = false;
  double *partials = nullptr, *dmat = nullptr, *dots = nullptr, *mbuf = nullptr;
  // split-float Gram products and block updates (the matrix runs on the split path)
  static constexpr bool kSplit = std::is_same<Arith, ArithF64Split>::value;

  Coupled(const ens_matrix *M_, int m_, int k_, const ens_solve_opts &o_, cudaStream_t s_, Scratch &sc_)
      : M(M_), n(M_->n), m(m_), k(k_), o(o_), s(s_), sc(sc_) {
    mp = k == 1 ? 1 : (k + 1) / 2 * 2;
    vec = mp == 1 ? 1 : 2;
    lanes = 1;
    while (lanes * vec < mp) lanes <<= 1;
    grid = M->num_sms * 8;
    // one wave of the Gram kernel (its blocks each take a contiguous share of the rows)
    int per_sm = 8;
    if (kSplit && mp % 2 == 0) {
      const cudaError_t oe =
          gram_wide() ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_split<4>, 256, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_split<1>, 256, 0);
      if (oe != cudaSuccess) {
        (void)cudaGetLastError();  // not a launch error: fall back to one block per SM
        per_sm = 1;
      }
      per_sm = std::max(per_sm, 1);
    }
    ggrid = (int)std::max<int64_t>(1, std::min<int64_t>((n + kGramRows - 1) / kGramRows, (int64_t)M->num_sms * per_sm));
  }

  // the widest Gram of an iteration (q = 2k: np = k mp pair entries) needs four per thread
  bool gram_wide() const { return k * mp > 256; }

  cudaError_t setup() {
    cudaError_t e = sc.get(&partials, (size_t)ggrid * kMaxCoupledM * 2 * kMaxCoupledM);
    if (e == cudaSuccess) e = sc.get(&dmat, (size_t)3 * kMaxCoupledM * kMaxCoupledM + 2 * kMaxCoupledM * kMaxCoupledM);
    if (e == cudaSuccess) e = sc.get(&dots, (size_t)4 * kMaxSolveM);
    // update matrices: 3 k x k doubles, then 3 ld x ld / 2 float4 (two doubles each) split copies
    if (e == cudaSuccess) e = sc.get(&mbuf, (size_t)6 * kMaxCoupledM * kMaxCoupledM);
    if (e != cudaSuccess) return e;
    if (o.precond == ENS_PRECOND_AMG) {
      use_pre = true;
      return pre.setup(sc, M->amg, mp, vec, lanes);
    }
    if (o.precond == ENS_PRECOND_CHEBYSHEV) {
      single.opts.theta = 0.0;
      single.opts.max_levels = 1;
      single.opts.coarse_size = 1;
      single.opts.smooth_steps = o.cheb_steps;
      single.opts.coarse_steps = o.cheb_steps;
      single.opts.cheb_lo = o.cheb_lo;
      single.opts.cheb_hi = o.cheb_hi;
      ens_amg_lev L;
      L.A = const_cast<ens_matrix *>(M);
      single.lev.assign(1, L);
      use_pre = true;
      return pre.setup(sc, &single, mp, vec, lanes);
    }
    return cudaSuccess;
  }

  cudaError_t prec(const double *in, double *out) {
    if (use_pre) return pre.apply(in, out, s);
    return cudaMemcpyAsync(out, in, (size_t)n * mp * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  cudaError_t spmv(const double *in, double *out) {
    const ens_status st = launch_gspmv(M, mp, ENS_F64, in, out, s);
    return st == ENS_OK ? cudaSuccess : cudaErrorLaunchFailure;
  }
  // host C (k x (q1 + q2)) = U^T [W1 W2]
  cudaError_t gram(const double *U, const double *W1, int q1, const double *W2, int q2, std::vector<double> &C) {
    const int q = q1 + q2, ne = k * q;
    if (kSplit && mp % 2 == 0 && (q2 > 0 ? k * mp : k * mp / 2) > 256)
      k_gram_split<4><<<ggrid, 256, 0, s>>>(n, mp, k, U, W1, q1, W2, q2, partials);
    else if (kSplit && mp % 2 == 0)
      k_gram_split<1><<<ggrid, 256, 0, s>>>(n, mp, k, U, W1, q1, W2, q2, partials);
    else
      k_gram<<<ggrid, 256, 0, s>>>(n, mp, k, U, W1, q1, W2, q2, partials);
    k_partials_final<<<partials_final_grid(ne), 256, 0, s>>>(ggrid, ne, partials, dmat);
    cudaError_t e = cudaGetLastError();
    C.assign(ne, 0.0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(C.data(), dmat, ne * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  }
  // per-column dots of up to 3 pairs over the mp columns -> host [npairs][k]
  cudaError_t coldots(std::vector<std::pair<const double *, const double *>> pairs, std::vector<double> &out) {
    const double *xs[4], *ys[4];
    for (size_t t = 0; t < pairs.size(); ++t) {
      xs[t] = pairs[t].first;
      ys[t] = pairs[t].second;
    }
    if (ens_block_dots(n, mp, (int32_t)pairs.size(), xs, ys, dots, s) != ENS_OK) return cudaErrorLaunchFailure;
    std::vector<double> all(pairs.size() * mp);
    cudaError_t e = cudaMemcpyAsync(all.data(), dots, all.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    out.assign(pairs.size() * k, 0.0);
    for (size_t t = 0; t < pairs.size(); ++t)
      for (int q = 0; q < k; ++q) out[t * k + q] = all[t * mp + q];
    return e;
  }
  // Y = Z0 + sum_t Z_t M_t (host matrices, k x k row-major)
  cudaError_t update(double *Y, const double *Z0, std::vector<std::pair<const double *, std::vector<double>>> terms) {
    const int nt = (int)terms.size();
    std::vector<double> hm((size_t)6 * kMaxCoupledM * kMaxCoupledM, 0.0);
    for (int t = 0; t < nt; ++t) std::copy(terms[t].second.begin(), terms[t].second.end(), hm.begin() + (size_t)t * k * k);
    const size_t soff = (size_t)3 * kMaxCoupledM * kMaxCoupledM;  // start of the split copies
    const bool split = kSplit && mp % 2 == 0 && split_matrices(terms, reinterpret_cast<float4 *>(hm.data() + soff));
    const size_t bytes = split ? hm.size() * sizeof(double) : (size_t)nt * k * k * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(mbuf, hm.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (split) {
      SplitTerms st{};
      const size_t sz = (size_t)mp * (mp / 2);
      for (int t = 0; t < nt; ++t) {
        st.Z[t] = terms[t].first;
        st.Md[t] = mbuf + (size_t)t * k * k;
        st.Ms[t] = reinterpret_cast<const float4 *>(mbuf + soff) + t * sz;
      }
      const int half = mp / 2;
      const int gsz = half <= 1 ? 1 : half <= 2 ? 2 : half <= 4 ? 4 : half <= 8 ? 8 : 16;
      const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n * gsz + 255) / 256, (int64_t)M->num_sms * 8));
      switch (gsz) {
        case 1: k_bupdate_split<1><<<blocks, 256, 0, s>>>(n, mp, k, Z0, st, nt, Y); break;
        case 2: k_bupdate_split<2><<<blocks, 256, 0, s>>>(n, mp, k, Z0, st, nt, Y); break;
        case 4: k_bupdate_split<4><<<blocks, 256, 0, s>>>(n, mp, k, Z0, st, nt, Y); break;
        case 8: k_bupdate_split<8><<<blocks, 256, 0, s>>>(n, mp, k, Z0, st, nt, Y); break;
        default: k_bupdate_split<16><<<blocks, 256, 0, s>>>(n, mp, k, Z0, st, nt, Y); break;
      }
      return cudaGetLastError();
    }
    Terms tm{};
    for (int t = 0; t < nt; ++t) {
      tm.Z[t] = terms[t].first;
      tm.M[t] = mbuf + (size_t)t * k * k;
    }
    const int gsz = k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n * gsz + 255) / 256, (int64_t)M->num_sms * 8));
    switch (gsz) {
      case 1: k_bupdate<1><<<blocks, 256, 0, s>>>(n, mp, k, Z0, tm, nt, Y); break;
      case 2: k_bupdate<2><<<blocks, 256, 0, s>>>(n, mp, k, Z0, tm, nt, Y); break;
      case 4: k_bupdate<4><<<blocks, 256, 0, s>>>(n, mp, k, Z0, tm, nt, Y); break;
      case 8: k_bupdate<8><<<blocks, 256, 0, s>>>(n, mp, k, Z0, tm, nt, Y); break;
      case 16: k_bupdate<16><<<blocks, 256, 0, s>>>(n, mp, k, Z0, tm, nt, Y); break;
      default: k_bupdate<32><<<blocks, 256, 0, s>>>(n, mp, k, Z0, tm, nt, Y); break;
    }
    return cudaGetLastError();
  }
  // The (hi, lo) float copies of the update matrices, zero-padded to mp x mp, in the layout of
  // SplitTerms::Ms; false when an entry is neither zero nor in [2^-80, 2^80] (the launch then runs
  // natively). hi is the float nearest to v and lo the float nearest to v - hi, so hi + lo is within
  // 2^-48 |v| of v.
  bool split_matrices(const std::vector<std::pair<const double *, std::vector<double>>> &terms, float4 *out) const {
    const int half = mp / 2;
    for (size_t t = 0; t < terms.size(); ++t)
      for (int p = 0; p < mp; ++p)
        for (int j = 0; j < half; ++j) {
          float hi[2], lo[2];
          for (int c = 0; c < 2; ++c) {
            const int col = 2 * j + c;
            const double v = (p < k && col < k) ? terms[t].second[(size_t)p * k + col] : 0.0;
            const double a = std::fabs(v);
            if (v != 0.0 && !(a >= 0x1p-80 && a <= 0x1p80)) return false;
            hi[c] = (float)v;
            lo[c] = (float)(v - (double)hi[c]);
          }
          out[t * (size_t)mp * half + (size_t)p * half + j] = make_float4(hi[0], hi[1], lo[0], lo[1]);
        }
    return true;
  }
};

std::vector<double> scaled_identity(int k, double c) {
  std::vector<double> I(k * k, 0.0);
  for (int q = 0; q < k; ++q) I[q * k + q] = c;
  return I;
}

// Per-column reduction of an n x m block through k_colred + k_partials_final; the NV * m results
// ([q][l]) are read back to the host.
template <int NV, typename F>
cudaError_t column_reduce(int64_t n, int32_t m, F f, int grid, double *partials, double *dout, double *hout,
                          cudaStream_t s) {
  const int64_t stride = (int64_t)grid * 256 / m * m;
  k_colred<NV><<<grid, 256, 0, s>>>(n * m, m, stride, f, partials);
  k_partials_final<<<partials_final_grid(NV * m), 256, 0, s>>>(grid, NV * m, partials, dout);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(hout, dout, (size_t)NV * m * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

template <typename Arith>
ens_status solve_coupled(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                         const ens_solve_opts &o, ens_solve_stats *st, cudaStream_t s) {
  const int64_t n = M->n;
  const bool singular = (M->flags & ENS_MATRIX_SINGULAR) != 0;
  std::vector<int32_t> status(m, ENS_COL_CONVERGED), iters(m, 0), idx;
  std::vector<double> relres(m, std::nan("")), bn(m, 0.0);
  std::vector<char> zero_b(m, 0);
  cudaError_t e = cudaSuccess;
  ens_status gst = ENS_OK;
  int it = 0;
  {
    Scratch sc(s, o);
    // per-column start checks on the device: ||b||^2, sum(b), non-finite entries of b and x0
    const int rgrid = (int)std::max<int64_t>(1, std::min<int64_t>((n * m + 255) / 256, (int64_t)M->num_sms * 4));
    double *rpart = nullptr, *rout = nullptr;
    e = sc.get(&rpart, (size_t)rgrid * 3 * m);
    if (e == cudaSuccess) e = sc.get(&rout, (size_t)3 * m);
    std::vector<double> cs(3 * m, 0.0);
    if (e == cudaSuccess)
      e = column_reduce<3>(n, m, StatsF{B, o.x0_zero ? nullptr : X}, rgrid, rpart, rout, cs.data(), s);
    if (e == cudaSuccess)
      for (int l = 0; l < m; ++l) {
        bn[l] = std::sqrt(cs[l]);
        if (cs[2 * m + l] != 0.0) status[l] = ENS_COL_NONFINITE;
        else if (bn[l] == 0.0) {
          zero_b[l] = 1;
          relres[l] = 0.0;
        } else if (singular && std::fabs(cs[m + l]) > 1e-10 * std::sqrt((double)n) * bn[l])
          status[l] = ENS_COL_INCOMPATIBLE;
        else idx.push_back(l);
      }
    const int k = (int)idx.size();
    Coupled<Arith> C(M, m, std::max(k, 1), o, s, sc);
    const int mp = C.mp;
    const size_t blk = (size_t)n * mp;
    double *Xb, *Bb, *R, *Rt, *P, *Ph, *V, *S, *Sh, *T;
    int32_t *didx = nullptr;
    Xb = Bb = R = Rt = P = Ph = V = S = Sh = T = nullptr;
    const int cg = M->num_sms * 8;
    if (e == cudaSuccess && k > 0) {
      for (double **p : {&Xb, &Bb, &R, &Rt, &P, &Ph, &V, &S, &Sh, &T})
        if (e == cudaSuccess) e = sc.get(p, blk);
      if (e == cudaSuccess) e = sc.get(&didx, (size_t)k);
      // every block starts at zero, so the padding column (odd k) stays zero through every product
      for (double *p : {Xb, Bb, R, Rt, P, Ph, V, S, Sh, T})
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, blk * sizeof(double), s);
      if (e == cudaSuccess) e = C.setup();
      if (e == cudaSuccess) e = cudaMemcpyAsync(didx, idx.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) {
        k_gather_cols<<<cg, 256, 0, s>>>(n, m, mp, k, didx, B, Bb);
        if (!o.x0_zero) k_gather_cols<<<cg, 256, 0, s>>>(n, m, mp, k, didx, X, Xb);
        e = cudaGetLastError();
      }
      // R = B - A X, R~ = R, P = R
      if (e == cudaSuccess) e = C.spmv(Xb, R);
      std::vector<double> I1 = scaled_identity(k, -1.0);
      if (e == cudaSuccess) e = C.update(R, Bb, {{R, I1}});
      if (e == cudaSuccess) e = cudaMemcpyAsync(Rt, R, blk * 8, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(P, R, blk * 8, cudaMemcpyDeviceToDevice, s);
      auto below = [&](const std::vector<double> &n2, int off) {
        for (int q = 0; q < k; ++q)
          if (!(std::sqrt(n2[off + q]) <= tol[idx[q]] * bn[idx[q]])) return false;
        return true;
      };
      std::vector<double> d, G, H, F, al, be;
      int state = ENS_COL_MAXITER;
      if (e == cudaSuccess) e = C.coldots({{R, R}}, d);
      if (e == cudaSuccess && below(d, 0)) state = ENS_COL_CONVERGED;
      std::vector<double> rn2 = d;
      for (int kk = 1; e == cudaSuccess && state == ENS_COL_MAXITER && kk <= o.max_iter; ++kk) {
        it = kk;
        e = C.prec(P, Ph);
        if (e == cudaSuccess) e = C.spmv(Ph, V);
        std::vector<double> GH;
        if (e == cudaSuccess) e = C.gram(Rt, V, k, R, k, GH);
        if (e != cudaSuccess) break;
        G.assign(k * k, 0.0);
        H.assign(k * k, 0.0);
        for (int i = 0; i < k; ++i)
          for (int j = 0; j < k; ++j) {
            G[i * k + j] = GH[i * 2 * k + j];
            H[i * k + j] = GH[i * 2 * k + k + j];
          }
        if (!lu_solve_multi(k, G, H, al)) {
          state = ENS_COL_BREAKDOWN;
          break;
        }
        std::vector<double> nal(al);
        for (double &v : nal) v = -v;
        e = C.update(S, R, {{V, nal}});  // S = R - V alpha
        if (e == cudaSuccess) e = C.prec(S, Sh);
        if (e == cudaSuccess) e = C.spmv(Sh, T);
        if (e == cudaSuccess) e = C.coldots({{S, S}, {T, S}, {T, T}}, d);
        if (e != cudaSuccess) break;
        if (below(d, 0)) {  // half step: X += P^ alpha
          e = C.update(Xb, Xb, {{Ph, al}});
          rn2.assign(d.begin(), d.begin() + k);
          state = ENS_COL_CONVERGED;
          break;
        }
        double ts = 0.0, tt = 0.0;
        for (int q = 0; q < k; ++q) {
          ts += d[k + q];
          tt += d[2 * k + q];
        }
        if (tt == 0.0 || !std::isfinite(ts / tt)) {
          state = ENS_COL_BREAKDOWN;
          break;
        }
        const double om = ts / tt;
        e = C.update(Xb, Xb, {{Ph, al}, {Sh, scaled_identity(k, om)}});
        if (e == cudaSuccess) e = C.update(R, S, {{T, scaled_identity(k, -om)}});
        std::vector<double> FT;
        if (e == cudaSuccess) e = C.coldots({{R, R}}, d);
        if (e == cudaSuccess) e = C.gram(Rt, T, k, nullptr, 0, FT);
        if (e != cudaSuccess) break;
        rn2 = d;
        bool fin = true;
        for (int q = 0; q < k; ++q) fin = fin && std::isfinite(d[q]);
        if (!fin) {
          state = ENS_COL_NONFINITE;
          break;
        }
        if (below(d, 0)) {
          state = ENS_COL_CONVERGED;
          break;
        }
        if (om == 0.0) {
          state = ENS_COL_BREAKDOWN;
          break;
        }
        for (double &v : FT) v = -v;
        if (!lu_solve_multi(k, G, FT, be)) {
          state = ENS_COL_BREAKDOWN;
          break;
        }
        std::vector<double> obe(be);
        for (double &v : obe) v = -om * v;
        e = C.update(P, R, {{P, be}, {V, obe}});  // P = R + P beta - omega V beta
      }
      for (int q = 0; q < k; ++q) {
        const int l = idx[q];
        iters[l] = it;
        status[l] = state != ENS_COL_MAXITER ? state
                    : (std::sqrt(rn2[q]) <= tol[l] * bn[l] ? ENS_COL_CONVERGED : ENS_COL_MAXITER);
      }
      if (e == cudaSuccess) {
        k_scatter_cols<<<cg, 256, 0, s>>>(n, m, mp, k, didx, Xb, X);
        e = cudaGetLastError();
      }
    }
    // zero right-hand sides: x = 0; singular operators: zero-mean solutions of the solved columns
    bool any_zero = false;
    for (int l = 0; l < m; ++l) any_zero = any_zero || zero_b[l];
    if (e == cudaSuccess && (any_zero || (singular && k > 0))) {
      std::vector<double> shift(m, 0.0);
      if (singular && k > 0) {
        std::vector<double> sums(m, 0.0);
        e = column_reduce<1>(n, m, SumF{X}, rgrid, rpart, rout, sums.data(), s);
        for (int l : idx) shift[l] = sums[l] / (double)n;
      }
      std::vector<int32_t> zf(m, 0);
      for (int l = 0; l < m; ++l) zf[l] = zero_b[l];
      double *dshift = nullptr;
      int32_t *dzero = nullptr;
      if (e == cudaSuccess) e = sc.get(&dshift, (size_t)m);
      if (e == cudaSuccess) e = sc.get(&dzero, (size_t)m);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dshift, shift.data(), m * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dzero, zf.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) {
        k_fix_cols<<<rgrid, 256, 0, s>>>(n * m, m, (int64_t)rgrid * 256 / m * m, X, dshift, dzero);
        e = cudaGetLastError();
      }
    }
    // true residuals ||b - A x|| / ||b|| of the solved columns
    if (e == cudaSuccess && k > 0) {
      double *AX = nullptr;
      e = sc.get(&AX, (size_t)n * m);
      if (e == cudaSuccess) gst = launch_gspmv(M, m, ENS_F64, X, AX, s);
      if (gst != ENS_OK) e = cudaErrorLaunchFailure;
      std::vector<double> r2(m, 0.0);
      if (e == cudaSuccess) e = column_reduce<1>(n, m, ResidF{B, AX}, rgrid, rpart, rout, r2.data(), s);
      if (e == cudaSuccess)
        for (int l : idx) relres[l] = std::sqrt(r2[l]) / bn[l];
    }
    const cudaError_t esync = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = esync;
  }
  if (gst != ENS_OK) return gst;
  if (e != cudaSuccess) return cuda_fail(e, "solve_block_coupled");
  if (st) {
    for (int l = 0; l < m; ++l) {
      if (st->iters) st->iters[l] = iters[l];
      if (st->status) st->status[l] = status[l];
      if (st->relres) st->relres[l] = relres[l];
      if (st->outer) st->outer[l] = 0;
    }
  }
  return ENS_OK;
}

}  // namespace coupled
}  // namespace ens

using namespace ens;

extern "C" ens_status ens_solve_block_coupled(const ens_matrix *A, int32_t m, const double *B, double *X,
                                              const double *tol, const ens_solve_opts *opts, ens_solve_stats *stats,
                                              void *stream) {
  clear_error();
  ens_solve_opts o;
  ens_default_solve_opts(&o);
  if (opts) o = *opts;
  if (!A) return fail(ENS_ERR_INVALID, "solve_block_coupled: matrix is NULL");
  if (A->ncols != A->n) return fail(ENS_ERR_INVALID, "solve_block_coupled: needs a square matrix");
  if (m < 1 || m > coupled::kMaxCoupledM)
    return fail(ENS_ERR_INVALID, "solve_block_coupled: m = %d outside [1, %d]", m, coupled::kMaxCoupledM);
  if (!B || !X || !tol) return fail(ENS_ERR_INVALID, "solve_block_coupled: NULL argument");
  for (int l = 0; l < m; ++l)
    if (!std::isfinite(tol[l]) || tol[l] < 0) return fail(ENS_ERR_INVALID, "solve_block_coupled: tol[%d] invalid", l);
  if ((uintptr_t)B % 8 || (uintptr_t)X % 8) return fail(ENS_ERR_INVALID, "solve_block_coupled: B/X not 8-byte aligned");
  if (o.max_iter < 0) return fail(ENS_ERR_INVALID, "solve_block_coupled: max_iter < 0");
  if (o.workspace) return fail(ENS_ERR_UNSUPPORTED, "solve_block_coupled: takes no caller workspace");
  if (o.precision != ENS_PREC_F64)
    return fail(ENS_ERR_UNSUPPORTED, "solve_block_coupled: only ENS_PREC_F64 (the coupled steps run in float64)");
  if (o.precond == ENS_PRECOND_AMG && !A->amg)
    return fail(ENS_ERR_INVALID, "solve_block_coupled: ENS_PRECOND_AMG needs ens_amg_setup on the matrix");
  if (o.precond != ENS_PRECOND_NONE && !A->full_diag)
    return fail(ENS_ERR_INVALID, "solve_block_coupled: the preconditioner needs a nonzero diagonal in every row");
  if (o.precond == ENS_PRECOND_CHEBYSHEV &&
      (o.cheb_steps < 1 || o.cheb_steps > 64 || !(o.cheb_lo > 0.0) || !(o.cheb_hi > o.cheb_lo)))
    return fail(ENS_ERR_INVALID, "solve_block_coupled: bad Chebyshev options");
  if (o.precond < ENS_PRECOND_NONE || o.precond > ENS_PRECOND_AMG)
    return fail(ENS_ERR_INVALID, "solve_block_coupled: unknown preconditioner %d", o.precond);
  cudaStream_t s = (cudaStream_t)stream;
  return use_split(A) ? coupled::solve_coupled<ArithF64Split>(A, m, B, X, tol, o, stats, s)
                      : coupled::solve_coupled<ArithF64Native>(A, m, B, X, tol, o, stats, s);
}
