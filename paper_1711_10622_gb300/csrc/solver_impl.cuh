// Multi-RHS BiCGStab on an n x m row-interleaved block (Sections 2.2 and 4.1), with an optional
// Jacobi-scaled Chebyshev polynomial preconditioner and an FP32-inner / FP64-outer
// mixed-precision mode.
//
// The m right-hand sides run m independent BiCGStab recurrences (per-column rho, alpha, omega,
// beta); every operator application is one GSpMV over the whole block, so the matrix is read
// once per product for all m columns. Per iteration (right preconditioning, M^-1 = Chebyshev
// polynomial or identity):
//   k_p     p = r + beta (p - omega v)            [+ d0 = D^-1 p / theta, ph = d0]
//   k_cheb  (cheb_steps - 1) x: GSpMV of d, fused 3-term update of d, z = ph, residual
//   k_v     v = A ph,  (rhat, v)  -> alpha       (dot fused into the GSpMV epilogue)
//   k_s     s = r - alpha v,  ||s||^2 -> half-step convergence   [+ Chebyshev start for s]
//   k_cheb  ... z = sh
//   k_t     t = A sh, (t, s), (t, t) -> omega     (dots fused into the GSpMV epilogue)
//   k_xr    x += alpha ph + omega sh, r = s - omega t, ||r||^2, (rhat, r) -> convergence, rho
// The per-column scalar step runs in the last block of each reduction (reduce.cuh), so the
// scalars never leave the device; the host only reads the m convergence flags every
// check_every iterations. Converged columns are frozen (their x is no longer updated).
//
// The solver works on internal copies of B and X whose row stride is m rounded up to an even
// width, so every kernel uses 16-byte row-segment accesses (m = 1 keeps stride 1).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "ens_internal.cuh"
#include "reduce.cuh"
#include "rowprod.cuh"

namespace ens {

bool use_split(const ens_matrix *A);

namespace solver {

enum : int32_t { ST_ACTIVE = 0, ST_HALF = 1, ST_DONE = 2 };
// FL_NOSTEP: the column broke down in its first iteration before x was updated (x is still x0).
enum : int32_t { FL_EARLY = 1, FL_ZERO_B = 2, FL_NOSTEP = 4 };

template <typename T>
struct Cols {
  T *rho, *rho_old, *alpha, *omega, *bn2, *thr2, *rh2, *rn2, *tol, *mean;
  int32_t *state, *iters, *status, *flags;
  double *relres;
  int32_t *it;  // [2]: iterations completed, "go" flag (some column active and it < max_iter)
};

template <typename T>
struct Tiny;
template <>
struct Tiny<double> {
  static constexpr double v = 1e-300;
};
template <>
struct Tiny<float> {
  static constexpr float v = 1e-30f;
};

#define ENS_ROWS(i)                                                                           \
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / LANES) + threadIdx.x / LANES; i < A.n; \
       i += (int64_t)gridDim.x * (kThreads / LANES))

// Kernels whose body is a GSpMV (tile_rows) are launched with a register cap of kTileMinBlocks
// resident blocks per SM and a grid of that many blocks per SM: without it the split kernels took
// 60 registers and 4 blocks per SM and ran their gathers at a lower occupancy than the standalone
// GSpMV (the hybrid tile's shared memory allows 5).
template <typename Arith>
struct TileBlocks {
  static constexpr int value = 6;
};
template <>
struct TileBlocks<ArithF64Hybrid> {
  static constexpr int value = 5;
};
#define ENS_TILE_BOUNDS(Arith) __launch_bounds__(kThreads, TileBlocks<Arith>::value)
// GSpMV kernels without column reductions (k_cheb, k_amg_resid, k_amg_smooth2) hold fewer live
// registers: their float32 forms run at 8 blocks and 32 registers, like the standalone float32
// GSpMV (10-12 % faster there than at 6 blocks); with the reductions' accumulators the float32
// k_start / k_v / k_t / k_resid would spill 56-300 bytes at 32 registers and stay at 6.
template <typename Arith>
struct LightBlocks {
  static constexpr int value = std::is_same<Arith, ArithF32>::value ? 8 : TileBlocks<Arith>::value;
};
#define ENS_LIGHT_BOUNDS(Arith) __launch_bounds__(kThreads, LightBlocks<Arith>::value)
// The Chebyshev step and the V-cycle's residual and two-update smoothing with four columns per lane
// in split float64 (solver_cheb4.cu) need 48 registers, as the standalone four-column GSpMV: 5 blocks
// per SM; every other form as LightBlocks.
template <typename Arith, int VEC>
struct ChebBlocks {
  static constexpr int value =
      std::is_same<Arith, ArithF64Split>::value && VEC == 4 ? 5 : LightBlocks<Arith>::value;
};

// ----------------------------------------------------------------------------- start
// r = b - A x (or r = b and x = 0 when x0_zero), rhat = r; per column ||b||^2, ||r||^2, sum(b).
template <typename Arith, int VEC, int LANES>
__global__ void ENS_TILE_BOUNDS(Arith)
    k_start(MatView A, int32_t m, const typename Arith::T *__restrict__ b, typename Arith::T *x,
            typename Arith::T *__restrict__ r, typename Arith::T *__restrict__ rh, int x0_zero, int singular,
            typename Arith::T incompat, Cols<typename Arith::T> cs, typename Arith::T *partials,
            unsigned *counter, uint32_t mask) {
  using T = typename Arith::T;
  T acc[3][VEC];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[d][q] = T(0);
  auto fin_row = [&](int64_t i, int32_t cc, const T (&ax)[VEC]) {
    T bv[VEC], rv[VEC];
    load_vec<T, VEC>(b + i * m + cc, bv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      rv[q] = bv[q] - ax[q];
      acc[0][q] += bv[q] * bv[q];
      acc[1][q] += rv[q] * rv[q];
      acc[2][q] += bv[q];
    }
    store_vec<T, VEC>(r + i * m + cc, rv);
    if (rh) store_vec<T, VEC>(rh + i * m + cc, rv);
  };
  if (x0_zero) {
    tile_order_rows<VEC, LANES>(A.n, m, [&](int64_t i, int32_t cc) {
      T ax[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) ax[q] = T(0);
      store_vec<T, VEC>(x + i * m + cc, ax);
      fin_row(i, cc, ax);
    });
  } else {
    tile_rows<Arith, VEC, LANES>(A, m, x, mask, fin_row);
  }
  reduce_cols<T, 3, VEC, LANES>(acc, m, partials, counter, [&](int l, const ColTotals<T, 3> &t) {
    const T bn2 = t.v[0][l], rn2 = t.v[1][l], sb = t.v[2][l];
    const T thr2 = cs.tol[l] * cs.tol[l] * bn2;
    int32_t st = ST_ACTIVE, status = ENS_COL_CONVERGED, fl = 0;
    if (!isfinite(bn2) || !isfinite(rn2)) {
      st = ST_DONE;
      status = ENS_COL_NONFINITE;
      fl = FL_EARLY;
    } else if (bn2 == T(0)) {
      st = ST_DONE;
      fl = FL_EARLY | FL_ZERO_B;
    } else if (singular && fabs(sb) > incompat * sqrt(bn2)) {
      st = ST_DONE;
      status = ENS_COL_INCOMPATIBLE;
      fl = FL_EARLY;
    } else if (rn2 <= thr2) {
      st = ST_DONE;
    }
    cs.bn2[l] = bn2;
    cs.thr2[l] = thr2;
    cs.rn2[l] = rn2;
    cs.rh2[l] = rn2;
    cs.rho[l] = rn2;  // rhat = r0, so rho_1 = (rhat, r0) = ||r0||^2
    cs.rho_old[l] = T(1);
    cs.alpha[l] = T(1);
    cs.omega[l] = T(1);
    cs.state[l] = st;
    cs.status[l] = status;
    cs.flags[l] = fl;
    cs.iters[l] = 0;
  }, [&]() {
    int32_t any = 0;
    for (int l = 0; l < m; ++l) any |= cs.state[l] != ST_DONE;
    cs.it[0] = 0;
    cs.it[1] = any;
  });
}

// ----------------------------------------------------------------------------- p update
// p = r + beta (p - omega v) for active columns; with the preconditioner also the first
// Chebyshev term d0 = D^-1 p / theta, written to da and to ph (= z).
template <typename Arith, int VEC, int LANES, bool PREC>
__global__ void __launch_bounds__(kThreads)
    k_p(MatView A, int32_t m, const typename Arith::T *__restrict__ r, typename Arith::T *p,
        const typename Arith::T *__restrict__ v, typename Arith::T *__restrict__ da, typename Arith::T *__restrict__ ph,
        typename Arith::T inv_theta, Cols<typename Arith::T> cs) {
  using T = typename Arith::T;
  const int32_t c = (threadIdx.x % LANES) * VEC;
  if (c >= m) return;
  T beta[VEC], om[VEC];
  bool act[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    const int l = c + q;
    act[q] = cs.state[l] == ST_ACTIVE;
    beta[q] = act[q] ? (cs.rho[l] / cs.rho_old[l]) * (cs.alpha[l] / cs.omega[l]) : T(0);
    om[q] = act[q] ? cs.omega[l] : T(0);
  }
  ENS_ROWS(i) {
    T rv[VEC], pv[VEC], vv[VEC];
    load_vec<T, VEC>(r + i * m + c, rv);
    load_vec_rw<T, VEC>(p + i * m + c, pv);
    load_vec<T, VEC>(v + i * m + c, vv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) pv[q] = act[q] ? rv[q] + beta[q] * (pv[q] - om[q] * vv[q]) : pv[q];
    store_vec<T, VEC>(p + i * m + c, pv);
    if (PREC) {
      const T sc = Arith::dinv(A, i) * inv_theta;
#pragma unroll
      for (int q = 0; q < VEC; ++q) pv[q] *= sc;
      store_vec<T, VEC>(da + i * m + c, pv);
      store_vec<T, VEC>(ph + i * m + c, pv);
    }
  }
}

// ----------------------------------------------------------------------------- Chebyshev step
// One step k >= 1 of the Chebyshev iteration z = p(D^-1 A) D^-1 src (Saad, Alg. 12.1, Jacobi
// scaled, zero start), fused with its GSpMV:
//   res_k = res_{k-1} - A d_{k-1}   (res_0 = src)
//   d_k   = c1 d_{k-1} + c2 D^-1 res_k,   z += d_k
// din is the GSpMV input (read by neighbouring rows), so d_k goes to a second buffer. The last
// step needs neither res_k nor d_k afterwards.
template <typename Arith, int VEC, int LANES, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads, ChebBlocks<Arith, VEC>::value)
    k_cheb(MatView A, int32_t m, const typename Arith::T *__restrict__ din, typename Arith::T *__restrict__ dout,
           const typename Arith::T *__restrict__ src, typename Arith::T *res, typename Arith::T *z,
           typename Arith::T c1, typename Arith::T c2, uint32_t mask) {
  using T = typename Arith::T;
  tile_rows<Arith, VEC, LANES>(A, m, din, mask, [&](int64_t i, int32_t cc, const T (&w)[VEC]) {
    T di[VEC], rs[VEC], zv[VEC], dn[VEC];
    load_vec<T, VEC>(din + i * m + cc, di);
    if (FIRST)
      load_vec<T, VEC>(src + i * m + cc, rs);
    else
      load_vec_rw<T, VEC>(res + i * m + cc, rs);
    load_vec_rw<T, VEC>(z + i * m + cc, zv);
    const T dv = Arith::dinv(A, i);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      rs[q] -= w[q];
      dn[q] = c1 * di[q] + c2 * (dv * rs[q]);
      zv[q] += dn[q];
    }
    store_vec<T, VEC>(z + i * m + cc, zv);
    if (!LAST) {
      store_vec<T, VEC>(res + i * m + cc, rs);
      store_vec<T, VEC>(dout + i * m + cc, dn);
    }
  });
}

// One Chebyshev step (k_cheb) in split float64 with four columns per lane, lanes4 lanes per row (one
// pass over a block of m columns, m a multiple of 4): 12-13 % faster than two columns per lane for
// the standalone GSpMV at m = 8 and 16 on GB300. Compiled in solver_cheb4.cu for lanes4 = 2, 4, 8;
// returns false (nothing launched) for any other lane count. grid_cap: blocks per launch at most.
bool launch_cheb4_split(int lanes4, bool first, bool last, const MatView &A, int32_t m, const double *din,
                        double *dout, const double *src, double *res, double *z, double c1, double c2,
                        uint32_t mask, int num_sms, int64_t grid_cap, cudaStream_t st);
// The V-cycle's res = r - A z (k_amg_resid) and two-update smoothing (k_amg_smooth2) in the same
// four-column form; false (nothing launched) for other lane counts.
bool launch_amg_resid4_split(int lanes4, const MatView &A, int32_t m, const double *z, const double *r, double *res,
                             uint32_t mask, int num_sms, int64_t grid_cap, cudaStream_t st);
bool launch_amg_smooth2_4_split(int lanes4, bool add, const MatView &As, const MatView &A, int32_t m, const double *src,
                                double *z, double inv_theta, double c1, double c2, uint32_t mask, int num_sms,
                                int64_t grid_cap, cudaStream_t st);

// ----------------------------------------------------------------------------- v = A ph
template <typename Arith, int VEC, int LANES>
__global__ void ENS_TILE_BOUNDS(Arith)
    k_v(MatView A, int32_t m, const typename Arith::T *__restrict__ ph, typename Arith::T *__restrict__ v,
        const typename Arith::T *__restrict__ rh, Cols<typename Arith::T> cs,
        typename Arith::T *partials, unsigned *counter, uint32_t mask) {
  using T = typename Arith::T;
  T acc[1][VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) acc[0][q] = T(0);
  tile_rows<Arith, VEC, LANES>(A, m, ph, mask, [&](int64_t i, int32_t cc, const T (&y)[VEC]) {
    T h[VEC];
    store_vec<T, VEC>(v + i * m + cc, y);
    load_vec<T, VEC>(rh + i * m + cc, h);
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[0][q] += h[q] * y[q];
  });
  reduce_cols<T, 1, VEC, LANES>(acc, m, partials, counter, [&](int l, const ColTotals<T, 1> &t) {
    if (cs.state[l] != ST_ACTIVE) return;
    cs.iters[l] = cs.it[0] + 1;
    const T rv = t.v[0][l];
    const T al = cs.rho[l] / rv;
    if (rv == T(0) || !isfinite(al)) {  // breakdown; x keeps its last finite iterate
      cs.state[l] = ST_DONE;
      cs.status[l] = ENS_COL_BREAKDOWN;
      if (cs.it[0] == 0) cs.flags[l] |= FL_NOSTEP;
      return;
    }
    cs.alpha[l] = al;
  });
}

// ----------------------------------------------------------------------------- s update
template <typename Arith, int VEC, int LANES, bool PREC>
__global__ void __launch_bounds__(kThreads)
    k_s(MatView A, int32_t m, const typename Arith::T *__restrict__ r, const typename Arith::T *__restrict__ v,
        typename Arith::T *__restrict__ s, typename Arith::T *__restrict__ da, typename Arith::T *__restrict__ sh,
        typename Arith::T inv_theta, Cols<typename Arith::T> cs, typename Arith::T *partials, unsigned *counter) {
  using T = typename Arith::T;
  const int32_t c = (threadIdx.x % LANES) * VEC;
  T acc[1][VEC], al[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    acc[0][q] = T(0);
    al[q] = (c + q < m && cs.state[c + q] == ST_ACTIVE) ? cs.alpha[c + q] : T(0);
  }
  if (c < m) {
    ENS_ROWS(i) {
      T rv[VEC], vv[VEC];
      load_vec<T, VEC>(r + i * m + c, rv);
      load_vec<T, VEC>(v + i * m + c, vv);
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        rv[q] = al[q] != T(0) ? rv[q] - al[q] * vv[q] : rv[q];
        acc[0][q] += rv[q] * rv[q];
      }
      store_vec<T, VEC>(s + i * m + c, rv);
      if (PREC) {
        const T sc = Arith::dinv(A, i) * inv_theta;
#pragma unroll
        for (int q = 0; q < VEC; ++q) rv[q] *= sc;
        store_vec<T, VEC>(da + i * m + c, rv);
        store_vec<T, VEC>(sh + i * m + c, rv);
      }
    }
  }
  reduce_cols<T, 1, VEC, LANES>(acc, m, partials, counter, [&](int l, const ColTotals<T, 1> &t) {
    if (cs.state[l] == ST_ACTIVE && t.v[0][l] <= cs.thr2[l]) cs.state[l] = ST_HALF;
  });
}

// ----------------------------------------------------------------------------- t = A sh
template <typename Arith, int VEC, int LANES>
__global__ void ENS_TILE_BOUNDS(Arith)
    k_t(MatView A, int32_t m, const typename Arith::T *__restrict__ sh, typename Arith::T *__restrict__ t,
        const typename Arith::T *__restrict__ s, Cols<typename Arith::T> cs, typename Arith::T *partials,
        unsigned *counter, uint32_t mask) {
  using T = typename Arith::T;
  T acc[2][VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) acc[0][q] = acc[1][q] = T(0);
  tile_rows<Arith, VEC, LANES>(A, m, sh, mask, [&](int64_t i, int32_t cc, const T (&y)[VEC]) {
    T sv[VEC];
    store_vec<T, VEC>(t + i * m + cc, y);
    load_vec<T, VEC>(s + i * m + cc, sv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      acc[0][q] += y[q] * sv[q];
      acc[1][q] += y[q] * y[q];
    }
  });
  reduce_cols<T, 2, VEC, LANES>(acc, m, partials, counter, [&](int l, const ColTotals<T, 2> &tt) {
    if (cs.state[l] != ST_ACTIVE) return;
    const T t2 = tt.v[1][l];
    const T om = tt.v[0][l] / t2;
    if (t2 == T(0) || !isfinite(om)) {  // breakdown before x is updated with a non-finite step
      cs.state[l] = ST_DONE;
      cs.status[l] = ENS_COL_BREAKDOWN;
      if (cs.it[0] == 0) cs.flags[l] |= FL_NOSTEP;
      return;
    }
    cs.omega[l] = om;
  });
}

// ----------------------------------------------------------------------------- x, r update
template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    k_xr(MatView A, int32_t m, typename Arith::T *x, const typename Arith::T *__restrict__ ph,
         const typename Arith::T *__restrict__ sh, const typename Arith::T *__restrict__ s,
         const typename Arith::T *__restrict__ t, typename Arith::T *__restrict__ r,
         const typename Arith::T *__restrict__ rh, int32_t max_iter, Cols<typename Arith::T> cs,
         typename Arith::T *partials, unsigned *counter) {
  using T = typename Arith::T;
  const int32_t c = (threadIdx.x % LANES) * VEC;
  T acc[2][VEC], al[VEC], om[VEC];
  int st[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    acc[0][q] = acc[1][q] = T(0);
    st[q] = c + q < m ? cs.state[c + q] : ST_DONE;
    al[q] = st[q] == ST_DONE ? T(0) : cs.alpha[c + q];
    om[q] = st[q] == ST_ACTIVE ? cs.omega[c + q] : T(0);
  }
  if (c < m) {
    ENS_ROWS(i) {
      T xv[VEC], pv[VEC], shv[VEC], sv[VEC], tv[VEC], hv[VEC];
      load_vec_rw<T, VEC>(x + i * m + c, xv);
      load_vec<T, VEC>(ph + i * m + c, pv);
      load_vec<T, VEC>(sh + i * m + c, shv);
      load_vec<T, VEC>(s + i * m + c, sv);
      load_vec<T, VEC>(t + i * m + c, tv);
      load_vec<T, VEC>(rh + i * m + c, hv);
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        // frozen columns keep x exactly (no 0 * v products that could turn NaN)
        const T xa = xv[q] + al[q] * pv[q];
        xv[q] = st[q] == ST_ACTIVE ? xa + om[q] * shv[q] : st[q] == ST_HALF ? xa : xv[q];
        sv[q] = st[q] == ST_ACTIVE ? sv[q] - om[q] * tv[q] : sv[q];  // r
        acc[0][q] += sv[q] * sv[q];
        acc[1][q] += hv[q] * sv[q];
      }
      store_vec<T, VEC>(x + i * m + c, xv);
      store_vec<T, VEC>(r + i * m + c, sv);
    }
  }
  const int32_t it = cs.it[0] + 1;  // the iteration this launch completes
  reduce_cols<T, 2, VEC, LANES>(acc, m, partials, counter, [&](int l, const ColTotals<T, 2> &tt) {
    const int st = cs.state[l];
    if (st == ST_HALF) {
      cs.state[l] = ST_DONE;
      cs.status[l] = ENS_COL_CONVERGED;
      return;
    }
    if (st != ST_ACTIVE) return;
    const T rn2 = tt.v[0][l], rr = tt.v[1][l];
    cs.rho_old[l] = cs.rho[l];
    cs.rn2[l] = rn2;
    if (!isfinite(rn2)) {
      cs.state[l] = ST_DONE;
      cs.status[l] = ENS_COL_NONFINITE;
    } else if (rn2 <= cs.thr2[l]) {
      cs.state[l] = ST_DONE;
      cs.status[l] = ENS_COL_CONVERGED;
    } else if (cs.omega[l] == T(0)) {
      cs.state[l] = ST_DONE;
      cs.status[l] = ENS_COL_BREAKDOWN;
    } else if (it < max_iter) {  // the next iteration begins: rho and its breakdown test
      if (!isfinite(rr)) {
        cs.state[l] = ST_DONE;
        cs.status[l] = ENS_COL_NONFINITE;
        cs.iters[l] = it + 1;
      } else if (fabs(rr) <= Tiny<T>::v * sqrt(cs.rh2[l]) * sqrt(rn2)) {
        cs.state[l] = ST_DONE;
        cs.status[l] = ENS_COL_BREAKDOWN;
        cs.iters[l] = it + 1;
      } else {
        cs.rho[l] = rr;
      }
    }
  }, [&]() {
    int32_t any = 0;
    for (int l = 0; l < m; ++l) any |= cs.state[l] != ST_DONE;
    cs.it[0] = it;
    cs.it[1] = any && it < max_iter;
  });
}

// Loop condition of the device-driven iteration graph (a conditional WHILE node).
static __global__ void k_loop_cond(cudaGraphConditionalHandle h, const int32_t *__restrict__ it) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h, it[1] ? 1u : 0u);
}

// ----------------------------------------------------------------------------- finishing
// Column sums of x (singular operators: the solution is normalised to zero mean).
template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    k_colsum(MatView A, int32_t m, const typename Arith::T *__restrict__ x, typename Arith::T inv_n,
             Cols<typename Arith::T> cs, typename Arith::T *partials, unsigned *counter) {
  using T = typename Arith::T;
  const int32_t c = (threadIdx.x % LANES) * VEC;
  T acc[1][VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) acc[0][q] = T(0);
  if (c < m) {
    ENS_ROWS(i) {
      T xv[VEC];
      load_vec<T, VEC>(x + i * m + c, xv);
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[0][q] += xv[q];
    }
  }
  reduce_cols<T, 1, VEC, LANES>(acc, m, partials, counter,
                                [&](int l, const ColTotals<T, 1> &t) { cs.mean[l] = t.v[0][l] * inv_n; });
}

// x = 0 for zero right-hand sides; x -= mean for singular operators (columns that iterated).
template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    k_fix(MatView A, int32_t m, typename Arith::T *x, int singular, Cols<typename Arith::T> cs) {
  using T = typename Arith::T;
  const int32_t c = (threadIdx.x % LANES) * VEC;
  if (c >= m) return;
  bool zero[VEC];
  T sub[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    const int fl = cs.flags[c + q];
    zero[q] = (fl & FL_ZERO_B) != 0;
    sub[q] = (singular && !(fl & FL_EARLY)) ? cs.mean[c + q] : T(0);
  }
  ENS_ROWS(i) {
    T xv[VEC];
    load_vec_rw<T, VEC>(x + i * m + c, xv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) xv[q] = zero[q] ? T(0) : xv[q] - sub[q];
    store_vec<T, VEC>(x + i * m + c, xv);
  }
}

// True residual ||b - A x||^2 per column -> relres. With `outer` set (mixed mode) the residual is
// also stored in r and the outer convergence test runs on it.
template <typename Arith, int VEC, int LANES>
__global__ void ENS_TILE_BOUNDS(Arith)
    k_resid(MatView A, int32_t m, const typename Arith::T *__restrict__ b, const typename Arith::T *__restrict__ x,
            typename Arith::T *__restrict__ r, int outer, Cols<typename Arith::T> cs, typename Arith::T *partials,
            unsigned *counter, uint32_t mask) {
  using T = typename Arith::T;
  T acc[1][VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) acc[0][q] = T(0);
  tile_rows<Arith, VEC, LANES>(A, m, x, mask, [&](int64_t i, int32_t cc, const T (&ax)[VEC]) {
    T y[VEC], bv[VEC];
    load_vec<T, VEC>(b + i * m + cc, bv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      y[q] = bv[q] - ax[q];
      acc[0][q] += y[q] * y[q];
    }
    if (r) store_vec<T, VEC>(r + i * m + cc, y);
  });
  reduce_cols<T, 1, VEC, LANES>(acc, m, partials, counter, [&](int l, const ColTotals<T, 1> &t) {
    const T rr = t.v[0][l];
    if (outer) {
      if (cs.state[l] != ST_ACTIVE) return;
      cs.rn2[l] = rr;
      if (!isfinite(rr)) {
        cs.state[l] = ST_DONE;
        cs.status[l] = ENS_COL_NONFINITE;
      } else if (rr <= cs.thr2[l]) {
        cs.state[l] = ST_DONE;
        cs.status[l] = ENS_COL_CONVERGED;
      }
      return;
    }
    const int fl = cs.flags[l];
    cs.relres[l] = (fl & FL_ZERO_B) ? 0.0 : (fl & FL_EARLY) ? (double)NAN : sqrt((double)rr / (double)cs.bn2[l]);
  });
}

// ----------------------------------------------------------------------------- mixed precision
// Inner right-hand side: r32 = r / ||r|| for active outer columns, 0 otherwise (so finished
// columns start converged in the inner solve).
template <int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    k_to32(int32_t n, int32_t m, const double *__restrict__ r, float *__restrict__ r32, Cols<double> cs) {
  const int32_t c = (threadIdx.x % LANES) * VEC;
  if (c >= m) return;
  double sc[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) sc[q] = cs.state[c + q] == ST_ACTIVE ? rsqrt(cs.rn2[c + q]) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / LANES) + threadIdx.x / LANES; i < n;
       i += (int64_t)gridDim.x * (kThreads / LANES)) {
    double rv[VEC];
    float o[VEC];
    load_vec<double, VEC>(r + i * m + c, rv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) o[q] = (float)(rv[q] * sc[q]);
    store_vec<float, VEC>(r32 + i * m + c, o);
  }
}

// Mixed precision, after an inner solve: an inner solve that broke down in its first iteration,
// before any update, returns d = 0 and leaves the outer residual as it was, so the next refinement
// step would repeat it exactly. Such a column ends with BREAKDOWN (x keeps its current iterate),
// as the FP64 solve of the same column does.
static __global__ void k_inner_nostep(int32_t mp, Cols<double> outer, const int32_t *__restrict__ inner_status,
                                      const int32_t *__restrict__ inner_flags) {
  for (int l = threadIdx.x; l < mp; l += blockDim.x)
    if (outer.state[l] == ST_ACTIVE && inner_status[l] == ENS_COL_BREAKDOWN && (inner_flags[l] & FL_NOSTEP)) {
      outer.state[l] = ST_DONE;
      outer.status[l] = ENS_COL_BREAKDOWN;
    }
}

// x += ||r|| d for active outer columns (the FP64 correction step).
template <int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    k_correct(int32_t n, int32_t m, double *x, const float *__restrict__ d, Cols<double> cs,
              const int32_t *__restrict__ inner_status) {
  const int32_t c = (threadIdx.x % LANES) * VEC;
  if (c >= m) return;
  double sc[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q)  // an inner solve that met a non-finite value contributes nothing
    sc[q] = cs.state[c + q] == ST_ACTIVE && inner_status[c + q] != ENS_COL_NONFINITE ? sqrt(cs.rn2[c + q]) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / LANES) + threadIdx.x / LANES; i < n;
       i += (int64_t)gridDim.x * (kThreads / LANES)) {
    double xv[VEC];
    float dv[VEC];
    load_vec_rw<double, VEC>(x + i * m + c, xv);
    load_vec<float, VEC>(d + i * m + c, dv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) xv[q] = sc[q] != 0.0 ? xv[q] + sc[q] * (double)dv[q] : xv[q];
    store_vec<double, VEC>(x + i * m + c, xv);
  }
}

// Copy between the caller's stride-m block and the internal stride-mp block (zero padding).
static __global__ void k_pad(int64_t n, int32_t m, int32_t mp, const double *__restrict__ src, double *__restrict__ dst) {
  const int64_t total = n * mp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / mp;
    const int32_t l = (int32_t)(e - i * mp);
    dst[e] = l < m ? src[i * m + l] : 0.0;
  }
}
static __global__ void k_unpad(int64_t n, int32_t m, int32_t mp, const double *__restrict__ src, double *__restrict__ dst) {
  const int64_t total = n * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / m;
    const int32_t l = (int32_t)(e - i * m);
    dst[e] = src[i * mp + l];
  }
}

// ----------------------------------------------------------------------------- host side
// VEC (1, 2, or 4 where kVec4) and LANES (a power of two) as compile-time constants.
template <bool kVec4 = false, typename F>
cudaError_t with_vl(int vec, int lanes, F &&f) {
  using std::integral_constant;
  if (vec == 1) return f(integral_constant<int, 1>{}, integral_constant<int, 1>{});
  if constexpr (kVec4) {
    if (vec == 4) {
      switch (lanes) {
        case 1: return f(integral_constant<int, 4>{}, integral_constant<int, 1>{});
        case 2: return f(integral_constant<int, 4>{}, integral_constant<int, 2>{});
        case 4: return f(integral_constant<int, 4>{}, integral_constant<int, 4>{});
        case 8: return f(integral_constant<int, 4>{}, integral_constant<int, 8>{});
        default: return f(integral_constant<int, 4>{}, integral_constant<int, 16>{});
      }
    }
  }
  switch (lanes) {
    case 1: return f(integral_constant<int, 2>{}, integral_constant<int, 1>{});
    case 2: return f(integral_constant<int, 2>{}, integral_constant<int, 2>{});
    case 4: return f(integral_constant<int, 2>{}, integral_constant<int, 4>{});
    case 8: return f(integral_constant<int, 2>{}, integral_constant<int, 8>{});
    case 16: return f(integral_constant<int, 2>{}, integral_constant<int, 16>{});
    default: return f(integral_constant<int, 2>{}, integral_constant<int, 32>{});
  }
}

// Stream-ordered scratch allocation, released when the object goes out of scope.
// Scratch memory of one solve call: stream-ordered allocations released at the end of the call,
// or, with a caller-provided workspace (ens_solve_opts.workspace), consecutive 256-byte aligned
// pieces of that memory (nothing is allocated). Either way the bytes taken are recorded for
// ens_last_workspace_bytes(); a workspace that is too small ends the call with ENS_ERR_BUDGET.
struct Scratch {
  cudaStream_t s;
  std::vector<void *> ptrs;
  char *arena = nullptr;
  size_t cap = 0, used = 0;
  bool overflow = false;
  explicit Scratch(cudaStream_t st) : s(st) {}
  Scratch(cudaStream_t st, const ens_solve_opts &o) : s(st), arena((char *)o.workspace), cap(o.workspace_bytes) {}
  ~Scratch() {
    for (void *p : ptrs) cudaFreeAsync(p, s);
    record_workspace(used, overflow);
  }
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    const size_t bytes = (std::max<size_t>(count, 1) * sizeof(T) + 255) / 256 * 256;
    if (arena) {
      if (overflow || used + bytes > cap) {
        overflow = true;
        used += bytes;  // what the call needed up to this request
        return cudaErrorMemoryAllocation;
      }
      *p = (T *)(arena + used);
      used += bytes;
      return cudaSuccess;
    }
    void *q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, bytes, s);
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    used += bytes;
    *p = (T *)q;
    return cudaSuccess;
  }
};

inline MatView view_of(const ens_matrix *A) {
  return MatView{(int32_t)A->n, A->row, A->col, A->val, A->val32, A->valsplit, A->dinv, A->dinv32};
}

template <typename T>
cudaError_t alloc_cols(Scratch &sc, int m, Cols<T> &cs) {
  cudaError_t e = cudaSuccess;
  T **tp[] = {&cs.rho, &cs.rho_old, &cs.alpha, &cs.omega, &cs.bn2, &cs.thr2, &cs.rh2, &cs.rn2, &cs.tol, &cs.mean};
  for (T **p : tp)
    if (e == cudaSuccess) e = sc.get(p, m);
  int32_t **ip[] = {&cs.state, &cs.iters, &cs.status, &cs.flags};
  for (int32_t **p : ip)
    if (e == cudaSuccess) e = sc.get(p, m);
  if (e == cudaSuccess) e = sc.get(&cs.relres, m);
  if (e == cudaSuccess) e = sc.get(&cs.it, 2);
  return e;
}

// One BiCGStab run over an mp-wide internal block in arithmetic Arith (float64 split/native or
// float32). b, x are device blocks of stride mp.
// ----------------------------------------------------------------------------- AMG V-cycle
// One V-cycle of the aggregation hierarchy (amg.cu) on an mp-wide block, every level's product a
// GSpMV of that level's matrix over the whole block:
//   z = S(r);  z += P V(P^T (r - A z));  z += S(r - A z);   coarsest level: z = S_coarse(r)
// with S the Jacobi-scaled Chebyshev iteration (first term below, further steps by k_cheb).

// d0 = D^-1 src / theta; z = d0 (or z += d0 for the post-smoothing).
template <typename Arith, int VEC, int LANES, bool ADD>
__global__ void __launch_bounds__(kThreads)
    k_amg_first(MatView A, int32_t m, const typename Arith::T *__restrict__ src, typename Arith::T *__restrict__ da,
                typename Arith::T *z, typename Arith::T inv_theta) {
  using T = typename Arith::T;
  const int32_t c = (threadIdx.x % LANES) * VEC;
  if (c >= m) return;
  ENS_ROWS(i) {
    T sv[VEC], zv[VEC];
    load_vec<T, VEC>(src + i * m + c, sv);
    const T sc = Arith::dinv(A, i) * inv_theta;
    if (ADD) load_vec_rw<T, VEC>(z + i * m + c, zv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      sv[q] *= sc;
      zv[q] = ADD ? zv[q] + sv[q] : sv[q];
    }
    store_vec<T, VEC>(da + i * m + c, sv);
    store_vec<T, VEC>(z + i * m + c, zv);
  }
}

// The coarsest level's whole smoothing z = S_steps(src) in one block (levels of at most
// kCoarseBlockRows rows): the first term of k_amg_first and then every step of k_cheb, with a block
// barrier where the separate launches had a kernel boundary. A step's product reads the previous
// step's d, written in this launch, so X is loaded with plain (coherent) loads and multiplied with
// native FMA (float values for the float32 solver): a few thousand products per step, where one
// launch per step cost more than its work.
constexpr int kCoarseBlockRows = 2048;
constexpr int kMaxCoarseSteps = 64;
template <typename T>
struct CoarseCoefs {
  T c1[kMaxCoarseSteps], c2[kMaxCoarseSteps];  // step k >= 1
};

template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    k_amg_coarse(MatView A, int32_t m, const typename Arith::T *__restrict__ src, typename Arith::T *da,
                 typename Arith::T *db, typename Arith::T *res, typename Arith::T *z, typename Arith::T inv_theta,
                 CoarseCoefs<typename Arith::T> cf, int32_t steps) {
  using T = typename Arith::T;
  constexpr int G = kThreads / LANES;
  const int32_t c = (threadIdx.x % LANES) * VEC;
  const bool act = c < m;
  if (act)
    for (int64_t i = threadIdx.x / LANES; i < A.n; i += G) {
      T sv[VEC];
      load_vec<T, VEC>(src + i * m + c, sv);
      const T sc = Arith::dinv(A, i) * inv_theta;
#pragma unroll
      for (int q = 0; q < VEC; ++q) sv[q] *= sc;
      store_vec<T, VEC>(da + i * m + c, sv);
      store_vec<T, VEC>(z + i * m + c, sv);
    }
  __syncthreads();
  T *din = da, *dout = db;
  for (int k = 1; k < steps; ++k) {
    const bool first = k == 1, last = k == steps - 1;
    const T c1 = cf.c1[k], c2 = cf.c2[k];
    if (act)
      for (int64_t i = threadIdx.x / LANES; i < A.n; i += G) {
        T w[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) w[q] = T(0);
        for (int32_t j = A.rp[i]; j < A.rp[i + 1]; ++j) {
          T a;
          if constexpr (std::is_same<T, float>::value)
            a = A.val32[j];
          else
            a = A.val[j];
          T x[VEC];
          load_vec_rw<T, VEC>(din + (int64_t)A.ci[j] * m + c, x);
#pragma unroll
          for (int q = 0; q < VEC; ++q) w[q] = fma(a, x[q], w[q]);
        }
        T di[VEC], rs[VEC], zv[VEC], dn[VEC];
        load_vec_rw<T, VEC>(din + i * m + c, di);
        if (first)
          load_vec<T, VEC>(src + i * m + c, rs);
        else
          load_vec_rw<T, VEC>(res + i * m + c, rs);
        load_vec_rw<T, VEC>(z + i * m + c, zv);
        const T dv = Arith::dinv(A, i);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          rs[q] -= w[q];
          dn[q] = c1 * di[q] + c2 * (dv * rs[q]);
          zv[q] += dn[q];
        }
        store_vec<T, VEC>(z + i * m + c, zv);
        if (!last) {
          store_vec<T, VEC>(res + i * m + c, rs);
          store_vec<T, VEC>(dout + i * m + c, dn);
        }
      }
    __syncthreads();
    T *t = din;
    din = dout;
    dout = t;
  }
}

// res = r - A z
template <typename Arith, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads, ChebBlocks<Arith, VEC>::value)
    k_amg_resid(MatView A, int32_t m, const typename Arith::T *__restrict__ z, const typename Arith::T *__restrict__ r,
                typename Arith::T *__restrict__ res, uint32_t mask) {
  using T = typename Arith::T;
  tile_rows<Arith, VEC, LANES>(A, m, z, mask, [&](int64_t i, int32_t cc, const T (&w)[VEC]) {
    T rv[VEC];
    load_vec<T, VEC>(r + i * m + cc, rv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) rv[q] -= w[q];
    store_vec<T, VEC>(res + i * m + cc, rv);
  });
}

// Both updates of a two-update Chebyshev smoothing in one pass, from the column-scaled copy
// As = A D^-1 of the level (A d0 = As src / theta for d0 = D^-1 src / theta):
//   d0 = D^-1 src / theta,  res1 = src - (As src) / theta,  d1 = c1 d0 + c2 D^-1 res1,
//   z = d0 + d1  (ADD: z += d0 + d1).
template <typename Arith, int VEC, int LANES, bool ADD>
__global__ void __launch_bounds__(kThreads, ChebBlocks<Arith, VEC>::value)
    k_amg_smooth2(MatView As, MatView A, int32_t m, const typename Arith::T *__restrict__ src, typename Arith::T *z,
                  typename Arith::T inv_theta, typename Arith::T c1, typename Arith::T c2, uint32_t mask) {
  using T = typename Arith::T;
  tile_rows<Arith, VEC, LANES>(As, m, src, mask, [&](int64_t i, int32_t cc, const T (&w)[VEC]) {
    T sv[VEC], zv[VEC];
    load_vec<T, VEC>(src + i * m + cc, sv);
    if (ADD) load_vec_rw<T, VEC>(z + i * m + cc, zv);
    const T dv = Arith::dinv(A, i);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      const T d0 = dv * sv[q] * inv_theta;
      const T r1 = sv[q] - w[q] * inv_theta;
      const T d1 = c1 * d0 + c2 * (dv * r1);
      zv[q] = ADD ? zv[q] + (d0 + d1) : d0 + d1;
    }
    store_vec<T, VEC>(z + i * m + cc, zv);
  });
}

// rc_I = sum of res_i over the rows i of aggregate I (ascending rows: a fixed order).
template <typename T, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    k_amg_restrict(int64_t nc, int32_t m, const int32_t *__restrict__ ptr, const int32_t *__restrict__ mem,
                   const T *__restrict__ res, T *__restrict__ rc) {
  const int32_t c = (threadIdx.x % LANES) * VEC;
  if (c >= m) return;
  for (int64_t I = (int64_t)blockIdx.x * (kThreads / LANES) + threadIdx.x / LANES; I < nc;
       I += (int64_t)gridDim.x * (kThreads / LANES)) {
    T acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = T(0);
    for (int32_t t = ptr[I]; t < ptr[I + 1]; ++t) {
      T v[VEC];
      load_vec<T, VEC>(res + (int64_t)mem[t] * m + c, v);
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] += v[q];
    }
    store_vec<T, VEC>(rc + I * m + c, acc);
  }
}

// z_i += zc_agg(i)
template <typename T, int VEC, int LANES>
__global__ void __launch_bounds__(kThreads)
    k_amg_prolong(int64_t n, int32_t m, const int32_t *__restrict__ agg, const T *__restrict__ zc, T *z) {
  const int32_t c = (threadIdx.x % LANES) * VEC;
  if (c >= m) return;
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / LANES) + threadIdx.x / LANES; i < n;
       i += (int64_t)gridDim.x * (kThreads / LANES)) {
    T zv[VEC], cv[VEC];
    load_vec_rw<T, VEC>(z + i * m + c, zv);
    load_vec<T, VEC>(zc + (int64_t)agg[i] * m + c, cv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) zv[q] += cv[q];
    store_vec<T, VEC>(z + i * m + c, zv);
  }
}

template <typename Arith>
struct AmgCycle {
  static constexpr bool kVec4 = std::is_same<Arith, ArithF32>::value;  // float32 blocks: 4 columns per lane
  using T = typename Arith::T;
  struct Level {
    MatView A, As;
    bool has_as = false;
    int64_t n = 0, nc = 0;
    const int32_t *agg = nullptr, *ptr = nullptr, *mem = nullptr;
    uint32_t mask = 0, as_mask = 0;
    bool split = false;     // float64 split arithmetic usable on this level
    bool as_split = false;  // ... and on its scaled copy
    int grid = 0, egrid = 0, cgrid = 0, sms = 1;
    T *r = nullptr, *z = nullptr, *res = nullptr, *cres = nullptr, *da = nullptr, *db = nullptr;
  };
  std::vector<Level> lev;
  ens_amg_opts o;
  int mp = 0, vec = 2, lanes = 1;

  cudaError_t setup(Scratch &sc, const ens_amg *H, int mp_, int vec_, int lanes_) {
    o = H->opts;
    mp = mp_;
    vec = vec_;
    lanes = lanes_;
    lev.clear();
    cudaError_t e = cudaSuccess;
    for (size_t l = 0; l < H->lev.size() && e == cudaSuccess; ++l) {
      const ens_amg_lev &h = H->lev[l];
      Level L;
      L.A = view_of(h.A);
      L.n = h.A->n;
      L.nc = h.nc;
      L.agg = h.agg;
      L.ptr = h.agg_ptr;
      L.mem = h.members;
      L.split = use_split(h.A);
      L.mask = std::is_same<Arith, ArithF64Split>::value && L.split ? share_mask(native_share(h.A, mp)) : 0u;
      if (h.As) {
        L.has_as = true;
        L.As = view_of(h.As);
        L.as_split = use_split(h.As);
        L.as_mask = std::is_same<Arith, ArithF64Split>::value && L.as_split ? share_mask(native_share(h.As, mp)) : 0u;
      }
      const int64_t rows_per_block = kThreads / lanes;
      const int64_t sms = h.A->num_sms;
      L.grid = (int)std::max<int64_t>(1, std::min<int64_t>((L.n + kTileRows - 1) / kTileRows, sms * LightBlocks<Arith>::value));
      L.sms = (int)sms;
      L.egrid = (int)std::max<int64_t>(1, std::min<int64_t>((L.n + rows_per_block - 1) / rows_per_block, sms * 8));
      L.cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((L.nc + rows_per_block - 1) / rows_per_block, sms * 8));
      const size_t blk = (size_t)L.n * mp;
      if (l > 0) {
        if (e == cudaSuccess) e = sc.get(&L.r, blk);
        if (e == cudaSuccess) e = sc.get(&L.z, blk);
      }
      T **bufs[] = {&L.res, &L.cres, &L.da, &L.db};
      for (T **b : bufs)
        if (e == cudaSuccess) e = sc.get(b, blk);
      lev.push_back(L);
    }
    return e;
  }

  // z (+)= S(src) on level l with `steps` Chebyshev updates, level arithmetic Ar.
  template <typename Ar, int V, int Ln>
  void smooth(const Level &L, const T *src, T *z, bool add, int steps, cudaStream_t st) {
    const double theta = 0.5 * (o.cheb_hi + o.cheb_lo), delta = 0.5 * (o.cheb_hi - o.cheb_lo);
    if (steps == 2 && L.has_as) {  // both updates in one pass over the scaled copy
      const double sigma = theta / delta, rho_prev = 1.0 / sigma, rho = 1.0 / (2.0 * sigma - rho_prev);
      const T c1 = (T)(rho * rho_prev), c2 = (T)(2.0 * rho / delta), it = (T)(1.0 / theta);
      if constexpr (std::is_same<Ar, ArithF64Split>::value || std::is_same<Ar, ArithF64Hybrid>::value) {
        if (!L.as_split) {  // the scaled copy's values leave the split range: native products
          if (add)
            k_amg_smooth2<ArithF64Native, V, Ln, true><<<L.grid, kThreads, 0, st>>>(L.As, L.A, mp, src, z, it, c1, c2, 0u);
          else
            k_amg_smooth2<ArithF64Native, V, Ln, false><<<L.grid, kThreads, 0, st>>>(L.As, L.A, mp, src, z, it, c1, c2, 0u);
          return;
        }
      }
      if constexpr (std::is_same<Ar, ArithF64Split>::value && V == 2 && Ln >= 2) {
        if (mp % 4 == 0 && launch_amg_smooth2_4_split(Ln / 2, add, L.As, L.A, mp, src, z, it, c1, c2, L.as_mask, L.sms,
                                                      (L.n + kTileRows - 1) / kTileRows, st))
          return;
      }
      if (add)
        k_amg_smooth2<Ar, V, Ln, true><<<L.grid, kThreads, 0, st>>>(L.As, L.A, mp, src, z, it, c1, c2, L.as_mask);
      else
        k_amg_smooth2<Ar, V, Ln, false><<<L.grid, kThreads, 0, st>>>(L.As, L.A, mp, src, z, it, c1, c2, L.as_mask);
      return;
    }
    if (add)
      k_amg_first<Ar, V, Ln, true><<<L.egrid, kThreads, 0, st>>>(L.A, mp, src, L.da, z, (T)(1.0 / theta));
    else
      k_amg_first<Ar, V, Ln, false><<<L.egrid, kThreads, 0, st>>>(L.A, mp, src, L.da, z, (T)(1.0 / theta));
    const double sigma = theta / delta;
    double rho_prev = 1.0 / sigma;
    T *din = L.da, *dout = L.db;
    for (int k = 1; k < steps; ++k) {
      const double rho = 1.0 / (2.0 * sigma - rho_prev);
      const T c1 = (T)(rho * rho_prev), c2 = (T)(2.0 * rho / delta);
      const bool first = k == 1, last = k == steps - 1;
      bool done = false;
      if constexpr (std::is_same<Ar, ArithF64Split>::value && V == 2 && Ln >= 2) {
        if (mp % 4 == 0)
          done = launch_cheb4_split(Ln / 2, first, last, L.A, mp, din, dout, src, L.cres, z, c1, c2, L.mask, L.sms,
                                    (L.n + kTileRows - 1) / kTileRows, st);
      }
      if (done)
        ;
      else if (first && last)
        k_cheb<Ar, V, Ln, true, true><<<L.grid, kThreads, 0, st>>>(L.A, mp, din, dout, src, L.cres, z, c1, c2, L.mask);
      else if (first)
        k_cheb<Ar, V, Ln, true, false><<<L.grid, kThreads, 0, st>>>(L.A, mp, din, dout, src, L.cres, z, c1, c2, L.mask);
      else if (last)
        k_cheb<Ar, V, Ln, false, true><<<L.grid, kThreads, 0, st>>>(L.A, mp, din, dout, src, L.cres, z, c1, c2, L.mask);
      else
        k_cheb<Ar, V, Ln, false, false><<<L.grid, kThreads, 0, st>>>(L.A, mp, din, dout, src, L.cres, z, c1, c2, L.mask);
      std::swap(din, dout);
      rho_prev = rho;
    }
  }

  // L.res = r - A z on level L
  template <typename Ar, int V, int Ln>
  void resid(const Level &L, const T *z, const T *r, cudaStream_t st) {
    if constexpr (std::is_same<Ar, ArithF64Split>::value && V == 2 && Ln >= 2) {
      if (mp % 4 == 0 &&
          launch_amg_resid4_split(Ln / 2, L.A, mp, z, r, L.res, L.mask, L.sms, (L.n + kTileRows - 1) / kTileRows, st))
        return;
    }
    k_amg_resid<Ar, V, Ln><<<L.grid, kThreads, 0, st>>>(L.A, mp, z, r, L.res, L.mask);
  }

  template <typename Ar, int V, int Ln>
  void level_cycle(size_t l, const T *r, T *z, cudaStream_t st) {
    const Level &L = lev[l];
    if (l + 1 == lev.size()) {
      if (L.n <= kCoarseBlockRows && o.coarse_steps <= kMaxCoarseSteps) {  // one block, one launch
        const double theta = 0.5 * (o.cheb_hi + o.cheb_lo), delta = 0.5 * (o.cheb_hi - o.cheb_lo);
        const double sigma = theta / delta;
        double rho_prev = 1.0 / sigma;
        CoarseCoefs<T> cf{};
        for (int k = 1; k < o.coarse_steps; ++k) {
          const double rho = 1.0 / (2.0 * sigma - rho_prev);
          cf.c1[k] = (T)(rho * rho_prev);
          cf.c2[k] = (T)(2.0 * rho / delta);
          rho_prev = rho;
        }
        k_amg_coarse<Ar, V, Ln><<<1, kThreads, 0, st>>>(L.A, mp, r, L.da, L.db, L.cres, z, (T)(1.0 / theta), cf,
                                                        o.coarse_steps);
        return;
      }
      this->template smooth<Ar, V, Ln>(L, r, z, false, o.coarse_steps, st);
      return;
    }
    const Level &C = lev[l + 1];
    this->template smooth<Ar, V, Ln>(L, r, z, false, o.smooth_steps, st);
    this->template resid<Ar, V, Ln>(L, z, r, st);
    k_amg_restrict<T, V, Ln><<<L.cgrid, kThreads, 0, st>>>(L.nc, mp, L.ptr, L.mem, L.res, C.r);
    this->template cycle<V, Ln>(l + 1, C.r, C.z, st);
    k_amg_prolong<T, V, Ln><<<L.egrid, kThreads, 0, st>>>(L.n, mp, L.agg, C.z, z);
    this->template resid<Ar, V, Ln>(L, z, r, st);
    this->template smooth<Ar, V, Ln>(L, L.res, z, true, o.smooth_steps, st);
  }

  // Levels where the split arithmetic cannot run (value range) use native DFMA.
  template <int V, int Ln>
  void cycle(size_t l, const T *r, T *z, cudaStream_t st) {
    if constexpr (std::is_same<Arith, ArithF64Split>::value || std::is_same<Arith, ArithF64Hybrid>::value) {
      if (!lev[l].split) {
        this->template level_cycle<ArithF64Native, V, Ln>(l, r, z, st);
        return;
      }
    }
    this->template level_cycle<Arith, V, Ln>(l, r, z, st);
  }

  // z = V(r) on the fine level (capturable: kernel launches only).
  cudaError_t apply(const T *r, T *z, cudaStream_t st) {
    return with_vl<kVec4>(vec, lanes, [&](auto Vc, auto Lc) {
      constexpr int V = decltype(Vc)::value, Ln = decltype(Lc)::value;
      this->template cycle<V, Ln>(0, r, z, st);
      return cudaGetLastError();
    });
  }
};

template <typename Arith>
struct Bicg {
  // float32 blocks whose padded width is a multiple of 4 take four columns per lane (16-byte
  // accesses, as the standalone float32 GSpMV); float64 blocks two.
  static constexpr bool kVec4 = std::is_same<Arith, ArithF32>::value;
  using T = typename Arith::T;
  MatView A;
  int64_t n = 0;
  int mp = 0, vec = 2, lanes = 1, grid = 0, tgrid = 0, lgrid = 0;  // grid: streaming kernels, tgrid / lgrid: GSpMV kernels
  int num_sms = 1;
  bool prec = false;
  bool use_amg = false;
  AmgCycle<Arith> amg;
  int cheb_steps = 4;
  uint32_t mask = 0;  // native-DFMA sweeps of the split arithmetic (hybrid tiles)
  double theta = 1, delta = 1;
  cudaStream_t s = nullptr;
  T *r, *rh, *p, *v, *ph, *s_, *sh, *t, *da, *db, *res;
  T *partials;
  unsigned *counter;
  Cols<T> cs;

  // outer_only: just the residual block, scalars and reduction scratch (mixed-mode outer loop).
  cudaError_t setup(Scratch &sc, const ens_matrix *M, int mp_, const ens_solve_opts &o, cudaStream_t st,
                    bool outer_only = false) {
    A = view_of(M);
    n = M->n;
    mp = mp_;
    mask = std::is_same<Arith, ArithF64Split>::value ? share_mask(native_share(M, mp_)) : 0u;
    s = st;
    vec = mp == 1 ? 1 : (kVec4 && mp % 4 == 0) ? 4 : 2;
    lanes = 1;
    while (lanes * vec < mp) lanes <<= 1;
    num_sms = M->num_sms;
    grid = M->num_sms * 4;
    tgrid = M->num_sms * TileBlocks<Arith>::value;
    lgrid = M->num_sms * LightBlocks<Arith>::value;
    prec = o.precond == ENS_PRECOND_CHEBYSHEV;
    cheb_steps = o.cheb_steps;
    theta = 0.5 * (o.cheb_hi + o.cheb_lo);
    delta = 0.5 * (o.cheb_hi - o.cheb_lo);
    const size_t blk = (size_t)n * mp;
    cudaError_t e = cudaSuccess;
    r = rh = p = v = ph = s_ = sh = t = da = db = res = nullptr;
    if (outer_only) {
      prec = false;
      e = sc.get(&r, blk);
    } else {
      T **bufs[] = {&r, &rh, &p, &v, &s_, &t};
      for (T **b : bufs)
        if (e == cudaSuccess) e = sc.get(b, blk);
    }
    use_amg = !outer_only && o.precond == ENS_PRECOND_AMG && M->amg != nullptr;
    if (outer_only) {
    } else if (prec) {
      T **pb[] = {&ph, &sh, &da, &db, &res};
      for (T **b : pb)
        if (e == cudaSuccess) e = sc.get(b, blk);
    } else if (use_amg) {
      if (e == cudaSuccess) e = sc.get(&ph, blk);
      if (e == cudaSuccess) e = sc.get(&sh, blk);
      if (e == cudaSuccess) e = amg.setup(sc, M->amg, mp, vec, lanes);
    } else {
      ph = p;
      sh = s_;
      da = db = res = nullptr;
    }
    if (e == cudaSuccess) e = sc.get(&partials, (size_t)std::max(grid, tgrid) * 3 * kMaxSolveM);
    if (e == cudaSuccess) e = sc.get(&counter, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = alloc_cols(sc, mp, cs);
    return e;
  }

  // Per-column tolerances to the device (a host copy: done before any graph capture).
  cudaError_t upload_tol(const std::vector<T> &tol) {
    return cudaMemcpyAsync(cs.tol, tol.data(), mp * sizeof(T), cudaMemcpyHostToDevice, s);
  }

  // r = b - A x, rhat = r, p = v = 0, column statuses (capturable: memsets and one kernel).
  cudaError_t enqueue_start(const T *b, T *x, bool x0_zero, int singular, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (p) e = cudaMemsetAsync(p, 0, (size_t)n * mp * sizeof(T), st);
    if (e == cudaSuccess && v) e = cudaMemsetAsync(v, 0, (size_t)n * mp * sizeof(T), st);
    if (e != cudaSuccess) return e;
    const T incompat = (T)(1e-10 * std::sqrt((double)n));
    return with_vl<kVec4>(vec, lanes, [&](auto Vc, auto Lc) {
      constexpr int V = decltype(Vc)::value, L = decltype(Lc)::value;
      k_start<Arith, V, L><<<tgrid, kThreads, 0, st>>>(A, mp, b, x, r, rh, x0_zero ? 1 : 0, singular, incompat, cs,
                                                      partials, counter, mask);
      return cudaGetLastError();
    });
  }

  cudaError_t start(const T *b, T *x, bool x0_zero, int singular, const std::vector<T> &tol) {
    cudaError_t e = upload_tol(tol);
    if (e == cudaSuccess) e = enqueue_start(b, x, x0_zero, singular, s);
    return e;
  }

  // Chebyshev application z = p(D^-1 A) D^-1 src; the first term is already in da and z.
  template <int V, int L>
  void cheb(const T *src, T *z, cudaStream_t st) {
    const double sigma = theta / delta;
    double rho_prev = 1.0 / sigma;
    T *din = da, *dout = db;
    for (int k = 1; k < cheb_steps; ++k) {
      const double rho = 1.0 / (2.0 * sigma - rho_prev);
      const T c1 = (T)(rho * rho_prev), c2 = (T)(2.0 * rho / delta);
      const bool first = k == 1, last = k == cheb_steps - 1;
      bool done = false;
      if constexpr (std::is_same<Arith, ArithF64Split>::value && V == 2 && L >= 2) {
        if (mp % 4 == 0)
          done = launch_cheb4_split(L / 2, first, last, A, mp, din, dout, src, res, z, c1, c2, mask, num_sms,
                                    INT64_MAX, st);
      }
      if (done)
        ;
      else if (first && last)
        k_cheb<Arith, V, L, true, true><<<lgrid, kThreads, 0, st>>>(A, mp, din, dout, src, res, z, c1, c2, mask);
      else if (first)
        k_cheb<Arith, V, L, true, false><<<lgrid, kThreads, 0, st>>>(A, mp, din, dout, src, res, z, c1, c2, mask);
      else if (last)
        k_cheb<Arith, V, L, false, true><<<lgrid, kThreads, 0, st>>>(A, mp, din, dout, src, res, z, c1, c2, mask);
      else
        k_cheb<Arith, V, L, false, false><<<lgrid, kThreads, 0, st>>>(A, mp, din, dout, src, res, z, c1, c2, mask);
      std::swap(din, dout);
      rho_prev = rho;
    }
  }

  // One BiCGStab iteration for every column (frozen columns are no-ops); the iteration number
  // lives on the device, so the same launches can be captured once and replayed.
  cudaError_t iteration(T *x, int max_iter, cudaStream_t st) {
    const T inv_theta = (T)(1.0 / theta);
    return with_vl<kVec4>(vec, lanes, [&](auto Vc, auto Lc) {
      constexpr int V = decltype(Vc)::value, L = decltype(Lc)::value;
      if (prec) {
        k_p<Arith, V, L, true><<<grid, kThreads, 0, st>>>(A, mp, r, p, v, da, ph, inv_theta, cs);
        cheb<V, L>(p, ph, st);
      } else {
        k_p<Arith, V, L, false><<<grid, kThreads, 0, st>>>(A, mp, r, p, v, da, ph, inv_theta, cs);
        if (use_amg) amg.template cycle<V, L>(0, p, ph, st);
      }
      k_v<Arith, V, L><<<tgrid, kThreads, 0, st>>>(A, mp, ph, v, rh, cs, partials, counter, mask);
      if (prec) {
        k_s<Arith, V, L, true><<<grid, kThreads, 0, st>>>(A, mp, r, v, s_, da, sh, inv_theta, cs, partials, counter);
        cheb<V, L>(s_, sh, st);
      } else {
        k_s<Arith, V, L, false><<<grid, kThreads, 0, st>>>(A, mp, r, v, s_, da, sh, inv_theta, cs, partials, counter);
        if (use_amg) amg.template cycle<V, L>(0, s_, sh, st);
      }
      k_t<Arith, V, L><<<tgrid, kThreads, 0, st>>>(A, mp, sh, t, s_, cs, partials, counter, mask);
      k_xr<Arith, V, L><<<grid, kThreads, 0, st>>>(A, mp, x, ph, sh, s_, t, r, rh, max_iter, cs, partials, counter);
      return cudaGetLastError();
    });
  }

  cudaError_t states(std::vector<int32_t> &h) {
    h.resize(mp);
    cudaError_t e = cudaMemcpyAsync(h.data(), cs.state, mp * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  }

  static bool all_done(const std::vector<int32_t> &h) {
    for (int32_t v : h)
      if (v != ST_DONE) return false;
    return true;
  }

  cudaError_t iterations_run(int *ran) {
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, cs.it, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *ran = h;
    return e;
  }

  // Host-driven loop: launch iterations, read the column states every check_every iterations.
  cudaError_t iterate_host(T *x, int max_iter, int check_every, int *ran) {
    std::vector<int32_t> h;
    cudaError_t e = states(h);
    *ran = 0;
    if (e != cudaSuccess || all_done(h)) return e;
    for (int it = 1; it <= max_iter; ++it) {
      e = iteration(x, max_iter, s);
      if (e != cudaSuccess) return e;
      if (it % check_every == 0 || it == max_iter) {
        e = states(h);
        if (e != cudaSuccess) return e;
        if (all_done(h)) break;
      }
    }
    return iterations_run(ran);
  }

  // Device-driven loop: one iteration is captured as the body of a conditional WHILE graph node
  // whose condition (some column active and fewer than max_iter iterations) is set on the device
  // by k_loop_cond; one graph launch runs the whole solve with no host round trip. The loop ends
  // after at most max_iter iterations.
  //
  // The instantiated loop is kept and replayed by later calls on the same x and max_iter (the mixed
  // solver's outer steps rerun the same inner loop on the same buffers; every value that changes
  // between them lives in device memory), so it is captured and instantiated once per solve.
  struct LoopGraph {
    cudaStream_t cap = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    const void *x = nullptr;
    int max_iter = 0;
    LoopGraph() = default;
    LoopGraph(const LoopGraph &) = delete;
    LoopGraph &operator=(const LoopGraph &) = delete;
    ~LoopGraph() { release(); }
    void release() {
      if (ge) cudaGraphExecDestroy(ge);
      if (g) cudaGraphDestroy(g);
      if (cap) cudaStreamDestroy(cap);
      ge = nullptr;
      g = nullptr;
      cap = nullptr;
      x = nullptr;
    }
  } loop;

  cudaError_t build_loop(T *x, int max_iter) {
    loop.release();
    cudaError_t e = cudaStreamCreateWithFlags(&loop.cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&loop.g, 0);
    cudaGraphConditionalHandle h{};
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, loop.g, 1, cudaGraphCondAssignDefault);
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      e = cudaGraphAddNode(&node, loop.g, nullptr, nullptr, 0, &np);
      if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(loop.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t ek = iteration(x, max_iter, loop.cap);
      if (ek == cudaSuccess) {
        k_loop_cond<<<1, 32, 0, loop.cap>>>(h, cs.it);
        ek = cudaGetLastError();
      }
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(loop.cap, &captured);
      if (e == cudaSuccess) e = ek;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&loop.ge, loop.g, 0);
    if (e == cudaSuccess) {
      loop.x = x;
      loop.max_iter = max_iter;
    } else {
      loop.release();
    }
    return e;
  }

  cudaError_t iterate_graph(T *x, int max_iter, int *ran) {
    *ran = 0;
    if (max_iter <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!loop.ge || loop.x != x || loop.max_iter != max_iter) e = build_loop(x, max_iter);
    // skip the launch when every column finished in the start phase
    std::vector<int32_t> st;
    if (e == cudaSuccess) e = states(st);
    if (e == cudaSuccess && !all_done(st)) e = cudaGraphLaunch(loop.ge, s);
    if (e == cudaSuccess) e = iterations_run(ran);
    return e;
  }

  cudaError_t iterate(T *x, int max_iter, int check_every, bool graph, int *ran) {
    return graph ? iterate_graph(x, max_iter, ran) : iterate_host(x, max_iter, check_every, ran);
  }

  cudaError_t finish(const T *b, T *x, int singular, cudaStream_t st = nullptr) {
    if (!st) st = s;
    return with_vl<kVec4>(vec, lanes, [&](auto Vc, auto Lc) {
      constexpr int V = decltype(Vc)::value, L = decltype(Lc)::value;
      if (singular) {
        k_colsum<Arith, V, L><<<grid, kThreads, 0, st>>>(A, mp, x, (T)(1.0 / (double)n), cs, partials, counter);
      }
      k_fix<Arith, V, L><<<grid, kThreads, 0, st>>>(A, mp, x, singular, cs);
      k_resid<Arith, V, L><<<tgrid, kThreads, 0, st>>>(A, mp, b, x, nullptr, 0, cs, partials, counter, mask);
      return cudaGetLastError();
    });
  }

  cudaError_t outer_residual(const T *b, const T *x, cudaStream_t st = nullptr) {
    if (!st) st = s;
    return with_vl<kVec4>(vec, lanes, [&](auto Vc, auto Lc) {
      constexpr int V = decltype(Vc)::value, L = decltype(Lc)::value;
      k_resid<Arith, V, L><<<tgrid, kThreads, 0, st>>>(A, mp, b, x, r, 1, cs, partials, counter, mask);
      return cudaGetLastError();
    });
  }
};

template <typename Arith64>
ens_status solve_f64(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                     const ens_solve_opts &o, ens_solve_stats *st, cudaStream_t s) {
  const int mp = m == 1 ? 1 : (m + 1) / 2 * 2;
  const int64_t n = M->n;
  const int singular = (M->flags & ENS_MATRIX_SINGULAR) ? 1 : 0;
  Scratch sc(s, o);
  double *b = nullptr, *x = nullptr;
  cudaError_t e = sc.get(&b, (size_t)n * mp);
  if (e == cudaSuccess) e = sc.get(&x, (size_t)n * mp);
  const int cgrid = M->num_sms * 8;
  if (e == cudaSuccess) {
    k_pad<<<cgrid, 256, 0, s>>>(n, m, mp, B, b);
    if (!o.x0_zero) k_pad<<<cgrid, 256, 0, s>>>(n, m, mp, X, x);
    e = cudaGetLastError();
  }
  std::vector<double> tolv(mp, 0.0);
  for (int l = 0; l < m; ++l) tolv[l] = tol[l];
  std::vector<int32_t> iters(mp, 0), status(mp, 0), state(mp, 0), outer(mp, 0);
  std::vector<double> relres(mp, 0.0);

  if (o.precision == ENS_PREC_F64) {
    Bicg<Arith64> S;
    if (e == cudaSuccess) e = S.setup(sc, M, mp, o, s);
    if (e == cudaSuccess) e = S.start(b, x, o.x0_zero != 0, singular, tolv);
    int ran = 0;
    if (e == cudaSuccess) e = S.iterate(x, o.max_iter, o.check_every, o.use_graph != 0, &ran);
    if (e == cudaSuccess) e = S.finish(b, x, singular);
    if (e == cudaSuccess) e = cudaMemcpyAsync(iters.data(), S.cs.iters, mp * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status.data(), S.cs.status, mp * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(state.data(), S.cs.state, mp * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(relres.data(), S.cs.relres, mp * 8, cudaMemcpyDeviceToHost, s);
  } else {
    // Outer FP64 loop: r = b - A x, inner FP32 solve of A d = r / ||r||, x += ||r|| d.
    Bicg<Arith64> O;  // only its residual, scalars and reduction scratch are used
    Bicg<ArithF32> I;
    float *r32 = nullptr, *d32 = nullptr;
    ens_solve_opts oo = o;
    oo.precond = ENS_PRECOND_NONE;
    if (e == cudaSuccess) e = O.setup(sc, M, mp, oo, s, true);
    if (e == cudaSuccess) e = I.setup(sc, M, mp, o, s);
    if (e == cudaSuccess) e = sc.get(&r32, (size_t)n * mp);
    if (e == cudaSuccess) e = sc.get(&d32, (size_t)n * mp);
    if (e == cudaSuccess) e = O.start(b, x, o.x0_zero != 0, singular, tolv);
    std::vector<float> itol(mp, (float)o.inner_tol);
    std::vector<int32_t> h, inner_it(mp);
    for (int k = 0; e == cudaSuccess && k < o.max_outer; ++k) {
      e = O.states(h);
      if (e != cudaSuccess || Bicg<Arith64>::all_done(h)) break;
      e = with_vl(O.vec, O.lanes, [&](auto Vc, auto Lc) {
        constexpr int V = decltype(Vc)::value, L = decltype(Lc)::value;
        k_to32<V, L><<<O.grid, kThreads, 0, s>>>((int32_t)n, mp, O.r, r32, O.cs);
        return cudaGetLastError();
      });
      if (e == cudaSuccess) e = I.start(r32, d32, true, 0, itol);
      int ran = 0;
      if (e == cudaSuccess) e = I.iterate(d32, o.inner_max_iter, o.check_every, o.use_graph != 0, &ran);
      if (e == cudaSuccess) e = cudaMemcpyAsync(inner_it.data(), I.cs.iters, mp * 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      for (int l = 0; l < mp; ++l)
        if (h[l] == ST_ACTIVE) {
          iters[l] += inner_it[l];
          outer[l] += 1;
        }
      k_inner_nostep<<<1, 64, 0, s>>>(mp, O.cs, I.cs.status, I.cs.flags);
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = with_vl(O.vec, O.lanes, [&](auto Vc, auto Lc) {
          constexpr int V = decltype(Vc)::value, L = decltype(Lc)::value;
          k_correct<V, L><<<O.grid, kThreads, 0, s>>>((int32_t)n, mp, x, d32, O.cs, I.cs.status);
          return cudaGetLastError();
        });
      if (e == cudaSuccess) e = O.outer_residual(b, x);
    }
    if (e == cudaSuccess) e = O.finish(b, x, singular);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status.data(), O.cs.status, mp * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(state.data(), O.cs.state, mp * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(relres.data(), O.cs.relres, mp * 8, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) {
    k_unpad<<<cgrid, 256, 0, s>>>(n, m, mp, x, X);
    e = cudaGetLastError();
  }
  // also on failure: work already queued may still use the scratch (or the caller's workspace)
  const cudaError_t esync = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = esync;
  if (e != cudaSuccess) return cuda_fail(e, "solve_block");
  for (int l = 0; l < m; ++l) {
    if (state[l] != ST_DONE) status[l] = ENS_COL_MAXITER;
    if (st) {
      if (st->iters) st->iters[l] = iters[l];
      if (st->status) st->status[l] = status[l];
      if (st->relres) st->relres[l] = relres[l];
      if (st->outer) st->outer[l] = outer[l];
    }
  }
  return ENS_OK;
}


// ============================================================================= batched solves
// Every system's whole solve (padding, start, iteration loop, finish) is stream-captured into one
// branch of a single CUDA graph; the iteration loops are conditional WHILE nodes inserted into the
// capture (nested outer/inner loops in mixed precision). One graph launch then runs all systems
// concurrently, each loop ending on the device when its columns are done or its limit is reached.

static __global__ void k_set_cond(cudaGraphConditionalHandle h, unsigned v) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h, v);
}

// Mixed precision, after an inner solve: columns still active in the outer loop add the inner
// iterations and one refinement step to their counts.
static __global__ void k_accum(int32_t mp, const int32_t *__restrict__ outer_state, const int32_t *__restrict__ inner_iters,
                               int32_t *iters_tot, int32_t *outer_cnt) {
  for (int l = threadIdx.x; l < mp; l += blockDim.x)
    if (outer_state[l] == ST_ACTIVE) {
      iters_tot[l] += inner_iters[l];
      outer_cnt[l] += 1;
    }
}

// Outer loop condition: some column still active and fewer than max_outer refinement steps.
static __global__ void k_outer_cond(cudaGraphConditionalHandle h, int32_t mp, const int32_t *__restrict__ state,
                                    int32_t *steps, int32_t max_outer) {
  if (threadIdx.x == 0) {
    int any = 0;
    for (int l = 0; l < mp; ++l) any |= state[l] != ST_DONE;
    const int k = ++steps[0];
    cudaGraphSetConditional(h, (any && k < max_outer) ? 1u : 0u);
  }
}

// Inside an active capture on `cap`: append a conditional WHILE node (handle created on the
// capturing graph, default 1) after the current capture dependencies, make it the new dependency
// and return its (empty) body graph.
inline cudaError_t capture_while(cudaStream_t cap, cudaGraphConditionalHandle *h, cudaGraph_t *body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cap, &cst, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cst != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  e = cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = *h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Captures `fill(stream)` into the given (empty) graph on a private stream.
template <typename F>
cudaError_t capture_into(cudaGraph_t body, F &&fill) {
  cudaStream_t c = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(c, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t ef = fill(c);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(c, &out);
    if (e == cudaSuccess) e = ef;
  }
  cudaStreamDestroy(c);
  return e;
}

struct SysBase {
  virtual ~SysBase() {}
  virtual cudaError_t setup(Scratch &sc) = 0;        // allocations and host-to-device uploads
  virtual cudaError_t record(cudaStream_t cap) = 0;  // the whole solve, captured
  virtual cudaError_t fetch() = 0;                   // stats to host (after the graph ran)
  virtual void write(ens_solve_stats *st) = 0;
};

template <typename Arith64>
struct SysImpl : SysBase {
  const ens_matrix *M;
  int32_t m, mp;
  const double *B;
  double *X;
  ens_solve_opts o;
  int singular;
  cudaStream_t s;
  double *b = nullptr, *x = nullptr;
  Bicg<Arith64> S;  // FP64 solver, or the outer residual/scalars in mixed mode
  Bicg<ArithF32> I; // mixed mode: FP32 inner solver
  float *r32 = nullptr, *d32 = nullptr;
  int32_t *iters_tot = nullptr, *outer_cnt = nullptr, *steps = nullptr;
  std::vector<double> tolv;
  std::vector<float> itol;
  std::vector<int32_t> h_iters, h_status, h_state, h_outer;
  std::vector<double> h_relres;

  SysImpl(const ens_matrix *M_, int32_t m_, const double *B_, double *X_, const double *tol, const ens_solve_opts &o_,
          cudaStream_t s_)
      : M(M_), m(m_), B(B_), X(X_), o(o_), s(s_) {
    mp = m == 1 ? 1 : (m + 1) / 2 * 2;
    singular = (M->flags & ENS_MATRIX_SINGULAR) ? 1 : 0;
    tolv.assign(mp, 0.0);
    for (int l = 0; l < m; ++l) tolv[l] = tol[l];
    itol.assign(mp, (float)o.inner_tol);
  }

  bool mixed() const { return o.precision == ENS_PREC_MIXED; }

  cudaError_t setup(Scratch &sc) override {
    const size_t blk = (size_t)M->n * mp;
    cudaError_t e = sc.get(&b, blk);
    if (e == cudaSuccess) e = sc.get(&x, blk);
    if (e == cudaSuccess) e = sc.get(&iters_tot, mp);
    if (e == cudaSuccess) e = sc.get(&outer_cnt, mp);
    if (e == cudaSuccess) e = sc.get(&steps, 1);
    if (mixed()) {
      ens_solve_opts oo = o;
      oo.precond = ENS_PRECOND_NONE;
      if (e == cudaSuccess) e = S.setup(sc, M, mp, oo, s, true);
      if (e == cudaSuccess) e = I.setup(sc, M, mp, o, s);
      if (e == cudaSuccess) e = sc.get(&r32, blk);
      if (e == cudaSuccess) e = sc.get(&d32, blk);
      if (e == cudaSuccess) e = I.upload_tol(itol);
    } else {
      if (e == cudaSuccess) e = S.setup(sc, M, mp, o, s);
    }
    if (e == cudaSuccess) e = S.upload_tol(tolv);
    return e;
  }

  cudaError_t record(cudaStream_t cap) override {
    const int64_t n = M->n;
    const int cgrid = M->num_sms * 8;
    k_pad<<<cgrid, 256, 0, cap>>>(n, m, mp, B, b);
    if (!o.x0_zero) k_pad<<<cgrid, 256, 0, cap>>>(n, m, mp, X, x);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(iters_tot, 0, mp * sizeof(int32_t), cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(outer_cnt, 0, mp * sizeof(int32_t), cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(steps, 0, sizeof(int32_t), cap);
    if (e == cudaSuccess) e = S.enqueue_start(b, x, o.x0_zero != 0, singular, cap);
    if (e != cudaSuccess) return e;
    if (!mixed()) {
      if (o.max_iter > 0) {
        cudaGraphConditionalHandle h{};
        cudaGraph_t body = nullptr;
        e = capture_while(cap, &h, &body);
        if (e == cudaSuccess)
          e = capture_into(body, [&](cudaStream_t c) {
            cudaError_t ek = S.iteration(x, o.max_iter, c);
            if (ek == cudaSuccess) {
              k_loop_cond<<<1, 32, 0, c>>>(h, S.cs.it);
              ek = cudaGetLastError();
            }
            return ek;
          });
      }
    } else {
      cudaGraphConditionalHandle ho{};
      cudaGraph_t obody = nullptr;
      e = capture_while(cap, &ho, &obody);
      if (e == cudaSuccess)
        e = capture_into(obody, [&](cudaStream_t c) {
          cudaError_t ek = with_vl(S.vec, S.lanes, [&](auto Vc, auto Lc) {
            constexpr int V = decltype(Vc)::value, L = decltype(Lc)::value;
            k_to32<V, L><<<S.grid, kThreads, 0, c>>>((int32_t)n, mp, S.r, r32, S.cs);
            return cudaGetLastError();
          });
          if (ek == cudaSuccess) ek = I.enqueue_start(r32, d32, true, 0, c);
          if (ek == cudaSuccess && o.inner_max_iter > 0) {
            cudaGraphConditionalHandle hi{};
            cudaGraph_t ibody = nullptr;
            ek = capture_while(c, &hi, &ibody);
            if (ek == cudaSuccess)
              ek = capture_into(ibody, [&](cudaStream_t c2) {
                cudaError_t ei = I.iteration(d32, o.inner_max_iter, c2);
                if (ei == cudaSuccess) {
                  k_loop_cond<<<1, 32, 0, c2>>>(hi, I.cs.it);
                  ei = cudaGetLastError();
                }
                return ei;
              });
            // the inner loop's condition starts at 1 when the graph is launched; re-arm it after the
            // loop ends so that the next outer step runs its inner solve again
            if (ek == cudaSuccess) {
              k_set_cond<<<1, 32, 0, c>>>(hi, 1u);
              ek = cudaGetLastError();
            }
          }
          if (ek == cudaSuccess) {
            k_accum<<<1, 64, 0, c>>>(mp, S.cs.state, I.cs.iters, iters_tot, outer_cnt);
            ek = cudaGetLastError();
          }
          if (ek == cudaSuccess) {
            k_inner_nostep<<<1, 64, 0, c>>>(mp, S.cs, I.cs.status, I.cs.flags);
            ek = cudaGetLastError();
          }
          if (ek == cudaSuccess)
            ek = with_vl(S.vec, S.lanes, [&](auto Vc, auto Lc) {
              constexpr int V = decltype(Vc)::value, L = decltype(Lc)::value;
              k_correct<V, L><<<S.grid, kThreads, 0, c>>>((int32_t)n, mp, x, d32, S.cs, I.cs.status);
              return cudaGetLastError();
            });
          if (ek == cudaSuccess) ek = S.outer_residual(b, x, c);
          if (ek == cudaSuccess) {
            k_outer_cond<<<1, 32, 0, c>>>(ho, mp, S.cs.state, steps, o.max_outer);
            ek = cudaGetLastError();
          }
          return ek;
        });
    }
    if (e == cudaSuccess) e = S.finish(b, x, singular, cap);
    if (e == cudaSuccess) {
      k_unpad<<<cgrid, 256, 0, cap>>>(n, m, mp, x, X);
      e = cudaGetLastError();
    }
    return e;
  }

  cudaError_t fetch() override {
    h_iters.assign(mp, 0);
    h_status.assign(mp, 0);
    h_state.assign(mp, 0);
    h_outer.assign(mp, 0);
    h_relres.assign(mp, 0.0);
    cudaError_t e = cudaMemcpyAsync(h_status.data(), S.cs.status, mp * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_state.data(), S.cs.state, mp * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_relres.data(), S.cs.relres, mp * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_iters.data(), mixed() ? iters_tot : S.cs.iters, mp * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && mixed()) e = cudaMemcpyAsync(h_outer.data(), outer_cnt, mp * 4, cudaMemcpyDeviceToHost, s);
    return e;
  }

  void write(ens_solve_stats *st) override {
    if (!st) return;
    for (int l = 0; l < m; ++l) {
      const int32_t status = h_state[l] != ST_DONE ? (int32_t)ENS_COL_MAXITER : h_status[l];
      if (st->iters) st->iters[l] = h_iters[l];
      if (st->status) st->status[l] = status;
      if (st->relres) st->relres[l] = h_relres[l];
      if (st->outer) st->outer[l] = h_outer[l];
    }
  }
};

SysBase *make_system_split(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                           const ens_solve_opts &o, cudaStream_t s);
SysBase *make_system_native(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                            const ens_solve_opts &o, cudaStream_t s);
SysBase *make_system_hybrid(const ens_matrix *M, int32_t m, const double *B, double *X, const double *tol,
                            const ens_solve_opts &o, cudaStream_t s);

extern template struct Bicg<ArithF32>;
extern template struct Bicg<ArithF64Split>;
extern template struct Bicg<ArithF64Native>;
extern template struct Bicg<ArithF64Hybrid>;

}  // namespace solver
}  // namespace ens
