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
// iteration). Gram products and updates cost O(n m^2) float64 multiply-adds per iteration, which on
// GB300's narrow FP64 pipe is the price of the coupling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
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
  double *partials = nullptr, *dmat = nullptr, *dots = nullptr;

  Coupled(const ens_matrix *M_, int m_, int k_, const ens_solve_opts &o_, cudaStream_t s_, Scratch &sc_)
      : M(M_), n(M_->n), m(m_), k(k_), o(o_), s(s_), sc(sc_) {
    mp = k == 1 ? 1 : (k + 1) / 2 * 2;
    vec = mp == 1 ? 1 : 2;
    lanes = 1;
    while (lanes * vec < mp) lanes <<= 1;
    grid = M->num_sms * 8;
    ggrid = (int)std::max<int64_t>(1, std::min<int64_t>((n + kGramRows - 1) / kGramRows, (int64_t)M->num_sms * 8));
  }

  cudaError_t setup() {
    cudaError_t e = sc.get(&partials, (size_t)ggrid * kMaxCoupledM * 2 * kMaxCoupledM);
    if (e == cudaSuccess) e = sc.get(&dmat, (size_t)3 * kMaxCoupledM * kMaxCoupledM + 2 * kMaxCoupledM * kMaxCoupledM);
    if (e == cudaSuccess) e = sc.get(&dots, (size_t)4 * kMaxSolveM);
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
    Terms tm{};
    std::vector<double> hm;
    for (auto &t : terms) hm.insert(hm.end(), t.second.begin(), t.second.end());
    cudaError_t e = cudaMemcpyAsync(dmat, hm.data(), hm.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    for (size_t t = 0; t < terms.size(); ++t) {
      tm.Z[t] = terms[t].first;
      tm.M[t] = dmat + t * (size_t)k * k;
    }
    if (e != cudaSuccess) return e;
    const int nt = (int)terms.size();
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
