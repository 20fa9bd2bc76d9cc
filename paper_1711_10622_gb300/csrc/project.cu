// The projection step around the pressure solve for m flow states (Section 2.2, Eqs. eq2/eq3):
// the divergence of m staggered velocity fields (the Poisson right-hand sides) and the pressure-
// gradient correction u -= tau G p. Both are streaming passes over the fluid cells with the m
// states of a face contiguous in memory (row-interleaved), one thread per (cell, group of 1, 2 or 4
// states).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "ens_internal.cuh"
#include "ensemble_project.h"
#include "rowprod.cuh"

struct ens_grid {
  int32_t N[3] = {0, 0, 0};
  int32_t F[3] = {0, 0, 0};  // faces per direction in each velocity component array
  int32_t bc[3] = {0, 0, 0};
  int32_t n = 0;  // fluid cells (rows)
  int64_t ncell = 0;
  int64_t nfaces[3] = {0, 0, 0};
  bool all_fluid = true;
  int device = 0;
  int num_sms = 0;
  int32_t *cell_of_row = nullptr;  // [n] (NULL when every cell is fluid: row = cell)
  int32_t *row_of_cell = nullptr;  // [ncell] (-1: solid; NULL when every cell is fluid)
  uint8_t *open = nullptr;         // [n] bit 2d: low face along d open, bit 2d+1: high face open
  double *width[3] = {nullptr, nullptr, nullptr};     // [N_d] cell widths
  double *inv_dist[3] = {nullptr, nullptr, nullptr};  // [N_d + 1] per face position (see below)
  double *area[3] = {nullptr, nullptr, nullptr};      // face areas normal to d, indexed by the other two
                                                      // coordinates (lower one fastest)
  bool split_area = false;  // every area lies in the split-float product range [2^-40, 2^60)
};

namespace ens {
namespace {

// Kernel view of a grid. inv_dist[d][i] belongs to the faces at position i along d: 1 / (distance
// between the centres of cells i-1 and i) inside, across the wrap for i = 0 of a periodic
// direction, 2 / width of the boundary cell on a Dirichlet boundary face (p = 0 half a cell out).
struct GridView {
  int32_t N[3], F[3], bc[3];
  int32_t n;
  bool all_fluid;
  const int32_t *__restrict__ cell_of_row;
  const int32_t *__restrict__ row_of_cell;
  const uint8_t *__restrict__ open;
  const double *__restrict__ width[3];
  const double *__restrict__ inv_dist[3];
  const double *__restrict__ area[3];
};

GridView view_of(const ens_grid *G) {
  GridView v;
  for (int d = 0; d < 3; ++d) {
    v.N[d] = G->N[d];
    v.F[d] = G->F[d];
    v.bc[d] = G->bc[d];
    v.width[d] = G->width[d];
    v.area[d] = G->area[d];
    v.inv_dist[d] = G->inv_dist[d];
  }
  v.n = G->n;
  v.all_fluid = G->all_fluid;
  v.cell_of_row = G->cell_of_row;
  v.row_of_cell = G->row_of_cell;
  v.open = G->open;
  return v;
}

// VEC consecutive doubles (VEC = 1, 2 or 4; 16-byte aligned for 2 and 4).
template <int VEC>
__device__ __forceinline__ void ldv(const double *p, double (&v)[VEC]) {
  if constexpr (VEC == 1) {
    v[0] = __ldg(p);
  } else {
#pragma unroll
    for (int h = 0; h < VEC / 2; ++h) {
      const double2 t = __ldg(reinterpret_cast<const double2 *>(p) + h);
      v[2 * h] = t.x;
      v[2 * h + 1] = t.y;
    }
  }
}
template <int VEC>
__device__ __forceinline__ void ldv_rw(const double *p, double (&v)[VEC]) {
  if constexpr (VEC == 1) {
    v[0] = *p;
  } else {
#pragma unroll
    for (int h = 0; h < VEC / 2; ++h) {
      const double2 t = reinterpret_cast<const double2 *>(p)[h];
      v[2 * h] = t.x;
      v[2 * h + 1] = t.y;
    }
  }
}
template <int VEC>
__device__ __forceinline__ void stv(double *p, const double (&v)[VEC]) {
  if constexpr (VEC == 1) {
    *p = v[0];
  } else {
#pragma unroll
    for (int h = 0; h < VEC / 2; ++h) reinterpret_cast<double2 *>(p)[h] = make_double2(v[2 * h], v[2 * h + 1]);
  }
}

// Face array index of the face at position (c0, c1, c2) along d (c_d is the face number).
__device__ __forceinline__ int64_t face_at(const GridView &g, int d, int32_t c0, int32_t c1, int32_t c2) {
  const int32_t s0 = d == 0 ? g.F[0] : g.N[0];
  const int32_t s1 = d == 1 ? g.F[1] : g.N[1];
  return (int64_t)c0 + (int64_t)s0 * ((int64_t)c1 + (int64_t)s1 * c2);
}

// D[r*m + c + q] = scale * sum_d area_d (u_hi - u_lo) over the open faces of the row's cell.
template <int VEC>
__global__ void __launch_bounds__(kThreads)
    k_divergence(GridView g, int32_t m, double scale, const double *__restrict__ U, const double *__restrict__ V,
                 const double *__restrict__ W, double *__restrict__ D) {
  const int32_t groups = m / VEC;
  const int64_t total = (int64_t)g.n * groups;
  const double *comp[3] = {U, V, W};
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / groups);
    const int32_t c = (int32_t)(t - (int64_t)r * groups) * VEC;
    const int32_t cell = g.all_fluid ? r : g.cell_of_row[r];
    const int32_t p[3] = {cell % g.N[0], (cell / g.N[0]) % g.N[1], cell / (g.N[0] * g.N[1])};
    const uint32_t op = g.open[r];
    // face areas of the cell (tables of the products of the other two widths)
    const double ar[3] = {g.area[0][p[1] + (int64_t)g.N[1] * p[2]], g.area[1][p[0] + (int64_t)g.N[0] * p[2]],
                          g.area[2][p[0] + (int64_t)g.N[0] * p[1]]};
    double acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double area = ar[d];
      int32_t lo[3] = {p[0], p[1], p[2]}, hi[3] = {p[0], p[1], p[2]};
      hi[d] = (g.bc[d] == ENS_BC_PERIODIC && p[d] + 1 == g.N[d]) ? 0 : p[d] + 1;
      if (op & (2u << (2 * d))) {
        double u[VEC];
        ldv<VEC>(comp[d] + face_at(g, d, hi[0], hi[1], hi[2]) * m + c, u);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = fma(area, u[q], acc[q]);
      }
      if (op & (1u << (2 * d))) {
        double u[VEC];
        ldv<VEC>(comp[d] + face_at(g, d, lo[0], lo[1], lo[2]) * m + c, u);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = fma(-area, u[q], acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] *= scale;
    stv<VEC>(D + (int64_t)r * m + c, acc);
  }
}

// The same divergence with split-float products (the GSpMV's arithmetic, rowprod.cuh): the FP64 pipe
// of GB300 is narrow, and the native form spends 7 FP64 operations per cell and state; here the six
// face products and their sum run on the FP32 pipe as packed pairs of states (split_acc2: each area and
// face value carried as hi + lo floats, the sum accumulated error-free), and each output costs one
// FP64 addition (the widening of hi + lo) and the scale multiply. A state whose face values leave the
// split range (zero among them) is recomputed with native DFMA. VEC = 2 or 4 states per thread.
template <int VEC>
__global__ void __launch_bounds__(kThreads, 4)
    k_divergence_split(GridView g, int32_t m, double scale, const double *__restrict__ U, const double *__restrict__ V,
                       const double *__restrict__ W, double *__restrict__ D) {
  constexpr int NP = VEC / 2;
  constexpr uint64_t kSign2 = 0x8000000080000000ull;
  const int32_t groups = m / VEC;
  const int64_t total = (int64_t)g.n * groups;
  const double *comp[3] = {U, V, W};
  const uint64_t g23 = f2_pack(__uint_as_float(kSplitG), __uint_as_float(kSplitG));
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / groups);
    const int32_t c = (int32_t)(t - (int64_t)r * groups) * VEC;
    const int32_t cell = g.all_fluid ? r : g.cell_of_row[r];
    const int32_t p[3] = {cell % g.N[0], (cell / g.N[0]) % g.N[1], cell / (g.N[0] * g.N[1])};
    const uint32_t op = g.open[r];
    const double ar[3] = {g.area[0][p[1] + (int64_t)g.N[1] * p[2]], g.area[1][p[0] + (int64_t)g.N[0] * p[2]],
                          g.area[2][p[0] + (int64_t)g.N[0] * p[1]]};
    uint64_t sh[NP], sl[NP];
    uint32_t rng[VEC];
#pragma unroll
    for (int q = 0; q < NP; ++q) sh[q] = sl[q] = 0ull;
#pragma unroll
    for (int q = 0; q < VEC; ++q) rng[q] = 0u;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float ah, al;
      split_f64(ar[d], ah, al);
      const SplitPair a = split_pair(make_float2(ah, al));
      int32_t lo[3] = {p[0], p[1], p[2]}, hi[3] = {p[0], p[1], p[2]};
      hi[d] = (g.bc[d] == ENS_BC_PERIODIC && p[d] + 1 == g.N[d]) ? 0 : p[d] + 1;
      if (op & (2u << (2 * d))) {
        double u[VEC];
        ldv<VEC>(comp[d] + face_at(g, d, hi[0], hi[1], hi[2]) * m + c, u);
#pragma unroll
        for (int q = 0; q < NP; ++q) split_acc2(a, u[2 * q], u[2 * q + 1], g23, sh[q], sl[q], rng[2 * q], rng[2 * q + 1]);
      }
      if (op & (1u << (2 * d))) {
        double u[VEC];
        ldv<VEC>(comp[d] + face_at(g, d, lo[0], lo[1], lo[2]) * m + c, u);
        const SplitPair na{a.ah ^ kSign2, a.al ^ kSign2};  // -area, exactly
#pragma unroll
        for (int q = 0; q < NP; ++q) split_acc2(na, u[2 * q], u[2 * q + 1], g23, sh[q], sl[q], rng[2 * q], rng[2 * q + 1]);
      }
    }
    double y[VEC];
    bool all_ok = true, ok[VEC];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      float h0, h1, l0, l1;
      f2_unpack(sh[q], h0, h1);
      f2_unpack(sl[q], l0, l1);
      ok[2 * q] = split_ok(rng[2 * q], h0, l0);
      ok[2 * q + 1] = split_ok(rng[2 * q + 1], h1, l1);
      y[2 * q] = split_to_double(h0, l0);
      y[2 * q + 1] = split_to_double(h1, l1);
      all_ok &= ok[2 * q] && ok[2 * q + 1];
    }
    if (!all_ok) {  // native products for the states the split form cannot carry
      double acc[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int32_t lo[3] = {p[0], p[1], p[2]}, hi[3] = {p[0], p[1], p[2]};
        hi[d] = (g.bc[d] == ENS_BC_PERIODIC && p[d] + 1 == g.N[d]) ? 0 : p[d] + 1;
        if (op & (2u << (2 * d))) {
          double u[VEC];
          ldv<VEC>(comp[d] + face_at(g, d, hi[0], hi[1], hi[2]) * m + c, u);
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[q] = fma(ar[d], u[q], acc[q]);
        }
        if (op & (1u << (2 * d))) {
          double u[VEC];
          ldv<VEC>(comp[d] + face_at(g, d, lo[0], lo[1], lo[2]) * m + c, u);
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[q] = fma(-ar[d], u[q], acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < VEC; ++q) y[q] = ok[q] ? y[q] : acc[q];
    }
#pragma unroll
    for (int q = 0; q < VEC; ++q) y[q] *= scale;
    stv<VEC>(D + (int64_t)r * m + c, y);
  }
}

// u -= tau (p_hi - p_lo) inv_dist on the open faces. Each fluid cell owns its low face in every
// direction (the cell is that face's high side) and, in a Dirichlet direction, the high boundary
// face when it is the last cell; together these are all open faces, each written once.
template <int VEC>
__global__ void __launch_bounds__(kThreads)
    k_grad_correct(GridView g, int32_t m, double tau, const double *__restrict__ P, double *U, double *V, double *W) {
  const int32_t groups = m / VEC;
  const int64_t total = (int64_t)g.n * groups;
  double *comp[3] = {U, V, W};
  const int32_t stride[3] = {1, g.N[0], g.N[0] * g.N[1]};
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / groups);
    const int32_t c = (int32_t)(t - (int64_t)r * groups) * VEC;
    const int32_t cell = g.all_fluid ? r : g.cell_of_row[r];
    const int32_t p[3] = {cell % g.N[0], (cell / g.N[0]) % g.N[1], cell / (g.N[0] * g.N[1])};
    const uint32_t op = g.open[r];
    double pc[VEC];
    ldv<VEC>(P + (int64_t)r * m + c, pc);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (op & (1u << (2 * d))) {  // low face open: a fluid neighbour or a Dirichlet boundary
        double pn[VEC];
        const bool boundary = p[d] == 0 && g.bc[d] != ENS_BC_PERIODIC;
        if (boundary) {
#pragma unroll
          for (int q = 0; q < VEC; ++q) pn[q] = 0.0;
        } else {
          const int32_t nb_cell = p[d] == 0 ? cell + (g.N[d] - 1) * stride[d] : cell - stride[d];
          const int32_t nb = g.all_fluid ? nb_cell : g.row_of_cell[nb_cell];
          ldv<VEC>(P + (int64_t)nb * m + c, pn);
        }
        const double coef = tau * g.inv_dist[d][p[d]];
        double *u = comp[d] + face_at(g, d, p[0], p[1], p[2]) * m + c;
        double v[VEC];
        ldv_rw<VEC>(u, v);
#pragma unroll
        for (int q = 0; q < VEC; ++q) v[q] = fma(-coef, pc[q] - pn[q], v[q]);
        stv<VEC>(u, v);
      }
      if (g.bc[d] == ENS_BC_DIRICHLET && p[d] == g.N[d] - 1 && (op & (2u << (2 * d)))) {
        const double coef = tau * g.inv_dist[d][g.N[d]];
        int32_t f[3] = {p[0], p[1], p[2]};
        f[d] = g.N[d];
        double *u = comp[d] + face_at(g, d, f[0], f[1], f[2]) * m + c;
        double v[VEC];
        ldv_rw<VEC>(u, v);
#pragma unroll
        for (int q = 0; q < VEC; ++q) v[q] = fma(-coef, 0.0 - pc[q], v[q]);
        stv<VEC>(u, v);
      }
    }
  }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int grid_blocks(const ens_grid *G, int64_t work) {
  const int64_t want = (work + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)G->num_sms * 8;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

void free_grid(ens_grid *G) {
  if (!G) return;
  cudaFree(G->cell_of_row);
  cudaFree(G->row_of_cell);
  cudaFree(G->open);
  for (int d = 0; d < 3; ++d) {
    cudaFree(G->width[d]);
    cudaFree(G->inv_dist[d]);
    cudaFree(G->area[d]);
  }
  delete G;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src, cudaStream_t s) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

}  // namespace
}  // namespace ens

using namespace ens;

static ens_status create_grid_impl(int32_t nx, int32_t ny, int32_t nz, const double *xn, const double *yn,
                                   const double *zn, const int32_t *bc, const uint8_t *solid, void *stream,
                                   ens_grid **out);

extern "C" ens_status ens_create_grid(int32_t nx, int32_t ny, int32_t nz, const double *xn, const double *yn,
                                      const double *zn, const int32_t *bc, const uint8_t *solid, void *stream,
                                      ens_grid **out) {
  clear_error();
  try {
    return create_grid_impl(nx, ny, nz, xn, yn, zn, bc, solid, stream, out);
  } catch (const std::bad_alloc &) {
    return fail(ENS_ERR_OOM, "create_grid: host allocation failed");
  }
}

static ens_status create_grid_impl(int32_t nx, int32_t ny, int32_t nz, const double *xn, const double *yn,
                                   const double *zn, const int32_t *bc, const uint8_t *solid, void *stream,
                                   ens_grid **out) {
  if (!out) return fail(ENS_ERR_INVALID, "create_grid: out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(ENS_ERR_INVALID, "create_grid: dimensions must be >= 1");
  if (!xn || !yn || !zn || !bc) return fail(ENS_ERR_INVALID, "create_grid: NULL coordinates or boundary codes");
  const int32_t N[3] = {nx, ny, nz};
  const double *nodes[3] = {xn, yn, zn};
  const int64_t ncell = (int64_t)nx * ny * nz;
  if (ncell > INT32_MAX) return fail(ENS_ERR_INVALID, "create_grid: %lld cells exceed int32 indexing", (long long)ncell);
  for (int d = 0; d < 3; ++d) {
    if (bc[d] != ENS_BC_WALL && bc[d] != ENS_BC_PERIODIC && bc[d] != ENS_BC_DIRICHLET)
      return fail(ENS_ERR_INVALID, "create_grid: unknown boundary code %d in direction %d", bc[d], d);
    if (bc[d] == ENS_BC_PERIODIC && N[d] < 3)
      return fail(ENS_ERR_INVALID, "create_grid: periodic direction %d needs at least 3 cells", d);
    for (int32_t i = 0; i <= N[d]; ++i)
      if (!std::isfinite(nodes[d][i]) || (i > 0 && !(nodes[d][i] > nodes[d][i - 1])))
        return fail(ENS_ERR_INVALID, "create_grid: node coordinates of direction %d not finite and increasing", d);
  }
  // cell <-> row maps and open-face masks (host)
  std::vector<int32_t> row_of_cell(ncell);
  std::vector<int32_t> cell_of_row;
  cell_of_row.reserve(ncell);
  for (int64_t cidx = 0; cidx < ncell; ++cidx) {
    if (solid && solid[cidx]) {
      row_of_cell[cidx] = -1;
    } else {
      row_of_cell[cidx] = (int32_t)cell_of_row.size();
      cell_of_row.push_back((int32_t)cidx);
    }
  }
  const int32_t n = (int32_t)cell_of_row.size();
  if (n == 0) return fail(ENS_ERR_INVALID, "create_grid: every cell is solid");
  const int64_t stride[3] = {1, nx, (int64_t)nx * ny};
  std::vector<uint8_t> open(n);
  for (int32_t r = 0; r < n; ++r) {
    const int64_t cell = cell_of_row[r];
    const int64_t p[3] = {cell % nx, (cell / nx) % ny, cell / ((int64_t)nx * ny)};
    uint8_t bits = 0;
    for (int d = 0; d < 3; ++d) {
      // low side
      if (p[d] > 0) {
        if (row_of_cell[cell - stride[d]] >= 0) bits |= (uint8_t)(1u << (2 * d));
      } else if (bc[d] == ENS_BC_PERIODIC) {
        if (row_of_cell[cell + (N[d] - 1) * stride[d]] >= 0) bits |= (uint8_t)(1u << (2 * d));
      } else if (bc[d] == ENS_BC_DIRICHLET) {
        bits |= (uint8_t)(1u << (2 * d));
      }
      // high side
      if (p[d] < N[d] - 1) {
        if (row_of_cell[cell + stride[d]] >= 0) bits |= (uint8_t)(2u << (2 * d));
      } else if (bc[d] == ENS_BC_PERIODIC) {
        if (row_of_cell[cell - (N[d] - 1) * stride[d]] >= 0) bits |= (uint8_t)(2u << (2 * d));
      } else if (bc[d] == ENS_BC_DIRICHLET) {
        bits |= (uint8_t)(2u << (2 * d));
      }
    }
    open[r] = bits;
  }
  std::vector<double> width[3], inv_dist[3];
  for (int d = 0; d < 3; ++d) {
    const int32_t Nd = N[d];
    width[d].resize(Nd);
    std::vector<double> centre(Nd);
    for (int32_t i = 0; i < Nd; ++i) {
      width[d][i] = nodes[d][i + 1] - nodes[d][i];
      centre[i] = 0.5 * (nodes[d][i] + nodes[d][i + 1]);
    }
    inv_dist[d].assign(Nd + 1, 0.0);
    for (int32_t i = 1; i < Nd; ++i) inv_dist[d][i] = 1.0 / (centre[i] - centre[i - 1]);
    if (bc[d] == ENS_BC_PERIODIC) {
      const double L = nodes[d][Nd] - nodes[d][0];
      inv_dist[d][0] = 1.0 / (centre[0] + L - centre[Nd - 1]);
    } else if (bc[d] == ENS_BC_DIRICHLET) {
      inv_dist[d][0] = 2.0 / width[d][0];
      inv_dist[d][Nd] = 2.0 / width[d][Nd - 1];
    }
  }

  // area of the faces normal to d: the product of the cell widths in the other two directions
  // (ascending direction order), tabulated over those two coordinates
  std::vector<double> area[3];
  for (int d = 0; d < 3; ++d) {
    const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;  // the other two directions, a < b
    area[d].resize((size_t)N[a] * N[b]);
    for (int32_t jb = 0; jb < N[b]; ++jb)
      for (int32_t ja = 0; ja < N[a]; ++ja) area[d][ja + (size_t)N[a] * jb] = width[a][ja] * width[b][jb];
  }

  bool split_area = true;
  for (int d = 0; d < 3; ++d)
    for (double a : area[d]) split_area = split_area && a >= 0x1p-40 && a < 0x1p60;

  ens_grid *G = new ens_grid();
  G->split_area = split_area;
  for (int d = 0; d < 3; ++d) {
    G->N[d] = N[d];
    G->bc[d] = bc[d];
    G->F[d] = bc[d] == ENS_BC_PERIODIC ? N[d] : N[d] + 1;
  }
  G->n = n;
  G->ncell = ncell;
  G->all_fluid = n == ncell;
  for (int d = 0; d < 3; ++d) {
    int64_t f = 1;
    for (int e = 0; e < 3; ++e) f *= e == d ? G->F[e] : G->N[e];
    G->nfaces[d] = f;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&G->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&G->num_sms, cudaDevAttrMultiProcessorCount, G->device);
  if (e == cudaSuccess && !G->all_fluid) e = upload(&G->cell_of_row, cell_of_row, s);
  if (e == cudaSuccess && !G->all_fluid) e = upload(&G->row_of_cell, row_of_cell, s);
  if (e == cudaSuccess) e = upload(&G->open, open, s);
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
    e = upload(&G->width[d], width[d], s);
    if (e == cudaSuccess) e = upload(&G->inv_dist[d], inv_dist[d], s);
    if (e == cudaSuccess) e = upload(&G->area[d], area[d], s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_grid(G);
    return cuda_fail(e, "create_grid");
  }
  *out = G;
  return ENS_OK;
}

extern "C" ens_status ens_destroy_grid(ens_grid *G) {
  clear_error();
  if (!G) return ENS_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_grid(G);
  if (e != cudaSuccess) return cuda_fail(e, "destroy_grid");
  return ENS_OK;
}

extern "C" ens_status ens_grid_info(const ens_grid *G, int64_t *n_rows, int64_t n_faces[3]) {
  clear_error();
  if (!G) return fail(ENS_ERR_INVALID, "grid_info: grid is NULL");
  if (n_rows) *n_rows = G->n;
  if (n_faces)
    for (int d = 0; d < 3; ++d) n_faces[d] = G->nfaces[d];
  return ENS_OK;
}

namespace {
ens_status check_common(const ens_grid *G, int32_t m, const char *who) {
  if (!G) return fail(ENS_ERR_INVALID, "%s: grid is NULL", who);
  if (m < 1) return fail(ENS_ERR_INVALID, "%s: m must be >= 1 (got %d)", who, m);
  int dev = 0;
  ENS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != G->device) return fail(ENS_ERR_INVALID, "%s: current device %d is not the grid's device %d", who, dev, G->device);
  return ENS_OK;
}
}  // namespace

extern "C" ens_status ens_divergence(const ens_grid *G, int32_t m, double scale, const double *U, const double *V,
                                     const double *W, double *D, void *stream) {
  clear_error();
  ens_status st = check_common(G, m, "divergence");
  if (st != ENS_OK) return st;
  if (!U || !V || !W || !D) return fail(ENS_ERR_INVALID, "divergence: NULL array");
  if (!std::isfinite(scale)) return fail(ENS_ERR_INVALID, "divergence: scale is not finite");
  const size_t nd = (size_t)G->n * m * sizeof(double);
  const double *comp[3] = {U, V, W};
  for (int d = 0; d < 3; ++d)
    if (overlaps(D, nd, comp[d], (size_t)G->nfaces[d] * m * sizeof(double)))
      return fail(ENS_ERR_INVALID, "divergence: D overlaps a velocity component");
  // four or two states per thread when the rows allow 16-byte accesses: the per-cell work (coordinates,
  // open faces, areas) is shared by those states
  const bool al = aligned16(U) && aligned16(V) && aligned16(W) && aligned16(D);
  const int vec = al && m % 4 == 0 ? 4 : (al && m % 2 == 0 ? 2 : 1);
  const GridView g = view_of(G);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t work = (int64_t)G->n * (m / vec);
  // split-float products on the FP32 pipe for two or four states per thread (native for one)
  if (vec == 4 && G->split_area)
    k_divergence_split<4><<<grid_blocks(G, work), kThreads, 0, s>>>(g, m, scale, U, V, W, D);
  else if (vec == 2 && G->split_area)
    k_divergence_split<2><<<grid_blocks(G, work), kThreads, 0, s>>>(g, m, scale, U, V, W, D);
  else if (vec == 4)
    k_divergence<4><<<grid_blocks(G, work), kThreads, 0, s>>>(g, m, scale, U, V, W, D);
  else if (vec == 2)
    k_divergence<2><<<grid_blocks(G, work), kThreads, 0, s>>>(g, m, scale, U, V, W, D);
  else
    k_divergence<1><<<grid_blocks(G, work), kThreads, 0, s>>>(g, m, scale, U, V, W, D);
  ENS_CUDA_TRY(cudaGetLastError());
  return ENS_OK;
}

extern "C" ens_status ens_grad_correct(const ens_grid *G, int32_t m, double tau, const double *P, double *U, double *V,
                                       double *W, void *stream) {
  clear_error();
  ens_status st = check_common(G, m, "grad_correct");
  if (st != ENS_OK) return st;
  if (!P || !U || !V || !W) return fail(ENS_ERR_INVALID, "grad_correct: NULL array");
  if (!std::isfinite(tau)) return fail(ENS_ERR_INVALID, "grad_correct: tau is not finite");
  const size_t np = (size_t)G->n * m * sizeof(double);
  double *comp[3] = {U, V, W};
  for (int d = 0; d < 3; ++d) {
    const size_t nb = (size_t)G->nfaces[d] * m * sizeof(double);
    if (overlaps(P, np, comp[d], nb)) return fail(ENS_ERR_INVALID, "grad_correct: P overlaps a velocity component");
    for (int e = d + 1; e < 3; ++e)
      if (overlaps(comp[d], nb, comp[e], (size_t)G->nfaces[e] * m * sizeof(double)))
        return fail(ENS_ERR_INVALID, "grad_correct: velocity components overlap");
  }
  const bool al = aligned16(P) && aligned16(U) && aligned16(V) && aligned16(W);
  const int vec = al && m % 4 == 0 ? 4 : (al && m % 2 == 0 ? 2 : 1);
  const GridView g = view_of(G);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t work = (int64_t)G->n * (m / vec);
  if (vec == 4)
    k_grad_correct<4><<<grid_blocks(G, work), kThreads, 0, s>>>(g, m, tau, P, U, V, W);
  else if (vec == 2)
    k_grad_correct<2><<<grid_blocks(G, work), kThreads, 0, s>>>(g, m, tau, P, U, V, W);
  else
    k_grad_correct<1><<<grid_blocks(G, work), kThreads, 0, s>>>(g, m, tau, P, U, V, W);
  ENS_CUDA_TRY(cudaGetLastError());
  return ENS_OK;
}
