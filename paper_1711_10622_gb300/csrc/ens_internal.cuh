// Internal declarations shared by the translation units of libensemble_solve.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "ensemble_solve.h"

struct ens_amg;  // aggregation multigrid hierarchy attached to a matrix (amg.cu)

constexpr int kTuneMaxM = 64;  // block widths the autotuner keeps a choice for
constexpr int kShareHybrid = 64;  // "native share" code of the column-hybrid FP64 arithmetic

struct ens_matrix {
  int64_t n = 0, nnz = 0;
  int64_t ncols = 0;          // columns (= n for the square matrices of the solver; a row block of a
                              // distributed matrix indexes an extended vector of ncols rows)
  int32_t max_row_len = 0;
  uint32_t flags = 0;
  int device = 0;
  int num_sms = 0;
  int32_t *row = nullptr;     // [n+1]
  int32_t *col = nullptr;     // [nnz]
  double *val = nullptr;      // [nnz]
  float *val32 = nullptr;     // [nnz] float32 copy of val (round to nearest)
  float2 *valsplit = nullptr; // [nnz] (hi, lo): hi = fl32(v), lo = fl32(v - hi)
  double *dinv = nullptr;     // [n] 1 / A[i,i] (0 where the diagonal is missing or zero)
  float *dinv32 = nullptr;    // [n]
  bool split_ok = false;      // every value lies in the split-float product range
  bool full_diag = false;     // every row has a nonzero diagonal entry
  int32_t f64_mode = ENS_F64_AUTO;
  int32_t native_share = -1;  // 32nds of row sweeps on native DFMA in split mode (-1: built-in table)
  int32_t untiled = -1;       // -1: the autotuner's choice; 0: always shared-memory tiles; 1: always untiled
  // autotuned launch choices by block width m (-1: none): lanes per row [0: FP64, 1: FP32], share
  int8_t tuned_lanes[2][kTuneMaxM + 1];
  int8_t tuned_share[kTuneMaxM + 1];
  int8_t tuned_direct[2][kTuneMaxM + 1];  // 1: rows straight from global memory (no tile), 0: tiled
  ens_matrix() {
    for (int i = 0; i <= kTuneMaxM; ++i)
      tuned_lanes[0][i] = tuned_lanes[1][i] = tuned_share[i] = tuned_direct[0][i] = tuned_direct[1][i] = -1;
  }
  // staging buffers of ens_gspmv_host (grown on demand)
  void *stage_x = nullptr, *stage_y = nullptr;
  size_t stage_bytes = 0;
  // ens_gspmv_host pipeline: X rows are split into blocks of pipe_block_rows rows, and row chunk
  // k = rows [pipe_row[k], pipe_row[k+1]) reads only the blocks whose bits are set in
  // pipe_mask[k * kPipeMaskWords ...] (from its column indices). X is copied in block runs in the
  // order the chunks first need them, so chunk k runs as soon as its blocks have arrived (with
  // periodic or other wrap-around couplings too), while later blocks are still being copied in and
  // earlier Y rows copied out. Streams and events are created by the first pipelined call.
  std::vector<int64_t> pipe_row;
  std::vector<uint64_t> pipe_mask;
  int64_t pipe_block_rows = 1;
  cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr;
  std::vector<cudaEvent_t> pipe_ev;
  // aggregation multigrid hierarchy (ens_amg_setup), owned
  ens_amg *amg = nullptr;
};

// One level of the aggregation hierarchy: its matrix (level 0 borrows the fine matrix) and, on
// every level but the coarsest, the map to the next level's rows.
struct ens_amg_lev {
  ens_matrix *A = nullptr;
  bool owned = false;
  ens_matrix *As = nullptr;     // A D^-1 (column-scaled copy, owned) on levels that are smoothed
  int64_t nc = 0;               // rows of the next level
  int32_t *agg = nullptr;       // [n] aggregate (next-level row) of each row
  int32_t *agg_ptr = nullptr;   // [nc + 1] start of each aggregate in members
  int32_t *members = nullptr;   // [n] rows grouped by aggregate, ascending within each
};
struct ens_amg {
  ens_amg_opts opts;
  std::vector<ens_amg_lev> lev;
};

namespace ens {

// Release a hierarchy (coarse matrices and maps; not the fine matrix).
void free_amg(ens_amg *H);

// Create a device matrix of n rows whose column indices lie in [0, ncols) (ncols = n: square).
ens_status create_matrix(int64_t n, int64_t ncols, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                         const double *val, uint32_t flags, void *stream, ens_matrix **out);

// Bytes of scratch the last solve call on this host thread took (or, if its caller-provided
// workspace was too small, needed up to the failing request), and whether it ran out.
void record_workspace(size_t bytes, bool overflow);
bool last_workspace_overflow();

// Record a formatted message for ens_last_error() and return `st`.
ens_status fail(ens_status st, const char *fmt, ...);
// Record a CUDA failure (message includes cudaGetErrorString) and return ENS_ERR_CUDA/OOM.
ens_status cuda_fail(cudaError_t e, const char *what);
void clear_error();

// Split-float path usable for this matrix (mode, value range, row lengths).
bool use_split(const ens_matrix *A);
// Native-DFMA share (32nds of row sweeps) used by the split path for block width m.
int native_share(const ens_matrix *A, int m);
uint32_t share_mask(int share);

// Time the launch candidates for block width m and keep the fastest (synchronous).
ens_status autotune(ens_matrix *A, int m, int dtype, cudaStream_t s, int32_t *lanes_out, int32_t *share_out,
                    double *best_us_out);

// Enqueue Y = A X; arguments already validated.
ens_status launch_gspmv(const ens_matrix *A, int m, int dtype, const void *X, void *Y, cudaStream_t s);
// Pipelined ens_gspmv_host: at most kPipeChunks row chunks, each a multiple of kPipeAlignRows rows
// (a multiple of the GSpMV tile).
constexpr int64_t kPipeChunks = 16;
constexpr int64_t kPipeBlocks = 128;  // X row blocks tracked per chunk
constexpr int64_t kPipeMaskWords = kPipeBlocks / 64;
constexpr int64_t kPipeAlignRows = 256;
// The product for rows [r0, r1) only (r0 a multiple of 256): Y rows r0..r1-1, reading X anywhere.
ens_status launch_gspmv_rows(const ens_matrix *A, int m, int dtype, const void *X, void *Y, int64_t r0, int64_t r1,
                             cudaStream_t s);

// Launch configuration shared by the streaming kernels: 256 threads, grid-stride.
constexpr int kThreads = 256;

}  // namespace ens

#define ENS_CUDA_TRY(call)                                   \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return ens::cuda_fail(_e, #call); \
  } while (0)
