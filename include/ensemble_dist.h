/*
 * ensemble_dist.h - building blocks of the multi-GPU forms of the multiple-ensemble solve
 * (arXiv 1711.10622), part of libensemble_solve.so.
 *
 * The paper runs its solver on a 3D geometric decomposition with MPI (Section 3): every process
 * owns a block of grid cells, i.e. a contiguous block of matrix rows, and each matrix-vector
 * product first exchanges the boundary values its neighbours need (Section 4.1 counts these
 * messages against m). On GPUs the same structure is one process per GPU: the rows a rank owns
 * form a row block of the matrix whose column indices point into an EXTENDED local vector
 * [owned rows | halo rows received from the neighbours]. The entry points below are the device
 * work of one rank; the exchange (NCCL or gloo send/recv) and the allreduce of the per-column dot
 * products run in the caller (the Python layer uses torch.distributed).
 *
 * Conventions are those of ensemble_solve.h: blocks are row-interleaved (element (k, l) at
 * k*m + l), pointers are DEVICE pointers owned by the caller unless stated, `stream` is a
 * cudaStream_t passed as void*, calls only enqueue work and return, errors are an ens_status with
 * a message from ens_last_error().
 */
#ifndef ENSEMBLE_DIST_H
#define ENSEMBLE_DIST_H

#include <stdint.h>

#include "ensemble_solve.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * A row block of a distributed matrix (Section 3's domain decomposition): n_rows rows whose
 * column indices lie in [0, n_cols) of an extended local vector (n_cols >= 1; the rows are the
 * owned rows of one rank, or a subset of them). HOST arrays as in ens_create_matrix (int32
 * row_ptr [n_rows + 1], col_idx and float64 val [nnz]); copied, synchronous. The handle works with
 * ens_gspmv (X has n_cols rows, Y n_rows rows) and ens_autotune; the solver, the AMG set-up and
 * the host-buffer products need square matrices and reject it with ENS_ERR_INVALID.
 */
ens_status ens_create_matrix_rect(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *row_ptr,
                                  const int32_t *col_idx, const double *val, void *stream, ens_matrix **out);

/* Rows and columns of a matrix (square or row block). */
ens_status ens_matrix_shape(const ens_matrix *A, int64_t *n_rows, int64_t *n_cols);

/*
 * Local partial block dots (Section 2.3's vector operations, per column): for k < npairs,
 *   out[k*m + l] = sum_{i < n} X_k[i*m + l] * Y_k[i*m + l],
 * summed in a fixed order (the same bits on every call with the same n, m). X, Y: HOST arrays of
 * npairs DEVICE pointers to float64 n x m blocks; out: DEVICE float64 [npairs * m]. A rank adds
 * its partial dots to the others' with one allreduce of npairs * m scalars.
 *   1 <= npairs <= 4, 1 <= m <= 256, n >= 0 (n = 0 writes zeros). Scratch for the partial sums of
 *   the blocks is allocated stream-ordered (cudaMallocAsync) and released in the call.
 */
ens_status ens_block_dots(int64_t n, int32_t m, int32_t npairs, const double *const *X, const double *const *Y,
                          double *out, void *stream);

/*
 * Block linear combination with per-column coefficients (the block axpy family of BiCGStab:
 * p = r + beta (p - omega v), s = r - alpha v, x += alpha p + omega s, r = s - omega t):
 *   out[i*m + l] = sum_{k < nterms} c_k[l] * V_k[i*m + l],   c_k = NULL means coefficient 1.
 * coef, vec: HOST arrays of nterms pointers (coef entries DEVICE float64 [m] or NULL; vec entries
 * DEVICE float64 n x m blocks). out may be one of the V_k (each element is read before it is
 * written, by the same thread). 1 <= nterms <= 4, 1 <= m <= 256.
 */
ens_status ens_block_lincomb(int64_t n, int32_t m, int32_t nterms, const double *const *coef, const double *const *vec,
                             double *out, void *stream);

/*
 * Row gather (packing the halo rows a neighbour needs): out[k*m + l] = X[idx[k]*m + l] for
 * k < count. idx: DEVICE int32 [count], each in [0, rows of X) (not checked on the device: the
 * caller builds idx from the partition). out must not overlap X. m >= 1.
 */
ens_status ens_gather_rows(int64_t count, int32_t m, const int32_t *idx, const double *X, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ENSEMBLE_DIST_H */
