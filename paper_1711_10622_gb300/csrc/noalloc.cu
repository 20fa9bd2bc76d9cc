// ens_gspmv_host_noalloc: the host-buffer GSpMV without any device allocation.
//
// ens_gspmv_host stages X and Y in device buffers that it allocates (and grows) on demand. Some
// callers cannot let a library allocate device memory at call time: applications that reserve all
// device memory up front for their own pool (a late cudaMalloc fails or fragments it), real-time
// loops where an allocation's latency and implicit synchronisation are not acceptable, and hosts
// that forbid plug-in libraries from allocating. This entry point stages through a fixed array
// compiled into the library instead, so the only device memory it uses exists from the moment the
// library's module is loaded on a GPU until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "ens_internal.cuh"

namespace ens {
namespace {

// Staging for X (first half) and Y (second half): kNoAllocStageBytes each.
constexpr size_t kNoAllocStageBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_stage[2 * kNoAllocStageBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_addr[kMaxDevices] = {};

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" ens_status ens_gspmv_host_noalloc(const ens_matrix *A, int32_t m, int32_t dtype, const void *X, void *Y,
                                             void *stream) {
  clear_error();
  if (!A) return fail(ENS_ERR_INVALID, "gspmv_host_noalloc: matrix is NULL");
  if (A->ncols != A->n) return fail(ENS_ERR_INVALID, "gspmv_host_noalloc: needs a square matrix");
  if (m < 1) return fail(ENS_ERR_INVALID, "gspmv_host_noalloc: m must be >= 1 (got %d)", m);
  if (dtype != ENS_F64 && dtype != ENS_F32) return fail(ENS_ERR_INVALID, "gspmv_host_noalloc: unknown dtype %d", dtype);
  if (!X || !Y) return fail(ENS_ERR_INVALID, "gspmv_host_noalloc: X or Y is NULL");
  const size_t es = dtype == ENS_F64 ? 8 : 4;
  if ((size_t)A->n > kNoAllocStageBytes / es / (size_t)m)
    return fail(ENS_ERR_INVALID, "gspmv_host_noalloc: n*m*%zu = %lld bytes exceeds the %zu-byte staging limit", es,
                (long long)((size_t)A->n * m * es), kNoAllocStageBytes);
  const size_t bytes = (size_t)A->n * m * es;
  int dev = 0;
  ENS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != A->device)
    return fail(ENS_ERR_INVALID, "gspmv_host_noalloc: current device %d is not the matrix's device %d", dev, A->device);
  if (dev < 0 || dev >= kMaxDevices) return fail(ENS_ERR_INVALID, "gspmv_host_noalloc: device %d unsupported", dev);
  cudaStream_t s = (cudaStream_t)stream;
  // One caller at a time: every call shares the staging array (see the header).
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    // Host code cannot use the array's name as a device address: ask the runtime, once per device,
    // with that device current.
    void *p = nullptr;
    ENS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_stage));
    g_noalloc_addr[dev] = (unsigned char *)p;
  }
  unsigned char *stage_x = g_noalloc_addr[dev];
  unsigned char *stage_y = stage_x + kNoAllocStageBytes;
  // Nothing has to start at zero: the copy overwrites the X part and the kernel writes all of Y.
  ENS_CUDA_TRY(cudaMemcpyAsync(stage_x, X, bytes, cudaMemcpyHostToDevice, s));
  // From here on work on the shared array may be queued: every exit waits for the stream while
  // the lock is still held, so the next caller never overwrites the array under running work.
  ens_status st = launch_gspmv(A, m, dtype, stage_x, stage_y, s);
  cudaError_t e = cudaSuccess;
  if (st == ENS_OK) e = cudaMemcpyAsync(Y, stage_y, bytes, cudaMemcpyDeviceToHost, s);
  const cudaError_t esync = cudaStreamSynchronize(s);
  if (st != ENS_OK) return st;
  if (e == cudaSuccess) e = esync;
  if (e != cudaSuccess) return cuda_fail(e, "gspmv_host_noalloc");
  return ENS_OK;
}
