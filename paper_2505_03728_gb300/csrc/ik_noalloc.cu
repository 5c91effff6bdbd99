// ik_noalloc.cu -- pk_ik_solve_noalloc: the multi-start IK solve with its
// scratch in a fixed, file-scope device array instead of caller or library
// allocations.
//
// Some callers cannot call cudaMalloc while they run: real-time control loops
// that must not allocate on their hot path (an allocation can block and take
// unbounded time), and plugin hosts whose device memory is owned by another
// allocator.  For them the work-queue head, the per-target cancellation flags
// and the per-seed result records live in g_ik_scratch below.  Every GPU that
// loads the library holds this array until the process exits.
#include <stdio.h>

#include <mutex>

#include "pk_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_ik_scratch[kNoallocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[pk::kMaxDevices] = {};

}  // namespace

extern "C" pk_status pk_ik_solve_noalloc(const pk_robot* robot, const pk_ik_params* params,
                                         int32_t k, const int32_t* target_links,
                                         const int32_t* target_kinds, int32_t batch,
                                         int32_t n_seeds, const float* d_targets,
                                         const float* d_seeds, float* d_q_out, float* d_err_out,
                                         int32_t* d_iters_out, int32_t* d_status_out,
                                         void* stream) {
  if (!robot) return pk::set_error(PK_ERR_INVALID_ARG, "robot is NULL");
  if (batch < 0 || n_seeds < 1)
    return pk::set_error(PK_ERR_INVALID_ARG, "batch must be >= 0 and n_seeds >= 1");
  const size_t need = pk_ik_workspace_bytes(robot, batch, n_seeds);
  if (need > kNoallocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "pk_ik_solve_noalloc: batch %d x %d seeds needs %zu bytes of scratch, more than the "
             "%zu-byte static scratch; split the batch or use pk_ik_solve",
             batch, n_seeds, need, kNoallocScratchBytes);
    return pk::set_error(PK_ERR_INVALID_ARG, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pk::set_error(PK_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= pk::kMaxDevices)
    return pk::set_error(PK_ERR_UNSUPPORTED, "device ordinal beyond the supported range");
  void* ptr = nullptr;
  {
    // One-time set-up per device, with that device current: the host-side
    // name g_ik_scratch is only a stand-in, so its device address is looked up.
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_ik_scratch);
      if (e != cudaSuccess) return pk::set_error(PK_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_ptr[dev] = p;
    }
    ptr = g_scratch_ptr[dev];
  }
  // pk_ik_solve zeroes the queue head, counters and flags in the scratch
  // before its kernel runs; the result records are fully rewritten.
  return pk_ik_solve(robot, params, k, target_links, target_kinds, batch, n_seeds, d_targets,
                     d_seeds, d_q_out, d_err_out, d_iters_out, d_status_out, ptr,
                     kNoallocScratchBytes, stream);
}
