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

// Device address of g_ik_scratch on the current device.  The host-side name
// is only a stand-in, so the address is looked up with the device current:
// on every call outside stream capture (the lookup allocates nothing, and a
// fresh lookup stays valid after a device or context reset), and from the
// copy kept by the last such call while `st` is being captured.
pk_status scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pk::set_error(PK_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= pk::kMaxDevices)
    return pk::set_error(PK_ERR_UNSUPPORTED, "device ordinal beyond the supported range");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!capturing) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_ik_scratch);
    if (e != cudaSuccess) return pk::set_error(PK_ERR_CUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  } else if (!g_scratch_ptr[dev]) {
    return pk::set_error(PK_ERR_INVALID_ARG,
                         "pk_ik_solve_noalloc: the first call on a device must come before any stream capture");
  }
  *out = g_scratch_ptr[dev];
  return PK_OK;
}

}  // namespace

extern "C" pk_status pk_ik_solve_noalloc(const pk_robot* robot, const pk_ik_params* params,
                                         int32_t k, const int32_t* target_links,
                                         const int32_t* target_kinds, int32_t batch,
                                         int32_t n_seeds, const float* d_targets,
                                         const float* d_seeds, float* d_q_out, float* d_err_out,
                                         int32_t* d_iters_out, int32_t* d_status_out,
                                         void* stream) {
  // the argument checks of pk_ik_solve first, so that a bad argument is
  // reported as such; an empty batch returns before any set-up
  bool empty = false;
  pk_status s = pk::ik_check_args(robot, params, k, target_links, target_kinds, batch, n_seeds, d_targets, d_seeds,
                                  d_q_out, d_err_out, d_iters_out, d_status_out, &empty);
  if (s != PK_OK || empty) return s;
  const size_t need = pk_ik_workspace_bytes(robot, batch, n_seeds);
  if (need > kNoallocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "pk_ik_solve_noalloc: batch %d x %d seeds needs %zu bytes of scratch, more than the "
             "%zu-byte static scratch; split the batch or use pk_ik_solve",
             batch, n_seeds, need, kNoallocScratchBytes);
    return pk::set_error(PK_ERR_INVALID_ARG, msg);
  }
  void* ptr = nullptr;
  if ((s = scratch_address((cudaStream_t)stream, &ptr)) != PK_OK) return s;
  // pk_ik_solve zeroes the queue head, counters and cancellation flags in the
  // scratch before its kernel runs; the result records are fully rewritten.
  return pk_ik_solve(robot, params, k, target_links, target_kinds, batch, n_seeds, d_targets,
                     d_seeds, d_q_out, d_err_out, d_iters_out, d_status_out, ptr,
                     kNoallocScratchBytes, stream);
}
