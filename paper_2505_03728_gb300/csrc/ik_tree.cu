// ik_tree.cu -- the warp-per-problem LM kernel for kinematic trees and
// several targets (ik_tree.cuh), and its host-side constants.
#include <vector>

#include "ik_tree.cuh"

namespace pk {

constexpr int kTreeThreads = 128;

template <int N>
__global__ void __launch_bounds__(kTreeThreads) tree_lm_kernel(const RobotDev* __restrict__ rb,
                                                               const __grid_constant__ TreeInfo ti,
                                                               const __grid_constant__ LmParams lp,
                                                               const float* __restrict__ targets,
                                                               const float* __restrict__ seeds, int n_seeds, int P,
                                                               IkWorkspace ws) {
  __shared__ TreeWarpSmem sm[kTreeThreads / 32];
  WorkCount wc;
  tree_lm_run<N>(rb, ti, lp, targets, seeds, n_seeds, P, ws.head, ws.flags, ws.rec, sm[threadIdx.x >> 5], wc);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(ws.stats + 0, (unsigned long long)wc.eval);
    atomicAdd(ws.stats + 1, (unsigned long long)wc.build);
    atomicAdd(ws.stats + 2, (unsigned long long)wc.solve);
    atomicAdd(ws.stats + 3, (unsigned long long)wc.done);
  }
}

bool build_tree_info(const pk_robot* rb, int k, const int32_t* links, const int32_t* kinds, TreeInfo* ti) {
  if (rb->n_dof > kTreeMaxDof || k > kTreeMaxTargets || rb->n_joints > kMaxJoints) return false;
  *ti = TreeInfo{};
  ti->n_joints = rb->n_joints;
  ti->n_dof = rb->n_dof;
  ti->k = k;
  std::vector<int> depth(rb->n_joints, 0);
  int max_depth = 0;
  for (int j = 0; j < rb->n_joints; ++j) {
    depth[j] = rb->parent[j] < 0 ? 0 : depth[rb->parent[j]] + 1;
    if (depth[j] > max_depth) max_depth = depth[j];
  }
  ti->n_levels = max_depth + 1;
  int pos = 0;
  for (int l = 0; l <= max_depth; ++l) {
    ti->level_start[l] = pos;
    for (int j = 0; j < rb->n_joints; ++j)
      if (depth[j] == l) ti->order[pos++] = j;
  }
  ti->level_start[max_depth + 1] = pos;
  std::vector<int> slot(rb->n_joints, -1);  // a mimic joint's index in its variable's list
  for (int j = 0; j < rb->n_joints; ++j) {
    const int v = rb->var[j];
    if (v < 0) continue;
    if (rb->mimic[j] < 0) {
      ti->dof_joint[v] = j;
      ti->lo[v] = rb->lower[j];
      ti->hi[v] = rb->upper[j];
    } else {
      if (ti->n_mim[v] >= kTreeMaxMimic) return false;
      slot[j] = ti->n_mim[v]++;
      ti->mim_joint[v][slot[j]] = j;
      ti->mim_mult[v][slot[j]] = rb->mult[j];
    }
  }
  for (int t = 0; t < k; ++t) {
    ti->links[t] = links[t];
    ti->kinds[t] = kinds ? kinds[t] : PK_TARGET_POSE;
    for (int j = links[t]; j >= 0; j = rb->parent[j]) {
      const int v = rb->var[j];
      if (v < 0) continue;
      ti->dof_targets[v] |= 1u << t;
      if (rb->mimic[j] < 0)
        ti->own_targets[v] |= 1u << t;
      else
        ti->mim_targets[v][slot[j]] |= 1u << t;
    }
  }
  return true;
}

cudaError_t launch_tree_lm(const pk_robot* rb, const TreeInfo& ti, const LmParams& lp, const float* d_targets,
                           const float* d_seeds, int batch, int n_seeds, IkWorkspace ws, float* d_q, float* d_err,
                           int32_t* d_iters, int32_t* d_status, cudaStream_t stream) {
  static int blocks_per_sm = 0, sms = 0;
  if (!blocks_per_sm) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, tree_lm_kernel<kTreeMaxDof>,
                                                                  kTreeThreads, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const long P = (long)batch * n_seeds;
  long grid = (long)blocks_per_sm * sms;
  const long need = (P + kTreeThreads / 32 - 1) / (kTreeThreads / 32);
  if (grid > need) grid = need;
  {
    TraceScope tr("ik_tree", stream);
    tree_lm_kernel<kTreeMaxDof><<<(unsigned)grid, kTreeThreads, 0, stream>>>(
        (const RobotDev*)rb->d_blob, ti, lp, d_targets, d_seeds, n_seeds, (int)P, ws);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_ik_reduce(ws.rec, rb->n_dof, batch, n_seeds, d_q, d_err, d_iters, d_status, stream);
}

}  // namespace pk
